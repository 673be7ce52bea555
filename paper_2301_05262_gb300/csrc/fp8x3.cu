// Three-term FP8 (E4M3) layers (network of Sec. 3.5 / 3.6; 8-bit storage is
// among the paper's Sec. 3.5 directions): y = relu?(conv_k(relu?(x)) + b), k = 3
// (zero padded) or 1, FP32 NHWC tensors in and out, products on tcgen05
// kind::f8f6f4 (E4M3 x E4M3, FP32 accumulation).
//
// Every activation is held as three E4M3 terms at fixed scales 1, 2^-4, 2^-8:
//   a_0 = e4m3(x),  a_1 = e4m3(16 (x - a_0)),  a_2 = e4m3(256 (x - a_0 - a_1 / 16))
// (round to nearest even, saturating at +-448), x ~ a_0 + a_1 / 16 + a_2 / 256;
// every weight of output channel o as s_o (b_0 + b_1 / 16 + b_2 / 256) with the
// same split of W / s_o, s_o = max |W[o]| / 448.  Term j of an activation times
// term k of a weight carries the scale 2^-4 (j + k) s_o: the nine products of
// a K step accumulate in five tensor-memory blocks, one per j + k, which the
// epilogue sums with their scales (times s_o, plus the bias).  About 12 bits
// of each operand survive (three 4-bit significands), against 3 for one term.
//
// Tile: 128 pixels of one image row x 32 output channels (16 for a 16-channel
// layer); K = taps x C_in in
// chunks of 32 input channels (one K = 32 step per tap and term pair).  The
// 1x1 kernel has two stages (the threads stage chunk c + 1, FP32 -> three E4M3
// planes, and one bulk copy brings its weights while the tensor core works on
// chunk c); the 3x3 kernel one, with two CTAs per SM overlapping instead.
#include <cuda_fp8.h>

#include "nsm_internal.h"
#include "tc_pipeline.cuh"
#include "train_internal.h"

namespace nsm {
namespace tr {

using namespace tc;

namespace {

constexpr int kF8Threads = 256;
constexpr int kF8T = 3;                 // E4M3 terms per value
constexpr int kF8Blk = 2 * kF8T - 1;    // accumulator blocks (j + k = 0 .. 4)
constexpr int kF8CC = 32;               // input channels per K chunk
constexpr int kF8ErrCode = 10;          // error word value of a wait in f8x3_conv_kernel that gave up

// NB: output channels per CTA (32, or 16 for a 16-channel layer).  PAIR (3x3
// layers with at most 16 input channels): one K = 32 step covers two
// horizontal taps -- its K halves are staged pixels m + kx and m + kx + 1 of the
// one 16-channel plane (16 bytes apart) -- so a kernel row takes 2 steps
// (kx = 0, 1 and kx = 2 with zero weights for the missing fourth tap), not 3.
template <int K, int NB, bool PAIR = false>
struct F8Cfg {
    // stages of (A, B): the 3x3 kernel keeps one (68 KB, so two CTAs share an SM
    // and one's staging overlaps the other's MMAs), the 1x1 kernel two
    static constexpr int NS = K == 3 ? 1 : 2;
    static constexpr int SR = K;                        // staged rows
    static constexpr int SP = K == 3 ? (PAIR ? 131 : 130) : 128;  // staged pixels used
    static constexpr int G = PAIR ? 1 : kF8CC / 16;     // 16-channel groups per term (the K halves unless PAIR)
    static constexpr int NSTEP = PAIR ? 2 * K : K * K;  // K = 32 steps per chunk and term pair
    static constexpr uint32_t PLANE = SR * kSW * 16;    // bytes per (term, group) plane
    static constexpr uint32_t A_BYTES = kF8T * G * PLANE;
    static constexpr uint32_t B_BYTES = NSTEP * kF8T * 2 * NB * 16;
    static constexpr uint32_t STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t OFF_BAR = NS * STAGE;
    static constexpr uint32_t BYTES = OFF_BAR + 64;     // 4 mbarriers, TMEM address slot
    static constexpr int ITEMS = SR * SP * G;
    static constexpr int S = (ITEMS + kF8Threads - 1) / kF8Threads;
    static constexpr int TMEM_COLS = kF8Blk * NB <= 128 ? 128 : 256;  // 5 blocks of NB columns
    static_assert(kF8Blk * NB <= TMEM_COLS, "accumulator blocks");
    static_assert(NB == 16 || NB == 32, "output block");
    static_assert(!PAIR || K == 3, "tap pairs are horizontal taps of a 3x3");
    static_assert(SP <= kSW, "staged row");
    static_assert(A_BYTES % 16 == 0 && B_BYTES % 16 == 0, "bulk-copy granularity");
    static_assert(BYTES <= 227 * 1024, "shared memory per CTA");
    static_assert(PLANE / 16 < (1u << 14), "LBO field");
};

__device__ __forceinline__ uint32_t f8_pack4(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}
__device__ __forceinline__ float2 f8_unpack2(uint32_t bits16) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(bits16), __NV_E4M3);
    return __half22float2(__half2(h));
}

// The three E4M3 terms of 16 values (chunk k holds term k, byte i = value i).
__device__ __forceinline__ void f8_split3(const float (&v)[16], uint4 (&t)[kF8T]) {
    float r[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = v[i];
#pragma unroll
    for (int k = 0; k < kF8T; ++k) {
        const float s = k == 0 ? 1.f : (k == 1 ? 16.f : 256.f), is = 1.f / s;  // exact powers of two
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            w[q] = f8_pack4(r[4 * q] * s, r[4 * q + 1] * s, r[4 * q + 2] * s, r[4 * q + 3] * s);
        t[k] = make_uint4(w[0], w[1], w[2], w[3]);
        if (k + 1 < kF8T) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 a = f8_unpack2(w[q] & 0xFFFFu), b = f8_unpack2(w[q] >> 16);
                r[4 * q] -= a.x * is; r[4 * q + 1] -= a.y * is; r[4 * q + 2] -= b.x * is; r[4 * q + 3] -= b.y * is;
            }
        }
    }
}

// s_o = max |W[o]| / 448 (1 for an all-zero channel)
__global__ void f8_scale_kernel(const float* __restrict__ w, int cin, int cout, int taps, float* __restrict__ scale) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= cout) return;
    float m = 0.f;
    for (int i = 0; i < cin * taps; ++i) m = fmaxf(m, fabsf(__ldg(w + static_cast<size_t>(o) * cin * taps + i)));
    scale[o] = m > 0.f ? m / 448.f : 1.f;
}

// Weight image of one layer: block (ob, c) = outputs nb ob .. + nb, inputs
// 32 c .. + 32; inside it chunk (step, term k, half h, row n) holds term k of
// W[nb ob + n][32 c + 16 h .. + 16][tap = step] / s_o as 16 E4M3 codes, or with
// tap pairs (pair) W[nb ob + n][0 .. 16][kernel row step / 2, column
// 2 (step % 2) + h] (zero for column 3).
__global__ void f8_pack_kernel(const float* __restrict__ w, const float* __restrict__ scale, int cin, int cout, int k,
                               int nb, int pair, uint4* __restrict__ img) {
    const int taps = k * k, nc = (cin + kF8CC - 1) / kF8CC, nob = (cout + nb - 1) / nb;
    const int nstep = pair ? 2 * k : taps;
    const size_t chunks = static_cast<size_t>(nob) * nc * nstep * kF8T * 2 * nb;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < chunks;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int n = static_cast<int>(i % nb);
        size_t r = i / nb;
        const int h = static_cast<int>(r % 2); r /= 2;
        const int term = static_cast<int>(r % kF8T); r /= kF8T;
        const int step = static_cast<int>(r % nstep); r /= nstep;
        const int c = static_cast<int>(r % nc);
        const int ob = static_cast<int>(r / nc);
        const int o = ob * nb + n;
        // a pair step's half h is horizontal tap 2 (step % 2) + h of kernel row step / 2 (none past kx = 2)
        const int kx = pair ? 2 * (step % 2) + h : 0;
        const int tap = pair ? (kx < k ? (step / 2) * k + kx : -1) : step;
        float v[16];
        const float s = o < cout ? __ldg(scale + o) : 1.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int ch = pair ? j : c * kF8CC + h * 16 + j;
            v[j] = (o < cout && ch < cin && tap >= 0)
                       ? __ldg(w + (static_cast<size_t>(o) * cin + ch) * taps + tap) / s : 0.f;
        }
        uint4 t[kF8T];
        f8_split3(v, t);
        img[i] = t[term];
    }
}

template <int K, int NB, bool PAIR>
struct F8Regs {
    float4 v[F8Cfg<K, NB, PAIR>::S][4];
};

// Chunk c of tile (row yr, x0): item i = (staged row sr, group g, staged
// pixel sp; pixel fastest) covers image row yr - K / 2 + sr, column
// x0 - K / 2 + sp, input channels 32 c + 16 g .. + 16; zeros outside the image
// and beyond C_in.
template <int K, int NB, bool PAIR>
__device__ __forceinline__ void f8_load(F8Regs<K, NB, PAIR>& R, const float* __restrict__ x, int H, int W, int CIN, int yr,
                                        int x0, int c) {
    using C = F8Cfg<K, NB, PAIR>;
#pragma unroll
    for (int s = 0; s < C::S; ++s) {
        const int i = threadIdx.x + s * kF8Threads;
        const int sp = i % C::SP, rest = i / C::SP;
        const int g = rest % C::G, sr = rest / C::G;
        const int yy = yr - K / 2 + sr, xx = x0 - K / 2 + sp;
        const bool in = i < C::ITEMS && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const int ch0 = c * kF8CC + 16 * g;
        const float4* p = reinterpret_cast<const float4*>(x + (static_cast<size_t>(in ? yy : 0) * W + (in ? xx : 0)) * CIN);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ch = ch0 + 4 * q;
            R.v[s][q] = (in && ch < CIN) ? __ldg(p + ch / 4) : z;
        }
    }
}

template <int K, int NB, bool PAIR>
__device__ __forceinline__ void f8_store(const F8Regs<K, NB, PAIR>& R, uint32_t abase, int relu_in) {
    using C = F8Cfg<K, NB, PAIR>;
#pragma unroll
    for (int s = 0; s < C::S; ++s) {
        const int i = threadIdx.x + s * kF8Threads;
        if (i >= C::ITEMS) break;
        const int sp = i % C::SP, rest = i / C::SP;
        const int g = rest % C::G, sr = rest / C::G;
        float v[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[4 * q] = R.v[s][q].x; v[4 * q + 1] = R.v[s][q].y; v[4 * q + 2] = R.v[s][q].z; v[4 * q + 3] = R.v[s][q].w;
        }
        if (relu_in)
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        uint4 t[kF8T];
        f8_split3(v, t);
        const uint32_t off = static_cast<uint32_t>(g) * C::PLANE + static_cast<uint32_t>(sr * kSW + sp) * 16;
#pragma unroll
        for (int k = 0; k < kF8T; ++k) st_shared_v4(abase + static_cast<uint32_t>(k * C::G) * C::PLANE + off, t[k]);
    }
}

// The chunk's MMAs (one thread): per K step, weight term k and activation
// term j, D block j + k; the first product into each block of a tile starts it.
template <int K, int NB, bool PAIR>
__device__ __forceinline__ void f8_mma(uint32_t abase, uint32_t bbase, uint32_t tbase, bool first_chunk) {
    using C = F8Cfg<K, NB, PAIR>;
    constexpr uint32_t idesc = idesc_e4m3(kTileM, NB);
#pragma unroll
    for (int step = 0; step < C::NSTEP; ++step) {
        // the step's first tap (ky, kx); its K halves: channel groups 0 and 1 of
        // that tap's pixels, or (PAIR) the 16 channels of pixels m + kx and m + kx + 1
        const int ky = PAIR ? step / 2 : step / K, kx = PAIR ? 2 * (step % 2) : step % K;
        const uint32_t lbo = PAIR ? 16u : C::PLANE;
#pragma unroll
        for (int k = 0; k < kF8T; ++k) {
            const uint64_t bdesc =
                smem_desc(bbase + static_cast<uint32_t>((step * kF8T + k) * 2 * NB) * 16, NB * 16, 128);
#pragma unroll
            for (int j = 0; j < kF8T; ++j) {
                // in the (k, j) order above, block j + k is first written by (0, j) or, for j + k > 2, by (k, 2)
                const bool starts = step == 0 && (k == 0 || j == kF8T - 1);
                const uint32_t a = abase + static_cast<uint32_t>(j * C::G) * C::PLANE +
                                   static_cast<uint32_t>(ky * kSW + kx) * 16;
                mma_e4m3(tbase + static_cast<uint32_t>((j + k) * NB), smem_desc(a, lbo, 128), bdesc, idesc,
                         (first_chunk && starts) ? 0u : 1u);
            }
        }
    }
}

template <int K, int NB, bool PAIR>
__global__ void __launch_bounds__(kF8Threads, 2) f8x3_conv_kernel(const float* __restrict__ x, int relu_in, int H, int W,
                                                               int CIN, int COUT, const uint4* __restrict__ img,
                                                               const float* __restrict__ scale,
                                                               const float* __restrict__ bias, float* __restrict__ y,
                                                               int relu_out, int* err) {
    using C = F8Cfg<K, NB, PAIR>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);       // [2] weights landed
    uint64_t* done = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR + 16);  // [2] MMAs of the stage finished
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 32);
    const uint32_t sbase = smem_u32(smem);
    if (tid == 0) {
        mbar_init(&full[0], 1); mbar_init(&full[1], 1);
        mbar_init(&done[0], 1); mbar_init(&done[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, C::TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    const int tiles_x = (W + kTileM - 1) / kTileM, nob = (COUT + NB - 1) / NB, nc = (CIN + kF8CC - 1) / kF8CC;
    const long long ntiles = static_cast<long long>(H) * tiles_x * nob;
    const uint32_t block_chunks = C::B_BYTES / 16;
    uint32_t fph[2] = {0u, 0u}, dph[2] = {0u, 0u};
    int pend[2] = {0, 0};
    bool ok = true;
    int it = 0;
    F8Regs<K, NB, PAIR> R;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int ob = static_cast<int>(t % nob);
        const long long r = t / nob;
        const int x0 = static_cast<int>(r % tiles_x) * kTileM, yr = static_cast<int>(r / tiles_x);
        for (int c = 0; c < nc; ++c, ++it) {
            const int s = C::NS == 2 ? (it & 1) : 0;
            const uint32_t abase = sbase + s * C::STAGE, bbase = abase + C::A_BYTES;
            f8_load<K, NB, PAIR>(R, x, H, W, CIN, yr, x0, c);  // in flight while the other stage's MMAs run
            if (pend[s]) {
                ok = mbar_wait_bounded(&done[s], dph[s], kWaitNs);
                dph[s] ^= 1u;
                pend[s] = 0;
            }
            if (__syncthreads_or(!ok)) { ok = false; break; }
            if (tid == 0) {
                mbar_arrive_expect_tx(&full[s], C::B_BYTES);
                bulk_load(bbase, img + (static_cast<size_t>(ob) * nc + c) * block_chunks, C::B_BYTES, &full[s]);
            }
            f8_store<K, NB, PAIR>(R, abase, relu_in);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                if (mbar_wait_bounded(&full[s], fph[s], kWaitNs)) {
                    fence_after_sync();
                    f8_mma<K, NB, PAIR>(abase, bbase, tbase, c == 0);
                } else {
                    atomicExch(err, kF8ErrCode);
                }
                mma_commit(&done[s]);
            }
            fph[s] ^= 1u;
            pend[s] = 1;
        }
        if (!ok) break;
        const int sl = C::NS == 2 ? ((it - 1) & 1) : 0;
        ok = mbar_wait_bounded(&done[sl], dph[sl], kWaitNs);
        dph[sl] ^= 1u;
        pend[sl] = 0;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        fence_after_sync();
        // warp w: TMEM lane quarter w % 4 (pixels), outputs NB / 2 (w / 4) .. + NB / 2 of the block
        const int lq = warp & 3, o0 = ob * NB + (NB / 2) * (warp >> 2);
        const int px = x0 + 32 * lq + lane;
        // passes of 8 columns: the five blocks' values of 8 outputs live at a time
#pragma unroll
        for (int hp = 0; hp < NB / 16; ++hp) {
            float d[kF8Blk][8];
            const uint32_t tq = tbase + (static_cast<uint32_t>(32 * lq) << 16) +
                                static_cast<uint32_t>((NB / 2) * (warp >> 2) + 8 * hp);
#pragma unroll
            for (int b = 0; b < kF8Blk; ++b) tmem_ld8(tq + static_cast<uint32_t>(b * NB), d[b]);
            tmem_ld_wait();
            if (px < W && o0 < COUT) {
                float* out = y + (static_cast<size_t>(yr) * W + px) * COUT + o0 + 8 * hp;
#pragma unroll
                for (int o = 0; o < 8; o += 4) {
                    float v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        // smallest-scale blocks first
                        float a = d[4][o + e];
                        a = fmaf(a, 1.f / 16.f, d[3][o + e]);
                        a = fmaf(a, 1.f / 16.f, d[2][o + e]);
                        a = fmaf(a, 1.f / 16.f, d[1][o + e]);
                        a = fmaf(a, 1.f / 16.f, d[0][o + e]);
                        const int oc = o0 + 8 * hp + o + e;
                        v[e] = fmaf(a, __ldg(scale + oc), __ldg(bias + oc));
                        if (relu_out) v[e] = fmaxf(v[e], 0.f);
                    }
                    *reinterpret_cast<float4*>(out + o) = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    for (int s = 0; s < 2; ++s)
        if (pend[s]) {
            if (!mbar_wait_bounded(&done[s], dph[s], kWaitNs)) atomicExch(err, kF8ErrCode);
            dph[s] ^= 1u;
        }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, C::TMEM_COLS);
}

template <int K, int NB, bool PAIR>
cudaError_t launch_f8x3(const float* x, int relu_in, int H, int W, int cin, int cout, const uint4* img,
                        const float* scale, const float* bias, float* y, int relu_out, int* err, cudaStream_t st) {
    using C = F8Cfg<K, NB, PAIR>;
    static int per_sm = 0;  // CTAs resident per SM (per instantiation, set on first use)
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(f8x3_conv_kernel<K, NB, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C::BYTES));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f8x3_conv_kernel<K, NB, PAIR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        const int occ = resident_ctas_per_sm(reinterpret_cast<const void*>(f8x3_conv_kernel<K, NB, PAIR>), kF8Threads,
                                             C::BYTES);
        per_sm = occ < 512 / C::TMEM_COLS ? occ : 512 / C::TMEM_COLS;
    }
    const long long tiles = static_cast<long long>(H) * ((W + kTileM - 1) / kTileM) * ((cout + NB - 1) / NB);
    if (tiles == 0) return cudaSuccess;
    const long long cap = static_cast<long long>(num_sms()) * per_sm;
    const int grid = static_cast<int>(tiles < cap ? tiles : cap);
    f8x3_conv_kernel<K, NB, PAIR><<<grid, kF8Threads, C::BYTES, st>>>(x, relu_in, H, W, cin, cout, img, scale, bias, y,
                                                                        relu_out, err);
    return cudaGetLastError();
}

// output channels per CTA: 16 for a 16-channel layer, else 32; tap pairs for a
// 3x3 layer with at most 16 input channels
constexpr int f8_nb(int cout) { return cout % 32 == 0 ? 32 : 16; }
constexpr bool f8_pair(int cin, int k) { return k == 3 && cin <= 16; }

}  // namespace

bool f8x3_supported(int cin, int cout, int k) {
    return (k == 3 || k == 1) && cin > 0 && cin % 4 == 0 && cout > 0 && cout % 16 == 0;
}

size_t f8x3_image_bytes(int cin, int cout, int k) {
    if (!f8x3_supported(cin, cout, k)) return 0;
    const size_t nb = f8_nb(cout), nob = (cout + nb - 1) / nb, nc = (cin + kF8CC - 1) / kF8CC;
    const size_t nstep = f8_pair(cin, k) ? 2 * k : k * k;
    return nob * nc * nstep * kF8T * 2 * nb * 16 + align_up(nob * nb * sizeof(float), 256);
}

// the weight terms' chunks of a layer's image (the scales follow them)
static size_t f8x3_chunks(int cin, int cout, int k) {
    const size_t nb = f8_nb(cout), nob = (cout + nb - 1) / nb, nc = (cin + kF8CC - 1) / kF8CC;
    const size_t nstep = f8_pair(cin, k) ? 2 * k : k * k;
    return nob * nc * nstep * kF8T * 2 * nb;
}

cudaError_t f8x3_pack(const float* w, int cin, int cout, int k, void* img, cudaStream_t st) {
    if (!f8x3_supported(cin, cout, k)) return cudaErrorInvalidValue;
    const size_t chunks = f8x3_chunks(cin, cout, k);
    float* scale = reinterpret_cast<float*>(static_cast<char*>(img) + chunks * 16);
    f8_scale_kernel<<<(cout + 127) / 128, 128, 0, st>>>(w, cin, cout, k * k, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t blocks = (chunks + 255) / 256, cap = static_cast<size_t>(num_sms()) * 8;
    f8_pack_kernel<<<static_cast<int>(blocks < cap ? blocks : cap), 256, 0, st>>>(
        w, scale, cin, cout, k, f8_nb(cout), f8_pair(cin, k) ? 1 : 0, static_cast<uint4*>(img));
    return cudaGetLastError();
}

cudaError_t f8x3_conv(int cin, int cout, int k, const float* x, int relu_in, int H, int W, const void* img,
                      const float* bias, float* y, int relu_out, int* err, cudaStream_t st) {
    if (!f8x3_supported(cin, cout, k)) return cudaErrorInvalidValue;
    const uint4* im = static_cast<const uint4*>(img);
    const float* scale =
        reinterpret_cast<const float*>(static_cast<const char*>(img) + f8x3_chunks(cin, cout, k) * 16);
    const bool nb16 = f8_nb(cout) == 16;
    if (k == 3) {
        if (f8_pair(cin, k))
            return nb16 ? launch_f8x3<3, 16, true>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st)
                        : launch_f8x3<3, 32, true>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st);
        return nb16 ? launch_f8x3<3, 16, false>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st)
                    : launch_f8x3<3, 32, false>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st);
    }
    return nb16 ? launch_f8x3<1, 16, false>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st)
                : launch_f8x3<1, 32, false>(x, relu_in, H, W, cin, cout, im, scale, bias, y, relu_out, err, st);
}

}  // namespace tr
}  // namespace nsm
