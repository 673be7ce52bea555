// Tensor-core layers of the deeper networks' inner levels (Sec. 3.6; layers
// of Sec. 3.5 with widths 16 * 2^l): y = relu?(conv_k(relu?(x)) + b) for k = 3
// (zero padded) and k = 1, FP32 NHWC tensors in and out, 32 .. 1024
// channels.  The products run on tcgen05 in compensated BF16: every
// activation and weight is a pair hi = bf16(v), lo = bf16(v - hi); all four
// part products accumulate in FP32 in tensor memory.
//
// Implicit GEMM, D[R x 128 pixels x 64 outputs] per CTA and tile (R image
// rows of a 128-pixel column segment, one block of 64 output channels; R = 4,
// 2 or 1 for a 3x3 layer, the largest that still gives every SM a tile, so a
// streamed weight chunk serves R MMA row blocks), K = taps x C_in walked in
// chunks of CC input channels:
//   A  the chunk's rows y - 1 .. y + R (y for a 1x1 layer) with a one-pixel
//      halo, staged by all threads from FP32 as [part][channel group][staged
//      row][staged pixel] 16-byte chunks (the no-swizzle K-major layout, so
//      tap (ky, kx) is the same planes started ky rows and kx chunks on)
//   B  the chunk's weights for the 64 outputs, hi and lo parts side by side
//      along N (N = 128), packed once per call into one contiguous block per
//      (output block, chunk) and fetched by a single bulk copy
// Two stages of (A, B): while the tensor core works on chunk c, the threads
// stage chunk c + 1 and the bulk copy brings its weights.  The accumulators
// of a tile are read out (hi and lo columns summed, bias added) after its
// last chunk.
#include <cuda_bf16.h>

#include "nsm_internal.h"
#include "tc_pipeline.cuh"
#include "train_internal.h"

namespace nsm {
namespace tr {

using namespace tc;

namespace {

constexpr int kDcThreads = 256;
constexpr int kDcNB = 64;          // output channels per CTA
constexpr int kDcN = 2 * kDcNB;    // MMA width: W_hi | W_lo
constexpr int kDcErrCode = 9;      // error word value of a wait in deep_conv_kernel that gave up

template <int K, int CC, int R>
struct DcCfg {
    static constexpr int SR = R + K - 1;                // staged rows
    static constexpr int SP = K == 3 ? 130 : 128;       // staged pixels used
    static constexpr int G = CC / 8;                    // channel groups per part
    static constexpr int KS = CC / 16;                  // K = 16 steps per tap
    static constexpr uint32_t PLANE = SR * kSW * 16;    // bytes per (part, group) plane
    static constexpr uint32_t A_BYTES = 2 * G * PLANE;
    static constexpr uint32_t B_BYTES = K * K * KS * 2 * kDcN * 16;
    static constexpr uint32_t STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t OFF_BAR = 2 * STAGE;
    static constexpr uint32_t BYTES = OFF_BAR + 64;     // 4 mbarriers, TMEM address slot
    static constexpr int ITEMS = SR * SP * G;
    static constexpr int S = (ITEMS + kDcThreads - 1) / kDcThreads;
    static constexpr int TMEM_COLS = R * kDcN;          // one accumulator block per image row
    static_assert(CC % 16 == 0, "whole K = 16 steps");
    static_assert(A_BYTES % 16 == 0 && B_BYTES % 16 == 0, "bulk-copy granularity");
    static_assert(BYTES <= 227 * 1024, "shared memory per CTA");
    static_assert(TMEM_COLS <= 512, "tensor memory");
    static_assert(PLANE / 16 < (1u << 14), "LBO field");
};

// Weight image of one layer: block (ob, c) = output channels 64 ob .. + 64,
// input channels CC c .. + CC; inside it chunk (tap, ks, half, n) holds the 8
// BF16 weights of MMA row n (n < 64: hi part of output 64 ob + n, else lo part
// of output 64 ob + n - 64) and input channels CC c + 16 ks + 8 half .. + 8.
__global__ void deep_pack_kernel(const float* __restrict__ w, int cin, int cout, int k, int cc, uint4* __restrict__ img) {
    const int taps = k * k, ks_n = cc / 16, nc = cin / cc, nob = (cout + kDcNB - 1) / kDcNB;
    const size_t chunks = static_cast<size_t>(nob) * nc * taps * ks_n * 2 * kDcN;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < chunks;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int n = static_cast<int>(i % kDcN);
        size_t r = i / kDcN;
        const int half = static_cast<int>(r % 2); r /= 2;
        const int ks = static_cast<int>(r % ks_n); r /= ks_n;
        const int tap = static_cast<int>(r % taps); r /= taps;
        const int c = static_cast<int>(r % nc);
        const int ob = static_cast<int>(r / nc);
        const int o = ob * kDcNB + n % kDcNB, part = n / kDcNB;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ch = c * cc + ks * 16 + half * 8 + j;
            const float x = o < cout ? __ldg(w + (static_cast<size_t>(o) * cin + ch) * taps + tap) : 0.f;
            const float hi = __bfloat162float(__float2bfloat16_rn(x));
            v[j] = part ? x - hi : x;
        }
        img[i] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                            pack_bf16x2(v[6], v[7]));
    }
}

template <int K, int CC, int R>
struct DcRegs {
    float4 a[DcCfg<K, CC, R>::S], b[DcCfg<K, CC, R>::S];
};

// Chunk c of tile (rows yr .. yr + R - 1, x0): item i = (staged row sr,
// group g, staged pixel sp; pixel fastest, so a warp's 16-byte stores fill
// whole rows of banks) covers image row yr - (K / 2) + sr, column
// x0 - (K / 2) + sp, channels CC c + 8 g .. + 8; zeros outside the image.
template <int K, int CC, int RR>
__device__ __forceinline__ void dc_load(DcRegs<K, CC, RR>& R, const float* __restrict__ x, int H, int W, int CIN,
                                        int yr, int x0, int c) {
    using C = DcCfg<K, CC, RR>;
#pragma unroll
    for (int s = 0; s < C::S; ++s) {
        const int i = threadIdx.x + s * kDcThreads;
        const int sp = i % C::SP, rest = i / C::SP;
        const int g = rest % C::G, sr = rest / C::G;
        const int yy = yr - K / 2 + sr, xx = x0 - K / 2 + sp;
        const bool in = i < C::ITEMS && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const float4* p = reinterpret_cast<const float4*>(
            x + (static_cast<size_t>(in ? yy : 0) * W + (in ? xx : 0)) * CIN + c * CC + 8 * g);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        R.a[s] = in ? __ldg(p) : z;
        R.b[s] = in ? __ldg(p + 1) : z;
    }
}

__device__ __forceinline__ uint32_t dc_bits(float v) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v)));
}

template <int K, int CC, int RR>
__device__ __forceinline__ void dc_store(const DcRegs<K, CC, RR>& R, uint32_t abase, int relu_in) {
    using C = DcCfg<K, CC, RR>;
#pragma unroll
    for (int s = 0; s < C::S; ++s) {
        const int i = threadIdx.x + s * kDcThreads;
        if (i >= C::ITEMS) break;
        const int sp = i % C::SP, rest = i / C::SP;
        const int g = rest % C::G, sr = rest / C::G;
        float f[8] = {R.a[s].x, R.a[s].y, R.a[s].z, R.a[s].w, R.b[s].x, R.b[s].y, R.b[s].z, R.b[s].w};
        uint32_t h[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float v0 = relu_in ? fmaxf(f[2 * k], 0.f) : f[2 * k];
            const float v1 = relu_in ? fmaxf(f[2 * k + 1], 0.f) : f[2 * k + 1];
            const uint32_t h0 = dc_bits(v0), h1 = dc_bits(v1);
            h[k] = h0 | (h1 << 16);
            l[k] = dc_bits(v0 - __uint_as_float(h0 << 16)) | (dc_bits(v1 - __uint_as_float(h1 << 16)) << 16);
        }
        const uint32_t off = static_cast<uint32_t>(g) * C::PLANE + static_cast<uint32_t>(sr * kSW + sp) * 16;
        st_shared_v4(abase + off, make_uint4(h[0], h[1], h[2], h[3]));
        st_shared_v4(abase + static_cast<uint32_t>(C::G) * C::PLANE + off, make_uint4(l[0], l[1], l[2], l[3]));
    }
}

// The chunk's MMAs (one thread): every image row of the tile, tap, K step and
// activation part; row r accumulates in tensor-memory columns r N .. + N.
template <int K, int CC, int R>
__device__ __forceinline__ void dc_mma(uint32_t abase, uint32_t bbase, uint32_t tbase, uint32_t acc0) {
    using C = DcCfg<K, CC, R>;
    constexpr uint32_t idesc = idesc_bf16(kTileM, kDcN);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        uint32_t acc = acc0;
#pragma unroll
        for (int tap = 0; tap < K * K; ++tap) {
            const int ky = tap / K, kx = tap % K;
#pragma unroll
            for (int ks = 0; ks < C::KS; ++ks) {
                const uint64_t bdesc =
                    smem_desc(bbase + static_cast<uint32_t>((tap * C::KS + ks) * 2 * kDcN) * 16, kDcN * 16, 128);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const uint32_t a = abase + static_cast<uint32_t>(p * C::G + 2 * ks) * C::PLANE +
                                       static_cast<uint32_t>((r + ky) * kSW + kx) * 16;
                    mma_bf16(tbase + static_cast<uint32_t>(r * kDcN), smem_desc(a, C::PLANE, 128), bdesc, idesc, acc);
                    acc = 1;
                }
            }
        }
    }
}

template <int K, int CC, int RR>
__global__ void __launch_bounds__(kDcThreads) deep_conv_kernel(const float* __restrict__ x, int relu_in, int H, int W,
                                                               int CIN, int COUT, const uint4* __restrict__ img,
                                                               const float* __restrict__ bias, float* __restrict__ y,
                                                               int relu_out, int* err) {
    using C = DcCfg<K, CC, RR>;
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

    const int tiles_x = (W + kTileM - 1) / kTileM, nob = (COUT + kDcNB - 1) / kDcNB, nc = CIN / CC;
    const int tiles_y = (H + RR - 1) / RR;
    const long long ntiles = static_cast<long long>(tiles_y) * tiles_x * nob;
    const uint32_t block_chunks = C::B_BYTES / 16;
    uint32_t fph[2] = {0u, 0u}, dph[2] = {0u, 0u};  // phase parities of full[] (thread 0) and done[]
    int pend[2] = {0, 0};                           // commits on done[s] not yet waited for
    bool ok = true;
    int it = 0;
    DcRegs<K, CC, RR> R;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int ob = static_cast<int>(t % nob);
        const long long r = t / nob;
        const int x0 = static_cast<int>(r % tiles_x) * kTileM, yr = static_cast<int>(r / tiles_x) * RR;
        for (int c = 0; c < nc; ++c, ++it) {
            const int s = it & 1;
            const uint32_t abase = sbase + s * C::STAGE, bbase = abase + C::A_BYTES;
            dc_load<K, CC, RR>(R, x, H, W, CIN, yr, x0, c);  // in flight while the other stage's MMAs run
            if (pend[s]) {                               // stage s free: its last MMAs finished
                ok = mbar_wait_bounded(&done[s], dph[s], kWaitNs);
                dph[s] ^= 1u;
                pend[s] = 0;
            }
            if (__syncthreads_or(!ok)) { ok = false; break; }
            if (tid == 0) {
                mbar_arrive_expect_tx(&full[s], C::B_BYTES);
                bulk_load(bbase, img + (static_cast<size_t>(ob) * nc + c) * block_chunks, C::B_BYTES, &full[s]);
            }
            dc_store<K, CC, RR>(R, abase, relu_in);
            fence_proxy_async_smem();  // the staged operand, visible to the tensor core
            __syncthreads();
            if (tid == 0) {
                if (mbar_wait_bounded(&full[s], fph[s], kWaitNs)) {
                    fence_after_sync();
                    dc_mma<K, CC, RR>(abase, bbase, tbase, c > 0 ? 1u : 0u);
                } else {
                    atomicExch(err, kDcErrCode);
                }
                mma_commit(&done[s]);  // also when nothing was issued: the phase still completes
            }
            fph[s] ^= 1u;
            pend[s] = 1;
        }
        if (!ok) break;
        // the tile's accumulators: its last commit covers every earlier MMA
        const int sl = (it - 1) & 1;
        ok = mbar_wait_bounded(&done[sl], dph[sl], kWaitNs);
        dph[sl] ^= 1u;
        pend[sl] = 0;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        fence_after_sync();
        // warp w: TMEM lane quarter w % 4 (pixels); (row, 32-output half) pairs
        // j = w / 4, w / 4 + 4, ... of the tile
        const int lq = warp & 3;
        const int px = x0 + 32 * lq + lane;
#pragma unroll 1
        for (int j = warp >> 2; j < 2 * RR; j += kDcThreads / 128) {
            const int rr = j >> 1, o0 = ob * kDcNB + 32 * (j & 1);
            float a[32], b[32];
            const uint32_t tq = tbase + (static_cast<uint32_t>(32 * lq) << 16) +
                                static_cast<uint32_t>(rr * kDcN + 32 * (j & 1));
            tmem_ld32(tq, a);
            tmem_ld32(tq + kDcNB, b);
            tmem_ld_wait();
            if (px < W && yr + rr < H && o0 < COUT) {
                float* out = y + (static_cast<size_t>(yr + rr) * W + px) * COUT + o0;
#pragma unroll
                for (int o = 0; o < 32; o += 4) {
                    float4 v = make_float4(a[o] + b[o] + __ldg(bias + o0 + o), a[o + 1] + b[o + 1] + __ldg(bias + o0 + o + 1),
                                           a[o + 2] + b[o + 2] + __ldg(bias + o0 + o + 2),
                                           a[o + 3] + b[o + 3] + __ldg(bias + o0 + o + 3));
                    if (relu_out) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
                    *reinterpret_cast<float4*>(out + o) = v;
                }
            }
        }
        // accumulators read out before the next tile's first MMA overwrites them
        fence_before_sync();
        __syncthreads();
    }
    // no MMA of this CTA left running on its shared memory or tensor memory
    for (int s = 0; s < 2; ++s)
        if (pend[s]) {
            if (!mbar_wait_bounded(&done[s], dph[s], kWaitNs)) atomicExch(err, kDcErrCode);
            dph[s] ^= 1u;
        }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, C::TMEM_COLS);
}

template <int K, int CC, int RR>
cudaError_t launch_deep_conv(const float* x, int relu_in, int H, int W, int cin, int cout, const uint4* img,
                             const float* bias, float* y, int relu_out, int* err, cudaStream_t st) {
    using C = DcCfg<K, CC, RR>;
    static int per_sm = 0;  // CTAs resident per SM (per instantiation, set on first use)
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(deep_conv_kernel<K, CC, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C::BYTES));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(deep_conv_kernel<K, CC, RR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        const int occ = resident_ctas_per_sm(reinterpret_cast<const void*>(deep_conv_kernel<K, CC, RR>), kDcThreads,
                                             C::BYTES);
        per_sm = occ < 512 / C::TMEM_COLS ? occ : 512 / C::TMEM_COLS;
    }
    const long long tiles =
        static_cast<long long>((H + RR - 1) / RR) * ((W + kTileM - 1) / kTileM) * ((cout + kDcNB - 1) / kDcNB);
    if (tiles == 0) return cudaSuccess;
    const long long cap = static_cast<long long>(num_sms()) * per_sm;
    const int grid = static_cast<int>(tiles < cap ? tiles : cap);
    deep_conv_kernel<K, CC, RR><<<grid, kDcThreads, C::BYTES, st>>>(x, relu_in, H, W, cin, cout, img, bias, y,
                                                                      relu_out, err);
    return cudaGetLastError();
}

constexpr int cc_of(int k) { return k == 3 ? 16 : 64; }

}  // namespace

bool deep_tc_supported(int cin, int cout, int k) {
    return (k == 3 || k == 1) && cin > 0 && cin % cc_of(k) == 0 && cout > 0 && cout % 32 == 0;
}

size_t deep_tc_image_bytes(int cin, int cout, int k) {
    if (!deep_tc_supported(cin, cout, k)) return 0;
    return static_cast<size_t>((cout + kDcNB - 1) / kDcNB) * cin * k * k / 16 * 2 * kDcN * 16;
}

cudaError_t deep_tc_pack(const float* w, int cin, int cout, int k, uint4* img, cudaStream_t st) {
    if (!deep_tc_supported(cin, cout, k)) return cudaErrorInvalidValue;
    const size_t chunks = deep_tc_image_bytes(cin, cout, k) / 16;
    const size_t blocks = (chunks + 255) / 256;
    const size_t cap = static_cast<size_t>(num_sms()) * 8;
    deep_pack_kernel<<<static_cast<int>(blocks < cap ? blocks : cap), 256, 0, st>>>(w, cin, cout, k, cc_of(k), img);
    return cudaGetLastError();
}

cudaError_t deep_tc_conv(int cin, int cout, int k, const float* x, int relu_in, int H, int W, const uint4* img,
                         const float* bias, float* y, int relu_out, int* err, cudaStream_t st) {
    if (!deep_tc_supported(cin, cout, k)) return cudaErrorInvalidValue;
    if (k == 1) return launch_deep_conv<1, 64, 1>(x, relu_in, H, W, cin, cout, img, bias, y, relu_out, err, st);
    // a 3x3 tile of R image rows reuses each streamed weight chunk R times:
    // the largest R whose tiles still give every SM one
    const long long per_row = static_cast<long long>((W + kTileM - 1) / kTileM) * ((cout + kDcNB - 1) / kDcNB);
    const long long sms = num_sms();
    if (static_cast<long long>((H + 3) / 4) * per_row >= sms)
        return launch_deep_conv<3, 16, 4>(x, relu_in, H, W, cin, cout, img, bias, y, relu_out, err, st);
    if (static_cast<long long>((H + 1) / 2) * per_row >= sms)
        return launch_deep_conv<3, 16, 2>(x, relu_in, H, W, cin, cout, img, bias, y, relu_out, err, st);
    return launch_deep_conv<3, 16, 1>(x, relu_in, H, W, cin, cout, img, bias, y, relu_out, err, st);
}

}  // namespace tr
}  // namespace nsm
