// Tensor-core 3x3 convolutions of the training backward (Sec. 3.3, Eq. 2
// adjoint; network of Sec. 3.5): the recomputed 3x3 pre-activations
//   y[n, p, o] = b[o] + sum_{c, tap} W[o][c][tap] x[n, p + off(tap), c]
// and the data gradients, which are the same convolution with the
// transposed, flipped weights Wd[c][o][tap] = W[o][c][8 - tap] applied to
// the output gradient.  FP32 NHWC tensors in and out, as the rest of the
// training path; the products run on tcgen05 in compensated BF16: every
// activation and weight is a pair hi = bf16(v), lo = bf16(v - hi), and the
// four products hi.hi + hi.lo + lo.hi + lo.lo accumulate in FP32 in tensor
// memory (about 2^-16 relative per operand instead of BF16's 2^-9).
//
// Implicit GEMM, D[pixels x C_out] = A[pixels x 9 C_in] B[C_out x 9 C_in]^T:
//   tile      R image rows x 128 pixels; one 128 x N x 16 MMA row block per
//             row, N = 2 C_out (the hi and lo weight parts side by side along
//             N, summed in the epilogue)
//   A         the tile with its one-pixel halo staged once in shared memory
//             as [part][channel group][staged row][staged pixel] 16-byte
//             chunks of 8 channels: the no-swizzle K-major operand layout, so
//             the operand of tap (ky, kx) is the same planes started ky rows
//             and kx chunks further on (no im2col); one K = 16 step covers
//             two channel groups of one part
//   B         every tap's weight image of the layer, packed once per step by
//             pack_conv3_kernel into the same chunk layout and staged once
//             per CTA
// Each CTA loops over tiles: all threads stage the tile (FP32 -> hi + lo),
// one thread issues the tile's MMAs and commits them to an mbarrier while
// every thread loads part of the next tile into registers, then all
// threads read the accumulators out (hi + lo parts summed, bias added) and
// store FP32.  Shared memory and TMEM are sized so that two to four CTAs
// share an SM and one CTA's staging overlaps another's MMAs and stores.
#include <cuda_bf16.h>

#include "nsm_internal.h"
#include "tc_pipeline.cuh"
#include "train_internal.h"

namespace nsm {
namespace tr {

using namespace tc;

template <int CIN, int COUT>
struct Conv3Cfg {
    static constexpr int CINP = (CIN + 15) / 16 * 16;        // K padded to whole K = 16 steps
    static constexpr int COUTP = COUT < 8 ? 8 : COUT;        // N = 2 COUTP >= 16
    static constexpr int G = CINP / 8;                       // channel groups per part
    static constexpr int KP = CINP / 16;                     // K = 16 steps per tap and part
    static constexpr int N = 2 * COUTP;                      // MMA width: W_hi | W_lo
    static constexpr int R = (CINP <= 16 && COUTP <= 16) ? 4 : 2;  // image rows per tile
    static constexpr int SR = R + 2;                         // staged rows
    static constexpr int SP = 130;                           // staged pixels used (128 + halo)
    static constexpr uint32_t PLANE = SR * kSW * 16;         // bytes per (part, group) plane
    static constexpr uint32_t A_BYTES = 2 * G * PLANE;
    static constexpr uint32_t B_CHUNKS = 9 * KP * 2 * N;     // weight image, 16-byte chunks
    static constexpr uint32_t OFF_B = A_BYTES;
    static constexpr uint32_t OFF_BIAS = OFF_B + B_CHUNKS * 16;
    static constexpr uint32_t OFF_BAR = OFF_BIAS + COUTP * 4;
    static constexpr uint32_t BYTES_USED = OFF_BAR + 16 + 16;  // mbarrier, TMEM address slot
    static constexpr int TMEM_RAW = R * N;
    static constexpr int TMEM_COLS = TMEM_RAW <= 32 ? 32 : TMEM_RAW <= 64 ? 64 : TMEM_RAW <= 128 ? 128 : 256;
    // enough shared memory per CTA that the CTAs resident on one SM never ask
    // for more than its 512 TMEM columns (at most 228 KB of shared memory per SM)
    static constexpr int TMEM_CAP = 512 / TMEM_COLS;
    static constexpr uint32_t BYTES_MIN = (236u * 1024u) / (TMEM_CAP + 1);
    static constexpr uint32_t BYTES = BYTES_USED < BYTES_MIN ? BYTES_MIN : BYTES_USED;
    static_assert(CIN == 4 || CIN % 16 == 0, "C_in: 4 or a multiple of 16");
    static_assert(COUT == 4 || COUT % 8 == 0, "C_out: 4 or a multiple of 8");
    static_assert(N <= 256, "MMA width");
    static_assert(BYTES_USED <= 227 * 1024, "shared memory per CTA");
    static_assert(PLANE / 16 < (1u << 14), "LBO field");
};

// ------------------------------------------------------------------ weight images
// One image per (layer, orientation): chunk (tap, kp, h, n) holds the 8 BF16
// weights of output row n (n < COUTP: hi part of output n, else lo part of
// output n - COUTP) and input channels 8 (2 kp + h) .. + 8.  Orientation 0
// is the layer's own convolution (C_in -> C_out of the layer); orientation 1
// its data gradient (C_out -> C_in, weights transposed and flipped).
struct Conv3Pack {
    int w_off;       // OIHW weights of the layer in the parameter vector
    int cin, cout;   // the layer's own shape
    int flip;        // orientation
    int img_off;     // first chunk of the image in the image buffer
};

struct Conv3Table { Conv3Pack e[kConv3Images]; };

// grid.y = one image each
__global__ void pack_conv3_kernel(const float* __restrict__ theta, const Conv3Table tab, uint4* __restrict__ img) {
    const Conv3Pack d = tab.e[blockIdx.y];
    const int cin = d.flip ? d.cout : d.cin, cout = d.flip ? d.cin : d.cout;  // of the convolution computed
    const int cinp = (cin + 15) / 16 * 16, coutp = cout < 8 ? 8 : cout;
    const int kp = cinp / 16, n = 2 * coutp;
    const int chunks = 9 * kp * 2 * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < chunks; i += gridDim.x * blockDim.x) {
        const int row = i % n, h = (i / n) % 2, k = (i / (2 * n)) % kp, tap = i / (2 * n * kp);
        const int o = row % coutp, part = row / coutp;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = (2 * k + h) * 8 + j;
            float w = 0.f;
            if (c < cin && o < cout)
                w = d.flip ? theta[d.w_off + (c * d.cin + o) * 9 + (8 - tap)]   // W[c][o][8 - tap]
                           : theta[d.w_off + (o * d.cin + c) * 9 + tap];        // W[o][c][tap]
            const float hi = __bfloat162float(__float2bfloat16_rn(w));
            v[j] = part ? w - hi : w;
        }
        img[d.img_off + i] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                                        pack_bf16x2(v[6], v[7]));
    }
}

// BF16 hi + lo chunks of 8 FP32 values (v - hi is exact in FP32)
__device__ __forceinline__ void split8(const float* f, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = pack_bf16x2(f[2 * k], f[2 * k + 1]);
        l[k] = pack_bf16x2(f[2 * k] - __uint_as_float(h[k] << 16), f[2 * k + 1] - __uint_as_float(h[k] & 0xffff0000u));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

constexpr int kConv3Threads = 256;
constexpr int kConv3ErrCode = 7;  // error word value of a wait in conv3_tc_kernel that gave up

// One tile's input with its halo, item by item: thread t takes items t,
// t + 256, ... (item = staged row sr, channel group g of 8 channels, staged
// pixel sp; pixel fastest, so a warp's 16-byte stores fill whole rows of
// banks); staged row sr = image row y0 - 1 + sr, staged pixel sp = column
// x0 - 1 + sp; zeros outside the image and beyond C_in.  The first PS items of
// a thread are loaded into registers one tile ahead (in flight while the
// current tile's MMAs run), the rest when the tile is staged; a thread issues
// all of a phase's loads before it uses any.
template <int CIN, int COUT>
struct Conv3Regs {
    using C = Conv3Cfg<CIN, COUT>;
    static constexpr int ITEMS = C::SR * C::SP * C::G;
    static constexpr int S = (ITEMS + kConv3Threads - 1) / kConv3Threads;
    static constexpr int PS = S < 4 ? S : 4;  // items loaded ahead (registers)
    float4 a[PS], b[PS];
};

template <int CIN, int COUT>
__device__ __forceinline__ void conv3_item_load(const float* __restrict__ x, int i, int n, int H, int W, int y0,
                                                int x0, float4& a, float4& b) {
    using C = Conv3Cfg<CIN, COUT>;
    const int sp = i % C::SP, rest = i / C::SP;
    const int g = rest % C::G, sr = rest / C::G;
    const int yy = y0 - 1 + sr, xx = x0 - 1 + sp;
    const bool in = i < Conv3Regs<CIN, COUT>::ITEMS && yy >= 0 && yy < H && xx >= 0 && xx < W && 8 * g < CIN;
    const float4* p = reinterpret_cast<const float4*>(
        x + ((static_cast<size_t>(n) * H + (in ? yy : 0)) * W + (in ? xx : 0)) * CIN + (in ? 8 * g : 0));
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    a = in ? __ldg(p) : z;
    b = (in && CIN >= 8) ? __ldg(p + 1) : z;
}

template <int CIN, int COUT>
__device__ __forceinline__ void conv3_load(Conv3Regs<CIN, COUT>& R, const float* __restrict__ x, int n, int H, int W,
                                           int y0, int x0) {
#pragma unroll
    for (int s = 0; s < Conv3Regs<CIN, COUT>::PS; ++s)
        conv3_item_load<CIN, COUT>(x, threadIdx.x + s * kConv3Threads, n, H, W, y0, x0, R.a[s], R.b[s]);
}

template <int CIN, int COUT>
__device__ __forceinline__ void conv3_store(const Conv3Regs<CIN, COUT>& R, uint32_t sbase, const float* __restrict__ x,
                                            int n, int H, int W, int y0, int x0) {
    using C = Conv3Cfg<CIN, COUT>;
    using RT = Conv3Regs<CIN, COUT>;
    constexpr int NL = RT::S - RT::PS;  // items loaded now
    float4 la[NL > 0 ? NL : 1], lb[NL > 0 ? NL : 1];
#pragma unroll
    for (int s = 0; s < NL; ++s)
        conv3_item_load<CIN, COUT>(x, threadIdx.x + (RT::PS + s) * kConv3Threads, n, H, W, y0, x0, la[s], lb[s]);
#pragma unroll
    for (int s = 0; s < RT::S; ++s) {
        const int i = threadIdx.x + s * kConv3Threads;
        if (i >= RT::ITEMS) break;
        const int sp = i % C::SP, rest = i / C::SP;
        const int g = rest % C::G, sr = rest / C::G;
        const float4 a = s < RT::PS ? R.a[s < RT::PS ? s : 0] : la[s < RT::PS ? 0 : s - RT::PS];
        const float4 b = s < RT::PS ? R.b[s < RT::PS ? s : 0] : lb[s < RT::PS ? 0 : s - RT::PS];
        const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint4 hi, lo;
        split8(f, hi, lo);
        const uint32_t off = static_cast<uint32_t>(g) * C::PLANE + static_cast<uint32_t>(sr * kSW + sp) * 16;
        st_shared_v4(sbase + off, hi);
        st_shared_v4(sbase + static_cast<uint32_t>(C::G) * C::PLANE + off, lo);
    }
}

// The tile's MMAs (one thread): output row r accumulates, over taps (ky, kx),
// parts p and K steps k, the planes (p, 2k), (p, 2k + 1) started at staged row
// r + ky and pixel kx against the weight chunks of (tap, k).
template <int CIN, int COUT>
__device__ __forceinline__ void conv3_mma(uint32_t sbase, uint32_t tbase) {
    using C = Conv3Cfg<CIN, COUT>;
    constexpr uint32_t idesc = idesc_bf16(kTileM, C::N);
#pragma unroll 1
    for (int r = 0; r < C::R; ++r) {
        uint32_t acc = 0;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int k = 0; k < C::KP; ++k) {
                const uint64_t bdesc =
                    smem_desc(sbase + C::OFF_B + static_cast<uint32_t>((tap * C::KP + k) * 2 * C::N) * 16, C::N * 16, 128);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const uint32_t a = sbase + static_cast<uint32_t>(p * C::G + 2 * k) * C::PLANE +
                                       static_cast<uint32_t>((r + ky) * kSW + kx) * 16;
                    mma_bf16(tbase + static_cast<uint32_t>(r * C::N), smem_desc(a, C::PLANE, 128), bdesc, idesc, acc);
                    acc = 1;
                }
            }
        }
    }
}

// Accumulators of row r of the tile -> FP32 outputs (hi + lo weight parts
// summed, bias added); warp w reads TMEM lane quarter w % 4 (pixels
// 32 (w % 4) .. + 32) of rows r = w / 4, w / 4 + 2, ...  C1 > 0: the pixel's
// 1x1 outputs y1 = b1 + sum_c W1[.][c] relu(y[c]) as well, c ascending (the
// separate 1x1 layer's order), from w1s [c][o] and b1s in shared memory.
template <int CIN, int COUT, int C1>
__device__ __forceinline__ void conv3_epilogue(uint32_t tbase, const float* bias_s, float* __restrict__ y, int n, int H,
                                               int W, int y0, int x0, const float* w1s, const float* b1s,
                                               float* __restrict__ y1) {
    using C = Conv3Cfg<CIN, COUT>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
    const int xx = x0 + 32 * q + lane;
    const uint32_t tq = tbase + (static_cast<uint32_t>(32 * q) << 16);
#pragma unroll 1
    for (int r = warp >> 2; r < C::R; r += kConv3Threads / 128) {
        const int yy = y0 + r;
        const bool ok = yy < H && xx < W;
        const size_t pix = (static_cast<size_t>(n) * H + (ok ? yy : 0)) * W + (ok ? xx : 0);
        float* out = y + pix * COUT;
        const uint32_t tr = tq + static_cast<uint32_t>(r * C::N);
        float z[C1 > 0 ? C1 : 1];
        if constexpr (C1 > 0) {
#pragma unroll
            for (int o = 0; o < C1; ++o) z[o] = b1s[o];
        }
        // the 1x1's products with channels c0 .. c0 + nc of the 3x3 output
        auto fuse = [&](const float* v, int c0, int nc) {
            if constexpr (C1 > 0) {
#pragma unroll
                for (int c = 0; c < nc; ++c) {
                    const float xr = fmaxf(v[c], 0.f);
                    const float4* w4 = reinterpret_cast<const float4*>(w1s + (c0 + c) * C1);
#pragma unroll
                    for (int o = 0; o < C1; o += 4) {
                        const float4 w = w4[o / 4];
                        z[o] = fmaf(xr, w.x, z[o]);
                        z[o + 1] = fmaf(xr, w.y, z[o + 1]);
                        z[o + 2] = fmaf(xr, w.z, z[o + 2]);
                        z[o + 3] = fmaf(xr, w.w, z[o + 3]);
                    }
                }
            }
        };
        if constexpr (C::N <= 32) {
            float v[32];
            if constexpr (C::N == 16) tmem_ld16(tr, *reinterpret_cast<float(*)[16]>(v));
            else tmem_ld32(tr, v);
            tmem_ld_wait();
            float s[COUT];
#pragma unroll
            for (int o = 0; o < COUT; ++o) s[o] = v[o] + v[C::COUTP + o] + bias_s[o];
            if (ok) {
#pragma unroll
                for (int o = 0; o < COUT; o += 4)
                    *reinterpret_cast<float4*>(out + o) = make_float4(s[o], s[o + 1], s[o + 2], s[o + 3]);
            }
            fuse(s, 0, COUT);
        } else {
#pragma unroll 1
            for (int o0 = 0; o0 < COUT; o0 += 32) {
                float a[32], b[32];
                tmem_ld32(tr + o0, a);
                tmem_ld32(tr + C::COUTP + o0, b);
                tmem_ld_wait();
#pragma unroll
                for (int o = 0; o < 32; ++o) a[o] = a[o] + b[o] + bias_s[o0 + o];
                if (ok) {
#pragma unroll
                    for (int o = 0; o < 32; o += 4)
                        *reinterpret_cast<float4*>(out + o0 + o) = make_float4(a[o], a[o + 1], a[o + 2], a[o + 3]);
                }
                fuse(a, o0, 32);
            }
        }
        if constexpr (C1 > 0) {
            if (ok) {
                float* out1 = y1 + pix * C1;
#pragma unroll
                for (int o = 0; o < C1; o += 4)
                    *reinterpret_cast<float4*>(out1 + o) = make_float4(z[o], z[o + 1], z[o + 2], z[o + 3]);
            }
        }
    }
}

// Shared memory of the kernel with a fused 1x1 (C1 > 0): its weights [c][o]
// and bias after the 3x3 kernel's own regions.
template <int CIN, int COUT, int C1>
struct Conv3Fuse {
    using C = Conv3Cfg<CIN, COUT>;
    static constexpr uint32_t OFF_W1 = (C::BYTES_USED + 15) / 16 * 16;
    static constexpr uint32_t USED = OFF_W1 + (C1 > 0 ? static_cast<uint32_t>(COUT * C1 + C1) * 4 : 0);
    static constexpr uint32_t BYTES = USED < C::BYTES_MIN ? C::BYTES_MIN : USED;
    static_assert(USED <= 227 * 1024, "shared memory per CTA");
    static_assert(C1 % 4 == 0 && COUT % 4 == 0, "float4 rows");
};

template <int CIN, int COUT, int C1>
__global__ void __launch_bounds__(kConv3Threads) conv3_tc_kernel(const float* __restrict__ x, int NI, int H, int W,
                                                                 const uint4* __restrict__ img,
                                                                 const float* __restrict__ bias, float* __restrict__ y,
                                                                 int* err, const float* __restrict__ w1,
                                                                 const float* __restrict__ b1,
                                                                 float* __restrict__ y1) {
    using C = Conv3Cfg<CIN, COUT>;
    using F = Conv3Fuse<CIN, COUT, C1>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 16);
    float* bias_s = reinterpret_cast<float*>(smem + C::OFF_BIAS);
    const uint32_t sbase = smem_u32(smem);
    // the weight image and the bias, once per CTA
    for (int i = tid; i < static_cast<int>(C::B_CHUNKS); i += kConv3Threads)
        st_shared_v4(sbase + C::OFF_B + 16u * i, __ldg(img + i));
    for (int i = tid; i < C::COUTP; i += kConv3Threads) bias_s[i] = (bias != nullptr && i < COUT) ? bias[i] : 0.f;
    float* w1s = reinterpret_cast<float*>(smem + F::OFF_W1);  // [c][o], then b1
    if constexpr (C1 > 0) {
        for (int i = tid; i < COUT * C1; i += kConv3Threads) w1s[i] = __ldg(w1 + (i % C1) * COUT + i / C1);
        for (int i = tid; i < C1; i += kConv3Threads) w1s[COUT * C1 + i] = b1 != nullptr ? __ldg(b1 + i) : 0.f;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, C::TMEM_COLS);
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    const int tiles_x = (W + kTileM - 1) / kTileM, tiles_y = (H + C::R - 1) / C::R;
    const long long ntiles = static_cast<long long>(NI) * tiles_y * tiles_x;
    auto tile_origin = [&](long long t, int& n, int& y0, int& x0) {
        const int tx = static_cast<int>(t % tiles_x);
        const long long t2 = t / tiles_x;
        n = static_cast<int>(t2 / tiles_y);
        y0 = static_cast<int>(t2 % tiles_y) * C::R;
        x0 = tx * kTileM;
    };
    Conv3Regs<CIN, COUT> Rg;
    if (blockIdx.x < ntiles) {
        int n, y0, x0;
        tile_origin(blockIdx.x, n, y0, x0);
        conv3_load<CIN, COUT>(Rg, x, n, H, W, y0, x0);
    }
    uint32_t phase = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int n, y0, x0;
        tile_origin(t, n, y0, x0);
        conv3_store<CIN, COUT>(Rg, sbase, x, n, H, W, y0, x0);
        fence_proxy_async_smem();  // the staged operand, visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            conv3_mma<CIN, COUT>(sbase, tbase);
            mma_commit(bar);
        }
        if (t + gridDim.x < ntiles) {  // the next tile's loads, in flight during the MMAs
            int n2, y2, x2;
            tile_origin(t + gridDim.x, n2, y2, x2);
            conv3_load<CIN, COUT>(Rg, x, n2, H, W, y2, x2);
        }
        bool ok = mbar_wait_bounded(bar, phase, kWaitNs);
        phase ^= 1u;
        if (!ok) {
            atomicExch(err, kConv3ErrCode);
        } else {
            fence_after_sync();
            conv3_epilogue<CIN, COUT, C1>(tbase, bias_s, y, n, H, W, y0, x0, w1s, w1s + COUT * C1, y1);
        }
        // TMEM read out and the operand consumed before the next tile
        fence_before_sync();
        if (__syncthreads_or(!ok)) break;
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, C::TMEM_COLS);
}

// ------------------------------------------------------------------ host side
template <int CIN, int COUT, int C1>
static cudaError_t launch_conv3(const float* x, int N, int H, int W, const uint4* img, const float* bias, float* y,
                                int* err, cudaStream_t st, const float* w1, const float* b1, float* y1) {
    using C = Conv3Cfg<CIN, COUT>;
    using F = Conv3Fuse<CIN, COUT, C1>;
    auto kern = conv3_tc_kernel<CIN, COUT, C1>;
    static int grid_cap = 0;  // CTAs resident on the device (per instantiation, set on first use)
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F::BYTES));
        if (e != cudaSuccess) return e;
        // all of the unified L1 / shared storage as shared memory: two to four CTAs per SM
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        per_sm = resident_ctas_per_sm(reinterpret_cast<const void*>(kern), kConv3Threads, F::BYTES);
        grid_cap = sms * (per_sm < C::TMEM_CAP ? per_sm : C::TMEM_CAP);
    }
    const long long tiles = static_cast<long long>(N) * ((H + C::R - 1) / C::R) * ((W + kTileM - 1) / kTileM);
    if (tiles == 0) return cudaSuccess;
    const int grid = tiles < grid_cap ? static_cast<int>(tiles) : grid_cap;
    kern<<<grid, kConv3Threads, F::BYTES, st>>>(x, N, H, W, img, bias, y, err, w1, b1, y1);
    return cudaGetLastError();
}

cudaError_t conv3_tc(int cin, int cout, const float* x, int N, int H, int W, const uint4* img, const float* bias,
                     float* y, int* err, cudaStream_t st, const float* w1, const float* b1, int c1, float* y1) {
#define NSM_CONV3(a, b, c)                \
    if (cin == a && cout == b && c1 == c) \
        return launch_conv3<a, b, c>(x, N, H, W, img, bias, y, err, st, w1, b1, y1);
    NSM_CONV3(4, 16, 0) NSM_CONV3(16, 16, 0) NSM_CONV3(16, 32, 0) NSM_CONV3(32, 16, 0) NSM_CONV3(32, 32, 0)
    NSM_CONV3(32, 64, 0) NSM_CONV3(64, 32, 0) NSM_CONV3(16, 4, 0)
    // the levels' 3x3 + 1x1 pairs (enc0 and dec0, enc1, bottleneck, dec1)
    NSM_CONV3(4, 16, 16) NSM_CONV3(16, 16, 16) NSM_CONV3(16, 32, 32) NSM_CONV3(32, 64, 32) NSM_CONV3(32, 32, 16)
#undef NSM_CONV3
    return cudaErrorInvalidValue;
}

// The 3x3 layers of the network in image order; images 2 l (the layer) and
// 2 l + 1 (its data gradient).
static const int kConv3Layers[kConv3Images / 2] = {ENC0_3, ENC1_3, BOTT_3, DEC1_3, DEC0_3};
static const int kConv3Shape[kConv3Images / 2][2] = {{4, 16}, {16, 32}, {32, 64}, {32, 32}, {16, 16}};

static int conv3_image_chunks(int cin, int cout) {
    const int cinp = (cin + 15) / 16 * 16, coutp = cout < 8 ? 8 : cout;
    return 9 * (cinp / 16) * 2 * (2 * coutp);
}

Conv3Images conv3_images() {
    Conv3Images t{};
    int off = 0;
    for (int l = 0; l < kConv3Images / 2; ++l)
        for (int f = 0; f < 2; ++f) {
            const int cin = kConv3Shape[l][0], cout = kConv3Shape[l][1];
            t.off[2 * l + f] = off;
            off += f ? conv3_image_chunks(cout, cin) : conv3_image_chunks(cin, cout);
        }
    t.total_chunks = off;
    return t;
}

cudaError_t conv3_pack(const float* theta, uint4* img, cudaStream_t st) {
    Conv3Table tab{};
    const LayerOffsets o = layer_offsets();
    const Conv3Images im = conv3_images();
    for (int l = 0; l < kConv3Images / 2; ++l)
        for (int f = 0; f < 2; ++f)
            tab.e[2 * l + f] = Conv3Pack{static_cast<int>(o.w[kConv3Layers[l]]), kConv3Shape[l][0], kConv3Shape[l][1],
                                         f, im.off[2 * l + f]};
    pack_conv3_kernel<<<dim3(8, kConv3Images), 256, 0, st>>>(theta, tab, img);
    return cudaGetLastError();
}

}  // namespace tr
}  // namespace nsm
