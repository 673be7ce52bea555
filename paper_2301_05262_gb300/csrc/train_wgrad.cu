// Tensor-core weight gradients of the training backward (Sec. 3.3, Eq. 2
// adjoint; network of Sec. 3.5):
//   dW[o][c][ky][kx] = sum_p g~[p][o] x~[p + (ky - 1, kx - 1)][c],   db[o] = sum_p g~[p][o]
// for the 3x3 layers (x zero outside the image) and, with the single tap, for
// the 1x1 layers (x~ = relu(x) where the layer reads a pre-activation, g~ = g
// masked by (m > 0) where the caller passes the layer output's ReLU mask m).
//
// The sum over every pixel of the batch is the K dimension of a GEMM
//   D[(kx, part_g, o)][(ky, part_x, c)] = sum_q A[q][(kx, part_g, o)] B[q][(ky, part_x, c)]
// over the pixels q of a tile of 8 image rows x TW columns; one 16-byte K
// chunk (8 BF16 values) holds one image column of the tile's 8 rows.  Both
// operands use the no-swizzle K-major layout with the row groups of one K
// column side by side (the 8-row stride is 128 bytes, the K-half stride one
// column's groups):
//   A  g~ at image column x0 + q - (kx - 1): one staged copy per horizontal
//      tap offset, so the offset is a shift by whole chunks, stacked along M
//   B  x~ at image rows y0 + r + ky - 1: one staged copy per vertical offset
//      (rows y0 - 1 .. y0 + 8 loaded once), stacked along N, then 8 rows of
//      ones (the bias gradient) and 8 rows of zeros
// Compensated BF16: every value v of g~ and x~ is a pair hi = bf16(v),
// lo = bf16(v - hi), both parts stacked (g along M, x along N), so D holds the
// four part products of every weight; the epilogue sums them in FP32.  One
// MMA (M = 128, N = 8 (6 C_in + 2)) per K step covers every tap held by the
// CTA; a layer too wide for one CTA's tensor memory takes one horizontal
// offset per CTA (grid.y = 3).  M rows beyond the real (kx, part, o) rows read
// whatever the neighbouring groups hold; their accumulators are never read.
//
// Each CTA accumulates all of its tiles in tensor memory and writes one slot
// of partial sums to global memory (every entry of its taps, zero when it
// gave up); a second kernel adds the slots in a fixed order to the gradient.
// No atomics: the gradient is the same bits from run to run on a device.
#include <cuda_bf16.h>

#include "nsm_internal.h"
#include "tc_pipeline.cuh"
#include "train_internal.h"

namespace nsm {
namespace tr {

using namespace tc;

namespace {

constexpr int kWgThreads = 256;
constexpr int kWgErrCode = 8;  // error word value of a wait in wgrad_tc_kernel that gave up

template <int CIN, int COUT, int K, int KXS, int TW>
struct WgCfg {
    static constexpr int CINP = CIN < 8 ? 8 : CIN;         // input channels padded to whole chunks
    static constexpr int CG = CINP / 8;
    static constexpr int OG = COUT / 8;
    static constexpr int NKY = K;                          // staged copies of x (vertical offsets)
    static constexpr int NKX = K == 3 ? KXS : 1;           // staged copies of g (horizontal offsets)
    static constexpr int NGA = NKX * 2 * OG;               // A row groups (kx, part, o / 8)
    static constexpr int MA = 8 * NGA;                     // rows of D that are read
    static constexpr int MB = (MA + 127) / 128;            // M = 128 blocks
    static constexpr int NGB = NKY * 2 * CG + 2;           // B row groups (ky, part, c / 8), ones, zeros
    static constexpr int N = 8 * NGB;
    static constexpr int XCOLS = (K == 3 && KXS == 3) ? TW + 2 : TW;  // g columns loaded per tile
    static constexpr int XROWS = K == 3 ? 10 : 8;          // x rows loaded per tile
    static constexpr int COLS = NKY * CINP;                // D columns per row after the part sum
    static constexpr int RS = COLS + 1;                    // epilogue row stride (floats, odd)
    static constexpr uint32_t A_BYTES = TW * NGA * 128;
    static constexpr uint32_t B_OFF = A_BYTES;
    static constexpr uint32_t B_BYTES = TW * NGB * 128;
    static constexpr uint32_t OPER = A_BYTES + B_BYTES;
    static constexpr uint32_t RED = static_cast<uint32_t>(MB * 128 * RS * 4);
    static constexpr uint32_t OFF_BAR = ((OPER > RED ? OPER : RED) + 15) / 16 * 16;
    static constexpr uint32_t BYTES_USED = OFF_BAR + 32;   // mbarrier, TMEM address slot
    static constexpr int TMEM_RAW = MB * N;
    static constexpr int TMEM_COLS = TMEM_RAW <= 32 ? 32 : TMEM_RAW <= 64 ? 64 : TMEM_RAW <= 128 ? 128
                                   : TMEM_RAW <= 256 ? 256 : 512;
    // enough shared memory per CTA that the CTAs resident on one SM never ask
    // for more than its 512 TMEM columns (at most 228 KB of shared memory per SM)
    static constexpr int TMEM_CAP = 512 / TMEM_COLS;
    static constexpr uint32_t BYTES_MIN = (236u * 1024u) / (TMEM_CAP + 1);
    static constexpr uint32_t BYTES = BYTES_USED < BYTES_MIN ? BYTES_MIN : BYTES_USED;
    static constexpr int ENTRIES = COUT * CIN * K * K + COUT;  // one slot: weights (OIHW), then biases
    static_assert(K == 1 || K == 3, "kernel size");
    static_assert(KXS == 1 || KXS == 3, "horizontal offsets per CTA");
    static_assert(CIN == 4 || CIN % 8 == 0, "C_in");
    static_assert(COUT % 8 == 0 && 2 * COUT * NKX <= 256, "C_out");
    static_assert(TW % 2 == 0, "two K columns per K = 16 step");
    static_assert(N % 16 == 0 && N <= 256, "MMA width");
    static_assert(TMEM_RAW <= 512, "tensor memory");
    // the last M block of the last K step reads (16 MB - NGA) groups past A, inside B
    static_assert((16 * MB - NGA) * 128 <= static_cast<int>(B_BYTES), "A overrun stays inside B");
    static_assert(BYTES_USED <= 227 * 1024, "shared memory per CTA");
    static_assert(NGA * 128 / 16 < (1 << 14) && NGB * 128 / 16 < (1 << 14), "LBO field");
};

__device__ __forceinline__ uint32_t bf16_bits(float v) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v)));
}

// One tile's operands in registers: thread t holds items t, t + 256, ... of
// g~ (SG items: one (column, output channel), 8 rows) and of x~ (SX items:
// one (column, input channel), XROWS rows).  Every load of a tile is issued
// before any is used, so a thread waits for one memory latency per tile, and
// the next tile's loads are in flight while the current tile's MMAs run.
template <int CIN, int COUT, int K, int KXS, int TW>
struct WgRegs {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    static constexpr int SG = (C::XCOLS * COUT + kWgThreads - 1) / kWgThreads;
    static constexpr int SX = (TW * C::CINP + kWgThreads - 1) / kWgThreads;
    float g[SG][8];
    float m[K == 1 ? SG : 1][8];  // ReLU mask of the 1x1 layers' g (raw values, applied on use)
    float x[SX][C::XROWS];
};

// g~ of tile (n, y0, x0): item i = (column xi, output o) covers image column
// x0 + xi - xoff, rows y0 .. y0 + 7; zeros outside the image.  x~: item
// i = (column q, input c) covers image column x0 + q, rows y0 + R0 .. (R0 = -1
// for a 3x3 layer); zeros outside the image and beyond C_in.
template <int CIN, int COUT, int K, int KXS, int TW>
__device__ __forceinline__ void wg_load(WgRegs<CIN, COUT, K, KXS, TW>& R, const float* __restrict__ g,
                                        const float* __restrict__ gm, const float* __restrict__ x, int n, int H, int W,
                                        int y0, int x0, int kx0) {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    using RT = WgRegs<CIN, COUT, K, KXS, TW>;
    const int xoff = K == 3 ? (KXS == 3 ? 1 : kx0 - 1) : 0;  // first loaded g column = x0 - xoff
#pragma unroll
    for (int s = 0; s < RT::SG; ++s) {
        const int i = threadIdx.x + s * kWgThreads;
        const int o = i % COUT, xi = i / COUT;
        const int X = x0 + xi - xoff;
        const bool col = i < C::XCOLS * COUT && X >= 0 && X < W;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const bool in = col && y0 + r < H;
            const size_t idx = in ? ((static_cast<size_t>(n) * H + y0 + r) * W + X) * COUT + o : 0;
            R.g[s][r] = in ? __ldg(g + idx) : 0.f;
            if constexpr (K == 1) R.m[s][r] = (in && gm != nullptr) ? __ldg(gm + idx) : 1.f;
        }
    }
    constexpr int R0 = K == 3 ? -1 : 0;
#pragma unroll
    for (int s = 0; s < RT::SX; ++s) {
        const int i = threadIdx.x + s * kWgThreads;
        const int c = i % C::CINP, q = i / C::CINP;
        const int X = x0 + q;
        const bool col = i < TW * C::CINP && c < CIN && X < W;
#pragma unroll
        for (int r = 0; r < C::XROWS; ++r) {
            const int yy = y0 + R0 + r;
            const bool in = col && yy >= 0 && yy < H;
            R.x[s][r] = in ? __ldg(x + ((static_cast<size_t>(n) * H + (in ? yy : 0)) * W + X) * CIN + c) : 0.f;
        }
    }
}

// Registers -> BF16 hi / lo chunks in shared memory.  Copy kxi of g (offset
// kx = kx0 + kxi) holds at K column q the column x0 + q - (kx - 1) (x0 + q for
// a 1x1 layer); copy ky of x holds at K column q the rows y0 + ky - 1 .. + 8
// (y0 .. y0 + 7 for a 1x1 layer).
template <int CIN, int COUT, int K, int KXS, int TW>
__device__ __forceinline__ void wg_store(const WgRegs<CIN, COUT, K, KXS, TW>& R, uint32_t sbase, const float* gm,
                                         int relu_in, int kx0) {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    using RT = WgRegs<CIN, COUT, K, KXS, TW>;
    const int xoff = K == 3 ? (KXS == 3 ? 1 : kx0 - 1) : 0;
#pragma unroll
    for (int s = 0; s < RT::SG; ++s) {
        const int i = threadIdx.x + s * kWgThreads;
        if (i >= C::XCOLS * COUT) break;
        const int o = i % COUT, xi = i / COUT;
        float v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            v[r] = R.g[s][r];
            if constexpr (K == 1)
                if (gm != nullptr && !(R.m[s][r] > 0.f)) v[r] = 0.f;
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t h0 = bf16_bits(v[2 * k]), h1 = bf16_bits(v[2 * k + 1]);
            h[k] = h0 | (h1 << 16);
            l[k] = bf16_bits(v[2 * k] - __uint_as_float(h0 << 16)) |
                   (bf16_bits(v[2 * k + 1] - __uint_as_float(h1 << 16)) << 16);
        }
        const uint4 hi = make_uint4(h[0], h[1], h[2], h[3]), lo = make_uint4(l[0], l[1], l[2], l[3]);
        const int og = o / 8, j = o % 8;
#pragma unroll
        for (int kxi = 0; kxi < C::NKX; ++kxi) {
            const int q = K == 3 ? xi - xoff + (kx0 + kxi) - 1 : xi;
            if (q >= 0 && q < TW) {
                const uint32_t a = sbase + static_cast<uint32_t>((q * C::NGA + 2 * kxi * C::OG + og) * 128 + j * 16);
                st_shared_v4(a, hi);
                st_shared_v4(a + C::OG * 128, lo);
            }
        }
    }
#pragma unroll
    for (int s = 0; s < RT::SX; ++s) {
        const int i = threadIdx.x + s * kWgThreads;
        if (i >= TW * C::CINP) break;
        const int c = i % C::CINP, q = i / C::CINP;
        uint32_t h[C::XROWS], l[C::XROWS];
#pragma unroll
        for (int r = 0; r < C::XROWS; ++r) {
            const float v = relu_in ? fmaxf(R.x[s][r], 0.f) : R.x[s][r];
            h[r] = bf16_bits(v);
            l[r] = bf16_bits(v - __uint_as_float(h[r] << 16));
        }
        const int cg = c / 8, j = c % 8;
#pragma unroll
        for (int ky = 0; ky < C::NKY; ++ky) {
            const uint4 hi = make_uint4(h[ky] | (h[ky + 1] << 16), h[ky + 2] | (h[ky + 3] << 16),
                                        h[ky + 4] | (h[ky + 5] << 16), h[ky + 6] | (h[ky + 7] << 16));
            const uint4 lo = make_uint4(l[ky] | (l[ky + 1] << 16), l[ky + 2] | (l[ky + 3] << 16),
                                        l[ky + 4] | (l[ky + 5] << 16), l[ky + 6] | (l[ky + 7] << 16));
            const uint32_t a =
                sbase + C::B_OFF + static_cast<uint32_t>((q * C::NGB + 2 * ky * C::CG + cg) * 128 + j * 16);
            st_shared_v4(a, hi);
            st_shared_v4(a + C::CG * 128, lo);
        }
    }
}

// The tile's MMAs (one thread): K step k covers K columns 2k and 2k + 1.
template <int CIN, int COUT, int K, int KXS, int TW>
__device__ __forceinline__ void wg_mma(uint32_t sbase, uint32_t tbase, uint32_t acc) {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    constexpr uint32_t idesc = idesc_bf16(kTileM, C::N);
#pragma unroll 1
    for (int k = 0; k < TW / 2; ++k) {
        const uint64_t bdesc = smem_desc(sbase + C::B_OFF + static_cast<uint32_t>(2 * k * C::NGB * 128), C::NGB * 128, 128);
#pragma unroll
        for (int mb = 0; mb < C::MB; ++mb) {
            const uint64_t adesc =
                smem_desc(sbase + static_cast<uint32_t>((2 * k * C::NGA + 16 * mb) * 128), C::NGA * 128, 128);
            mma_bf16(tbase + static_cast<uint32_t>(mb * C::N), adesc, bdesc, idesc, acc);
        }
        acc = 1;
    }
}

template <int CIN, int COUT, int K, int KXS, int TW>
__global__ void __launch_bounds__(kWgThreads) wgrad_tc_kernel(const float* __restrict__ x, int relu_in,
                                                              const float* __restrict__ g, const float* __restrict__ gm,
                                                              int NI, int H, int W, float* __restrict__ part, int* err) {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 16);
    const uint32_t sbase = smem_u32(smem);
    const int kx0 = (K == 3 && KXS == 1) ? static_cast<int>(blockIdx.y) : 0;
    // ones (group NGB - 2) and zeros (group NGB - 1) of every K column; staging never writes them
    for (int i = tid; i < TW * 16; i += kWgThreads) {
        const int q = i / 16, r = i % 16;
        const uint32_t v = r < 8 ? 0x3F803F80u : 0u;
        st_shared_v4(sbase + C::B_OFF + static_cast<uint32_t>((q * C::NGB + C::NGB - 2) * 128 + r * 16),
                     make_uint4(v, v, v, v));
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, C::TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + 7) / 8;
    const long long ntiles = static_cast<long long>(NI) * tiles_y * tiles_x;
    uint32_t phase = 0;
    int done = 0;
    bool ok = true;
    auto tile_origin = [&](long long t, int& n, int& y0, int& x0) {
        const int tx = static_cast<int>(t % tiles_x);
        const long long t2 = t / tiles_x;
        n = static_cast<int>(t2 / tiles_y);
        y0 = static_cast<int>(t2 % tiles_y) * 8;
        x0 = tx * TW;
    };
    WgRegs<CIN, COUT, K, KXS, TW> R;
    if (blockIdx.x < ntiles) {
        int n, y0, x0;
        tile_origin(blockIdx.x, n, y0, x0);
        wg_load<CIN, COUT, K, KXS, TW>(R, g, gm, x, n, H, W, y0, x0, kx0);
    }
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        wg_store<CIN, COUT, K, KXS, TW>(R, sbase, gm, relu_in, kx0);
        fence_proxy_async_smem();  // the staged operands, visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            wg_mma<CIN, COUT, K, KXS, TW>(sbase, tbase, done > 0 ? 1u : 0u);
            mma_commit(bar);
        }
        if (t + gridDim.x < ntiles) {  // the next tile's loads, in flight during the MMAs
            int n, y0, x0;
            tile_origin(t + gridDim.x, n, y0, x0);
            wg_load<CIN, COUT, K, KXS, TW>(R, g, gm, x, n, H, W, y0, x0, kx0);
        }
        ok = mbar_wait_bounded(bar, phase, kWaitNs);
        phase ^= 1u;
        if (!ok) atomicExch(err, kWgErrCode);
        ++done;
        // operands consumed before the next tile is staged
        fence_before_sync();
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
    }
    fence_after_sync();

    // accumulators -> shared memory (operands no longer needed): row m, column
    // ky C_inp + c = the two x parts summed
    float* red = reinterpret_cast<float*>(smem);
    const bool have = ok && done > 0;
    const int lq = warp & 3, half = warp >> 2;
#pragma unroll 1
    for (int mb = 0; mb < C::MB; ++mb) {
        const int m = 128 * mb + 32 * lq + lane;
        const uint32_t trow = tbase + (static_cast<uint32_t>(32 * lq) << 16) + static_cast<uint32_t>(mb * C::N);
#pragma unroll 1
        for (int it = half; it <= C::NKY * C::CG; it += kWgThreads / 128) {
            float a[8], b[8];
            if (it < C::NKY * C::CG) {
                const int ky = it / C::CG, c0 = 8 * (it % C::CG);
                tmem_ld8(trow + static_cast<uint32_t>(2 * ky * C::CINP + c0), a);
                tmem_ld8(trow + static_cast<uint32_t>((2 * ky + 1) * C::CINP + c0), b);
                tmem_ld_wait();
                if (m < C::MA)
#pragma unroll
                    for (int j = 0; j < 8; ++j) red[m * C::RS + ky * C::CINP + c0 + j] = have ? a[j] + b[j] : 0.f;
            } else {
                tmem_ld8(trow + static_cast<uint32_t>(8 * (C::NGB - 2)), a);
                tmem_ld_wait();
                if (m < C::MA) red[m * C::RS + C::COLS] = have ? a[0] : 0.f;
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    // the two g parts summed; slot blockIdx.x of the partial sums (OIHW, then biases)
    float* slot = part + static_cast<size_t>(blockIdx.x) * C::ENTRIES;
    constexpr int NE = C::NKX * COUT * CIN * C::NKY;
    for (int e = tid; e < NE; e += kWgThreads) {
        const int ky = e % C::NKY;
        int r = e / C::NKY;
        const int c = r % CIN;
        r /= CIN;
        const int o = r % COUT, kxi = r / COUT;
        const int m0 = 2 * kxi * COUT + o;
        const float v = red[m0 * C::RS + ky * C::CINP + c] + red[(m0 + COUT) * C::RS + ky * C::CINP + c];
        slot[((o * CIN + c) * K + ky) * K + (K == 3 ? kx0 + kxi : 0)] = v;
    }
    // the bias: the copy without horizontal offset (kx = 1, or the 1x1 layer's only copy)
    const int kxc = K == 3 ? 1 - kx0 : 0;
    if (kxc >= 0 && kxc < C::NKX)
        for (int o = tid; o < COUT; o += kWgThreads) {
            const int m0 = 2 * kxc * COUT + o;
            slot[COUT * CIN * K * K + o] = red[m0 * C::RS + C::COLS] + red[(m0 + COUT) * C::RS + C::COLS];
        }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, C::TMEM_COLS);
}

// dW[e] += sum over slots s of part[s][e] for e < nw, db[e - nw] += ... beyond.
// 32 entries per block (one per lane); the 32 warps take slots w, w + 32, ...
// into four accumulators (slot s to accumulator (s / 32) % 4, the tail to the
// first) and meet in shared memory in warp order: a fixed order, so the same
// sums every run.
constexpr int kRedThreads = 1024;
__global__ void __launch_bounds__(kRedThreads) wg_reduce_kernel(const float* __restrict__ part, int slots, int entries,
                                                                int nw, float* __restrict__ dW, float* __restrict__ db) {
    constexpr int NWp = kRedThreads / 32;
    __shared__ float red[NWp][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (e < entries) {
        int s = warp;
        for (; s + 3 * NWp < slots; s += 4 * NWp) {  // four loads in flight per thread
            a0 += __ldg(part + static_cast<size_t>(s) * entries + e);
            a1 += __ldg(part + static_cast<size_t>(s + NWp) * entries + e);
            a2 += __ldg(part + static_cast<size_t>(s + 2 * NWp) * entries + e);
            a3 += __ldg(part + static_cast<size_t>(s + 3 * NWp) * entries + e);
        }
        for (; s < slots; s += NWp) a0 += __ldg(part + static_cast<size_t>(s) * entries + e);
    }
    red[warp][lane] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (warp == 0 && e < entries) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < NWp; ++w) v += red[w][lane];
        if (e < nw) dW[e] += v;
        else if (db != nullptr) db[e - nw] += v;
    }
}

template <int CIN, int COUT, int K, int KXS, int TW>
cudaError_t launch_wgrad(const float* x, int relu_in, const float* g, const float* gm, int NI, int H, int W,
                         float* part, float* dW, float* db, int* err, cudaStream_t st) {
    using C = WgCfg<CIN, COUT, K, KXS, TW>;
    static int per_sm = 0;  // CTAs resident per SM (per instantiation, set on first use)
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<CIN, COUT, K, KXS, TW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(C::BYTES));
        if (e != cudaSuccess) return e;
        // all of the unified L1 / shared storage as shared memory: several CTAs per SM
        e = cudaFuncSetAttribute(wgrad_tc_kernel<CIN, COUT, K, KXS, TW>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        const int occ = resident_ctas_per_sm(reinterpret_cast<const void*>(wgrad_tc_kernel<CIN, COUT, K, KXS, TW>),
                                             kWgThreads, C::BYTES);
        per_sm = occ < C::TMEM_CAP ? occ : C::TMEM_CAP;
    }
    const long long tiles = static_cast<long long>(NI) * ((H + 7) / 8) * ((W + TW - 1) / TW);
    if (tiles == 0) return cudaSuccess;
    const int gy = (K == 3 && KXS == 1) ? 3 : 1;
    long long cap = static_cast<long long>(num_sms()) * per_sm / gy;
    const long long slots_fit = kWgPartFloats / C::ENTRIES;
    if (cap > slots_fit) cap = slots_fit;
    if (cap < 1) cap = 1;
    const int gx = static_cast<int>(tiles < cap ? tiles : cap);
    wgrad_tc_kernel<CIN, COUT, K, KXS, TW><<<dim3(gx, gy), kWgThreads, C::BYTES, st>>>(x, relu_in, g, gm, NI, H, W,
                                                                                        part, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wg_reduce_kernel<<<(C::ENTRIES + 31) / 32, kRedThreads, 0, st>>>(part, gx, C::ENTRIES, COUT * CIN * K * K, dW, db);
    return cudaGetLastError();
}

}  // namespace

cudaError_t wgrad_tc(int cin, int cout, int k, const float* x, int relu_in, const float* g, const float* gm, int N,
                     int H, int W, float* part, float* dW, float* db, int* err, cudaStream_t st) {
#define NSM_WG(a, b, kk, kxs, tw) \
    if (cin == a && cout == b && k == kk) return launch_wgrad<a, b, kk, kxs, tw>(x, relu_in, g, gm, N, H, W, part, dW, db, err, st);
    // 3x3 layers: (C_in, C_out, 3, horizontal offsets per CTA, tile columns)
    NSM_WG(4, 16, 3, 3, 32) NSM_WG(16, 32, 3, 3, 16) NSM_WG(32, 64, 3, 1, 16) NSM_WG(32, 32, 3, 1, 16)
    NSM_WG(16, 16, 3, 3, 32)
    // 1x1 layers
    NSM_WG(16, 16, 1, 1, 32) NSM_WG(32, 16, 1, 1, 32) NSM_WG(64, 32, 1, 1, 32) NSM_WG(32, 32, 1, 1, 32)
#undef NSM_WG
    return cudaErrorInvalidValue;
}

cudaError_t slot_reduce(const float* part, int slots, int entries, int nw, float* dW, float* db, cudaStream_t st) {
    if (slots < 1 || entries < 1) return cudaSuccess;
    wg_reduce_kernel<<<(entries + 31) / 32, kRedThreads, 0, st>>>(part, slots, entries, nw, dW, db);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ 1x1 weight gradients
// dW[o][c] += sum_p g~[p][o] x~[p][c], db[o] += sum_p g~[p][o] of a 1x1 layer.
// Two reads per pixel and 16 to 64 channels each: bound by HBM, not a dense
// contraction, so FP32 on CUDA cores.  CTA b takes the contiguous tiles
// [T b / G, T (b + 1) / G) of 256 pixels (T tiles, G CTAs); each tile's x~
// (rectified) and g~ (masked) rows arrive with coalesced float4 loads in a
// shared tile.  Thread t keeps the 4 x 4 block (o-block, c-block) = t % NB of
// dW (NB = C_out C_in / 16 blocks) over pixels t / NB, t / NB + NG, ... (NG =
// 256 / NB pixel groups) of every tile, plus the bias for c-block 0; the
// groups meet in shared memory in group order and the CTA's sums go to its
// slot, which slot_reduce adds in slot order: a fixed order throughout.
constexpr int kW1P = 256;  // pixels per tile = threads per CTA

template <int CIN, int COUT>
struct W1Shape {
    static constexpr int CI4 = CIN / 4, CO4 = COUT / 4, NB = CI4 * CO4, NG = kW1P / NB;
    static constexpr int SX = CIN + 4, SG = COUT + 4;  // padded rows (conflict-free float4 reads)
    static constexpr int ENTRIES = COUT * CIN + COUT;
    static constexpr size_t SMEM = sizeof(float) * static_cast<size_t>(kW1P) * (SX + SG);
    static_assert(CIN % 4 == 0 && COUT % 4 == 0 && kW1P % NB == 0 && NG >= 1, "1x1 weight-gradient shape");
    static_assert(NG * NB * 20 <= kW1P * (SX + SG), "group sums fit the tile storage");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kW1P) wgrad1x1_tile_kernel(const float* __restrict__ x, int relu_in,
                                                             const float* __restrict__ g, const float* __restrict__ gm,
                                                             size_t npx, float* __restrict__ part) {
    using S = W1Shape<CIN, COUT>;
    extern __shared__ float4 w1smem[];
    float* xs = reinterpret_cast<float*>(w1smem);  // [kW1P][SX]
    float* gs = xs + kW1P * S::SX;                  // [kW1P][SG]
    const int t = threadIdx.x, blk = t % S::NB, pg = t / S::NB;
    const int ob = blk / S::CI4, cb = blk % S::CI4;
    float acc[4][4] = {};
    float bacc[4] = {0.f, 0.f, 0.f, 0.f};
    const long long tiles = static_cast<long long>((npx + kW1P - 1) / kW1P);
    const long long t0 = tiles * blockIdx.x / gridDim.x, t1 = tiles * (blockIdx.x + 1) / gridDim.x;
    for (long long tile = t0; tile < t1; ++tile) {
        const size_t p0 = static_cast<size_t>(tile) * kW1P;
        const int np = static_cast<int>(npx - p0 < static_cast<size_t>(kW1P) ? npx - p0 : kW1P);
        const float4* x4 = reinterpret_cast<const float4*>(x + p0 * CIN);
        const float4* g4 = reinterpret_cast<const float4*>(g + p0 * COUT);
        const float4* m4 = gm ? reinterpret_cast<const float4*>(gm + p0 * COUT) : nullptr;
        // rows past the last pixel are zero, so the products need no bound
#pragma unroll
        for (int k = 0; k < S::CI4; ++k) {
            const int i = t + kW1P * k;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < np * S::CI4) {
                v = __ldg(x4 + i);
                if (relu_in) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
            }
            *reinterpret_cast<float4*>(xs + (i / S::CI4) * S::SX + 4 * (i % S::CI4)) = v;
        }
#pragma unroll
        for (int k = 0; k < S::CO4; ++k) {
            const int i = t + kW1P * k;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < np * S::CO4) {
                v = __ldg(g4 + i);
                if (m4) {
                    const float4 m = __ldg(m4 + i);
                    v = make_float4(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f, m.z > 0.f ? v.z : 0.f,
                                    m.w > 0.f ? v.w : 0.f);
                }
            }
            *reinterpret_cast<float4*>(gs + (i / S::CO4) * S::SG + 4 * (i % S::CO4)) = v;
        }
        __syncthreads();
        for (int p = pg; p < np; p += S::NG) {
            const float4 xv = *reinterpret_cast<const float4*>(xs + p * S::SX + 4 * cb);
            const float4 gv = *reinterpret_cast<const float4*>(gs + p * S::SG + 4 * ob);
            const float gq[4] = {gv.x, gv.y, gv.z, gv.w}, xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(gq[i], xq[j], acc[i][j]);
                bacc[i] += gq[i];
            }
        }
        __syncthreads();  // the tile's rows are free for the next tile
    }
    // group sums, in group order, into the CTA's slot
    float* red = xs;  // [NG][NB][20]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(pg * S::NB + blk) * 20 + 4 * i + j] = acc[i][j];
        red[(pg * S::NB + blk) * 20 + 16 + i] = bacc[i];
    }
    __syncthreads();
    float* slot = part + static_cast<size_t>(blockIdx.x) * S::ENTRIES;
    for (int e = t; e < S::NB * 20; e += kW1P) {
        const int b2 = e / 20, k = e % 20;
        float v = 0.f;
        for (int q = 0; q < S::NG; ++q) v += red[(q * S::NB + b2) * 20 + k];
        const int o0 = 4 * (b2 / S::CI4), c0 = 4 * (b2 % S::CI4);
        if (k < 16) slot[(o0 + k / 4) * CIN + c0 + k % 4] = v;
        else if (c0 == 0) slot[COUT * CIN + o0 + (k - 16)] = v;
    }
}

template <int CIN, int COUT>
static cudaError_t launch_wgrad1x1(const float* x, int relu_in, const float* g, const float* gm, size_t npx,
                                   float* part, float* dW, float* db, cudaStream_t st) {
    using S = W1Shape<CIN, COUT>;
    auto kern = wgrad1x1_tile_kernel<CIN, COUT>;
    static int per_sm = 0;  // resident CTAs per SM, from the tile storage
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(S::SMEM));
        if (e != cudaSuccess) return e;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kW1P, S::SMEM) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    const long long tiles = static_cast<long long>((npx + kW1P - 1) / kW1P);
    long long grid = static_cast<long long>(num_sms()) * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid * S::ENTRIES > kWgPartFloats) grid = kWgPartFloats / S::ENTRIES;
    kern<<<static_cast<unsigned>(grid), kW1P, S::SMEM, st>>>(x, relu_in, g, gm, npx, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return slot_reduce(part, static_cast<int>(grid), S::ENTRIES, COUT * CIN, dW, db, st);
}

cudaError_t wgrad1x1_tiles(int cin, int cout, const float* x, int relu_in, const float* g, const float* gm, int N,
                           int H, int W, float* part, float* dW, float* db, cudaStream_t st) {
    const size_t npx = static_cast<size_t>(N) * H * W;
    if (npx == 0) return cudaSuccess;
#define NSM_W1(a, b) \
    if (cin == a && cout == b) return launch_wgrad1x1<a, b>(x, relu_in, g, gm, npx, part, dW, db, st);
    NSM_W1(16, 16) NSM_W1(32, 16) NSM_W1(32, 32) NSM_W1(64, 32)
#undef NSM_W1
    return cudaErrorInvalidValue;
}


}  // namespace tr
}  // namespace nsm
