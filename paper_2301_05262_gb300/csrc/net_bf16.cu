// BF16 tensor-core form of the compact encoder/decoder (Sec. 3.5) on
// Blackwell tcgen05: every convolution is an implicit GEMM
//   D[pixels x C_out] = A[pixels x K] * B[C_out x K]^T,  K = 9 C_in (3x3) or C_mid (1x1),
// issued as 128 x N x 16 MMAs by one thread, accumulated in FP32 in tensor
// memory (TMEM).  One fused kernel per level ("stage") runs
// "3x3 conv + ReLU -> 1x1 conv + ReLU" with one of these prologues / epilogues:
//   prologue  GATHER (features from G-buffer + shadow map: the gather fused
//             into the first level), PLAIN, UP_SKIP, UP;
//   epilogue  POOL, SKIP_POOL, STORE, HEAD (1x1 16 -> 1 + sigmoid).
//
// Each launch is persistent and serves a job table of up to kMaxViews views
// of any sizes (one view for nsm_infer, many for nsm_infer_batched): the
// CTAs walk one global list of tiles, each tile belonging to one view.
//
// Compensated BF16: every value the tensor cores read is a pair of BF16
// numbers, v = hi + lo with hi = bf16(v), lo = bf16(v - hi) (about 16
// significant bits): the weights (hi and lo stacked along N, so one MMA
// yields x W_hi and x W_lo side by side in TMEM, summed in the epilogue), the
// features, the 3x3 -> 1x1 intermediate and every activation stored between
// stages ([pixel][part][C] in global memory, 4 bytes per channel like FP32).
// The products are BF16 x BF16 with FP32 accumulation; what rounding remains
// is ~2^-16 relative per stored value instead of BF16's 2^-9, which a deep
// chain of unnormalised convolutions otherwise amplifies well past 1e-2 in
// the visibility.
//
// Tile: R rows x 128 pixels of the level; MMA row block = one 128-pixel row
// segment.  The input tile with its 1-pixel halo is staged in shared memory
// as 16-byte chunks of 8 channels, [plane][staged row][staged pixel], which
// is the tensor core's no-swizzle K-major operand layout: the A operand of
// tap (ky, kx) and a channel pair is the same buffer started (ky, kx) chunks
// further on, so the im2col matrix is never built.  A plane is one channel
// group of one part (hi or lo); both parts are multiplied by the same weight
// chunk.  Large inputs are staged in K slices (KS > 1: an input buffer holds
// the hi and lo planes of 8 C_in / KS channels), each slice one pipeline
// step.  Row-stacked 3x3 (when 3 x 2 C_mid <= 256): the kernel rows ky are
// stacked along N too, so one MMA over staged input row j accumulates into
// output rows j, j-1, j-2 (accumulators in descending column order, cleared
// by one MMA with a zero A operand).  The 3x3 result goes TMEM -> registers
// (bias, ReLU) -> shared memory as hi + lo parts, the A operand of the 1x1
// MMAs (written into the same TMEM columns).
//
// First level: the four FP32 features are split into hi + lo parts, 8
// "channels" per pixel; K steps pair two taps (two 16-byte chunks).
//
// Warp-specialised pipeline (NEW epilogue warps, NPW producer warps, one MMA
// warp; the autotuner picks the split):
//   producers  PLAIN copies step i (a tile's K slice) straight into input
//              buffer i % 2 with cp.async; GATHER / UP* prefetch tile t + 1's
//              raw inputs (G-buffer, or the coarser level) into raw buffer
//              (t + 1) % 2 with cp.async while they compute tile t from raw
//              buffer t % 2 (texel lookups, features / bilinear x2 + skip)
//   MMA warp   one thread issues the 3x3 of tile t, slice by slice, into
//              accumulator buffer t % 2, then its 1x1 into the same columns;
//              it also owns the TMEM allocation
//   epilogue   TMEM lane quarter = warp % 4, tile rows r = warp / 4 (mod
//              NEW / 4); 3x3 result -> 1x1 operand, 1x1 result -> outputs
// mbarriers (every wait is bounded and gives up when another role aborted):
//   gfull[b]  producers' cp.async -> producers: raw buffer b landed
//   rfree[b]  producers -> producers: raw buffer b consumed
//   full[b]   producers -> MMA: input buffer b staged
//   mma3[b]   MMA -> producers: input buffer b consumed
//   accf[t]   MMA -> epilogue: 3x3 accumulators of buffer t complete
//   a1full    epilogue -> MMA: 1x1 operand written
//   mma1      MMA -> epilogue: 1x1 done (and its operand free)
//   tfree[t]  epilogue -> MMA: accumulator buffer t read out
#include <cudaTypedefs.h>

#include "nsm_internal.h"
#include "tc_common.cuh"
#include "tc_stage.h"
#include "tc_pipeline.cuh"

namespace nsm {

using namespace tc;

// Warp roles of a CTA (NEW epilogue warps, NPW producer warps, one MMA warp):
// warps [0, NEW) epilogue (warp w reads TMEM lane quarter w % 4 and the tile
// rows r = w / 4 (mod NEW / 4)), [NEW, NEW + NPW) producers, NEW + NPW MMA.
// PAR: the level-0 decoder on the coarse grid (C_mid = 4 output parities x
// C_out channels of the 3x3; the 1x1 applies per parity, so its weight image
// is the plain C_out -> C_out one).
template <int CIN, int CMID, int COUT, int R, int PRO, int KS, bool PAR = false>
struct TcCfg {
    static constexpr bool SPLIT = (PRO == TPRO_GATHER);
    static constexpr bool UP = (PRO == TPRO_UP || PRO == TPRO_UP_SKIP);
    static constexpr int CG_IN = SPLIT ? 1 : CIN / 8;           // channel groups of each part of the input
    // K slices: an input buffer holds the hi and lo planes of CGS channel
    // groups, [part][group of the slice] (the first level: one plane)
    static constexpr int CGS = SPLIT ? 1 : CG_IN / KS;
    static constexpr int PLN = SPLIT ? 1 : 2 * CGS;
    static constexpr int KSTEPS3 = SPLIT ? 5 : 9 * (CIN / 16);
    static constexpr int A0_CHUNKS = PLN * (R + 2) * kSW;        // one input buffer
    // Staged rows form rings, so a tile that continues the previous one down
    // its column reuses the two overlapping rows and stages only R new ones.
    // KS == 1: the two input buffers form one ring of 2 (R + 2) rows per plane
    // (the next tile's rows are staged while the MMAs read the current ones);
    // KS > 1: each input buffer holds one K slice as its own ring of R + 2
    // rows, refilled once the MMAs of the same slice of the previous tile are
    // done (the new rows take the slots of that tile's rows 0 .. R - 1)
    static constexpr bool RING = true;
    static constexpr bool ONE_RING = (KS == 1);
    static constexpr int NRW = ONE_RING ? 2 * (R + 2) : R + 2;  // staged rows per plane
    static constexpr uint32_t PLANE = NRW * kSW * 16;            // bytes per plane
    // 3x3 -> 1x1 intermediate as BF16 hi + lo parts: [row][part][channel group][pixel]
    static constexpr int A1_CHUNKS = R * 2 * (CMID / 8) * kTileM;
    // raw prefetch buffer (two): the staged G-buffer (pos, nrm) or the coarse rows (hi + lo)
    static constexpr int NCR = R / 2 + 2;
    static constexpr int RAW_BYTES = SPLIT ? (R + 2) * 130 * 32 : (UP ? NCR * kNCC * (CIN / 4 + 1) * 16 : 0);
    // weights as BF16 hi + lo parts stacked along the output rows (2 C rows per K block)
    static constexpr int N3 = 2 * CMID, N1 = 2 * COUT;             // MMA widths
    // row-stacked 3x3: the kernel rows ky = 0, 1, 2 stacked along N as well, so
    // one MMA over staged input row j accumulates into output rows j, j-1, j-2
    static constexpr bool STACK = 3 * N3 <= 256;
    static constexpr int B3_CHUNKS = STACK ? (SPLIT ? 12 * N3 : 9 * CG_IN * N3) : KSTEPS3 * 2 * N3;
    static constexpr int B1_CHUNKS = (PAR ? COUT / 8 : CMID / 8) * N1;
    static constexpr int OFF_A0 = 0;                                // two input buffers
    static constexpr int OFF_A1 = OFF_A0 + 2 * A0_CHUNKS * 16;
    static constexpr int OFF_RAW = OFF_A1 + A1_CHUNKS * 16;         // two raw buffers
    static constexpr int OFF_B3 = OFF_RAW + 2 * RAW_BYTES;
    static constexpr int OFF_B1 = OFF_B3 + B3_CHUNKS * 16;
    static constexpr int OFF_BIAS3 = OFF_B1 + B1_CHUNKS * 16;
    static constexpr int OFF_BIAS1 = OFF_BIAS3 + CMID * 4;
    static constexpr int OFF_HEAD = OFF_BIAS1 + COUT * 4;
    // PAR: FP32 3x3 [tap][c][o] and 1x1 [c][o] weights for the exact border ring
    static constexpr int OFF_RINGW = OFF_HEAD + 4 * (COUT + 1) * 4;
    static constexpr int RINGW_BYTES = PAR ? (9 * COUT * COUT + COUT * COUT + 8 * 2 * 9 * COUT) * 4 : 0;
    static constexpr int OFF_ZERO = ((OFF_RINGW + RINGW_BYTES) + 127) / 128 * 128;  // zero A operand
    static constexpr int ZERO_BYTES = STACK ? kTileM * 16 + 128 : 0;
    static constexpr int OFF_BAR = OFF_ZERO + ZERO_BYTES;
    static constexpr int BYTES_USED = OFF_BAR + 144;
    static constexpr int TMEM_BUF = R * N3;                         // columns of one accumulator buffer
    static constexpr int TMEM_COLS_RAW = 2 * TMEM_BUF;
    static constexpr int TMEM_COLS = TMEM_COLS_RAW < 32 ? 32 : TMEM_COLS_RAW;
    // enough shared memory per CTA that the CTAs resident on one SM can never
    // ask for more than its 512 TMEM columns (228 KB of shared memory per SM)
    static constexpr int TMEM_CAP = 512 / TMEM_COLS;
    static constexpr int BYTES_MIN = (236 * 1024) / (TMEM_CAP + 1);
    static constexpr int BYTES = BYTES_USED < BYTES_MIN ? BYTES_MIN : BYTES_USED;
    static_assert(TMEM_COLS == 32 || TMEM_COLS == 64 || TMEM_COLS == 128 || TMEM_COLS == 256 || TMEM_COLS == 512,
                  "TMEM columns");
    static_assert(CMID % 16 == 0 && COUT % 16 == 0 && COUT <= CMID, "channel shapes");
    static_assert(!PAR || (CMID == 4 * COUT && PRO == TPRO_PLAIN && KS == 1 && !STACK), "coarse-grid decoder shape");
    static_assert(!UP || (R % 2 == 0), "up-sampling stages need an even tile height");
    static_assert(!STACK || R * N3 <= 256, "row-stacked accumulators are cleared by one MMA");
    static_assert(SPLIT ? KS == 1 : (CG_IN % KS == 0 && CGS % 2 == 0), "a K slice holds whole 16-channel K steps");
    static_assert(BYTES_USED <= 227 * 1024, "shared memory");
};

// ------------------------------------------------------------------ producer pieces
// (pt = producer thread 0..NP-1 of NP; staged rows y0-1 .. y0+R, pixels x0-1 .. x0+128;
// staged row sr of a tile lives in row slot (base + sr) mod NRW of every plane,
// and a producer call writes the staged rows [first, R + 2))
// Activations in global memory: [pixel][part][C] BF16, part 0 = hi, 1 = lo, so
// chunk part * CG + g of a pixel holds channels 8g .. 8g+7 of that part.

// PLAIN: K slice s of an NHWC tile straight into the input buffer, zeros
// outside the image, or (CLAMP) the nearest pixel of the image: the
// edge-replicated input of the coarse-grid level-0 decoder (planes [part][group
// of the slice])
template <int NP, int CIN, int R, int KS, int NRW, bool CLAMP = false>
__device__ __forceinline__ void copy_slice(const uint16_t* src, int H, int W, int y0, int x0, uint32_t a0, int s,
                                           int base, int first, int pt) {
    constexpr int CG = CIN / 8, CGS = CG / KS, PLN = 2 * CGS;
    constexpr uint32_t kPlane = NRW * kSW * 16;
    // each thread owns (pixel column, plane) items and walks the staged rows
    for (int ci = pt; ci < 130 * PLN; ci += NP) {
        const int pl = ci % PLN, sp = ci / PLN;
        const int chunk = (pl / CGS) * CG + s * CGS + pl % CGS;
        int gx = x0 - 1 + sp;
        const bool okx = gx >= 0 && gx < W;
        if (CLAMP) gx = gx < 0 ? 0 : (gx > W - 1 ? W - 1 : gx);
        const uint32_t dst = a0 + pl * kPlane + 16 * sp;
#pragma unroll 2
        for (int sr = first; sr < R + 2; ++sr) {
            int gy = y0 - 1 + sr;
            const bool ok = CLAMP || (okx && gy >= 0 && gy < H);
            if (CLAMP) gy = gy < 0 ? 0 : (gy > H - 1 ? H - 1 : gy);
            const uint16_t* p = ok ? src + ((static_cast<size_t>(gy) * W + gx) * 2 * CG + chunk) * 8 : src;
            cp_async16(dst + 16 * (row_slot<NRW>(base, sr) * kSW), p, ok ? 16u : 0u);
        }
    }
}

// TMA: K slice s of an NHWC tile by tensor copies, one per (plane, staged row):
// a box of kSW pixels starting at the halo column lands in the row's ring slot
// (rows 2176 bytes apart, so every destination is 128-byte aligned); the tensor
// map fills zeros outside the image.  One thread; `bar` receives the bytes.
template <int CIN, int R, int KS, int NRW>
__device__ __forceinline__ void tma_slice(const CUtensorMap* map, int y0, int x0, uint32_t a0, int s, int base,
                                          int first, uint64_t* bar) {
    constexpr int CG = CIN / 8, CGS = CG / KS, PLN = 2 * CGS;
    constexpr uint32_t kPlane = NRW * kSW * 16;
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(PLN * (R + 2 - first) * kSW * 16));
#pragma unroll
    for (int pl = 0; pl < PLN; ++pl) {
        const int chunk = (pl / CGS) * CG + s * CGS + pl % CGS;
        for (int sr = first; sr < R + 2; ++sr)
            tma_load_4d(a0 + pl * kPlane + 16 * (row_slot<NRW>(base, sr) * kSW), map, 0, chunk, x0 - 1, y0 - 1 + sr,
                        bar);
    }
}

// GATHER raw: pos4 / nrm4 of the staged pixels in bounds, [part][staged row][pixel]
template <int NP, int R>
__device__ __forceinline__ void prefetch_gbuffer(const TcJob& job, int y0, int x0, uint32_t raw, int first, int pt) {
    const int H = job.H, W = job.W;
    for (int idx = pt; idx < (R + 2 - first) * 130 * 2; idx += NP) {
        const int part = idx & 1, q = idx >> 1;
        const int sr = first + q / 130, sp = q % 130;
        const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            cp_async16(raw + 16 * (part * (R + 2) * 130 + sr * 130 + sp),
                       (part ? job.g.nrm4 : job.g.pos4) + static_cast<size_t>(gy) * W + gx, 16);
    }
}

// UP raw: the coarse rows y0/2-1 .. y0/2+R/2 and columns x0/2-1 .. x0/2+64 in
// bounds, FP32, CIN / 4 chunks of each coarse pixel, pixels CIN / 4 + 1 chunks
// apart (the pad chunk spreads neighbouring pixels over the banks)
template <int NP, int CIN, int R>
__device__ __forceinline__ void prefetch_coarse(const TcJob& job, int y0, int x0, uint32_t raw, int pt) {
    constexpr int C2 = CIN / 4, NCR = R / 2 + 2;
    const int Hl = job.H / 2, Wl = job.W / 2;
    const int cy0 = y0 / 2 - 1, cx0 = x0 / 2 - 1;
    for (int idx = pt; idx < NCR * kNCC * C2; idx += NP) {
        const int ch = idx % C2, q = idx / C2;
        const int gy = cy0 + q / kNCC, gx = cx0 + q % kNCC;
        if (gy >= 0 && gy < Hl && gx >= 0 && gx < Wl)
            cp_async16(raw + 16 * (q * (C2 + 1) + ch), job.in_f + (static_cast<size_t>(gy) * Wl + gx) * CIN + 4 * ch, 16);
    }
}

// GATHER compute: features of the staged pixels from the raw G-buffer, the
// shadow-map texel fetched per pixel (all of a thread's fetches in flight
// together), BF16 hi + lo chunks into the input buffer
template <int NP, int R, int NRW>
__device__ __forceinline__ void compute_gather(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0, int base,
                                               int first, int pt) {
    constexpr int NSP = 131;  // staged pixel 130 is the zero pad read by the dummy tap
    constexpr int NPT = ((R + 2) * NSP + NP - 1) / NP;
    const int ITEMS = (R + 2 - first) * NSP;
    const GatherParams g = job.g;  // one copy per tile: the view index is only known at run time
    const int H = job.H, W = job.W;
    float4 P[NPT], Nv[NPT];
    float z[NPT];
    bool ok[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = pt + NP * k;
        const int sr = first + idx / NSP, sp = idx % NSP;
        const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
        ok[k] = idx < ITEMS && sp < 130 && gy >= 0 && gy < H && gx >= 0 && gx < W;
        z[k] = g.z_far;
        if (ok[k]) {
            const uint32_t q = static_cast<uint32_t>(sr * 130 + sp);
            P[k] = ld_shared_f4(raw + 16 * q);
            Nv[k] = ld_shared_f4(raw + 16 * ((R + 2) * 130 + q));
            const int tx = texel_index(g, P[k].x, P[k].y, P[k].z);
            if (tx >= 0) z[k] = __ldg(g.sm + tx);
        }
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = pt + NP * k;
        if (idx < ITEMS) {
            const int sr = first + idx / NSP, sp = idx % NSP;
            uint4 chunk = make_uint4(0, 0, 0, 0);
            if (ok[k]) {
                float f[4];
                pixel_features(g, P[k], Nv[k], z[k], f);
                if (g.feat_eps)
                    f[g.eps_ch] += g.eps_scale * __ldg(g.feat_eps + static_cast<size_t>(y0 - 1 + sr) * W + (x0 - 1 + sp));
                float hl[8];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float hf = __bfloat162float(__float2bfloat16_rn(f[c]));
                    hl[c] = hf;
                    hl[4 + c] = f[c] - hf;
                }
                chunk = f32_to_chunk(hl);
            }
            st_shared_v4(a0 + 16 * (row_slot<NRW>(base, sr) * kSW + sp), chunk);
        }
    }
}

// BF16 hi + lo chunks of 8 FP32 values: hi = bf16(v), lo = bf16(v - hi) (v - hi
// is exact in FP32).  One packed rounding per pair of values and part; the hi
// values are read back from the packed bits.
__device__ __forceinline__ void split_chunks(const float* f, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = pack_bf16x2(f[2 * k], f[2 * k + 1]);
        l[k] = pack_bf16x2(f[2 * k] - __uint_as_float(h[k] << 16), f[2 * k + 1] - __uint_as_float(h[k] & 0xffff0000u));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
// FP32 value of a hi + lo chunk pair
__device__ __forceinline__ void pair_to_f32(uint4 hi, uint4 lo, float (&f)[8]) {
    float l[8];
    chunk_to_f32(hi, f);
    chunk_to_f32(lo, l);
#pragma unroll
    for (int c = 0; c < 8; ++c) f[c] += l[c];
}

// UP / UP_SKIP compute: bilinear x2 of the raw FP32 coarse rows (+ the FP32
// skip, read from global memory) -> BF16 hi + lo planes of the input buffer.  Separable:
// a coarse row is interpolated horizontally once and kept while the staged
// rows that need it are produced (two coarse rows live at a time).
// Column sp, channel group cgl of K slice s, staged rows [sr0, sr0 + NROWS).
template <int CIN, int R, int KS, bool SKIP, int NROWS, int NRW>
__device__ __forceinline__ void up_column(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0, int s, int sp,
                                          int cgl, int sr0, int base) {
    constexpr int CG = CIN / 8, CGS = CG / KS, C4 = CIN / 4;
    constexpr uint32_t kPlane = NRW * kSW * 16;
    const int H = job.H, W = job.W, Hl = H / 2, Wl = W / 2;
    const int cy0 = y0 / 2 - 1, cx0 = x0 / 2 - 1;
    const int cg = s * CGS + cgl;
    const int gx = x0 - 1 + sp;
    const bool okx = gx >= 0 && gx < W;
    const BilinTap tx = bilin_tap(okx ? gx : 0, Wl);
    const uint32_t c0 = raw + 16 * ((tx.i0 - cx0) * (C4 + 1) + 2 * cg);  // coarse column i0, row cy0
    const uint32_t c1 = raw + 16 * ((tx.i1 - cx0) * (C4 + 1) + 2 * cg);
    const uint32_t dst = a0 + cgl * kPlane + 16 * sp;          // hi plane; lo plane CGS planes on
    // the skip chunks of all rows first (global loads in flight together)
    float4 ska[NROWS], skb[NROWS];
    if constexpr (SKIP) {
#pragma unroll
        for (int k = 0; k < NROWS; ++k) {
            const int gy = y0 - 1 + sr0 + k;
            ska[k] = skb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (okx && gy >= 0 && gy < H) {
                const float4* p = reinterpret_cast<const float4*>(job.skip + (static_cast<size_t>(gy) * W + gx) * CIN) +
                                  2 * cg;
                ska[k] = __ldg(p);
                skb[k] = __ldg(p + 1);
            }
        }
    }
    // horizontal interpolation of coarse row ci
    auto hrow = [&](int ci, float (&h)[8]) {
        const uint32_t ro = 16 * ((ci - cy0) * kNCC * (C4 + 1));
        const float4 a0 = ld_shared_f4(c0 + ro), a1 = ld_shared_f4(c0 + ro + 16);
        const float4 b0 = ld_shared_f4(c1 + ro), b1 = ld_shared_f4(c1 + ro + 16);
        const float p0[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float p1[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) h[c] = p0[c] * tx.w0 + p1[c] * tx.w1;
    };
    // All coarse rows the item's staged rows need, interpolated horizontally up
    // front (their shared-memory loads in flight together).  Fine row gy takes
    // coarse rows i0 = gy odd ? (gy - 1) / 2 : gy / 2 - 1 and i0 + 1, weights
    // (3/4, 1/4) for odd gy and (1/4, 3/4) for even gy, both indices clamped to
    // the level (bilin_tap); items of several rows start on an odd row (tile
    // origins are even), so row k uses rows k / 2 and k / 2 + 1 of the preload,
    // single-row items rows 0 and 1.  Rows are loaded through the same clamp.
    const int gy0 = y0 - 1 + sr0;
    const int cu = (gy0 & 1) ? (gy0 - 1) / 2 : gy0 / 2 - 1;
    constexpr int NCRI = (NROWS + 1) / 2 + 1;
    // (only for a column inside the view: outside it c0 / c1 are not raw-buffer
    // addresses, and the staged values are zeros)
    float hv[NCRI][8];
#pragma unroll
    for (int j = 0; j < NCRI; ++j) {
        const int ci = cu + j < 0 ? 0 : (cu + j > Hl - 1 ? Hl - 1 : cu + j);
        if (okx) {
            hrow(ci, hv[j]);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) hv[j][c] = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < NROWS; ++k) {
        const int sr = sr0 + k;
        const int gy = y0 - 1 + sr;
        uint4 vh = make_uint4(0, 0, 0, 0), vl = vh;
        if (okx && gy >= 0 && gy < H) {
            const int j0 = NROWS == 1 ? 0 : k / 2;
            const float w0 = (gy & 1) ? 0.75f : 0.25f, w1 = (gy & 1) ? 0.25f : 0.75f;
            float o[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) o[c] = hv[j0][c] * w0 + hv[j0 + 1][c] * w1;
            if constexpr (SKIP) {
                const float sk[8] = {ska[k].x, ska[k].y, ska[k].z, ska[k].w, skb[k].x, skb[k].y, skb[k].z, skb[k].w};
#pragma unroll
                for (int c = 0; c < 8; ++c) o[c] += sk[c];
            }
            split_chunks(o, vh, vl);
        }
        const uint32_t ro = 16 * (row_slot<NRW>(base, sr) * kSW);
        st_shared_v4(dst + ro, vh);
        st_shared_v4(dst + CGS * kPlane + ro, vl);
    }
}

// K slice s: the 128 interior columns x channel groups walk all staged rows
// (one item per producer thread per pass); the two halo columns are split
// into single rows.
template <int NP, int CIN, int R, int KS, bool SKIP, int NRW>
__device__ __forceinline__ void compute_up(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0, int s,
                                           int base, int first, int pt) {
    constexpr int CGS = CIN / 8 / KS;
    constexpr int MAIN = kTileM * CGS;
    const int nrows = R + 2 - first;
    // channel-group-major items: a warp writes 32 consecutive chunks of one plane
    for (int i = pt; i < MAIN; i += NP) {
        if (first == 0)
            up_column<CIN, R, KS, SKIP, R + 2, NRW>(job, y0, x0, raw, a0, s, 1 + i % kTileM, i / kTileM, 0, base);
        else
            up_column<CIN, R, KS, SKIP, R, NRW>(job, y0, x0, raw, a0, s, 1 + i % kTileM, i / kTileM, 2, base);
    }
    // halo items go to the threads without an interior item when there are
    // enough of them (their loads then overlap the interior items' instead of
    // following them on the same threads)
    const int nhalo = 2 * CGS * nrows;
    const int hp = NP - MAIN >= nhalo ? pt - MAIN : pt;
    for (int i = hp; i >= 0 && i < nhalo; i += NP) {
        const int sr = first + i % nrows, q = i / nrows;
        up_column<CIN, R, KS, SKIP, 1, NRW>(job, y0, x0, raw, a0, s, (q / CGS) ? 129 : 0, q % CGS, sr, base);
    }
}

// Coalesced FP32 row output of the epilogue: each lane (pixel) puts its C values
// into a per-warp shared-memory staging area ([pixel][16-byte chunk], chunks
// XOR-swizzled by the pixel so a warp's writes and reads spread over the
// banks), then the warp writes its 32 pixels' contiguous 32 * C * 4 bytes with
// 16-byte stores (512 contiguous bytes per instruction).
template <int C>
__device__ __forceinline__ void stage_put(uint32_t stg, int lane, int c0, const float* v16) {
    constexpr int Q = C / 4;  // chunks per pixel
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int q = c0 / 4 + j;
        st_shared_v4(stg + 16 * (lane * Q + (q ^ (lane & (Q - 1)))),
                     make_uint4(__float_as_uint(v16[4 * j]), __float_as_uint(v16[4 * j + 1]),
                                __float_as_uint(v16[4 * j + 2]), __float_as_uint(v16[4 * j + 3])));
    }
}
template <int C>
__device__ __forceinline__ void stage_flush(uint32_t stg, int lane, float* gdst, int npix) {
    constexpr int Q = C / 4;
    uint4* g = reinterpret_cast<uint4*>(gdst);
#pragma unroll
    for (int t = 0; t < Q; ++t) {
        const int j = lane + 32 * t, px = j / Q, q = j % Q;
        if (px < npix) g[j] = ld_shared_v4(stg + 16 * (px * Q + (q ^ (px & (Q - 1)))));
    }
}

// ------------------------------------------------------------------ exact border ring of the coarse-grid decoder
// The coarse-grid level-0 decoder reads the edge-replicated coarse input,
// which reproduces the up-sampled input on every fine row and column of the
// image but also one step outside it, where the 3x3 convolution reads zero
// padding instead: on its outermost ring of fine pixels (rows 0 and H - 1,
// columns 0 and W - 1) the epilogue writes nothing, and the producer warps,
// idle between their tiles' copies, compute those pixels exactly as the level
// is defined (Sec. 3.5): bilinear x2 up-sampling of the coarse input, 3x3 +
// ReLU, 1x1 + ReLU, head, sigmoid, in FP32 with the FP32 weights; a producer
// warp takes one pair of ring pixels after each tile's copies.
__host__ __device__ inline int ring_pixels(int Hf, int Wf) {
    return (Hf <= 0 || Wf <= 0) ? 0 : (Hf <= 2 ? Hf * Wf : 2 * Wf + 2 * (Hf - 2));
}

// ring pixel `item` of the batch -> view, fine row and column (false past the
// end); vh / vbase: a view at or before the item's and the number of ring pixels
// of the views before it (a search hint carried between calls; 0, 0 = none)
__device__ __forceinline__ bool ring_locate(const TcBatch& a, int item, int& v, int& fy, int& fx, int& vh,
                                            int& vbase) {
    if (item < vbase) vh = vbase = 0;
    item -= vbase;
    for (v = vh; v < a.nviews; ++v) {
        const int n = ring_pixels(2 * a.job[v].H, 2 * a.job[v].W);
        if (item < n) break;
        item -= n;
        vbase += n;
    }
    vh = v;
    if (v >= a.nviews) return false;
    const int Hf = 2 * a.job[v].H, Wf = 2 * a.job[v].W;
    if (Hf <= 2) { fy = item / Wf; fx = item % Wf; }
    else if (item < Wf) { fy = 0; fx = item; }
    else if (item < 2 * Wf) { fy = Hf - 1; fx = item - Wf; }
    else if (item < 2 * Wf + Hf - 2) { fy = 1 + item - 2 * Wf; fx = 0; }
    else { fy = 1 + item - 2 * Wf - (Hf - 2); fx = Wf - 1; }
    return true;
}

// One more finished unit (a tile row group of an epilogue warp, or a ring
// pixel) of view v; the arrival that completes the view stamps its time.
__device__ __forceinline__ void view_unit_done(const TcBatch& a, int v, unsigned expected) {
    __threadfence();
    unsigned long long* cnt = a.timing + 1 + kMaxViews + v;
    if (atomicAdd(cnt, 1ull) + 1 == expected) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        a.timing[1 + v] = t;
    }
}

// units of view v that view_unit_done counts in the level-0 decoder: every
// epilogue warp's pass over each tile, and every ring pixel
__device__ __forceinline__ unsigned view_units(const TcBatch& a, int v, int new_warps) {
    return static_cast<unsigned>(a.tile_start[v + 1] - a.tile_start[v]) * new_warps +
           ring_pixels(2 * a.job[v].H, 2 * a.job[v].W);
}

// Two ring pixels per warp pass, items `item` and `item + 1` (below n_end):
// half-warp h takes item + h, lane o of it output channel o.  FP32 weights in
// shared memory: w3s [tap][c][o], w1s [c][o]; b3 / b1 biases; hs the head
// weights then its bias; us a per-warp scratch of 2 x 9 x 16 floats (C = 16);
// vh / vbase the view-search hint of ring_locate.
__device__ __forceinline__ void ring_pair(const TcBatch& a, int item, int n_end, const float* w3s, const float* w1s,
                                          const float* b3, const float* b1, const float* hs, float* us, int lane,
                                          int new_warps, int& vh, int& vbase) {
    constexpr int C = 16;
    const int h = lane >> 4, o = lane & 15;
    int v = 0, fy = 0, fx = 0;
    const bool live = item + h < n_end && ring_locate(a, item + h, v, fy, fx, vh, vbase);
    // channel o of the up-sampled input at the pixel's nine taps (0 outside the image),
    // from the (at most 3 x 3) coarse pixels those taps read, each loaded once
    float u[9];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) u[tap] = 0.f;
    if (live) {
        const TcJob& job = a.job[v];
        const int Hl = job.H, Wl = job.W;
        const int cy0 = max(0, min(Hl - 1, (fy - 2) >> 1)), cx0 = max(0, min(Wl - 1, (fx - 2) >> 1));
        float pc[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int ci = min(Hl - 1, cy0 + r), cj = min(Wl - 1, cx0 + q);
                const uint16_t* p = job.in + (static_cast<size_t>(ci) * Wl + cj) * 2 * C + o;
                pc[r][q] = __bfloat162float(__ushort_as_bfloat16(p[0])) + __bfloat162float(__ushort_as_bfloat16(p[C]));
            }
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int y = fy + tap / 3 - 1, x = fx + tap % 3 - 1;
            if (y >= 0 && y < 2 * Hl && x >= 0 && x < 2 * Wl) {
                const BilinTap ty = bilin_tap(y, Hl), tx = bilin_tap(x, Wl);
                const int r0 = ty.i0 - cy0, r1 = ty.i1 - cy0, q0 = tx.i0 - cx0, q1 = tx.i1 - cx0;
                u[tap] = ty.w0 * (tx.w0 * pc[r0][q0] + tx.w1 * pc[r0][q1]) + ty.w1 * (tx.w0 * pc[r1][q0] + tx.w1 * pc[r1][q1]);
            }
        }
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) us[(h * 9 + tap) * C + o] = u[tap];
    __syncwarp();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int c = 0; c < C; c += 4) {
            const float4 u4 = *reinterpret_cast<const float4*>(us + (h * 9 + tap) * C + c);
            acc[0] = fmaf(w3s[(tap * C + c) * C + o], u4.x, acc[0]);
            acc[1] = fmaf(w3s[(tap * C + c + 1) * C + o], u4.y, acc[1]);
            acc[2] = fmaf(w3s[(tap * C + c + 2) * C + o], u4.z, acc[2]);
            acc[3] = fmaf(w3s[(tap * C + c + 3) * C + o], u4.w, acc[3]);
        }
    const float hv = fmaxf((acc[0] + acc[1]) + (acc[2] + acc[3]) + b3[o], 0.f);
    float z = b1[o];
#pragma unroll
    for (int c = 0; c < C; ++c) z = fmaf(w1s[c * C + o], __shfl_sync(0xffffffffu, hv, (lane & 16) | c), z);
    float t = hs[o] * fmaxf(z, 0.f);
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
    if (live && o == 0) {
        a.job[v].vis[static_cast<size_t>(fy) * (2 * a.job[v].W) + fx] = sigmoidf_fast(t + hs[C]);
        if (a.timing) view_unit_done(a, v, view_units(a, v, new_warps));
    }
    __syncwarp();  // us is reused by the next pass
}

// warps of a CTA: NEW epilogue, NPW producer, one MMA
constexpr int tc_warps(int NEW, int NPW, int EPI) { return NEW + NPW + 1 + 0 * EPI; }

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW, int KS, int ORD>
__global__ void __launch_bounds__(32 * tc_warps(NEW, NPW, EPI), 1) level_tc_kernel(const __grid_constant__ TcBatch a) {
    constexpr bool PAR = (EPI == TEPI_HEAD_PAR);
    using C = TcCfg<CIN, CMID, COUT, R, PRO, KS, PAR>;
    constexpr int NP = 32 * NPW, NT = 32 * tc_warps(NEW, NPW, EPI), MW = NEW + NPW, NE = 32 * NEW;
    static_assert(NEW == 4 || NEW == 8, "epilogue warps cover the four TMEM lane quarters");
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sA0 = sbase + C::OFF_A0, sA1 = sbase + C::OFF_A1, sRAW = sbase + C::OFF_RAW;
    const uint32_t sB3 = sbase + C::OFF_B3, sB1 = sbase + C::OFF_B1;
    float* bias3_s = reinterpret_cast<float*>(smem + C::OFF_BIAS3);
    float* bias1_s = reinterpret_cast<float*>(smem + C::OFF_BIAS1);
    float* head_s = reinterpret_cast<float*>(smem + C::OFF_HEAD);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint64_t* full = bar;          // [2] per input buffer
    uint64_t* mma3 = bar + 2;      // [2] per input buffer
    uint64_t* tfree = bar + 4;     // [2] per accumulator buffer
    uint64_t* a1full = bar + 6;
    uint64_t* mma1 = bar + 7;
    uint64_t* gfull = bar + 8;     // [2] per raw buffer
    uint64_t* rfree = bar + 10;    // [2] per raw buffer
    uint64_t* accf = bar + 12;     // [2] per accumulator buffer
    uint64_t* sfree = bar + 14;    // epilogue -> epilogue: output staging (in the 1x1 operand) done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 128);
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + 132);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    // ---- one-time set-up: weights, barriers, TMEM
    for (int i = tid; i < C::B3_CHUNKS; i += NT) st_shared_v4(sB3 + 16 * i, __ldg(a.b3img + i));
    for (int i = tid; i < C::B1_CHUNKS; i += NT) st_shared_v4(sB1 + 16 * i, __ldg(a.b1img + i));
    for (int i = tid; i < CMID; i += NT) bias3_s[i] = __ldg(a.bias3 + (PAR ? i % COUT : i));
    for (int i = tid; i < COUT; i += NT) bias1_s[i] = __ldg(a.bias1 + i);
    if (EPI == TEPI_HEAD || EPI == TEPI_HEAD4 || EPI == TEPI_HEAD_PAR)
        for (int i = tid; i < (EPI == TEPI_HEAD4 ? 4 : 1) * (COUT + 1); i += NT) head_s[i] = __ldg(a.head + i);
    for (int i = tid; i < C::ZERO_BYTES / 16; i += NT) st_shared_v4(sbase + C::OFF_ZERO + 16 * i, make_uint4(0, 0, 0, 0));
    float* ringw = reinterpret_cast<float*>(smem + C::OFF_RINGW);
    if constexpr (PAR) {
        for (int i = tid; i < 9 * COUT * COUT; i += NT) {
            const int o = i % COUT, c = (i / COUT) % COUT, tap = i / (COUT * COUT);
            ringw[i] = __ldg(a.w3 + (o * COUT + c) * 9 + tap);
        }
        for (int i = tid; i < COUT * COUT; i += NT) ringw[9 * COUT * COUT + i] = __ldg(a.w1 + (i % COUT) * COUT + i / COUT);
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(full + k, PRO == TPRO_TMA ? 1 : NP);
            mbar_init(mma3 + k, 1);
            mbar_init(tfree + k, NE);
            mbar_init(gfull + k, NP);
            mbar_init(rfree + k, NP);
            mbar_init(accf + k, 1);
        }
        mbar_init(a1full, NE);
        mbar_init(mma1, 1);
        mbar_init(sfree, NE);
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == MW) tmem_alloc(tslot, C::TMEM_COLS);
    fence_proxy_async_smem();  // the weights are read by the tensor core
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    // The set-up above reads only weights and parameters, which no stage kernel
    // writes: with a programmatic launch it overlaps the previous stage's tail.
    // The next stage may start its own set-up now; this stage's inputs are read
    // only after the previous stage has completed.
    griddep_launch_dependents();
    griddep_wait();
    if (PRO == TPRO_GATHER && a.timing && blockIdx.x == 0 && tid == 0) {
        // batched serving: the batch starts now (after the previous kernel of the
        // stream, which may be the previous batch's level-0 decoder still writing
        // these records); clear the views' completion records
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        a.timing[0] = t;
        for (int v = 0; v < a.nviews; ++v) a.timing[1 + v] = a.timing[1 + kMaxViews + v] = 0;
    }
    const uint32_t tbase = *tslot;
    // this CTA's tiles: a contiguous range of the tile list, which runs
    // column-major within each view (vertical strips of 128-pixel columns)
    const long long ntl = a.tile_start[a.nviews];
    const int t_lo = static_cast<int>(ntl * blockIdx.x / gridDim.x);
    const int t_hi = static_cast<int>(ntl * (blockIdx.x + 1) / gridDim.x);
    // view, origin and continuation (the tile right below the CTA's previous one)
    auto locate = [&](int tile, int& v, int& y0, int& x0, bool& cont) -> const TcJob& {
        while (tile >= a.tile_start[v + 1]) ++v;
        const TcJob& job = a.job[v];
        const int local = tile - a.tile_start[v];
        const int ys = local % job.tiles_y;
        y0 = ys * R;
        x0 = (local / job.tiles_y) * kTileM;
        cont = C::RING && tile > t_lo && ys > 0;
        return job;
    };
    // ring slots: staged row 0 of a tile sits in slot `base` (of every plane,
    // and of both slice buffers when KS > 1); the counter `ring` is the slot
    // after the last staged row produced so far
    auto ring_next = [&](bool cont, int& ring, int& base, int& first) {
        if constexpr (C::RING) {
            first = cont ? 2 : 0;
            base = cont ? (ring >= 2 ? ring - 2 : ring - 2 + C::NRW) : ring;
            ring = base + R + 2;
            if (ring >= C::NRW) ring -= C::NRW;
        } else {
            first = 0;
            base = 0;
        }
    };

    if (warp >= NEW && warp < MW) {
        // ================= producers: step st = (tile it, K slice s) fills input buffer st % 2
        const int pt = tid - NE;
        constexpr bool RAWP = (PRO == TPRO_GATHER || C::UP);  // raw inputs prefetched by cp.async
        int v = 0, vn = 0, it = 0, ring = 0;
        if constexpr (RAWP) {
            // prefetch the first tile's raw inputs into raw buffer 0
            if (t_lo < t_hi) {
                int y0, x0;
                bool cont;
                const TcJob& job = locate(t_lo, vn, y0, x0, cont);
                if constexpr (PRO == TPRO_GATHER) prefetch_gbuffer<NP, R>(job, y0, x0, sRAW, 0, pt);
                else prefetch_coarse<NP, CIN, R>(job, y0, x0, sRAW, pt);
                cp_async_arrive(gfull + 0);
            }
        }
        bool failed = false;
        // PAR: this CTA's share [ring_lo, ring_hi) of the batch's border-ring
        // pixels; producer warp w takes pairs w, w + NPW, ... one per tile
        int ring_lo = 0, ring_hi = 0, ring_vh = 0, ring_vb = 0;
        float* ring_us = ringw + 10 * COUT * COUT + (pt / 32) * 2 * 9 * COUT;
        if constexpr (PAR) {
            static_assert(NPW <= 8, "ring scratch per producer warp");
            long long nr = 0;
            for (int q = 0; q < a.nviews; ++q) nr += ring_pixels(2 * a.job[q].H, 2 * a.job[q].W);
            ring_lo = static_cast<int>(nr * blockIdx.x / gridDim.x);
            ring_hi = static_cast<int>(nr * (blockIdx.x + 1) / gridDim.x);
        }
        for (int tile = t_lo; tile < t_hi && !failed; ++tile, ++it) {
            int y0, x0, base, first;
            bool cont;
            const TcJob& job = locate(tile, v, y0, x0, cont);
            ring_next(cont, ring, base, first);
            const int rb = it & 1;
            if constexpr (RAWP) {
                // prefetch tile it + 1 into the other raw buffer
                const int next = tile + 1;
                if (next < t_hi) {
                    const int nb = rb ^ 1;
                    const int un = (it + 1) >> 1;  // use index of raw buffer nb for tile it + 1
                    if (un >= 1 && !wait_phase(rfree + nb, (un - 1) & 1, s_abort)) { failed = true; break; }
                    int ny0, nx0;
                    bool ncont;
                    const TcJob& nj = locate(next, vn, ny0, nx0, ncont);
                    const uint32_t nraw = sRAW + nb * C::RAW_BYTES;
                    if constexpr (PRO == TPRO_GATHER) prefetch_gbuffer<NP, R>(nj, ny0, nx0, nraw, ncont ? 2 : 0, pt);
                    else prefetch_coarse<NP, CIN, R>(nj, ny0, nx0, nraw, pt);
                    cp_async_arrive(gfull + nb);
                }
                // this tile's raw inputs
                if (!wait_phase(gfull + rb, (it >> 1) & 1, s_abort)) { failed = true; break; }
            }
            const uint32_t raw = sRAW + rb * C::RAW_BYTES;
#pragma unroll 1
            for (int s = 0; s < KS; ++s) {
                const int st = it * KS + s, b = st & 1;
                const uint32_t A0 = C::ONE_RING ? sA0 : sA0 + b * (C::A0_CHUNKS * 16);
                // the rows written now are free once the MMAs of step st - 2 are done
                if (PRO == TPRO_TMA && pt != 0) continue;  // one thread issues the tensor copies
                if (st >= 2 && !wait_phase(mma3 + b, ((st >> 1) - 1) & 1, s_abort)) { failed = true; break; }
                if constexpr (PRO == TPRO_PLAIN) {
                    copy_slice<NP, CIN, R, KS, C::NRW, PAR>(job.in, job.H, job.W, y0, x0, A0, s, base, first, pt);
                    cp_async_arrive(full + b);
                } else if constexpr (PRO == TPRO_TMA) {
                    tma_slice<CIN, R, KS, C::NRW>(&job.tmap, y0, x0, A0, s, base, first, full + b);
                } else {
                    if constexpr (PRO == TPRO_GATHER)
                        compute_gather<NP, R, C::NRW>(job, y0, x0, raw, A0, base, first, pt);
                    else
                        compute_up<NP, CIN, R, KS, PRO == TPRO_UP_SKIP, C::NRW>(job, y0, x0, raw, A0, s, base, first,
                                                                                pt);
                    fence_proxy_async_smem();
                    mbar_arrive(full + b);
                }
            }
            if (failed) break;
            if constexpr (RAWP) mbar_arrive(rfree + rb);
            if constexpr (PAR) {
                const int k = ring_lo + 2 * (it * NPW + pt / 32);
                if (k < ring_hi)
                    ring_pair(a, k, ring_hi, ringw, ringw + 9 * COUT * COUT, bias3_s, bias1_s, head_s, ring_us, tid & 31,
                              NEW, ring_vh, ring_vb);
            }
        }
        if constexpr (PAR) {
            for (int k = ring_lo + 2 * (it * NPW + pt / 32); !failed && k < ring_hi; k += 2 * NPW)
                ring_pair(a, k, ring_hi, ringw, ringw + 9 * COUT * COUT, bias3_s, bias1_s, head_s, ring_us, tid & 31,
                          NEW, ring_vh, ring_vb);
        }
        if (failed) {
            atomicExch(a.err, 3);
            *s_abort = 1;
        }
    } else if (warp == MW) {
        // ================= MMA issuer
        if ((tid & 31) == 0) {
            constexpr uint32_t id3 = idesc_bf16(128, C::N3);
            constexpr uint32_t id1 = idesc_bf16(128, C::N1);
            constexpr uint32_t kPlane = C::PLANE;
            constexpr int kA1Part = (CMID / 8) * kTileM;
            // 1x1 of tile index j once the epilogue has written its operand:
            // (A_hi + A_lo) [B_hi; B_lo] into the tile's accumulator buffer
            auto issue_1x1 = [&](int j) -> bool {
                if (!wait_phase(a1full, j & 1, s_abort)) return false;
                fence_after_sync();
                const uint32_t Dj = tbase + (j & 1) * C::TMEM_BUF;
                if constexpr (PAR) {
                    // per output parity p: its C_out channels (K = 16) times the
                    // C_out -> C_out weights, into columns [p N1, (p + 1) N1)
                    static_assert(COUT == 16, "one K step per parity");
                    const uint64_t bd = smem_desc(sB1, C::N1 * 16, 128);
                    for (int r = 0; r < R; ++r) {
                        const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const uint64_t ahi = smem_desc(row + 16 * (2 * p * kTileM), kTileM * 16, 128);
                            const uint64_t alo = smem_desc(row + 16 * (kA1Part + 2 * p * kTileM), kTileM * 16, 128);
                            mma_bf16(Dj + r * C::N3 + p * C::N1, ahi, bd, id1, 0);
                            mma_bf16(Dj + r * C::N3 + p * C::N1, alo, bd, id1, 1);
                        }
                    }
                    mma_commit(mma1);
                    return true;
                }
                for (int r = 0; r < R; ++r) {
                    const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
#pragma unroll
                    for (int kk = 0; kk < CMID / 16; ++kk) {
                        const uint64_t ahi = smem_desc(row + 16 * (2 * kk * kTileM), kTileM * 16, 128);
                        const uint64_t alo = smem_desc(row + 16 * (kA1Part + 2 * kk * kTileM), kTileM * 16, 128);
                        const uint64_t bd = smem_desc(sB1 + 16 * (2 * kk * C::N1), C::N1 * 16, 128);
                        mma_bf16(Dj + r * C::N3, ahi, bd, id1, kk > 0);
                        mma_bf16(Dj + r * C::N3, alo, bd, id1, 1);
                    }
                }
                mma_commit(mma1);
                return true;
            };
            int it = 0, v = 0, ring = 0;
            bool failed = false;
            for (int tile = t_lo; tile < t_hi; ++tile, ++it) {
                int y0, x0, rbase, first;
                bool cont;
                locate(tile, v, y0, x0, cont);
                ring_next(cont, ring, rbase, first);
                const int tb = it & 1;
                const uint32_t D = tbase + tb * C::TMEM_BUF;
#pragma unroll 1
                for (int s = 0; s < KS; ++s) {
                    const int st = it * KS + s, b = st & 1;
                    if (!wait_phase(full + b, (st >> 1) & 1, s_abort) ||
                        (s == 0 && it >= 2 && !wait_phase(tfree + tb, ((it >> 1) - 1) & 1, s_abort))) {
                        failed = true;
                        break;
                    }
                    fence_proxy_async_smem();  // cp.async / st.shared data -> tensor core
                    fence_after_sync();
                    const uint32_t A0 = C::ONE_RING ? sA0 : sA0 + b * (C::A0_CHUNKS * 16);
                    if constexpr (C::STACK) {
                        // clear the R x N3 accumulator columns (zero A operand), then
                        // one MMA per (staged row j, K step) of width (#ky) x N3:
                        // output row r accumulates at column (R - 1 - r) N3, kernel
                        // row ky of input row j at (R - 1 - j + ky) N3
                        if (s == 0)
                            mma_bf16(D, smem_desc(sbase + C::OFF_ZERO, 16, 128), smem_desc(sB3, 16, 128),
                                     idesc_bf16(128, R * C::N3), 0);
                        constexpr uint32_t kBL = 3 * C::N3 * 16;  // B: next K chunk
                        const uint64_t bdesc = smem_desc(sB3, kBL, 128);
#pragma unroll
                        for (int j = 0; j < R + 2; ++j) {
                            const int ka = j - (R - 1) > 0 ? j - (R - 1) : 0, kb = j < 2 ? j : 2;
                            const uint32_t id = idesc_bf16(128, (kb - ka + 1) * C::N3);
                            const uint32_t d = D + (R - 1 - j + ka) * C::N3;
                            if constexpr (C::SPLIT) {
                                // K = staged pixels m + 2p, m + 2p + 1 (4 features hi | lo each)
                                const uint64_t adesc = smem_desc(A0 + 16 * (row_slot<C::NRW>(rbase, j) * kSW), 16, 128);
#pragma unroll
                                for (int p2 = 0; p2 < 2; ++p2)
                                    mma_bf16(d, adesc + 2 * p2, bdesc + ((2 * p2 * 3 + ka) * C::N3), id, 1);
                            } else {
                                // K step = planes (2q, 2q + 1) of one part; both parts use the same weights
                                const uint64_t adesc = smem_desc(A0 + 16 * (row_slot<C::NRW>(rbase, j) * kSW), kPlane, 128);
#pragma unroll
                                for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                                    for (int q = 0; q < C::CGS / 2; ++q)
#pragma unroll
                                        for (int part = 0; part < 2; ++part)
                                            mma_bf16(d, adesc + ((part * C::CGS + 2 * q) * kPlane / 16 + kx),
                                                     bdesc + (((kx * C::CG_IN + s * C::CGS + 2 * q) * 3 + ka) * C::N3),
                                                     id, 1);
                            }
                        }
                    } else {
                        // 3x3: one MMA of width 2 CMID per (row, tap, K step, part)
                        for (int r = 0; r < R; ++r) {
                            const uint32_t d = D + r * C::N3;
#pragma unroll
                            for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                                for (int q = 0; q < C::CGS / 2; ++q) {
#pragma unroll
                                    for (int part = 0; part < 2; ++part) {
                                        const uint32_t a0 = A0 + (part * C::CGS + 2 * q) * kPlane +
                                                            16 * (row_slot<C::NRW>(rbase, r + tap / 3) * kSW + tap % 3);
                                        const uint32_t b0 = sB3 + 16 * ((tap * C::CG_IN + s * C::CGS + 2 * q) * C::N3);
                                        mma_bf16(d, smem_desc(a0, kPlane, 128), smem_desc(b0, C::N3 * 16, 128), id3,
                                                 (s | tap | q | part) != 0);
                                    }
                                }
                            }
                        }
                    }
                    mma_commit(mma3 + b);  // input buffer b consumed
                }
                if (failed) break;
                mma_commit(accf + tb);     // 3x3 accumulators of this tile complete
                // ORD 0: this tile's 1x1 next; ORD 1: the previous tile's 1x1 now, so
                // that this tile's 3x3 runs on the tensor core while the epilogue
                // prepares the previous tile's 1x1 operand
                if (ORD == 0 ? !issue_1x1(it) : (it > 0 && !issue_1x1(it - 1))) {
                    failed = true;
                    break;
                }
            }
            if (ORD == 1 && !failed && it > 0 && !issue_1x1(it - 1)) failed = true;
            if (failed) {
                atomicExch(a.err, 4);
                *s_abort = 1;
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue (warps 0 .. NEW-1; TMEM lane quarter = warp % 4)
        constexpr int G = NEW / 4;
        const int m = (warp & 3) * 32 + (tid & 31);  // pixel of the row block = TMEM lane
        const int rg = G == 1 ? 0 : warp >> 2;         // row group of this warp
        const uint32_t tlane = tbase + (static_cast<uint32_t>((warp & 3) * 32) << 16);
        constexpr int kA1Part = (CMID / 8) * kTileM;
        // FP32 rows go out through a per-warp staging area in the 1x1 operand
        // buffer (free between the 1x1 MMAs and the next tile's 3x3 result) when
        // it has room for every epilogue warp
        constexpr int kStg = 32 * COUT * 4;                              // one row of a warp
        constexpr int kRows = EPI == TEPI_SKIP_POOL ? 2 : 1;            // rows staged at once
        constexpr bool kStage = (EPI == TEPI_STORE || EPI == TEPI_STORE_PAIR || EPI == TEPI_SKIP_POOL) &&
                                NEW * kRows * kStg <= C::A1_CHUNKS * 16;
        static_assert(EPI != TEPI_STORE_PAIR || (kStage && COUT == 16), "pair rows go out through the staging area");
        int v = 0, it = 0;
        for (int tile = t_lo; tile < t_hi; ++tile, ++it) {
            const int tb = it & 1;
            int y0, x0;
            bool cont;
            const TcJob& job = locate(tile, v, y0, x0, cont);
            const int H = job.H, W = job.W;
            const uint32_t Dl = tlane + tb * C::TMEM_BUF;
            if (!wait_phase(accf + tb, (it >> 1) & 1, s_abort)) {
                atomicExch(a.err, 1);
                *s_abort = 1;
                break;
            }
            fence_after_sync();
            if constexpr (kStage) {
                // every epilogue warp has flushed the previous tile's staged rows
                if (it >= 1 && !wait_phase(sfree, (it - 1) & 1, s_abort)) {
                    atomicExch(a.err, 6);
                    *s_abort = 1;
                    break;
                }
            }
            // ---- 3x3 result: bias + ReLU -> BF16 hi + lo -> operand of the 1x1
            if constexpr (PAR) {
                // two parities (32 columns of each weight part) in flight at once
                for (int r = rg; r < R; r += G) {
                    const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
#pragma unroll
                    for (int q = 0; q < CMID; q += 32) {
                        float val[32], lo[32];
                        tmem_ld32(Dl + r * C::N3 + q, val);
                        tmem_ld32(Dl + r * C::N3 + CMID + q, lo);
                        tmem_ld_wait();
#pragma unroll
                        for (int c0 = 0; c0 < 32; c0 += 8) {
                            float x[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) x[j] = fmaxf(val[c0 + j] + lo[c0 + j] + bias3_s[q + c0 + j], 0.f);
                            uint4 h, l;
                            split_chunks(x, h, l);
                            st_shared_v4(row + 16 * (((q + c0) / 8) * kTileM + m), h);
                            st_shared_v4(row + 16 * (kA1Part + ((q + c0) / 8) * kTileM + m), l);
                        }
                    }
                }
            } else
            for (int r = rg; r < R; r += G) {
#pragma unroll
                for (int c0 = 0; c0 < CMID; c0 += 16) {
                    float val[16], lo[16];
                    const uint32_t col = (C::STACK ? R - 1 - r : r) * C::N3;
                    tmem_ld16(Dl + col + c0, val);         // x W_hi
                    tmem_ld16(Dl + col + CMID + c0, lo);   // x W_lo
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) val[j] = fmaxf(val[j] + lo[j] + bias3_s[c0 + j], 0.f);
                    const int cg = c0 / 8;
                    const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
                    uint4 h0, l0, h1, l1;
                    split_chunks(val, h0, l0);
                    split_chunks(val + 8, h1, l1);
                    st_shared_v4(row + 16 * (cg * kTileM + m), h0);
                    st_shared_v4(row + 16 * ((cg + 1) * kTileM + m), h1);
                    st_shared_v4(row + 16 * (kA1Part + cg * kTileM + m), l0);
                    st_shared_v4(row + 16 * (kA1Part + (cg + 1) * kTileM + m), l1);
                }
            }
            fence_proxy_async_smem();
            fence_before_sync();
            mbar_arrive(a1full);
            if (!wait_phase(mma1, it & 1, s_abort)) {
                atomicExch(a.err, 2);
                *s_abort = 1;
                break;
            }
            fence_after_sync();
            // ---- 1x1 result -> outputs (pooled: BF16 hi + lo [pixel][part][COUT]; else FP32)
            const int ox = x0 + m;
            const int lane = tid & 31;
            const uint32_t stg = sA1 + warp * (kRows * kStg);
            const int px0 = x0 + 32 * (warp & 3);
            const int npix = min(32, W - px0);
            if constexpr (EPI == TEPI_POOL || EPI == TEPI_SKIP_POOL) {
                for (int r = 2 * rg; r < R; r += 2 * G) {
                    float s[COUT];
#pragma unroll
                    for (int c0 = 0; c0 < COUT; c0 += 16) {
                        float v0[16], v1[16], w0[16], w1[16];
                        tmem_ld16(Dl + r * C::N3 + c0, v0);
                        tmem_ld16(Dl + r * C::N3 + COUT + c0, w0);
                        tmem_ld16(Dl + (r + 1) * C::N3 + c0, v1);
                        tmem_ld16(Dl + (r + 1) * C::N3 + COUT + c0, w1);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            v0[j] = fmaxf(v0[j] + w0[j] + bias1_s[c0 + j], 0.f);
                            v1[j] = fmaxf(v1[j] + w1[j] + bias1_s[c0 + j], 0.f);
                            s[c0 + j] = v0[j] + v1[j];
                        }
                        if constexpr (EPI == TEPI_SKIP_POOL) {
                            const int oy = y0 + r;
                            if constexpr (kStage) {
                                stage_put<COUT>(stg, lane, c0, v0);
                                stage_put<COUT>(stg + kStg, lane, c0, v1);
                            } else if (oy < H && ox < W) {
                                float4* dst = reinterpret_cast<float4*>(job.out_skip +
                                                                        (static_cast<size_t>(oy) * W + ox) * COUT + c0);
                                float4* dst1 = dst + static_cast<size_t>(W) * (COUT / 4);
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    dst[q] = make_float4(v0[4 * q], v0[4 * q + 1], v0[4 * q + 2], v0[4 * q + 3]);
                                    dst1[q] = make_float4(v1[4 * q], v1[4 * q + 1], v1[4 * q + 2], v1[4 * q + 3]);
                                }
                            }
                        }
                    }
                    if constexpr (EPI == TEPI_SKIP_POOL && kStage) {
                        __syncwarp();
                        const int oy = y0 + r;
                        if (oy < H && npix > 0) {
                            float* g0 = job.out_skip + (static_cast<size_t>(oy) * W + px0) * COUT;
                            stage_flush<COUT>(stg, lane, g0, npix);
                            stage_flush<COUT>(stg + kStg, lane, g0 + static_cast<size_t>(W) * COUT, npix);
                        }
                        __syncwarp();
                    }
#pragma unroll
                    for (int c = 0; c < COUT; ++c) s[c] = 0.25f * (s[c] + __shfl_xor_sync(0xffffffffu, s[c], 1));
                    const int oy = y0 + r;
                    if (oy < H && ox < W) {
                        // even pixel writes the hi part, odd pixel the lo part
                        const int part = m & 1;
                        uint4* dst = reinterpret_cast<uint4*>(job.out + (static_cast<size_t>(oy / 2) * (W / 2) + ox / 2) *
                                                                            2 * COUT) + part * (COUT / 8);
#pragma unroll
                        for (int c = 0; c < COUT; c += 8) {
                            uint4 h, l;
                            split_chunks(s + c, h, l);
                            dst[c / 8] = part ? l : h;
                        }
                    }
                }
            } else if constexpr (EPI == TEPI_HEAD_PAR) {
                // coarse pixel (oy, ox) -> fine pixels (2 oy + a, 2 ox + b), parity
                // p = 2a + b in TMEM columns [p N1, (p + 1) N1): 1x1 hi | lo parts
                const int Wf = 2 * W;
                for (int r = rg; r < R; r += G) {
                    const int oy = y0 + r;
                    float o4[4];
#pragma unroll
                    for (int q = 0; q < 4; q += 2) {
                        // parities q, q + 1: columns [q N1, (q + 2) N1), hi | lo parts of each
                        float d[2][32];
                        tmem_ld32(Dl + r * C::N3 + q * C::N1, d[0]);
                        tmem_ld32(Dl + r * C::N3 + (q + 1) * C::N1, d[1]);
                        tmem_ld_wait();
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            float hsum = 0.f;
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                hsum = fmaf(head_s[j], fmaxf(d[k][j] + d[k][COUT + j] + bias1_s[j], 0.f), hsum);
                            o4[q + k] = sigmoidf_fast(hsum + head_s[COUT]);
                        }
                    }
                    if (oy < H && ox < W) {
                        float* v0 = job.vis + static_cast<size_t>(2 * oy) * Wf + 2 * ox;
                        if (oy > 0 && oy < H - 1 && ox > 0 && ox < W - 1) {
                            reinterpret_cast<float2*>(v0)[0] = make_float2(o4[0], o4[1]);
                            reinterpret_cast<float2*>(v0 + Wf)[0] = make_float2(o4[2], o4[3]);
                        } else {
                            // the outermost fine ring is the producers' (exact path)
#pragma unroll
                            for (int p = 0; p < 4; ++p) {
                                const int fy = 2 * oy + (p >> 1), fx = 2 * ox + (p & 1);
                                if (fy > 0 && fy < 2 * H - 1 && fx > 0 && fx < Wf - 1) v0[(p >> 1) * Wf + (p & 1)] = o4[p];
                            }
                        }
                    }
                }
            } else {
                for (int r = rg; r < R; r += G) {
                    const int oy = y0 + r;
                    float hsum = 0.f;
                    float h4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int c0 = 0; c0 < COUT; c0 += 16) {
                        float val[16], lo[16];
                        tmem_ld16(Dl + r * C::N3 + c0, val);
                        tmem_ld16(Dl + r * C::N3 + COUT + c0, lo);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) val[j] = fmaxf(val[j] + lo[j] + bias1_s[c0 + j], 0.f);
                        if constexpr (EPI == TEPI_STORE_PAIR) {
                            // [part][16 channels] of the pixel: hi chunks, then lo chunks
                            uint4 h0, l0, h1, l1;
                            split_chunks(val, h0, l0);
                            split_chunks(val + 8, h1, l1);
                            const float pk[16] = {
                                __uint_as_float(h0.x), __uint_as_float(h0.y), __uint_as_float(h0.z), __uint_as_float(h0.w),
                                __uint_as_float(h1.x), __uint_as_float(h1.y), __uint_as_float(h1.z), __uint_as_float(h1.w),
                                __uint_as_float(l0.x), __uint_as_float(l0.y), __uint_as_float(l0.z), __uint_as_float(l0.w),
                                __uint_as_float(l1.x), __uint_as_float(l1.y), __uint_as_float(l1.z), __uint_as_float(l1.w)};
                            stage_put<COUT>(stg, lane, c0, pk);
                        } else if constexpr (EPI == TEPI_STORE) {
                            if constexpr (kStage) {
                                stage_put<COUT>(stg, lane, c0, val);
                            } else if (oy < H && ox < W) {
                                float4* dst = reinterpret_cast<float4*>(job.out_f +
                                                                        (static_cast<size_t>(oy) * W + ox) * COUT + c0);
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    dst[q] = make_float4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
                            }
                        } else if constexpr (EPI == TEPI_HEAD4) {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
#pragma unroll
                                for (int j = 0; j < 16; ++j) h4[k] = fmaf(head_s[k * COUT + c0 + j], val[j], h4[k]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) hsum = fmaf(head_s[c0 + j], val[j], hsum);
                        }
                    }
                    if (EPI == TEPI_HEAD && oy < H && ox < W)
                        job.vis[static_cast<size_t>(oy) * W + ox] = sigmoidf_fast(hsum + head_s[COUT]);
                    if (EPI == TEPI_HEAD4 && oy < H && ox < W)
                        reinterpret_cast<float4*>(job.out_f)[static_cast<size_t>(oy) * W + ox] =
                            make_float4(h4[0] + head_s[4 * COUT], h4[1] + head_s[4 * COUT + 1],
                                        h4[2] + head_s[4 * COUT + 2], h4[3] + head_s[4 * COUT + 3]);
                    if constexpr ((EPI == TEPI_STORE || EPI == TEPI_STORE_PAIR) && kStage) {
                        __syncwarp();
                        float* orow = EPI == TEPI_STORE_PAIR ? reinterpret_cast<float*>(job.out) : job.out_f;
                        if (oy < H && npix > 0)
                            stage_flush<COUT>(stg, lane, orow + (static_cast<size_t>(oy) * W + px0) * COUT, npix);
                        __syncwarp();
                    }
                }
            }
            if (PAR && a.timing) {
                __syncwarp();
                if ((tid & 31) == 0) view_unit_done(a, v, view_units(a, v, NEW));
            }
            // the next tile's 3x3 result goes where the rows were staged
            if constexpr (kStage) mbar_arrive(sfree);
            fence_before_sync();
            mbar_arrive(tfree + tb);
        }
    }

    // wait for every cp.async of this thread before the CTA ends
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    fence_after_sync();
    if (warp == MW) tmem_dealloc(tbase, C::TMEM_COLS);
}

// ------------------------------------------------------------------ variants and launch
// pdl: launch with programmatic stream serialisation (the kernel's set-up may
// overlap the previous kernel of the stream, see griddep_wait)
template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW, int KS, int ORD>
static cudaError_t launch_variant(const TcBatch& a, int ctas_per_sm, cudaStream_t stream, bool pdl) {
    using C = TcCfg<CIN, CMID, COUT, R, PRO, KS, EPI == TEPI_HEAD_PAR>;
    auto kern = level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI, NEW, NPW, KS, ORD>;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::BYTES);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the kernel's own resources: registers,
        // shared memory (228 KB per SM, 1 KB reserved per CTA) and TMEM columns
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int regs = ((fa.numRegs + 7) / 8) * 8 * (32 * tc_warps(NEW, NPW, EPI));
        const int by_regs = regs > 0 ? 65536 / regs : 8;
        const int by_smem = (228 * 1024) / (C::BYTES + 1024);
        int o = by_regs < by_smem ? by_regs : by_smem;
        if (o > C::TMEM_CAP) o = C::TMEM_CAP;
        if (o > 8) o = 8;
        occ = o < 1 ? 1 : o;
    }
    const int tiles = a.tile_start[a.nviews];
    if (tiles == 0) return cudaSuccess;
    const int per_sm = (ctas_per_sm <= 0 || ctas_per_sm > occ) ? occ : ctas_per_sm;
    const int cap = per_sm * num_sms();
    const int grid = tiles < cap ? tiles : cap;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * tc_warps(NEW, NPW, EPI));
    cfg.dynamicSmemBytes = C::BYTES;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW, int KS, int ORD>
static const void* kernel_of() {
    return reinterpret_cast<const void*>(level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI, NEW, NPW, KS, ORD>);
}

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW, int KS, int ORD>
static int occupancy_of() {
    using C = TcCfg<CIN, CMID, COUT, R, PRO, KS, EPI == TEPI_HEAD_PAR>;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI, NEW, NPW, KS, ORD>) != cudaSuccess) return 1;
    const int regs = ((fa.numRegs + 7) / 8) * 8 * (32 * tc_warps(NEW, NPW, EPI));
    const int by_regs = regs > 0 ? 65536 / regs : 8;
    const int by_smem = (228 * 1024) / (C::BYTES + 1024);
    int o = by_regs < by_smem ? by_regs : by_smem;
    if (o > C::TMEM_CAP) o = C::TMEM_CAP;
    if (o > 8) o = 8;
    return o < 1 ? 1 : o;
}

// Variant tables: tile height R and warp roles of every stage (the
// autotuner's search space).
using LaunchFn = cudaError_t (*)(const TcBatch&, int, cudaStream_t, bool);
struct Variant { int R, ew, pw, ks, ord; LaunchFn fn; const void* (*func)(); int (*occ)(); int tma, cin; };
#define NSM_VARIANT(R_, EW_, PW_, KS_, ORD_, CIN_, CMID_, COUT_, PRO_, EPI_)                              \
    {R_, EW_, PW_, KS_, ORD_, launch_variant<CIN_, CMID_, COUT_, R_, PRO_, EPI_, EW_, PW_, KS_, ORD_>,      \
     kernel_of<CIN_, CMID_, COUT_, R_, PRO_, EPI_, EW_, PW_, KS_, ORD_>,                                  \
     occupancy_of<CIN_, CMID_, COUT_, R_, PRO_, EPI_, EW_, PW_, KS_, ORD_>, (PRO_) == TPRO_TMA, CIN_}
// both MMA schedules of one tile shape / warp split
#define NSM_VARIANT2(R_, EW_, PW_, KS_, CIN_, CMID_, COUT_, PRO_, EPI_)                                   \
    NSM_VARIANT(R_, EW_, PW_, KS_, 0, CIN_, CMID_, COUT_, PRO_, EPI_),                                     \
    NSM_VARIANT(R_, EW_, PW_, KS_, 1, CIN_, CMID_, COUT_, PRO_, EPI_)

// (rows, epilogue warps, producer warps, K slices, [MMA order,] C_in, C_mid, C_out, prologue, epilogue)
static const Variant kVarEnc0[] = {
    NSM_VARIANT(4, 4, 8, 1, 0, 4, 16, 16, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT(4, 8, 8, 1, 0, 4, 16, 16, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT2(8, 4, 8, 1, 4, 16, 16, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT2(8, 4, 16, 1, 4, 16, 16, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT(8, 8, 12, 1, 0, 4, 16, 16, TPRO_GATHER, TEPI_POOL)};
static const Variant kVarEnc1[] = {
    NSM_VARIANT(2, 4, 8, 1, 0, 16, 32, 32, TPRO_PLAIN, TEPI_SKIP_POOL),
    NSM_VARIANT(2, 8, 8, 1, 0, 16, 32, 32, TPRO_PLAIN, TEPI_SKIP_POOL),
    NSM_VARIANT2(4, 4, 8, 1, 16, 32, 32, TPRO_PLAIN, TEPI_SKIP_POOL),
    NSM_VARIANT2(4, 8, 8, 1, 16, 32, 32, TPRO_PLAIN, TEPI_SKIP_POOL),
    NSM_VARIANT2(4, 4, 1, 1, 16, 32, 32, TPRO_TMA, TEPI_SKIP_POOL),
    NSM_VARIANT2(4, 8, 1, 1, 16, 32, 32, TPRO_TMA, TEPI_SKIP_POOL)};
static const Variant kVarBott[] = {
    NSM_VARIANT(1, 4, 8, 1, 0, 32, 64, 32, TPRO_PLAIN, TEPI_STORE),
    NSM_VARIANT2(2, 4, 8, 2, 32, 64, 32, TPRO_PLAIN, TEPI_STORE),
    NSM_VARIANT2(2, 8, 8, 2, 32, 64, 32, TPRO_PLAIN, TEPI_STORE),
    NSM_VARIANT2(2, 4, 1, 2, 32, 64, 32, TPRO_TMA, TEPI_STORE),
    NSM_VARIANT2(2, 8, 1, 2, 32, 64, 32, TPRO_TMA, TEPI_STORE)};
static const Variant kVarDec1[] = {
    NSM_VARIANT2(2, 4, 8, 2, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR),
    NSM_VARIANT2(2, 8, 8, 2, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR),
    NSM_VARIANT(2, 4, 9, 2, 0, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR),
    NSM_VARIANT(2, 8, 9, 2, 0, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR),
    NSM_VARIANT(2, 4, 12, 2, 0, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR),
    NSM_VARIANT(2, 8, 12, 2, 0, 32, 32, 16, TPRO_UP_SKIP, TEPI_STORE_PAIR)};
// level-0 decoder on the coarse grid: the tile is R coarse rows x 128 coarse
// pixels (2R fine rows x 256 fine pixels), C_mid = 4 parities x 16 channels
static const Variant kVarDec0[] = {
    NSM_VARIANT2(1, 4, 4, 1, 16, 64, 16, TPRO_PLAIN, TEPI_HEAD_PAR),
    NSM_VARIANT2(2, 4, 4, 1, 16, 64, 16, TPRO_PLAIN, TEPI_HEAD_PAR),
    NSM_VARIANT2(2, 8, 4, 1, 16, 64, 16, TPRO_PLAIN, TEPI_HEAD_PAR),
    NSM_VARIANT2(2, 4, 8, 1, 16, 64, 16, TPRO_PLAIN, TEPI_HEAD_PAR),
    NSM_VARIANT2(2, 8, 8, 1, 16, 64, 16, TPRO_PLAIN, TEPI_HEAD_PAR)};

static const Variant kVarDec1Head4[] = {
    NSM_VARIANT2(2, 4, 8, 2, 32, 32, 16, TPRO_UP_SKIP, TEPI_HEAD4)};

struct StageTable { const Variant* v; int n; };
#define NSM_STAGE(t) {t, static_cast<int>(sizeof(t) / sizeof(t[0]))}
static const StageTable kStages[kTcStages] = {
    NSM_STAGE(kVarEnc0), NSM_STAGE(kVarEnc1), NSM_STAGE(kVarBott), NSM_STAGE(kVarDec1), NSM_STAGE(kVarDec0)};

int tc_stage_variants(int stage) { return (stage >= 0 && stage < kTcStages) ? kStages[stage].n : 0; }
int tc_stage_rows(int stage, int variant) { return kStages[stage].v[variant].R; }
const void* tc_stage_kernel(int stage, int variant) { return kStages[stage].v[variant].func(); }
int tc_stage_occupancy(int stage, int variant) { return kStages[stage].v[variant].occ(); }

int tc_stage_order(int stage, int variant) { return kStages[stage].v[variant].ord; }

int tc_stage_warps(int stage, int variant, int* producer_warps) {
    if (producer_warps) *producer_warps = kStages[stage].v[variant].pw;
    return kStages[stage].v[variant].ew;
}

int tc_default_variant(int stage) {
    // the fastest plan of the 1080p autotuning runs: enc0 8 rows with 16 producer
    // warps, enc1 / bottleneck on TMA rows, dec1 9 producer warps, dec0 8 epilogue
    // and 8 producer warps
    static const int def[kTcStages] = {4, 8, 6, 4, 9};
    return def[stage];
}

// Fill the tile table of a stage for the given tile height.
void tc_fill_tiles(TcBatch& b, int rows) {
    b.tile_start[0] = 0;
    for (int i = 0; i < b.nviews; ++i) {
        TcJob& j = b.job[i];
        j.tiles_x = (j.W + kTileM - 1) / kTileM;
        j.tiles_y = (j.H + rows - 1) / rows;
        b.tile_start[i + 1] = b.tile_start[i] + j.tiles_x * j.tiles_y;
    }
}

cudaError_t tc_encode_input_map(CUtensorMap* map, const uint16_t* in, int H, int W, int cin) {
    // cuTensorMapEncodeTiled, resolved through the runtime (the library does not link the driver library)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                                                                     : nullptr;
    }();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t nch = 2 * cin / 8;  // 16-byte chunks per pixel: [part][channel group]
    const cuuint64_t dims[4] = {8, nch, static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
    const cuuint64_t strides[3] = {16, nch * 16, static_cast<cuuint64_t>(W) * nch * 16};
    const cuuint32_t box[4] = {8, 1, kSW, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<uint16_t*>(in), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_prepare_stage(int stage, int variant, TcBatch& b) {
    if (stage < 0 || stage >= kTcStages || variant < 0 || variant >= kStages[stage].n) return cudaErrorInvalidValue;
    const Variant& v = kStages[stage].v[variant];
    tc_fill_tiles(b, v.R);
    if (v.tma)
        for (int i = 0; i < b.nviews; ++i) {
            TcJob& j = b.job[i];
            if (j.H > 0 && j.W > 0) {
                cudaError_t e = tc_encode_input_map(&j.tmap, j.in, j.H, j.W, v.cin);
                if (e != cudaSuccess) return e;
            }
        }
    return cudaSuccess;
}

cudaError_t tc_launch_stage(int stage, int variant, TcBatch& b, int ctas_per_sm, cudaStream_t stream) {
    cudaError_t e = tc_prepare_stage(stage, variant, b);
    if (e != cudaSuccess) return e;
    // every stage overlaps its set-up with the tail of the previous kernel of the
    // stream (for the first stage: the previous frame's level-0 decoder); each
    // reads its inputs only after griddepcontrol.wait
    return kStages[stage].v[variant].fn(b, ctas_per_sm, stream, true);
}

const char* const kInferKernelNamesBf16[kInferKernelsBf16] = {
    "bf16_enc0_gather", "bf16_enc1", "bf16_bottleneck", "bf16_dec1", "bf16_dec0_head"};

// Jobs of the five stages for a list of views (one Activations per view).
void tc_make_batches(const GatherParams* g, const Activations* act, float* const* vis, int n, const float* params,
                     const uint16_t* img, int* err, TcBatch* out) {
    const LayerOffsets off = layer_offsets();
    const BF16Images im = bf16_images();
    auto I = [&](int layer) { return reinterpret_cast<const uint4*>(img + im.img_off[layer]); };
    const int l3[kTcStages] = {ENC0_3, ENC1_3, BOTT_3, DEC1_3, DEC0_3};
    const int l1[kTcStages] = {ENC0_1, ENC1_1, BOTT_1, DEC1_1, DEC0_1};
    for (int s = 0; s < kTcStages; ++s) {
        TcBatch& b = out[s];
        b = TcBatch{};
        b.nviews = n;
        b.b3img = I(l3[s]);
        b.b1img = I(l1[s]);
        b.bias3 = params + off.b[l3[s]];
        b.bias1 = params + off.b[l1[s]];
        b.head = params + off.w[HEAD];  // head weights followed by its bias
        b.w3 = params + off.w[l3[s]];
        b.w1 = params + off.w[l1[s]];
        b.err = err;
        for (int i = 0; i < n; ++i) {
            TcJob& j = b.job[i];
            j.g = g[i];
            const int H = g[i].H, W = g[i].W;
            const Activations& A = act[i];
            switch (s) {
                case 0: j.H = H; j.W = W; j.out = static_cast<uint16_t*>(A.e0); break;
                case 1: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(A.e0);
                        j.out_skip = static_cast<float*>(A.s1); j.out = static_cast<uint16_t*>(A.p1); break;
                case 2: j.H = H / 4; j.W = W / 4; j.in = static_cast<const uint16_t*>(A.p1);
                        j.out_f = static_cast<float*>(A.bo); break;
                case 3: j.H = H / 2; j.W = W / 2; j.in_f = static_cast<const float*>(A.bo);
                        j.skip = static_cast<const float*>(A.s1); j.out = static_cast<uint16_t*>(A.d1); break;
                // the level-0 decoder runs on the coarse (level-1) grid
                default: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(A.d1); j.vis = vis[i]; break;
            }
        }
    }
}

cudaError_t launch_infer_bf16(const GatherParams& g, const float* params, const uint16_t* img,
                              const Activations& act, float* vis, int* err, cudaStream_t stream,
                              const StageEvents& se, const int* variant, const int* ctas) {
    TcBatch b[kTcStages];
    float* vp[1] = {vis};
    tc_make_batches(&g, &act, vp, 1, params, img, err, b);
    for (int s = 0; s < kTcStages; ++s) {
        se.rec(s);
        cudaError_t e = tc_launch_stage(s, variant ? variant[s] : tc_default_variant(s), b[s],
                                        ctas ? ctas[s] : 0, stream);
        if (e != cudaSuccess) return e;
    }
    se.rec(kTcStages);
    return cudaSuccess;
}

const char* const kInferKernelNamesS2d[kInferKernelsS2d] = {
    "s2d_gather_flatten", "s2d_bf16_enc1", "s2d_bf16_bottleneck", "s2d_bf16_dec1_head4", "s2d_recombine"};

// Space-to-depth topology (Sec. 3.5), BF16 form: the gather writes the 2x2
// flattened features (16 channels, BF16 hi + lo) where the 3-level net keeps
// its pooled level-0 output, so the level-1 encoder and the bottleneck run
// unchanged; dec1 ends in the 4-channel head; a last kernel recombines.
cudaError_t launch_infer_s2d_bf16(const GatherParams& g, const float* params, const uint16_t* img,
                                  const Activations& A, float* vis, int* err, cudaStream_t stream,
                                  const StageEvents& se) {
    const LayerOffsets off = layer_offsets_s2d();
    const BF16Images im = bf16_images(true);
    auto I = [&](int layer) { return reinterpret_cast<const uint4*>(img + im.img_off[layer]); };
    const int H = g.H, W = g.W;
    se.rec(0);
    cudaError_t e = launch_s2d_features(g, static_cast<uint16_t*>(A.e0), stream);
    if (e != cudaSuccess) return e;
    const int l3[3] = {ENC1_3, BOTT_3, DEC1_3}, l1[3] = {ENC1_1, BOTT_1, DEC1_1};
    for (int s = 0; s < 3; ++s) {
        TcBatch b{};
        b.nviews = 1;
        b.b3img = I(l3[s]);
        b.b1img = I(l1[s]);
        b.bias3 = params + off.b[l3[s]];
        b.bias1 = params + off.b[l1[s]];
        b.head = params + off.w[HEAD];  // [4][16] weights followed by the 4 biases
        b.err = err;
        TcJob& j = b.job[0];
        j.g = g;
        se.rec(1 + s);
        if (s == 0) {
            j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(A.e0);
            j.out_skip = static_cast<float*>(A.s1); j.out = static_cast<uint16_t*>(A.p1);
            e = tc_launch_stage(1, tc_default_variant(1), b, 0, stream);
        } else if (s == 1) {
            j.H = H / 4; j.W = W / 4; j.in = static_cast<const uint16_t*>(A.p1); j.out_f = static_cast<float*>(A.bo);
            e = tc_launch_stage(2, tc_default_variant(2), b, 0, stream);
        } else {
            j.H = H / 2; j.W = W / 2; j.in_f = static_cast<const float*>(A.bo);
            j.skip = static_cast<const float*>(A.s1); j.out_f = static_cast<float*>(A.d1);
            tc_fill_tiles(b, kVarDec1Head4[0].R);
            e = kVarDec1Head4[0].fn(b, 0, stream, true);
        }
        if (e != cudaSuccess) return e;
    }
    se.rec(4);
    e = launch_s2d_output(static_cast<const float*>(A.d1), H, W, vis, stream);
    se.rec(5);
    return e;
}

}  // namespace nsm
