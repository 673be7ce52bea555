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
// Tile: R rows x 128 pixels of the level; MMA row block = one 128-pixel row
// segment.  The input tile with its 1-pixel halo is staged in shared memory
// as 16-byte chunks of 8 channels, [channel group][staged row][staged pixel],
// which is the tensor core's no-swizzle K-major operand layout: the A operand
// of tap (ky, kx) and channel pair (2g, 2g+1) is the same buffer started
// (ky, kx) chunks further on, so the im2col matrix is never built.  The 3x3
// result goes TMEM -> registers (bias, ReLU) -> shared memory as BF16 hi + lo
// parts, the A operand of the 1x1 MMA (written into the same TMEM columns).
// Weights are BF16 hi + lo images: each K step runs against both, and the
// 1x1 adds A_hi B_hi + A_hi B_lo + A_lo B_hi, so weight and intermediate
// rounding leave no trace beyond ~2^-16; only the level outputs are BF16.
//
// First level: the four FP32 features are split into BF16 hi + lo parts
// (f = hi + lo to ~2^-16 relative), 8 "channels" per pixel; K steps pair two
// taps (two 16-byte chunks), so the 3x3 4 -> 16 convolution is five K = 16
// steps with a zero-weight pad.  This keeps the depth-test features
// (z / z_f near 1, z - z_f near 0) at near-FP32 resolution.
//
// 256 threads (8 warps) per CTA: all stage the input; warp w reads TMEM lane
// quarter w % 4 and the two warpgroups split the epilogue rows.
#include "nsm_internal.h"
#include "tc_common.cuh"
#include "tc_stage.h"

namespace nsm {

using namespace tc;

constexpr int kNT = 256;         // threads per CTA
constexpr int kTileM = 128;      // pixels per MMA row block
constexpr int kSW = 136;         // staged pixels per row (128 + halo + pad)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait

template <int CIN, int CMID, int COUT, int R, int PRO>
struct TcCfg {
    static constexpr bool SPLIT = (PRO == TPRO_GATHER);
    static constexpr int CG_IN = SPLIT ? 1 : CIN / 8;
    static constexpr int KSTEPS3 = SPLIT ? 5 : 9 * (CIN / 16);
    static constexpr int A0_CHUNKS = CG_IN * (R + 2) * kSW;
    // 3x3 -> 1x1 intermediate as BF16 hi + lo parts: [row][part][channel group][pixel]
    static constexpr int A1_CHUNKS = R * 2 * (CMID / 8) * kTileM;
    // weights as BF16 hi + lo images (hi image first, then lo image)
    static constexpr int B3_IMG = KSTEPS3 * 2 * CMID;
    static constexpr int B1_IMG = (CMID / 8) * COUT;
    static constexpr int B3_CHUNKS = 2 * B3_IMG;
    static constexpr int B1_CHUNKS = 2 * B1_IMG;
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_A1 = OFF_A0 + A0_CHUNKS * 16;
    static constexpr int OFF_B3 = OFF_A1 + A1_CHUNKS * 16;
    static constexpr int OFF_B1 = OFF_B3 + B3_CHUNKS * 16;
    static constexpr int OFF_BIAS3 = OFF_B1 + B1_CHUNKS * 16;
    static constexpr int OFF_BIAS1 = OFF_BIAS3 + CMID * 4;
    static constexpr int OFF_HEAD = OFF_BIAS1 + COUT * 4;
    static constexpr int OFF_BAR = ((OFF_HEAD + (COUT + 1) * 4) + 15) / 16 * 16;
    static constexpr int BYTES_USED = OFF_BAR + 32;
    static constexpr int TMEM_COLS_RAW = R * CMID;
    static constexpr int TMEM_COLS = TMEM_COLS_RAW < 32 ? 32 : TMEM_COLS_RAW;
    // enough shared memory per CTA that the CTAs resident on one SM can never
    // ask for more than its 512 TMEM columns (228 KB of shared memory per SM)
    static constexpr int TMEM_CAP = 512 / TMEM_COLS;
    static constexpr int BYTES_MIN = (236 * 1024) / (TMEM_CAP + 1);
    static constexpr int BYTES = BYTES_USED < BYTES_MIN ? BYTES_MIN : BYTES_USED;
    static_assert(TMEM_COLS == 32 || TMEM_COLS == 64 || TMEM_COLS == 128 || TMEM_COLS == 256, "TMEM columns");
    static_assert(CMID % 16 == 0 && COUT % 16 == 0 && COUT <= CMID, "channel shapes");
    static_assert(BYTES_USED <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 ldg_v4(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// 8 BF16 values of a chunk -> FP32
__device__ __forceinline__ void chunk_to_f32(uint4 c, float (&f)[8]) {
    float2 a = unpack_bf16x2(c.x), b = unpack_bf16x2(c.y), d = unpack_bf16x2(c.z), e = unpack_bf16x2(c.w);
    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y; f[4] = d.x; f[5] = d.y; f[6] = e.x; f[7] = e.y;
}
__device__ __forceinline__ uint4 f32_to_chunk(const float* f) {
    return make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                      pack_bf16x2(f[6], f[7]));
}

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI>
__global__ void __launch_bounds__(kNT, 2) level_tc_kernel(const __grid_constant__ TcBatch a) {
    using C = TcCfg<CIN, CMID, COUT, R, PRO>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sA0 = sbase + C::OFF_A0, sA1 = sbase + C::OFF_A1;
    const uint32_t sB3 = sbase + C::OFF_B3, sB1 = sbase + C::OFF_B1;
    float* bias3_s = reinterpret_cast<float*>(smem + C::OFF_BIAS3);
    float* bias1_s = reinterpret_cast<float*>(smem + C::OFF_BIAS1);
    float* head_s = reinterpret_cast<float*>(smem + C::OFF_HEAD);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 8);
    int* s_abort = reinterpret_cast<int*>(smem + C::OFF_BAR + 12);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int wg = warp >> 2;          // warpgroup: splits the epilogue rows
    const int m = tid & 127;           // pixel of the row block = TMEM lane

    // ---- one-time set-up: weights, barrier, TMEM
    for (int i = tid; i < C::B3_CHUNKS; i += kNT) st_shared_v4(sB3 + 16 * i, __ldg(a.b3img + i));
    for (int i = tid; i < C::B1_CHUNKS; i += kNT) st_shared_v4(sB1 + 16 * i, __ldg(a.b1img + i));
    for (int i = tid; i < CMID; i += kNT) bias3_s[i] = __ldg(a.bias3 + i);
    for (int i = tid; i < COUT; i += kNT) bias1_s[i] = __ldg(a.bias1 + i);
    if (EPI == TEPI_HEAD)
        for (int i = tid; i <= COUT; i += kNT) head_s[i] = __ldg(a.head + i);
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 0) tmem_alloc(tslot, C::TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t tlane = tbase + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    uint32_t phase = 0;

    constexpr uint32_t kPlane = (R + 2) * kSW * 16;  // bytes between channel groups of A0
    const int ntiles = a.tile_start[a.nviews];
    int v = 0;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        while (tile >= a.tile_start[v + 1]) ++v;
        const TcJob& job = a.job[v];
        const int H = job.H, W = job.W;
        const int local = tile - a.tile_start[v];
        const int y0 = (local / job.tiles_x) * R;
        const int x0 = (local % job.tiles_x) * kTileM;

        // ---------------- prologue: stage the (R+2) x 130 input tile (zero padded)
        if constexpr (PRO == TPRO_GATHER) {
            // staged pixels -1 .. 129 of each row (129 = zero pad read by the dummy tap);
            // each thread gathers NPT of them in three batched phases so that its
            // G-buffer loads, then its shadow-map loads, are all in flight together
            constexpr int NSP = 131;
            constexpr int ITEMS = (R + 2) * NSP;
            constexpr int NPT = (ITEMS + kNT - 1) / kNT;
            const GatherParams& g = job.g;
            float4 P[NPT], Nv[NPT];
            bool ok[NPT];
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int idx = tid + kNT * k;
                const int sr = idx / NSP, sp = idx % NSP;
                const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
                ok[k] = idx < ITEMS && sp < 130 && gy >= 0 && gy < H && gx >= 0 && gx < W;
                if (ok[k]) {
                    const size_t p = static_cast<size_t>(gy) * W + gx;
                    P[k] = __ldg(g.pos4 + p);
                    Nv[k] = __ldg(g.nrm4 + p);
                }
            }
            float z[NPT];
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int tx = ok[k] ? texel_index(g, P[k].x, P[k].y, P[k].z) : -1;
                z[k] = g.z_far;
                if (tx >= 0) z[k] = __ldg(g.sm + tx);
            }
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int idx = tid + kNT * k;
                if (idx < ITEMS) {
                    const int sr = idx / NSP, sp = idx % NSP;
                    uint4 chunk = make_uint4(0, 0, 0, 0);
                    if (ok[k]) {
                        float f[4];
                        pixel_features(g, P[k], Nv[k], z[k], f);
                        float hl[8];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float hf = __bfloat162float(__float2bfloat16_rn(f[c]));
                            hl[c] = hf;
                            hl[4 + c] = f[c] - hf;
                        }
                        chunk = f32_to_chunk(hl);
                    }
                    st_shared_v4(sA0 + 16 * (sr * kSW + sp), chunk);
                }
            }
        } else if constexpr (PRO == TPRO_PLAIN) {
            constexpr int CG = CIN / 8;
#pragma unroll 4
            for (int idx = tid; idx < (R + 2) * 130 * CG; idx += kNT) {
                const int cg = idx % CG;
                const int t = idx / CG;
                const int sp = t % 130, sr = t / 130;
                const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                    val = ldg_v4(job.in + (static_cast<size_t>(gy) * W + gx) * CIN + cg * 8);
                st_shared_v4(sA0 + cg * kPlane + 16 * (sr * kSW + sp), val);
            }
        } else {  // UP_SKIP / UP
            constexpr int CG = CIN / 8;
            const int Hl = H / 2, Wl = W / 2;
#pragma unroll 2
            for (int idx = tid; idx < (R + 2) * 130 * CG; idx += kNT) {
                const int cg = idx % CG;
                const int t = idx / CG;
                const int sp = t % 130, sr = t / 130;
                const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const BilinTap ty = bilin_tap(gy, Hl), tx = bilin_tap(gx, Wl);
                    float p00[8], p01[8], p10[8], p11[8], o[8];
                    chunk_to_f32(ldg_v4(job.in + (static_cast<size_t>(ty.i0) * Wl + tx.i0) * CIN + cg * 8), p00);
                    chunk_to_f32(ldg_v4(job.in + (static_cast<size_t>(ty.i0) * Wl + tx.i1) * CIN + cg * 8), p01);
                    chunk_to_f32(ldg_v4(job.in + (static_cast<size_t>(ty.i1) * Wl + tx.i0) * CIN + cg * 8), p10);
                    chunk_to_f32(ldg_v4(job.in + (static_cast<size_t>(ty.i1) * Wl + tx.i1) * CIN + cg * 8), p11);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float r0 = p00[c] * tx.w0 + p01[c] * tx.w1;
                        const float r1 = p10[c] * tx.w0 + p11[c] * tx.w1;
                        o[c] = r0 * ty.w0 + r1 * ty.w1;
                    }
                    if constexpr (PRO == TPRO_UP_SKIP) {
                        float s[8];
                        chunk_to_f32(ldg_v4(job.skip + (static_cast<size_t>(gy) * W + gx) * CIN + cg * 8), s);
#pragma unroll
                        for (int c = 0; c < 8; ++c) o[c] += s[c];
                    }
                    val = f32_to_chunk(o);
                }
                st_shared_v4(sA0 + cg * kPlane + 16 * (sr * kSW + sp), val);
            }
        }
        fence_proxy_async_smem();
        fence_before_sync();
        __syncthreads();

        // ---------------- 3x3 convolution: R row blocks of 128 x CMID; each K step
        // twice, against the hi and the lo image of the weights
        if (tid == 0) {
            fence_after_sync();
            constexpr uint32_t id3 = idesc_bf16(128, CMID);
            constexpr uint32_t kB3lo = 16 * C::B3_IMG;  // byte offset of the lo image
            for (int r = 0; r < R; ++r) {
                const uint32_t d = tbase + r * CMID;
                if constexpr (C::SPLIT) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const int t0 = 2 * k, t1 = 2 * k + 1;
                        const uint32_t a0 = sA0 + 16 * ((r + t0 / 3) * kSW + t0 % 3);
                        const uint32_t lbo = (t1 < 9) ? 16 * ((r + t1 / 3) * kSW + t1 % 3) - 16 * ((r + t0 / 3) * kSW + t0 % 3) : 16;
                        const uint64_t ad = smem_desc(a0, lbo, 128);
                        const uint32_t b0 = sB3 + 16 * (k * 2 * CMID);
                        mma_bf16(d, ad, smem_desc(b0, CMID * 16, 128), id3, k > 0);
                        mma_bf16(d, ad, smem_desc(b0 + kB3lo, CMID * 16, 128), id3, 1);
                    }
                } else {
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                        for (int kk = 0; kk < CIN / 16; ++kk) {
                            const uint32_t a0 = sA0 + (2 * kk) * kPlane + 16 * ((r + tap / 3) * kSW + tap % 3);
                            const uint64_t ad = smem_desc(a0, kPlane, 128);
                            const uint32_t b0 = sB3 + 16 * ((tap * C::CG_IN + 2 * kk) * CMID);
                            mma_bf16(d, ad, smem_desc(b0, CMID * 16, 128), id3, (tap | kk) != 0);
                            mma_bf16(d, ad, smem_desc(b0 + kB3lo, CMID * 16, 128), id3, 1);
                        }
                    }
                }
            }
            mma_commit(mbar);
        }
        if (!mbar_wait_bounded(mbar, phase, kWaitNs)) {
            atomicExch(a.err, 1);
            *s_abort = 1;
        }
        phase ^= 1;
        __syncthreads();
        if (*s_abort) break;
        fence_after_sync();

        // ---------------- epilogue 1: bias + ReLU -> BF16 hi + lo -> A operand of the 1x1
        constexpr int kA1Part = (CMID / 8) * kTileM;  // chunks per part of one row
        for (int r = wg; r < R; r += 2) {
#pragma unroll
            for (int c0 = 0; c0 < CMID; c0 += 16) {
                float val[16], lo[16];
                tmem_ld16(tlane + r * CMID + c0, val);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    val[j] = fmaxf(val[j] + bias3_s[c0 + j], 0.f);
                    const float hi = __bfloat162float(__float2bfloat16_rn(val[j]));
                    lo[j] = val[j] - hi;
                    val[j] = hi;
                }
                const int cg = c0 / 8;
                const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
                st_shared_v4(row + 16 * (cg * kTileM + m), f32_to_chunk(val));
                st_shared_v4(row + 16 * ((cg + 1) * kTileM + m), f32_to_chunk(val + 8));
                st_shared_v4(row + 16 * (kA1Part + cg * kTileM + m), f32_to_chunk(lo));
                st_shared_v4(row + 16 * (kA1Part + (cg + 1) * kTileM + m), f32_to_chunk(lo + 8));
            }
        }
        fence_proxy_async_smem();
        fence_before_sync();
        __syncthreads();

        // ---------------- 1x1 convolution into the same TMEM columns:
        // A_hi B_hi + A_hi B_lo + A_lo B_hi per K step
        if (tid == 0) {
            fence_after_sync();
            constexpr uint32_t id1 = idesc_bf16(128, COUT);
            constexpr uint32_t kB1lo = 16 * C::B1_IMG;
            for (int r = 0; r < R; ++r) {
                const uint32_t row = sA1 + 16 * (r * 2 * kA1Part);
#pragma unroll
                for (int kk = 0; kk < CMID / 16; ++kk) {
                    const uint64_t ahi = smem_desc(row + 16 * (2 * kk * kTileM), kTileM * 16, 128);
                    const uint64_t alo = smem_desc(row + 16 * (kA1Part + 2 * kk * kTileM), kTileM * 16, 128);
                    const uint32_t b0 = sB1 + 16 * (2 * kk * COUT);
                    const uint64_t bhi = smem_desc(b0, COUT * 16, 128);
                    const uint64_t blo = smem_desc(b0 + kB1lo, COUT * 16, 128);
                    mma_bf16(tbase + r * CMID, ahi, bhi, id1, kk > 0);
                    mma_bf16(tbase + r * CMID, ahi, blo, id1, 1);
                    mma_bf16(tbase + r * CMID, alo, bhi, id1, 1);
                }
            }
            mma_commit(mbar);
        }
        if (!mbar_wait_bounded(mbar, phase, kWaitNs)) {
            atomicExch(a.err, 2);
            *s_abort = 1;
        }
        phase ^= 1;
        __syncthreads();
        if (*s_abort) break;
        fence_after_sync();

        // ---------------- epilogue 2
        const int ox = x0 + m;
        if constexpr (EPI == TEPI_POOL || EPI == TEPI_SKIP_POOL) {
            for (int r = 2 * wg; r < R; r += 4) {  // row pairs (r, r + 1), alternating warpgroups
                float s[COUT];
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float v0[16], v1[16];
                    tmem_ld16(tlane + r * CMID + c0, v0);
                    tmem_ld16(tlane + (r + 1) * CMID + c0, v1);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v0[j] = fmaxf(v0[j] + bias1_s[c0 + j], 0.f);
                        v1[j] = fmaxf(v1[j] + bias1_s[c0 + j], 0.f);
                        s[c0 + j] = v0[j] + v1[j];
                    }
                    if constexpr (EPI == TEPI_SKIP_POOL) {
                        const int oy = y0 + r;
                        if (oy < H && ox < W) {
                            uint16_t* dst = job.out_skip + (static_cast<size_t>(oy) * W + ox) * COUT + c0;
                            reinterpret_cast<uint4*>(dst)[0] = f32_to_chunk(v0);
                            reinterpret_cast<uint4*>(dst)[1] = f32_to_chunk(v0 + 8);
                            dst += static_cast<size_t>(W) * COUT;
                            reinterpret_cast<uint4*>(dst)[0] = f32_to_chunk(v1);
                            reinterpret_cast<uint4*>(dst)[1] = f32_to_chunk(v1 + 8);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < COUT; ++c) s[c] = 0.25f * (s[c] + __shfl_xor_sync(0xffffffffu, s[c], 1));
                const int oy = y0 + r;
                if (oy < H && ox < W) {
                    // even pixel writes the first half of the channels, odd the second
                    const int half = (m & 1) * (COUT / 2);
                    uint16_t* dst = job.out + (static_cast<size_t>(oy / 2) * (W / 2) + ox / 2) * COUT + half;
#pragma unroll
                    for (int c = 0; c < COUT / 2; c += 8) {
                        float t8[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) t8[j] = s[half + c + j];
                        reinterpret_cast<uint4*>(dst + c)[0] = f32_to_chunk(t8);
                    }
                }
            }
        } else {
            for (int r = wg; r < R; r += 2) {
                const int oy = y0 + r;
                float hsum = 0.f;
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float val[16];
                    tmem_ld16(tlane + r * CMID + c0, val);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) val[j] = fmaxf(val[j] + bias1_s[c0 + j], 0.f);
                    if constexpr (EPI == TEPI_STORE) {
                        if (oy < H && ox < W) {
                            uint16_t* dst = job.out + (static_cast<size_t>(oy) * W + ox) * COUT + c0;
                            reinterpret_cast<uint4*>(dst)[0] = f32_to_chunk(val);
                            reinterpret_cast<uint4*>(dst)[1] = f32_to_chunk(val + 8);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) hsum = fmaf(head_s[c0 + j], val[j], hsum);
                    }
                }
                if (EPI == TEPI_HEAD && oy < H && ox < W)
                    job.vis[static_cast<size_t>(oy) * W + ox] = sigmoidf_acc(hsum + head_s[COUT]);
            }
        }
        fence_before_sync();
        __syncthreads();  // TMEM columns, A0 and A1 are free for the next tile
    }

    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, C::TMEM_COLS);
}

// ------------------------------------------------------------------ variants and launch
template <int CIN, int CMID, int COUT, int R, int PRO, int EPI>
static cudaError_t launch_variant(const TcBatch& a, int ctas_per_sm, cudaStream_t stream) {
    using C = TcCfg<CIN, CMID, COUT, R, PRO>;
    auto kern = level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI>;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::BYTES);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the kernel's own resources: registers,
        // shared memory (228 KB per SM, 1 KB reserved per CTA) and TMEM columns
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int regs = ((fa.numRegs + 7) / 8) * 8 * kNT;
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
    kern<<<grid, kNT, C::BYTES, stream>>>(a);
    return cudaGetLastError();
}

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI>
static const void* kernel_of() {
    return reinterpret_cast<const void*>(level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI>);
}

template <int CIN, int CMID, int COUT, int R, int PRO, int EPI>
static int occupancy_of() {
    using C = TcCfg<CIN, CMID, COUT, R, PRO>;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, level_tc_kernel<CIN, CMID, COUT, R, PRO, EPI>) != cudaSuccess) return 1;
    const int regs = ((fa.numRegs + 7) / 8) * 8 * kNT;
    const int by_regs = regs > 0 ? 65536 / regs : 8;
    const int by_smem = (228 * 1024) / (C::BYTES + 1024);
    int o = by_regs < by_smem ? by_regs : by_smem;
    if (o > C::TMEM_CAP) o = C::TMEM_CAP;
    if (o > 8) o = 8;
    return o < 1 ? 1 : o;
}

// Variant tables: the tile height R of every stage (the autotuner's search space).
using LaunchFn = cudaError_t (*)(const TcBatch&, int, cudaStream_t);
struct Variant { int R; LaunchFn fn; const void* (*func)(); int (*occ)(); };
#define NSM_VARIANT(R_, ...) {R_, launch_variant<__VA_ARGS__>, kernel_of<__VA_ARGS__>, occupancy_of<__VA_ARGS__>}

static const Variant kVarEnc0[] = {
    NSM_VARIANT(2, 4, 16, 16, 2, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT(4, 4, 16, 16, 4, TPRO_GATHER, TEPI_POOL),
    NSM_VARIANT(8, 4, 16, 16, 8, TPRO_GATHER, TEPI_POOL)};
static const Variant kVarEnc1[] = {
    NSM_VARIANT(2, 16, 32, 32, 2, TPRO_PLAIN, TEPI_SKIP_POOL),
    NSM_VARIANT(4, 16, 32, 32, 4, TPRO_PLAIN, TEPI_SKIP_POOL)};
static const Variant kVarBott[] = {
    NSM_VARIANT(1, 32, 64, 32, 1, TPRO_PLAIN, TEPI_STORE),
    NSM_VARIANT(2, 32, 64, 32, 2, TPRO_PLAIN, TEPI_STORE)};
static const Variant kVarDec1[] = {
    NSM_VARIANT(2, 32, 32, 16, 2, TPRO_UP_SKIP, TEPI_STORE),
    NSM_VARIANT(4, 32, 32, 16, 4, TPRO_UP_SKIP, TEPI_STORE)};
static const Variant kVarDec0[] = {
    NSM_VARIANT(2, 16, 16, 16, 2, TPRO_UP, TEPI_HEAD),
    NSM_VARIANT(4, 16, 16, 16, 4, TPRO_UP, TEPI_HEAD),
    NSM_VARIANT(8, 16, 16, 16, 8, TPRO_UP, TEPI_HEAD)};

struct StageTable { const Variant* v; int n; };
static const StageTable kStages[kTcStages] = {
    {kVarEnc0, 3}, {kVarEnc1, 2}, {kVarBott, 2}, {kVarDec1, 2}, {kVarDec0, 3}};

int tc_stage_variants(int stage) { return (stage >= 0 && stage < kTcStages) ? kStages[stage].n : 0; }
int tc_stage_rows(int stage, int variant) { return kStages[stage].v[variant].R; }
const void* tc_stage_kernel(int stage, int variant) { return kStages[stage].v[variant].func(); }
int tc_stage_occupancy(int stage, int variant) { return kStages[stage].v[variant].occ(); }

int tc_default_variant(int stage) {
    // R = 4 for the full-resolution stages, the smaller tiles for the others
    static const int def[kTcStages] = {1, 1, 1, 0, 1};
    return def[stage];
}

// Fill the tile table of a stage for the given tile height.
static void fill_tiles(TcBatch& b, int rows) {
    b.tile_start[0] = 0;
    for (int i = 0; i < b.nviews; ++i) {
        TcJob& j = b.job[i];
        j.tiles_x = (j.W + kTileM - 1) / kTileM;
        const int ty = (j.H + rows - 1) / rows;
        b.tile_start[i + 1] = b.tile_start[i] + j.tiles_x * ty;
    }
}

cudaError_t tc_launch_stage(int stage, int variant, TcBatch& b, int ctas_per_sm, cudaStream_t stream) {
    if (stage < 0 || stage >= kTcStages || variant < 0 || variant >= kStages[stage].n) return cudaErrorInvalidValue;
    const Variant& v = kStages[stage].v[variant];
    fill_tiles(b, v.R);
    return v.fn(b, ctas_per_sm, stream);
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
        b.err = err;
        for (int i = 0; i < n; ++i) {
            TcJob& j = b.job[i];
            j.g = g[i];
            const int H = g[i].H, W = g[i].W;
            const Activations& A = act[i];
            switch (s) {
                case 0: j.H = H; j.W = W; j.out = static_cast<uint16_t*>(A.e0); break;
                case 1: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(A.e0);
                        j.out_skip = static_cast<uint16_t*>(A.s1); j.out = static_cast<uint16_t*>(A.p1); break;
                case 2: j.H = H / 4; j.W = W / 4; j.in = static_cast<const uint16_t*>(A.p1);
                        j.out = static_cast<uint16_t*>(A.bo); break;
                case 3: j.H = H / 2; j.W = W / 2; j.in = static_cast<const uint16_t*>(A.bo);
                        j.skip = static_cast<const uint16_t*>(A.s1); j.out = static_cast<uint16_t*>(A.d1); break;
                default: j.H = H; j.W = W; j.in = static_cast<const uint16_t*>(A.d1); j.vis = vis[i]; break;
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

}  // namespace nsm
