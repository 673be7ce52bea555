// FP8 (E4M3) tensor-core form of the compact encoder/decoder (Sec. 3.5):
// the stage structure of the BF16 form (net_bf16.cu: persistent
// warp-specialised kernels, one per level, producers -> MMA warp -> TMEM ->
// epilogue, row-stacked 3x3, ring of staged rows) with
// tcgen05.mma.kind::f8f6f4 (E4M3 x E4M3, FP32 accumulation in TMEM).
//
//   weights      E4M3 with one scale per output channel, s_o = max|W[o]| / 448
//                (pack_fp8.cu); the epilogue computes acc * s_o + bias
//   activations  E4M3 with unit scale (saturating at +-448): the staged
//                inputs, the 3x3 -> 1x1 intermediate and every tensor stored
//                between stages ([pixel][C], 1 byte per channel)
//   features     computed in FP32 (texel index and depth test as in every
//                form), then E4M3
//
// A K = 32 MMA step reads two 16-byte chunks of 16 E4M3 values:
//   C_in = 16    staged pixels m + 2p and m + 2p + 1 (p = 0, 1; the kx = 3
//                weights are zero and the pad pixels of every staged row are
//                kept zero)
//   C_in = 32    the two channel-group planes of staged pixel m + kx
//   first level  one "triplet" chunk per staged pixel m holding the four
//                features of staged pixels m, m+1, m+2 (all three kx taps)
//                and a chunk of a plane that stays zero
// The kernel rows ky are stacked along N (3 C_mid <= 192), so one MMA per
// (staged row, K step) feeds up to three output rows, as in the BF16 form.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "nsm_internal.h"
#include "tc_pipeline.cuh"
#include "tc_stage.h"

namespace nsm {

template <int CIN, int CMID, int COUT, int R, int PRO>
struct F8Cfg {
    static constexpr bool SPLIT = (PRO == TPRO_GATHER);
    static constexpr bool UP = (PRO == TPRO_UP || PRO == TPRO_UP_SKIP);
    static constexpr int CG = SPLIT ? 1 : CIN / 16;               // 16-channel chunks per staged pixel
    static constexpr int PLN = SPLIT ? 2 : CG;                    // first level: triplet plane + zero plane
    static constexpr int NRW = 2 * (R + 2);                       // ring of staged rows per plane
    static constexpr uint32_t PLANE = NRW * kSW * 16;
    static constexpr int MP = CMID / 16, MPP = (MP + 1) / 2 * 2;  // intermediate planes (even: zero pad plane)
    static constexpr int A1_BYTES = R * MPP * kTileM * 16;        // [row][plane][pixel]
    static constexpr int NCR = R / 2 + 2;
    static constexpr int RAW_BYTES = SPLIT ? (R + 2) * 130 * 32 : (UP ? NCR * kNCC * (CG + 1) * 16 : 0);
    static constexpr int N3 = CMID, N1 = COUT;
    static constexpr int B3_CHUNKS = (SPLIT ? 6 : (CG == 1 ? 12 : 18)) * N3;
    static constexpr int B1_CHUNKS = MPP * N1;
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_A1 = OFF_A0 + PLN * PLANE;
    static constexpr int OFF_RAW = OFF_A1 + A1_BYTES;             // two raw buffers
    static constexpr int OFF_B3 = OFF_RAW + 2 * RAW_BYTES;
    static constexpr int OFF_B1 = OFF_B3 + B3_CHUNKS * 16;
    static constexpr int OFF_BIAS3 = OFF_B1 + B1_CHUNKS * 16;
    static constexpr int OFF_S3 = OFF_BIAS3 + CMID * 4;
    static constexpr int OFF_BIAS1 = OFF_S3 + CMID * 4;
    static constexpr int OFF_S1 = OFF_BIAS1 + COUT * 4;
    static constexpr int OFF_HEAD = OFF_S1 + COUT * 4;
    static constexpr int OFF_ZERO = ((OFF_HEAD + (COUT + 1) * 4) + 127) / 128 * 128;
    static constexpr int ZERO_BYTES = 256 * 16 + 128;  // zero A and B operands of the clearing MMA
    static constexpr int OFF_BAR = OFF_ZERO + ZERO_BYTES;
    static constexpr int BYTES_USED = OFF_BAR + 128;
    static constexpr int TMEM_BUF = R * N3;
    static constexpr int TMEM_COLS = 2 * TMEM_BUF < 32 ? 32 : 2 * TMEM_BUF;
    static constexpr int TMEM_CAP = 512 / TMEM_COLS;
    static constexpr int BYTES_MIN = (236 * 1024) / (TMEM_CAP + 1);
    static constexpr int BYTES = BYTES_USED < BYTES_MIN ? BYTES_MIN : BYTES_USED;
    static_assert(SPLIT ? CIN == 4 : (CIN == 16 || CIN == 32), "input widths of the FP8 stages");
    static_assert(CMID % 16 == 0 && COUT % 16 == 0 && 3 * N3 <= 256 && R * N3 <= 256, "channel shapes");
    static_assert(TMEM_COLS == 32 || TMEM_COLS == 64 || TMEM_COLS == 128 || TMEM_COLS == 256 || TMEM_COLS == 512,
                  "TMEM columns");
    static_assert(!UP || (R % 2 == 0), "up-sampling stages need an even tile height");
    static_assert(BYTES_USED <= 227 * 1024, "shared memory");
};

// ------------------------------------------------------------------ E4M3 conversions
__device__ __forceinline__ uint32_t pack4_e4m3(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}
__device__ __forceinline__ uint4 pack16_e4m3(const float* f) {
    return make_uint4(pack4_e4m3(f[0], f[1], f[2], f[3]), pack4_e4m3(f[4], f[5], f[6], f[7]),
                      pack4_e4m3(f[8], f[9], f[10], f[11]), pack4_e4m3(f[12], f[13], f[14], f[15]));
}
__device__ __forceinline__ float2 e4m3x2_to_f32(uint32_t bits16) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(bits16), __NV_E4M3);
    return __half22float2(__half2(h));
}
__device__ __forceinline__ void unpack16_e4m3(uint4 c, float (&f)[16]) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 a = e4m3x2_to_f32(w[k] & 0xFFFFu), b = e4m3x2_to_f32(w[k] >> 16);
        f[4 * k] = a.x; f[4 * k + 1] = a.y; f[4 * k + 2] = b.x; f[4 * k + 3] = b.y;
    }
}
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
}

// ------------------------------------------------------------------ producer pieces
// (staged rows y0-1 .. y0+R, pixels x0-1 .. x0+128; staged row sr of a tile in
// ring slot (base + sr) mod NRW; a producer call writes staged rows [first, R + 2))

// PLAIN: the E4M3 chunks of the tile straight into the ring, zeros outside the image
template <int NP, int CIN, int R, int NRW>
__device__ __forceinline__ void f8_copy(const uint8_t* src, int H, int W, int y0, int x0, uint32_t a0, int base,
                                        int first, int pt) {
    constexpr int CG = CIN / 16;
    constexpr uint32_t kPlane = NRW * kSW * 16;
    for (int ci = pt; ci < 130 * CG; ci += NP) {
        const int pl = ci % CG, sp = ci / CG;
        const int gx = x0 - 1 + sp;
        const bool okx = gx >= 0 && gx < W;
        const uint32_t dst = a0 + pl * kPlane + 16 * sp;
#pragma unroll 2
        for (int sr = first; sr < R + 2; ++sr) {
            const int gy = y0 - 1 + sr;
            const bool ok = okx && gy >= 0 && gy < H;
            const uint8_t* p = ok ? src + ((static_cast<size_t>(gy) * W + gx) * CG + pl) * 16 : src;
            cp_async16(dst + 16 * (row_slot<NRW>(base, sr) * kSW), p, ok ? 16u : 0u);
        }
    }
}

// GATHER raw: pos4 / nrm4 of the staged pixels in bounds, [part][staged row][pixel]
template <int NP, int R>
__device__ __forceinline__ void f8_prefetch_gbuffer(const TcJob& job, int y0, int x0, uint32_t raw, int first, int pt) {
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

// UP raw: the E4M3 coarse rows y0/2-1 .. y0/2+R/2 and columns x0/2-1 .. x0/2+64
// in bounds, pixels CIN / 16 + 1 chunks apart
template <int NP, int CIN, int R>
__device__ __forceinline__ void f8_prefetch_coarse(const TcJob& job, int y0, int x0, uint32_t raw, int pt) {
    constexpr int CG = CIN / 16, NCR = R / 2 + 2;
    const int Hl = job.H / 2, Wl = job.W / 2;
    const int cy0 = y0 / 2 - 1, cx0 = x0 / 2 - 1;
    for (int idx = pt; idx < NCR * kNCC * CG; idx += NP) {
        const int ch = idx % CG, q = idx / CG;
        const int gy = cy0 + q / kNCC, gx = cx0 + q % kNCC;
        if (gy >= 0 && gy < Hl && gx >= 0 && gx < Wl)
            cp_async16(raw + 16 * (q * (CG + 1) + ch), job.in8 + ((static_cast<size_t>(gy) * Wl + gx) * CG + ch) * 16, 16);
    }
}

// GATHER compute: features in FP32 (texel fetches of a thread in flight
// together) -> E4M3 -> the triplet chunks: the 4 bytes of staged pixel sp go to
// bytes 0-3 of chunk sp, 4-7 of chunk sp - 1 and 8-11 of chunk sp - 2; chunk
// sp's bytes 12-15 are written as zeros with its bytes 0-3.
template <int NP, int R, int NRW>
__device__ __forceinline__ void f8_compute_gather(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0,
                                                  int base, int first, int pt) {
    constexpr int NSP = 130;
    constexpr int NPT = ((R + 2) * NSP + NP - 1) / NP;
    const int ITEMS = (R + 2 - first) * NSP;
    const GatherParams g = job.g;
    const int H = job.H, W = job.W;
    float4 P[NPT], Nv[NPT];
    float z[NPT];
    bool ok[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = pt + NP * k;
        const int sr = first + idx / NSP, sp = idx % NSP;
        const int gy = y0 - 1 + sr, gx = x0 - 1 + sp;
        ok[k] = idx < ITEMS && gy >= 0 && gy < H && gx >= 0 && gx < W;
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
            uint32_t word = 0;
            if (ok[k]) {
                float f[4];
                pixel_features(g, P[k], Nv[k], z[k], f);
                word = pack4_e4m3(f[0], f[1], f[2], f[3]);
            }
            const uint32_t row = a0 + 16 * (row_slot<NRW>(base, sr) * kSW);
            if (sp < kTileM) {
                st_shared_u32(row + 16 * sp, word);
                st_shared_u32(row + 16 * sp + 12, 0u);
            }
            if (sp >= 1 && sp - 1 < kTileM) st_shared_u32(row + 16 * (sp - 1) + 4, word);
            if (sp >= 2 && sp - 2 < kTileM) st_shared_u32(row + 16 * (sp - 2) + 8, word);
        }
    }
}

// UP / UP_SKIP compute: bilinear x2 of the E4M3 coarse rows in FP32 (+ the
// E4M3 skip from global memory) -> E4M3 chunks of plane g.  Separable, two
// coarse rows live at a time (as in the BF16 form).
template <int CIN, int R, bool SKIP, int NROWS, int NRW>
__device__ __forceinline__ void f8_up_column(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0, int sp,
                                             int g, int sr0, int base) {
    constexpr int CG = CIN / 16;
    constexpr uint32_t kPlane = NRW * kSW * 16;
    const int H = job.H, W = job.W, Hl = H / 2, Wl = W / 2;
    const int cy0 = y0 / 2 - 1, cx0 = x0 / 2 - 1;
    const int gx = x0 - 1 + sp;
    const bool okx = gx >= 0 && gx < W;
    const BilinTap tx = bilin_tap(okx ? gx : 0, Wl);
    const uint32_t c0 = raw + 16 * ((tx.i0 - cx0) * (CG + 1) + g);
    const uint32_t c1 = raw + 16 * ((tx.i1 - cx0) * (CG + 1) + g);
    const uint32_t dst = a0 + g * kPlane + 16 * sp;
    uint4 sk[NROWS];
    if constexpr (SKIP) {
#pragma unroll
        for (int k = 0; k < NROWS; ++k) {
            const int gy = y0 - 1 + sr0 + k;
            sk[k] = make_uint4(0, 0, 0, 0);
            if (okx && gy >= 0 && gy < H)
                sk[k] = __ldg(reinterpret_cast<const uint4*>(job.skip8 + (static_cast<size_t>(gy) * W + gx) * CIN) + g);
        }
    }
    auto hrow = [&](int ci, float (&h)[16]) {
        const uint32_t ro = 16 * ((ci - cy0) * kNCC * (CG + 1));
        float p0[16], p1[16];
        unpack16_e4m3(ld_shared_v4(c0 + ro), p0);
        unpack16_e4m3(ld_shared_v4(c1 + ro), p1);
#pragma unroll
        for (int c = 0; c < 16; ++c) h[c] = p0[c] * tx.w0 + p1[c] * tx.w1;
    };
    int ia = -4, ib = -4;
    float ha[16], hb[16];
#pragma unroll
    for (int k = 0; k < NROWS; ++k) {
        const int sr = sr0 + k;
        const int gy = y0 - 1 + sr;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (okx && gy >= 0 && gy < H) {
            const BilinTap ty = bilin_tap(gy, Hl);
            if (ty.i0 != ia) {
                if (ty.i0 == ib) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) ha[c] = hb[c];
                } else {
                    hrow(ty.i0, ha);
                }
                ia = ty.i0;
                ib = ia;
            }
            if (ty.i1 != ia && ty.i1 != ib) {
                hrow(ty.i1, hb);
                ib = ty.i1;
            }
            const bool same = ty.i1 == ia;
            float o[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) o[c] = ha[c] * ty.w0 + (same ? ha[c] : hb[c]) * ty.w1;
            if constexpr (SKIP) {
                float s[16];
                unpack16_e4m3(sk[k], s);
#pragma unroll
                for (int c = 0; c < 16; ++c) o[c] += s[c];
            }
            v = pack16_e4m3(o);
        }
        st_shared_v4(dst + 16 * (row_slot<NRW>(base, sr) * kSW), v);
    }
}

template <int NP, int CIN, int R, bool SKIP, int NRW>
__device__ __forceinline__ void f8_compute_up(const TcJob& job, int y0, int x0, uint32_t raw, uint32_t a0, int base,
                                              int first, int pt) {
    constexpr int CG = CIN / 16;
    constexpr int MAIN = kTileM * CG;
    const int nrows = R + 2 - first;
    for (int i = pt; i < MAIN; i += NP) {
        if (first == 0)
            f8_up_column<CIN, R, SKIP, R + 2, NRW>(job, y0, x0, raw, a0, 1 + i % kTileM, i / kTileM, 0, base);
        else
            f8_up_column<CIN, R, SKIP, R, NRW>(job, y0, x0, raw, a0, 1 + i % kTileM, i / kTileM, 2, base);
    }
    for (int i = pt; i < 2 * CG * nrows; i += NP) {
        const int sr = first + i % nrows, q = i / nrows;
        f8_up_column<CIN, R, SKIP, 1, NRW>(job, y0, x0, raw, a0, (q / CG) ? 129 : 0, q % CG, sr, base);
    }
}

// ------------------------------------------------------------------ stage kernel
template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW>
__global__ void __launch_bounds__(32 * (NEW + NPW + 1), 1) level_f8_kernel(const __grid_constant__ TcBatch a) {
    using C = F8Cfg<CIN, CMID, COUT, R, PRO>;
    constexpr int NP = 32 * NPW, NT = 32 * (NEW + NPW + 1), MW = NEW + NPW, NE = 32 * NEW;
    static_assert(NEW == 4 || NEW == 8, "epilogue warps cover the four TMEM lane quarters");
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sA0 = sbase + C::OFF_A0, sA1 = sbase + C::OFF_A1, sRAW = sbase + C::OFF_RAW;
    const uint32_t sB3 = sbase + C::OFF_B3, sB1 = sbase + C::OFF_B1;
    float* bias3_s = reinterpret_cast<float*>(smem + C::OFF_BIAS3);
    float* s3_s = reinterpret_cast<float*>(smem + C::OFF_S3);
    float* bias1_s = reinterpret_cast<float*>(smem + C::OFF_BIAS1);
    float* s1_s = reinterpret_cast<float*>(smem + C::OFF_S1);
    float* head_s = reinterpret_cast<float*>(smem + C::OFF_HEAD);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint64_t* full = bar;          // [2]
    uint64_t* mma3 = bar + 2;      // [2]
    uint64_t* tfree = bar + 4;     // [2]
    uint64_t* a1full = bar + 6;
    uint64_t* mma1 = bar + 7;
    uint64_t* gfull = bar + 8;     // [2]
    uint64_t* rfree = bar + 10;    // [2]
    uint64_t* accf = bar + 12;     // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 112);
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + 116);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    // ---- one-time set-up: zero the input ring and the 1x1 operand (pad pixels,
    // the first level's zero plane and the pad plane stay zero), weights, barriers, TMEM
    for (int i = tid; i < (C::OFF_RAW - C::OFF_A0) / 16; i += NT) st_shared_v4(sA0 + 16 * i, make_uint4(0, 0, 0, 0));
    for (int i = tid; i < C::B3_CHUNKS; i += NT) st_shared_v4(sB3 + 16 * i, __ldg(a.b3img + i));
    for (int i = tid; i < C::B1_CHUNKS; i += NT) st_shared_v4(sB1 + 16 * i, __ldg(a.b1img + i));
    for (int i = tid; i < CMID; i += NT) { bias3_s[i] = __ldg(a.bias3 + i); s3_s[i] = __ldg(a.scale3 + i); }
    for (int i = tid; i < COUT; i += NT) { bias1_s[i] = __ldg(a.bias1 + i); s1_s[i] = __ldg(a.scale1 + i); }
    if (EPI == TEPI_HEAD)
        for (int i = tid; i <= COUT; i += NT) head_s[i] = __ldg(a.head + i);
    for (int i = tid; i < C::ZERO_BYTES / 16; i += NT) st_shared_v4(sbase + C::OFF_ZERO + 16 * i, make_uint4(0, 0, 0, 0));
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(full + k, NP);
            mbar_init(mma3 + k, 1);
            mbar_init(tfree + k, NE);
            mbar_init(gfull + k, NP);
            mbar_init(rfree + k, NP);
            mbar_init(accf + k, 1);
        }
        mbar_init(a1full, NE);
        mbar_init(mma1, 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == MW) tmem_alloc(tslot, C::TMEM_COLS);
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;
    const long long ntl = a.tile_start[a.nviews];
    const int t_lo = static_cast<int>(ntl * blockIdx.x / gridDim.x);
    const int t_hi = static_cast<int>(ntl * (blockIdx.x + 1) / gridDim.x);
    auto locate = [&](int tile, int& v, int& y0, int& x0, bool& cont) -> const TcJob& {
        while (tile >= a.tile_start[v + 1]) ++v;
        const TcJob& job = a.job[v];
        const int local = tile - a.tile_start[v];
        const int ys = local % job.tiles_y;
        y0 = ys * R;
        x0 = (local / job.tiles_y) * kTileM;
        cont = tile > t_lo && ys > 0;
        return job;
    };
    auto ring_next = [&](bool cont, int& ring, int& base, int& first) {
        first = cont ? 2 : 0;
        base = cont ? (ring >= 2 ? ring - 2 : ring - 2 + C::NRW) : ring;
        ring = base + R + 2;
        if (ring >= C::NRW) ring -= C::NRW;
    };

    if (warp >= NEW && warp < MW) {
        // ================= producers: tile it fills its new rows of the ring
        const int pt = tid - NE;
        int v = 0, vn = 0, it = 0, ring = 0;
        if constexpr (PRO != TPRO_PLAIN) {
            if (t_lo < t_hi) {
                int y0, x0;
                bool cont;
                const TcJob& job = locate(t_lo, vn, y0, x0, cont);
                if constexpr (PRO == TPRO_GATHER) f8_prefetch_gbuffer<NP, R>(job, y0, x0, sRAW, 0, pt);
                else f8_prefetch_coarse<NP, CIN, R>(job, y0, x0, sRAW, pt);
                cp_async_arrive(gfull + 0);
            }
        }
        bool failed = false;
        for (int tile = t_lo; tile < t_hi && !failed; ++tile, ++it) {
            int y0, x0, base, first;
            bool cont;
            const TcJob& job = locate(tile, v, y0, x0, cont);
            ring_next(cont, ring, base, first);
            const int rb = it & 1, b = it & 1;
            if constexpr (PRO != TPRO_PLAIN) {
                const int next = tile + 1;
                if (next < t_hi) {
                    const int nb = rb ^ 1;
                    const int un = (it + 1) >> 1;
                    if (un >= 1 && !wait_phase(rfree + nb, (un - 1) & 1, s_abort)) { failed = true; break; }
                    int ny0, nx0;
                    bool ncont;
                    const TcJob& nj = locate(next, vn, ny0, nx0, ncont);
                    const uint32_t nraw = sRAW + nb * C::RAW_BYTES;
                    if constexpr (PRO == TPRO_GATHER) f8_prefetch_gbuffer<NP, R>(nj, ny0, nx0, nraw, ncont ? 2 : 0, pt);
                    else f8_prefetch_coarse<NP, CIN, R>(nj, ny0, nx0, nraw, pt);
                    cp_async_arrive(gfull + nb);
                }
                if (!wait_phase(gfull + rb, (it >> 1) & 1, s_abort)) { failed = true; break; }
            }
            // the rows written now are free once the MMAs of tile it - 2 are done
            if (it >= 2 && !wait_phase(mma3 + b, ((it >> 1) - 1) & 1, s_abort)) { failed = true; break; }
            const uint32_t raw = sRAW + rb * C::RAW_BYTES;
            if constexpr (PRO == TPRO_PLAIN) {
                f8_copy<NP, CIN, R, C::NRW>(job.in8, job.H, job.W, y0, x0, sA0, base, first, pt);
                cp_async_arrive(full + b);
            } else {
                if constexpr (PRO == TPRO_GATHER) f8_compute_gather<NP, R, C::NRW>(job, y0, x0, raw, sA0, base, first, pt);
                else f8_compute_up<NP, CIN, R, PRO == TPRO_UP_SKIP, C::NRW>(job, y0, x0, raw, sA0, base, first, pt);
                fence_proxy_async_smem();
                mbar_arrive(full + b);
                mbar_arrive(rfree + rb);
            }
        }
        if (failed) {
            atomicExch(a.err, 3);
            *s_abort = 1;
        }
    } else if (warp == MW) {
        // ================= MMA issuer
        if ((tid & 31) == 0) {
            constexpr uint32_t id1 = idesc_e4m3(128, C::N1);
            int it = 0, v = 0, ring = 0;
            bool failed = false;
            for (int tile = t_lo; tile < t_hi; ++tile, ++it) {
                int y0, x0, rbase, first;
                bool cont;
                locate(tile, v, y0, x0, cont);
                ring_next(cont, ring, rbase, first);
                const int tb = it & 1, b = it & 1;
                const uint32_t D = tbase + tb * C::TMEM_BUF;
                if (!wait_phase(full + b, (it >> 1) & 1, s_abort) ||
                    (it >= 2 && !wait_phase(tfree + tb, ((it >> 1) - 1) & 1, s_abort))) {
                    failed = true;
                    break;
                }
                fence_proxy_async_smem();
                fence_after_sync();
                // clear the accumulators (zero A and B operands), then per staged row
                // j one MMA per K step of width (#ky) x C_mid into output rows j - ky
                mma_e4m3(D, smem_desc(sbase + C::OFF_ZERO, 16, 128), smem_desc(sbase + C::OFF_ZERO, 16, 128),
                         idesc_e4m3(128, R * C::N3), 0);
                const uint64_t bdesc = smem_desc(sB3, 3 * C::N3 * 16, 128);
#pragma unroll
                for (int j = 0; j < R + 2; ++j) {
                    const int ka = j - (R - 1) > 0 ? j - (R - 1) : 0, kb = j < 2 ? j : 2;
                    const uint32_t id = idesc_e4m3(128, (kb - ka + 1) * C::N3);
                    const uint32_t d = D + (R - 1 - j + ka) * C::N3;
                    const uint32_t row = sA0 + 16 * (row_slot<C::NRW>(rbase, j) * kSW);
                    if constexpr (C::SPLIT) {
                        // triplet chunk of plane 0 + the zero plane
                        mma_e4m3(d, smem_desc(row, C::PLANE, 128), bdesc + ka * C::N3, id, 1);
                    } else if constexpr (C::CG == 1) {
                        // staged pixels (m + 2p, m + 2p + 1)
                        const uint64_t adesc = smem_desc(row, 16, 128);
#pragma unroll
                        for (int p2 = 0; p2 < 2; ++p2)
                            mma_e4m3(d, adesc + 2 * p2, bdesc + ((2 * p2 * 3 + ka) * C::N3), id, 1);
                    } else {
                        // the two channel-group planes of staged pixel m + kx
                        const uint64_t adesc = smem_desc(row, C::PLANE, 128);
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            mma_e4m3(d, adesc + kx, bdesc + ((kx * 2 * 3 + ka) * C::N3), id, 1);
                    }
                }
                mma_commit(mma3 + b);
                mma_commit(accf + tb);
                if (!wait_phase(a1full, it & 1, s_abort)) {
                    failed = true;
                    break;
                }
                fence_after_sync();
                for (int r = 0; r < R; ++r) {
#pragma unroll
                    for (int q = 0; q < C::MPP / 2; ++q) {
                        const uint64_t ad = smem_desc(sA1 + 16 * ((r * C::MPP + 2 * q) * kTileM), kTileM * 16, 128);
                        const uint64_t bd = smem_desc(sB1 + 16 * (2 * q * C::N1), C::N1 * 16, 128);
                        mma_e4m3(D + r * C::N3, ad, bd, id1, q > 0);
                    }
                }
                mma_commit(mma1);
            }
            if (failed) {
                atomicExch(a.err, 4);
                *s_abort = 1;
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue (warps 0 .. NEW-1; TMEM lane quarter = warp % 4)
        constexpr int G = NEW / 4;
        const int m = (warp & 3) * 32 + (tid & 31);
        const int rg = G == 1 ? 0 : warp >> 2;
        const uint32_t tlane = tbase + (static_cast<uint32_t>((warp & 3) * 32) << 16);
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
            // ---- 3x3 result: scale, bias, ReLU -> E4M3 -> operand of the 1x1
            for (int r = rg; r < R; r += G) {
#pragma unroll
                for (int c0 = 0; c0 < CMID; c0 += 16) {
                    float val[16];
                    tmem_ld16(Dl + (R - 1 - r) * C::N3 + c0, val);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) val[j] = fmaxf(fmaf(val[j], s3_s[c0 + j], bias3_s[c0 + j]), 0.f);
                    st_shared_v4(sA1 + 16 * ((r * C::MPP + c0 / 16) * kTileM + m), pack16_e4m3(val));
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
            // ---- 1x1 result -> outputs (E4M3 [pixel][COUT]; the head writes FP32 visibility)
            const int ox = x0 + m;
            if constexpr (EPI == TEPI_POOL || EPI == TEPI_SKIP_POOL) {
                for (int r = 2 * rg; r < R; r += 2 * G) {
                    const int oy = y0 + r;
                    float s[COUT];
#pragma unroll
                    for (int c0 = 0; c0 < COUT; c0 += 16) {
                        float v0[16], v1[16];
                        tmem_ld16(Dl + r * C::N3 + c0, v0);
                        tmem_ld16(Dl + (r + 1) * C::N3 + c0, v1);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            v0[j] = fmaxf(fmaf(v0[j], s1_s[c0 + j], bias1_s[c0 + j]), 0.f);
                            v1[j] = fmaxf(fmaf(v1[j], s1_s[c0 + j], bias1_s[c0 + j]), 0.f);
                            s[c0 + j] = v0[j] + v1[j];
                        }
                        if constexpr (EPI == TEPI_SKIP_POOL) {
                            if (oy < H && ox < W) {
                                uint8_t* dst = job.out_skip8 + (static_cast<size_t>(oy) * W + ox) * COUT + c0;
                                *reinterpret_cast<uint4*>(dst) = pack16_e4m3(v0);
                                *reinterpret_cast<uint4*>(dst + static_cast<size_t>(W) * COUT) = pack16_e4m3(v1);
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < COUT; ++c) s[c] = 0.25f * (s[c] + __shfl_xor_sync(0xffffffffu, s[c], 1));
                    if (oy < H && ox < W && (m & 1) == 0) {
                        uint8_t* dst = job.out8 + (static_cast<size_t>(oy / 2) * (W / 2) + ox / 2) * COUT;
#pragma unroll
                        for (int c0 = 0; c0 < COUT; c0 += 16) *reinterpret_cast<uint4*>(dst + c0) = pack16_e4m3(s + c0);
                    }
                }
            } else {
                for (int r = rg; r < R; r += G) {
                    const int oy = y0 + r;
                    float hsum = 0.f;
#pragma unroll
                    for (int c0 = 0; c0 < COUT; c0 += 16) {
                        float val[16];
                        tmem_ld16(Dl + r * C::N3 + c0, val);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) val[j] = fmaxf(fmaf(val[j], s1_s[c0 + j], bias1_s[c0 + j]), 0.f);
                        if constexpr (EPI == TEPI_STORE) {
                            if (oy < H && ox < W)
                                *reinterpret_cast<uint4*>(job.out8 + (static_cast<size_t>(oy) * W + ox) * COUT + c0) =
                                    pack16_e4m3(val);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) hsum = fmaf(head_s[c0 + j], val[j], hsum);
                        }
                    }
                    if (EPI == TEPI_HEAD && oy < H && ox < W)
                        job.vis[static_cast<size_t>(oy) * W + ox] = sigmoidf_fast(hsum + head_s[COUT]);
                }
            }
            fence_before_sync();
            mbar_arrive(tfree + tb);
        }
    }

    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    fence_after_sync();
    if (warp == MW) tmem_dealloc(tbase, C::TMEM_COLS);
}

// ------------------------------------------------------------------ launch
template <int CIN, int CMID, int COUT, int R, int PRO, int EPI, int NEW, int NPW>
static cudaError_t f8_launch(const TcBatch& a, cudaStream_t stream) {
    using C = F8Cfg<CIN, CMID, COUT, R, PRO>;
    constexpr int NT = 32 * (NEW + NPW + 1);
    auto kern = level_f8_kernel<CIN, CMID, COUT, R, PRO, EPI, NEW, NPW>;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::BYTES);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int regs = ((fa.numRegs + 7) / 8) * 8 * NT;
        const int by_regs = regs > 0 ? 65536 / regs : 8;
        const int by_smem = (228 * 1024) / (C::BYTES + 1024);
        int o = by_regs < by_smem ? by_regs : by_smem;
        if (o > C::TMEM_CAP) o = C::TMEM_CAP;
        occ = o < 1 ? 1 : o;
    }
    const int tiles = a.tile_start[a.nviews];
    if (tiles == 0) return cudaSuccess;
    const int cap = occ * num_sms();
    kern<<<tiles < cap ? tiles : cap, NT, C::BYTES, stream>>>(a);
    return cudaGetLastError();
}

const char* const kInferKernelNamesFp8[kInferKernelsFp8] = {
    "fp8_enc0_gather", "fp8_enc1", "fp8_bottleneck", "fp8_dec1", "fp8_dec0_head"};

cudaError_t launch_infer_fp8(const GatherParams& g, const float* params, const uint8_t* img, const float* scales,
                             const Activations& A, float* vis, int* err, cudaStream_t stream,
                             const StageEvents& se) {
    const LayerOffsets off = layer_offsets();
    const F8Images im = fp8_images();
    const int l3[kTcStages] = {ENC0_3, ENC1_3, BOTT_3, DEC1_3, DEC0_3};
    const int l1[kTcStages] = {ENC0_1, ENC1_1, BOTT_1, DEC1_1, DEC0_1};
    const int rows[kTcStages] = {8, 4, 2, 4, 8};
    const int H = g.H, W = g.W;
    for (int s = 0; s < kTcStages; ++s) {
        TcBatch b{};
        b.nviews = 1;
        b.b3img = reinterpret_cast<const uint4*>(img + im.img_off[l3[s]]);
        b.b1img = reinterpret_cast<const uint4*>(img + im.img_off[l1[s]]);
        b.bias3 = params + off.b[l3[s]];
        b.bias1 = params + off.b[l1[s]];
        b.scale3 = scales + im.scale_off[l3[s]];
        b.scale1 = scales + im.scale_off[l1[s]];
        b.head = params + off.w[HEAD];
        b.err = err;
        TcJob& j = b.job[0];
        j.g = g;
        switch (s) {
            case 0: j.H = H; j.W = W; j.out8 = static_cast<uint8_t*>(A.e0); break;
            case 1: j.H = H / 2; j.W = W / 2; j.in8 = static_cast<const uint8_t*>(A.e0);
                    j.out_skip8 = static_cast<uint8_t*>(A.s1); j.out8 = static_cast<uint8_t*>(A.p1); break;
            case 2: j.H = H / 4; j.W = W / 4; j.in8 = static_cast<const uint8_t*>(A.p1);
                    j.out8 = static_cast<uint8_t*>(A.bo); break;
            case 3: j.H = H / 2; j.W = W / 2; j.in8 = static_cast<const uint8_t*>(A.bo);
                    j.skip8 = static_cast<const uint8_t*>(A.s1); j.out8 = static_cast<uint8_t*>(A.d1); break;
            default: j.H = H; j.W = W; j.in8 = static_cast<const uint8_t*>(A.d1); j.vis = vis; break;
        }
        tc_fill_tiles(b, rows[s]);
        se.rec(s);
        cudaError_t e;
        switch (s) {
            case 0: e = f8_launch<4, 16, 16, 8, TPRO_GATHER, TEPI_POOL, 4, 16>(b, stream); break;
            case 1: e = f8_launch<16, 32, 32, 4, TPRO_PLAIN, TEPI_SKIP_POOL, 4, 8>(b, stream); break;
            case 2: e = f8_launch<32, 64, 32, 2, TPRO_PLAIN, TEPI_STORE, 4, 8>(b, stream); break;
            case 3: e = f8_launch<32, 32, 16, 4, TPRO_UP_SKIP, TEPI_STORE, 4, 8>(b, stream); break;
            default: e = f8_launch<16, 16, 16, 8, TPRO_UP, TEPI_HEAD, 8, 8>(b, stream); break;
        }
        if (e != cudaSuccess) return e;
    }
    se.rec(kTcStages);
    return cudaSuccess;
}

}  // namespace nsm
