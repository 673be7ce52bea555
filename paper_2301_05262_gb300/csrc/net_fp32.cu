// FP32 CUDA-core form of the compact encoder/decoder (Sec. 3.5).
//
// One fused kernel per level pair "3x3 conv + ReLU -> 1x1 conv + ReLU", with
// the level's input staged in shared memory (tile + 1-pixel halo, zero
// padded) by one of four prologues and its output written by one of four
// epilogues:
//   prologue  GATHER   features computed from the G-buffer and shadow map
//             PLAIN    NHWC activation tensor of this level
//             UP_SKIP  bilinear x2 of the coarser tensor + the skip tensor
//             UP       bilinear x2 of the coarser tensor
//   epilogue  POOL      2x2 average -> NHWC at half resolution
//             SKIP_POOL NHWC at this resolution (decoder skip) + pooled
//             STORE     NHWC at this resolution
//             HEAD      1x1 16 -> 1 + sigmoid -> visibility image
// Each thread owns a 2x2 quad of output pixels; CTAs are persistent and load
// the level's weights into shared memory once.
#include "nsm_internal.h"

namespace nsm {

enum Pro { PRO_GATHER = 0, PRO_PLAIN = 1, PRO_UP_SKIP = 2, PRO_UP = 3 };
enum Epi { EPI_POOL = 0, EPI_SKIP_POOL = 1, EPI_STORE = 2, EPI_HEAD = 3 };

struct LevelArgs {
    GatherParams g;
    int H, W;                 // resolution of this level
    const float* in;          // PLAIN: [H][W][CIN]; UP*: [H/2][W/2][CIN]
    const float* skip;        // UP_SKIP: [H][W][CIN]
    const float* w3; const float* b3;  // OIHW [CMID][CIN][3][3]
    const float* w1; const float* b1;  // [COUT][CMID]
    const float* wh; const float* bh;  // head [1][COUT]
    float* out;
    float* out_skip;
};

template <int CIN, int CMID, int COUT, int QH, int QW>
struct Smem {
    static constexpr int TH = 2 * QH, TW = 2 * QW;
    static constexpr int RH = TH + 2, RW = TW + 2;
    static constexpr int PLANE = RH * RW;
    static constexpr int IN = CIN * PLANE;
    static constexpr int W3 = 9 * CIN * CMID;
    static constexpr int W1 = CMID * COUT;
    static constexpr int TOTAL = IN + W3 + W1 + CMID + COUT + COUT + 4;
    static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

template <int CIN, int CMID, int COUT, int QH, int QW, int PRO, int EPI>
__global__ void __launch_bounds__(QH * QW) level_fp32_kernel(LevelArgs a) {
    using S = Smem<CIN, CMID, COUT, QH, QW>;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* in_s = sm;
    float* w3_s = in_s + S::IN;      // [tap][ci][co]
    float* w1_s = w3_s + S::W3;      // [ci][co]
    float* b3_s = w1_s + S::W1;
    float* b1_s = b3_s + CMID;
    float* wh_s = b1_s + COUT;       // head weights (EPI_HEAD), + bias at [COUT]

    const int tid = threadIdx.x;
    constexpr int NT = QH * QW;

    // weights: OIHW -> [tap][ci][co]
    for (int idx = tid; idx < S::W3; idx += NT) {
        const int co = idx % CMID;
        const int ci = (idx / CMID) % CIN;
        const int tap = idx / (CMID * CIN);
        w3_s[idx] = __ldg(a.w3 + (co * CIN + ci) * 9 + tap);
    }
    for (int idx = tid; idx < S::W1; idx += NT) {
        const int co = idx % COUT;
        const int ci = idx / COUT;
        w1_s[idx] = __ldg(a.w1 + co * CMID + ci);
    }
    for (int idx = tid; idx < CMID; idx += NT) b3_s[idx] = __ldg(a.b3 + idx);
    for (int idx = tid; idx < COUT; idx += NT) b1_s[idx] = __ldg(a.b1 + idx);
    if (EPI == EPI_HEAD) {
        for (int idx = tid; idx < COUT; idx += NT) wh_s[idx] = __ldg(a.wh + idx);
        if (tid == 0) wh_s[COUT] = __ldg(a.bh);
    }

    const int H = a.H, W = a.W;
    const int tiles_x = (W + S::TW - 1) / S::TW;
    const int tiles_y = (H + S::TH - 1) / S::TH;
    const int ntiles = tiles_x * tiles_y;
    const int qy = tid / QW, qx = tid % QW;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int y0 = (tile / tiles_x) * S::TH;
        const int x0 = (tile % tiles_x) * S::TW;
        __syncthreads();  // previous tile's readers are done with in_s (and weights are loaded)

        // ---------------- prologue: stage (TH+2) x (TW+2) x CIN, zero padded
        if (PRO == PRO_GATHER) {
            for (int r = tid; r < S::PLANE; r += NT) {
                const int ry = r / S::RW, rx = r % S::RW;
                const int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
                float f[4] = {0.f, 0.f, 0.f, 0.f};
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    gather_features(a.g, gy, gx, f);
                    if (a.g.feat_eps)
                        f[a.g.eps_ch] += a.g.eps_scale * __ldg(a.g.feat_eps + static_cast<size_t>(gy) * W + gx);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) in_s[c * S::PLANE + r] = f[c];
            }
        } else if (PRO == PRO_PLAIN) {
            constexpr int C4 = CIN / 4;
            for (int idx = tid; idx < S::PLANE * C4; idx += NT) {
                const int c4 = idx % C4;
                const int r = idx / C4;
                const int ry = r / S::RW, rx = r % S::RW;
                const int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                    v = __ldg(reinterpret_cast<const float4*>(a.in + (static_cast<size_t>(gy) * W + gx) * CIN) + c4);
                in_s[(4 * c4 + 0) * S::PLANE + r] = v.x;
                in_s[(4 * c4 + 1) * S::PLANE + r] = v.y;
                in_s[(4 * c4 + 2) * S::PLANE + r] = v.z;
                in_s[(4 * c4 + 3) * S::PLANE + r] = v.w;
            }
        } else {  // UP_SKIP / UP: bilinear x2 of in (H/2 x W/2) (+ skip)
            constexpr int C4 = CIN / 4;
            const int Hl = H / 2, Wl = W / 2;
            for (int idx = tid; idx < S::PLANE * C4; idx += NT) {
                const int c4 = idx % C4;
                const int r = idx / C4;
                const int ry = r / S::RW, rx = r % S::RW;
                const int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const BilinTap ty = bilin_tap(gy, Hl), tx = bilin_tap(gx, Wl);
                    auto ld = [&](int yy, int xx) {
                        return __ldg(reinterpret_cast<const float4*>(a.in + (static_cast<size_t>(yy) * Wl + xx) * CIN) + c4);
                    };
                    const float4 a00 = ld(ty.i0, tx.i0), a01 = ld(ty.i0, tx.i1);
                    const float4 a10 = ld(ty.i1, tx.i0), a11 = ld(ty.i1, tx.i1);
                    auto mix = [&](float p00, float p01, float p10, float p11) {
                        const float r0 = p00 * tx.w0 + p01 * tx.w1;
                        const float r1 = p10 * tx.w0 + p11 * tx.w1;
                        return r0 * ty.w0 + r1 * ty.w1;
                    };
                    v = make_float4(mix(a00.x, a01.x, a10.x, a11.x), mix(a00.y, a01.y, a10.y, a11.y),
                                    mix(a00.z, a01.z, a10.z, a11.z), mix(a00.w, a01.w, a10.w, a11.w));
                    if (PRO == PRO_UP_SKIP) {
                        const float4 s = __ldg(reinterpret_cast<const float4*>(a.skip + (static_cast<size_t>(gy) * W + gx) * CIN) + c4);
                        v.x += s.x; v.y += s.y; v.z += s.z; v.w += s.w;
                    }
                }
                in_s[(4 * c4 + 0) * S::PLANE + r] = v.x;
                in_s[(4 * c4 + 1) * S::PLANE + r] = v.y;
                in_s[(4 * c4 + 2) * S::PLANE + r] = v.z;
                in_s[(4 * c4 + 3) * S::PLANE + r] = v.w;
            }
        }
        __syncthreads();

        // ---------------- compute: each thread a 2x2 quad; PXQ of its pixels at a
        // time share every weight load (all four for narrow layers)
        constexpr int PXQ = (CMID <= 16) ? 4 : 1;
        float pool[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) pool[c] = 0.f;
        const int oyq = y0 + 2 * qy, oxq = x0 + 2 * qx;
#pragma unroll 1
        for (int q0 = 0; q0 < 4; q0 += PXQ) {
            float acc[PXQ][CMID];
#pragma unroll
            for (int j = 0; j < PXQ; ++j)
#pragma unroll
                for (int c = 0; c < CMID; ++c) acc[j][c] = b3_s[c];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const float4* wt = reinterpret_cast<const float4*>(w3_s + tap * CIN * CMID);
#pragma unroll 4
                for (int ci = 0; ci < CIN; ++ci) {
                    float xv[PXQ];
#pragma unroll
                    for (int j = 0; j < PXQ; ++j) {
                        const int q = q0 + j;
                        const int ly = 2 * qy + (q >> 1), lx = 2 * qx + (q & 1);
                        xv[j] = in_s[ci * S::PLANE + (ly + tap / 3) * S::RW + (lx + tap % 3)];
                    }
#pragma unroll
                    for (int c4 = 0; c4 < CMID / 4; ++c4) {
                        const float4 w = wt[ci * (CMID / 4) + c4];
#pragma unroll
                        for (int j = 0; j < PXQ; ++j) {
                            acc[j][4 * c4 + 0] = fmaf(xv[j], w.x, acc[j][4 * c4 + 0]);
                            acc[j][4 * c4 + 1] = fmaf(xv[j], w.y, acc[j][4 * c4 + 1]);
                            acc[j][4 * c4 + 2] = fmaf(xv[j], w.z, acc[j][4 * c4 + 2]);
                            acc[j][4 * c4 + 3] = fmaf(xv[j], w.w, acc[j][4 * c4 + 3]);
                        }
                    }
                }
            }
            float o[PXQ][COUT];
#pragma unroll
            for (int j = 0; j < PXQ; ++j)
#pragma unroll
                for (int c = 0; c < COUT; ++c) o[j][c] = b1_s[c];
            const float4* w1v = reinterpret_cast<const float4*>(w1_s);
#pragma unroll
            for (int ci = 0; ci < CMID; ++ci) {
#pragma unroll
                for (int c4 = 0; c4 < COUT / 4; ++c4) {
                    const float4 w = w1v[ci * (COUT / 4) + c4];
#pragma unroll
                    for (int j = 0; j < PXQ; ++j) {
                        const float hv = fmaxf(acc[j][ci], 0.f);
                        o[j][4 * c4 + 0] = fmaf(hv, w.x, o[j][4 * c4 + 0]);
                        o[j][4 * c4 + 1] = fmaf(hv, w.y, o[j][4 * c4 + 1]);
                        o[j][4 * c4 + 2] = fmaf(hv, w.z, o[j][4 * c4 + 2]);
                        o[j][4 * c4 + 3] = fmaf(hv, w.w, o[j][4 * c4 + 3]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < PXQ; ++j) {
                const int q = q0 + j;
                const int oy = oyq + (q >> 1), ox = oxq + (q & 1);
                const bool inb = oy < H && ox < W;
#pragma unroll
                for (int c = 0; c < COUT; ++c) o[j][c] = fmaxf(o[j][c], 0.f);
                if (EPI == EPI_POOL || EPI == EPI_SKIP_POOL) {
#pragma unroll
                    for (int c = 0; c < COUT; ++c) pool[c] += o[j][c];
                }
                if (inb) {
                    if (EPI == EPI_STORE || EPI == EPI_SKIP_POOL) {
                        float* dst = (EPI == EPI_STORE ? a.out : a.out_skip) + (static_cast<size_t>(oy) * W + ox) * COUT;
#pragma unroll
                        for (int c4 = 0; c4 < COUT / 4; ++c4)
                            reinterpret_cast<float4*>(dst)[c4] =
                                make_float4(o[j][4 * c4], o[j][4 * c4 + 1], o[j][4 * c4 + 2], o[j][4 * c4 + 3]);
                    } else if (EPI == EPI_HEAD) {
                        float l = wh_s[COUT];
#pragma unroll
                        for (int c = 0; c < COUT; ++c) l = fmaf(wh_s[c], o[j][c], l);
                        a.out[static_cast<size_t>(oy) * W + ox] = sigmoidf_acc(l);
                    }
                }
            }
        }
        if ((EPI == EPI_POOL || EPI == EPI_SKIP_POOL) && oyq < H && oxq < W) {
            float* dst = a.out + (static_cast<size_t>(oyq / 2) * (W / 2) + oxq / 2) * COUT;
#pragma unroll
            for (int c4 = 0; c4 < COUT / 4; ++c4)
                reinterpret_cast<float4*>(dst)[c4] = make_float4(0.25f * pool[4 * c4], 0.25f * pool[4 * c4 + 1],
                                                                 0.25f * pool[4 * c4 + 2], 0.25f * pool[4 * c4 + 3]);
        }
    }
}

template <int CIN, int CMID, int COUT, int QH, int QW, int PRO, int EPI>
static cudaError_t launch_level(const LevelArgs& a, cudaStream_t stream) {
    using S = Smem<CIN, CMID, COUT, QH, QW>;
    auto kern = level_fp32_kernel<CIN, CMID, COUT, QH, QW, PRO, EPI>;
    static int occ = -1;  // per instantiation; the library targets one device model
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(S::BYTES));
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, QH * QW, S::BYTES);
        if (e != cudaSuccess) return e;
        occ = o > 0 ? o : 1;
    }
    const int tiles = ((a.H + S::TH - 1) / S::TH) * ((a.W + S::TW - 1) / S::TW);
    if (tiles == 0) return cudaSuccess;
    const int cap = occ * num_sms();
    const int grid = tiles < cap ? tiles : cap;
    kern<<<grid, QH * QW, S::BYTES, stream>>>(a);
    return cudaGetLastError();
}

const char* const kInferKernelNamesFp32[kInferKernelsFp32] = {
    "fp32_enc0_gather", "fp32_enc1", "fp32_bottleneck", "fp32_dec1", "fp32_dec0_head"};

cudaError_t launch_infer_fp32(const GatherParams& g, const float* params, const Activations& act,
                              float* vis, cudaStream_t stream, const StageEvents& se) {
    const LayerOffsets off = layer_offsets();
    const int H = g.H, W = g.W;
    cudaError_t e;
    LevelArgs a{};
    a.g = g;
    // level 0 encoder, fused with the gather: 4 -> 16 -> 16, pooled
    a.H = H; a.W = W;
    a.w3 = params + off.w[ENC0_3]; a.b3 = params + off.b[ENC0_3];
    a.w1 = params + off.w[ENC0_1]; a.b1 = params + off.b[ENC0_1];
    a.out = static_cast<float*>(act.e0);
    se.rec(0);
    if ((e = launch_level<4, 16, 16, 8, 16, PRO_GATHER, EPI_POOL>(a, stream)) != cudaSuccess) return e;
    // level 1 encoder: 16 -> 32 -> 32, skip + pooled
    a = LevelArgs{}; a.g = g;
    a.H = H / 2; a.W = W / 2;
    a.in = static_cast<const float*>(act.e0);
    a.w3 = params + off.w[ENC1_3]; a.b3 = params + off.b[ENC1_3];
    a.w1 = params + off.w[ENC1_1]; a.b1 = params + off.b[ENC1_1];
    a.out_skip = static_cast<float*>(act.s1);
    a.out = static_cast<float*>(act.p1);
    se.rec(1);
    if ((e = launch_level<16, 32, 32, 8, 16, PRO_PLAIN, EPI_SKIP_POOL>(a, stream)) != cudaSuccess) return e;
    // bottleneck: 32 -> 64 -> 32
    a = LevelArgs{}; a.g = g;
    a.H = H / 4; a.W = W / 4;
    a.in = static_cast<const float*>(act.p1);
    a.w3 = params + off.w[BOTT_3]; a.b3 = params + off.b[BOTT_3];
    a.w1 = params + off.w[BOTT_1]; a.b1 = params + off.b[BOTT_1];
    a.out = static_cast<float*>(act.bo);
    se.rec(2);
    if ((e = launch_level<32, 64, 32, 4, 16, PRO_PLAIN, EPI_STORE>(a, stream)) != cudaSuccess) return e;
    // level 1 decoder: up(bottleneck) + skip -> 32 -> 16
    a = LevelArgs{}; a.g = g;
    a.H = H / 2; a.W = W / 2;
    a.in = static_cast<const float*>(act.bo);
    a.skip = static_cast<const float*>(act.s1);
    a.w3 = params + off.w[DEC1_3]; a.b3 = params + off.b[DEC1_3];
    a.w1 = params + off.w[DEC1_1]; a.b1 = params + off.b[DEC1_1];
    a.out = static_cast<float*>(act.d1);
    se.rec(3);
    if ((e = launch_level<32, 32, 16, 4, 16, PRO_UP_SKIP, EPI_STORE>(a, stream)) != cudaSuccess) return e;
    // level 0 decoder + head: up(level-1 decoder) -> 16 -> 16 -> 1, sigmoid
    a = LevelArgs{}; a.g = g;
    a.H = H; a.W = W;
    a.in = static_cast<const float*>(act.d1);
    a.w3 = params + off.w[DEC0_3]; a.b3 = params + off.b[DEC0_3];
    a.w1 = params + off.w[DEC0_1]; a.b1 = params + off.b[DEC0_1];
    a.wh = params + off.w[HEAD]; a.bh = params + off.b[HEAD];
    a.out = vis;
    se.rec(4);
    e = launch_level<16, 16, 16, 8, 16, PRO_UP, EPI_HEAD>(a, stream);
    se.rec(5);
    return e;
}

}  // namespace nsm
