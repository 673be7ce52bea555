// Training path: forward with level checkpoints, hand-written adjoint
// (backward) with per-level recomputation, the Eq. 2 loss and Adam
// (Sec. 3.3, Eq. 2; network of Sec. 3.5).
//
// All tensors here are FP32 NHWC batches [N][H][W][C].  The forward keeps
// only the level boundaries (features, pooled level-0 output, level-1 skip,
// pooled level-1 output, bottleneck output, level-1 decoder output); the
// backward recomputes each level's 3x3 / 1x1 pre-activations from its
// checkpoint right before back-propagating through it, so at most one
// level's internals are alive at a time.
//
// Kernels (CUDA cores, FP32):
//   conv_fwd   y = conv(x~) (+ b) (masked by m > 0), x~ = x, relu(x) or x (m_in > 0);
//              also the data gradient, as a convolution with the transposed,
//              flipped weights.  In the checkpointed forward one launch covers
//              a whole level: the input up-sampled while staging (decoders),
//              3x3, ReLU, the 1x1 in the epilogue, then the rectified
//              checkpoint, the 2x2 pooling (encoders) or the head (level 0);
//   conv1x1    1x1 layers: coalesced pixel tiles through shared memory, one
//              thread per pixel for the products;
//   conv_wgrad dW += sum_p g~(p) x~(p + tap), db += sum_p g~(p) of the 3x3
//              layers: 8 x 8 register blocks of outer products per thread, one
//              atomicAdd per weight per CTA (the 1x1 layers' weight gradients:
//              wgrad1x1_tiles, fixed order);
//   pooling, bilinear x2 and their adjoints, head, loss, Adam.
#include <vector>

#include "nsm_internal.h"
#include "train_internal.h"

namespace nsm {
namespace tr {


// ------------------------------------------------------------------ convolution
// y[n,p,o] = b[o] + sum_{c,tap} Wc[o][c][tap] * xin(n, p + off(tap), c), zero padded,
// xin = relu(x) if relu_in, x * (xm > 0) if xm, else x;  y *= (ym > 0) if ym.
// Weights come as canonical OIHW (transpose_flip = 0), as the weights of the
// layer whose data gradient this is (transpose_flip = 1): Wc[o][c][tap] =
// W[c][o][8 - tap], or pre-transposed to [tap][c][o] (transpose_flip = 2,
// so a chunk's weights are contiguous rows of outputs: coalesced staging).
// Tile: 8 rows x 16 PX columns; thread (r, j) computes the PX pixels of row r
// at columns j, j + 16, ... (neighbouring threads read neighbouring words) for
// every output; per (tap, input channel) PX input words and COUT / 4
// broadcast float4 weight words feed PX COUT FMAs.  The input tile is staged
// as channel planes with an odd plane stride (conflict-free transposing
// stores from 16-byte NHWC loads).
constexpr int TH = 8, TJ = 16, NT = TH * TJ;  // conv tile rows, threads per row
static int ew_grid(size_t n);                  // grid of the element-wise kernels

// Bilinear x2 up-sampling (half-pixel centres, clamped) of channel group c4
// (4 channels) of the coarse NHWC tensor lo (Hl x Wl, C4 groups) at fine
// pixel (yy, x); one definition for every kernel that up-samples.
__device__ __forceinline__ float4 up_sample4(const float4* __restrict__ lo4, int n, int Hl, int Wl, int C4, int yy,
                                             int x, int c4) {
    const BilinTap ty = bilin_tap(yy, Hl), tx = bilin_tap(x, Wl);
    auto L = [&](int a, int b2) { return __ldg(lo4 + ((static_cast<size_t>(n) * Hl + a) * Wl + b2) * C4 + c4); };
    const float4 a00 = L(ty.i0, tx.i0), a01 = L(ty.i0, tx.i1), a10 = L(ty.i1, tx.i0), a11 = L(ty.i1, tx.i1);
    auto mix = [&](float v00, float v01, float v10, float v11) {
        return (v00 * tx.w0 + v01 * tx.w1) * ty.w0 + (v10 * tx.w0 + v11 * tx.w1) * ty.w1;
    };
    return make_float4(mix(a00.x, a01.x, a10.x, a11.x), mix(a00.y, a01.y, a10.y, a11.y),
                       mix(a00.z, a01.z, a10.z, a11.z), mix(a00.w, a01.w, a10.w, a11.w));
}

// pixels per thread: 4, or 2 where 64 channels in or out would need too many
// accumulators or too much shared memory
template <int CIN, int COUT>
struct FwdShape { static constexpr int PX = (COUT >= 64 || CIN >= 64) ? 2 : 4; };

// CB input channels are staged at a time (CB < CIN: the weights of each chunk
// are staged with it), and a CTA computes the OB outputs of block blockIdx.y
// (OB < COUT for wide layers); CB = CIN, OB = COUT stage everything once.
// C1 > 0 fuses the level's 1x1 convolution (C1 outputs, OIHW weights w1, bias
// b1) into the epilogue: y gets b1 + W1 relu(conv), rectified as well with
// relu_out; the 3x3 result itself is not stored (the checkpointed forward
// needs only the 1x1 output); the sums run in the order of the separate 1x1
// layer, so the result is the same.  POOL also writes yp = 2x2 average of
// relu(y) (H, W even): the four pixels of a block are lanes l, l + 1, l + 16,
// l + 17 of one warp, summed in the separate pooling kernel's order; y may
// then be null.  UPIN: the input is up(x) + xm, x the coarse (H/2 x W/2)
// tensor and xm the skip (nullable), up-sampled while staging (no mask).
// HEAD (C1 = 16): also vis = sigmoid(wh[16] + sum_o wh[o] relu(y_o)), summed
// in the head kernel's order; y may then be null.
template <int CIN, int COUT, int K, int CB = CIN, int OB = COUT, int C1 = 0, int POOL = 0, int UPIN = 0,
          int HEAD = 0>
__global__ void __launch_bounds__(NT) conv_fwd_kernel(const float* __restrict__ x, const float* __restrict__ xm,
                                                      int relu_in, int N, int H, int W,
                                                      const float* __restrict__ w, int transpose_flip,
                                                      const float* __restrict__ b, const float* __restrict__ ym,
                                                      float* __restrict__ y, const float* __restrict__ w1,
                                                      const float* __restrict__ b1, int relu_out,
                                                      float* __restrict__ yp, const float* __restrict__ wh,
                                                      float* __restrict__ vis) {
    constexpr int P = K / 2, PX = FwdShape<CB, OB>::PX, TW = TJ * PX;
    constexpr int RH = TH + 2 * P, RW = TW + 2 * P, PS = (RH * RW) | 1;  // odd plane stride
    constexpr bool ONCE = (CB == CIN);
    static_assert(CIN % CB == 0 && COUT % OB == 0 && CB % 4 == 0 && OB % 4 == 0, "channel blocks");
    static_assert(C1 == 0 || (OB == COUT && C1 % 4 == 0), "the fused 1x1 needs every 3x3 output of a pixel");
    static_assert(POOL == 0 || C1 > 0, "pooling follows the fused 1x1");
    static_assert(HEAD == 0 || (C1 == 16 && POOL == 0), "the head reads the 16 outputs of the fused 1x1");
    extern __shared__ float sm[];
    float* xs = sm;                       // [CB][PS]
    float* ws = xs + CB * PS;             // [tap][ci of the chunk][co of the block]
    float* w1s = ws + K * K * CB * OB;    // fused 1x1: [c][o]
    const int tid = threadIdx.x;
    if constexpr (C1 > 0) {
        for (int i = tid; i < C1 * COUT; i += NT) w1s[i] = __ldg(w1 + (i % C1) * COUT + i / C1);
    }
    const int ob0 = blockIdx.y * OB;
    auto stage_w = [&](int c0) {
        if (transpose_flip == 2) {
            for (int i = tid; i < K * K * CB * (OB / 4); i += NT) {  // float4 rows of OB outputs
                const int o4 = i % (OB / 4), ci = c0 + (i / (OB / 4)) % CB, tap = i / ((OB / 4) * CB);
                reinterpret_cast<float4*>(ws)[i] =
                    __ldg(reinterpret_cast<const float4*>(w + (static_cast<size_t>(tap) * CIN + ci) * COUT + ob0) + o4);
            }
            return;
        }
        for (int i = tid; i < K * K * CB * OB; i += NT) {
            const int co = ob0 + i % OB, ci = c0 + (i / OB) % CB, tap = i / (OB * CB);
            ws[i] = transpose_flip ? __ldg(w + (static_cast<size_t>(ci) * COUT + co) * K * K + (K * K - 1 - tap))
                                   : __ldg(w + (static_cast<size_t>(co) * CIN + ci) * K * K + tap);
        }
    };
    if (ONCE) stage_w(0);
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
    const long long ntiles = static_cast<long long>(N) * tx * ty;
    const int lr = tid / TJ, lj = tid % TJ;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int n = static_cast<int>(t / (tx * ty));
        const int r = static_cast<int>(t % (tx * ty));
        const int y0 = (r / tx) * TH, x0 = (r % tx) * TW;
        float acc[PX][OB];
#pragma unroll
        for (int o = 0; o < OB; ++o) {
            const float bo = b ? __ldg(b + ob0 + o) : 0.f;
#pragma unroll
            for (int p = 0; p < PX; ++p) acc[p][o] = bo;
        }
#pragma unroll 1
        for (int c0 = 0; c0 < CIN; c0 += CB) {
            __syncthreads();
            if (!ONCE) stage_w(c0);
            for (int i = tid; i < RH * RW * (CB / 4); i += NT) {
                const int c4 = i % (CB / 4), q = i / (CB / 4);
                const int gy = y0 - P + q / RW, gx = x0 - P + q % RW;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (UPIN && gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    v = up_sample4(reinterpret_cast<const float4*>(x), n, H / 2, W / 2, CIN / 4, gy, gx, c0 / 4 + c4);
                    if (xm) {
                        const float4 sk = __ldg(reinterpret_cast<const float4*>(
                                                    xm + ((static_cast<size_t>(n) * H + gy) * W + gx) * CIN + c0) + c4);
                        v.x += sk.x; v.y += sk.y; v.z += sk.z; v.w += sk.w;
                    }
                } else if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const size_t idx = ((static_cast<size_t>(n) * H + gy) * W + gx) * CIN + c0;
                    v = __ldg(reinterpret_cast<const float4*>(x + idx) + c4);
                    if (relu_in) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
                    if (xm) {
                        const float4 m = __ldg(reinterpret_cast<const float4*>(xm + idx) + c4);
                        v = make_float4(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f, m.z > 0.f ? v.z : 0.f,
                                        m.w > 0.f ? v.w : 0.f);
                    }
                }
                xs[(4 * c4 + 0) * PS + q] = v.x;
                xs[(4 * c4 + 1) * PS + q] = v.y;
                xs[(4 * c4 + 2) * PS + q] = v.z;
                xs[(4 * c4 + 3) * PS + q] = v.w;
            }
            __syncthreads();
#pragma unroll
            for (int tap = 0; tap < K * K; ++tap) {
                const float* xin = xs + (lr + tap / K) * RW + (lj + tap % K);
                const float4* wt = reinterpret_cast<const float4*>(ws + tap * CB * OB);
#pragma unroll 2
                for (int c = 0; c < CB; ++c) {
                    float xv[PX];
#pragma unroll
                    for (int p = 0; p < PX; ++p) xv[p] = xin[c * PS + TJ * p];
#pragma unroll
                    for (int o4 = 0; o4 < OB / 4; ++o4) {
                        const float4 wv = wt[c * (OB / 4) + o4];
#pragma unroll
                        for (int p = 0; p < PX; ++p) {
                            acc[p][4 * o4 + 0] = fmaf(xv[p], wv.x, acc[p][4 * o4 + 0]);
                            acc[p][4 * o4 + 1] = fmaf(xv[p], wv.y, acc[p][4 * o4 + 1]);
                            acc[p][4 * o4 + 2] = fmaf(xv[p], wv.z, acc[p][4 * o4 + 2]);
                            acc[p][4 * o4 + 3] = fmaf(xv[p], wv.w, acc[p][4 * o4 + 3]);
                        }
                    }
                }
            }
        }
        const int oy = y0 + lr;
        if constexpr (C1 > 0) {
            const float4* w14 = reinterpret_cast<const float4*>(w1s);
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const int ox = x0 + lj + TJ * p;
                const bool ok = oy < H && ox < W;  // a 2x2 block is wholly in or out (H, W even)
                if (!POOL && !ok) continue;
#pragma unroll
                for (int c = 0; c < COUT; ++c) acc[p][c] = fmaxf(acc[p][c], 0.f);
                const size_t pix = (static_cast<size_t>(n) * H + oy) * W + ox;
                float logit = HEAD ? __ldg(wh + 16) : 0.f;
#pragma unroll 1
                for (int o4 = 0; o4 < C1 / 4; ++o4) {
                    float4 s = __ldg(reinterpret_cast<const float4*>(b1) + o4);
#pragma unroll
                    for (int c = 0; c < COUT; ++c) {
                        const float4 wv = w14[c * (C1 / 4) + o4];
                        s.x = fmaf(acc[p][c], wv.x, s.x);
                        s.y = fmaf(acc[p][c], wv.y, s.y);
                        s.z = fmaf(acc[p][c], wv.z, s.z);
                        s.w = fmaf(acc[p][c], wv.w, s.w);
                    }
                    if (relu_out) s = make_float4(fmaxf(s.x, 0.f), fmaxf(s.y, 0.f), fmaxf(s.z, 0.f), fmaxf(s.w, 0.f));
                    if (ok && y) reinterpret_cast<float4*>(y + pix * C1)[o4] = s;
                    if constexpr (HEAD) {
                        logit = fmaf(__ldg(wh + 4 * o4), fmaxf(s.x, 0.f), logit);
                        logit = fmaf(__ldg(wh + 4 * o4 + 1), fmaxf(s.y, 0.f), logit);
                        logit = fmaf(__ldg(wh + 4 * o4 + 2), fmaxf(s.z, 0.f), logit);
                        logit = fmaf(__ldg(wh + 4 * o4 + 3), fmaxf(s.w, 0.f), logit);
                    }
                    if constexpr (POOL) {
                        const float v[4] = {fmaxf(s.x, 0.f), fmaxf(s.y, 0.f), fmaxf(s.z, 0.f), fmaxf(s.w, 0.f)};
                        float q[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float v01 = __shfl_down_sync(0xffffffffu, v[e], 1);
                            const float v10 = __shfl_down_sync(0xffffffffu, v[e], 16);
                            const float v11 = __shfl_down_sync(0xffffffffu, v[e], 17);
                            q[e] = 0.25f * (((v[e] + v01) + v10) + v11);
                        }
                        if (ok && ((lr | lj) & 1) == 0)
                            reinterpret_cast<float4*>(
                                yp + ((static_cast<size_t>(n) * (H / 2) + oy / 2) * (W / 2) + ox / 2) * C1)[o4] =
                                make_float4(q[0], q[1], q[2], q[3]);
                    }
                }
                if (HEAD && ok) vis[pix] = sigmoidf_acc(logit);
            }
        } else {
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const int ox = x0 + lj + TJ * p;
                if (oy < H && ox < W) {
                    const size_t base = ((static_cast<size_t>(n) * H + oy) * W + ox) * COUT + ob0;
#pragma unroll
                    for (int o4 = 0; o4 < OB / 4; ++o4) {
                        float4 v = make_float4(acc[p][4 * o4], acc[p][4 * o4 + 1], acc[p][4 * o4 + 2], acc[p][4 * o4 + 3]);
                        if (ym) {
                            const float4 m = __ldg(reinterpret_cast<const float4*>(ym + base) + o4);
                            v = make_float4(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f, m.z > 0.f ? v.z : 0.f,
                                            m.w > 0.f ? v.w : 0.f);
                        }
                        reinterpret_cast<float4*>(y + base)[o4] = v;
                    }
                }
            }
        }
    }
}

// dW[o][c][tap] += sum_p g~[p][o] xin[p + off(tap)][c];  db[o] += sum_p g~[p][o],
// g~ = g * (gm > 0) if gm.  Register-blocked outer products: the weights are
// cut into blocks of 8 outputs x 8 inputs (4 where C_in = 4) of one tap;
// thread t owns blocks t, t + WNT, ... (64 accumulators each, kept in
// registers over every tile the CTA visits) and, when there are fewer blocks
// than threads, one residue class of the tile's pixels.  Per pixel a block
// takes two 16-byte loads of g~ and two of xin for 64 FMAs.  WNT = 9 x 32:
// every layer's block count times its pixel classes fills it exactly.  Pixel
// classes meet in shared memory at the end; one atomicAdd per weight per CTA.
constexpr int WTH = 8, WTW = 32, WNT = 288;  // wgrad pixel tile, threads

template <int CIN, int COUT, int K>
__global__ void __launch_bounds__(WNT, 2) conv_wgrad_kernel(const float* __restrict__ x, int relu_in,
                                                            const float* __restrict__ g, const float* __restrict__ gm,
                                                            int N, int H, int W, float* __restrict__ dW,
                                                            float* __restrict__ db) {
    constexpr int P = K / 2;
    constexpr int RH = WTH + 2 * P, RW = WTW + 2 * P, NPX = WTH * WTW;
    constexpr int BO = 8, BI = CIN % 8 == 0 ? 8 : 4, BE = BO * BI;
    constexpr int OB = COUT / BO, CB = CIN / BI, TAPS = K * K;
    constexpr int NB = TAPS * OB * CB;                  // weight blocks
    constexpr int PL = NB >= WNT ? 1 : WNT / NB;        // pixel classes
    constexpr int NBT = (NB + WNT - 1) / WNT;           // blocks per thread
    constexpr int NW = NB * BE;
    static_assert(CIN % BI == 0 && COUT % BO == 0, "channel blocks");
    static_assert(PL == 1 || NW <= RH * RW * CIN, "pixel-class reduction reuses the input tile");
    extern __shared__ float4 sm4[];
    float* xs = reinterpret_cast<float*>(sm4);  // [RH][RW][CIN]
    float* gs = xs + RH * RW * CIN;             // [NPX][COUT]
    float* dbs = gs + NPX * COUT;               // [COUT]
    const int tid = threadIdx.x;
    const int pl = PL == 1 ? 0 : tid / NB;
    const bool active = PL == 1 || tid < NB * PL;
    float acc[NBT][BE];
#pragma unroll
    for (int k = 0; k < NBT; ++k)
#pragma unroll
        for (int e = 0; e < BE; ++e) acc[k][e] = 0.f;
    for (int i = tid; i < COUT; i += WNT) dbs[i] = 0.f;
    const int tx = (W + WTW - 1) / WTW, ty = (H + WTH - 1) / WTH;
    const long long ntiles = static_cast<long long>(N) * tx * ty;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int n = static_cast<int>(t / (tx * ty));
        const int r = static_cast<int>(t % (tx * ty));
        const int y0 = (r / tx) * WTH, x0 = (r % tx) * WTW;
        __syncthreads();
        for (int i = tid; i < RH * RW * (CIN / 4); i += WNT) {
            const int c4 = i % (CIN / 4), q = i / (CIN / 4);
            const int gy = y0 - P + q / RW, gx = x0 - P + q % RW;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                v = __ldg(reinterpret_cast<const float4*>(x + ((static_cast<size_t>(n) * H + gy) * W + gx) * CIN) + c4);
                if (relu_in) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
            }
            reinterpret_cast<float4*>(xs)[i] = v;
        }
        for (int i = tid; i < NPX * (COUT / 4); i += WNT) {
            const int o4 = i % (COUT / 4), q = i / (COUT / 4);
            const int gy = y0 + q / WTW, gx = x0 + q % WTW;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy < H && gx < W) {
                const size_t idx = ((static_cast<size_t>(n) * H + gy) * W + gx) * COUT;
                v = __ldg(reinterpret_cast<const float4*>(g + idx) + o4);
                if (gm) {
                    const float4 m = __ldg(reinterpret_cast<const float4*>(gm + idx) + o4);
                    v = make_float4(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f, m.z > 0.f ? v.z : 0.f,
                                    m.w > 0.f ? v.w : 0.f);
                }
            }
            reinterpret_cast<float4*>(gs)[i] = v;
        }
        __syncthreads();
        for (int o = tid; o < COUT; o += WNT) {
            float s = 0.f;
            for (int q = 0; q < NPX; ++q) s += gs[q * COUT + o];
            dbs[o] += s;
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < NBT; ++k) {
                const int b = PL == 1 ? tid + k * WNT : tid % NB;
                if (b >= NB) continue;
                const int cb = b % CB, ob = (b / CB) % OB, tap = b / (CB * OB);
                const float* gp = gs + BO * ob;
                const float* xp = xs + ((tap / K) * RW + (tap % K)) * CIN + BI * cb;
#pragma unroll 2
                for (int q = pl; q < NPX; q += PL) {
                    float gv[BO], xv[BI];
#pragma unroll
                    for (int h = 0; h < BO / 4; ++h) {
                        const float4 g4 = *reinterpret_cast<const float4*>(gp + q * COUT + 4 * h);
                        gv[4 * h] = g4.x; gv[4 * h + 1] = g4.y; gv[4 * h + 2] = g4.z; gv[4 * h + 3] = g4.w;
                    }
#pragma unroll
                    for (int h = 0; h < BI / 4; ++h) {
                        const float4 x4 =
                            *reinterpret_cast<const float4*>(xp + ((q / WTW) * RW + (q % WTW)) * CIN + 4 * h);
                        xv[4 * h] = x4.x; xv[4 * h + 1] = x4.y; xv[4 * h + 2] = x4.z; xv[4 * h + 3] = x4.w;
                    }
#pragma unroll
                    for (int i = 0; i < BO; ++i)
#pragma unroll
                        for (int j = 0; j < BI; ++j) acc[k][BI * i + j] = fmaf(gv[i], xv[j], acc[k][BI * i + j]);
                }
            }
        }
    }
    __syncthreads();
    // weight e = (o CIN + c) TAPS + tap of block b, element (i, j): o = BO ob + i, c = BI cb + j
    auto widx = [&](int b, int i, int j) {
        const int cb = b % CB, ob = (b / CB) % OB, tap = b / (CB * OB);
        return ((BO * ob + i) * CIN + BI * cb + j) * TAPS + tap;
    };
    if constexpr (PL == 1) {
#pragma unroll
        for (int k = 0; k < NBT; ++k) {
            const int b = tid + k * WNT;
            if (b >= NB) continue;
#pragma unroll
            for (int e = 0; e < BE; ++e) atomicAdd(dW + widx(b, e / BI, e % BI), acc[k][e]);
        }
    } else {
        float* red = xs;  // the pixel classes' partial sums meet here
        for (int e = tid; e < NW; e += WNT) red[e] = 0.f;
        __syncthreads();
        if (active) {
            const int b = tid % NB;
#pragma unroll
            for (int e = 0; e < BE; ++e) atomicAdd(red + widx(b, e / BI, e % BI), acc[0][e]);
        }
        __syncthreads();
        for (int e = tid; e < NW; e += WNT) atomicAdd(dW + e, red[e]);
    }
    if (db)
        for (int o = tid; o < COUT; o += WNT) atomicAdd(db + o, dbs[o]);
}

// 1x1 layers (no halo): tiles of kP1 pixels, whose NHWC rows are contiguous in
// memory, move between HBM and a shared tile with consecutive threads on
// consecutive float4s (coalesced); the input rectification / mask is applied
// while loading and the output mask while storing, both in that layout.  In
// between one thread per pixel reads its row, the weights ws[c][o] broadcast
// from shared memory; same operand semantics as conv_fwd_kernel with K = 1 and
// the same summation order (bias, then c = 0, 1, ...), so the same values.
// Rows are padded to S = max(C_in, C_out) + 4 floats (conflict-free float4
// row reads); the output rows overwrite the input rows of the same tile.
constexpr int kP1 = 256;  // pixels per tile = threads per CTA

template <int CIN, int COUT>
struct Conv1x1Shape {
    static constexpr int S = (CIN > COUT ? CIN : COUT) + 4;
    static constexpr size_t SMEM = sizeof(float) * (static_cast<size_t>(kP1) * S + CIN * COUT);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kP1) conv1x1_kernel(const float* __restrict__ x, const float* __restrict__ xm,
                                                      int relu_in, size_t npx, const float* __restrict__ w, int tf,
                                                      const float* __restrict__ b, const float* __restrict__ ym,
                                                      float* __restrict__ y) {
    static_assert(CIN % 4 == 0 && COUT % 4 == 0, "float4 channels");
    constexpr int S = Conv1x1Shape<CIN, COUT>::S, CI4 = CIN / 4, CO4 = COUT / 4;
    extern __shared__ float4 smem1[];
    float* rows = reinterpret_cast<float*>(smem1);             // [kP1][S]
    float4* ws4 = smem1 + kP1 * S / 4;                          // [CIN][COUT]
    float* ws = reinterpret_cast<float*>(ws4);
    const int t = threadIdx.x;
    for (int i = t; i < CIN * COUT; i += kP1) {
        const int c = i / COUT, o = i % COUT;
        ws[i] = tf ? __ldg(w + c * COUT + o) : __ldg(w + o * CIN + c);
    }
    const size_t tiles = (npx + kP1 - 1) / kP1;
    for (size_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const size_t p0 = tile * kP1;
        const int np = static_cast<int>(npx - p0 < static_cast<size_t>(kP1) ? npx - p0 : kP1);
        // coalesced input rows -> shared tile (rectified / masked)
        const float4* x4 = reinterpret_cast<const float4*>(x + p0 * CIN);
        const float4* xm4 = xm ? reinterpret_cast<const float4*>(xm + p0 * CIN) : nullptr;
#pragma unroll
        for (int k = 0; k < CI4; ++k) {
            const int i = t + kP1 * k;  // float4 index within the tile
            if (i < np * CI4) {
                float4 v = __ldg(x4 + i);
                if (relu_in) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
                if (xm4) {
                    const float4 m = __ldg(xm4 + i);
                    v = make_float4(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f, m.z > 0.f ? v.z : 0.f,
                                    m.w > 0.f ? v.w : 0.f);
                }
                *reinterpret_cast<float4*>(rows + (i / CI4) * S + 4 * (i % CI4)) = v;
            }
        }
        __syncthreads();
        float xv[CIN];
        if (t < np) {
#pragma unroll
            for (int c4 = 0; c4 < CI4; ++c4) {
                const float4 v = *reinterpret_cast<const float4*>(rows + t * S + 4 * c4);
                xv[4 * c4] = v.x; xv[4 * c4 + 1] = v.y; xv[4 * c4 + 2] = v.z; xv[4 * c4 + 3] = v.w;
            }
        }
        __syncthreads();  // every input row read before the output rows overwrite them
        if (t < np) {
#pragma unroll 2
            for (int o4 = 0; o4 < CO4; ++o4) {
                float4 s = b ? __ldg(reinterpret_cast<const float4*>(b) + o4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < CIN; ++c) {
                    const float4 wv = ws4[c * CO4 + o4];
                    s.x = fmaf(xv[c], wv.x, s.x);
                    s.y = fmaf(xv[c], wv.y, s.y);
                    s.z = fmaf(xv[c], wv.z, s.z);
                    s.w = fmaf(xv[c], wv.w, s.w);
                }
                *reinterpret_cast<float4*>(rows + t * S + 4 * o4) = s;
            }
        }
        __syncthreads();
        // shared tile -> coalesced output rows (masked)
        float4* y4 = reinterpret_cast<float4*>(y + p0 * COUT);
        const float4* ym4 = ym ? reinterpret_cast<const float4*>(ym + p0 * COUT) : nullptr;
#pragma unroll
        for (int k = 0; k < CO4; ++k) {
            const int i = t + kP1 * k;
            if (i < np * CO4) {
                float4 s = *reinterpret_cast<const float4*>(rows + (i / CO4) * S + 4 * (i % CO4));
                if (ym4) {
                    const float4 m = __ldg(ym4 + i);
                    s = make_float4(m.x > 0.f ? s.x : 0.f, m.y > 0.f ? s.y : 0.f, m.z > 0.f ? s.z : 0.f,
                                    m.w > 0.f ? s.w : 0.f);
                }
                y4[i] = s;
            }
        }
        __syncthreads();  // the tile's rows are free for the next tile
    }
}

template <int CIN, int COUT, int K, int CB = CIN, int OB = COUT, int C1 = 0, int POOL = 0, int UPIN = 0,
          int HEAD = 0>
cudaError_t conv_fwd(const float* x, const float* xm, int relu_in, int N, int H, int W, const float* w, int tf,
                     const float* b, const float* ym, float* y, cudaStream_t st, const float* w1 = nullptr,
                     const float* b1 = nullptr, int relu_out = 0, float* yp = nullptr, const float* wh = nullptr,
                     float* vis = nullptr) {
    if constexpr (K == 1 && CB == CIN && OB == COUT && C1 == 0 && !UPIN && !HEAD && CIN * COUT <= 4096) {
        const size_t npx = static_cast<size_t>(N) * H * W;
        if (npx == 0) return cudaSuccess;
        constexpr size_t smem = Conv1x1Shape<CIN, COUT>::SMEM;
        auto kern = conv1x1_kernel<CIN, COUT>;
        static int per_sm = 0;  // resident CTAs per SM, from the shared tile's size
        if (per_sm == 0) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return e;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kP1, smem) != cudaSuccess || per_sm < 1)
                per_sm = 1;
        }
        const size_t tiles = (npx + kP1 - 1) / kP1, cap = static_cast<size_t>(num_sms()) * per_sm;
        kern<<<static_cast<unsigned>(tiles < cap ? tiles : cap), kP1, smem, st>>>(x, xm, relu_in, npx, w, tf, b, ym, y);
        return cudaGetLastError();
    }
    constexpr int P = K / 2, TW = TJ * FwdShape<CB, OB>::PX;
    const size_t smem = sizeof(float) * (CB * (((TH + 2 * P) * (TW + 2 * P)) | 1) + K * K * CB * OB + C1 * COUT);
    auto kern = conv_fwd_kernel<CIN, COUT, K, CB, OB, C1, POOL, UPIN, HEAD>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long tiles = static_cast<long long>(N) * ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
    if (tiles == 0) return cudaSuccess;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    const long long cap = static_cast<long long>(num_sms()) * per_sm;
    const dim3 grid(static_cast<unsigned>(tiles < cap ? tiles : cap), COUT / OB);
    kern<<<grid, NT, smem, st>>>(x, xm, relu_in, N, H, W, w, tf, b, ym, y, w1, b1, relu_out, yp, wh, vis);
    return cudaGetLastError();
}

template <int CIN, int COUT, int K>
cudaError_t conv_wgrad(const float* x, int relu_in, const float* g, const float* gm, int N, int H, int W, float* dW,
                       float* db, cudaStream_t st) {
    constexpr int P = K / 2;
    const size_t smem = sizeof(float) * ((WTH + 2 * P) * (WTW + 2 * P) * CIN + WTH * WTW * COUT + COUT);
    auto kern = conv_wgrad_kernel<CIN, COUT, K>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long tiles = static_cast<long long>(N) * ((W + WTW - 1) / WTW) * ((H + WTH - 1) / WTH);
    if (tiles == 0) return cudaSuccess;
    const long long cap = static_cast<long long>(num_sms()) * 2;
    kern<<<static_cast<int>(tiles < cap ? tiles : cap), WNT, smem, st>>>(x, relu_in, g, gm, N, H, W, dW, db);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pooling / upsampling
// y[n,Y,X,c] = 1/4 sum of relu?(x) over the 2x2 block; H, W of x even
__global__ void pool_fwd_kernel(const float* __restrict__ x, int relu_in, int N, int H, int W, int C,
                                float* __restrict__ y) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t total = static_cast<size_t>(N) * Ho * Wo * C;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % C);
        size_t q = i / C;
        const int X = static_cast<int>(q % Wo); q /= Wo;
        const int Y = static_cast<int>(q % Ho);
        const int n = static_cast<int>(q / Ho);
        float s = 0.f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                float v = x[((static_cast<size_t>(n) * H + 2 * Y + dy) * W + 2 * X + dx) * C + c];
                if (relu_in) v = fmaxf(v, 0.f);
                s += v;
            }
        y[i] = 0.25f * s;
    }
}

// gx[n,y,x,c] (+)= 1/4 gy[n,y/2,x/2,c]
__global__ void pool_adj_kernel(const float* __restrict__ gy, int NH, int W, int c4s, const float* __restrict__ add,
                                float* __restrict__ gx) {
    // rows of the fine grid on grid.y (fine row r = n H + y, its coarse row r / 2:
    // H is even), four channels (one float4) per thread, C / 4 = 2^c4s
    const int C4 = 1 << c4s, per_row = W << c4s;
    const float4* g4 = reinterpret_cast<const float4*>(gy);
    const float4* a4 = reinterpret_cast<const float4*>(add);
    float4* o4 = reinterpret_cast<float4*>(gx);
    for (int r = blockIdx.y; r < NH; r += gridDim.y) {
        const size_t rin = static_cast<size_t>(r >> 1) * ((W >> 1) << c4s);
        const size_t rout = static_cast<size_t>(r) * per_row;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < per_row; t += gridDim.x * blockDim.x) {
            const int x = t >> c4s, c4 = t & (C4 - 1);
            float4 v = __ldg(g4 + rin + ((x >> 1) << c4s) + c4);
            v = make_float4(0.25f * v.x, 0.25f * v.y, 0.25f * v.z, 0.25f * v.w);
            if (a4) {
                const float4 a = __ldg(a4 + rout + t);
                v.x += a.x; v.y += a.y; v.z += a.z; v.w += a.w;
            }
            o4[rout + t] = v;
        }
    }
}

// y[n,y,x,c] = bilinear x2 of lo (H/2 x W/2) (+ skip[n,y,x,c])
__global__ void up_fwd_kernel(const float* __restrict__ lo, const float* __restrict__ skip, int N, int H, int W,
                              int c4s, float* __restrict__ y) {
    // rows of the fine grid on grid.y (r = n H + yy), four channels (one float4)
    // per thread, C / 4 = 2^c4s
    const int Hl = H / 2, Wl = W / 2, C4 = 1 << c4s, per_row = W << c4s;
    const float4* lo4 = reinterpret_cast<const float4*>(lo);
    for (int r = blockIdx.y; r < N * H; r += gridDim.y) {
        const int n = r / H, yy = r - n * H;
        const size_t row = static_cast<size_t>(r) * per_row;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < per_row; t += gridDim.x * blockDim.x) {
            const int x = t >> c4s, c4 = t & (C4 - 1);
            float4 v = up_sample4(lo4, n, Hl, Wl, C4, yy, x, c4);
            if (skip) {
                const float4 sk = __ldg(reinterpret_cast<const float4*>(skip) + row + t);
                v.x += sk.x; v.y += sk.y; v.z += sk.z; v.w += sk.w;
            }
            reinterpret_cast<float4*>(y)[row + t] = v;
        }
    }
}

// Adjoint of the bilinear x2 upsampling in gather form: each coarse pixel
// sums the fine-grid cotangents of the (at most 4 x 4) fine pixels whose taps
// reach it, with those taps' weights.
__global__ void up_adj_kernel(const float* __restrict__ g, int N, int H, int W, int c4s, float* __restrict__ glo) {
    // coarse rows on grid.y (R = n Hl + Y), four channels (one float4) per
    // thread, C / 4 = 2^c4s.  Only fine indices 2X - 1 .. 2X + 2 reach coarse
    // X (bilin_tap clamps at the borders, where the clamped tap also falls in
    // that window): their 16 cotangents are loaded together from clamped
    // (always valid) addresses, and the terms of nonzero weight are summed in
    // row-major order.
    const int Hl = H / 2, Wl = W / 2, C4 = 1 << c4s, per_row = Wl << c4s;
    const float4* g4 = reinterpret_cast<const float4*>(g);
    for (int R = blockIdx.y; R < N * Hl; R += gridDim.y) {
        const int n = R / Hl, Y = R - n * Hl;
        float wy[4];
        int yc[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int yy = 2 * Y - 1 + d;
            yc[d] = yy < 0 ? 0 : (yy >= H ? H - 1 : yy);
            const BilinTap ty = bilin_tap(yc[d], Hl);
            wy[d] = (yy < 0 || yy >= H) ? 0.f : (ty.i0 == Y ? ty.w0 : 0.f) + (ty.i1 == Y ? ty.w1 : 0.f);
        }
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < per_row; t += gridDim.x * blockDim.x) {
            const int X = t >> c4s, c4 = t & (C4 - 1);
            float wx[4];
            int xc[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int xx = 2 * X - 1 + d;
                xc[d] = xx < 0 ? 0 : (xx >= W ? W - 1 : xx);
                const BilinTap tx = bilin_tap(xc[d], Wl);
                wx[d] = (xx < 0 || xx >= W) ? 0.f : (tx.i0 == X ? tx.w0 : 0.f) + (tx.i1 == X ? tx.w1 : 0.f);
            }
            float4 v[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    v[i][j] = __ldg(g4 + ((static_cast<size_t>(n) * H + yc[i]) * W + xc[j]) * C4 + c4);
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (wy[i] == 0.f) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (wx[j] == 0.f) continue;
                    const float wt = wy[i] * wx[j];
                    s.x += wt * v[i][j].x; s.y += wt * v[i][j].y; s.z += wt * v[i][j].z; s.w += wt * v[i][j].w;
                }
            }
            reinterpret_cast<float4*>(glo)[static_cast<size_t>(R) * per_row + t] = s;
        }
    }
}

__global__ void relu_copy_kernel(const float* __restrict__ x, size_t n, float* __restrict__ y) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        y[i] = fmaxf(x[i], 0.f);
}

// ------------------------------------------------------------------ head, loss
// vis = sigmoid(bh + sum_c wh[c] relu(a1[c])), C = 16
__global__ void head_fwd_kernel(const float* __restrict__ a1, const float* __restrict__ wh, size_t npx,
                                float* __restrict__ vis) {
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < npx;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float l = __ldg(wh + 16);
#pragma unroll
        for (int c = 0; c < 16; ++c) l = fmaf(__ldg(wh + c), fmaxf(a1[p * 16 + c], 0.f), l);
        vis[p] = sigmoidf_acc(l);
    }
}

// g_logit = g_vis vis (1 - vis); g_a1[c] = wh[c] g_logit (a1[c] > 0);
// dwh[c] += sum g_logit relu(a1[c]); dbh += sum g_logit
__global__ void head_bwd_kernel(const float* __restrict__ a1, const float* __restrict__ vis,
                                const float* __restrict__ gvis, const float* __restrict__ wh, size_t npx,
                                float* __restrict__ ga1, float* __restrict__ dwh, float* __restrict__ slots) {
    __shared__ float red[17][8];
    float part[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) part[c] = 0.f;
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < npx;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float v = vis[p];
        const float gl = gvis[p] * v * (1.f - v);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(a1 + p * 16) + c4);
            const float av[4] = {a.x, a.y, a.z, a.w};
            float gv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * c4 + e;
                gv[e] = (av[e] > 0.f) ? __ldg(wh + c) * gl : 0.f;
                part[c] = fmaf(gl, fmaxf(av[e], 0.f), part[c]);
            }
            reinterpret_cast<float4*>(ga1 + p * 16)[c4] = make_float4(gv[0], gv[1], gv[2], gv[3]);
        }
        part[16] += gl;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 17; ++c) {
        float s = part[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[c][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        float s = 0.f;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) s += red[threadIdx.x][w];
        if (slots) slots[blockIdx.x * 17 + threadIdx.x] = s;  // slot of this block, summed in order afterwards
        else atomicAdd(dwh + threadIdx.x, s);
    }
}

// Eq. 2 with the L1 term: per item b, alpha mean|x0 - target| + sum_i alpha mean|x0 - x_i|
// (x_i detached), averaged over the B items.  vis is [T][B][npx] (instance 0
// first).  Writes g_vis for x0 ([B][npx]) and adds the loss to *loss.
__global__ void loss_l1_kernel(const float* __restrict__ vis, const float* __restrict__ target, int B, int T,
                               size_t npx, float alpha, float* __restrict__ gvis, float* __restrict__ loss) {
    __shared__ float red[8];
    const float scale = alpha / (static_cast<float>(npx) * B);
    float part = 0.f;
    const size_t total = static_cast<size_t>(B) * npx;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float x0 = vis[i];
        float d = x0 - target[i];
        float g = (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
        float l = fabsf(d);
        for (int t = 1; t < T; ++t) {
            const float xi = vis[static_cast<size_t>(t) * total + i];
            d = x0 - xi;
            g += (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
            l += fabsf(d);
        }
        gvis[i] = scale * g;
        part += l;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) s += red[w];
        atomicAdd(loss, s * scale);
    }
}

// Adam (Kingma & Ba 2015) with bias correction; step >= 1
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Features of a batch of views, NHWC [N][H][W][4]; one GatherParams per view.
__global__ void features_batch_kernel(const GatherParams* __restrict__ gp, int N, int H, int W,
                                      float* __restrict__ feat) {
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t total = npx * N;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int n = static_cast<int>(i / npx);
        const size_t p = i % npx;
        const GatherParams& g = gp[n];
        const float4 P = __ldg(g.pos4 + p);
        const float4 Nn = __ldg(g.nrm4 + p);
        PixelGather o = gather_pixel(g, P, Nn);
        reinterpret_cast<float4*>(feat)[i] = make_float4(o.f[0], o.f[1], o.f[2], o.f[3]);
    }
}

// grid of the row kernels: rows on y (at most 65,535, grid-stride beyond),
// about 8 CTAs per SM in all
static dim3 row_grid(int rows, int per_row) {
    const int gx = (per_row + 255) / 256;
    const int want_y = num_sms() * 8 / (gx > 0 ? gx : 1);
    int gy = rows < want_y ? rows : want_y;
    gy = gy < 1 ? 1 : (gy > 65535 ? 65535 : gy);
    return dim3(gx < 1 ? 1 : gx, gy);
}
static int log2_c4(int C) {  // C / 4 = 2^result (C a power of two, >= 4)
    int s = 0;
    while ((4 << s) < C) ++s;
    return s;
}

static int ew_grid(size_t n) {
    const size_t b = (n + 255) / 256;
    const size_t cap = static_cast<size_t>(num_sms()) * 8;
    return static_cast<int>(b < 1 ? 1 : (b < cap ? b : cap));
}

// ------------------------------------------------------------------ network driver
struct Level {  // offsets into the canonical vector
    const float *w3, *b3, *w1, *b1;
    float *dw3, *db3, *dw1, *db1;
};

static Level level(const float* th, float* gr, int l3, int l1) {
    const LayerOffsets o = layer_offsets();
    return {th + o.w[l3], th + o.b[l3], th + o.w[l1], th + o.b[l1],
            gr ? gr + o.w[l3] : nullptr, gr ? gr + o.b[l3] : nullptr,
            gr ? gr + o.w[l1] : nullptr, gr ? gr + o.b[l1] : nullptr};
}

#define NSM_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

size_t workspace_floats(int N, int Nb, int H, int W) {
    const size_t p0 = static_cast<size_t>(H) * W, p1 = p0 / 4, p2 = p0 / 16;
    size_t f = 0;
    f += N * p0 * 4;            // feat
    f += N * p1 * 16;           // e0
    f += N * p1 * 32;           // s1
    f += N * p2 * 32;           // p1
    f += N * p2 * 32;           // bo
    f += N * p1 * 16;           // d1
    f += N * p0;                // vis
    f += Nb * p0;               // g_vis
    // per-level scratch (largest level: level 0): x_in, a3, a1, g_a1, g_a3, g_x, g_low, g_skip
    f += Nb * p0 * 16 * 6 + Nb * p1 * 32 * 2;
    f += Nb * p0 * 16;          // conv scratch (level-0 1x1 input gradient)
    f += kWgPartFloats;         // weight-gradient partial sums
    return f + 128;
}

Buffers carve(float* base, int N, int Nb, int H, int W) {
    const size_t p0 = static_cast<size_t>(H) * W, p1 = p0 / 4, p2 = p0 / 16;
    Buffers b{};
    float* q = base;
    auto take = [&](size_t n) { float* r = q; q += (n + 63) / 64 * 64; return r; };
    b.feat = take(N * p0 * 4);
    b.e0 = take(N * p1 * 16);
    b.s1 = take(N * p1 * 32);
    b.p1 = take(N * p2 * 32);
    b.bo = take(N * p2 * 32);
    b.d1 = take(N * p1 * 16);
    b.vis = take(N * p0);
    b.gvis = take(Nb * p0);
    b.xin = take(Nb * p0 * 16);
    b.a3 = take(Nb * p0 * 16);
    b.a1 = take(Nb * p0 * 16);
    b.ga1 = take(Nb * p0 * 16);
    b.ga3 = take(Nb * p0 * 16);
    b.gx = take(Nb * p0 * 16);
    b.glo = take(Nb * p1 * 32);
    b.gskip = take(Nb * p1 * 32);
    b.gtmp = take(Nb * p0 * 16);
    b.wpart = take(kWgPartFloats);
    return b;
}

// Forward of N views (features already in b.feat) keeping the level
// checkpoints; uses xin / a3 / a1 of the scratch, sized for Nb views, in
// chunks of Nb views.
cudaError_t forward(const float* th, const Buffers& b, int N, int Nb, int H, int W, cudaStream_t st) {
    const size_t p0 = static_cast<size_t>(H) * W, p1 = p0 / 4, p2 = p0 / 16;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    const LayerOffsets o = layer_offsets();
    for (int n0 = 0; n0 < N; n0 += Nb) {
        const int n = (N - n0) < Nb ? (N - n0) : Nb;
        const float* feat = b.feat + n0 * p0 * 4;
        float* e0 = b.e0 + n0 * p1 * 16;
        float* s1 = b.s1 + n0 * p1 * 32;
        float* pp1 = b.p1 + n0 * p2 * 32;
        float* bo = b.bo + n0 * p2 * 32;
        float* d1 = b.d1 + n0 * p1 * 16;
        float* vis = b.vis + n0 * p0;
        Level L;
        // level 0 encoder
        L = level(th, nullptr, ENC0_3, ENC0_1);
        NSM_TRY((conv_fwd<4, 16, 3, 4, 16, 16, 1>(feat, nullptr, 0, n, H, W, L.w3, 0, L.b3, nullptr, nullptr, st, L.w1,
                                                  L.b1, 0, e0)));
        // level 1 encoder
        L = level(th, nullptr, ENC1_3, ENC1_1);
        // the decoder skip relu(a1) of level 1 is written directly
        NSM_TRY((conv_fwd<16, 32, 3, 16, 32, 32, 1>(e0, nullptr, 0, n, H1, W1, L.w3, 0, L.b3, nullptr, s1, st, L.w1,
                                                    L.b1, 1, pp1)));
        // bottleneck
        L = level(th, nullptr, BOTT_3, BOTT_1);
        NSM_TRY((conv_fwd<32, 64, 3, 16, 64, 32>(pp1, nullptr, 0, n, H2, W2, L.w3, 0, L.b3, nullptr, bo, st, L.w1, L.b1,
                                                 1)));
        // level 1 decoder
        L = level(th, nullptr, DEC1_3, DEC1_1);
        NSM_TRY((conv_fwd<32, 32, 3, 16, 32, 16, 0, 1>(bo, s1, 0, n, H1, W1, L.w3, 0, L.b3, nullptr, d1, st, L.w1, L.b1,
                                                       1)));  // input up(bo) + s1
        // level 0 decoder + head
        L = level(th, nullptr, DEC0_3, DEC0_1);
        NSM_TRY((conv_fwd<16, 16, 3, 16, 16, 16, 0, 1, 1>(d1, nullptr, 0, n, H, W, L.w3, 0, L.b3, nullptr, nullptr, st,
                                                          L.w1, L.b1, 0, nullptr, th + o.w[HEAD], vis)));  // up(d1)
        NSM_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// Backward of the first Nb views (cotangent b.gvis) into grad (canonical
// layout, accumulated), recomputing each level from its checkpoint.
// With gfeat != nullptr also the feature gradient [Nb][H][W][4].  With img
// != nullptr (the conv3_pack images of th) the 3x3 recomputations (with the
// level's 1x1 in their epilogue) and data gradients (conv3_tc) and the 3x3
// weight gradients (wgrad_tc) run on the tensor cores, every weight gradient
// (the head's by per-block slots) reduced in a fixed order; else the FP32
// kernels.  The 1x1 weight gradients run on CUDA cores in both forms
// (wgrad1x1_tiles: memory-bound, fixed order).
cudaError_t backward(const float* th, float* grad, const Buffers& b, int Nb, int H, int W, float* gfeat,
                     cudaStream_t st, const uint4* img, int* err) {
    const Conv3Images im = conv3_images();
    auto I = [&](int i) { return img + im.off[i]; };
    const size_t p0 = static_cast<size_t>(H) * W, p1 = p0 / 4, p2 = p0 / 16;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    const LayerOffsets o = layer_offsets();
    const int n = Nb;
    Level L;
    // ---- level 0 decoder + head: recompute x = up(d1), a3, a1
    L = level(th, grad, DEC0_3, DEC0_1);
    up_fwd_kernel<<<row_grid(n * H, W * 4), 256, 0, st>>>(b.d1, nullptr, n, H, W, log2_c4(16), b.xin);
    if (img) {
        NSM_TRY(conv3_tc(16, 16, b.xin, n, H, W, I(8), L.b3, b.a3, err, st, L.w1, L.b1, 16, b.a1));
    } else {
        NSM_TRY((conv_fwd<16, 16, 3>(b.xin, nullptr, 0, n, H, W, L.w3, 0, L.b3, nullptr, b.a3, st)));
        NSM_TRY((conv_fwd<16, 16, 1>(b.a3, nullptr, 1, n, H, W, L.w1, 0, L.b1, nullptr, b.a1, st)));
    }
    {
        const int hb = ew_grid(n * p0);
        head_bwd_kernel<<<hb, 256, 0, st>>>(b.a1, b.vis, b.gvis, th + o.w[HEAD], n * p0, b.ga1, grad + o.w[HEAD],
                                            img ? b.wpart : nullptr);
        if (img) NSM_TRY(slot_reduce(b.wpart, hb, 17, 17, grad + o.w[HEAD], nullptr, st));
    }
    NSM_TRY(wgrad1x1_tiles(16, 16, b.a3, 1, b.ga1, nullptr, n, H, W, b.wpart, L.dw1, L.db1, st));  // FP32, both forms
    NSM_TRY((conv_fwd<16, 16, 1>(b.ga1, nullptr, 0, n, H, W, L.w1, 1, nullptr, b.a3, b.ga3, st)));
    if (img) NSM_TRY(wgrad_tc(16, 16, 3, b.xin, 0, b.ga3, nullptr, n, H, W, b.wpart, L.dw3, L.db3, err, st));
    else NSM_TRY((conv_wgrad<16, 16, 3>(b.xin, 0, b.ga3, nullptr, n, H, W, L.dw3, L.db3, st)));
    if (img) NSM_TRY(conv3_tc(16, 16, b.ga3, n, H, W, I(9), nullptr, b.gx, err, st));
    else NSM_TRY((conv_fwd<16, 16, 3>(b.ga3, nullptr, 0, n, H, W, L.w3, 1, nullptr, nullptr, b.gx, st)));
    up_adj_kernel<<<row_grid(n * H1, W1 * 4), 256, 0, st>>>(b.gx, n, H, W, log2_c4(16), b.glo);  // g d1 [n][H1][W1][16]
    // ---- level 1 decoder: recompute x = up(bo) + s1, a3, a1
    L = level(th, grad, DEC1_3, DEC1_1);
    up_fwd_kernel<<<row_grid(n * H1, W1 * 8), 256, 0, st>>>(b.bo, b.s1, n, H1, W1, log2_c4(32), b.xin);
    if (img) {
        NSM_TRY(conv3_tc(32, 32, b.xin, n, H1, W1, I(6), L.b3, b.a3, err, st, L.w1, L.b1, 16, b.a1));
    } else {
        NSM_TRY((conv_fwd<32, 32, 3, 16>(b.xin, nullptr, 0, n, H1, W1, L.w3, 0, L.b3, nullptr, b.a3, st)));
        NSM_TRY((conv_fwd<32, 16, 1>(b.a3, nullptr, 1, n, H1, W1, L.w1, 0, L.b1, nullptr, b.a1, st)));
    }
    // g_a1 = g_d1 (a1 > 0)
    NSM_TRY(wgrad1x1_tiles(32, 16, b.a3, 1, b.glo, b.a1, n, H1, W1, b.wpart, L.dw1, L.db1, st));  // FP32, both forms
    NSM_TRY((conv_fwd<16, 32, 1>(b.glo, b.a1, 0, n, H1, W1, L.w1, 1, nullptr, b.a3, b.ga3, st)));
    if (img) NSM_TRY(wgrad_tc(32, 32, 3, b.xin, 0, b.ga3, nullptr, n, H1, W1, b.wpart, L.dw3, L.db3, err, st));
    else NSM_TRY((conv_wgrad<32, 32, 3>(b.xin, 0, b.ga3, nullptr, n, H1, W1, L.dw3, L.db3, st)));
    if (img) NSM_TRY(conv3_tc(32, 32, b.ga3, n, H1, W1, I(7), nullptr, b.gskip, err, st));  // g x1
    else NSM_TRY((conv_fwd<32, 32, 3, 16>(b.ga3, nullptr, 0, n, H1, W1, L.w3, 1, nullptr, nullptr, b.gskip, st)));
    up_adj_kernel<<<row_grid(n * H2, W2 * 8), 256, 0, st>>>(b.gskip, n, H1, W1, log2_c4(32), b.glo);  // g bo [n][H2][W2][32]
    // ---- bottleneck: recompute a3 = conv3(p1), a1
    L = level(th, grad, BOTT_3, BOTT_1);
    if (img) {
        NSM_TRY(conv3_tc(32, 64, b.p1, n, H2, W2, I(4), L.b3, b.a3, err, st, L.w1, L.b1, 32, b.a1));
    } else {
        NSM_TRY((conv_fwd<32, 64, 3, 16>(b.p1, nullptr, 0, n, H2, W2, L.w3, 0, L.b3, nullptr, b.a3, st)));
        NSM_TRY((conv_fwd<64, 32, 1>(b.a3, nullptr, 1, n, H2, W2, L.w1, 0, L.b1, nullptr, b.a1, st)));
    }
    NSM_TRY(wgrad1x1_tiles(64, 32, b.a3, 1, b.glo, b.a1, n, H2, W2, b.wpart, L.dw1, L.db1, st));  // FP32, both forms
    NSM_TRY((conv_fwd<32, 64, 1>(b.glo, b.a1, 0, n, H2, W2, L.w1, 1, nullptr, b.a3, b.ga3, st)));
    if (img) NSM_TRY(wgrad_tc(32, 64, 3, b.p1, 0, b.ga3, nullptr, n, H2, W2, b.wpart, L.dw3, L.db3, err, st));
    else NSM_TRY((conv_wgrad<32, 64, 3>(b.p1, 0, b.ga3, nullptr, n, H2, W2, L.dw3, L.db3, st)));
    if (img) NSM_TRY(conv3_tc(64, 32, b.ga3, n, H2, W2, I(5), nullptr, b.gx, err, st));  // g p1
    else NSM_TRY((conv_fwd<64, 32, 3, 16>(b.ga3, nullptr, 0, n, H2, W2, L.w3, 1, nullptr, nullptr, b.gx, st)));
    // ---- level 1 encoder: g_h1 = pool_adj(g p1) + g s1 ; recompute a3 = conv3(e0), a1
    L = level(th, grad, ENC1_3, ENC1_1);
    pool_adj_kernel<<<row_grid(n * H1, W1 * 8), 256, 0, st>>>(b.gx, n * H1, W1, log2_c4(32), b.gskip, b.glo);
    if (img) {
        NSM_TRY(conv3_tc(16, 32, b.e0, n, H1, W1, I(2), L.b3, b.a3, err, st, L.w1, L.b1, 32, b.a1));
    } else {
        NSM_TRY((conv_fwd<16, 32, 3>(b.e0, nullptr, 0, n, H1, W1, L.w3, 0, L.b3, nullptr, b.a3, st)));
        NSM_TRY((conv_fwd<32, 32, 1>(b.a3, nullptr, 1, n, H1, W1, L.w1, 0, L.b1, nullptr, b.a1, st)));
    }
    NSM_TRY(wgrad1x1_tiles(32, 32, b.a3, 1, b.glo, b.a1, n, H1, W1, b.wpart, L.dw1, L.db1, st));  // FP32, both forms
    NSM_TRY((conv_fwd<32, 32, 1>(b.glo, b.a1, 0, n, H1, W1, L.w1, 1, nullptr, b.a3, b.ga3, st)));
    if (img) NSM_TRY(wgrad_tc(16, 32, 3, b.e0, 0, b.ga3, nullptr, n, H1, W1, b.wpart, L.dw3, L.db3, err, st));
    else NSM_TRY((conv_wgrad<16, 32, 3>(b.e0, 0, b.ga3, nullptr, n, H1, W1, L.dw3, L.db3, st)));
    if (img) NSM_TRY(conv3_tc(32, 16, b.ga3, n, H1, W1, I(3), nullptr, b.gx, err, st));  // g e0
    else NSM_TRY((conv_fwd<32, 16, 3>(b.ga3, nullptr, 0, n, H1, W1, L.w3, 1, nullptr, nullptr, b.gx, st)));
    // ---- level 0 encoder: g_h1 = pool_adj(g e0); recompute a3 = conv3(feat), a1
    L = level(th, grad, ENC0_3, ENC0_1);
    pool_adj_kernel<<<row_grid(n * H, W * 4), 256, 0, st>>>(b.gx, n * H, W, log2_c4(16), nullptr, b.gtmp);
    if (img) {
        NSM_TRY(conv3_tc(4, 16, b.feat, n, H, W, I(0), L.b3, b.a3, err, st, L.w1, L.b1, 16, b.a1));
    } else {
        NSM_TRY((conv_fwd<4, 16, 3>(b.feat, nullptr, 0, n, H, W, L.w3, 0, L.b3, nullptr, b.a3, st)));
        NSM_TRY((conv_fwd<16, 16, 1>(b.a3, nullptr, 1, n, H, W, L.w1, 0, L.b1, nullptr, b.a1, st)));
    }
    NSM_TRY(wgrad1x1_tiles(16, 16, b.a3, 1, b.gtmp, b.a1, n, H, W, b.wpart, L.dw1, L.db1, st));  // FP32, both forms
    NSM_TRY((conv_fwd<16, 16, 1>(b.gtmp, b.a1, 0, n, H, W, L.w1, 1, nullptr, b.a3, b.ga3, st)));
    if (img) NSM_TRY(wgrad_tc(4, 16, 3, b.feat, 0, b.ga3, nullptr, n, H, W, b.wpart, L.dw3, L.db3, err, st));
    else NSM_TRY((conv_wgrad<4, 16, 3>(b.feat, 0, b.ga3, nullptr, n, H, W, L.dw3, L.db3, st)));
    if (gfeat && img) NSM_TRY(conv3_tc(16, 4, b.ga3, n, H, W, I(1), nullptr, gfeat, err, st));
    else if (gfeat) NSM_TRY((conv_fwd<16, 4, 3>(b.ga3, nullptr, 0, n, H, W, L.w3, 1, nullptr, nullptr, gfeat, st)));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ layers of the deeper networks
// Forward layers by runtime shape for the 2- to 7-level networks (Sec. 3.6):
// the (C_in, C_out, k) of their layer tables, weights pre-transposed to
// [tap][C_in][C_out] (transpose_to_tap_major).  Layers with 64 or more
// channels in or out are staged in 32-channel input chunks and computed in
// blocks of 64 outputs; where that gives fewer than two CTAs per SM (the
// coarse levels: few pixels, many channels) they take blocks of 16 outputs
// and 16-channel chunks instead (4 pixels per thread, ~51 KB of shared
// memory, several CTAs per SM).
cudaError_t conv_layer(int cin, int cout, int k, const float* x, int relu_in, int N, int H, int W, const float* w,
                       const float* b, float* y, cudaStream_t st) {
    const long long t64 = static_cast<long long>(N) * ((W + 31) / 32) * ((H + TH - 1) / TH) * (cout >= 64 ? cout / 64 : 1);
    const bool narrow = t64 < 2LL * num_sms();
#define NSM_L(ci, co, kk, cb, ob)                                                                           \
    if (cin == ci && cout == co && k == kk)                                                                 \
        return conv_fwd<ci, co, kk, cb, ob>(x, nullptr, relu_in, N, H, W, w, 2, b, nullptr, y, st);
#define NSM_W(ci, co, kk, cb, ob)                                                                           \
    if (cin == ci && cout == co && k == kk)                                                                 \
        return narrow ? conv_fwd<ci, co, kk, 16, 16>(x, nullptr, relu_in, N, H, W, w, 2, b, nullptr, y, st)  \
                      : conv_fwd<ci, co, kk, cb, ob>(x, nullptr, relu_in, N, H, W, w, 2, b, nullptr, y, st);
    NSM_L(4, 16, 3, 4, 16) NSM_L(16, 16, 1, 16, 16) NSM_L(16, 16, 3, 16, 16) NSM_L(16, 32, 3, 16, 32)
    NSM_L(32, 32, 1, 32, 32) NSM_L(32, 32, 3, 32, 32) NSM_L(32, 16, 1, 32, 16) NSM_W(32, 64, 3, 32, 64)
    NSM_W(64, 64, 1, 64, 64) NSM_W(64, 64, 3, 16, 64) NSM_W(64, 32, 1, 64, 32) NSM_W(64, 128, 3, 16, 64)
    NSM_W(128, 128, 1, 16, 64) NSM_W(128, 128, 3, 16, 64) NSM_W(128, 64, 1, 16, 64) NSM_W(128, 256, 3, 16, 64)
    NSM_W(256, 128, 1, 16, 64) NSM_W(256, 256, 1, 16, 64) NSM_W(256, 256, 3, 16, 64) NSM_W(256, 512, 3, 16, 64)
    NSM_W(512, 512, 1, 16, 64) NSM_W(512, 512, 3, 16, 64) NSM_W(512, 256, 1, 16, 64) NSM_W(512, 1024, 3, 16, 64)
    NSM_W(1024, 512, 1, 16, 64)
#undef NSM_W
#undef NSM_L
    return cudaErrorInvalidValue;
}

// wt[(tap C_in + c) C_out + o] = w[(o C_in + c) k^2 + tap] for one layer
__global__ void transpose_tap_major_kernel(const float* __restrict__ w, int cin, int cout, int kk,
                                           float* __restrict__ wt) {
    const size_t n = static_cast<size_t>(cin) * cout * kk;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int o = static_cast<int>(i % cout);
        const size_t r = i / cout;
        const int c = static_cast<int>(r % cin), tap = static_cast<int>(r / cin);
        wt[i] = __ldg(w + (static_cast<size_t>(o) * cin + c) * kk + tap);
    }
}

cudaError_t transpose_to_tap_major(const float* w, int cin, int cout, int k, float* wt, cudaStream_t st) {
    transpose_tap_major_kernel<<<ew_grid(static_cast<size_t>(cin) * cout * k * k), 256, 0, st>>>(w, cin, cout, k * k,
                                                                                                 wt);
    return cudaGetLastError();
}

// Levels of the deeper networks with the shapes of the 3-level network's
// levels 0 and 1 run as the training forward's fused kernels (3x3 weights
// tap-major, 1x1 weights OIHW).  Encoder: skip (nullable) = relu(1x1), pooled =
// its 2x2 average.  Decoder: y (nullable) = 1x1 of the 3x3 of up(lo) + skip
// (nullable), rectified with relu_out; with vis (16 outputs) also the head.
bool enc_level_fusable(int cin, int cout) { return (cin == 4 && cout == 16) || (cin == 16 && cout == 32); }
bool dec_level_fusable(int cin, int cout1) { return (cin == 32 && cout1 == 16) || (cin == 16 && cout1 == 16); }

cudaError_t enc_level_fused(int cin, int cout, const float* x, int N, int H, int W, const float* wt3, const float* b3,
                            const float* w1, const float* b1, float* skip, float* pooled, cudaStream_t st) {
    if (cin == 4 && cout == 16)
        return conv_fwd<4, 16, 3, 4, 16, 16, 1>(x, nullptr, 0, N, H, W, wt3, 2, b3, nullptr, skip, st, w1, b1, 1,
                                                pooled);
    if (cin == 16 && cout == 32)
        return conv_fwd<16, 32, 3, 16, 32, 32, 1>(x, nullptr, 0, N, H, W, wt3, 2, b3, nullptr, skip, st, w1, b1, 1,
                                                  pooled);
    return cudaErrorInvalidValue;
}

cudaError_t dec_level_fused(int cin, int cout1, const float* lo, const float* skip, int N, int H, int W,
                            const float* wt3, const float* b3, const float* w1, const float* b1, int relu_out, float* y,
                            const float* wh, float* vis, cudaStream_t st) {
    if (cin == 32 && cout1 == 16)
        return conv_fwd<32, 32, 3, 16, 32, 16, 0, 1>(lo, skip, 0, N, H, W, wt3, 2, b3, nullptr, y, st, w1, b1, relu_out);
    if (cin == 16 && cout1 == 16 && vis)
        return conv_fwd<16, 16, 3, 16, 16, 16, 0, 1, 1>(lo, skip, 0, N, H, W, wt3, 2, b3, nullptr, y, st, w1, b1,
                                                         relu_out, nullptr, wh, vis);
    if (cin == 16 && cout1 == 16)
        return conv_fwd<16, 16, 3, 16, 16, 16, 0, 1>(lo, skip, 0, N, H, W, wt3, 2, b3, nullptr, y, st, w1, b1, relu_out);
    return cudaErrorInvalidValue;
}

cudaError_t pool_relu(const float* x, int N, int H, int W, int C, float* y, cudaStream_t st) {
    pool_fwd_kernel<<<ew_grid(static_cast<size_t>(N) * (H / 2) * (W / 2) * C), 256, 0, st>>>(x, 1, N, H, W, C, y);
    return cudaGetLastError();
}

cudaError_t up_add(const float* lo, const float* skip, int N, int H, int W, int C, float* y, cudaStream_t st) {
    if (C < 4 || (C & (C - 1)) != 0) return cudaErrorInvalidValue;  // a power of two
    up_fwd_kernel<<<row_grid(N * H, W * (C / 4)), 256, 0, st>>>(lo, skip, N, H, W, log2_c4(C), y);
    return cudaGetLastError();
}

cudaError_t relu_copy(const float* x, size_t n, float* y, cudaStream_t st) {
    relu_copy_kernel<<<ew_grid(n), 256, 0, st>>>(x, n, y);
    return cudaGetLastError();
}

cudaError_t head(const float* a1, const float* wh, size_t npx, float* vis, cudaStream_t st) {
    head_fwd_kernel<<<ew_grid(npx), 256, 0, st>>>(a1, wh, npx, vis);
    return cudaGetLastError();
}

cudaError_t features_batch(const GatherParams* dev_params, int N, int H, int W, float* feat, cudaStream_t st) {
    const size_t total = static_cast<size_t>(N) * H * W;
    if (total == 0) return cudaSuccess;
    features_batch_kernel<<<ew_grid(total), 256, 0, st>>>(dev_params, N, H, W, feat);
    return cudaGetLastError();
}

cudaError_t loss_l1(const float* vis, const float* target, int B, int T, size_t npx, float alpha, float* gvis,
                    float* loss, cudaStream_t st) {
    loss_l1_kernel<<<ew_grid(static_cast<size_t>(B) * npx), 256, 0, st>>>(vis, target, B, T, npx, alpha, gvis, loss);
    return cudaGetLastError();
}

cudaError_t adam(float* theta, const float* grad, float* m, float* v, size_t n, float lr, float b1, float b2,
                 float eps, int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, static_cast<float>(step));
    const float c2 = 1.f - powf(b2, static_cast<float>(step));
    adam_kernel<<<ew_grid(n), 256, 0, st>>>(theta, grad, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace tr
}  // namespace nsm
