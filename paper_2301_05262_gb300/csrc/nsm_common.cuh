// Shared device-side pieces of the GB300 Neural Shadow Mapping path:
// the per-pixel shadow-map gather (Sec. 3.1, 3.2, Fig. 2) and small helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nsm {

// Emitter, camera and shadow-map description, passed by value as a kernel
// parameter (lives in the constant bank: broadcast to every thread).
struct GatherParams {
    float M[16];        // world -> light clip, row-major
    float L[3];         // emitter centre
    float C[3];         // camera centre
    float r_hat;        // emitter-size input (DC offset on c_e)
    float z_far;        // depth read outside the map
    float beta;         // relative depth bias
    float radius;       // emitter radius (blocker window)
    float tan_half_fov; // map frustum (blocker window)
    float Ws_f, Hs_f;   // map size as floats (exact, <= 2^24)
    float half_Ws;      // 0.5 * Ws
    int Ws, Hs;
    int H, W;
    const float4* __restrict__ pos4;
    const float4* __restrict__ nrm4;
    const float* __restrict__ sm;
    // Feature perturbation of the sensitivity analysis (Sec. 3.2, Eq. 1): when
    // set, feature channel eps_ch of pixel p gets eps_scale * feat_eps[p] added
    // in the gather (FP32 and BF16 forms); null otherwise
    const float* __restrict__ feat_eps;
    float eps_scale;
    int eps_ch;
};

// Texel choice for world position P, binary32 with the operation order that
// defines it:  clip_r = ((M[r][0] Px + M[r][1] Py) + M[r][2] Pz) + M[r][3];
// ndc = clip.xy / clip.w; u = ndc * 0.5 + 0.5; (i, j) = floor(u * (Ws, Hs)).
// Every product and sum is rounded separately (no FMA contraction).
// Returns the texel index j * Ws + i, or -1 outside the frustum / map.
__device__ __forceinline__ int texel_index(const GatherParams& g, float px, float py, float pz,
                                           int* oi = nullptr, int* oj = nullptr) {
    auto row = [&](int r) {
        const float* m = g.M + 4 * r;
        float s = __fadd_rn(__fmul_rn(m[0], px), __fmul_rn(m[1], py));
        s = __fadd_rn(s, __fmul_rn(m[2], pz));
        return __fadd_rn(s, m[3]);
    };
    const float cx = row(0), cy = row(1), cw = row(3);
    if (!(cw > 0.0f)) return -1;
    const float nx = __fdiv_rn(cx, cw);
    const float ny = __fdiv_rn(cy, cw);
    const float u = __fadd_rn(__fmul_rn(nx, 0.5f), 0.5f);
    const float v = __fadd_rn(__fmul_rn(ny, 0.5f), 0.5f);
    const float fi = floorf(__fmul_rn(u, g.Ws_f));
    const float fj = floorf(__fmul_rn(v, g.Hs_f));
    if (!(fi >= 0.0f && fi < g.Ws_f && fj >= 0.0f && fj < g.Hs_f)) return -1;
    const int i = static_cast<int>(fi), j = static_cast<int>(fj);
    if (oi) *oi = i;
    if (oj) *oj = j;
    return j * g.Ws + i;
}

// z_f = sqrt((dx dx + dy dy) + dz dz), d = L - P, binary32 without contraction.
__device__ __forceinline__ float emitter_distance(const GatherParams& g, float px, float py, float pz) {
    const float dx = __fsub_rn(g.L[0], px), dy = __fsub_rn(g.L[1], py), dz = __fsub_rn(g.L[2], pz);
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    s = __fadd_rn(s, __fmul_rn(dz, dz));
    return __fsqrt_rn(s);
}

// Hard depth test: lit iff z_f <= z + beta z_f (binary32).
__device__ __forceinline__ bool depth_test(const GatherParams& g, float zf, float z) {
    return zf <= __fadd_rn(z, __fmul_rn(g.beta, zf));
}

// The four features from the pixel's G-buffer entry and the fetched depth z.
// Ordinary FP32 accuracy (not part of the bit-exact contract): the quotients
// use the hardware reciprocal / reciprocal square root (a few ulp each), which
// keeps every feature within ~1e-6 relative of its FP64 value at a fraction of
// the instructions of correctly rounded division.
__device__ __forceinline__ void pixel_features(const GatherParams& g, float4 P, float4 N, float z, float f[4]) {
    const float zf = emitter_distance(g, P.x, P.y, P.z);
    const float izf = __fdividef(1.0f, zf);
    const float lx = g.L[0] - P.x, ly = g.L[1] - P.y, lz = g.L[2] - P.z;
    const float ce = (N.x * lx + N.y * ly + N.z * lz) * izf;
    const float cxv = g.C[0] - P.x, cyv = g.C[1] - P.y, czv = g.C[2] - P.z;
    const float icl = rsqrtf(cxv * cxv + cyv * cyv + czv * czv);
    const float cc = (N.x * cxv + N.y * cyv + N.z * czv) * icl;
    f[0] = ce + g.r_hat;
    f[1] = z * izf;
    f[2] = z - zf;
    f[3] = cc * __fdividef(1.0f, P.w);
}

struct PixelGather {
    float f[4];  // c_e + r_hat, z / z_f, z - z_f, c_c / d
    float zf;    // binary32 z_f
    float z;     // fetched depth
    int tex;     // texel index or -1
    bool lit;    // hard bit
};

// Full gather for one pixel: texel lookup, depth test, the four features.
__device__ __forceinline__ PixelGather gather_pixel(const GatherParams& g, float4 P, float4 N) {
    PixelGather o;
    o.tex = texel_index(g, P.x, P.y, P.z);
    o.z = (o.tex >= 0) ? __ldg(g.sm + o.tex) : g.z_far;
    o.zf = emitter_distance(g, P.x, P.y, P.z);
    o.lit = depth_test(g, o.zf, o.z);
    // features (ordinary FP32 arithmetic; not part of the bit-exact contract)
    pixel_features(g, P, N, o.z, o.f);
    return o;
}

// Features only (used by the fused first level for staged halo pixels).
__device__ __forceinline__ void gather_features(const GatherParams& g, int y, int x, float f[4]) {
    const size_t p = static_cast<size_t>(y) * g.W + x;
    const float4 P = __ldg(g.pos4 + p);
    const float4 N = __ldg(g.nrm4 + p);
    PixelGather o = gather_pixel(g, P, N);
    f[0] = o.f[0]; f[1] = o.f[1]; f[2] = o.f[2]; f[3] = o.f[3];
}

__device__ __forceinline__ float sigmoidf_acc(float x) { return 1.0f / (1.0f + expf(-x)); }
// The hardware exponential and reciprocal (a few ulp, ~1e-6 relative): for
// the tensor-core forms, whose stored values carry far larger rounding.  The
// argument is clamped at -80 so the divisor stays below 2^126, where the fast
// reciprocal is specified (the sigmoid is ~1.8e-35 there).
__device__ __forceinline__ float sigmoidf_fast(float x) {
    return __fdividef(1.0f, 1.0f + __expf(-fmaxf(x, -80.0f)));
}

// Bilinear x2 upsampling with half-pixel centres (align_corners = false) and
// edge clamping: output index o samples the source at o / 2 - 1 / 4.
struct BilinTap { int i0, i1; float w0, w1; };
__device__ __forceinline__ BilinTap bilin_tap(int o, int n) {
    // o even: src = o/2 - 0.25 -> i0 = o/2 - 1, w1 = 0.75 ; o odd: src = (o-1)/2 + 0.25 -> w1 = 0.25
    BilinTap t;
    const int k = o >> 1;
    if (o & 1) { t.i0 = k; t.i1 = k + 1; t.w0 = 0.75f; t.w1 = 0.25f; }
    else { t.i0 = k - 1; t.i1 = k; t.w0 = 0.25f; t.w1 = 0.75f; }
    t.i0 = t.i0 < 0 ? 0 : (t.i0 > n - 1 ? n - 1 : t.i0);
    t.i1 = t.i1 < 0 ? 0 : (t.i1 > n - 1 ? n - 1 : t.i1);
    return t;
}

}  // namespace nsm
