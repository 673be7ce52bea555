// Scene generation on the GPU: the ray-cast G-buffer, shadow map and
// Monte-Carlo visibility targets the method trains on (Sec. 3.1: G-buffer and
// shadow-map pass from rasterisation, converged hard / soft shadows from ray
// tracing).  There is no rasteriser here; every buffer is produced by casting
// rays into an analytic scene: the ground plane z = 0 (normal +z) plus spheres
// and axis-aligned boxes.  FP32 arithmetic throughout.
//
//   gen_gbuffer     one thread per pixel: pinhole camera ray through the pixel
//                   centre (row 0 at the top), nearest hit -> P, n, view depth d
//   gen_shadowmap   one thread per texel: ray from the emitter centre through
//                   the texel centre, distance to the nearest hit (z_far if none)
//   gen_visibility  one warp per pixel: spp_side^2 stratified jittered samples on
//                   the emitter's silhouette disk (radius r, perpendicular to
//                   L - P, concentric disk map), shadow rays from P + eps n, the
//                   unoccluded fraction by a warp reduction; r = 0 gives the
//                   hard (point-light) visibility.  Jitter from SplitMix64
//                   (Steele, Lea and Flood, 2014) keyed by (pixel, sample).
// Nearest hit wins; an exact tie goes to the lower object index and the plane
// is tested last.
#include "nsm_internal.h"

namespace nsm {

constexpr int kGenMaxObjects = 256;
struct GenScene {
    int n;
    float obj[kGenMaxObjects][5];  // type (0 sphere, 1 box), centre x, y, z, size
};
struct GenCam { float o[3], fwd[3], right[3], up[3], th, aspect; };

struct Hit { float t, n[3]; bool hit; };

__device__ __forceinline__ bool hit_sphere(const float* o, const float* d, const float* c, float s, float tmin,
                                           float tmax, float& t_out, float* n_out) {
    const float oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    const float b = d[0] * oc[0] + d[1] * oc[1] + d[2] * oc[2];
    const float cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - s * s;
    const float disc = b * b - cc;
    if (disc < 0.f) return false;
    const float sq = sqrtf(disc);
    float t = -b - sq;
    if (!(t > tmin)) t = -b + sq;
    if (!(t > tmin) || !(t < tmax)) return false;
    t_out = t;
    for (int k = 0; k < 3; ++k) n_out[k] = (o[k] + t * d[k] - c[k]) / s;
    return true;
}

__device__ __forceinline__ bool hit_box(const float* o, const float* d, const float* c, float s, float tmin,
                                        float tmax, float& t_out, float* n_out) {
    float tn = -INFINITY, tf = INFINITY, sn = 0.f, sf = 0.f;
    int an = -1, af = -1;
    for (int k = 0; k < 3; ++k) {
        const float lo = c[k] - s, hi = c[k] + s;
        if (d[k] == 0.f) {
            if (o[k] < lo || o[k] > hi) return false;
            continue;
        }
        float t0 = (lo - o[k]) / d[k], t1 = (hi - o[k]) / d[k];
        float s0 = -1.f, s1 = 1.f;  // outward normal sign of the lo / hi face
        if (t0 > t1) { const float tt = t0; t0 = t1; t1 = tt; s0 = 1.f; s1 = -1.f; }
        if (t0 > tn) { tn = t0; an = k; sn = s0; }
        if (t1 < tf) { tf = t1; af = k; sf = s1; }
    }
    if (tn > tf) return false;
    float t, sg;
    int ax;
    if (tn > tmin) { t = tn; ax = an; sg = sn; }
    else { t = tf; ax = af; sg = sf; }  // origin inside the box
    if (!(t > tmin) || !(t < tmax) || ax < 0) return false;
    t_out = t;
    n_out[0] = n_out[1] = n_out[2] = 0.f;
    n_out[ax] = sg;
    return true;
}

__device__ __forceinline__ bool hit_plane(const float* o, const float* d, float tmin, float tmax, float& t_out,
                                          float* n_out) {
    if (d[2] == 0.f) return false;
    const float t = -o[2] / d[2];
    if (!(t > tmin) || !(t < tmax)) return false;
    t_out = t;
    n_out[0] = 0.f; n_out[1] = 0.f; n_out[2] = o[2] >= 0.f ? 1.f : -1.f;
    return true;
}

__device__ __forceinline__ Hit trace(const GenScene& sc, const float* o, const float* d, float tmin, float tmax) {
    Hit h;
    h.hit = false;
    h.t = tmax;
    float t, n[3];
    for (int i = 0; i < sc.n; ++i) {
        const float* ob = sc.obj[i];
        const bool ok = ob[0] == 0.f ? hit_sphere(o, d, ob + 1, ob[4], tmin, h.t, t, n)
                                     : hit_box(o, d, ob + 1, ob[4], tmin, h.t, t, n);
        if (ok && t < h.t) { h.t = t; h.n[0] = n[0]; h.n[1] = n[1]; h.n[2] = n[2]; h.hit = true; }
    }
    if (hit_plane(o, d, tmin, h.t, t, n) && t < h.t) {
        h.t = t; h.n[0] = n[0]; h.n[1] = n[1]; h.n[2] = n[2]; h.hit = true;
    }
    return h;
}

__device__ __forceinline__ bool occluded(const GenScene& sc, const float* o, const float* d, float tmax) {
    float t, n[3];
    for (int i = 0; i < sc.n; ++i) {
        const float* ob = sc.obj[i];
        const bool ok = ob[0] == 0.f ? hit_sphere(o, d, ob + 1, ob[4], 0.f, tmax, t, n)
                                     : hit_box(o, d, ob + 1, ob[4], 0.f, tmax, t, n);
        if (ok) return true;
    }
    return hit_plane(o, d, 0.f, tmax, t, n);
}

__device__ __forceinline__ void normalize3(float* v) {
    const float l = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

__global__ void __launch_bounds__(256) gen_gbuffer_kernel(GenScene sc, GenCam cam, int H, int W,
                                                          float4* __restrict__ pos4, float4* __restrict__ nrm4,
                                                          uint8_t* __restrict__ mask) {
    const size_t n = static_cast<size_t>(H) * W;
    for (size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(p / W), x = static_cast<int>(p % W);
        const float nx = 2.f * (x + 0.5f) / W - 1.f, ny = 1.f - 2.f * (y + 0.5f) / H;
        float d[3];
        for (int k = 0; k < 3; ++k) d[k] = cam.fwd[k] + nx * cam.th * cam.aspect * cam.right[k] + ny * cam.th * cam.up[k];
        normalize3(d);
        const Hit h = trace(sc, cam.o, d, 0.f, INFINITY);
        if (h.hit) {
            const float P[3] = {cam.o[0] + h.t * d[0], cam.o[1] + h.t * d[1], cam.o[2] + h.t * d[2]};
            const float dv = (P[0] - cam.o[0]) * cam.fwd[0] + (P[1] - cam.o[1]) * cam.fwd[1] +
                             (P[2] - cam.o[2]) * cam.fwd[2];
            pos4[p] = make_float4(P[0], P[1], P[2], dv);
            nrm4[p] = make_float4(h.n[0], h.n[1], h.n[2], 0.f);
            mask[p] = 1;
        } else {
            pos4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            nrm4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            mask[p] = 0;
        }
    }
}

__global__ void __launch_bounds__(256) gen_shadowmap_kernel(GenScene sc, GenCam lc, int Hs, int Ws, float z_far,
                                                            float* __restrict__ depth) {
    const size_t n = static_cast<size_t>(Hs) * Ws;
    for (size_t q = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; q < n;
         q += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(q / Ws), i = static_cast<int>(q % Ws);
        const float nx = 2.f * (i + 0.5f) / Ws - 1.f, ny = 2.f * (j + 0.5f) / Hs - 1.f;
        float d[3];
        for (int k = 0; k < 3; ++k) d[k] = lc.fwd[k] + nx * lc.th * lc.right[k] + ny * lc.th * lc.up[k];
        normalize3(d);
        const Hit h = trace(sc, lc.o, d, 0.f, z_far);
        depth[q] = h.hit ? h.t : z_far;
    }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Shirley-Chiu concentric map of the unit square onto the unit disk
__device__ __forceinline__ void concentric(float a, float b, float& dx, float& dy) {
    const float sx = 2.f * a - 1.f, sy = 2.f * b - 1.f;
    if (sx == 0.f && sy == 0.f) { dx = dy = 0.f; return; }
    const float q = 0.78539816339744831f;  // pi / 4
    float r, phi;
    if (fabsf(sx) > fabsf(sy)) { r = sx; phi = q * (sy / sx); }
    else { r = sy; phi = 2.f * q - q * (sx / sy); }
    dx = r * cosf(phi);
    dy = r * sinf(phi);
}

__global__ void __launch_bounds__(256) gen_visibility_kernel(GenScene sc, const float4* __restrict__ pos4,
                                                             const float4* __restrict__ nrm4,
                                                             const uint8_t* __restrict__ mask, float3 L, float r,
                                                             int spp_side, uint64_t seed, float eps, size_t npx,
                                                             float* __restrict__ vis) {
    const int lane = threadIdx.x & 31;
    const size_t warps = static_cast<size_t>(gridDim.x) * (blockDim.x / 32);
    const int total = spp_side * spp_side;
    for (size_t p = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) / 32; p < npx; p += warps) {
        if (!mask[p]) {
            if (lane == 0) vis[p] = 1.f;
            continue;
        }
        const float4 P = __ldg(pos4 + p), N = __ldg(nrm4 + p);
        const float o[3] = {P.x + eps * N.x, P.y + eps * N.y, P.z + eps * N.z};
        float w[3] = {L.x - o[0], L.y - o[1], L.z - o[2]};
        normalize3(w);
        // orthonormal frame (e1, e2) of the disk plane
        float a[3] = {1.f, 0.f, 0.f};
        if (fabsf(w[0]) > 0.9f) { a[0] = 0.f; a[1] = 1.f; }
        float e1[3] = {a[1] * w[2] - a[2] * w[1], a[2] * w[0] - a[0] * w[2], a[0] * w[1] - a[1] * w[0]};
        normalize3(e1);
        const float e2[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
        int unocc = 0;
        for (int s = lane; s < total; s += 32) {
            const uint64_t h1 = splitmix64(seed ^ splitmix64((static_cast<uint64_t>(p) << 20) | (2ull * s)));
            const uint64_t h2 = splitmix64(seed ^ splitmix64((static_cast<uint64_t>(p) << 20) | (2ull * s + 1)));
            const float u1 = static_cast<float>(h1 >> 40) * (1.f / 16777216.f);
            const float u2 = static_cast<float>(h2 >> 40) * (1.f / 16777216.f);
            const float su = ((s % spp_side) + u1) / spp_side, sv = ((s / spp_side) + u2) / spp_side;
            float dx, dy;
            concentric(su, sv, dx, dy);
            const float tgt[3] = {L.x + r * (dx * e1[0] + dy * e2[0]), L.y + r * (dx * e1[1] + dy * e2[1]),
                                  L.z + r * (dx * e1[2] + dy * e2[2])};
            float d[3] = {tgt[0] - o[0], tgt[1] - o[1], tgt[2] - o[2]};
            const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            d[0] /= dist; d[1] /= dist; d[2] /= dist;
            unocc += occluded(sc, o, d, dist) ? 0 : 1;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) unocc += __shfl_xor_sync(0xffffffffu, unocc, off);
        if (lane == 0) vis[p] = static_cast<float>(unocc) / static_cast<float>(total);
    }
}

static bool load_scene(int n_obj, const float* obj, GenScene& sc) {
    if (n_obj < 0 || n_obj > kGenMaxObjects || (n_obj > 0 && !obj)) return false;
    sc.n = n_obj;
    for (int i = 0; i < n_obj; ++i)
        for (int k = 0; k < 5; ++k) sc.obj[i][k] = obj[5 * i + k];
    return true;
}

static unsigned gen_blocks(size_t items, int per_block) {
    const size_t cap = static_cast<size_t>(num_sms()) * 16;
    const size_t b = (items + per_block - 1) / per_block;
    return static_cast<unsigned>(b < cap ? b : cap);
}

}  // namespace nsm

using namespace nsm;

extern "C" {

nsm_status nsm_gen_gbuffer(int H, int W, const float* cam, int n_obj, const float* objects, float* pos4,
                           float* nrm4, uint8_t* mask, void* stream) {
    if (H < 0 || W < 0 || !cam) return fail(NSM_ERR_INVALID_ARG, "H, W must be >= 0 and cam non-NULL");
    GenScene sc;
    if (!load_scene(n_obj, objects, sc)) return fail(NSM_ERR_INVALID_ARG, "0..%d objects", kGenMaxObjects);
    if (static_cast<size_t>(H) * W == 0) return NSM_OK;
    nsm_status s;
    if ((s = check_dev_ptr(pos4, "pos4", 16)) != NSM_OK || (s = check_dev_ptr(nrm4, "nrm4", 16)) != NSM_OK ||
        (s = check_dev_ptr(mask, "mask", 1)) != NSM_OK)
        return s;
    GenCam c{};
    for (int k = 0; k < 3; ++k) { c.o[k] = cam[k]; c.fwd[k] = cam[3 + k]; c.right[k] = cam[6 + k]; c.up[k] = cam[9 + k]; }
    c.th = cam[12];
    c.aspect = cam[13];
    gen_gbuffer_kernel<<<gen_blocks(static_cast<size_t>(H) * W, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        sc, c, H, W, reinterpret_cast<float4*>(pos4), reinterpret_cast<float4*>(nrm4), mask);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "gen_gbuffer launch");
}

nsm_status nsm_gen_shadowmap(int Hs, int Ws, const float* lcam, float z_far, int n_obj, const float* objects,
                             float* depth, void* stream) {
    if (Hs < 0 || Ws < 0 || !lcam || !(z_far > 0.f))
        return fail(NSM_ERR_INVALID_ARG, "Hs, Ws must be >= 0, lcam non-NULL and z_far > 0");
    GenScene sc;
    if (!load_scene(n_obj, objects, sc)) return fail(NSM_ERR_INVALID_ARG, "0..%d objects", kGenMaxObjects);
    if (static_cast<size_t>(Hs) * Ws == 0) return NSM_OK;
    nsm_status s;
    if ((s = check_dev_ptr(depth, "depth", 4)) != NSM_OK) return s;
    GenCam c{};
    for (int k = 0; k < 3; ++k) { c.o[k] = lcam[k]; c.fwd[k] = lcam[3 + k]; c.right[k] = lcam[6 + k]; c.up[k] = lcam[9 + k]; }
    c.th = lcam[12];
    gen_shadowmap_kernel<<<gen_blocks(static_cast<size_t>(Hs) * Ws, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        sc, c, Hs, Ws, z_far, depth);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "gen_shadowmap launch");
}

nsm_status nsm_gen_visibility(int H, int W, const float* pos4, const float* nrm4, const uint8_t* mask,
                              const float* light_pos, float radius, int spp_side, uint64_t seed, float eps,
                              int n_obj, const float* objects, float* vis, void* stream) {
    if (H < 0 || W < 0 || !light_pos || spp_side < 1 || spp_side > 1024 || !(radius >= 0.f))
        return fail(NSM_ERR_INVALID_ARG, "H, W >= 0, light_pos non-NULL, 1 <= spp_side <= 1024, radius >= 0");
    GenScene sc;
    if (!load_scene(n_obj, objects, sc)) return fail(NSM_ERR_INVALID_ARG, "0..%d objects", kGenMaxObjects);
    const size_t npx = static_cast<size_t>(H) * W;
    if (npx == 0) return NSM_OK;
    nsm_status s;
    if ((s = check_dev_ptr(pos4, "pos4", 16)) != NSM_OK || (s = check_dev_ptr(nrm4, "nrm4", 16)) != NSM_OK ||
        (s = check_dev_ptr(mask, "mask", 1)) != NSM_OK || (s = check_dev_ptr(vis, "vis", 4)) != NSM_OK)
        return s;
    gen_visibility_kernel<<<gen_blocks(npx * 32, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        sc, reinterpret_cast<const float4*>(pos4), reinterpret_cast<const float4*>(nrm4), mask,
        make_float3(light_pos[0], light_pos[1], light_pos[2]), radius, spp_side, seed, eps, npx, vis);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NSM_OK : cuda_fail(e, "gen_visibility launch");
}

}  // extern "C"
