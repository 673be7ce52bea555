/*
 * Seeded synthetic-scene ray caster (input generator, FP64).
 *
 * Produces the screen-space buffers that a rasteriser would hand to the
 * neural shadow method (Sec. 3.1: view-space depth d and normal n per pixel;
 * emitter-to-occluder depth z per shadow-map texel) and the ray-traced
 * visibility targets (Sec. 3.1: Monte-Carlo hard/soft shadows).  There is no
 * graphics stack here, so every buffer is produced by ray casting an analytic
 * scene: an infinite ground plane z = 0 (normal +z) plus spheres and
 * axis-aligned boxes.
 *
 * This file holds no part of the shadow method itself (no texel lookup, no
 * features, no network): both the FP64 oracle and the CUDA path consume the
 * buffers it writes.
 *
 * Object record (5 doubles): type (0 = sphere, 1 = box), cx, cy, cz, s.
 *   sphere: centre c, radius s;  box: axis-aligned, centre c, half-extent s.
 * Nearest hit wins; an exact tie goes to the lower object index and the
 * plane is tested last, so it wins only when strictly closer.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define SG_INF 1e300

typedef struct { double t; double n[3]; int hit; } sg_hit;

static inline double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ray o + t d, |d| = 1; returns the smallest t in (tmin, tmax) */
static int hit_sphere(const double* o, const double* d, const double* c, double s,
                      double tmin, double tmax, double* t_out, double* n_out) {
    double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    double b = dot3(d, oc);
    double cc = dot3(oc, oc) - s * s;
    double disc = b * b - cc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double t = -b - sq;
    if (!(t > tmin)) t = -b + sq;
    if (!(t > tmin) || !(t < tmax)) return 0;
    *t_out = t;
    for (int k = 0; k < 3; ++k) n_out[k] = (o[k] + t * d[k] - c[k]) / s;
    return 1;
}

static int hit_box(const double* o, const double* d, const double* c, double s,
                   double tmin, double tmax, double* t_out, double* n_out) {
    double tn = -SG_INF, tf = SG_INF;
    int an = -1, af = -1;
    double sn = 0.0, sf = 0.0;
    for (int k = 0; k < 3; ++k) {
        double lo = c[k] - s, hi = c[k] + s;
        if (d[k] == 0.0) {
            if (o[k] < lo || o[k] > hi) return 0;
            continue;
        }
        double t0 = (lo - o[k]) / d[k], t1 = (hi - o[k]) / d[k];
        double s0 = -1.0, s1 = 1.0; /* outward normal sign of the lo / hi face */
        if (t0 > t1) { double tt = t0; t0 = t1; t1 = tt; s0 = 1.0; s1 = -1.0; }
        if (t0 > tn) { tn = t0; an = k; sn = s0; }
        if (t1 < tf) { tf = t1; af = k; sf = s1; }
    }
    if (tn > tf) return 0;
    double t; int ax; double sg;
    if (tn > tmin) { t = tn; ax = an; sg = sn; }
    else { t = tf; ax = af; sg = sf; }  /* origin inside the box */
    if (!(t > tmin) || !(t < tmax) || ax < 0) return 0;
    *t_out = t;
    n_out[0] = n_out[1] = n_out[2] = 0.0;
    n_out[ax] = sg;
    return 1;
}

static int hit_plane(const double* o, const double* d, double tmin, double tmax,
                     double* t_out, double* n_out) {
    if (d[2] == 0.0) return 0;
    double t = -o[2] / d[2];
    if (!(t > tmin) || !(t < tmax)) return 0;
    *t_out = t;
    n_out[0] = 0.0; n_out[1] = 0.0; n_out[2] = (o[2] >= 0.0) ? 1.0 : -1.0;
    return 1;
}

static sg_hit trace(const double* o, const double* d, int n_obj, const double* obj,
                    double tmin, double tmax, int with_plane) {
    sg_hit h; h.hit = 0; h.t = tmax;
    double t, n[3];
    for (int i = 0; i < n_obj; ++i) {
        const double* ob = obj + 5 * i;
        int ok = (ob[0] == 0.0) ? hit_sphere(o, d, ob + 1, ob[4], tmin, h.t, &t, n)
                                : hit_box(o, d, ob + 1, ob[4], tmin, h.t, &t, n);
        if (ok && t < h.t) { h.t = t; h.n[0] = n[0]; h.n[1] = n[1]; h.n[2] = n[2]; h.hit = 1; }
    }
    if (with_plane && hit_plane(o, d, tmin, h.t, &t, n) && t < h.t) {
        h.t = t; h.n[0] = n[0]; h.n[1] = n[1]; h.n[2] = n[2]; h.hit = 1;
    }
    return h;
}

/* any hit with t in (tmin, tmax): shadow-ray query */
static int occluded(const double* o, const double* d, int n_obj, const double* obj,
                    double tmin, double tmax) {
    double t, n[3];
    for (int i = 0; i < n_obj; ++i) {
        const double* ob = obj + 5 * i;
        int ok = (ob[0] == 0.0) ? hit_sphere(o, d, ob + 1, ob[4], tmin, tmax, &t, n)
                                : hit_box(o, d, ob + 1, ob[4], tmin, tmax, &t, n);
        if (ok) return 1;
    }
    return hit_plane(o, d, tmin, tmax, &t, n);
}

static void normalize3(double* v) {
    double l = sqrt(dot3(v, v));
    v[0] /= l; v[1] /= l; v[2] /= l;
}

/*
 * Pinhole camera G-buffer.  cam = {C[3], fwd[3], right[3], up[3], tan_half_fovy, aspect}
 * (orthonormal basis).  Pixel (x, y) centre, row 0 at the top.
 * pos4[p] = (P.x, P.y, P.z, d) with d = (P - C)·fwd (positive view depth);
 * nrm4[p] = (n.x, n.y, n.z, 0).  mask[p] = 1 where the ray hits something.
 */
void sg_gbuffer(int H, int W, const double* cam, int n_obj, const double* obj,
                float* pos4, float* nrm4, uint8_t* mask) {
    const double* C = cam;
    const double* fwd = cam + 3;
    const double* right = cam + 6;
    const double* up = cam + 9;
    double th = cam[12], aspect = cam[13];
    #pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double nx = 2.0 * (x + 0.5) / W - 1.0;
            double ny = 1.0 - 2.0 * (y + 0.5) / H;
            double d[3];
            for (int k = 0; k < 3; ++k)
                d[k] = fwd[k] + nx * th * aspect * right[k] + ny * th * up[k];
            normalize3(d);
            sg_hit h = trace(C, d, n_obj, obj, 0.0, SG_INF, 1);
            size_t p = (size_t)y * W + x;
            if (h.hit) {
                double P[3] = {C[0] + h.t * d[0], C[1] + h.t * d[1], C[2] + h.t * d[2]};
                double dv = (P[0] - C[0]) * fwd[0] + (P[1] - C[1]) * fwd[1] + (P[2] - C[2]) * fwd[2];
                pos4[4 * p + 0] = (float)P[0]; pos4[4 * p + 1] = (float)P[1];
                pos4[4 * p + 2] = (float)P[2]; pos4[4 * p + 3] = (float)dv;
                nrm4[4 * p + 0] = (float)h.n[0]; nrm4[4 * p + 1] = (float)h.n[1];
                nrm4[4 * p + 2] = (float)h.n[2]; nrm4[4 * p + 3] = 0.0f;
                mask[p] = 1;
            } else {
                for (int k = 0; k < 4; ++k) { pos4[4 * p + k] = 0.0f; nrm4[4 * p + k] = 0.0f; }
                mask[p] = 0;
            }
        }
    }
}

/*
 * Vanilla (single-frustum) shadow map.  lcam = {L[3], fwd[3], right[3], up[3], tan_half_fov}.
 * Texel (i, j) holds the Euclidean distance from L to the first hit along the
 * ray through the texel centre (ndc = 2 (i + 1/2) / Ws - 1, 2 (j + 1/2) / Hs - 1;
 * row j = 0 at ndc_y = -1), or z_far when nothing is hit before z_far.
 */
void sg_shadowmap(int Hs, int Ws, const double* lcam, int n_obj, const double* obj,
                  double z_far, float* depth) {
    const double* L = lcam;
    const double* fwd = lcam + 3;
    const double* right = lcam + 6;
    const double* up = lcam + 9;
    double th = lcam[12];
    #pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < Hs; ++j) {
        for (int i = 0; i < Ws; ++i) {
            double nx = 2.0 * (i + 0.5) / Ws - 1.0;
            double ny = 2.0 * (j + 0.5) / Hs - 1.0;
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = fwd[k] + nx * th * right[k] + ny * th * up[k];
            normalize3(d);
            sg_hit h = trace(L, d, n_obj, obj, 0.0, z_far, 1);
            depth[(size_t)j * Ws + i] = h.hit ? (float)h.t : (float)z_far;
        }
    }
}

/* brute-force hard visibility: shadow ray from P + eps n to the point light L */
void sg_hard_visibility(size_t npx, const float* pos4, const float* nrm4, const uint8_t* mask,
                        const double* L, int n_obj, const double* obj, double eps, uint8_t* vis) {
    #pragma omp parallel for schedule(dynamic, 256)
    for (long long q = 0; q < (long long)npx; ++q) {
        size_t p = (size_t)q;
        if (!mask[p]) { vis[p] = 1; continue; }
        double o[3], d[3];
        for (int k = 0; k < 3; ++k) o[k] = (double)pos4[4 * p + k] + eps * (double)nrm4[4 * p + k];
        for (int k = 0; k < 3; ++k) d[k] = L[k] - o[k];
        double dist = sqrt(dot3(d, d));
        for (int k = 0; k < 3; ++k) d[k] /= dist;
        vis[p] = occluded(o, d, n_obj, obj, 0.0, dist) ? 0 : 1;
    }
}

/* SplitMix64 (Steele, Lea, Flood 2014): counter-based stream for the MC jitter */
static inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Shirley-Chiu concentric map of the unit square onto the unit disk */
static void concentric(double a, double b, double* dx, double* dy) {
    double sx = 2.0 * a - 1.0, sy = 2.0 * b - 1.0;
    if (sx == 0.0 && sy == 0.0) { *dx = 0.0; *dy = 0.0; return; }
    double r, phi;
    const double q = 0.78539816339744830962; /* pi / 4 */
    if (fabs(sx) > fabs(sy)) { r = sx; phi = q * (sy / sx); }
    else { r = sy; phi = 2.0 * q - q * (sx / sy); }
    *dx = r * cos(phi); *dy = r * sin(phi);
}

/*
 * Monte-Carlo visibility of a spherical emitter (centre L, radius r) seen as
 * its silhouette disk: the disk of radius r centred at L, perpendicular to
 * L - P.  spp_side^2 stratified jittered samples per pixel, mapped to the
 * disk with the concentric map; shadow rays start at P + eps n.
 * vis[p] = fraction of unoccluded samples (1 where mask is 0).
 * r = 0 degenerates to the hard (point-light) visibility.
 */
void sg_soft_visibility(size_t npx, const float* pos4, const float* nrm4, const uint8_t* mask,
                        const double* L, double r, int n_obj, const double* obj,
                        int spp_side, uint64_t seed, double eps, float* vis) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (long long q = 0; q < (long long)npx; ++q) {
        size_t p = (size_t)q;
        if (!mask[p]) { vis[p] = 1.0f; continue; }
        double o[3], w[3];
        for (int k = 0; k < 3; ++k) o[k] = (double)pos4[4 * p + k] + eps * (double)nrm4[4 * p + k];
        for (int k = 0; k < 3; ++k) w[k] = L[k] - o[k];
        normalize3(w);
        /* orthonormal frame (e1, e2) of the disk plane */
        double a[3] = {1.0, 0.0, 0.0};
        if (fabs(w[0]) > 0.9) { a[0] = 0.0; a[1] = 1.0; }
        double e1[3] = {a[1] * w[2] - a[2] * w[1], a[2] * w[0] - a[0] * w[2], a[0] * w[1] - a[1] * w[0]};
        normalize3(e1);
        double e2[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
        int unocc = 0, total = spp_side * spp_side;
        for (int s = 0; s < total; ++s) {
            uint64_t h1 = splitmix64(seed ^ splitmix64(((uint64_t)p << 20) | (uint64_t)(2 * s)));
            uint64_t h2 = splitmix64(seed ^ splitmix64(((uint64_t)p << 20) | (uint64_t)(2 * s + 1)));
            double su = ((s % spp_side) + u01(h1)) / spp_side;
            double sv = ((s / spp_side) + u01(h2)) / spp_side;
            double dx, dy;
            concentric(su, sv, &dx, &dy);
            double tgt[3], d[3];
            for (int k = 0; k < 3; ++k) tgt[k] = L[k] + r * (dx * e1[k] + dy * e2[k]);
            for (int k = 0; k < 3; ++k) d[k] = tgt[k] - o[k];
            double dist = sqrt(dot3(d, d));
            for (int k = 0; k < 3; ++k) d[k] /= dist;
            if (!occluded(o, d, n_obj, obj, 0.0, dist)) ++unocc;
        }
        vis[p] = (float)((double)unocc / (double)total);
    }
}

/* single-ray query for tests: nearest hit distance (or -1) and normal */
double sg_trace_one(const double* o, const double* d, int n_obj, const double* obj,
                    int with_plane, double* n_out) {
    sg_hit h = trace(o, d, n_obj, obj, 0.0, SG_INF, with_plane);
    if (!h.hit) return -1.0;
    n_out[0] = h.n[0]; n_out[1] = h.n[1]; n_out[2] = h.n[2];
    return h.t;
}

/* distance from L to the first hit along the exact ray L -> P (per pixel) */
void sg_light_depth(size_t npx, const float* pos4, const double* L, int n_obj, const double* obj,
                    double* out) {
    #pragma omp parallel for schedule(dynamic, 256)
    for (long long q = 0; q < (long long)npx; ++q) {
        size_t p = (size_t)q;
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = (double)pos4[4 * p + k] - L[k];
        double dist = sqrt(dot3(d, d));
        for (int k = 0; k < 3; ++k) d[k] /= dist;
        sg_hit h = trace(L, d, n_obj, obj, 0.0, SG_INF, 1);
        out[p] = h.hit ? h.t : SG_INF;
    }
}
