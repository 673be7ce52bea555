"""Oracle: shadow-map lookup, hard depth test, features and blocker search.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.1 lists the rasteriser buffers: view-space depth d and normal n, the
emitter-to-occluder depth z read from a vanilla shadow map, the
pixel-to-emitter distance z_f, the emitter size r_e, and the cosines c_e
(normal vs emitter direction) and c_c (normal vs view direction).  Sec. 3.2
and Fig. 2 / Fig. 3 fix the selected input set and its order:
    f = [c_e + r_e, z / z_f, z - z_f, c_c / d]
with the emitter size added to c_e as a DC offset (Sec. 3.1.1).

Texel choice and hard depth test (readings: nearest texel, texel centres at
+1/2, outside the frustum reads z_far, a depth bias proportional to the
receiver distance, lit iff z_f <= z + beta z_f) are evaluated in
IEEE binary32 with a fixed operation order and no fused multiply-add; this
routine *defines* the texel index and the hard bit.  numpy float32 ufuncs
round every single operation correctly, which is exactly that definition.

Features are evaluated in FP64 from the FP32 inputs, with z taken from the
texel that the binary32 routine chose.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32


def project_fp32(P: np.ndarray, M: np.ndarray, Ws: int, Hs: int):
    """Light-space projection and nearest-texel index in binary32.

    P: (..., 3) float32 world positions; M: (4, 4) float32 world->clip (row-major).
    clip_r = ((M[r,0] Px + M[r,1] Py) + M[r,2] Pz) + M[r,3]  (left to right)
    ndc = clip.xy / clip.w;  u = ndc * 0.5 + 0.5;  (i, j) = floor(u * (Ws, Hs))
    inside iff clip.w > 0 and 0 <= i < Ws and 0 <= j < Hs.
    Returns (i, j, inside, clip_w) with i, j as int64 (valid where inside).
    """
    P = np.asarray(P, F32)
    M = np.asarray(M, F32)
    px, py, pz = P[..., 0], P[..., 1], P[..., 2]

    def row(r):
        return ((M[r, 0] * px + M[r, 1] * py) + M[r, 2] * pz) + M[r, 3]

    cx, cy, cw = row(0), row(1), row(3)
    with np.errstate(divide="ignore", invalid="ignore"):
        nx = cx / cw
        ny = cy / cw
        u = nx * F32(0.5) + F32(0.5)
        v = ny * F32(0.5) + F32(0.5)
        fi = np.floor(u * F32(Ws))
        fj = np.floor(v * F32(Hs))
        inside = (cw > F32(0)) & (fi >= F32(0)) & (fi < F32(Ws)) & (fj >= F32(0)) & (fj < F32(Hs))
    i = np.where(inside, fi, 0).astype(np.int64)
    j = np.where(inside, fj, 0).astype(np.int64)
    return i, j, inside, cw


def depth_test_fp32(zf: np.ndarray, z: np.ndarray, beta: float) -> np.ndarray:
    """Hard bit in binary32: lit iff z_f <= z + (beta * z_f)."""
    zf = np.asarray(zf, F32)
    return zf <= (np.asarray(z, F32) + F32(beta) * zf)


def emitter_distance_fp32(P: np.ndarray, L: np.ndarray) -> np.ndarray:
    """z_f = sqrt((dx dx + dy dy) + dz dz) in binary32, d = L - P."""
    P = np.asarray(P, F32)
    L = np.asarray(L, F32)
    dx = L[0] - P[..., 0]
    dy = L[1] - P[..., 1]
    dz = L[2] - P[..., 2]
    return np.sqrt((dx * dx + dy * dy) + dz * dz)


def lookup_and_test(pos4: np.ndarray, sm: np.ndarray, M: np.ndarray, L: np.ndarray,
                    z_far: float, bias: float):
    """Texel index (j*Ws + i, or -1 outside), fetched depth z (float32) and the
    hard bit (z_f <= z + beta z_f, binary32, beta = bias) for every pixel."""
    Hs, Ws = sm.shape
    P = pos4[..., :3]
    i, j, inside, _ = project_fp32(P, M, Ws, Hs)
    z = np.where(inside, sm[j, i], F32(z_far)).astype(F32)
    zf = emitter_distance_fp32(P, L)
    hard = depth_test_fp32(zf, z, bias)
    tex = np.where(inside, j * Ws + i, -1).astype(np.int64)
    return tex, z, hard


def project_fp64_index(P: np.ndarray, M: np.ndarray, Ws: int, Hs: int) -> np.ndarray:
    """The same texel choice in FP64 (for reporting how many pixels differ)."""
    P = np.asarray(P, np.float64)
    M = np.asarray(M, np.float64)
    h = np.concatenate([P, np.ones(P.shape[:-1] + (1,))], axis=-1)
    clip = h @ M.T
    with np.errstate(divide="ignore", invalid="ignore"):
        u = clip[..., 0] / clip[..., 3] * 0.5 + 0.5
        v = clip[..., 1] / clip[..., 3] * 0.5 + 0.5
        fi = np.floor(u * Ws)
        fj = np.floor(v * Hs)
        inside = (clip[..., 3] > 0) & (fi >= 0) & (fi < Ws) & (fj >= 0) & (fj < Hs)
    return np.where(inside, np.where(inside, fj, 0).astype(np.int64) * Ws
                    + np.where(inside, fi, 0).astype(np.int64), -1)


def features(pos4, nrm4, sm, M, L, C, r_hat, z_far, bias):
    """The four network inputs, FP64, channel-first (4, H, W).

    z_f = |L - P|,  c_e = n . (L - P) / z_f,  c_c = n . (C - P) / |C - P|,
    d = view depth (pos4 w),  z = depth of the binary32-chosen texel.
    f = [c_e + r_hat, z / z_f, z - z_f, c_c / d]   (Fig. 2 order)
    Returns (feat, tex, hard).
    """
    tex, z, hard = lookup_and_test(pos4, sm, M, L, z_far, bias)
    P = pos4[..., :3].astype(np.float64)
    n = nrm4[..., :3].astype(np.float64)
    d = pos4[..., 3].astype(np.float64)
    Lv = np.asarray(L, np.float64)
    Cv = np.asarray(C, np.float64)
    toL = Lv - P
    zf = np.sqrt(np.sum(toL * toL, axis=-1))
    ce = np.sum(n * toL, axis=-1) / zf
    toC = Cv - P
    cc = np.sum(n * toC, axis=-1) / np.sqrt(np.sum(toC * toC, axis=-1))
    z64 = z.astype(np.float64)
    feat = np.stack([ce + float(r_hat), z64 / zf, z64 - zf, cc / d], axis=0)
    return feat, tex, hard


def blocker_window_half(zf32, light_radius, Ws, tan_half_fov, kmax=32):
    """Half-size k of the square blocker-search window (binary32):
    k = min(kmax, ceil((r * (Ws/2)) / (z_f * tan(fov/2)))), the emitter's
    footprint in texels at the receiver distance (PCSS-style search region)."""
    zf32 = np.asarray(zf32, F32)
    num = F32(light_radius) * F32(0.5 * Ws)
    den = zf32 * F32(tan_half_fov)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.ceil(num / den)
    k = np.where(np.isfinite(k), k, kmax)
    return np.minimum(k, kmax).astype(np.int64)


def blocker_search(pos4, sm, M, L, light_radius, tan_half_fov, z_far, bias, kmax=32):
    """Occluder distances seen from the emitter around each pixel's texel.

    Over the texels (i + a, j + b), |a|, |b| <= k (clipped to the map), the
    blockers are those with z < z_f - beta z_f (binary32); returns (z_min, z_max, found)
    with z_min/z_max = 0 where no blocker was found or the pixel projects
    outside the map.  z_min / z_max are the nearest / farthest occluder
    distances of the penumbra model (Sec. 3.6, Fig. 7)."""
    Hs, Ws = sm.shape
    P = pos4[..., :3]
    i, j, inside, _ = project_fp32(P, M, Ws, Hs)
    zf = emitter_distance_fp32(P, L)
    thr = zf - F32(bias) * zf
    k = blocker_window_half(zf, light_radius, Ws, tan_half_fov, kmax)
    shp = zf.shape
    zmin = np.zeros(shp, F32)
    zmax = np.zeros(shp, F32)
    found = np.zeros(shp, bool)
    for idx in np.ndindex(shp):
        if not inside[idx]:
            continue
        kk = int(k[idx])
        ci, cj = int(i[idx]), int(j[idx])
        win = sm[max(0, cj - kk):min(Hs, cj + kk + 1), max(0, ci - kk):min(Ws, ci + kk + 1)]
        sel = win[win < thr[idx]]
        if sel.size:
            found[idx] = True
            zmin[idx] = sel.min()
            zmax[idx] = sel.max()
    return zmin, zmax, found


def penumbra_width(z_f, z_min, z_max, r_e):
    """Penumbra width x_a + x_b of the spherical-occluder model (suppl. Sec. 4):
    z_m = (z_max + z_min)/2, r_s = (z_max - z_min)/2,
    theta_d = asin(r_s / sqrt(z_m^2 + r_e^2)), BQ = r_e (z_f - z_m) / z_m,
    theta = atan((BQ + r_e) / z_f),  x_{a,b} = z_f tan(theta -/+ theta_d) - r_e.
    FP64; returns (x_a, x_b)."""
    z_f = np.asarray(z_f, np.float64)
    z_min = np.asarray(z_min, np.float64)
    z_max = np.asarray(z_max, np.float64)
    zm = 0.5 * (z_max + z_min)
    rs = 0.5 * (z_max - z_min)
    td = np.arcsin(rs / np.sqrt(zm * zm + r_e * r_e))
    bq = r_e * (z_f - zm) / zm
    th = np.arctan((bq + r_e) / z_f)
    xa = z_f * np.tan(th - td) - r_e
    xb = z_f * np.tan(th + td) - r_e
    return xa, xb


def receptive_field(levels: int) -> int:
    """Receptive field 3 * 2^l of an l-level net of 3x3 kernels (Sec. 3.6)."""
    return 3 * (2 ** levels)


def levels_for_penumbra(p_w: float) -> float:
    """l = log2(p_w / 3) (Sec. 3.6)."""
    return math.log2(p_w / 3.0)
