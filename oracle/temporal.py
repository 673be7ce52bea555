"""Oracle: the temporal-instability metric (Sec. 3.4, Eq. 3) and the
penumbra-size histogram that selects the network depth (Sec. 3.6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. 3:  E = (1 / P) sum_{p, t} (exp(alpha D_t(p)) - 1),
        D_t(p) = |I_t(p) - I_{t-1}(m(p))|,  alpha = 3,
where m(p) is the motion-vector adjusted position of p in the previous frame
and pixels that fail a depth and normal comparison with their reprojection
are rejected.  Readings (the paper fixes none of these):
  * m(p): the world position of p (G-buffer) projected with the previous
    frame's pinhole camera, nearest pixel (pixel centres at +1/2, row 0 at the
    top).  Scene motion is not tracked: a point on a moving object reprojects
    to where the static world would be, and the depth / normal test rejects it
    when the surface seen there differs.
  * The comparison: the previous frame covers m(p) (view depth > 0), its view
    depth is within 1% of the reprojected depth, and the two unit normals have
    a dot product >= 0.9.
  * P is the total number of pixels of the compared frame pairs, H W (T - 1)
    (rejected pixels add 0); the count of accepted pixels is returned too.
  * The accept decisions and D are taken in binary32 with a fixed operation
    order and no contraction (the GPU takes them the same way, so the counts
    agree exactly); exp and the sum are FP64.

Sec. 3.6 depth rule: a histogram of per-pixel screen-space penumbra widths
over the training frames; its 95th percentile p_w bounds the receptive field;
l = log2(p_w / 3) levels of 3x3 kernels.  Readings: the world-space width
x_a + x_b of the spherical-occluder model (suppl. Sec. 4) is projected at the
pixel's view depth, w_px = w H / (2 d tan(fovy / 2)); only pixels with a
blocker count; the histogram has nbins bins of bin_px pixels, the last one
open-ended; the percentile is the upper edge of the first bin at which the
cumulative count reaches 95% of the total; the depth is ceil(l), at least 1.
"""
from __future__ import annotations

import math

import numpy as np

_F = np.float32


def _f(x):
    return np.asarray(x, np.float32)


def reproject_fp32(P: np.ndarray, cam: np.ndarray, H: int, W: int):
    """Pixel (i, j) of world points P (..., 3) in the pinhole camera cam = (C,
    forward, right, up, tan(fovy / 2), aspect W / H), binary32 in this order:
      v = P - C;  z = (v.f_x + v.f_y) + v.f_z  (the same for v.right, v.up);
      ndc_x = (v.right) / (z * (tan * aspect));  ndc_y = (v.up) / (z * tan);
      i = floor((ndc_x * 0.5 + 0.5) * W);  j = floor((0.5 - ndc_y * 0.5) * H).
    Returns (i, j, z, ok) with ok = z > 0 and (i, j) inside the image."""
    cam = _f(cam)
    P = _f(P)
    C, fw, rt, up = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    th, asp = cam[12], cam[13]
    with np.errstate(all="ignore"):
        v = [(P[..., k] - C[k]).astype(_F) for k in range(3)]

        def dot(a):
            s = (v[0] * a[0]).astype(_F) + (v[1] * a[1]).astype(_F)
            return (s.astype(_F) + (v[2] * a[2]).astype(_F)).astype(_F)

        z = dot(fw)
        xr, yu = dot(rt), dot(up)
        tha = _F(th * asp)
        nx = (xr / (z * tha).astype(_F)).astype(_F)
        ny = (yu / (z * th).astype(_F)).astype(_F)
        u = ((nx * _F(0.5)).astype(_F) + _F(0.5)).astype(_F)
        w = (_F(0.5) - (ny * _F(0.5)).astype(_F)).astype(_F)
        fi = np.floor((u * _F(W)).astype(_F))
        fj = np.floor((w * _F(H)).astype(_F))
        ok = (z > 0) & (fi >= 0) & (fi < W) & (fj >= 0) & (fj < H)
    i = np.where(ok, fi, 0).astype(np.int64)
    j = np.where(ok, fj, 0).astype(np.int64)
    return i, j, z, ok


def accept_fp32(z_reproj, d_prev, n_cur, n_prev, d_tol: float = 0.01, n_cos: float = 0.9):
    """Depth / normal comparison in binary32: d_prev > 0,
    |d_prev - z| <= d_tol * z and (n_x n'_x + n_y n'_y) + n_z n'_z >= n_cos."""
    z = _f(z_reproj)
    dp = _f(d_prev)
    dd = np.abs((dp - z).astype(_F))
    lim = (_F(d_tol) * z).astype(_F)
    nc, npv = _f(n_cur), _f(n_prev)
    s = (nc[..., 0] * npv[..., 0]).astype(_F) + (nc[..., 1] * npv[..., 1]).astype(_F)
    s = (s.astype(_F) + (nc[..., 2] * npv[..., 2]).astype(_F)).astype(_F)
    return (dp > 0) & (dd <= lim) & (s >= _F(n_cos))


def instability_pair(I_t, I_prev, pos4_t, nrm4_t, pos4_prev, nrm4_prev, cam_prev, alpha: float = 3.0):
    """One frame pair of Eq. 3: (sum of exp(alpha D) - 1 over accepted pixels,
    number of accepted pixels).  Images (H, W); G-buffers (H, W, 4) with the
    view depth in pos4[..., 3] (0 where the pixel sees nothing)."""
    H, W = I_t.shape
    i, j, z, ok = reproject_fp32(pos4_t[..., :3], cam_prev, H, W)
    ok &= _f(pos4_t[..., 3]) > 0
    d_prev = np.where(ok, _f(pos4_prev[..., 3])[j, i], _F(0))
    n_prev = _f(nrm4_prev[..., :3])[j, i]
    acc = ok & accept_fp32(z, d_prev, nrm4_t[..., :3], n_prev)
    D = np.abs((_f(I_t) - _f(I_prev)[j, i]).astype(_F)).astype(np.float64)
    contrib = np.where(acc, np.exp(alpha * D) - 1.0, 0.0)
    return float(contrib.sum()), int(acc.sum())


def temporal_instability(images, pos4s, nrm4s, cams, alpha: float = 3.0):
    """Eq. 3 over a sequence: E = (1 / P) sum over consecutive pairs, P = H W
    (T - 1).  Returns (E, accepted pixel count)."""
    T = len(images)
    H, W = images[0].shape
    tot, cnt = 0.0, 0
    for t in range(1, T):
        s, c = instability_pair(images[t], images[t - 1], pos4s[t], nrm4s[t], pos4s[t - 1], nrm4s[t - 1],
                                cams[t - 1], alpha)
        tot += s
        cnt += c
    return tot / float(H * W * (T - 1)), cnt


# ------------------------------------------------------------------ depth from the penumbra size (Sec. 3.6)

def screen_width_px(width_world, d, H: int, tan_half_fovy: float):
    """World-space width at view depth d in pixels: w H / (2 d tan(fovy / 2))."""
    return np.asarray(width_world, np.float64) * H / (2.0 * np.asarray(d, np.float64) * tan_half_fovy)


def penumbra_histogram(width_px, bin_px: float, nbins: int) -> np.ndarray:
    """Counts of floor(w / bin_px) (negative widths in bin 0, the last bin
    open-ended)."""
    b = np.floor(np.asarray(width_px, np.float64) / bin_px)
    b = np.clip(b, 0, nbins - 1).astype(np.int64)
    return np.bincount(b.ravel(), minlength=nbins).astype(np.int64)


def p95_from_histogram(hist, bin_px: float) -> float:
    """Upper edge of the first bin at which the cumulative count reaches 95%
    of the total (0 for an empty histogram)."""
    h = np.asarray(hist, np.int64)
    total = int(h.sum())
    if total == 0:
        return 0.0
    # cumulative >= 95% of the total, compared exactly in integers (19 / 20)
    k = int(np.nonzero(20 * np.cumsum(h) >= 19 * total)[0][0])
    return (k + 1) * bin_px


def depth_for_width(p_w: float) -> int:
    """ceil(log2(p_w / 3)), at least 1: the levels whose receptive field
    3 * 2^l covers a penumbra of p_w pixels."""
    if p_w <= 6.0:
        return 1
    return max(1, int(math.ceil(math.log2(p_w / 3.0))))
