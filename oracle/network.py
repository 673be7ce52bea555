"""Oracle: the compact encoder/decoder, its adjoint, the loss and Adam (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Architecture (Sec. 3.5): each level has one 3x3 convolution and one 1x1
convolution; average pooling (2x2, stride 2) on the way down; bilinear x2
upsampling on the way up; decoder skips merged by an algebraic sum; no skip
connection at level 0.  Readings where the paper is silent: ReLU after every
convolution except the output head, which is a 1x1 convolution 16 -> 1
followed by a sigmoid; zero "same" padding; biases present; bilinear x2 with
half-pixel centres (align_corners = False) and edge clamping.

Per-level channel plan (w_l = 16 * 2^l): encoder 3x3 w_{l-1} -> w_l (4 input
features at level 0), encoder 1x1 w_l -> w_l; decoder 3x3 w_l -> w_l,
decoder 1x1 w_l -> w_{l-1} (16 -> 16 at level 0); the bottleneck level L-1
has 3x3 w_{L-2} -> w_{L-1} and 1x1 w_{L-1} -> w_{L-2}.  This plan gives
exactly the parameter and per-pixel MAC counts the paper prints for the 3-
and 5-level nets (suppl. Tab. 3 and Tab. 5): 39,248 / 8,528 and
653,648 / 16,208, and 7.15 / 8.05 / 8.05 / 8.05 / 2.68 GMAC per level at
1024 x 2048.

Tensors are channel-first (C, H, W) float64.  Weight layout: a flat vector,
for each layer in `layer_table` order its OIHW weights then its bias.
"""
from __future__ import annotations

import numpy as np

# ------------------------------------------------------------------ topology


def layer_table(levels: int = 3, base: int = 16, in_ch: int = 4):
    """[(name, c_in, c_out, k)] in canonical order: encoder levels 0..L-2
    (3x3, 1x1), bottleneck (3x3, 1x1), decoder levels L-2..0 (3x3, 1x1), head."""
    w = [base * (2 ** l) for l in range(levels)]
    t = []
    for l in range(levels - 1):
        cin = in_ch if l == 0 else w[l - 1]
        t.append((f"enc{l}_3x3", cin, w[l], 3))
        t.append((f"enc{l}_1x1", w[l], w[l], 1))
    b = levels - 1
    t.append((f"bott_3x3", w[b - 1], w[b], 3))
    t.append((f"bott_1x1", w[b], w[b - 1], 1))
    for l in range(levels - 2, -1, -1):
        cout = w[l - 1] if l > 0 else w[0]
        t.append((f"dec{l}_3x3", w[l], w[l], 3))
        t.append((f"dec{l}_1x1", w[l], cout, 1))
    t.append(("head", w[0], 1, 1))
    return t


def param_count(levels: int = 3, with_bias: bool = False) -> int:
    n = 0
    for (_, ci, co, k) in layer_table(levels):
        n += ci * co * k * k + (co if with_bias else 0)
    return n


def macs_per_pixel_by_level(levels: int = 3):
    """MACs per full-resolution pixel, per level (level l runs at 1/4^l pixels)."""
    out = [0.0] * levels
    for (name, ci, co, k) in layer_table(levels):
        if name == "head":
            lvl = 0
        elif name.startswith("bott"):
            lvl = levels - 1
        else:
            lvl = int(name[3])
        out[lvl] += ci * co * k * k / (4.0 ** lvl)
    return out


def unpack(theta: np.ndarray, levels: int = 3):
    """Flat canonical vector -> {name: (W (O,I,k,k), b (O,))}."""
    theta = np.asarray(theta, np.float64)
    out = {}
    off = 0
    for (name, ci, co, k) in layer_table(levels):
        n = co * ci * k * k
        W = theta[off:off + n].reshape(co, ci, k, k)
        off += n
        b = theta[off:off + co]
        off += co
        out[name] = (W, b)
    if off != theta.size:
        raise ValueError(f"weight vector has {theta.size} entries, expected {off}")
    return out


def pack(params, levels: int = 3) -> np.ndarray:
    parts = []
    for (name, ci, co, k) in layer_table(levels):
        W, b = params[name]
        parts.append(np.asarray(W, np.float64).reshape(-1))
        parts.append(np.asarray(b, np.float64).reshape(-1))
    return np.concatenate(parts)


# ------------------------------------------------------------------ operators


def conv2d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' cross-correlation: y[o,y,x] = b[o] +
    sum_{c,u,v} W[o,c,u,v] x[c, y+u-p, x+v-p], p = (k-1)/2.  The channel sum
    of each tap is one tensordot; taps are summed in (u, v) order."""
    co, ci, k, _ = W.shape
    p = (k - 1) // 2
    C, H, Wd = x.shape
    assert C == ci
    xp = np.pad(x, ((0, 0), (p, p), (p, p)))
    y = np.broadcast_to(b[:, None, None], (co, H, Wd)).astype(np.float64).copy()
    for u in range(k):
        for v in range(k):
            y += np.tensordot(W[:, :, u, v], xp[:, u:u + H, v:v + Wd], axes=(1, 0))
    return y


def conv2d_adjoint(gy: np.ndarray, x: np.ndarray, W: np.ndarray):
    """Adjoint of conv2d: (dx, dW, db) for output cotangent gy."""
    co, ci, k, _ = W.shape
    p = (k - 1) // 2
    C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for u in range(k):
        for v in range(k):
            dxp[:, u:u + H, v:v + Wd] += np.tensordot(W[:, :, u, v], gy, axes=(0, 0))
            dW[:, :, u, v] = np.tensordot(gy, xp[:, u:u + H, v:v + Wd], axes=([1, 2], [1, 2]))
    dx = dxp[:, p:p + H, p:p + Wd] if p else dxp
    db = gy.sum(axis=(1, 2))
    return dx, dW, db


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x: np.ndarray) -> np.ndarray:
    """2x2 average pooling, stride 2 (H, W even)."""
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_adjoint(gy: np.ndarray) -> np.ndarray:
    return 0.25 * np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2)


def _bilinear_taps(n: int):
    """Output index o of a x2 upsample samples the input at o/2 - 1/4
    (half-pixel centres).  Returns (i0, i1, w0, w1) with clamped indices."""
    o = np.arange(2 * n)
    src = (o + 0.5) / 2.0 - 0.5
    i0 = np.floor(src).astype(np.int64)
    w1 = src - i0
    w0 = 1.0 - w1
    i1 = i0 + 1
    return np.clip(i0, 0, n - 1), np.clip(i1, 0, n - 1), w0, w1


def upsample2(x: np.ndarray) -> np.ndarray:
    """Bilinear x2 upsampling, align_corners = False, edge clamp."""
    C, H, W = x.shape
    y0, y1, wy0, wy1 = _bilinear_taps(H)
    x0, x1, wx0, wx1 = _bilinear_taps(W)
    rows = x[:, y0, :] * wy0[None, :, None] + x[:, y1, :] * wy1[None, :, None]
    return rows[:, :, x0] * wx0[None, None, :] + rows[:, :, x1] * wx1[None, None, :]


def upsample2_adjoint(gy: np.ndarray) -> np.ndarray:
    C, H2, W2 = gy.shape
    H, W = H2 // 2, W2 // 2
    y0, y1, wy0, wy1 = _bilinear_taps(H)
    x0, x1, wx0, wx1 = _bilinear_taps(W)
    g_rows = np.zeros((C, H2, W))
    np.add.at(g_rows, (slice(None), slice(None), x0), gy * wx0[None, None, :])
    np.add.at(g_rows, (slice(None), slice(None), x1), gy * wx1[None, None, :])
    gx = np.zeros((C, H, W))
    np.add.at(gx, (slice(None), y0, slice(None)), g_rows * wy0[None, :, None])
    np.add.at(gx, (slice(None), y1, slice(None)), g_rows * wy1[None, :, None])
    return gx


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


# ------------------------------------------------------------------ network


def forward(feat: np.ndarray, theta: np.ndarray, levels: int = 3, keep: bool = False):
    """Visibility (H, W) from features (4, H, W); H, W multiples of 2^(levels-1).
    With keep=True also returns the dict of every intermediate (for the adjoint)."""
    P = unpack(theta, levels)
    t = {}
    h = np.asarray(feat, np.float64)
    skips = {}
    for l in range(levels - 1):
        t[f"enc{l}_in"] = h
        a = conv2d(h, *P[f"enc{l}_3x3"])
        t[f"enc{l}_a3"] = a
        h3 = relu(a)
        t[f"enc{l}_h3"] = h3
        a1 = conv2d(h3, *P[f"enc{l}_1x1"])
        t[f"enc{l}_a1"] = a1
        h1 = relu(a1)
        t[f"enc{l}_h1"] = h1
        if l >= 1:
            skips[l] = h1
        h = avgpool2(h1)
    t["bott_in"] = h
    a = conv2d(h, *P["bott_3x3"])
    t["bott_a3"] = a
    h3 = relu(a)
    t["bott_h3"] = h3
    a1 = conv2d(h3, *P["bott_1x1"])
    t["bott_a1"] = a1
    h = relu(a1)
    t["bott_out"] = h
    for l in range(levels - 2, -1, -1):
        u = upsample2(h)
        x = u + skips[l] if l >= 1 else u
        t[f"dec{l}_in"] = x
        a = conv2d(x, *P[f"dec{l}_3x3"])
        t[f"dec{l}_a3"] = a
        h3 = relu(a)
        t[f"dec{l}_h3"] = h3
        a1 = conv2d(h3, *P[f"dec{l}_1x1"])
        t[f"dec{l}_a1"] = a1
        h = relu(a1)
        t[f"dec{l}_out"] = h
    logit = conv2d(h, *P["head"])[0]
    t["logit"] = logit
    vis = sigmoid(logit)
    t["vis"] = vis
    return (vis, t) if keep else vis


def backward(gvis: np.ndarray, theta: np.ndarray, t: dict, levels: int = 3):
    """Adjoint of `forward`: returns (dtheta flat, dfeat) for cotangent gvis (H, W)."""
    P = unpack(theta, levels)
    G = {}
    vis = t["vis"]
    glogit = (gvis * vis * (1.0 - vis))[None]
    gh, dW, db = conv2d_adjoint(glogit, t["dec0_out"], P["head"][0])
    G["head"] = (dW, db)
    gskip = {}
    for l in range(0, levels - 1):
        ga1 = gh * (t[f"dec{l}_a1"] > 0)
        gh3, dW, db = conv2d_adjoint(ga1, t[f"dec{l}_h3"], P[f"dec{l}_1x1"][0])
        G[f"dec{l}_1x1"] = (dW, db)
        ga3 = gh3 * (t[f"dec{l}_a3"] > 0)
        gx, dW, db = conv2d_adjoint(ga3, t[f"dec{l}_in"], P[f"dec{l}_3x3"][0])
        G[f"dec{l}_3x3"] = (dW, db)
        if l >= 1:
            gskip[l] = gx
        gh = upsample2_adjoint(gx)
    ga1 = gh * (t["bott_a1"] > 0)
    gh3, dW, db = conv2d_adjoint(ga1, t["bott_h3"], P["bott_1x1"][0])
    G["bott_1x1"] = (dW, db)
    ga3 = gh3 * (t["bott_a3"] > 0)
    gx, dW, db = conv2d_adjoint(ga3, t["bott_in"], P["bott_3x3"][0])
    G["bott_3x3"] = (dW, db)
    gh = gx
    for l in range(levels - 2, -1, -1):
        gh1 = avgpool2_adjoint(gh)
        if l >= 1:
            gh1 = gh1 + gskip[l]
        ga1 = gh1 * (t[f"enc{l}_a1"] > 0)
        gh3, dW, db = conv2d_adjoint(ga1, t[f"enc{l}_h3"], P[f"enc{l}_1x1"][0])
        G[f"enc{l}_1x1"] = (dW, db)
        ga3 = gh3 * (t[f"enc{l}_a3"] > 0)
        gx, dW, db = conv2d_adjoint(ga3, t[f"enc{l}_in"], P[f"enc{l}_3x3"][0])
        G[f"enc{l}_3x3"] = (dW, db)
        gh = gx
    return pack(G, levels), gh


# ------------------------------------------------------------------ reduced-precision storage


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits
    of an IEEE binary32 value.  (Inputs are first rounded to binary32.)"""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    u = (u & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def round_bf16_pair(x):
    """hi + lo with hi = bf16(x) and lo = bf16(x - hi): x to about 16 bits."""
    x32 = np.asarray(x, np.float32).astype(np.float64)
    hi = round_bf16(x32)
    lo = round_bf16((x32 - hi).astype(np.float32))
    return hi + lo


def e4m3_values():
    """All finite non-negative values of the FP8 E4M3 format (1 sign bit, 4
    exponent bits with bias 7, 3 mantissa bits; exponent field 0 encodes the
    subnormals m/8 * 2^-6; the all-ones exponent with mantissa 7 is NaN, so
    the largest finite value is 1.75 * 2^8 = 448; there are no infinities),
    enumerated from the bit fields: 127 values, ascending."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue
            vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(sorted(vals))


_E4M3 = None


def round_e4m3(x):
    """Round to the nearest E4M3 value, ties to the even mantissa, saturating
    at +-448 (the conversion an FP8 tensor-core form applies to values it
    stores).  Inputs are first rounded to binary32; returned as float64."""
    global _E4M3
    if _E4M3 is None:
        _E4M3 = e4m3_values()
    v = _E4M3
    a = np.abs(np.asarray(x, np.float32).astype(np.float64))
    a = np.minimum(a, v[-1])
    hi = np.clip(np.searchsorted(v, a, side="left"), 1, v.size - 1)
    lo_v, hi_v = v[hi - 1], v[hi]
    dl, dh = a - lo_v, hi_v - a
    # ties: the neighbour whose mantissa field is even (index parity follows the
    # mantissa field, since each binade holds 8 consecutive codes)
    pick_hi = (dh < dl) | ((dh == dl) & (hi % 2 == 0))
    q = np.where(a == hi_v, hi_v, np.where(pick_hi, hi_v, lo_v))
    return np.sign(np.asarray(x, np.float64)) * q


def round_e4m3_per_out_channel(W):
    """E4M3 weights with one scale per output channel (axis 0): s_o =
    max|W[o]| / 448 (1 for an all-zero channel), W ~ e4m3(W / s_o) * s_o."""
    W = np.asarray(W, np.float64)
    s = np.abs(W).reshape(W.shape[0], -1).max(axis=1) / 448.0
    s = np.where(s > 0, s, 1.0).reshape((-1,) + (1,) * (W.ndim - 1))
    return round_e4m3(W / s) * s


def round_e4m3_terms(x, terms: int = 3):
    """x held as the sum of `terms` E4M3 values at fixed scales 1, 2^-4, 2^-8,
    ...: a_0 = e4m3(x) and a_k = e4m3(16^k r_k) 16^-k for the residual r_k = x
    - (a_0 + ... + a_{k-1}) (each conversion rounds to nearest even and
    saturates at +-448, as `round_e4m3`), returned as the float64 sum.  Each
    term keeps the residual's top four significant bits, so ~12 bits survive
    for three terms; magnitudes beyond 448 (1 + 1/16 + 1/256 + ...) saturate."""
    x = np.asarray(x, np.float32).astype(np.float64)
    acc = np.zeros_like(x)
    for k in range(terms):
        s = 16.0 ** k
        acc = acc + round_e4m3((x - acc) * s) / s
    return acc


def round_e4m3_terms_per_out_channel(W, terms: int = 3):
    """`round_e4m3_terms` of W / s_o times s_o, one scale per output channel
    (axis 0): s_o = max|W[o]| / 448 (1 for an all-zero channel)."""
    W = np.asarray(W, np.float64)
    s = np.abs(W).reshape(W.shape[0], -1).max(axis=1) / 448.0
    s = np.where(s > 0, s, 1.0).reshape((-1,) + (1,) * (W.ndim - 1))
    return round_e4m3_terms(W / s, terms) * s


def upsample_coef(a: int, k: int, d: int) -> float:
    """Bilinear weight of coarse index i + d - 1 in fine index 2i + a + k - 1
    (half-pixel centres, as `upsample2` away from the clamped edge): fine
    index 2j takes coarse j - 1 and j with 1/4 and 3/4, fine 2j + 1 takes j
    and j + 1 with 3/4 and 1/4."""
    t = a + k - 1
    m, par = t // 2, t % 2
    taps = {m - 1: 0.25, m: 0.75} if par == 0 else {m: 0.75, m + 1: 0.25}
    return taps.get(d - 1, 0.0)


def upsample_conv_weights(W: np.ndarray) -> np.ndarray:
    """Effective 3x3 weights E[a, b] (O, C, 3, 3) on the coarse grid of a 3x3
    convolution W (O, C, 3, 3) that follows a bilinear x2 up-sampling: output
    pixel (2i + a, 2j + b) = sum_{dy,dx} E[a, b][:, :, dy, dx] x[:, i+dy-1, j+dx-1]
    wherever the up-sampled pixels it reads are inside the image (and their
    coarse taps unclamped, or the coarse input extended by edge replication)."""
    E = np.zeros((2, 2) + W.shape)
    for a in range(2):
        for b in range(2):
            for dy in range(3):
                for dx in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            q = upsample_coef(a, ky, dy) * upsample_coef(b, kx, dx)
                            if q:
                                E[a, b, :, :, dy, dx] += q * W[:, :, ky, kx]
    return E


def _coarse_grid_dec0(h, W3, b3, Weff, W1, b1, rnd_mid, Wexact):
    """Level-0 decoder pair (3x3 + ReLU -> 1x1 + ReLU) of the coarse input h,
    evaluated as the coarse-grid form does: the four output parities from the
    effective weights `Weff` over h extended by edge replication; the
    outermost ring of fine pixels exactly, from the up-sampled h with the
    unrounded weights `Wexact` (and no rounding of its 3x3 output)."""
    C, hh, ww = h.shape
    hp = np.pad(h, ((0, 0), (1, 1), (1, 1)), mode="edge")
    y = np.zeros((W3.shape[0], 2 * hh, 2 * ww))
    for a in range(2):
        for b in range(2):
            y[:, a::2, b::2] = conv2d(hp, Weff[a, b], b3)[:, 1:-1, 1:-1]
    out = relu(conv2d(rnd_mid(relu(y)), W1, b1))
    exact = relu(conv2d(relu(conv2d(upsample2(h), *Wexact[0])), *Wexact[1]))
    ring = np.ones(y.shape[1:], bool)
    ring[1:-1, 1:-1] = False
    out[:, ring] = exact[:, ring]
    return out


def forward_rounded(feat, theta, rnd, rnd_in=None, rnd_w=None, rnd_mid=None, levels: int = 3,
                    coarse_dec0: bool = False, ckpt: dict | None = None):
    """`forward` with values rounded wherever a reduced-precision form stores
    them: every convolution weight by `rnd_w` (not biases or the head), the
    3x3 output that feeds each 1x1 by `rnd_mid`, and by `rnd` each level's
    output (after pooling where the level pools; the level-1 skip separately;
    the up-sampled (+ skip) decoder inputs).  The input features are rounded
    by `rnd_in`.  `rnd_w` / `rnd_mid` default to `rnd`.  All arithmetic between
    those points is exact (FP64).
    coarse_dec0: the level-0 decoder as a coarse-grid form evaluates it
    (`_coarse_grid_dec0`): no rounding of its up-sampled input, its 3x3 from
    the effective weights of `upsample_conv_weights` rounded by `rnd_w`, and
    the outermost fine ring with the unrounded weights.
    ckpt: if a dict is given, it receives the stored level outputs as a form
    keeps them for a backward pass: "e0" (pooled level-0 encoder output),
    "s1" (level-1 skip), "p1" (pooled level-1 output), "bo" (bottleneck
    output), "d1" (level-1 decoder output) and "vis" (3-level network)."""
    rnd_w = rnd if rnd_w is None else rnd_w
    rnd_mid = rnd if rnd_mid is None else rnd_mid
    P = unpack(theta, levels)
    Wr = {k: ((rnd_w(W) if k != "head" else W), b) for k, (W, b) in P.items()}
    h = np.asarray(feat, np.float64) if rnd_in is None else rnd_in(feat)
    skips = {}

    def pair(x, l3, l1):
        a = rnd_mid(relu(conv2d(x, *Wr[l3])))
        return relu(conv2d(a, *Wr[l1]))

    store = ckpt if ckpt is not None else {}
    for l in range(levels - 1):
        h1 = pair(h, f"enc{l}_3x3", f"enc{l}_1x1")
        if l >= 1:
            skips[l] = rnd(h1)
            store[f"s{l}"] = skips[l]
        h = rnd(avgpool2(h1))
        store["e0" if l == 0 else f"p{l}"] = h
    h = rnd(pair(h, "bott_3x3", "bott_1x1"))
    store["bo"] = h
    for l in range(levels - 2, -1, -1):
        if l == 0 and coarse_dec0:
            W3, b3 = P["dec0_3x3"]
            Weff = rnd_w(upsample_conv_weights(W3))
            h = _coarse_grid_dec0(h, W3, b3, Weff, *Wr["dec0_1x1"], rnd_mid,
                                  (P["dec0_3x3"], P["dec0_1x1"]))
            continue
        u = upsample2(h)
        x = rnd(u + skips[l]) if l >= 1 else rnd(u)
        h = pair(x, f"dec{l}_3x3", f"dec{l}_1x1")
        if l >= 1:
            h = rnd(h)
            store[f"d{l}"] = h
    vis = sigmoid(conv2d(h, *Wr["head"])[0])
    store["vis"] = vis
    return vis


def recompute_from_checkpoints(feat, ckpt: dict, theta) -> dict:
    """The intermediates `backward` needs (the `t` of `forward(keep=True)`,
    3-level network), recomputed exactly level by level from stored level
    inputs, as a backward with activation recomputation does: the level-0
    encoder from the features, the level-1 encoder from ckpt["e0"], the
    bottleneck from ckpt["p1"], the level-1 decoder from up(ckpt["bo"]) +
    ckpt["s1"], the level-0 decoder from up(ckpt["d1"]); the output
    visibility is the stored ckpt["vis"].  With exact checkpoints this is
    `forward`'s t."""
    P = unpack(theta, 3)
    t = {}

    def level(name, x):
        t[f"{name}_in"] = x
        a = conv2d(x, *P[f"{name}_3x3"])
        t[f"{name}_a3"] = a
        h3 = relu(a)
        t[f"{name}_h3"] = h3
        a1 = conv2d(h3, *P[f"{name}_1x1"])
        t[f"{name}_a1"] = a1
        return relu(a1)

    t["enc0_h1"] = level("enc0", np.asarray(feat, np.float64))
    t["enc1_h1"] = level("enc1", ckpt["e0"])
    t["bott_out"] = level("bott", ckpt["p1"])
    t["dec1_out"] = level("dec1", upsample2(ckpt["bo"]) + ckpt["s1"])
    t["dec0_out"] = level("dec0", upsample2(ckpt["d1"]))
    t["logit"] = conv2d(t["dec0_out"], *P["head"])[0]
    t["vis"] = ckpt["vis"]
    return t


# ------------------------------------------------------------------ space-to-depth topology (Sec. 3.5)
# The paper's final first-layer optimisation: the level-0 convolutions are
# removed; a 2x2 square of full-resolution pixels is flattened into channels,
# so the 4 input features become 16 channels at half resolution and feed the
# second level directly; on the decoder side 4 output channels are rearranged
# into the 2x2 square, the first one bilinearly upscaled to full resolution
# and the other three added to it as the details.
# Readings (the text fixes neither): input channel order 4 * (2 a + b) + c for
# feature c of the pixel at offset (a, b) = (row, column) in the square; the
# three detail channels go to offsets (0, 1), (1, 0), (1, 1) (none to (0, 0));
# the sigmoid is applied to the recombined sum; the decoder's 1x1 output
# (16 channels) feeds a 1x1 head with 4 outputs.


def layer_table_s2d(levels: int = 3, base: int = 16):
    """The level-0 layers of `layer_table` removed and the head widened to 4
    outputs: the level-1 encoder takes the 16 space-to-depth channels."""
    t = [(n, ci, co, k) for (n, ci, co, k) in layer_table(levels, base) if not n.startswith(("enc0", "dec0"))]
    return [(n, ci, 4 if n == "head" else co, k) for (n, ci, co, k) in t]


def unpack_s2d(theta: np.ndarray, levels: int = 3):
    theta = np.asarray(theta, np.float64)
    out, off = {}, 0
    for (name, ci, co, k) in layer_table_s2d(levels):
        n = co * ci * k * k
        out[name] = (theta[off:off + n].reshape(co, ci, k, k), theta[off + n:off + n + co])
        off += n + co
    if off != theta.size:
        raise ValueError(f"weight vector has {theta.size} entries, expected {off}")
    return out


def space_to_depth(x: np.ndarray) -> np.ndarray:
    """(C, H, W) -> (4C, H/2, W/2): out[4 * (2a + b) + c, i, j] = x[c, 2i + a, 2j + b]."""
    C, H, W = x.shape
    y = np.empty((4 * C, H // 2, W // 2), x.dtype)
    for a in range(2):
        for b in range(2):
            y[C * (2 * a + b):C * (2 * a + b + 1)] = x[:, a::2, b::2]
    return y


def s2d_output(o: np.ndarray) -> np.ndarray:
    """(4, H/2, W/2) head outputs -> (H, W) pre-sigmoid values: the bilinear x2
    of channel 0 plus channels 1, 2, 3 at square offsets (0, 1), (1, 0), (1, 1)."""
    up = upsample2(o[0:1])[0]
    up[0::2, 1::2] += o[1]
    up[1::2, 0::2] += o[2]
    up[1::2, 1::2] += o[3]
    return up


def pack_s2d(params, levels: int = 3) -> np.ndarray:
    parts = []
    for (name, ci, co, k) in layer_table_s2d(levels):
        W, b = params[name]
        parts.append(np.asarray(W, np.float64).reshape(-1))
        parts.append(np.asarray(b, np.float64).reshape(-1))
    return np.concatenate(parts)


def space_to_depth_adjoint(g: np.ndarray) -> np.ndarray:
    """Adjoint (= inverse) of space_to_depth: (4C, H/2, W/2) -> (C, H, W)."""
    C4, H2, W2 = g.shape
    C = C4 // 4
    x = np.empty((C, 2 * H2, 2 * W2), g.dtype)
    for a in range(2):
        for b in range(2):
            x[:, a::2, b::2] = g[C * (2 * a + b):C * (2 * a + b + 1)]
    return x


def s2d_output_adjoint(g: np.ndarray) -> np.ndarray:
    """Adjoint of s2d_output: (H, W) cotangent -> (4, H/2, W/2)."""
    o = np.empty((4, g.shape[0] // 2, g.shape[1] // 2), g.dtype)
    o[0] = upsample2_adjoint(g[None])[0]
    o[1] = g[0::2, 1::2]
    o[2] = g[1::2, 0::2]
    o[3] = g[1::2, 1::2]
    return o


def forward_s2d(feat: np.ndarray, theta: np.ndarray, levels: int = 3, keep: bool = False):
    """Visibility of the space-to-depth network: the levels 1 .. L-1 of
    `forward` on space_to_depth(features), then the 4-channel head and the
    2x2 recombination (Sec. 3.5).  With keep=True also the intermediates."""
    P = unpack_s2d(theta, levels)
    t = {}
    h = space_to_depth(np.asarray(feat, np.float64))
    skips = {}

    def pair(x, name):
        t[f"{name}_in"] = x
        a3 = conv2d(x, *P[f"{name}_3x3"])
        h3 = relu(a3)
        a1 = conv2d(h3, *P[f"{name}_1x1"])
        t[f"{name}_a3"], t[f"{name}_h3"], t[f"{name}_a1"] = a3, h3, a1
        return relu(a1)

    for l in range(1, levels - 1):
        h1 = pair(h, f"enc{l}")
        skips[l] = h1
        h = avgpool2(h1)
    h = pair(h, "bott")
    for l in range(levels - 2, 0, -1):
        h = pair(upsample2(h) + skips[l], f"dec{l}")
    t["head_in"] = h
    vis = sigmoid(s2d_output(conv2d(h, *P["head"])))
    t["vis"] = vis
    return (vis, t) if keep else vis


def backward_s2d(gvis: np.ndarray, theta: np.ndarray, t: dict, levels: int = 3):
    """Adjoint of `forward_s2d`: (dtheta flat in layer_table_s2d order, dfeat)
    for the cotangent gvis (H, W)."""
    P = unpack_s2d(theta, levels)
    G = {}
    vis = t["vis"]
    go = s2d_output_adjoint(gvis * vis * (1.0 - vis))
    gh, dW, db = conv2d_adjoint(go, t["head_in"], P["head"][0])
    G["head"] = (dW, db)

    def pair_adj(gout, name):
        ga1 = gout * (t[f"{name}_a1"] > 0)
        gh3, dW1, db1 = conv2d_adjoint(ga1, t[f"{name}_h3"], P[f"{name}_1x1"][0])
        G[f"{name}_1x1"] = (dW1, db1)
        ga3 = gh3 * (t[f"{name}_a3"] > 0)
        gx, dW3, db3 = conv2d_adjoint(ga3, t[f"{name}_in"], P[f"{name}_3x3"][0])
        G[f"{name}_3x3"] = (dW3, db3)
        return gx

    gskip = {}
    for l in range(1, levels - 1):
        gx = pair_adj(gh, f"dec{l}")
        gskip[l] = gx
        gh = upsample2_adjoint(gx)
    gh = pair_adj(gh, "bott")
    for l in range(levels - 2, 0, -1):
        gh = pair_adj(avgpool2_adjoint(gh) + gskip[l], f"enc{l}")
    return pack_s2d(G, levels), space_to_depth_adjoint(gh)


def train_step_s2d(batch_feats, targets, theta, m, v, step, lr=1e-3, alpha=0.9, levels=3):
    """`train_step` for the space-to-depth network (same Eq. 2 loss, Adam)."""
    B = len(batch_feats)
    grad = np.zeros_like(np.asarray(theta, np.float64))
    total = 0.0
    for b in range(B):
        insts = batch_feats[b]
        x0, t = forward_s2d(insts[0], theta, levels, keep=True)
        xs = [forward_s2d(f, theta, levels) for f in insts[1:]]
        loss, g = loss_l1(x0, targets[b], xs, alpha)
        total += loss / B
        dth, _ = backward_s2d(g / B, theta, t, levels)
        grad += dth
    theta2, m2, v2 = adam_update(theta, grad, m, v, step, lr)
    return theta2, m2, v2, total, grad


# ------------------------------------------------------------------ loss (Eq. 2)


def loss_l1(x0: np.ndarray, target: np.ndarray, xs, alpha: float = 0.9):
    """Eq. 2 with the per-pixel term L(y, y~) = alpha |y - y~| (the VGG-19 term
    is not evaluated: its ImageNet weights are unavailable), averaged over
    pixels:  alpha mean|x0 - x~| + sum_i alpha mean|x0 - x_i|.
    Gradient flows through x0 only; d|u|/du at u = 0 is taken as 0.
    Returns (loss, dloss/dx0)."""
    n = x0.size
    loss = alpha * np.abs(x0 - target).sum() / n
    g = alpha * np.sign(x0 - target) / n
    for xi in xs:
        loss += alpha * np.abs(x0 - xi).sum() / n
        g = g + alpha * np.sign(x0 - xi) / n
    return float(loss), g


def adam_update(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; step >= 1.
    Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta, m, v


def train_step(batch_feats, targets, theta, m, v, step, lr=1e-3, alpha=0.9, levels=3, detached_forward=None,
               target_forward=None):
    """One temporal-window training step (Sec. 3.3, Eq. 2).

    batch_feats: list over batch items of lists over window instances of
    features (4, H, W); instance 0 carries the target and the gradient, the
    others are evaluated without gradient.  The per-item losses are averaged
    over the batch.  detached_forward(features, theta) evaluates the
    instances without gradient (default: `forward`; a reduced-precision
    form's rounding model, e.g. `forward_rounded`, for a form that runs them
    at lower precision).  target_forward(features, theta), if given, gives
    the visibility of instance 0 that enters the loss (a form that runs the
    target's forward at lower precision); the adjoint is still taken at the
    exact activations of `forward`.  Returns (theta, m, v, loss, grad)."""
    B = len(batch_feats)
    grad = np.zeros_like(np.asarray(theta, np.float64))
    total = 0.0
    fwd_detached = detached_forward if detached_forward is not None else (lambda f, th: forward(f, th, levels))
    for b in range(B):
        insts = batch_feats[b]
        x0, t = forward(insts[0], theta, levels, keep=True)
        if target_forward is not None:
            x0 = target_forward(insts[0], theta)
        xs = [fwd_detached(f, theta) for f in insts[1:]]
        loss, g = loss_l1(x0, targets[b], xs, alpha)
        total += loss / B
        dth, _ = backward(g / B, theta, t, levels)
        grad += dth
    theta2, m2, v2 = adam_update(theta, grad, m, v, step, lr)
    return theta2, m2, v2, total, grad
