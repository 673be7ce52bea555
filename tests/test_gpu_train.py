"""GPU checks of the hand-written backward (nsm_backward), the training step
(nsm_train_step, Eq. 2 with Adam) and the torch.autograd.Function wrapper,
against the FP64 oracle's adjoint and central finite differences."""
import math

import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, device_batch, train_batch_frames  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = nsm.Context()
    yield c
    c.check()
    c.close()


def _theta(seed):
    """He-normal weights and small random biases (non-zero, so every bias
    gradient path is exercised)."""
    rng = np.random.default_rng(seed)
    parts = []
    for (_, ci, co, k) in N.layer_table(3):
        parts.append(rng.standard_normal(co * ci * k * k) * math.sqrt(2.0 / (ci * k * k)))
        parts.append(rng.standard_normal(co) * 0.05)
    return np.concatenate(parts).astype(np.float32)


def _layer_slices():
    out, off = [], 0
    for (name, ci, co, k) in N.layer_table(3):
        nw = ci * co * k * k
        out.append((name + ".w", slice(off, off + nw)))
        out.append((name + ".b", slice(off + nw, off + nw + co)))
        off += nw + co
    return out


def _gpu_backward(ctx, f, theta, gvis, precision=None):
    df = DeviceFrame(f)
    params = torch.from_numpy(theta).cuda()
    gv = torch.from_numpy(gvis.astype(np.float32)).cuda()
    gp = torch.zeros_like(params)
    gf = torch.empty((f.H, f.W, 4), device="cuda")
    vis = torch.empty((f.H, f.W), device="cuda")
    ws = torch.empty((nsm.nsm_backward_workspace_bytes(f.H, f.W),), dtype=torch.uint8, device="cuda")
    nsm.nsm_backward(ctx, df.frame, params, gv, gp, ws, grad_feat=gf, vis_out=vis, precision=precision)
    torch.cuda.synchronize()
    ctx.check()
    return gp.cpu().numpy().astype(np.float64), gf.cpu().numpy().astype(np.float64), vis.cpu().numpy()


@pytest.mark.parametrize("size", [(32, 32), (36, 68)])
def test_backward_matches_oracle_adjoint(ctx, size):
    H, W = size
    f = scenegen.soft_frame(H, W, 128, 128, 8, 31)
    theta = _theta(1)
    gvis = np.random.default_rng(2).standard_normal((H, W))
    gp, gf, vis = _gpu_backward(ctx, f, theta, gvis)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref_vis, t = N.forward(feat, theta.astype(np.float64), keep=True)
    ref_g, ref_gf = N.backward(gvis, theta.astype(np.float64), t)
    assert np.abs(vis - ref_vis).max() < 1e-4
    for name, sl in _layer_slices():
        a, b = gp[sl], ref_g[sl]
        scale = max(np.abs(b).max(), 1e-12)
        assert np.abs(a - b).max() <= 2e-4 * scale, (name, np.abs(a - b).max(), scale)
    scale = np.abs(ref_gf).max()
    assert np.abs(gf - ref_gf.transpose(1, 2, 0)).max() <= 2e-4 * scale


def _relu_tie_columns(gvis, theta, t, tau=1e-5):
    """ReLU masks a recomputation with ~2^-17 relative operand rounding may
    decide either way: for every pre-activation (*_a3, *_a1) within tau of 0,
    relative to its tensor's largest, the change of the FP64 adjoint's
    (dtheta, dfeat) when that mask bit flips.  A correct gradient is the
    adjoint plus a 0 / 1 combination of these columns."""
    g0, f0 = N.backward(gvis, theta, t)
    cg, cf = [], []
    for k, v in t.items():
        if not k.endswith(("_a3", "_a1")):
            continue
        m = np.abs(v).max()
        for idx in zip(*np.nonzero(np.abs(v) < tau * m)):
            v2 = v.copy()
            v2[idx] = -v2[idx] if v2[idx] != 0 else -1e-300
            g2, f2 = N.backward(gvis, theta, {**t, k: v2})
            cg.append(g2 - g0)
            cf.append((f2 - f0).ravel())
    if not cg:
        return g0, f0, np.zeros((g0.size, 0)), np.zeros((f0.size, 0))
    return g0, f0, np.stack(cg, axis=1), np.stack(cf, axis=1)


def _fit_flips(gp, gf, ref_g, ref_gf, Cg, Cf):
    """Greedy 0 / 1 choice of the flipped masks (columns of _relu_tie_columns):
    add, one at a time, the column that most reduces the squared residual, on
    the even-indexed parameters and the feature gradient, each normalised by
    its layer's largest entry (the odd-indexed half is left to check it)."""
    even = np.arange(ref_g.size) % 2 == 0
    rows = [(sl.start + np.nonzero(even[sl])[0], max(np.abs(ref_g[sl]).max(), 1e-12)) for _, sl in _layer_slices()]
    fs = np.abs(ref_gf).max()
    A = np.concatenate([Cg[i] / sc for i, sc in rows] + [Cf / fs])
    r = np.concatenate([(gp - ref_g)[i] / sc for i, sc in rows] + [(gf - ref_gf) / fs])
    sgn = np.zeros(Cg.shape[1])
    norms = (A * A).sum(axis=0)
    while True:
        gain = 2.0 * (r @ A) - norms       # |r|^2 - |r - a_j|^2
        gain[sgn > 0] = -np.inf
        j = int(np.argmax(gain)) if gain.size else -1
        if j < 0 or gain[j] <= 0.0:
            break
        sgn[j] = 1.0
        r = r - A[:, j]
    return sgn


@pytest.mark.parametrize("size", [(32, 32), (36, 68), (40, 260)])
def test_backward_bf16_convolutions_match_oracle_adjoint(ctx, size):
    """The backward with its 3x3 recomputations, data gradients and every
    weight gradient on the tcgen05 kernels (compensated BF16 operands, FP32
    accumulation, per-CTA slots added in a fixed order) against the FP64
    adjoint, layer by layer and for the feature gradient.  The sizes span
    several 128-pixel tiles with ragged tails at every level (260 = 2 x 128 + 4
    columns at level 0, 130 at level 1; 260 = 8 x 32 + 4 and 130 = 8 x 16 + 2
    columns of the weight-gradient tiles) and rows that are not a multiple of
    the tiles'.  Each operand keeps ~2^-17 of relative rounding, which can flip the
    recomputed ReLU mask of a pre-activation within ~1e-6 of 0: those flips
    are fitted (0 / 1 per near-zero pre-activation, on the even-indexed
    parameters), and the rest must meet the FP32 backward's bar on every
    parameter and on the feature gradient."""
    H, W = size
    f = scenegen.soft_frame(H, W, 128, 128, 8, 31)
    theta = _theta(1)
    gvis = np.random.default_rng(2).standard_normal((H, W))
    gp, gf, vis = _gpu_backward(ctx, f, theta, gvis, precision=nsm.NSM_BF16)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    th64 = theta.astype(np.float64)
    ref_vis, t = N.forward(feat, th64, keep=True)
    ref_g, ref_gf, Cg, Cf = _relu_tie_columns(gvis, th64, t)
    assert np.abs(vis - ref_vis).max() < 1e-4
    gf_flat = gf.transpose(2, 0, 1).ravel()
    sgn = _fit_flips(gp, gf_flat, ref_g, ref_gf.ravel(), Cg, Cf)
    print(f"near-zero pre-activations: {Cg.shape[1]}, fitted as flipped: {int(sgn.sum())}")
    fit_g, fit_f = ref_g + Cg @ sgn, ref_gf.ravel() + Cf @ sgn
    worst = 0.0
    for name, sl in _layer_slices():
        scale = max(np.abs(ref_g[sl]).max(), 1e-12)
        err = np.abs(gp[sl] - fit_g[sl]).max() / scale
        worst = max(worst, err)
        assert err <= 2e-4, (name, err)
    gerr = np.abs(gf_flat - fit_f).max() / np.abs(ref_gf).max()
    print(f"worst per-layer gradient error {worst:.2e}, feature gradient {gerr:.2e} (relative to the largest)")
    assert gerr <= 2e-4


def test_bf16_backward_gradient_is_the_same_bits_every_run(ctx):
    """With the backward on the tensor cores no gradient is summed by atomics:
    every weight gradient (and the head's) is reduced from per-CTA slots in a
    fixed order, so two steps' gradients from the same state and batch are
    bit-identical.  B = 8 items of 128 x 128 crops: hundreds of CTAs at every
    level.  The FP32 backward, whose weight gradients are summed by atomics,
    agrees with it to FP32 accuracy."""
    B, T, H, W, S = 8, 1, 128, 128, 256
    frames, targets = train_batch_frames(B, T, H, W, S, seed=47)
    theta = _theta(10)
    bt = device_batch(frames, targets)
    grads = []
    for prec in (nsm.NSM_BF16, nsm.NSM_BF16, nsm.NSM_FP32):
        st = nsm.TrainState(ctx, theta, B, T, H, W)
        st.set_backward_precision(prec)
        for _ in range(2):
            st.grad(bt, alpha=0.9)
            g = torch.empty(theta.size, device="cuda")
            st.read(1, g)
            torch.cuda.synchronize()
            grads.append(g.cpu().numpy())
        st.close()
    a, b, c, d, e, _ = grads
    for other in (b, c, d):
        assert np.array_equal(a, other)
    for name, sl in _layer_slices():
        scale = max(np.abs(e[sl]).max(), 1e-12)
        assert np.abs(a[sl] - e[sl]).max() <= 1e-3 * scale, name


def test_backward_central_finite_differences(ctx):
    """GPU gradient against central differences (h = 1e-3) of the FP64 oracle
    forward on a 32 x 32 crop; coordinates whose stencil flips a ReLU are skipped."""
    H = W = 32
    f = scenegen.soft_frame(H, W, 128, 128, 8, 33)
    theta = _theta(3)
    gvis = np.random.default_rng(4).standard_normal((H, W))
    gp, _, _ = _gpu_backward(ctx, f, theta, gvis)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    th = theta.astype(np.float64)
    _, t0 = N.forward(feat, th, keep=True)

    def pattern(tt):
        return np.concatenate([(tt[k] > 0).ravel() for k in tt if k.endswith(("_a3", "_a1"))])

    p0 = pattern(t0)
    rng = np.random.default_rng(5)
    idx = list(rng.choice(th.size, 50, replace=False))
    idx += [sl.start for _, sl in _layer_slices()]
    h = 1e-3
    checked = 0
    for i in idx:
        tp = th.copy(); tp[i] += h
        tm = th.copy(); tm[i] -= h
        vp, ttp = N.forward(feat, tp, keep=True)
        vm, ttm = N.forward(feat, tm, keep=True)
        if not (np.array_equal(pattern(ttp), p0) and np.array_equal(pattern(ttm), p0)):
            continue
        fd = (np.sum(gvis * vp) - np.sum(gvis * vm)) / (2 * h)
        assert abs(gp[i] - fd) <= 1e-3 * abs(fd) + 1e-5, (i, gp[i], fd)
        checked += 1
    assert checked >= 40


def test_autograd_function_matches_oracle(ctx):
    H = W = 32
    f = scenegen.hard_frame(H, W, 128, 128, 8, 35)
    theta = _theta(6)
    df = DeviceFrame(f)
    F = nsm.autograd_function()
    params = torch.from_numpy(theta).cuda().requires_grad_(True)
    vis = F.apply(params, ctx, df.frame)
    g = torch.from_numpy(np.random.default_rng(7).standard_normal((H, W)).astype(np.float32)).cuda()
    (vis * g).sum().backward()
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref_vis, t = N.forward(feat, theta.astype(np.float64), keep=True)
    ref_g, _ = N.backward(g.cpu().numpy().astype(np.float64), theta.astype(np.float64), t)
    assert np.abs(vis.detach().cpu().numpy() - ref_vis).max() < 1e-4
    got = params.grad.cpu().numpy()
    assert np.abs(got - ref_g).max() <= 2e-4 * np.abs(ref_g).max()


def _near_tie_split(feats, targets, theta, alpha, tau=1e-5, detached=None, target_fwd=None, target_t=None):
    """The Eq. 2 gradient split at the kink of |u| at 0.  Where |x0 - x_i| (or
    |x0 - target|) is below tau an FP32 evaluation may take either sign of the
    L1 term (or 0 at an exact tie), so the FP64 gradient with those terms left
    out (g_rest) is returned together with one column per such pixel: its
    contribution alpha / n / B * d x0(p) / d theta with sign +1.  A correct FP32
    gradient is g_rest + C s with every s_p in [-1, 1]."""
    B = len(feats)
    g_rest = np.zeros_like(theta)
    cols = []
    for b in range(B):
        x0, t = (target_t or (lambda f, th: N.forward(f, th, keep=True)))(feats[b][0], theta)
        if target_fwd is not None:
            x0 = target_fwd(feats[b][0], theta)
        fwd = detached if detached is not None else N.forward
        others = [np.asarray(targets[b], np.float64)] + [fwd(f, theta) for f in feats[b][1:]]
        n = x0.size
        cot = np.zeros_like(x0)
        for o in others:
            d = x0 - o
            tie = np.abs(d) < tau
            cot += alpha / n / B * np.where(tie, 0.0, np.sign(d))
            for (y, x) in zip(*np.nonzero(tie)):
                one = np.zeros_like(x0)
                one[y, x] = alpha / n / B
                cols.append(N.backward(one, theta, t)[0])
        g_rest += N.backward(cot, theta, t)[0]
    C = np.stack(cols, axis=1) if cols else np.zeros((theta.size, 0))
    return g_rest, C


@pytest.mark.parametrize("backward", ["fp32", "bf16"])
def test_train_step_matches_oracle(ctx, backward):
    """One temporal-window step (B = 2 items, T = 3 instances, 32 x 32 crops):
    loss, gradient and Adam-updated weights against the oracle's train_step;
    the backward's 3x3 layers on the FP32 kernels or on the tcgen05 kernels
    (compensated BF16 operands)."""
    B, T, H, W, S = 2, 3, 32, 32, 128
    frames, targets = train_batch_frames(B, T, H, W, S, seed=41)
    theta = _theta(8)
    st = nsm.TrainState(ctx, theta, B, T, H, W)
    if backward == "bf16":
        st.set_backward_precision(nsm.NSM_BF16)
    bt = device_batch(frames, targets)
    loss = torch.zeros(1, device="cuda")
    lr = 1e-3
    st.step(bt, lr=lr, alpha=0.9, loss_out=loss)
    out = {k: torch.empty(theta.size, device="cuda") for k in (0, 1)}
    for k, v in out.items():
        st.read(k, v)
    torch.cuda.synchronize()
    feats = []
    for b in range(B):
        insts = []
        for t in range(T):
            fr = frames[t][b]
            ft, _, _ = G.features(fr.pos4, fr.nrm4, fr.sm, fr.view_proj, fr.light_pos, fr.cam_pos, fr.r_hat,
                                  fr.z_far, fr.bias)
            insts.append(ft)
        feats.append(insts)
    th64 = theta.astype(np.float64)
    th2, _, _, ref_loss, ref_grad = N.train_step(feats, [targets[b].astype(np.float64) for b in range(B)], th64,
                                                 np.zeros_like(th64), np.zeros_like(th64), 1, lr=lr, alpha=0.9)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    grad = out[1].cpu().numpy().astype(np.float64)
    # FP32 may take either sign of |x0 - x_i| at near-ties: fit those signs, then
    # the rest must agree to FP32 accuracy and every fitted sign lie in [-1, 1]
    # (one free sign per near-tie term, so their number is bounded, and the
    # signs are fitted on the even-indexed parameters only: the odd-indexed
    # half, held out, checks the fit)
    g_rest, Ct = _near_tie_split(feats, [targets[b] for b in range(B)], th64, alpha=0.9)
    n_terms = B * T * H * W
    print(f"near-tie L1 terms: {Ct.shape[1]} of {n_terms}")
    assert Ct.shape[1] <= 0.01 * n_terms
    even = np.arange(th64.size) % 2 == 0
    sgn = np.linalg.lstsq(Ct[even], (grad - g_rest)[even], rcond=None)[0] if Ct.shape[1] else np.zeros(0)
    assert np.all(np.abs(sgn) <= 1.05), sgn
    fit = g_rest + Ct @ sgn
    for name, sl in _layer_slices():
        scale = max(np.abs(ref_grad[sl]).max(), 1e-12)
        assert np.abs(grad[sl] - fit[sl]).max() <= 2e-3 * scale, name
        held = sl.start + np.nonzero(~even[sl])[0]
        assert np.abs(grad[held] - fit[held]).max(initial=0.0) <= 2e-3 * scale, name
    # Adam's first step moves every weight by about lr * sign(g); compare where the
    # gradient is clearly non-zero and no near-tie can change its sign
    new = out[0].cpu().numpy().astype(np.float64)
    big = (np.abs(ref_grad) > 1e-3 * np.abs(ref_grad).max()) & (np.abs(ref_grad) > 2.0 * np.abs(Ct).sum(axis=1))
    np.testing.assert_allclose((new - th64)[big], (th2 - th64)[big], rtol=1e-3, atol=1e-7)


def test_training_reduces_the_loss(ctx):
    B, T, H, W, S = 4, 3, 64, 64, 256
    frames, targets = train_batch_frames(B, T, H, W, S, seed=43)
    theta = scenegen.he_init_weights(9, N.layer_table(3)).astype(np.float32)
    st = nsm.TrainState(ctx, theta, B, T, H, W)
    bt = device_batch(frames, targets)
    loss = torch.zeros(1, device="cuda")
    losses = []
    for _ in range(60):
        st.step(bt, lr=3e-3, loss_out=loss)
        losses.append(float(loss.item()))
    assert all(np.isfinite(losses))
    assert min(losses[-10:]) < 0.7 * losses[0], (losses[0], losses[-10:])


def test_grad_apply_and_data_parallel_trainer_match_train_step(ctx):
    """nsm_train_grad + nsm_train_apply is nsm_train_step; a gradient written
    back through nsm_train_state_write is the one applied; the data-parallel
    trainer on one rank (the exchange is the identity) takes the same steps."""
    from paper_2301_05262_gb300.data_parallel import DataParallelTrainer
    B, T, H, W, S = 2, 3, 32, 32, 128
    frames, targets = train_batch_frames(B, T, H, W, S, seed=43)
    theta = _theta(9)
    bt = device_batch(frames, targets)
    a = nsm.TrainState(ctx, theta, B, T, H, W)
    b = nsm.TrainState(ctx, theta, B, T, H, W)
    c = nsm.TrainState(ctx, theta, B, T, H, W)
    dp = DataParallelTrainer(c)
    g = torch.empty(theta.size, device="cuda")
    for _ in range(2):
        a.step(bt, lr=1e-3)
        b.grad(bt)
        b.read(1, g)
        b.write(1, g.clone())
        b.apply(lr=1e-3)
        dp.step(bt, lr=1e-3)
    out = [torch.empty(theta.size, device="cuda") for _ in range(3)]
    for st, o in zip((a, b, c), out):
        st.read(0, o)
    torch.cuda.synchronize()
    # weight gradients are summed with FP32 atomics across CTAs, so two runs of
    # the same step agree to rounding, not bit for bit
    np.testing.assert_allclose(out[0].cpu().numpy(), out[1].cpu().numpy(), rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(out[0].cpu().numpy(), out[2].cpu().numpy(), rtol=1e-5, atol=1e-7)
    # a gradient set by hand moves the weights by lr * sign(g) on the first Adam step
    d = nsm.TrainState(ctx, theta, B, T, H, W)
    gh = torch.from_numpy(np.where(np.arange(theta.size) % 2 == 0, 1.0, -1.0).astype(np.float32)).cuda()
    d.write(1, gh)
    d.apply(lr=1e-3)
    w = torch.empty(theta.size, device="cuda")
    d.read(0, w)
    torch.cuda.synchronize()
    np.testing.assert_allclose(w.cpu().numpy() - theta, -1e-3 * gh.cpu().numpy(), rtol=1e-4, atol=1e-7)


def test_train_step_with_bf16_detached_instances(ctx):
    """The detached instances x_1, x_2 of Eq. 2 on the BF16 tensor-core stage
    kernels: their visibilities follow the BF16 form's rounding model (and lie
    within 1e-2 of FP64), x_0 stays FP32, and the loss, gradient and Adam step
    match the oracle's step with that rounding model as the detached forward."""
    B, T, H, W, S = 2, 3, 32, 32, 128
    frames, targets = train_batch_frames(B, T, H, W, S, seed=41)
    theta = _theta(8)
    st = nsm.TrainState(ctx, theta, B, T, H, W)
    st.set_detached_precision(nsm.NSM_BF16)
    bt = device_batch(frames, targets)
    loss = torch.zeros(1, device="cuda")
    lr = 1e-3
    st.step(bt, lr=lr, alpha=0.9, loss_out=loss)
    vis = torch.empty(T * B * H * W, device="cuda")
    st.read_vis(vis)
    out = {k: torch.empty(theta.size, device="cuda") for k in (0, 1)}
    for k, v in out.items():
        st.read(k, v)
    torch.cuda.synchronize()
    v = vis.cpu().numpy().astype(np.float64).reshape(T, B, H, W)
    th64 = theta.astype(np.float64)
    model = lambda f, th: N.forward_rounded(f, th, N.round_bf16_pair, rnd_in=N.round_bf16_pair, coarse_dec0=True)
    feats = []
    for b in range(B):
        insts = []
        for t in range(T):
            fr = frames[t][b]
            insts.append(G.features(fr.pos4, fr.nrm4, fr.sm, fr.view_proj, fr.light_pos, fr.cam_pos, fr.r_hat,
                                    fr.z_far, fr.bias)[0])
        feats.append(insts)
        assert np.abs(v[0, b] - N.forward(insts[0], th64)).max() <= 1e-4          # x_0: FP32
        for t in range(1, T):
            q = model(insts[t], th64)
            assert float(np.mean((v[t, b] - q) ** 2)) <= 1e-8
            assert np.abs(v[t, b] - q).max() <= 1e-3
            assert np.abs(v[t, b] - N.forward(insts[t], th64)).max() <= 1e-2
    th2, _, _, ref_loss, ref_grad = N.train_step(feats, [targets[b].astype(np.float64) for b in range(B)], th64,
                                                 np.zeros_like(th64), np.zeros_like(th64), 1, lr=lr, alpha=0.9,
                                                 detached_forward=model)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    grad = out[1].cpu().numpy().astype(np.float64)
    g_rest, Ct = _near_tie_split(feats, [targets[b] for b in range(B)], th64, alpha=0.9, detached=model)
    n_terms = B * T * H * W
    print(f"near-tie L1 terms: {Ct.shape[1]} of {n_terms}")
    assert Ct.shape[1] <= 0.01 * n_terms
    even = np.arange(th64.size) % 2 == 0
    sgn = np.linalg.lstsq(Ct[even], (grad - g_rest)[even], rcond=None)[0] if Ct.shape[1] else np.zeros(0)
    assert np.all(np.abs(sgn) <= 1.05), sgn
    fit = g_rest + Ct @ sgn
    for name, sl in _layer_slices():
        scale = max(np.abs(ref_grad[sl]).max(), 1e-12)
        assert np.abs(grad[sl] - fit[sl]).max() <= 2e-3 * scale, name
    new = out[0].cpu().numpy().astype(np.float64)
    big = (np.abs(ref_grad) > 1e-3 * np.abs(ref_grad).max()) & (np.abs(ref_grad) > 2.0 * np.abs(Ct).sum(axis=1))
    np.testing.assert_allclose((new - th64)[big], (th2 - th64)[big], rtol=1e-3, atol=1e-7)
    st.close()


@pytest.mark.parametrize("backward", ["fp32", "bf16"])
def test_train_step_with_every_forward_on_the_tensor_cores(ctx, backward):
    """x_0 and the detached instances on the BF16 tcgen05 stage kernels (the
    backward FP32 from the converted checkpoints): every visibility follows the
    BF16 rounding model; loss and gradient match the oracle's with x_0's
    visibility and level checkpoints from that model and the adjoint's
    activations recomputed exactly from the checkpoints, as the backward does
    (near-tie signs fitted on half the parameters and checked on the rest)."""
    B, T, H, W, S = 2, 3, 32, 32, 128
    frames, targets = train_batch_frames(B, T, H, W, S, seed=41)
    theta = _theta(8)
    st = nsm.TrainState(ctx, theta, B, T, H, W)
    st.set_detached_precision(nsm.NSM_BF16)
    st.set_forward_precision(nsm.NSM_BF16)
    if backward == "bf16":
        st.set_backward_precision(nsm.NSM_BF16)
    bt = device_batch(frames, targets)
    loss = torch.zeros(1, device="cuda")
    lr = 1e-3
    st.step(bt, lr=lr, alpha=0.9, loss_out=loss)
    vis = torch.empty(T * B * H * W, device="cuda")
    st.read_vis(vis)
    out = {k: torch.empty(theta.size, device="cuda") for k in (0, 1)}
    for k, v in out.items():
        st.read(k, v)
    torch.cuda.synchronize()
    v = vis.cpu().numpy().astype(np.float64).reshape(T, B, H, W)
    th64 = theta.astype(np.float64)
    model = lambda f, th: N.forward_rounded(f, th, N.round_bf16_pair, rnd_in=N.round_bf16_pair, coarse_dec0=True)
    feats = []
    for b in range(B):
        insts = []
        for t in range(T):
            fr = frames[t][b]
            insts.append(G.features(fr.pos4, fr.nrm4, fr.sm, fr.view_proj, fr.light_pos, fr.cam_pos, fr.r_hat,
                                    fr.z_far, fr.bias)[0])
        feats.append(insts)
        for t in range(T):
            q = model(insts[t], th64)
            assert float(np.mean((v[t, b] - q) ** 2)) <= 1e-8
            assert np.abs(v[t, b] - q).max() <= 1e-3
    # the reference a backward with recomputation takes: x_0's visibility and
    # level checkpoints from the BF16 form's rounding model, the adjoint's
    # activations recomputed exactly from those checkpoints
    def target_t(f, th):
        ck = {}
        x0 = N.forward_rounded(f, th, N.round_bf16_pair, rnd_in=N.round_bf16_pair, coarse_dec0=True, ckpt=ck)
        return x0, N.recompute_from_checkpoints(f, ck, th)

    ref_loss = 0.0
    ref_grad = np.zeros_like(th64)
    for b in range(B):
        x0, t = target_t(feats[b][0], th64)
        xs = [model(f, th64) for f in feats[b][1:]]
        l, g = N.loss_l1(x0, targets[b].astype(np.float64), xs, 0.9)
        ref_loss += l / B
        ref_grad += N.backward(g / B, th64, t)[0]
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    grad = out[1].cpu().numpy().astype(np.float64)
    g_rest, Ct = _near_tie_split(feats, [targets[b] for b in range(B)], th64, alpha=0.9, detached=model,
                                 target_t=target_t)
    n_terms = B * T * H * W
    print(f"near-tie L1 terms: {Ct.shape[1]} of {n_terms}")
    assert Ct.shape[1] <= 0.01 * n_terms
    even = np.arange(th64.size) % 2 == 0
    sgn = np.linalg.lstsq(Ct[even], (grad - g_rest)[even], rcond=None)[0] if Ct.shape[1] else np.zeros(0)
    assert np.all(np.abs(sgn) <= 1.05), sgn
    fit = g_rest + Ct @ sgn
    worst = 0.0
    for name, sl in _layer_slices():
        scale = max(np.abs(ref_grad[sl]).max(), 1e-12)
        err = np.abs(grad[sl] - fit[sl]).max() / scale
        worst = max(worst, err)
        assert err <= 2e-3, (name, err)
        held = sl.start + np.nonzero(~even[sl])[0]
        assert np.abs(grad[held] - fit[held]).max(initial=0.0) <= 2e-3 * scale, name
    print(f"worst per-layer gradient error relative to the layer's largest: {worst:.2e}")
    st.close()
