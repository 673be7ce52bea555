"""Host-only checks of the C-ABI library: it builds, loads, exports every
symbol include/nsm.h declares, and its host-side sizes and validation paths
behave as documented (no GPU work is issued)."""
import ctypes

import numpy as np
import pytest

import paper_2301_05262_gb300 as nsm
from paper_2301_05262_gb300 import build as nsm_build
from oracle import network as N


@pytest.fixture(scope="module")
def lib():
    nsm_build.build()
    return nsm.lib()


def test_exports_every_declared_symbol(lib):
    declared = nsm.declared_symbols()
    assert "nsm_features" in declared and "nsm_infer" in declared
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing


def test_abi_version_and_param_count(lib):
    assert lib.nsm_abi_version() == 1
    biases = sum(co for (_, _, co, _) in N.layer_table(3))
    assert nsm.nsm_param_count() == N.param_count(3) + biases == 39521
    assert [(c, o, k) for (_, c, o, k) in nsm.LAYERS] == [(c, o, k) for (_, c, o, k) in N.layer_table(3)]


def test_workspace_bytes(lib):
    # FP32 activations, or BF16 hi + lo pairs: 4 bytes per channel in both forms
    for prec, eb in ((nsm.NSM_FP32, 4), (nsm.NSM_BF16, 4)):
        H, W = 1080, 1920
        n = nsm.nsm_infer_workspace_bytes(H, W, prec)
        h2, h4 = (H // 2) * (W // 2), (H // 4) * (W // 4)
        assert n >= eb * (h2 * (16 + 32 + 16) + h4 * (32 + 32))
        assert n < eb * (h2 * (16 + 32 + 16) + h4 * (32 + 32)) + 5 * 256
    assert nsm.nsm_infer_workspace_bytes(0, 64, nsm.NSM_FP32) == 0


def test_host_validation_errors(lib):
    # NULL frame / NULL context are rejected before any CUDA call
    assert lib.nsm_features(None, None, None, None, None, None) == 1
    assert b"frame" in lib.nsm_last_error()
    assert lib.nsm_infer(None, None, None, 0, None, 0, None, None) == 1
    assert b"ctx" in lib.nsm_last_error()
    out = ctypes.c_void_p()
    assert lib.nsm_weights_create(None, None, 0, ctypes.byref(out)) == 1
    # host-frame entry point: missing buffers
    fr = nsm.nsm_frame(H=4, W=4)
    assert lib.nsm_infer_host(None, ctypes.byref(fr), None, 0, None, 0, None, 0, None, None) == 1
    assert nsm.nsm_infer_host_stage_bytes(4, 4, 8, 8) >= 4 * 4 * 32 + 8 * 8 * 4 + 4 * 4 * 4
    # pipelined host entry point: NULL context / weights, negative count
    assert lib.nsm_infer_host_sequence(None, 1, ctypes.byref(fr), None, 0, None, 0, None, 0, None, None) == 1
    assert b"ctx" in lib.nsm_last_error()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(nsm, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nsm, "_lib", None)
    with pytest.raises(ImportError):
        nsm.lib()


def test_depth_for_penumbra_host_logic(lib):
    """nsm_depth_for_penumbra (host only) against the oracle's 95th-percentile
    and depth rule on random histograms, and its argument checks."""
    from oracle import temporal as TM
    rng = np.random.default_rng(1)
    for _ in range(500):
        h = rng.integers(0, 50, size=int(rng.integers(1, 40)))
        if rng.random() < 0.1:
            h[:] = 0
        b = float(rng.choice([0.25, 0.5, 1.0, 3.0]))
        p95, lv = nsm.depth_for_penumbra(h, b)
        assert p95 == pytest.approx(TM.p95_from_histogram(h, b), abs=1e-6)
        assert lv == (TM.depth_for_width(p95) if p95 > 0 else 1)
    # the paper's receptive fields: 24 / 96 / 384 pixels -> 3 / 5 / 7 levels
    for w, l in ((24, 3), (96, 5), (384, 7)):
        h = np.zeros(400, np.uint32)
        h[w - 1] = 10
        assert nsm.depth_for_penumbra(h, 1.0) == (float(w), l)
    with pytest.raises(nsm.NSMError):
        nsm.depth_for_penumbra(np.zeros(4, np.uint32), 0.0)


def test_deep_network_sizes(lib):
    """Parameter counts of the 2- to 7-level networks equal the oracle's layer
    tables (the paper prints 39,248 / 653,648 weights for 3 / 5 levels)."""
    for L in range(2, 8):
        assert nsm.nsm_param_count_levels(L) == N.param_count(L, with_bias=True)
    assert N.param_count(5) == 653648
    assert nsm.nsm_param_count_levels(1) == 0 and nsm.nsm_param_count_levels(8) == 0
    assert nsm.nsm_infer_deep_workspace_bytes(64, 64, 5) >= (64 * 64 * 84 + N.param_count(5, with_bias=True)) * 4
    assert nsm.nsm_infer_deep_workspace_bytes(64, 64, 9) == 0


def test_features_workspace_size(lib):
    # two float2 tables (8 x 8 and 4 x 4 squares) per map texel
    assert nsm.nsm_features_workspace_bytes(2048, 2048) == 2048 * 2048 * 16
    assert nsm.nsm_features_workspace_bytes(0, 16) == 0


def test_host_validation_of_the_newer_entry_points(lib):
    # rejected before any CUDA call: NULL frame / context, depth out of range
    # (through the prototypes the binding declares)
    assert lib.nsm_features_ws(None, None, None, None, None, None, 0, None) == 1
    assert b"frame" in lib.nsm_last_error()
    typed = nsm._gen_sigs()
    assert typed.nsm_infer_deep(None, None, None, 5, None, 0, None, None) == 1
    assert b"ctx" in lib.nsm_last_error()
    assert nsm.nsm_infer_deep_workspace_bytes(0, 64, 5) == 0
    assert nsm.nsm_infer_deep_workspace_bytes(64, 64, 1) == 0
    assert typed.nsm_infer_deep_ex(None, None, None, 5, nsm.NSM_BF16, None, 0, None, None) == 1
    assert b"ctx" in lib.nsm_last_error()
    # the tensor-core form: 3 .. 7 levels, FP32 and BF16 only; its workspace
    # holds the FP32 form's plus the stage activations and weight images
    for L in (3, 5, 7):
        fp32 = nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_FP32)
        assert fp32 == nsm.nsm_infer_deep_workspace_bytes(64, 128, L)
        assert nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_BF16) > fp32
    assert nsm.nsm_infer_deep_workspace_bytes(64, 128, 2, nsm.NSM_BF16) == 0
    # the three-term FP8 form: 2 .. 7 levels, the FP32 form's tensors plus the
    # E4M3 images (in place of the FP32 form's weight copy)
    for L in (2, 3, 5, 7):
        assert nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_FP8) > 64 * 128 * 84 * 4
    assert nsm.nsm_infer_deep_workspace_bytes(64, 128, 5, 3) == 0


def test_packed_deep_weights_host_checks_and_workspace(lib):
    """The packed-weights entry points reject NULL handles before any CUDA
    call; their workspace is the per-call one without the packed images (for
    FP32: the tap-major copy of the vector, 256-byte aligned)."""
    typed = nsm._gen_sigs()
    h = ctypes.c_void_p()
    assert typed.nsm_deep_weights_create(None, None, 0, 5, nsm.NSM_FP32, ctypes.byref(h)) == 1
    assert b"ctx" in lib.nsm_last_error()
    assert typed.nsm_infer_deep_packed(None, None, None, None, 0, None, None) == 1
    assert b"weights" in lib.nsm_last_error()
    assert typed.nsm_deep_weights_load_device(None, None, 0, None) == 1
    typed.nsm_deep_weights_destroy(None)  # a no-op
    for L in (2, 3, 5, 7):
        n = N.param_count(L, with_bias=True)
        ex = nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_FP32)
        packed = nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, L, nsm.NSM_FP32)
        assert ex - packed == (n * 4 + 255) // 256 * 256
        assert nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, L, nsm.NSM_FP8) == packed
        assert nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_FP8) > packed
        if L >= 3:
            bf = nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, L, nsm.NSM_BF16)
            assert packed < bf < nsm.nsm_infer_deep_workspace_bytes(64, 128, L, nsm.NSM_BF16)
    assert nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, 2, nsm.NSM_BF16) == 0
    assert nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, 8, nsm.NSM_FP32) == 0
    assert nsm.nsm_infer_deep_packed_workspace_bytes(64, 128, 5, 3) == 0


def test_host_validation_of_the_static_entry_point(lib):
    """nsm_infer_fp32_static rejects bad frames before any CUDA call: NULL
    frame, sizes that are not multiples of 4, views above its fixed scratch
    limit, non-finite or out-of-range light values."""
    import math
    f = lib.nsm_infer_fp32_static
    assert f(None, None, None, None) == 1
    assert b"frame" in lib.nsm_last_error()

    def frame(H, W, **light):
        fr = nsm.nsm_frame(H=H, W=W, Hs=64, Ws=64)
        fr.light.tan_half_fov = 1.0
        fr.light.z_far = 10.0
        for k, v in light.items():
            setattr(fr.light, k, v)
        return fr

    assert f(ctypes.byref(frame(6, 8)), None, None, None) == 2          # H % 4 != 0
    assert b"multiples of 4" in lib.nsm_last_error()
    assert f(ctypes.byref(frame(516, 512)), None, None, None) == 2      # 264,192 > 262,144 pixels
    assert b"static scratch limit" in lib.nsm_last_error()
    assert f(ctypes.byref(frame(65536, 4)), None, None, None) == 2      # outside [0, 16384]
    bad = frame(64, 64)
    bad.light.pos[1] = math.nan
    assert f(ctypes.byref(bad), None, None, None) == 1
    assert b"finite" in lib.nsm_last_error()
    assert f(ctypes.byref(frame(64, 64, tan_half_fov=0.0)), None, None, None) == 1
    assert f(ctypes.byref(frame(64, 64, radius=-0.1)), None, None, None) == 1
    assert f(ctypes.byref(frame(64, 64, bias=-1e-3)), None, None, None) == 1
    assert f(ctypes.byref(frame(0, 64)), None, None, None) == 0         # empty view: nothing to do


def test_host_validation_of_the_sensitivity_entry_points(lib):
    typed = nsm._sens_sigs()
    assert typed.nsm_feature_moments(None, None, None) == 1
    assert b"frame" in lib.nsm_last_error()
    assert typed.nsm_sensitivity(None, None, None, 0, None, 1, None, None, 0, None, None) == 1
    assert b"ctx" in lib.nsm_last_error()
    assert nsm.nsm_sensitivity_workspace_bytes(0, 64) == 0
    H, W = 64, 96
    assert nsm.nsm_sensitivity_workspace_bytes(H, W) >= nsm.nsm_infer_workspace_bytes(H, W, nsm.NSM_FP32) + 2 * H * W * 4


def test_row_band_workspace_and_validation(lib):
    H, W = 1080, 1920
    n = nsm.nsm_infer_rows_workspace_bytes(H, W, 540, 1080, 32, nsm.NSM_BF16)
    rows = 1080 - 508
    assert n >= nsm.nsm_infer_workspace_bytes(rows, W, nsm.NSM_BF16) + rows * W * 4
    assert nsm.nsm_infer_rows_workspace_bytes(H, W, 540, 540, 32, nsm.NSM_BF16) == 0
    assert lib.nsm_infer_rows(None, None, None, 0, 0, 4, 0, None, 0, None, None) == 1


def test_host_validation_of_the_training_precision_entry_points(lib):
    # rejected before any CUDA call: NULL state / context
    typed = nsm._train_sigs()
    for f in ("nsm_train_state_set_detached_precision", "nsm_train_state_set_forward_precision",
              "nsm_train_state_set_backward_precision"):
        assert getattr(typed, f)(None, nsm.NSM_BF16) == 1
        assert b"state" in lib.nsm_last_error()
    assert typed.nsm_backward_ex(None, None, None, None, None, None, None, nsm.NSM_BF16, None, 0, None) == 1
    assert b"ctx" in lib.nsm_last_error()
    # the backward's workspace also holds the 3x3 weight images of the tensor-core form
    # (18,144 chunks of 16 bytes: 9 taps x K steps x 2 halves x 2 C_out rows per image)
    chunks = 0
    for ci, co in ((4, 16), (16, 32), (32, 64), (32, 32), (16, 16)):
        for a, b in ((ci, co), (co, ci)):
            chunks += 9 * ((a + 15) // 16) * 2 * 2 * max(b, 8)
    assert chunks == 18144
    small = nsm.nsm_backward_workspace_bytes(4, 4)
    assert small >= chunks * 16
