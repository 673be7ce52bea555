"""Python binding of libnsm.so (include/nsm.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
turns torch tensors (device memory, streams) and numpy arrays (host memory)
into the C structs and pointers of the ABI and raises NSMError on failure.
There is no fallback: if libnsm.so has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnsm.so")

NSM_FP32, NSM_BF16, NSM_FP8 = 0, 1, 2
NSM_TOPO_LEVELS3, NSM_TOPO_S2D = 0, 1
PRECISIONS = {"fp32": NSM_FP32, "bf16": NSM_BF16, "fp8": NSM_FP8}
STATUS = {0: "NSM_OK", 1: "NSM_ERR_INVALID_ARG", 2: "NSM_ERR_SHAPE", 3: "NSM_ERR_ALIGNMENT",
          4: "NSM_ERR_DEVICE", 5: "NSM_ERR_CUDA", 6: "NSM_ERR_TIMEOUT", 7: "NSM_ERR_UNSUPPORTED",
          8: "NSM_ERR_WORKSPACE"}

# canonical layer order of the parameter vector: (name, c_in, c_out, k)
LAYERS = [("enc0_3x3", 4, 16, 3), ("enc0_1x1", 16, 16, 1), ("enc1_3x3", 16, 32, 3),
          ("enc1_1x1", 32, 32, 1), ("bott_3x3", 32, 64, 3), ("bott_1x1", 64, 32, 1),
          ("dec1_3x3", 32, 32, 3), ("dec1_1x1", 32, 16, 1), ("dec0_3x3", 16, 16, 3),
          ("dec0_1x1", 16, 16, 1), ("head", 16, 1, 1)]


class NSMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class nsm_light(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("radius", ctypes.c_float), ("r_hat", ctypes.c_float),
                ("view_proj", ctypes.c_float * 16), ("z_far", ctypes.c_float), ("bias", ctypes.c_float),
                ("tan_half_fov", ctypes.c_float)]


class nsm_camera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3)]


class nsm_frame(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("pos4", ctypes.c_void_p),
                ("nrm4", ctypes.c_void_p), ("Hs", ctypes.c_int), ("Ws", ctypes.c_int),
                ("sm", ctypes.c_void_p), ("light", nsm_light), ("camera", nsm_camera)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        FP = ctypes.POINTER(nsm_frame)
        sig = {
            "nsm_abi_version": ([], I),
            "nsm_last_error": ([], ctypes.c_char_p),
            "nsm_ctx_create": ([ctypes.POINTER(P)], I),
            "nsm_ctx_destroy": ([P], None),
            "nsm_ctx_check": ([P], I),
            "nsm_ctx_set_stage_events": ([P, P, I], I),
            "nsm_infer_kernel_count": ([I], I),
            "nsm_infer_kernel_name": ([I, I], ctypes.c_char_p),
            "nsm_param_count": ([], Z),
            "nsm_weights_create": ([P, P, Z, ctypes.POINTER(P)], I),
            "nsm_param_count_topology": ([I], Z),
            "nsm_weights_create_topology": ([P, I, P, Z, ctypes.POINTER(P)], I),
            "nsm_weights_load_device": ([P, P, Z, P], I),
            "nsm_weights_destroy": ([P], None),
            "nsm_features": ([FP, P, P, P, P, P], I),
            "nsm_features_workspace_bytes": ([ctypes.c_int, ctypes.c_int], Z),
            "nsm_features_ws": ([FP, P, P, P, P, P, Z, P], I),
            "nsm_infer_workspace_bytes": ([I, I, I], Z),
            "nsm_infer": ([P, FP, P, I, P, Z, P, P], I),
            "nsm_infer_host_stage_bytes": ([I, I, I, I], Z),
            "nsm_infer_host": ([P, FP, P, I, P, Z, P, Z, P, P], I),
            "nsm_infer_host_sequence": ([P, I, FP, P, I, P, Z, P, Z, P, P], I),
            "nsm_infer_fp32_static": ([FP, P, P, P], I),
            "nsm_infer_rows_workspace_bytes": ([I, I, I, I, I, I], Z),
            "nsm_infer_rows": ([P, FP, P, I, I, I, I, P, Z, P, P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def declared_symbols():
    """Names declared by include/nsm.h (for the ABI completeness test)."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "nsm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(nsm_[a-z0-9_]+)\s*\(", hdr)))


def _check(status: int, where: str):
    if status != 0:
        raise NSMError(status, where, lib().nsm_last_error().decode())


def _ptr(x):
    """Address of a torch tensor / numpy array / None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


@dataclass
class LightDesc:
    pos: tuple
    radius: float
    r_hat: float
    view_proj: np.ndarray  # (4, 4) row-major
    z_far: float
    bias: float
    tan_half_fov: float


def make_frame(pos4, nrm4, sm, light: LightDesc, cam_pos) -> nsm_frame:
    """Build an nsm_frame from (H, W, 4) pos4 / nrm4 and (Hs, Ws) sm buffers
    (torch device tensors or numpy host arrays; the caller keeps them alive)."""
    H, W = int(pos4.shape[0]), int(pos4.shape[1])
    Hs, Ws = int(sm.shape[0]), int(sm.shape[1])
    L = nsm_light()
    L.pos[:] = [float(v) for v in light.pos]
    L.radius = float(light.radius)
    L.r_hat = float(light.r_hat)
    L.view_proj[:] = [float(v) for v in np.asarray(light.view_proj, np.float32).reshape(-1)]
    L.z_far = float(light.z_far)
    L.bias = float(light.bias)
    L.tan_half_fov = float(light.tan_half_fov)
    C = nsm_camera()
    C.pos[:] = [float(v) for v in cam_pos]
    return nsm_frame(H=H, W=W, pos4=_ptr(pos4), nrm4=_ptr(nrm4), Hs=Hs, Ws=Ws, sm=_ptr(sm), light=L, camera=C)


class Context:
    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().nsm_ctx_create(ctypes.byref(h)), "nsm_ctx_create")
        self.h = h

    def check(self):
        _check(lib().nsm_ctx_check(self.h), "nsm_ctx_check")

    def set_stage_events(self, events):
        """events: list of torch.cuda.Event (timing enabled), or [] to turn the hook off."""
        handles = [ctypes.c_void_p(e.cuda_event) for e in events]
        arr = (ctypes.c_void_p * max(1, len(handles)))(*handles)
        _check(lib().nsm_ctx_set_stage_events(self.h, arr if handles else None, len(handles)),
               "nsm_ctx_set_stage_events")

    def close(self):
        if self.h:
            lib().nsm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Weights:
    """Network weights on the device; topology NSM_TOPO_LEVELS3 (default) or NSM_TOPO_S2D."""

    def __init__(self, ctx: Context, params: np.ndarray, topology: int = 0):
        p = np.ascontiguousarray(params, np.float32)
        h = ctypes.c_void_p()
        _check(lib().nsm_weights_create_topology(ctx.h, topology, _ptr(p), p.size, ctypes.byref(h)),
               "nsm_weights_create_topology")
        self.h = h
        self.topology = topology

    def load_device(self, dev_params, stream=None):
        _check(lib().nsm_weights_load_device(self.h, _ptr(dev_params), int(dev_params.numel()), _stream(stream)),
               "nsm_weights_load_device")

    def close(self):
        if self.h:
            lib().nsm_weights_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nsm_infer_kernel_names(precision: int):
    n = lib().nsm_infer_kernel_count(precision)
    return [lib().nsm_infer_kernel_name(precision, i).decode() for i in range(n)]


def nsm_param_count() -> int:
    return int(lib().nsm_param_count())


def nsm_features(frame: nsm_frame, feat_out, texel_out=None, hard_out=None, blocker_out=None, stream=None):
    _check(lib().nsm_features(ctypes.byref(frame), _ptr(feat_out), _ptr(texel_out), _ptr(hard_out),
                              _ptr(blocker_out), _stream(stream)), "nsm_features")


def nsm_features_workspace_bytes(Hs: int, Ws: int) -> int:
    return int(lib().nsm_features_workspace_bytes(Hs, Ws))


def nsm_features_ws(frame: nsm_frame, feat_out, texel_out=None, hard_out=None, blocker_out=None, workspace=None,
                    stream=None):
    """nsm_features with the blocker search's table scratch taken from `workspace`."""
    nbytes = 0 if workspace is None else int(workspace.numel() * workspace.element_size())
    _check(lib().nsm_features_ws(ctypes.byref(frame), _ptr(feat_out), _ptr(texel_out), _ptr(hard_out),
                                 _ptr(blocker_out), _ptr(workspace), nbytes, _stream(stream)), "nsm_features_ws")


def nsm_infer_workspace_bytes(H: int, W: int, precision: int) -> int:
    return int(lib().nsm_infer_workspace_bytes(H, W, precision))


def nsm_infer(ctx: Context, frame: nsm_frame, weights: Weights, precision: int, workspace, vis_out, stream=None,
              workspace_bytes=None):
    nbytes = workspace_bytes if workspace_bytes is not None else (
        0 if workspace is None else int(workspace.numel() * workspace.element_size()))
    _check(lib().nsm_infer(ctx.h, ctypes.byref(frame), weights.h, precision, _ptr(workspace), nbytes,
                           _ptr(vis_out), _stream(stream)), "nsm_infer")


def nsm_infer_host_stage_bytes(H, W, Hs, Ws) -> int:
    return int(lib().nsm_infer_host_stage_bytes(H, W, Hs, Ws))


def nsm_infer_host(ctx: Context, host_frame: nsm_frame, weights: Weights, precision: int, dev_stage, workspace,
                   vis_host: np.ndarray, stream=None):
    _check(lib().nsm_infer_host(ctx.h, ctypes.byref(host_frame), weights.h, precision, _ptr(dev_stage),
                                int(dev_stage.numel() * dev_stage.element_size()), _ptr(workspace),
                                int(workspace.numel() * workspace.element_size()), _ptr(vis_host),
                                _stream(stream)), "nsm_infer_host")


def nsm_infer_host_sequence(ctx: Context, host_frames, weights: Weights, precision: int, dev_stage, workspace,
                            vis_hosts, stream=None):
    """Pipelined nsm_infer_host over a list of host frames; vis_hosts: one
    C-contiguous float32 host array per frame (pinned for overlap)."""
    n = len(host_frames)
    arr = (nsm_frame * max(n, 1))(*host_frames)
    outs = (ctypes.c_void_p * max(n, 1))(*[v.ctypes.data if isinstance(v, np.ndarray) else v.data_ptr()
                                           for v in vis_hosts])
    _check(lib().nsm_infer_host_sequence(ctx.h, n, arr, weights.h, precision, _ptr(dev_stage),
                                         int(dev_stage.numel() * dev_stage.element_size()), _ptr(workspace),
                                         int(workspace.numel() * workspace.element_size()),
                                         ctypes.cast(outs, ctypes.c_void_p), _stream(stream)),
           "nsm_infer_host_sequence")


def nsm_infer_rows_workspace_bytes(H: int, W: int, y0: int, y1: int, halo: int, precision: int) -> int:
    return int(lib().nsm_infer_rows_workspace_bytes(H, W, y0, y1, halo, precision))


def nsm_infer_rows(ctx: Context, frame: nsm_frame, weights: Weights, precision: int, y0: int, y1: int, halo: int,
                   workspace, vis_rows, stream=None):
    """Rows [y0, y1) of the frame's visibility from a slab with `halo` rows of context."""
    _check(lib().nsm_infer_rows(ctx.h, ctypes.byref(frame), weights.h, precision, y0, y1, halo, _ptr(workspace),
                                int(workspace.numel() * workspace.element_size()), _ptr(vis_rows), _stream(stream)),
           "nsm_infer_rows")


def frame_rows(H: int, rank: int, world: int):
    """The band of rows [y0, y1) of an H-row frame that `rank` of `world` devices
    computes when one frame is split across them: contiguous bands, bounds on
    the 4-row pooling grid, sizes within 4 rows of each other (empty bands when
    H / 4 < world)."""
    q = H // 4
    return 4 * (q * rank // world), 4 * (q * (rank + 1) // world)


def nsm_infer_fp32_static(frame: nsm_frame, dev_params, vis_out, stream=None):
    """FP32 inference without allocation or workspace (views up to 262,144 pixels)."""
    _check(lib().nsm_infer_fp32_static(ctypes.byref(frame), _ptr(dev_params), _ptr(vis_out), _stream(stream)),
           "nsm_infer_fp32_static")


# ---------------------------------------------------------------- backward / training
class nsm_batch(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("T", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("Hs", ctypes.c_int), ("Ws", ctypes.c_int), ("pos4", ctypes.c_void_p), ("nrm4", ctypes.c_void_p),
                ("sm", ctypes.c_void_p), ("lights", ctypes.POINTER(nsm_light)),
                ("cameras", ctypes.POINTER(nsm_camera)), ("target", ctypes.c_void_p)]


class nsm_train_cfg(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("alpha", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


def _train_sigs():
    L = lib()
    if getattr(L, "_train_sigs", False):
        return L
    P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sig = {
        "nsm_backward_workspace_bytes": ([I, I], Z),
        "nsm_backward": ([P, ctypes.POINTER(nsm_frame), P, P, P, P, P, P, Z, P], I),
        "nsm_backward_ex": ([P, ctypes.POINTER(nsm_frame), P, P, P, P, P, I, P, Z, P], I),
        "nsm_train_state_create": ([P, P, Z, I, I, I, I, ctypes.POINTER(P)], I),
        "nsm_train_state_destroy": ([P], None),
        "nsm_train_step": ([P, P, ctypes.POINTER(nsm_batch), ctypes.POINTER(nsm_train_cfg), P, P], I),
        "nsm_train_state_read": ([P, I, P, Z, P], I),
        "nsm_train_state_write": ([P, I, P, Z, P], I),
        "nsm_train_grad": ([P, P, ctypes.POINTER(nsm_batch), ctypes.POINTER(nsm_train_cfg), P, P], I),
        "nsm_train_apply": ([P, P, ctypes.POINTER(nsm_train_cfg), P], I),
        "nsm_train_state_set_detached_precision": ([P, I], I),
        "nsm_train_state_set_forward_precision": ([P, I], I),
        "nsm_train_state_set_backward_precision": ([P, I], I),
        "nsm_train_state_read_vis": ([P, P, Z, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    L._train_sigs = True
    return L


def nsm_backward_workspace_bytes(H: int, W: int) -> int:
    return int(_train_sigs().nsm_backward_workspace_bytes(H, W))


def nsm_backward(ctx: Context, frame: nsm_frame, dev_params, grad_vis, grad_params, workspace, grad_feat=None,
                 vis_out=None, stream=None, precision=None):
    """precision None: nsm_backward; NSM_FP32 / NSM_BF16: nsm_backward_ex with that form of the 3x3 layers."""
    L = _train_sigs()
    if precision is None:
        _check(L.nsm_backward(ctx.h, ctypes.byref(frame), _ptr(dev_params), _ptr(grad_vis), _ptr(grad_params),
                              _ptr(grad_feat), _ptr(vis_out), _ptr(workspace),
                              int(workspace.numel() * workspace.element_size()), _stream(stream)), "nsm_backward")
        return
    _check(L.nsm_backward_ex(ctx.h, ctypes.byref(frame), _ptr(dev_params), _ptr(grad_vis), _ptr(grad_params),
                             _ptr(grad_feat), _ptr(vis_out), int(precision), _ptr(workspace),
                             int(workspace.numel() * workspace.element_size()), _stream(stream)), "nsm_backward_ex")


class TrainState:
    """FP32 master weights + Adam state for nsm_train_step."""

    def __init__(self, ctx: Context, params: np.ndarray, max_B: int, max_T: int, H: int, W: int):
        L = _train_sigs()
        p = np.ascontiguousarray(params, np.float32)
        h = ctypes.c_void_p()
        _check(L.nsm_train_state_create(ctx.h, _ptr(p), p.size, max_B, max_T, H, W, ctypes.byref(h)),
               "nsm_train_state_create")
        self.h, self.ctx, self.n = h, ctx, p.size

    def step(self, batch: nsm_batch, lr=1e-3, alpha=0.9, beta1=0.9, beta2=0.999, eps=1e-8, loss_out=None,
             stream=None):
        cfg = nsm_train_cfg(lr=lr, alpha=alpha, beta1=beta1, beta2=beta2, eps=eps)
        _check(_train_sigs().nsm_train_step(self.ctx.h, self.h, ctypes.byref(batch), ctypes.byref(cfg),
                                            _ptr(loss_out), _stream(stream)), "nsm_train_step")

    def grad(self, batch: nsm_batch, alpha=0.9, loss_out=None, stream=None):
        """Loss and gradient of the batch into the state (no weight update)."""
        cfg = nsm_train_cfg(lr=1e-3, alpha=alpha, beta1=0.9, beta2=0.999, eps=1e-8)
        _check(_train_sigs().nsm_train_grad(self.ctx.h, self.h, ctypes.byref(batch), ctypes.byref(cfg),
                                            _ptr(loss_out), _stream(stream)), "nsm_train_grad")

    def apply(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """One Adam step with the state's gradient."""
        cfg = nsm_train_cfg(lr=lr, alpha=0.9, beta1=beta1, beta2=beta2, eps=eps)
        _check(_train_sigs().nsm_train_apply(self.ctx.h, self.h, ctypes.byref(cfg), _stream(stream)),
               "nsm_train_apply")

    def read(self, what: int, out, stream=None):
        _check(_train_sigs().nsm_train_state_read(self.h, what, _ptr(out), self.n, _stream(stream)),
               "nsm_train_state_read")

    def write(self, what: int, src, stream=None):
        _check(_train_sigs().nsm_train_state_write(self.h, what, _ptr(src), self.n, _stream(stream)),
               "nsm_train_state_write")

    def set_detached_precision(self, precision: int):
        """Form of the detached instances' forward (NSM_FP32 or NSM_BF16)."""
        _check(_train_sigs().nsm_train_state_set_detached_precision(self.h, precision),
               "nsm_train_state_set_detached_precision")

    def set_forward_precision(self, precision: int):
        """Form of the target instances' forward (NSM_FP32 or NSM_BF16)."""
        _check(_train_sigs().nsm_train_state_set_forward_precision(self.h, precision),
               "nsm_train_state_set_forward_precision")

    def set_backward_precision(self, precision: int):
        """Form of the backward's 3x3 recomputations and data gradients (NSM_FP32 or NSM_BF16)."""
        _check(_train_sigs().nsm_train_state_set_backward_precision(self.h, precision),
               "nsm_train_state_set_backward_precision")

    def read_vis(self, out, stream=None):
        """Visibility [T][B][H][W] of the last step's instances into a device tensor."""
        _check(_train_sigs().nsm_train_state_read_vis(self.h, _ptr(out), int(out.numel()), _stream(stream)),
               "nsm_train_state_read_vis")

    def close(self):
        if self.h:
            _train_sigs().nsm_train_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_batch(pos4, nrm4, sm, lights, cams, target, B, T):
    """nsm_batch from device tensors pos4/nrm4 [T,B,H,W,4], sm [T,B,Hs,Ws],
    target [B,H,W] and T*B LightDesc / camera positions (instance order t*B+b)."""
    H, W = int(pos4.shape[2]), int(pos4.shape[3])
    Hs, Ws = int(sm.shape[2]), int(sm.shape[3])
    LA = (nsm_light * (T * B))()
    CA = (nsm_camera * (T * B))()
    for i, (ld, cp) in enumerate(zip(lights, cams)):
        fr = make_frame(np.zeros((1, 1, 4), np.float32), np.zeros((1, 1, 4), np.float32),
                        np.zeros((1, 1), np.float32), ld, cp)
        LA[i] = fr.light
        CA[i] = fr.camera
    bt = nsm_batch(B=B, T=T, H=H, W=W, Hs=Hs, Ws=Ws, pos4=_ptr(pos4), nrm4=_ptr(nrm4), sm=_ptr(sm),
                   lights=ctypes.cast(LA, ctypes.POINTER(nsm_light)),
                   cameras=ctypes.cast(CA, ctypes.POINTER(nsm_camera)), target=_ptr(target))
    bt._keep = (LA, CA)
    return bt


def autograd_function():
    """torch.autograd.Function whose forward is nsm_infer (FP32) and whose
    backward is the library's hand-written adjoint (nsm_backward).
    Usage: vis = F.apply(params, ctx, frame) with params a device FP32 tensor
    of nsm_param_count() floats; the frame's buffers must stay alive."""
    import torch

    class NSMFunction(torch.autograd.Function):
        @staticmethod
        def forward(fctx, params, ctx, frame):
            H, W = frame.H, frame.W
            vis = torch.empty((H, W), dtype=torch.float32, device=params.device)
            ws = torch.empty((nsm_backward_workspace_bytes(H, W),), dtype=torch.uint8, device=params.device)
            gp = torch.zeros_like(params)
            g0 = torch.zeros((H, W), dtype=torch.float32, device=params.device)
            # the adjoint call also returns the forward visibility; with a zero
            # cotangent it leaves the gradient untouched
            nsm_backward(ctx, frame, params.contiguous(), g0, gp, ws, vis_out=vis)
            fctx.save_for_backward(params)
            fctx.nsm = (ctx, frame)
            return vis

        @staticmethod
        def backward(fctx, grad_vis):
            (params,) = fctx.saved_tensors
            ctx, frame = fctx.nsm
            ws = torch.empty((nsm_backward_workspace_bytes(frame.H, frame.W),), dtype=torch.uint8,
                             device=params.device)
            gp = torch.zeros_like(params)
            nsm_backward(ctx, frame, params.contiguous(), grad_vis.contiguous().float(), gp, ws)
            return gp, None, None

    return NSMFunction


# ---------------------------------------------------------------- batched serving, graphs, autotuner
class nsm_view(ctypes.Structure):
    _fields_ = [("frame", nsm_frame), ("vis_out", ctypes.c_void_p)]


def _batch_sigs():
    L = lib()
    if getattr(L, "_batch_sigs", False):
        return L
    P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    VP = ctypes.POINTER(nsm_view)
    sig = {
        "nsm_infer_batched_workspace_bytes": ([I, VP], Z),
        "nsm_infer_batched": ([P, I, VP, P, P, Z, P], I),
        "nsm_ctx_set_graph": ([P, I], I),
        "nsm_ctx_set_view_timing": ([P, P], I),
        "nsm_ctx_graph_replays": ([P], I),
        "nsm_autotune": ([P, I, VP, P, P, Z, I, P], I),
        "nsm_autotune_report": ([P, P, P, P], I),
        "nsm_autotune_report_warps": ([P, P, P], I),
        "nsm_autotune_report_order": ([P, P], I),
        "nsm_plan_variants": ([I], I),
        "nsm_plan_set": ([P, I, I, I], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    L._batch_sigs = True
    return L


def make_views(frames, vis_outs):
    arr = (nsm_view * len(frames))()
    for i, (fr, vo) in enumerate(zip(frames, vis_outs)):
        arr[i].frame = fr
        arr[i].vis_out = _ptr(vo)
    return arr


def nsm_infer_batched_workspace_bytes(views) -> int:
    return int(_batch_sigs().nsm_infer_batched_workspace_bytes(len(views), views))


def nsm_infer_batched(ctx: Context, views, weights: Weights, workspace, stream=None):
    _check(_batch_sigs().nsm_infer_batched(ctx.h, len(views), views, weights.h, _ptr(workspace),
                                           int(workspace.numel() * workspace.element_size()), _stream(stream)),
           "nsm_infer_batched")


def nsm_ctx_set_graph(ctx: Context, enable: bool):
    _check(_batch_sigs().nsm_ctx_set_graph(ctx.h, 1 if enable else 0), "nsm_ctx_set_graph")


def nsm_ctx_set_view_timing(ctx: Context, records=None):
    """Per-view completion records of later batched calls: a device int64[65]
    tensor ([0] start, [1 + v] view v done, %globaltimer ns), or None (off)."""
    _check(_batch_sigs().nsm_ctx_set_view_timing(ctx.h, _ptr(records)), "nsm_ctx_set_view_timing")


def nsm_ctx_graph_replays(ctx: Context) -> int:
    return int(_batch_sigs().nsm_ctx_graph_replays(ctx.h))


def nsm_autotune(ctx: Context, views, weights: Weights, workspace, reps=3, stream=None):
    _check(_batch_sigs().nsm_autotune(ctx.h, len(views), views, weights.h, _ptr(workspace),
                                      int(workspace.numel() * workspace.element_size()), reps, _stream(stream)),
           "nsm_autotune")


def nsm_autotune_report(ctx: Context):
    rows = (ctypes.c_int * 5)()
    ctas = (ctypes.c_int * 5)()
    ms = (ctypes.c_float * 5)()
    _check(_batch_sigs().nsm_autotune_report(ctx.h, rows, ctas, ms), "nsm_autotune_report")
    return list(rows), list(ctas), list(ms)


def nsm_plan_variants(stage: int) -> int:
    return int(_batch_sigs().nsm_plan_variants(stage))


def nsm_plan_set(ctx: Context, stage: int, variant: int, ctas_per_sm: int = 0):
    _check(_batch_sigs().nsm_plan_set(ctx.h, stage, variant, ctas_per_sm), "nsm_plan_set")


def nsm_autotune_report_order(ctx: Context):
    """MMA schedule (0 or 1) of every stage of the context's plan."""
    o = (ctypes.c_int * 5)()
    _check(_batch_sigs().nsm_autotune_report_order(ctx.h, o), "nsm_autotune_report_order")
    return list(o)


def nsm_autotune_report_warps(ctx: Context):
    """(epilogue warps, producer warps) of every stage of the context's plan."""
    ew = (ctypes.c_int * 5)()
    pw = (ctypes.c_int * 5)()
    _check(_batch_sigs().nsm_autotune_report_warps(ctx.h, ew, pw), "nsm_autotune_report_warps")
    return list(ew), list(pw)


def nsm_param_count_topology(topology: int) -> int:
    return int(lib().nsm_param_count_topology(topology))


# ------------------------------------------------------------------ scene generation (GPU ray casting)
_GEN = None


def _gen_sigs():
    global _GEN
    if _GEN is None:
        L = lib()
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        for name, args in {
            "nsm_gen_gbuffer": [I, I, P, I, P, P, P, P, P],
            "nsm_gen_shadowmap": [I, I, P, F, I, P, P, P],
            "nsm_gen_visibility": [I, I, P, P, P, P, F, I, ctypes.c_uint64, F, I, P, P, P],
            "nsm_temporal_instability": [I, I, P, P, P, P, P, P, P, F, P, P, P],
            "nsm_infer_deep": [P, ctypes.POINTER(nsm_frame), P, I, P, ctypes.c_size_t, P, P],
            "nsm_infer_deep_ex": [P, ctypes.POINTER(nsm_frame), P, I, I, P, ctypes.c_size_t, P, P],
            "nsm_deep_weights_create": [P, P, ctypes.c_size_t, I, I, ctypes.POINTER(P)],
            "nsm_deep_weights_load_device": [P, P, ctypes.c_size_t, P],
            "nsm_infer_deep_packed": [P, ctypes.POINTER(nsm_frame), P, P, ctypes.c_size_t, P, P],
            "nsm_penumbra_histogram": [I, I, P, P, F, F, I, P, P],
            "nsm_depth_for_penumbra": [P, I, F, P, P],
        }.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = I
        L.nsm_deep_weights_destroy.argtypes = [P]
        L.nsm_deep_weights_destroy.restype = None
        L.nsm_infer_deep_packed_workspace_bytes.argtypes = [I, I, I, I]
        L.nsm_infer_deep_packed_workspace_bytes.restype = ctypes.c_size_t
        _GEN = L
    return _GEN


def _host_f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1))


def gen_gbuffer(H, W, cam, objects, pos4, nrm4, mask, stream=None):
    """cam: 14 floats (eye, forward, right, up, tan(fovy/2), aspect); objects: (n, 5)."""
    c, o = _host_f32(cam), _host_f32(objects)
    _check(_gen_sigs().nsm_gen_gbuffer(H, W, _ptr(c), o.size // 5, _ptr(o) if o.size else None, _ptr(pos4),
                                       _ptr(nrm4), _ptr(mask), _stream(stream)), "nsm_gen_gbuffer")


def gen_shadowmap(Hs, Ws, lcam, z_far, objects, depth, stream=None):
    c, o = _host_f32(lcam), _host_f32(objects)
    _check(_gen_sigs().nsm_gen_shadowmap(Hs, Ws, _ptr(c), float(z_far), o.size // 5, _ptr(o) if o.size else None,
                                         _ptr(depth), _stream(stream)), "nsm_gen_shadowmap")


def gen_visibility(H, W, pos4, nrm4, mask, light_pos, radius, spp_side, seed, eps, objects, vis, stream=None):
    L, o = _host_f32(light_pos), _host_f32(objects)
    _check(_gen_sigs().nsm_gen_visibility(H, W, _ptr(pos4), _ptr(nrm4), _ptr(mask), _ptr(L), float(radius),
                                          int(spp_side), ctypes.c_uint64(seed), float(eps), o.size // 5,
                                          _ptr(o) if o.size else None, _ptr(vis), _stream(stream)),
           "nsm_gen_visibility")


def temporal_instability(vis, vis_prev, pos4, nrm4, pos4_prev, nrm4_prev, cam_prev, sum_inout, count_inout,
                         alpha=3.0, stream=None):
    """Adds one frame pair's Eq. 3 terms to sum_inout (float64 device scalar)
    and its accepted-pixel count to count_inout (int64 device scalar)."""
    H, W = int(vis.shape[0]), int(vis.shape[1])
    c = _host_f32(cam_prev)
    _check(_gen_sigs().nsm_temporal_instability(H, W, _ptr(vis), _ptr(vis_prev), _ptr(pos4), _ptr(nrm4),
                                                _ptr(pos4_prev), _ptr(nrm4_prev), _ptr(c), float(alpha),
                                                _ptr(sum_inout), _ptr(count_inout), _stream(stream)),
           "nsm_temporal_instability")


def penumbra_histogram(blocker, pos4, tan_half_fovy, bin_px, hist_inout, stream=None):
    """Adds the frame's screen-space penumbra widths to hist_inout (int32
    device array; its length is the bin count)."""
    H, W = int(pos4.shape[0]), int(pos4.shape[1])
    _check(_gen_sigs().nsm_penumbra_histogram(H, W, _ptr(blocker), _ptr(pos4), float(tan_half_fovy), float(bin_px),
                                              int(hist_inout.numel()), _ptr(hist_inout), _stream(stream)),
           "nsm_penumbra_histogram")


def nsm_param_count_levels(levels: int) -> int:
    L = lib()
    L.nsm_param_count_levels.restype = ctypes.c_size_t
    L.nsm_param_count_levels.argtypes = [ctypes.c_int]
    return int(L.nsm_param_count_levels(levels))


def nsm_infer_deep_workspace_bytes(H: int, W: int, levels: int, precision=None) -> int:
    """Workspace of nsm_infer_deep (precision None) or nsm_infer_deep_ex."""
    L = lib()
    if precision is None:
        L.nsm_infer_deep_workspace_bytes.restype = ctypes.c_size_t
        L.nsm_infer_deep_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        return int(L.nsm_infer_deep_workspace_bytes(H, W, levels))
    L.nsm_infer_deep_ex_workspace_bytes.restype = ctypes.c_size_t
    L.nsm_infer_deep_ex_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    return int(L.nsm_infer_deep_ex_workspace_bytes(H, W, levels, int(precision)))


def nsm_infer_deep(ctx: Context, frame: nsm_frame, dev_params, levels: int, workspace, vis_out, stream=None,
                   precision=None):
    """Forward of the L-level network (L = 2 .. 7) on a device frame: FP32
    (precision None: nsm_infer_deep) or the form nsm_infer_deep_ex runs."""
    nbytes = int(workspace.numel() * workspace.element_size())
    if precision is None:
        _check(_gen_sigs().nsm_infer_deep(ctx.h, ctypes.byref(frame), _ptr(dev_params), int(levels), _ptr(workspace),
                                          nbytes, _ptr(vis_out), _stream(stream)), "nsm_infer_deep")
    else:
        _check(_gen_sigs().nsm_infer_deep_ex(ctx.h, ctypes.byref(frame), _ptr(dev_params), int(levels),
                                             int(precision), _ptr(workspace), nbytes, _ptr(vis_out),
                                             _stream(stream)), "nsm_infer_deep_ex")


class DeepWeights:
    """Packed weights of the L-level network in one form (FP32, BF16 or FP8),
    made once from a host vector of nsm_param_count_levels(levels) floats."""

    def __init__(self, ctx: Context, params: np.ndarray, levels: int, precision: int = 0):
        p = np.ascontiguousarray(params, np.float32).reshape(-1)
        h = ctypes.c_void_p()
        _check(_gen_sigs().nsm_deep_weights_create(ctx.h, _ptr(p), p.size, int(levels), int(precision),
                                                   ctypes.byref(h)), "nsm_deep_weights_create")
        self.h = h
        self.levels = int(levels)
        self.precision = int(precision)

    def load_device(self, dev_params, stream=None):
        _check(_gen_sigs().nsm_deep_weights_load_device(self.h, _ptr(dev_params), int(dev_params.numel()),
                                                        _stream(stream)), "nsm_deep_weights_load_device")

    def close(self):
        if self.h:
            _gen_sigs().nsm_deep_weights_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nsm_infer_deep_packed_workspace_bytes(H: int, W: int, levels: int, precision: int) -> int:
    return int(_gen_sigs().nsm_infer_deep_packed_workspace_bytes(H, W, levels, int(precision)))


def nsm_infer_deep_packed(ctx: Context, frame: nsm_frame, weights: DeepWeights, workspace, vis_out, stream=None):
    """Forward of the L-level network from packed weights (nsm_infer_deep_ex's
    result, without the per-call packing)."""
    nbytes = int(workspace.numel() * workspace.element_size())
    _check(_gen_sigs().nsm_infer_deep_packed(ctx.h, ctypes.byref(frame), weights.h, _ptr(workspace), nbytes,
                                             _ptr(vis_out), _stream(stream)), "nsm_infer_deep_packed")


def depth_for_penumbra(hist, bin_px):
    """(95th-percentile width in pixels, levels) from a host histogram."""
    h = np.ascontiguousarray(np.asarray(hist, np.uint32).reshape(-1))
    p95 = ctypes.c_float()
    lv = ctypes.c_int()
    _check(_gen_sigs().nsm_depth_for_penumbra(_ptr(h), h.size, float(bin_px), ctypes.byref(p95), ctypes.byref(lv)),
           "nsm_depth_for_penumbra")
    return float(p95.value), int(lv.value)


# ------------------------------------------------------------------ feature sensitivity (Sec. 3.2, Eq. 1)
_SENS = None


def _sens_sigs():
    global _SENS
    if _SENS is None:
        L = lib()
        P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        FP = ctypes.POINTER(nsm_frame)
        for name, (args, res) in {
            "nsm_feature_moments": ([FP, P, P], I),
            "nsm_sensitivity_workspace_bytes": ([I, I], Z),
            "nsm_sensitivity": ([P, FP, P, I, P, I, P, P, Z, P, P], I),
        }.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _SENS = L
    return _SENS


def feature_moments(frame: nsm_frame, moments_inout, stream=None):
    """Adds the frame's per-channel sums of f and f^2 to a device float64[8]."""
    _check(_sens_sigs().nsm_feature_moments(ctypes.byref(frame), _ptr(moments_inout), _stream(stream)),
           "nsm_feature_moments")


def nsm_sensitivity_workspace_bytes(H: int, W: int) -> int:
    return int(_sens_sigs().nsm_sensitivity_workspace_bytes(H, W))


def sensitivity(ctx: Context, frame: nsm_frame, weights: Weights, precision: int, noise, sigma, workspace, s_inout,
                stream=None):
    """Adds sum_p |phi_pert - phi| / (0.1 sigma_i) over pixels and draws to a
    device float64[4]; noise is a device float32 [draws][4][H][W] of standard
    normal draws, sigma 4 host floats."""
    sig = _host_f32(sigma)
    draws = int(noise.shape[0])
    _check(_sens_sigs().nsm_sensitivity(ctx.h, ctypes.byref(frame), weights.h, precision, _ptr(noise), draws,
                                        _ptr(sig), _ptr(workspace), int(workspace.numel() * workspace.element_size()),
                                        _ptr(s_inout), _stream(stream)), "nsm_sensitivity")
