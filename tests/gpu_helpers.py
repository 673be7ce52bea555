"""Shared helpers for the GPU tests: move a seeded scenegen frame to the
device and run the library's calls through the Python binding."""
import numpy as np
import torch

import paper_2301_05262_gb300 as nsm


def light_desc(f):
    return nsm.LightDesc(pos=tuple(float(v) for v in f.light_pos), radius=f.light_radius, r_hat=f.r_hat,
                         view_proj=f.view_proj, z_far=f.z_far, bias=f.bias, tan_half_fov=f.tan_half_fov)


class DeviceFrame:
    """Device copies of a frame's buffers plus the nsm_frame struct."""

    def __init__(self, f, device="cuda"):
        self.f = f
        self.pos4 = torch.from_numpy(f.pos4).to(device)
        self.nrm4 = torch.from_numpy(f.nrm4).to(device)
        self.sm = torch.from_numpy(f.sm).to(device)
        self.frame = nsm.make_frame(self.pos4, self.nrm4, self.sm, light_desc(f), f.cam_pos)


def run_features(df, blocker=False):
    f = df.f
    H, W = f.H, f.W
    feat = torch.empty((4, H, W), dtype=torch.float32, device="cuda")
    tex = torch.empty((H, W), dtype=torch.int32, device="cuda")
    hard = torch.empty(((H * W + 31) // 32,), dtype=torch.int32, device="cuda")
    blk = torch.empty((3, H, W), dtype=torch.float32, device="cuda") if blocker else None
    nsm.nsm_features(df.frame, feat, tex, hard, blk)
    torch.cuda.synchronize()
    return feat, tex, hard, blk


def unpack_hard_bits(words: np.ndarray, n: int) -> np.ndarray:
    w = words.astype(np.uint32)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1
    return bits.reshape(-1)[:n].astype(bool)


def run_infer(ctx, weights, df, precision, vis=None):
    f = df.f
    nbytes = nsm.nsm_infer_workspace_bytes(f.H, f.W, precision)
    ws = torch.empty((max(nbytes, 1),), dtype=torch.uint8, device="cuda")
    if vis is None:
        vis = torch.empty((f.H, f.W), dtype=torch.float32, device="cuda")
    nsm.nsm_infer(ctx, df.frame, weights, precision, ws, vis)
    torch.cuda.synchronize()
    return vis


def train_batch_frames(B, T, H, W, S, seed, n_obj=8, spp_side=8):
    """Frames [t][b] of a temporal-window batch (instance 0 = the seeded soft
    scene, instances 1..T-1 = its perturbations) and the MC targets [b]."""
    import scenegen
    rng = scenegen.SplitMix64(seed ^ 0xBA7C4)
    frames = [[None] * B for _ in range(T)]
    targets = []
    for b in range(B):
        base = scenegen.random_scene(seed * 100 + b, n_obj, soft=True)
        frames[0][b] = scenegen.render_frame(base, H, W, S, S)
        for t in range(1, T):
            frames[t][b] = scenegen.render_frame(scenegen.perturbed(base, rng), H, W, S, S)
        targets.append(scenegen.soft_visibility(frames[0][b], spp_side=spp_side))
    return frames, np.stack(targets).astype(np.float32)


def device_batch(frames, targets):
    T, B = len(frames), len(frames[0])
    pos = torch.from_numpy(np.stack([[frames[t][b].pos4 for b in range(B)] for t in range(T)])).cuda()
    nrm = torch.from_numpy(np.stack([[frames[t][b].nrm4 for b in range(B)] for t in range(T)])).cuda()
    sm = torch.from_numpy(np.stack([[frames[t][b].sm for b in range(B)] for t in range(T)])).cuda()
    tgt = torch.from_numpy(targets).cuda()
    lights = [light_desc(frames[t][b]) for t in range(T) for b in range(B)]
    cams = [frames[t][b].cam_pos for t in range(T) for b in range(B)]
    bt = nsm.make_batch(pos, nrm, sm, lights, cams, tgt, B, T)
    bt._tensors = (pos, nrm, sm, tgt)
    return bt


def oracle_band(frame, theta64, y0, y1, margin=32):
    """FP64 oracle visibility of rows [y0, y1) (multiples of 4) from the rows
    [y0 - margin, y1 + margin) of the frame: the network's receptive field is
    about 20 level-0 pixels, so these rows equal the full-frame forward (a CPU
    test pins the band forward to the full one)."""
    from oracle import gather as G
    from oracle import network as N
    a, b = max(0, y0 - margin), min(frame.H, y1 + margin)
    sub = slice(a, b)
    feat, _, _ = G.features(frame.pos4[sub], frame.nrm4[sub], frame.sm, frame.view_proj, frame.light_pos,
                            frame.cam_pos, frame.r_hat, frame.z_far, frame.bias)
    return N.forward(feat, theta64)[y0 - a:y1 - a]
