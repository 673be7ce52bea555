"""Seeded trained weights for the 3-level network and the space-to-depth
network (Sec. 3.5), made with the FP64 oracle.

TEST INFRASTRUCTURE (see oracle/__init__.py): this script is run by hand and
writes scenegen/weights_trained_3level.npy (--topology levels3) or
scenegen/weights_trained_s2d.npy (--topology s2d), the trained weight sets the
parity tests and the benchmark feed to both the oracle and the GPU path as an
input.
The weights never come from the GPU path: every step below is the oracle's
own arithmetic (features, forward, adjoint, Eq. 2 loss, Adam).

Recipe (Sec. 3.3: supervised training on ray-traced targets with the temporal
perturbation term of Eq. 2; a single network for every emitter size, the
emitter size entering through the r_hat feature of Sec. 3.1):
  scenes   n_scenes seeded scenes (seeds 1000 + k), 64 objects each; even k
           point light (hard target: brute-force shadow rays), odd k spherical
           emitter of radius U[0.05, 0.2] (soft target: 16 x 16 stratified
           Monte-Carlo samples of the emitter disk).
  frames   480 x 272 view (about the 1080p aspect) with a 1024^2 shadow map,
           near the 1080p / 2048^2 texel-to-pixel ratio; each scene is rendered
           once as x0 and twice with seeded light / camera perturbations
           (scenegen.perturbed) as x1, x2.
  steps    `steps` Adam steps (lr 2e-3, then 1e-3 from half-way and 3e-4 for the
           last fifth) on batches
           of 8 random 64 x 64 crops; the loss is Eq. 2's L1 part with
           alpha = 0.9 and the perturbed instances detached.
  start    He-normal weights, seed 3.

Usage:  python -m oracle.train_weights [--topology levels3|s2d] [--steps N] [--scenes N]
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

import scenegen
from oracle import gather as G
from oracle import network as N

OUTS = {"levels3": os.path.join(os.path.dirname(scenegen.__file__), "weights_trained_3level.npy"),
        "s2d": os.path.join(os.path.dirname(scenegen.__file__), "weights_trained_s2d.npy")}
H, W, HS, WS, N_OBJ = 272, 480, 1024, 1024, 64
CROP, BATCH = 64, 8


def frame_features(f) -> np.ndarray:
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    return feat


def make_scene_data(k: int):
    soft = (k % 2) == 1
    scene = scenegen.random_scene(1000 + k, N_OBJ, soft=soft)
    f0 = scenegen.render_frame(scene, H, W, HS, WS)
    if soft:
        target = scenegen.soft_visibility(f0, spp_side=16, seed=k).astype(np.float64)
    else:
        target = scenegen.hard_visibility(f0).astype(np.float64)
    rng = scenegen.SplitMix64(0xC0FFEE + k)
    insts = [frame_features(f0)]
    for _ in range(2):
        insts.append(frame_features(scenegen.render_frame(scenegen.perturbed(scene, rng), H, W, HS, WS)))
    return insts, target


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--scenes", type=int, default=48)
    ap.add_argument("--topology", choices=sorted(OUTS), default="levels3")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or OUTS[args.topology]
    s2d = args.topology == "s2d"
    layers = N.layer_table_s2d(3) if s2d else N.layer_table(3)
    fwd = N.forward_s2d if s2d else N.forward
    step_fn = N.train_step_s2d if s2d else N.train_step

    t0 = time.time()
    data = [make_scene_data(k) for k in range(args.scenes)]
    val = [make_scene_data(k) for k in range(args.scenes, args.scenes + 2)]
    print(f"data: {args.scenes} scenes + 2 held out in {time.time() - t0:.0f} s", flush=True)

    theta = scenegen.he_init_weights(3, layers).astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    rng = np.random.Generator(np.random.PCG64(2301))

    def val_mse(th):
        errs = []
        for insts, target in val:
            y = fwd(insts[0], th)
            errs.append(float(np.mean((y - target) ** 2)))
        return errs

    print(f"start: held-out MSE vs ray-cast target {val_mse(theta)}", flush=True)
    t0 = time.time()
    for step in range(1, args.steps + 1):
        feats, targets = [], []
        for _ in range(BATCH):
            insts, target = data[rng.integers(len(data))]
            y0 = int(rng.integers(0, H - CROP + 1))
            x0 = int(rng.integers(0, W - CROP + 1))
            feats.append([f[:, y0:y0 + CROP, x0:x0 + CROP] for f in insts])
            targets.append(target[y0:y0 + CROP, x0:x0 + CROP])
        lr = 2e-3 if 2 * step <= args.steps else (1e-3 if 5 * step <= 4 * args.steps else 3e-4)
        theta, m, v, loss, _ = step_fn(feats, targets, theta, m, v, step, lr=lr)
        if step % 100 == 0 or step == 1:
            print(f"step {step}: loss {loss:.5f} ({time.time() - t0:.0f} s)", flush=True)
    print(f"end: held-out MSE vs ray-cast target {val_mse(theta)}", flush=True)
    np.save(out, theta.astype(np.float32))
    print(f"wrote {out}", flush=True)


if __name__ == "__main__":
    main()
