"""Oracle: feature sensitivity (Sec. 3.2, Eq. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The absolute sensitivity of input channel i measures how much the network
output moves when that channel alone is perturbed by a random texture of
normal noise whose standard deviation is a tenth of the channel's own
standard deviation, normalised by that noise level:

    S_i = E[ |phi(f with f_i + eps_i) - phi(f)| ] / (0.1 sigma_i),
    eps_i ~ N(0, (0.1 sigma_i)^2) per pixel,

the expectation taken over pixels, frames and repeated draws; sigma_i is the
standard deviation of channel i over all pixels of the frames.  The relative
sensitivity is s_i = S_i / sum_j S_j.

Readings (the printed equation is ambiguous): the expectation is of the
absolute change (the signed change averages to about zero for symmetric
noise, which would make every sensitivity vanish); the second parameter of
N(0, 0.1 sigma_i) is the standard deviation.  The noise textures are inputs
(standard normal draws), so any implementation can be fed the same ones.
"""
from __future__ import annotations

import numpy as np


def feature_std(feats) -> np.ndarray:
    """sigma_i of each channel over every pixel of the frames; feats is a list
    of (C, H, W) arrays (population standard deviation, FP64)."""
    x = np.concatenate([np.asarray(f, np.float64).reshape(f.shape[0], -1) for f in feats], axis=1)
    return x.std(axis=1)


def sensitivity(phi, feats, sigma, noise) -> np.ndarray:
    """Absolute sensitivities S (C,) of the network `phi` ((C, H, W) -> (H, W)).
    noise[f][k][i] is a standard normal (H, W) texture: draw k of channel i for
    frame f; the perturbation is 0.1 sigma_i times it."""
    sigma = np.asarray(sigma, np.float64)
    C = sigma.size
    total = np.zeros(C)
    count = 0
    for f, nf in zip(feats, noise):
        f = np.asarray(f, np.float64)
        base = phi(f)
        for draw in nf:
            for i in range(C):
                fp = f.copy()
                fp[i] = fp[i] + 0.1 * sigma[i] * np.asarray(draw[i], np.float64)
                total[i] += np.abs(phi(fp) - base).sum() / (0.1 * sigma[i])
        count += len(nf) * base.size
    return total / count


def relative(S) -> np.ndarray:
    S = np.asarray(S, np.float64)
    return S / S.sum()
