"""Pins for the oracle's feature sensitivity (Sec. 3.2, Eq. 1): closed forms
of pixel-wise linear networks, an ignored channel, the standard normal's mean
absolute value, and the relative form."""
import math

import numpy as np
import pytest

from oracle import sensitivity as SE


def _linear(a):
    a = np.asarray(a, np.float64)
    return lambda f: np.tensordot(a, f, axes=(0, 0))


def test_linear_network_closed_form_given_the_draws():
    """phi = sum_i a_i f_i: the change from channel i is a_i 0.1 sigma_i n, so
    S_i = |a_i| mean|n| exactly for the draws used; a_2 = 0 gives S_2 = 0 and a
    wrong channel, scale or normalisation would change the values."""
    rng = np.random.default_rng(0)
    feats = [rng.normal(size=(4, 8, 12)) * np.array([1.0, 3.0, 0.5, 2.0])[:, None, None] for _ in range(2)]
    sigma = SE.feature_std(feats)
    noise = [[rng.normal(size=(4, 8, 12)) for _ in range(3)] for _ in range(2)]
    a = [0.7, -1.3, 0.0, 2.5]
    S = SE.sensitivity(_linear(a), feats, sigma, noise)
    for i in range(4):
        m = np.mean([np.abs(noise[f][k][i]).mean() for f in range(2) for k in range(3)])
        assert S[i] == pytest.approx(abs(a[i]) * m, rel=1e-12)
    assert S[2] == 0.0


def test_standard_normal_mean_absolute_value():
    """With many draws S_i of a linear network tends to |a_i| E|N(0,1)| =
    |a_i| sqrt(2/pi), independent of sigma_i (the normalisation cancels it)."""
    rng = np.random.default_rng(1)
    feats = [rng.normal(size=(4, 64, 64)) * np.array([0.01, 1.0, 100.0, 5.0])[:, None, None]]
    sigma = SE.feature_std(feats)
    noise = [[rng.normal(size=(4, 64, 64)) for _ in range(4)]]
    a = [2.0, 1.0, 0.5, 1.5]
    S = SE.sensitivity(_linear(a), feats, sigma, noise)
    np.testing.assert_allclose(S, np.abs(a) * math.sqrt(2 / math.pi), rtol=0.02)
    np.testing.assert_allclose(SE.relative(S).sum(), 1.0, rtol=1e-12)


def test_feature_std_is_over_all_frames_and_pixels():
    rng = np.random.default_rng(2)
    f1, f2 = rng.normal(size=(4, 5, 6)), rng.normal(size=(4, 7, 3)) + 4.0
    sig = SE.feature_std([f1, f2])
    for i in range(4):
        allv = np.concatenate([f1[i].ravel(), f2[i].ravel()])
        assert sig[i] == pytest.approx(math.sqrt(np.mean((allv - allv.mean()) ** 2)), rel=1e-12)


def test_saturating_network_is_less_sensitive_where_saturated():
    """A pixel-wise sigmoid of one channel: the change is largest where the
    input sits at the sigmoid's steepest point; far into saturation it tends
    to zero (checks that |phi(f + eps) - phi(f)| is taken, not a linearised
    slope)."""
    rng = np.random.default_rng(3)
    phi = lambda f: 1.0 / (1.0 + np.exp(-f[0]))
    centre = [np.zeros((1, 32, 32))]
    far = [np.full((1, 32, 32), 30.0)]
    sigma = np.array([1.0])
    noise = [[rng.normal(size=(1, 32, 32)) for _ in range(2)]]
    s_centre = SE.sensitivity(phi, centre, sigma, noise)[0]
    s_far = SE.sensitivity(phi, far, sigma, noise)[0]
    assert s_centre == pytest.approx(0.25 * math.sqrt(2 / math.pi), rel=0.05)
    assert s_far < 1e-10
