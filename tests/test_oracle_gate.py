"""Pins of the oracle's troubled-zone gate: MLP gradients against finite
differences, the FP32 decision forward against the FP64 forward, features and
flag dilation by hand, and labels on smooth vs discontinuous data."""
import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P


def bce(z, y):
    return np.mean(np.maximum(z, 0) - y * z + np.log1p(np.exp(-np.abs(z))))


def he_init(nin, nh, rng):
    W1 = rng.normal(0, np.sqrt(2.0 / nin), size=(nh, nin))
    W2 = rng.normal(0, np.sqrt(2.0 / nh), size=(nh, nh))
    w3 = rng.normal(0, np.sqrt(2.0 / nh), size=nh)
    b1 = rng.normal(0, 0.1, nh)
    b2 = rng.normal(0, 0.1, nh)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [0.05]]).astype(np.float32)


def test_mlp_parameter_count_and_layout():
    assert oracle.mlp_num_params(24, 32) == 32 * 24 + 32 + 32 * 32 + 32 + 32 + 1
    rng = np.random.default_rng(0)
    nin, nh = 5, 32
    p = he_init(nin, nh, rng)
    x = rng.normal(size=(7, nin)).astype(np.float32)
    # forward by hand from the packed layout
    W1 = p[:nh * nin].reshape(nh, nin).astype(np.float64)
    o = nh * nin
    b1 = p[o:o + nh]; o += nh
    W2 = p[o:o + nh * nh].reshape(nh, nh); o += nh * nh
    b2 = p[o:o + nh]; o += nh
    w3 = p[o:o + nh]; o += nh
    b3 = p[o]
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T.astype(np.float64) + b2, 0)
    z = h2 @ w3.astype(np.float64) + b3
    assert np.allclose(oracle.mlp_forward_f64(p, x), z, rtol=1e-12, atol=1e-12)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    nin, nh, B = 12, 32, 16
    p = he_init(nin, nh, rng)
    x = rng.normal(size=(B, nin)).astype(np.float32)
    y = (rng.uniform(size=B) < 0.5).astype(np.float32)
    loss, g = oracle.mlp_loss_grad_f64(p, x, y)
    assert abs(loss - bce(oracle.mlp_forward_f64(p, x), y)) < 1e-12
    # central differences in float64 on perturbed float32 parameters need a
    # parameter vector exactly representable after the shift: use h = 2^-10
    h = 2.0 ** -10
    idx = rng.choice(p.size, size=60, replace=False)
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (bce(oracle.mlp_forward_f64(pp, x), y) - bce(oracle.mlp_forward_f64(pm, x), y)) / (
            float(pp[i]) - float(pm[i]))
        assert abs(fd - g[i]) <= 1e-3 * max(1e-3, abs(g[i])) + 1e-6, (i, fd, g[i])


def test_f32_decision_forward_close_to_f64():
    rng = np.random.default_rng(2)
    nin = 24
    p = he_init(nin, 32, rng)
    x = rng.uniform(-1, 1, size=(200, nin)).astype(np.float32)
    z64 = oracle.mlp_forward_f64(p, x)
    z32 = oracle.mlp_forward_f32(p, x)
    assert np.abs(z32 - z64).max() < 1e-5 * max(1.0, np.abs(z64).max())


def test_features_by_hand():
    prob = P.sod(nx=16, ny=4, order=3)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    F = orc.features(U, 0.0)
    g, N = 3, 2
    assert F.shape[-1] == 2 * 2 * (2 * N + 1) == 20
    # zone at active x index 7 (last left zone): the x-stencil spans 5..9; the
    # only nonzero difference is f(8) - f(7), at k = 2
    f = F[0, g + 1, g + 7]
    # rho: differences (0, 0, -0.875, 0) -> shape (0, 0, -1, 0); magnitude
    # 100 * 0.875/1 squashed, in FP32 operations rounded once each
    f32 = np.float32
    assert list(f[0:4]) == [0.0, 0.0, -1.0, 0.0]
    x = f32(100.0) * (f32(0.875) / (f32(1.0) + f32(1e-12)))
    assert f[4] == x / (f32(1.0) + x)
    # E = p/(gamma-1): 2.5 | 0.25 -> shape (0, 0, -1, 0); magnitude 2.25/2.5
    assert list(f[5:9]) == [0.0, 0.0, -1.0, 0.0]
    x = f32(100.0) * (f32(2.25) / (f32(2.5) + f32(1e-12)))
    assert f[9] == x / (f32(1.0) + x)
    # y: constant data -> zeros
    assert np.all(f[10:] == 0)
    # zones without the full stencil get zero features
    assert np.all(F[0, 0, 0] == 0)


def test_flag_dilation_and_missing_stencils():
    prob = P.uniform(dim=2, n=8, order=3)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    nin = orc.num_features()
    p = np.zeros(oracle.mlp_num_params(nin, 32), dtype=np.float32)
    p[-1] = -1.0  # every logit -1 -> nothing troubled where a stencil exists
    fl = orc.gate_flags(U, 0.0, p)
    G = orc.G
    N = 2
    inner = np.zeros((G[1], G[0]), bool)
    inner[N:G[1] - N, N:G[0] - N] = True
    f2 = fl[0]
    # zones without stencil are troubled, and dilation reaches one zone inward
    assert np.all(f2[~inner] == 1)
    assert np.all(f2[N + 1:G[1] - N - 1, N + 1:G[0] - N - 1] == 0)
    assert np.all(f2[N, N + 1:G[0] - N - 1] == 1)
    p[-1] = 1.0
    assert np.all(orc.gate_flags(U, 0.0, p) == 1)


def test_labels_smooth_vs_shock():
    prob = P.sod(nx=32, ny=4, order=3)
    orc = oracle.Oracle(prob)
    lab = orc.labels(prob.initial_state(), 0.0, 0.1)
    g = 3
    row = lab[0, g + 1, g:g + 32]
    # zones whose central candidate crosses the jump at 15|16 are troubled;
    # at 14 and 17 only a candidate with linear weight 1/102 crosses it, so the
    # weights move by ~0.01 < tau
    assert np.all(row[15:17] == 1)
    assert np.all(row[:15] == 0) and np.all(row[17:] == 0)
    assert np.all(lab[0, 0, :] == 255)
