"""Pins of the oracle's multi-dimensional reconstruction (pure and mixed modes,
the z family included) against what the mathematics fixes.

1. Polynomial recovery.  Every WENO candidate is a full polynomial of degree N
   that matches the zone averages of its stencil, so a polynomial of total
   degree <= N is reproduced exactly by each candidate, whatever the weights.
   The mixed modes follow: the (a,0,0) mode field of a polynomial p is, zone
   by zone, the average over the transverse zone of the polynomial q_a(y, z)
   that multiplies P_a(xi) in p's local expansion, and q_a has total degree
   <= N - a; the same argument carries the (a,b,0) fields through the z pass.
   So every spatial mode (a, b, c) of the reconstruction must equal the
   coefficient of P_a(xi) P_b(eta) P_c(zeta) in p's expansion about the zone
   centre, to rounding.  The test writes the zone averages and the expected
   coefficients with exact rational arithmetic, from the basis of the method
   (P0 = 1, P1 = xi, P2 = xi^2 - 1/12, P3 = xi^3 - 3 xi / 20 on [-1/2, 1/2]),
   and runs the reconstruction with computed (nonlinear) weights, with the
   fixed linear weights, and with linear weights that pick one candidate
   alone (each candidate, in every pass, must reproduce the polynomial).

2. Design order in 3D.  A density wave advected along the diagonal of the
   periodic unit cube (every mixed derivative non-zero) must converge at the
   order of the scheme (Sec. IV.1 reports 3D rates of 2.94 at order 3 and
   4.22 at order 4, Table XII).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import _dp, _up
from paper_2211_13295_gb300 import problems as P

# xi^s in the basis: xi^0 = P0, xi = P1, xi^2 = P2 + P0/12, xi^3 = P3 + 3/20 P1
MONO_TO_BASIS = [
    [Fr(1), Fr(0), Fr(0), Fr(0)],
    [Fr(0), Fr(1), Fr(0), Fr(0)],
    [Fr(1, 12), Fr(0), Fr(1), Fr(0)],
    [Fr(0), Fr(3, 20), Fr(0), Fr(1)],
]


def _random_poly(rng, dim, N, half):
    """Coefficients {(p, q, r): Fraction} of a random polynomial of total degree
    <= N in zone-index coordinates, scaled so |p| = O(1) on [-half, half]^dim."""
    coef = {}
    for r in range(N + 1 if dim == 3 else 1):
        for q in range(N + 1 - r):
            for p in range(N + 1 - q - r):
                num = int(rng.integers(1, 10)) * int(rng.choice([-1, 1]))
                coef[(p, q, r)] = Fr(num, 10 * half ** (p + q + r))
    return coef


def _axis_averages(centres, N):
    """avg[s][i] = average of X^s over [c_i - 1/2, c_i + 1/2] (exact)."""
    out = []
    for s in range(N + 1):
        out.append([((c + Fr(1, 2)) ** (s + 1) - (c - Fr(1, 2)) ** (s + 1)) / (s + 1) for c in centres])
    return out


def _axis_expansion(centres, N):
    """E[p][a][i] = coefficient of P_a(xi) in (c_i + xi)^p (exact)."""
    E = [[[Fr(0)] * len(centres) for _ in range(N + 1)] for _ in range(N + 1)]
    for p in range(N + 1):
        for i, c in enumerate(centres):
            for s in range(p + 1):
                term = math.comb(p, s) * c ** (p - s)
                for a in range(N + 1):
                    E[p][a][i] += term * MONO_TO_BASIS[s][a]
    return E


def _recon_case(dim, order, weights, seed):
    N = order - 1
    n = (5, 4, 3) if dim == 3 else (5, 4, 1)
    prob = P.uniform(dim=dim, n=n[0], order=order).replace(n=n)
    if weights[0] == "one":
        lin = [0.0] * order
        lin[weights[1]] = 1.0
        prob = prob.replace(lin=tuple(lin))
    orc = oracle.Oracle(prob)
    G = orc.G
    rng = np.random.default_rng(seed)
    half = max(G[:dim]) // 2 + 1
    coef = _random_poly(rng, dim, N, half)
    # zone centres in zone-index units, centred on the grid
    cen = [[Fr(2 * i - (G[d] - 1), 2) for i in range(G[d])] if d < dim else [Fr(0)] for d in range(3)]
    av = [_axis_averages(cen[d], N) if d < dim else [[Fr(1)]] * (N + 1) for d in range(3)]
    Ug = np.zeros((orc.nv, G[2], G[1], G[0]))
    for (p, q, r), cf in coef.items():
        blk = np.array([[[float(cf * av[0][p][i] * av[1][q][j] * av[2][r][k]) for i in range(G[0])]
                         for j in range(G[1])] for k in range(G[2])])
        Ug[0] += blk
    # the other variables: scaled copies, so every variable runs the same path
    for v in range(1, orc.nv):
        Ug[v] = (v + 1) * Ug[0]
    ns = oracle.num_modes(dim, N)
    B = orc.box_shape()
    W = np.zeros((orc.nv, ns, B[2], B[1], B[0]))
    flags = None
    if weights[0] in ("linear", "one"):
        flags = np.zeros(int(np.prod(G)), dtype=np.uint8)
    rc = oracle.lib().ora_reconstruct(oracle.C.byref(orc.cfg), _dp(np.ascontiguousarray(Ug)), _up(flags), _dp(W))
    assert rc == 0
    # expected coefficients at the box zones (active zones + one layer)
    g = orc.g
    box_idx = [[ib - 1 + g for ib in range(B[d])] if d < dim else [0] for d in range(3)]
    Ex = [_axis_expansion([cen[d][i] for i in box_idx[d]], N) if d < dim else None for d in range(3)]
    modes = oracle.mode_list(dim, N)
    want = np.zeros((ns, B[2], B[1], B[0]))
    for m, (a, b, c) in enumerate(modes):
        for kb in range(B[2]):
            for jb in range(B[1]):
                for ib in range(B[0]):
                    acc = Fr(0)
                    for (p, q, r), cf in coef.items():
                        ez = Ex[2][r][c][kb] if dim == 3 else (Fr(1) if c == 0 and r == 0 else Fr(0))
                        if ez == 0:
                            continue
                        acc += cf * Ex[0][p][a][ib] * Ex[1][q][b][jb] * ez
                    want[m, kb, jb, ib] = float(acc)
    return W, want, modes, orc.nv


@pytest.mark.parametrize("dim,order", [(2, 3), (2, 4), (3, 3), (3, 4)])
@pytest.mark.parametrize("weights", [("nonlinear",), ("linear",), ("one", 0), ("one", 1), ("one", -1)],
                         ids=["nonlinear", "linear", "cand0", "cand1", "candlast"])
def test_reconstruction_recovers_every_mode_of_a_polynomial(dim, order, weights):
    W, want, modes, nv = _recon_case(dim, order, weights, seed=100 * dim + order)
    scale = np.abs(want).max()
    for v in range(nv):
        err = np.abs(W[v] - (v + 1) * want)
        worst = np.unravel_index(np.argmax(err), err.shape)
        assert err.max() <= 1e-13 * (v + 1) * scale, (v, tuple(modes[worst[0]]), err.max(), scale)
    # the test is not vacuous: every mode, pure and mixed, is present and non-zero
    for m in range(len(modes)):
        assert np.abs(want[m]).max() > 1e-6 * scale, modes[m]


def _run_to(orc, U, T, cfl):
    t, dt = 0.0, orc.cfl_dt(U, cfl)
    while t < T - 1e-12:
        dt = min(dt, T - t)
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        dt = cfl / smax
    return U


@pytest.mark.parametrize("order,ns,t_end,min_rate", [(3, (8, 16, 32), 0.04, 2.7), (4, (8, 12, 16), 0.05, 3.7)])
def test_design_order_on_a_3d_diagonal_density_wave(order, ns, t_end, min_rate):
    errs = []
    for n in ns:
        prob = P.wave3d(n=n, order=order, t_end=t_end)
        U = _run_to(oracle.Oracle(prob), prob.initial_state(), t_end, prob.cfl)
        errs.append(np.abs(U[0] - P.wave3d_exact(prob, t_end)[0]).mean())
    rates = [math.log(a / b) / math.log(m / n) for a, b, n, m in zip(errs, errs[1:], ns, ns[1:])]
    assert rates[-1] >= min_rate, (errs, rates)
