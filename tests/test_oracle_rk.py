"""Pins of the oracle's Runge-Kutta variant (the time stepping the paper
compares ADER with in Table IV: two stages at second order, three at third,
five at fourth) against facts independent of its code: the order conditions
of each scheme's Butcher tableau, the strong-stability-preserving property of
its Shu-Osher form, forward Euler through the ADER path with zero predictor
sweeps, free stream, conservation and the design order on the vortex."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P


def butcher(alpha, beta):
    """Shu-Osher (alpha, beta) -> Butcher (A, b, c): U(i) = U0 + dt sum_j
    Ahat[i][j] L(U(j)), Ahat[i] = sum_k alpha[i][k] Ahat[k] + beta[i]."""
    s = alpha.shape[1]
    Ahat = np.zeros((s + 1, s))
    for i in range(1, s + 1):
        Ahat[i] = sum(alpha[i][k] * Ahat[k] for k in range(i)) + beta[i]
    A, b = Ahat[:s], Ahat[s]
    return A, b, A.sum(axis=1)


ORDER_CONDITIONS = [
    (1, lambda A, b, c: b.sum(), 1.0),
    (2, lambda A, b, c: b @ c, 1 / 2),
    (3, lambda A, b, c: b @ c ** 2, 1 / 3),
    (3, lambda A, b, c: b @ A @ c, 1 / 6),
    (4, lambda A, b, c: b @ c ** 3, 1 / 4),
    (4, lambda A, b, c: (b * c) @ A @ c, 1 / 8),
    (4, lambda A, b, c: b @ A @ c ** 2, 1 / 12),
    (4, lambda A, b, c: b @ A @ A @ c, 1 / 24),
]


@pytest.mark.parametrize("stages,order", [(2, 2), (3, 3), (5, 4)])
def test_butcher_order_conditions(stages, order):
    A, b, c = butcher(*oracle.rk_coefficients(stages))
    assert np.allclose(np.tril(A, -1), A)                 # explicit
    for p, cond, value in ORDER_CONDITIONS:
        if p <= order:
            assert abs(cond(A, b, c) - value) < 2e-15, (p, cond(A, b, c), value)
    # and not of one order more (the schemes are exactly of their stated order)
    if order < 4:
        assert max(abs(cond(A, b, c) - v) for p, cond, v in ORDER_CONDITIONS if p == order + 1) > 1e-3


@pytest.mark.parametrize("stages,ssp", [(2, 1.0), (3, 1.0), (5, 1.508)])
def test_shu_osher_form_is_strong_stability_preserving(stages, ssp):
    """Every alpha and beta non-negative, each row of alpha sums to 1, and the
    SSP coefficient min alpha/beta is 1 for SSP(2,2) and SSP(3,3) and ~1.508
    for SSP(5,4)."""
    a, bt = oracle.rk_coefficients(stages)
    assert (a >= 0).all() and (bt >= 0).all()
    assert np.allclose(a[1:].sum(axis=1), 1.0, atol=2e-15)
    cfl = min(a[i, k] / bt[i, k] for i in range(1, stages + 1) for k in range(stages) if bt[i, k] > 0)
    assert abs(cfl - ssp) < 1e-3, cfl


@pytest.mark.parametrize("stages", [2, 3, 5])
def test_stages_see_the_boundary_at_their_abscissae(stages):
    """Double Mach reflection (top boundary moving with the shock): the step
    equals the stages composed here from L(U) evaluated with the boundary at
    t + c_k dt, c the Butcher abscissae of the scheme (0, 1 for SSP(2,2);
    0, 1, 1/2 for SSP(3,3))."""
    prob = P.dmr(nx=24, ny=8, order=3).replace(fallback=True, scheme="ssprk", rk_stages=stages)
    orc = oracle.Oracle(prob)
    U0 = prob.initial_state()
    dt = 0.3 / orc.signal_max(U0)
    # start so that the top boundary's shock passes the centre of the ghost
    # zone at x = 5.5 dx in the middle of the step
    xg, sq3 = 5.5 * prob.dx(0), math.sqrt(3.0)
    t = ((xg - 1.0 / 6.0 - 10.0 * dt / sq3) * sq3 - 1.0) / 20.0
    assert t > 0
    alpha, beta = oracle.rk_coefficients(stages)
    c = butcher(alpha, beta)[2]
    if stages == 2:
        assert np.array_equal(c, [0.0, 1.0])
    if stages == 3:
        assert np.array_equal(c, [0.0, 1.0, 0.5])
    Us, Ls = [U0.reshape((prob.nv,) + U0.shape[1:])], []
    for i in range(1, stages + 1):
        Ls.append(orc.rk_rhs(Us[i - 1], t + c[i - 1] * dt))
        Us.append(sum(alpha[i][k] * Us[k] + beta[i][k] * dt * Ls[k] for k in range(i)))
    U1, _, _ = orc.rk_step(U0, t, dt)
    assert np.abs(U1 - Us[-1]).max() <= 1e-13 * np.abs(U0).max()
    # and the boundary's motion matters at this resolution
    moved = max(np.abs(orc.rk_rhs(Us[k], t) - Ls[k]).max() for k in range(stages))
    assert moved > 1e-6 * np.abs(Ls[0]).max()


@pytest.mark.parametrize("dim,order", [(2, 2), (2, 3), (3, 3), (3, 4)])
def test_rhs_is_forward_euler_of_the_ader_step_without_sweeps(dim, order):
    """With zero predictor sweeps the ADER face states are the reconstructed
    polynomial at every time point, so the ADER step (time-and-face
    quadrature) equals U + dt L(U) (face quadrature only)."""
    if dim == 2:
        prob = P.vortex2d(n=10, order=order)
    else:
        prob = P.tgv3d(n=6, order=order)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    dt = 0.3 / orc.signal_max(U)
    orc.cfg.picard = 0
    Ua, _, rc = orc.step(U, 0.0, dt)
    assert rc == 0
    L = orc.rk_rhs(U, 0.0)
    Ue = U.reshape(L.shape) + dt * L
    assert np.abs(Ua.reshape(L.shape) - Ue).max() <= 1e-13 * np.abs(U).max()
    assert np.abs(L).max() > 1e-3


@pytest.mark.parametrize("order", [2, 3, 4])
def test_free_stream_and_conservation(order):
    prob = P.uniform(dim=3, n=6, order=order, vel=(0.3, -0.2, 0.1)).replace(scheme="ssprk")
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    # L vanishes bitwise; the stage combinations sum_k alpha_ik U leave a few
    # ulps (SSP(5,4)'s published 15-digit weights of the last stage sum to
    # 1 + 1e-15)
    assert not orc.rk_rhs(U, 0.0).any()
    U1, _, rc = orc.rk_step(U, 0.0, 0.4 / orc.signal_max(U))
    assert rc == 0 and np.abs(U1.reshape(U.shape) - U).max() <= 16 * np.finfo(float).eps * np.abs(U).max()
    prob = P.vortex2d(n=12, order=order).replace(scheme="ssprk")
    orc = oracle.Oracle(prob)
    U0 = U = prob.initial_state()
    t = 0.0
    for _ in range(5):
        dt = prob.cfl / orc.signal_max(U)
        U, _, rc = orc.rk_step(U, t, dt)
        U = U.reshape(U0.shape)
        t += dt
        assert rc == 0
    for v in range(prob.nv):
        a, b = math.fsum(U0[v].ravel()), math.fsum(U[v].ravel())
        scale = max(math.fsum(np.abs(U0[v]).ravel()), math.fsum(np.abs(U0[0]).ravel()))
        assert abs(a - b) <= 1e-13 * scale


@pytest.mark.parametrize("order,ns,min_rate", [(3, (64, 128), 2.7), (4, (32, 64), 3.7)])
def test_design_order_on_the_vortex(order, ns, min_rate):
    errs = []
    for n in ns:
        prob = P.vortex2d(n=n, order=order, t_end=1.0).replace(scheme="ssprk")
        orc = oracle.Oracle(prob)
        U, t = prob.initial_state(), 0.0
        dt = prob.cfl / orc.signal_max(U)
        while t < 1.0 - 1e-12:
            dt = min(dt, 1.0 - t)
            U, smax, rc = orc.rk_step(U, t, dt)
            U = U.reshape(prob.shape())
            assert rc == 0
            t += dt
            dt = prob.cfl / smax
        errs.append(np.abs(U[0] - P.vortex_exact(prob, 1.0)[0]).mean())
    assert math.log2(errs[0] / errs[1]) >= min_rate, errs
