"""Pins of the oracle's HLL, HLLEM and Rusanov fluxes (the Riemann solvers
named beside HLLC in Sec. I.1) against facts of the Euler equations:
consistency and symmetries, exactness on waves each solver must resolve (an
isolated shock for HLL and HLLEM through Roe's property; isolated contacts
and shear waves for HLLEM), the integral-average form of HLL, and the
linearisation of Rusanov's flux about a uniform state."""
import math

import numpy as np
import pytest

import oracle

G = 1.4
KINDS = ["hllc", "hll", "hllem", "rusanov"]


def euler_flux(U, d, dim):
    rho = U[0]
    v = U[1:1 + dim] / rho
    p = (G - 1) * (U[-1] - 0.5 * rho * (v ** 2).sum())
    F = np.zeros(dim + 2)
    F[0] = rho * v[d]
    F[1:1 + dim] = rho * v[d] * v
    F[1 + d] += p
    F[-1] = (U[-1] + p) * v[d]
    return F


def cons(rho, vel, p):
    vel = np.asarray(vel, dtype=float)
    return np.concatenate([[rho], rho * vel, [p / (G - 1) + 0.5 * rho * (vel ** 2).sum()]])


def prim(U, dim):
    rho = U[0]
    v = U[1:1 + dim] / rho
    p = (G - 1) * (U[-1] - 0.5 * rho * (v ** 2).sum())
    return rho, v, p


def rand_state(rng, dim):
    return cons(rng.uniform(0.2, 3), rng.uniform(-2, 2, size=dim), rng.uniform(0.1, 5))


def test_hllc_dispatch_is_the_hllc_routine():
    rng = np.random.default_rng(1)
    for _ in range(10):
        UL, UR = rand_state(rng, 3), rand_state(rng, 3)
        assert np.array_equal(oracle.riemann("hllc", 3, G, 1, UL, UR), oracle.hllc(3, G, 1, UL, UR))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dim", [2, 3])
def test_consistency_and_symmetries(kind, dim):
    rng = np.random.default_rng(7)
    for _ in range(30):
        UL, UR = rand_state(rng, dim), rand_state(rng, dim)
        for d in range(dim):
            F = oracle.riemann(kind, dim, G, d, UL, UL)
            assert np.allclose(F, euler_flux(UL, d, dim), rtol=1e-13, atol=1e-13)
            R = np.ones(dim + 2)
            R[1 + d] = -1
            F1 = oracle.riemann(kind, dim, G, d, UL, UR)
            F2 = oracle.riemann(kind, dim, G, d, R * UR, R * UL)
            assert np.allclose(F2, -R * F1, rtol=1e-12, atol=1e-12)
            if d > 0:
                perm = list(range(dim + 2))
                perm[1], perm[1 + d] = perm[1 + d], perm[1]
                Fx = oracle.riemann(kind, dim, G, 0, UL[perm], UR[perm])
                assert np.allclose(F1[perm], Fx, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["hll", "hllem"])
def test_isolated_shocks_are_exact(kind):
    """Roe's property makes the Roe speed of the shock family equal to the
    shock speed S; with S as the outer wave speed, the HLL flux collapses to
    the Godunov flux (F_L for a right-facing shock with S > 0, by
    Rankine-Hugoniot F_R - F_L = S (U_R - U_L)).  The jump across a shock lies
    along that family's Roe eigenvector, so HLLEM's restored waves have zero
    strength and it is exact as well.  w = -S0 makes the shock stationary."""
    for M in (1.5, 3.0, 6.0):
        rr, pr = 0.8, 1.1
        cr = math.sqrt(G * pr / rr)
        S0 = M * cr
        rl = rr * (G + 1) * M * M / ((G - 1) * M * M + 2)
        pl = pr * (2 * G * M * M - (G - 1)) / (G + 1)
        ul0 = S0 * (1 - rr / rl)
        for w in (0.0, -0.3 * S0, -0.6 * S0, -0.95 * S0, -S0, 0.5 * S0):
            for dim in (2, 3):
                vt = [0.25, -0.1][:dim - 1]
                UL = cons(rl, [ul0 + w] + vt, pl)
                UR = cons(rr, [w] + vt, pr)
                F = oracle.riemann(kind, dim, G, 0, UL, UR)
                assert np.allclose(F, euler_flux(UL, 0, dim), rtol=1e-12, atol=1e-12), (M, w, dim)
                R = np.ones(dim + 2)
                R[1] = -1
                Fm = oracle.riemann(kind, dim, G, 0, R * UR, R * UL)
                assert np.allclose(Fm, euler_flux(R * UL, 0, dim), rtol=1e-12, atol=1e-12), (M, w, dim)


def test_hllem_resolves_contacts_and_shear_waves_exactly():
    """Across a contact or shear wave only rho and the tangential velocity
    jump; the exact flux is the upwind physical flux (only the pressure flux
    at u = 0).  HLLEM restores exactly these waves; HLL and Rusanov smear
    them (their mass flux at a stationary contact is not zero)."""
    for dim in (2, 3):
        vt_l, vt_r = [0.3, -0.2][:dim - 1], [-1.0, 0.5][:dim - 1]
        UL, UR = cons(1.0, [0.0] + vt_l, 0.7), cons(0.2, [0.0] + vt_r, 0.7)
        F = oracle.riemann("hllem", dim, G, 0, UL, UR)
        expect = np.zeros(dim + 2)
        expect[1] = 0.7
        assert np.allclose(F, expect, atol=1e-14)
        for kind in ("hll", "rusanov"):
            assert abs(oracle.riemann(kind, dim, G, 0, UL, UR)[0]) > 1e-3
        for u in (0.4, -0.4, 1.7, -2.9):   # sub- and supersonic contact speeds
            UL, UR = cons(1.0, [u] + vt_l, 0.7), cons(0.2, [u] + vt_r, 0.7)
            up = UL if u > 0 else UR
            F = oracle.riemann("hllem", dim, G, 0, UL, UR)
            assert np.allclose(F, euler_flux(up, 0, dim), rtol=1e-13, atol=1e-13), (dim, u)
        # a pure shear wave (same density)
        UL, UR = cons(0.6, [0.5] + vt_l, 1.3), cons(0.6, [0.5] + vt_r, 1.3)
        F = oracle.riemann("hllem", dim, G, 0, UL, UR)
        assert np.allclose(F, euler_flux(UL, 0, dim), rtol=1e-13, atol=1e-13)


def roe_speeds(UL, UR, dim, d):
    """Davis-Einfeldt wave speeds from Roe averages (the reading shared with
    HLLC), restated here."""
    rl, vl, pl = prim(UL, dim)
    rr, vr, pr = prim(UR, dim)
    cl, cr = math.sqrt(G * pl / rl), math.sqrt(G * pr / rr)
    wl, wr = math.sqrt(rl), math.sqrt(rr)
    v = (wl * vl + wr * vr) / (wl + wr)
    H = (wl * (UL[-1] + pl) / rl + wr * (UR[-1] + pr) / rr) / (wl + wr)
    c = math.sqrt((G - 1) * (H - 0.5 * (v ** 2).sum()))
    return min(vl[d] - cl, v[d] - c), max(vr[d] + cr, v[d] + c)


def test_hll_is_the_flux_of_the_integral_average_state():
    """HLL's single state U* is the average of the exact solution over the
    fan [S_L t, S_R t] (conservation on the control volume gives
    U* = (S_R U_R - S_L U_L - (F_R - F_L))/(S_R - S_L)); its flux follows from
    the Rankine-Hugoniot conditions across either outer wave:
    F = F_L + S_L (U* - U_L) = F_R + S_R (U* - U_R)."""
    rng = np.random.default_rng(11)
    n_fan = 0
    for _ in range(60):
        dim = 3
        UL, UR = rand_state(rng, dim), rand_state(rng, dim)
        SL, SR = roe_speeds(UL, UR, dim, 0)
        FL, FR = euler_flux(UL, 0, dim), euler_flux(UR, 0, dim)
        F = oracle.riemann("hll", dim, G, 0, UL, UR)
        if SL < 0 < SR:
            n_fan += 1
            Us = (SR * UR - SL * UL - (FR - FL)) / (SR - SL)
            assert np.allclose(F, FL + SL * (Us - UL), rtol=1e-12, atol=1e-12)
            assert np.allclose(F, FR + SR * (Us - UR), rtol=1e-12, atol=1e-12)
        elif SL >= 0:
            assert np.array_equal(F, FL) or np.allclose(F, FL, rtol=1e-15)
        else:
            assert np.allclose(F, FR, rtol=1e-15)
    assert n_fan > 20


def test_rusanov_linearisation_and_dissipation_speed():
    """About a uniform state U, dF/dU_R = (A(U) - S I)/2 with A the flux
    Jacobian (finite differences of the physical flux here) and S = |u| + c;
    for unequal states the dissipation coefficient read off the flux,
    -2 (F - (F_L + F_R)/2) / (U_R - U_L), is the larger of the two states'
    |u| + c (the reading of the local Lax-Friedrichs speed)."""
    rng = np.random.default_rng(3)
    dim = 3
    for _ in range(5):
        U = rand_state(rng, dim)
        rho, v, p = prim(U, dim)
        S = abs(v[0]) + math.sqrt(G * p / rho)
        h = 1e-7   # the max() in S has a kink at U_R = U: an O(h) one-sided error
        for k in range(dim + 2):
            e = np.zeros(dim + 2)
            e[k] = h * max(1.0, abs(U[k]))
            dF = (oracle.riemann("rusanov", dim, G, 0, U, U + e) - oracle.riemann("rusanov", dim, G, 0, U, U - e)) / (2 * e[k])
            dA = (euler_flux(U + e, 0, dim) - euler_flux(U - e, 0, dim)) / (2 * e[k])
            expect = 0.5 * dA
            expect[k] -= 0.5 * S
            assert np.allclose(dF, expect, rtol=2e-6, atol=2e-6)
    for _ in range(20):
        UL, UR = rand_state(rng, dim), rand_state(rng, dim)
        F = oracle.riemann("rusanov", dim, G, 0, UL, UR)
        avg = 0.5 * (euler_flux(UL, 0, dim) + euler_flux(UR, 0, dim))
        k = int(np.argmax(np.abs(UR - UL)))
        S_read = -2 * (F[k] - avg[k]) / (UR[k] - UL[k])
        speeds = []
        for U in (UL, UR):
            rho, v, p = prim(U, dim)
            speeds.append(abs(v[0]) + math.sqrt(G * p / rho))
        assert abs(S_read - max(speeds)) < 1e-12 * max(speeds)


# --------------------------------------------------------------------------
# the whole step with each solver
# --------------------------------------------------------------------------
from paper_2211_13295_gb300 import problems as P  # noqa: E402


@pytest.mark.parametrize("kind", ["hll", "hllem", "rusanov"])
def test_free_stream_and_conservation(kind):
    prob = P.uniform(dim=3, n=6, order=4, vel=(0.3, -0.2, 0.1)).replace(riemann=kind)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    U1, _, rc = orc.step(U, 0.0, 0.4 / orc.signal_max(U))
    assert rc == 0 and np.array_equal(U1, U)
    prob = P.vortex2d(n=16, order=3).replace(riemann=kind)
    orc = oracle.Oracle(prob)
    U0 = U = prob.initial_state()
    t = 0.0
    for _ in range(10):
        dt = prob.cfl / orc.signal_max(U)
        U, _, rc = orc.step(U, t, dt)
        t += dt
        assert rc == 0
    for v in range(prob.nv):
        a, b = math.fsum(U0[v].ravel()), math.fsum(U[v].ravel())
        scale = max(math.fsum(np.abs(U0[v]).ravel()), math.fsum(np.abs(U0[0]).ravel()))
        assert abs(a - b) <= 1e-13 * scale


@pytest.mark.parametrize("kind", ["hll", "rusanov"])
def test_design_order_is_kept_on_the_vortex(kind):
    """The Riemann solver changes the error constant, not the order: the
    order-3 vortex still converges at rate >= 2.6 from 64^2 to 128^2 (the
    HLLC run measures 2.94 there)."""
    errs = []
    for n in (64, 128):
        prob = P.vortex2d(n=n, order=3, t_end=1.0).replace(riemann=kind)
        orc = oracle.Oracle(prob)
        U, t = prob.initial_state(), 0.0
        dt = prob.cfl / orc.signal_max(U)
        while t < 1.0 - 1e-12:
            dt = min(dt, 1.0 - t)
            U, smax, rc = orc.step(U, t, dt)
            assert rc == 0
            t += dt
            dt = prob.cfl / smax
        errs.append(np.abs(U[0] - P.vortex_exact(prob, 1.0)[0]).mean())
    assert math.log2(errs[0] / errs[1]) >= 2.6, errs
