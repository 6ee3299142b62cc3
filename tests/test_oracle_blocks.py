"""Pins of the oracle's building blocks against what mathematics fixes.

Each test checks the oracle (oracle/ora.c) against an independent fact: exact
integrals, exact rational stencil algebra done here by hand with fractions,
invariants of the Euler equations (Rankine-Hugoniot, Riemann invariants),
symmetries, or exact solutions (an isolated contact is advected exactly).
None of them re-calls the oracle's own routine to produce the expected value.
"""
import itertools
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

# --------------------------------------------------------------------------
# independent restatement of the basis (Legendre on [-1/2,1/2], unit leading
# coefficient) in exact rationals, used to produce expected values
# --------------------------------------------------------------------------
P_MONO = {0: {0: Fr(1)}, 1: {1: Fr(1)}, 2: {0: Fr(-1, 12), 2: Fr(1)}, 3: {1: Fr(-3, 20), 3: Fr(1)}}


def mono_zone_avg(j, s):
    """exact average of xi^j over [s-1/2, s+1/2]"""
    s = Fr(s)
    return ((s + Fr(1, 2)) ** (j + 1) - (s - Fr(1, 2)) ** (j + 1)) / (j + 1)


def mono_to_modes(m):
    """monomial coefficients m[j] (j <= 3) -> coefficients of P_0..P_3"""
    m = list(m) + [Fr(0)] * (4 - len(m))
    c3 = m[3]
    c2 = m[2]
    c1 = m[1] + Fr(3, 20) * c3
    c0 = m[0] + Fr(1, 12) * c2
    return [c0, c1, c2, c3]


def eval_P(a, x):
    return sum(float(c) * x ** j for j, c in P_MONO[a].items())


def shifted_L(e, t):
    return [1.0, 2 * t - 1, 6 * t * t - 6 * t + 1, 20 * t ** 3 - 30 * t * t + 12 * t - 1][e]


# --------------------------------------------------------------------------
def test_gauss_legendre_integrates_to_degree_2n_minus_1():
    for n in range(1, 6):
        x, w = oracle.gauss_legendre(n)
        assert np.all(np.diff(x) > 0)
        for j in range(2 * n):
            exact = float(mono_zone_avg(j, 0))
            assert abs(np.dot(w, x ** j) - exact) < 1e-15
        # degree 2n is not integrated exactly (a dropped node would pass the loop above)
        assert abs(np.dot(w, x ** (2 * n)) - float(mono_zone_avg(2 * n, 0))) > 1e-8


def test_basis_is_the_scaled_legendre_basis():
    xs = np.linspace(-0.5, 0.5, 7)
    for a in range(4):
        for x in xs:
            assert abs(oracle.basis(a, x) - eval_P(a, x)) < 1e-15
    # orthogonality and norms 1, 1/12, 1/180, 1/2800 (exact integrals of products)
    norms = [Fr(1), Fr(1, 12), Fr(1, 180), Fr(1, 2800)]
    for a in range(4):
        for b in range(4):
            prod = {}
            for i, ci in P_MONO[a].items():
                for j, cj in P_MONO[b].items():
                    prod[i + j] = prod.get(i + j, Fr(0)) + ci * cj
            integ = sum(c * mono_zone_avg(k, 0) for k, c in prod.items())
            assert integ == (norms[a] if a == b else 0)


@pytest.mark.parametrize("N", [2, 3])
def test_candidate_stencils_reproduce_polynomials_exactly(N):
    rng = np.random.default_rng(10 + N)
    for trial in range(20):
        m = [Fr(int(v), 7) for v in rng.integers(-20, 20, size=N + 1)]
        u = np.array([float(sum(m[j] * mono_zone_avg(j, s) for j in range(N + 1))) for s in range(-N, N + 1)])
        modes = mono_to_modes(m)
        for k in range(N + 1):
            c = oracle.candidate(N, k, u)
            assert np.allclose(c, [float(v) for v in modes[1:N + 1]], rtol=0, atol=1e-13), (k, c, modes)


@pytest.mark.parametrize("N", [2, 3])
def test_candidate_stencil_widths(N):
    """Candidate k uses exactly the zones k-N..k: perturbing any other zone leaves it unchanged."""
    rng = np.random.default_rng(3)
    u = rng.normal(size=2 * N + 1)
    for k in range(N + 1):
        base = oracle.candidate(N, k, u)
        for s in range(-N, N + 1):
            up = u.copy()
            up[N + s] += 1.0
            changed = not np.allclose(oracle.candidate(N, k, up), base, atol=1e-14)
            assert changed == (k - N <= s <= k), (k, s)


def test_beta_closed_forms():
    """beta = sum_l int (d^l p)^2 over the zone.  By hand:
    N=2: p' = ux + 2 uxx xi, p'' = 2 uxx -> ux^2 + (1/3 + 4) uxx^2 = ux^2 + 13/3 uxx^2.
    N=3: p' = (ux + uxxx/10) + 2 uxx xi + 3 uxxx (xi^2 - 1/12), int (xi^2-1/12)^2 = 1/180,
    p'' = 2 uxx + 6 uxxx xi, p''' = 6 uxxx ->
    (ux + uxxx/10)^2 + 13/3 uxx^2 + (1/20 + 3 + 36) uxxx^2."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        ux, uxx, uxxx = rng.normal(size=3)
        assert abs(oracle.beta(2, [ux, uxx]) - (ux ** 2 + 13.0 / 3.0 * uxx ** 2)) < 1e-12
        exp3 = (ux + uxxx / 10) ** 2 + 13.0 / 3.0 * uxx ** 2 + 781.0 / 20.0 * uxxx ** 2
        assert abs(oracle.beta(3, [ux, uxx, uxxx]) - exp3) < 1e-11 * max(1, exp3)


@pytest.mark.parametrize("N", [2, 3])
def test_weno_reproduces_polynomials_for_any_weights(N):
    from paper_2211_13295_gb300.problems import LINEAR_WEIGHTS
    lin = LINEAR_WEIGHTS[N + 1]
    rng = np.random.default_rng(20 + N)
    for _ in range(20):
        m = [Fr(int(v), 3) for v in rng.integers(-30, 30, size=N + 1)]
        u = np.array([float(sum(m[j] * mono_zone_avg(j, s) for j in range(N + 1))) for s in range(-N, N + 1)])
        modes = [float(v) for v in mono_to_modes(m)[1:N + 1]]
        for lin_only in (False, True):
            c, om = oracle.weno1d(N, u, 1e-12, lin, lin_only)
            assert abs(om.sum() - 1.0) < 1e-14
            assert np.allclose(c, modes, rtol=0, atol=1e-11 * max(1, np.abs(u).max()))


@pytest.mark.parametrize("N", [2, 3])
def test_weno_weights_smooth_and_discontinuous(N):
    from paper_2211_13295_gb300.problems import LINEAR_WEIGHTS
    lin = np.array(LINEAR_WEIGHTS[N + 1])
    # smooth: samples of sin at fine resolution -> weights near linear
    h = 1e-2
    s = np.arange(-N, N + 1)
    u = (np.cos((s - 0.5) * h + 0.3) - np.cos((s + 0.5) * h + 0.3)) / h
    _, om = oracle.weno1d(N, u, 1e-12, lin)
    assert np.abs(om - lin).max() < 0.05
    # a jump between zones 0 and +1: every candidate that crosses it gets ~0 weight
    u = np.where(s <= 0, 1.0, 0.1)
    _, om = oracle.weno1d(N, u, 1e-12, lin)
    assert om[0] > 0.999
    assert np.all(om[1:] < 1e-6)


# --------------------------------------------------------------------------
# HLLC
# --------------------------------------------------------------------------
G = 1.4


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


def rand_state(rng, dim):
    return cons(rng.uniform(0.2, 3), rng.uniform(-2, 2, size=dim), rng.uniform(0.1, 5))


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_consistency_and_symmetries(dim):
    rng = np.random.default_rng(5)
    for _ in range(40):
        UL, UR = rand_state(rng, dim), rand_state(rng, dim)
        for d in range(dim):
            F = oracle.hllc(dim, G, d, UL, UL)
            assert np.allclose(F, euler_flux(UL, d, dim), rtol=1e-13, atol=1e-13)
            # mirror: reflect the normal direction, swap sides -> flux negated, normal momentum kept
            R = np.ones(dim + 2)
            R[1 + d] = -1
            F1 = oracle.hllc(dim, G, d, UL, UR)
            F2 = oracle.hllc(dim, G, d, R * UR, R * UL)
            assert np.allclose(F2, -R * F1, rtol=1e-12, atol=1e-12)
            # rotation: direction d flux equals the x flux of the permuted states
            if d > 0:
                perm = list(range(dim + 2))
                perm[1], perm[1 + d] = perm[1 + d], perm[1]
                Fx = oracle.hllc(dim, G, 0, UL[perm], UR[perm])
                assert np.allclose(F1[perm], Fx, rtol=1e-12, atol=1e-12)


def test_hllc_resolves_isolated_contacts_exactly():
    dim = 3
    # stationary contact: only the pressure flux survives
    UL, UR = cons(1.0, [0, 0.3, -0.2], 0.7), cons(0.2, [0, -1.0, 0.5], 0.7)
    F = oracle.hllc(dim, G, 0, UL, UR)
    assert np.allclose(F, [0, 0.7, 0, 0, 0], atol=1e-14)
    # moving contact: the upwind physical flux
    for u in (0.4, -0.4):
        UL, UR = cons(1.0, [u, 0.3, -0.2], 0.7), cons(0.2, [u, -1.0, 0.5], 0.7)
        F = oracle.hllc(dim, G, 0, UL, UR)
        up = UL if u > 0 else UR
        assert np.allclose(F, euler_flux(up, 0, dim), rtol=1e-13, atol=1e-13)
    # supersonic to the right: left flux
    UL, UR = cons(1.0, [5.0, 0, 0], 1.0), cons(0.5, [4.0, 0, 0], 0.4)
    assert np.allclose(oracle.hllc(dim, G, 0, UL, UR), euler_flux(UL, 0, dim), rtol=1e-13)


# --------------------------------------------------------------------------
# exact Riemann solver
# --------------------------------------------------------------------------
def prim_to_cons1(r, u, p):
    return np.array([r, r * u, p / (G - 1) + 0.5 * r * u * u])


def flux1(r, u, p):
    E = p / (G - 1) + 0.5 * r * u * u
    return np.array([r * u, r * u * u + p, (E + p) * u])


def test_exact_riemann_sod_invariants():
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    (_, _, _), (ps, us) = oracle.exact_riemann(G, left, right, 0.0)
    # textbook star values of this problem (Toro, Riemann Solvers, Table 4.3, test 1)
    assert abs(ps - 0.30313) < 5e-6 and abs(us - 0.92745) < 5e-6
    ss = np.linspace(-2, 2, 4001)
    sol = np.array([oracle.exact_riemann(G, left, right, s)[0] for s in ss])
    # right shock: Rankine-Hugoniot with the speed implied by mass conservation
    post = sol[(ss > us + 1e-3) & (ss < us + 0.5)][0]
    S = (post[0] * post[1] - right[0] * right[1]) / (post[0] - right[0])
    lhs = flux1(*post) - S * prim_to_cons1(*post)
    rhs = flux1(*right) - S * prim_to_cons1(*right)
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-10)
    # left rarefaction: entropy and the Riemann invariant u + 2c/(g-1) constant through the fan
    fan = sol[(ss > -1.2) & (ss < -0.1)]
    ent = fan[:, 2] / fan[:, 0] ** G
    inv = fan[:, 1] + 2 * np.sqrt(G * fan[:, 2] / fan[:, 0]) / (G - 1)
    assert np.ptp(ent) < 1e-12 and np.ptp(inv) < 1e-12
    # contact: p and u continuous
    a = oracle.exact_riemann(G, left, right, us - 1e-9)[0]
    b = oracle.exact_riemann(G, left, right, us + 1e-9)[0]
    assert abs(a[1] - b[1]) < 1e-12 and abs(a[2] - b[2]) < 1e-12 and abs(a[0] - b[0]) > 0.1


def test_exact_riemann_two_shocks_rankine_hugoniot():
    left, right = (1.0, 2.0, 1.0), (1.0, -2.0, 1.0)
    (_, _, _), (ps, us) = oracle.exact_riemann(G, left, right, 0.0)
    assert abs(us) < 1e-12 and ps > 1.0
    for side, st in ((-1, left), (1, right)):
        ss = np.linspace(0, side * 5, 5001)
        sol = np.array([oracle.exact_riemann(G, left, right, s)[0] for s in ss])
        post = sol[1]
        S = (post[0] * post[1] - st[0] * st[1]) / (post[0] - st[0])
        assert np.allclose(flux1(*post) - S * prim_to_cons1(*post), flux1(*st) - S * prim_to_cons1(*st),
                           rtol=1e-10, atol=1e-10)


# --------------------------------------------------------------------------
# predictor
# --------------------------------------------------------------------------
def st_modes(dim, N):
    out = []
    cmax = N if dim == 3 else 0
    for e in range(N + 1):
        for c in range(min(cmax, N - e) + 1):
            for b in range(N - e - c + 1):
                for a in range(N - e - b - c + 1):
                    out.append((a, b, c, e))
    return out


def s_modes(dim, N):
    out = []
    cmax = N if dim == 3 else 0
    for c in range(cmax + 1):
        for b in range(N - c + 1):
            for a in range(N - b - c + 1):
                out.append((a, b, c))
    return out


def eval_st(coef, modes, xi, tau):
    acc = 0.0
    for cf, (a, b, c, e) in zip(coef, modes):
        acc += cf * eval_P(a, xi[0]) * eval_P(b, xi[1]) * eval_P(c, xi[2]) * shifted_L(e, tau)
    return acc


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (2, 3), (2, 4), (3, 3), (3, 4)])
def test_predictor_advects_an_isolated_contact_exactly(dim, order):
    """Constant velocity and pressure, polynomial density of degree <= N: the
    Euler equations reduce to linear advection and the exact space-time
    solution rho0(xi - lam*tau) is a polynomial of total degree <= N, which the
    predictor must return exactly after N Picard sweeps."""
    from paper_2211_13295_gb300 import problems as P
    N = order - 1
    prob = P.uniform(dim=dim, n=4, order=order)
    orc = oracle.Oracle(prob)
    rng = np.random.default_rng(order * 10 + dim)
    vel = np.array([0.7, -0.4, 0.25][:dim])
    p = 1.3
    sm = s_modes(dim, N)
    # density: random modal coefficients (small, mean 1)
    rho_m = np.array([1.0 if m == (0, 0, 0) else 0.05 * rng.normal() for m in sm])
    w = np.zeros((dim + 2, len(sm)))
    w[0] = rho_m
    for d in range(dim):
        w[1 + d] = vel[d] * rho_m
    w[-1] = 0.5 * (vel ** 2).sum() * rho_m
    w[-1][0] += p / (G - 1)
    dt = 0.3 * prob.dx(0)
    lam = [vel[d] * dt / prob.dx(d) for d in range(dim)] + [0.0] * (3 - dim)
    st = orc.predict_zone(w, dt)
    stm = st_modes(dim, N)

    def rho0(xi):
        return sum(cf * eval_P(a, xi[0]) * eval_P(b, xi[1]) * eval_P(c, xi[2]) for cf, (a, b, c) in zip(rho_m, sm))

    for _ in range(20):
        xi = list(rng.uniform(-0.5, 0.5, size=dim)) + [0.0] * (3 - dim)
        tau = rng.uniform(0, 1)
        shifted = [xi[d] - lam[d] * tau for d in range(3)]
        assert abs(eval_st(st[0], stm, xi, tau) - rho0(shifted)) < 1e-13
        for d in range(dim):
            assert abs(eval_st(st[1 + d], stm, xi, tau) - vel[d] * rho0(shifted)) < 1e-13
    if N < 2:
        return
    # with one sweep fewer the cubic/quadratic-in-time terms are missing (for N >= 2)
    prob2 = prob.replace(picard=N - 1)
    st2 = oracle.Oracle(prob2).predict_zone(w, dt)
    errs = [abs(eval_st(st2[0], stm, [0.5, 0.2, 0.1], 1.0) - rho0([0.5 - lam[0], 0.2 - lam[1], 0.1 - lam[2]]))]
    assert max(errs) > 1e-9


def eval_dP(a, x):
    """derivative of the scaled Legendre basis function P_a (closed form)"""
    return sum(float(c) * j * x ** (j - 1) for j, c in P_MONO[a].items() if j > 0)


def eval_st_ddx(coef, modes, xi, tau, d):
    """d/dxi_d of a space-time polynomial given by its modal coefficients"""
    acc = 0.0
    for cf, (a, b, c, e) in zip(coef, modes):
        f = [eval_P(a, xi[0]), eval_P(b, xi[1]), eval_P(c, xi[2])]
        f[d] = eval_dP((a, b, c)[d], xi[d])
        acc += cf * f[0] * f[1] * f[2] * shifted_L(e, tau)
    return acc


@pytest.mark.parametrize("dim,order", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3), (3, 4)])
def test_picard_mass_row_is_the_exact_momentum_divergence(dim, order):
    """The mass flux of direction d is the momentum q_{1+d}, which lies in the
    space the predictor projects onto (total degree <= N in space and time); the
    (N+1)-point Gauss rules integrate its products with the test functions
    exactly, so each Picard sweep must give, for a general (non-linear) state,
    rho^{k+1}(xi, tau) = w_rho(xi) - sum_d lam_d int_0^tau d/dxi_d q^k_{1+d}(xi, s) ds
    exactly: the space-time update of the method (the paper's predictor, Fig. 4)
    for the one conservation law with a linear flux.  The right side is evaluated
    here from the basis closed forms and a Gauss rule on [0, tau]."""
    from paper_2211_13295_gb300 import problems as P
    N = order - 1
    prob = P.uniform(dim=dim, n=4, order=order)
    rng = np.random.default_rng(100 * dim + order)
    sm = s_modes(dim, N)
    stm = st_modes(dim, N)
    w = 0.1 * rng.normal(size=(dim + 2, len(sm)))
    w[0][0], w[-1][0] = 1.0, 2.5
    for d in range(dim):
        w[1 + d][0] = 0.5 * rng.normal()
    dt = 0.2 * prob.dx(0)
    lam = [dt / prob.dx(d) for d in range(dim)]
    xg, wg = oracle.gauss_legendre(N + 1)

    def w_rho(xi):
        return sum(cf * eval_P(a, xi[0]) * eval_P(b, xi[1]) * eval_P(c, xi[2]) for cf, (a, b, c) in zip(w[0], sm))

    prev = None
    for K in range(1, N + 1):
        st = oracle.Oracle(prob.replace(picard=K)).predict_zone(w, dt)
        for _ in range(12):
            xi = list(rng.uniform(-0.5, 0.5, size=dim)) + [0.0] * (3 - dim)
            tau = rng.uniform(0, 1)
            rhs = w_rho(xi)
            for d in range(dim):
                if prev is None:   # q^0 = w: time-independent
                    div = sum(cf * (eval_dP(a, xi[0]) if d == 0 else eval_P(a, xi[0])) *
                              (eval_dP(b, xi[1]) if d == 1 else eval_P(b, xi[1])) *
                              (eval_dP(c, xi[2]) if d == 2 else eval_P(c, xi[2]))
                              for cf, (a, b, c) in zip(w[1 + d], sm))
                    rhs -= lam[d] * tau * div
                else:
                    integ = sum(wq * tau * eval_st_ddx(prev[1 + d], stm, xi, tau * (xq + 0.5), d)
                                for xq, wq in zip(xg, wg))
                    rhs -= lam[d] * integ
            assert abs(eval_st(st[0], stm, xi, tau) - rhs) < 1e-13
        prev = st


def test_fig5_face_state_convention(golden):
    """The paper's O2 flux builds the x-face states from the zone mean (mode 1),
    the x-slope (mode 2) and the time mode (mode 5) as U1 +/- U2/2 + U5/2
    (Fig. 5).  With a linear contact profile the oracle's face states, averaged
    over its time nodes, must follow that rule with U5 the coefficient of tau."""
    from paper_2211_13295_gb300 import problems as P
    fx = golden("fig5_face_state.json")
    dim, order = 2, 3
    prob = P.uniform(dim=dim, n=4, order=order)
    orc = oracle.Oracle(prob)
    u, p = fx["u"], 1.0
    rho_mean, rho_slope = fx["U1"], fx["U2"]
    sm = s_modes(dim, 2)
    rho_m = np.array([rho_mean if m == (0, 0, 0) else (rho_slope if m == (1, 0, 0) else 0.0) for m in sm])
    w = np.zeros((4, len(sm)))
    w[0] = rho_m
    w[1] = u * rho_m
    w[3] = 0.5 * u * u * rho_m
    w[3][0] += p / (G - 1)
    dt = fx["lam"] * prob.dx(0) / u
    st = orc.predict_zone(w, dt)
    stm = st_modes(dim, 2)
    x, _ = oracle.gauss_legendre(2)
    left_face = np.mean([eval_st(st[0], stm, [0.5, 0.0, 0.0], t + 0.5) for t in x])
    right_face = np.mean([eval_st(st[0], stm, [-0.5, 0.0, 0.0], t + 0.5) for t in x])
    U5 = fx["U5"]
    assert abs(left_face - (rho_mean + 0.5 * rho_slope + 0.5 * U5)) < 1e-14
    assert abs(right_face - (rho_mean - 0.5 * rho_slope + 0.5 * U5)) < 1e-14


def test_hllc_resolves_a_stationary_shock_exactly():
    """For two states joined by a single shock the Roe matrix has the shock
    speed as an eigenvalue (Roe's property A(UL,UR)(UR-UL) = F(UR)-F(UL)), so
    the Roe-average speed estimate of the shock family is exact; for a
    stationary shock the HLLC flux must then be the exact flux F(UL) = F(UR)."""
    for M in (1.5, 3.0, 8.0):
        for dim in (2, 3):
            rl, pl = 1.0, 1.0
            ul = M * math.sqrt(G * pl / rl)
            # Rankine-Hugoniot for a stationary normal shock
            rr = rl * (G + 1) * M * M / ((G - 1) * M * M + 2)
            pr = pl * (2 * G * M * M - (G - 1)) / (G + 1)
            ur = rl * ul / rr
            vt = [0.3, -0.2][:dim - 1]
            UL = cons(rl, [ul] + vt, pl)
            UR = cons(rr, [ur] + vt, pr)
            FL, FR = euler_flux(UL, 0, dim), euler_flux(UR, 0, dim)
            assert np.allclose(FL, FR, rtol=1e-13)
            F = oracle.hllc(dim, G, 0, UL, UR)
            assert np.allclose(F, FL, rtol=1e-12, atol=1e-12), (M, dim, F, FL)


def test_hllc_is_exact_for_an_isolated_moving_shock():
    """A right-facing shock of speed S > 0: Roe's property makes the Roe speed
    u~ + c~ equal S, and with that wave speed the HLLC middle wave speed is
    S* = u_L and the star state is U_L (both by Rankine-Hugoniot), so the flux
    is the exact Godunov flux F(U_L) in every frame with S > 0; mirrored, a
    left-facing shock with S < 0 gives F(U_R)."""
    for M in (1.5, 3.0, 6.0):
        rr, pr = 0.8, 1.1
        cr = math.sqrt(G * pr / rr)
        S0 = M * cr                       # pre-shock (right) state at rest
        rl = rr * (G + 1) * M * M / ((G - 1) * M * M + 2)
        pl = pr * (2 * G * M * M - (G - 1)) / (G + 1)
        ul0 = S0 * (1 - rr / rl)
        for w in (0.0, -0.3 * S0, -0.6 * S0, -0.95 * S0, 0.5 * S0):
            for dim in (2, 3):
                vt = [0.25, -0.1][:dim - 1]
                UL = cons(rl, [ul0 + w] + vt, pl)
                UR = cons(rr, [w] + vt, pr)
                F = oracle.hllc(dim, G, 0, UL, UR)
                assert np.allclose(F, euler_flux(UL, 0, dim), rtol=1e-12, atol=1e-12), (M, w, dim)
                # mirror image: left-facing shock moving left
                R = np.ones(dim + 2)
                R[1] = -1
                Fm = oracle.hllc(dim, G, 0, R * UR, R * UL)
                assert np.allclose(Fm, euler_flux(R * UL, 0, dim), rtol=1e-12, atol=1e-12), (M, w, dim)


def test_mc_limiter_of_fig3_by_hand():
    """Fig. 3: MC_Limiter(a, b, cfac) = MIN(0.5|a+b|, cfac|a|, cfac|b|) *
    (SIGN(0.5,a) + SIGN(0.5,b)), SIGN(A,B) = |A| with the sign of B."""
    cases = [((1.0, 3.0, 2.0), 2.0),     # min(2, 2, 6)
             ((3.0, 1.0, 1.5), 1.5),     # min(2, 4.5, 1.5)
             ((-1.0, -0.25, 2.0), -0.5),  # min(0.625, 2, 0.5) negative
             ((1.0, -1.0, 2.0), 0.0),     # opposite signs
             ((0.0, 2.0, 2.0), 0.0),      # cfac*|a| = 0
             ((0.4, 0.4, 1.5), 0.4)]      # smooth: the centred slope
    for (a, b, cf), exp in cases:
        assert oracle.mc_slope(a, b, cf) == exp, (a, b, cf)
