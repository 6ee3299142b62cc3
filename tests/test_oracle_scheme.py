"""Pins of the oracle's whole step against what the method and the PDE fix:
boundary zones by hand, free-stream preservation (bitwise), conservation on
periodic grids, mirror/swap symmetries, the design order of accuracy on the
isentropic vortex, the exact Sod solution, the CFL time step by hand, and the
non-physical status."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P

G = 1.4


def run(orc, U, t, nsteps=None, t_end=None, cfl=0.4):
    dt = orc.cfl_dt(U, cfl)
    k = 0
    while True:
        if t_end is not None:
            if t >= t_end - 1e-12:
                break
            dt = min(dt, t_end - t)
        elif k >= nsteps:
            break
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        k += 1
        dt = cfl / smax
    return U, t, k


# --------------------------------------------------------------------------
def test_ghost_zones_by_hand():
    prob = P.Problem("uniform", 2, (4, 3, 1), (0, 0, 0), (4.0, 3.0, 1.0), 3,
                     bc=("reflect", "outflow", "periodic", "periodic", "periodic", "periodic"))
    orc = oracle.Oracle(prob)
    g = 3
    U = np.zeros((4, 1, 3, 4))
    for v in range(4):
        for j in range(3):
            for i in range(4):
                U[v, 0, j, i] = 100 * v + 10 * j + i + 1
    Ug = orc.ghosted(U, 0.0)
    I = lambda v, j, i: Ug[v, 0, g + j, g + i]  # active-relative indexing
    # x low reflect: mirror with x-momentum negated
    assert I(0, 1, -1) == U[0, 0, 1, 0] and I(0, 1, -3) == U[0, 0, 1, 2]
    assert I(1, 1, -2) == -U[1, 0, 1, 1] and I(2, 1, -2) == U[2, 0, 1, 1]
    # x high outflow: copy of the last zone
    assert I(3, 2, 4) == U[3, 0, 2, 3] and I(1, 2, 6) == U[1, 0, 2, 3]
    # y periodic
    assert I(0, -1, 2) == U[0, 0, 2, 2] and I(0, 3, 2) == U[0, 0, 0, 2] and I(0, 5, 1) == U[0, 0, 2, 1]
    # corner: y image (periodic) of the x image (reflect): momentum flipped once
    assert I(1, -1, -1) == -U[1, 0, 2, 0] and I(0, 4, -2) == U[0, 0, 1, 1]
    # BCs that do not commute: x inflow then y reflect -> the corner is the
    # inflow state with its y-momentum negated
    inflow = (10.0, 2.0, 3.0, 40.0)
    prob2 = P.Problem("uniform", 2, (4, 3, 1), (0, 0, 0), (4.0, 3.0, 1.0), 3,
                      bc=("inflow", "outflow", "reflect", "outflow", "periodic", "periodic"),
                      inflow=(inflow, None, None, None, None, None))
    Ug2 = oracle.Oracle(prob2).ghosted(U, 0.0)
    assert list(Ug2[:, 0, g - 1, g - 1]) == [10.0, 2.0, -3.0, 40.0]
    assert list(Ug2[:, 0, g + 1, g - 2]) == list(inflow)


def test_ghost_zones_dmr():
    prob = P.dmr(nx=24, ny=6)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    g = 3
    t = 0.01
    Ug = orc.ghosted(U, t)
    post, pre = np.array(prob.inflow[0]), np.array(prob.pre)
    xs = (np.arange(-g, 24 + g) + 0.5) * prob.dx(0)
    for ii, x in enumerate(xs):
        i = ii - g
        col_bot = Ug[:, 0, g - 1, ii]
        if x < 1.0 / 6.0:
            assert np.array_equal(col_bot, post)
        elif 0 <= i < 24:
            m = U[:, 0, 0, i].copy()
            m[2] = -m[2]
            assert np.array_equal(col_bot, m)
        top = Ug[:, 0, g + 6, ii]
        xs_t = 1.0 / 6.0 + (1.0 + 20.0 * t) / math.sqrt(3.0)
        assert np.array_equal(top, post if x < xs_t else pre)


@pytest.mark.parametrize("dim,order,bc", [(2, 2, "periodic"), (3, 2, "reflect"), (2, 3, "periodic"),
                                          (2, 4, "outflow"), (3, 3, "periodic"), (3, 4, "reflect")])
def test_free_stream_is_preserved_bitwise(dim, order, bc):
    vel = (0.3, -0.2, 0.1) if bc != "reflect" else (0.0, 0.0, 0.0)
    prob = P.uniform(dim=dim, n=6 if dim == 3 else 10, order=order, vel=vel, bc=bc)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    U1, smax, rc = orc.step(U, 0.0, 0.4 / orc.signal_max(U))
    assert rc == 0 and np.array_equal(U1, U)


def test_cfl_time_step_by_hand():
    prob = P.Problem("uniform", 2, (8, 4, 1), (0, 0, 0), (1.0, 2.0, 1.0), 3,
                     params={"rho": 1.2, "vel": (0.3, -1.5), "p": 0.8})
    U = prob.initial_state()
    c = math.sqrt(G * 0.8 / 1.2)
    s = max((0.3 + c) / (1.0 / 8), (1.5 + c) / (2.0 / 4))
    assert abs(oracle.Oracle(prob).cfl_dt(U, 0.4) - 0.4 / s) < 1e-15


def _kahan_totals(U):
    return [math.fsum(U[v].ravel()) for v in range(U.shape[0])]


@pytest.mark.parametrize("dim,order,n,steps", [(2, 3, 16, 30), (2, 4, 12, 10), (3, 4, 6, 2)])
def test_conservation_on_periodic_grids(dim, order, n, steps):
    if dim == 2:
        prob = P.vortex2d(n=n, order=order)
    else:
        prob = P.tgv3d(n=n, order=order)
    orc = oracle.Oracle(prob)
    U0 = prob.initial_state()
    U, _, _ = run(orc, U0, 0.0, nsteps=steps, cfl=prob.cfl)
    a, b = _kahan_totals(U0), _kahan_totals(U)
    for v in range(prob.nv):
        scale = max(abs(a[v]), math.fsum(np.abs(U0[v]).ravel()), math.fsum(np.abs(U0[0]).ravel()))
        assert abs(b[v] - a[v]) <= 1e-13 * scale, (v, a[v], b[v])


def test_taylor_green_mirror_symmetries():
    """The TGV state is mirror symmetric in x, y and z (zone i -> n-1-i with the
    normal velocity odd, the rest even); the stencils and linear weights are
    mirror symmetric, so the scheme must keep each symmetry to round-off.  An
    index or sign error in any one direction breaks its symmetry."""
    prob = P.tgv3d(n=8, order=3)
    orc = oracle.Oracle(prob)
    U, _, _ = run(orc, prob.initial_state(), 0.0, nsteps=2, cfl=prob.cfl)
    scale = np.abs(U).max()
    for axis, comp in ((3, 1), (2, 2), (1, 3)):
        mir = np.flip(U, axis=axis).copy()
        mir[comp] *= -1
        assert np.abs(mir - U).max() < 1e-12 * scale, axis


def _smooth_state(prob, seed):
    """positive smooth periodic state on the active grid"""
    rng = np.random.default_rng(seed)
    sh = prob.shape()
    idx = np.meshgrid(*[np.arange(n) for n in sh[1:]], indexing="ij")
    f = lambda a: sum(a * np.sin(2 * np.pi * (k + 1) * (x + 0.5) / n + rng.uniform(0, 6))
                      for k, x, n in zip(range(3), idx, sh[1:]))
    U = np.zeros(sh)
    rho = 1.0 + 0.2 * f(0.3)
    vel = [0.5 * f(0.3) for _ in range(prob.dim)]
    p = 1.0 + 0.2 * f(0.3)
    c = P.conserved(G, rho, vel, p)
    for v in range(prob.nv):
        U[v] = c[v]
    return U


@pytest.mark.parametrize("dim,order", [(2, 3), (2, 4), (3, 4)])
def test_diagonal_reflection_on_an_anisotropic_grid(dim, order):
    """Reflecting the problem across the plane x=y (2D) or y=z (3D) swaps two
    axes, their zone sizes and their momenta; it is a symmetry of the Euler
    equations.  With linear weights the 1D stencils commute, so the reflected
    run must equal the reflected result to round-off.  dx != dy catches any
    transposed zone size, flux direction or momentum index."""
    a, b = (0, 1) if dim == 2 else (1, 2)
    n = [10, 6, 4] if dim == 2 else [4, 6, 5]
    hi = [1.0, 1.5, 1.0] if dim == 2 else [1.0, 1.5, 0.5]
    probA = P.Problem("uniform", dim, tuple(n if dim == 3 else n[:2] + [1]), (0, 0, 0), tuple(hi), order)
    n2, hi2 = list(n), list(hi)
    n2[a], n2[b] = n[b], n[a]
    hi2[a], hi2[b] = hi[b], hi[a]
    probB = P.Problem("uniform", dim, tuple(n2 if dim == 3 else n2[:2] + [1]), (0, 0, 0), tuple(hi2), order)
    UA = _smooth_state(probA, 7)
    ax = lambda d: 3 - d  # array axis of dimension d in [v][z][y][x]

    def reflect(U):
        R = np.swapaxes(U, ax(a), ax(b)).copy()
        R[[1 + a, 1 + b]] = R[[1 + b, 1 + a]]
        return R

    UB = reflect(UA)
    oA, oB = oracle.Oracle(probA), oracle.Oracle(probB)
    flA = np.zeros(oA.G[::-1], dtype=np.uint8)
    flB = np.zeros(oB.G[::-1], dtype=np.uint8)
    dt = 0.3 / oA.signal_max(UA)
    A1, _, rcA = oA.step(UA, 0.0, dt, flags=flA)
    B1, _, rcB = oB.step(UB, 0.0, dt, flags=flB)
    assert rcA == 0 and rcB == 0
    assert np.abs(reflect(A1) - B1).max() < 1e-13 * np.abs(A1).max()
    # and the step did something direction dependent
    assert np.abs(A1 - UA).max() > 1e-3


@pytest.mark.parametrize("order,ns,t_end,min_rate", [(2, (32, 64, 128), 1.0, 1.6), (3, (32, 64, 128), 1.0, 2.7),
                                                    (4, (16, 32, 64), 1.0, 3.7)])
def test_design_order_on_the_isentropic_vortex(order, ns, t_end, min_rate):
    errs = []
    for n in ns:
        prob = P.vortex2d(n=n, order=order, t_end=t_end)
        orc = oracle.Oracle(prob)
        U, t, _ = run(orc, prob.initial_state(), 0.0, t_end=t_end, cfl=prob.cfl)
        errs.append(np.abs(U[0] - P.vortex_exact(prob, t_end)[0]).mean())
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert rates[-1] >= min_rate, (errs, rates)


def test_sod_converges_to_the_exact_solution():
    errs = []
    for nx in (100, 200):
        prob = P.sod(nx=nx, ny=4, order=3)
        orc = oracle.Oracle(prob)
        U, t, _ = run(orc, prob.initial_state(), 0.0, t_end=0.2, cfl=prob.cfl)
        h = 1.0 / nx
        xs = (np.arange(nx) + 0.5) * h
        sub = (np.arange(16) + 0.5) / 16 - 0.5
        ex = np.array([np.mean([oracle.exact_riemann(G, P.SOD_LEFT, P.SOD_RIGHT, (x + s * h - 0.5) / 0.2)[0][0]
                                for s in sub]) for x in xs])
        assert np.abs(U[0] - U[0][0:1]).max() < 1e-12  # y-uniform
        errs.append(np.abs(U[0, 0, 0] - ex).mean())
    assert errs[0] < 0.01 and math.log2(errs[0] / errs[1]) >= 0.6, errs


def test_nonphysical_state_is_reported():
    prob = P.uniform(dim=2, n=8, order=3)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    U[3, 0, 4, 4] = 0.01  # energy below the kinetic energy: negative pressure
    _, _, rc = orc.step(U, 0.0, 1e-3)
    assert rc == -4


@pytest.mark.parametrize("order", [3, 4])
def test_lower_dimensional_consistency(order):
    """A 3D state that varies only along z is a 1D problem: one step must equal
    the step of the 2D state varying only along x (axes and momenta rotated)
    on the same zone size.  Transverse quadrature weights must sum to one and
    every direction must see the same face fluxes."""
    n = 12
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.1 * np.cos(6 * np.pi * x)
    un = 0.4 + 0.2 * np.cos(2 * np.pi * x)
    p = 1.0 + 0.2 * np.sin(4 * np.pi * x)
    vt = 0.3 * np.sin(2 * np.pi * x)
    c2 = P.conserved(G, rho, [un, vt], p)
    p2 = P.Problem("uniform", 2, (n, 4, 1), (0, 0, 0), (1.0, 4.0 / n, 1.0), order)
    U2 = np.zeros(p2.shape())
    for v in range(4):
        U2[v] = c2[v][None, None, :]
    p3 = P.Problem("uniform", 3, (4, 4, n), (0, 0, 0), (4.0 / n, 4.0 / n, 1.0), order)
    U3 = np.zeros(p3.shape())
    # 3D: normal direction z carries un, x carries the transverse velocity
    c3 = P.conserved(G, rho, [vt, 0.0 * x, un], p)
    for v in range(5):
        U3[v] = c3[v][:, None, None]
    o2, o3 = oracle.Oracle(p2), oracle.Oracle(p3)
    dt = 0.3 / o2.signal_max(U2)
    A, _, ra = o2.step(U2, 0.0, dt)
    B, _, rb = o3.step(U3, 0.0, dt)
    assert ra == 0 and rb == 0
    scale = np.abs(A).max()
    # rho, normal momentum, transverse momentum, energy
    for a_v, b_v in ((0, 0), (1, 3), (2, 1), (3, 4)):
        assert np.abs(B[b_v][:, 0, 0] - A[a_v][0, 0, :]).max() < 1e-13 * scale, (a_v, b_v)
    assert np.abs(B[2]).max() < 1e-15


def test_order2_face_state_is_fig5():
    """At order 2 the face state is the paper's U_L = U1 + U2/2 + U5/2 at the
    face centre and mid-step (Fig. 5): U1 the zone mean, U2 the MC slope
    (Fig. 3), U5 the coefficient of tau of the predicted polynomial."""
    prob = P.vortex2d(n=12, order=2)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    dt = orc.cfl_dt(U, 0.4)
    W = orc.reconstruct(U, 0.0)          # [v][mode][By][Bx]: modes 1, xi, eta
    FS = orc.face_states(U, 0.0, dt)     # [dir][side][1][v][...]
    for (jb, ib) in ((3, 4), (6, 2), (9, 10)):
        w = W[:, :, 0, jb, ib]
        st = orc.predict_zone(w.reshape(-1).copy(), dt)
        # space-time modes (a, b, e): e outermost: (0,0,0), (1,0,0), (0,1,0), (0,0,1)
        U5 = 2.0 * st[:, 3]              # L1 = 2 tau - 1: coefficient of tau is 2*c
        UL = w[:, 0] + 0.5 * w[:, 1] + 0.5 * U5
        UR = w[:, 0] - 0.5 * w[:, 1] + 0.5 * U5
        assert np.allclose(FS[0, 1, 0, :, 0, jb, ib], UL, rtol=0, atol=1e-14)
        assert np.allclose(FS[0, 0, 0, :, 0, jb, ib], UR, rtol=0, atol=1e-14)
