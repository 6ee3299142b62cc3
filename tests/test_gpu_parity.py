"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, row by
row: reconstructed modes, predictor face states, HLLC face fluxes, the full
step, the CFL time step, boundary conditions, the FP32-bulk form, slab
streaming, checkpoint/resume, conservation, free stream and error statuses.

Tolerance: FP64 form within 1e-12 relative L1 per variable per step (the
spec bar), elementwise within 1e-10 of the variable's scale for the
intermediate rows (modes, face states, fluxes: these sit before the
cancellation of the flux difference).  Grid sizes are ragged (not multiples
of any block size) and small enough for the oracle to finish in seconds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def smooth_state(prob, seed, amp=0.2):
    """positive smooth periodic state (seeded)"""
    rng = np.random.default_rng(seed)
    sh = prob.shape()
    idx = np.meshgrid(*[np.arange(n) for n in sh[1:]], indexing="ij")

    def f():
        return sum(np.sin(2 * np.pi * (k + 1) * (x + 0.5) / n + rng.uniform(0, 6))
                   for k, x, n in zip(range(3), idx, sh[1:]))
    rho = 1.0 + amp * 0.3 * f()
    vel = [amp * 2.0 * f() for _ in range(prob.dim)]
    p = 1.0 + amp * 0.3 * f()
    c = P.conserved(1.4, rho, vel, p)
    U = np.zeros(sh)
    for v in range(prob.nv):
        U[v] = c[v]
    return U


def shocky_state(prob, seed):
    """smooth state with a density/pressure jump across a tilted plane"""
    U = smooth_state(prob, seed, amp=0.1)
    sh = prob.shape()
    idx = np.meshgrid(*[np.arange(n) for n in sh[1:]], indexing="ij")
    plane = sum((0.7 + 0.3 * d) * x / n for d, (x, n) in enumerate(zip(idx, sh[1:]))) < 0.9
    U[:, plane] *= 2.5
    return U


CASES = [
    # (dim, order, n, state)
    (2, 2, (13, 11, 1), "shock"),
    (3, 2, (9, 7, 6), "smooth"),
    (2, 3, (13, 11, 1), "smooth"),
    (2, 4, (12, 9, 1), "shock"),
    (3, 3, (9, 7, 6), "shock"),
    (3, 4, (7, 6, 5), "smooth"),
    (3, 4, (6, 7, 5), "shock"),
]


def make(dim, order, n, state, bc="periodic"):
    prob = P.Problem("uniform", dim, n, (0, 0, 0), (1.0, 1.3, 0.8), order, bc=(bc,) * 6)
    U = smooth_state(prob, 3) if state == "smooth" else shocky_state(prob, 4)
    return prob, U


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_modes_match_the_oracle(awe, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    g = awe.Grid(prob)
    g.set_state(U)
    Wg = g.probe_modes()
    Wo = oracle.Oracle(prob).reconstruct(U, 0.0)
    assert Wg.shape == Wo.shape
    for v in range(prob.nv):
        scale = np.abs(Wo[v]).max()
        assert np.abs(Wg[v] - Wo[v]).max() <= 1e-11 * scale, v


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_face_states_match_the_oracle(awe, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Fg = g.probe_face_states(dt)
    Fo = orc.face_states(U, 0.0, dt)
    for v in range(prob.nv):
        scale = np.abs(Fo[:, :, :, v]).max()
        assert np.abs(Fg[:, :, :, v] - Fo[:, :, :, v]).max() <= 1e-10 * scale, v


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_fp32_face_states_and_fluxes_match_the_oracle(awe, dim, order, n, state):
    """The FP32-bulk form's stages one by one (the line kernel of the predictor
    at 3D order 4, the thread-per-zone kernel elsewhere; FP32 Riemann
    fluxes): face states within 2e-6 of each variable's scale (FP32 rounding,
    6e-8, through the reconstruction and the Picard sweeps) and fluxes within
    5e-6 of theirs, elementwise, against the FP64 oracle."""
    prob, U = make(dim, order, n, state)
    g = awe.Grid(prob, prec="fp32")
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Fg = g.probe_face_states(dt)
    Fo = orc.face_states(U, 0.0, dt)
    for v in range(prob.nv):
        scale = np.abs(Fo[:, :, :, v]).max()
        err = np.abs(Fg[:, :, :, v] - Fo[:, :, :, v]).max() / scale
        assert err <= 2e-6, (v, err)
    Gg = g.probe_fluxes(dt)
    Go = orc.fluxes(U, 0.0, dt)
    for d in range(dim):
        for v in range(prob.nv):
            scale = max(np.abs(Go[d][v]).max(), np.abs(Go[d][0]).max())
            err = np.abs(Gg[d][v] - Go[d][v]).max() / scale
            assert err <= 5e-6, (d, v, err)
    g.close()


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_fluxes_match_the_oracle(awe, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Fg = g.probe_fluxes(dt)
    Fo = orc.fluxes(U, 0.0, dt)
    for d in range(dim):
        for v in range(prob.nv):
            scale = np.abs(Fo[d][v]).max() + 1e-300
            assert np.abs(Fg[d][v] - Fo[d][v]).max() <= 1e-10 * scale, (d, v)


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_full_step_matches_the_oracle(awe, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    dn = g.step(dt)
    Ug = g.get_state()
    Uo, smax, rc = orc.step(U, 0.0, dt)
    assert rc == 0
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v
    assert abs(dn - prob.cfl / smax) <= 1e-13 * dn
    assert abs(g.time() - dt) <= 1e-15


def test_cfl_dt_matches_the_oracle(awe):
    prob, U = make(3, 4, (7, 6, 5), "shock")
    g = awe.Grid(prob)
    g.set_state(U)
    assert abs(g.cfl_dt(0.3) - oracle.Oracle(prob).cfl_dt(U, 0.3)) <= 1e-14 * g.cfl_dt(0.3)


def test_several_steps_with_device_resident_dt(awe):
    """20 steps of the 2D vortex (order 3) with dt kept on the device; the
    oracle gets the same dt sequence (read back at the end of each step)."""
    prob = P.vortex2d(n=24, order=3)
    U0 = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U0)
    orc = oracle.Oracle(prob)
    U = U0
    t = 0.0
    dt = g.cfl_dt()
    for k in range(20):
        dn = g.step(0.0)  # device-resident dt
        U, smax, rc = orc.step(U, t, dt)
        t += dt
        assert rc == 0
        assert abs(dn - prob.cfl / smax) <= 1e-12 * dn
        dt = dn
    Ug = g.get_state()
    for v in range(prob.nv):
        assert rel_l1(Ug[v], U[v]) <= 1e-12 * 20, v
    assert abs(g.time() - t) <= 1e-13


@pytest.mark.parametrize("bc", ["outflow", "reflect"])
def test_boundary_conditions_3d(awe, bc):
    prob, U = make(3, 4, (6, 7, 5), "shock", bc=bc)
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    g.step(dt)
    Uo, _, rc = orc.step(U, 0.0, dt)
    assert rc == 0
    Ug = g.get_state()
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v


def test_double_mach_reflection_status_parity(awe):
    """The plain method has no positivity limiter: at the initial Mach-10 shock
    of the double Mach reflection the order-3 face polynomials undershoot to
    negative pressure.  Both the oracle and the CUDA path must report it
    (status -4) on the first step, and agree on the updated state where it is
    finite."""
    prob = P.dmr(nx=48, ny=12)
    U = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = orc.cfl_dt(U, prob.cfl)
    Uo, _, rc = orc.step(U, 0.0, dt)
    assert rc == -4
    with pytest.raises(awe.AweError) as ei:
        g.step(dt)
    assert ei.value.code == awe.AWE_ERR_NONPHYSICAL
    Ug = g.get_state()
    fin = np.isfinite(Uo).all(axis=0) & np.isfinite(Ug).all(axis=0)
    assert fin.mean() > 0.9
    for v in range(prob.nv):
        assert np.abs(Ug[v][fin] - Uo[v][fin]).sum() <= 1e-12 * np.abs(Uo[v][fin]).sum(), v


def test_free_stream_bitwise_on_gpu(awe):
    for dim, order in ((2, 3), (3, 4)):
        prob = P.uniform(dim=dim, n=7 if dim == 3 else 11, order=order)
        U = prob.initial_state()
        g = awe.Grid(prob)
        g.set_state(U)
        g.step(0.01)
        assert np.array_equal(g.get_state(), U)


def test_conservation_on_gpu(awe):
    prob = P.tgv3d(n=12, order=4)
    U0 = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U0)
    g.cfl_dt(0.3)
    for _ in range(10):
        g.step(0.0, sync=False)
    g.check()
    U = g.get_state()
    for v in range(prob.nv):
        a, b = math.fsum(U0[v].ravel()), math.fsum(U[v].ravel())
        scale = max(math.fsum(np.abs(U0[v]).ravel()), math.fsum(np.abs(U0[0]).ravel()))
        assert abs(a - b) <= 1e-13 * scale, v


def test_slab_streaming_is_bitwise_identical(awe):
    prob, U = make(3, 4, (7, 6, 11), "shock")
    a = awe.Grid(prob)
    b = awe.Grid(prob, slab=3)
    a.set_state(U)
    b.set_state(U)
    for _ in range(2):
        a.step(0.002)
        b.step(0.002)
    assert np.array_equal(a.get_state(), b.get_state())


def test_checkpoint_resume_is_bitwise(awe):
    """N+M steps equal N steps -> get_state/time -> fresh grid -> M steps."""
    prob = P.vortex2d(n=20, order=4)
    U0 = prob.initial_state()
    ref = awe.Grid(prob)
    ref.set_state(U0)
    dts = [ref.cfl_dt()]
    for _ in range(6):
        dts.append(ref.step(dts[-1]))
    a = awe.Grid(prob)
    a.set_state(U0)
    for k in range(3):
        a.step(dts[k])
    snap, t = a.get_state(), a.time()
    b = awe.Grid(prob)
    b.set_state(snap)
    b.set_time(t)
    for k in range(3, 6):
        b.step(dts[k])
    assert np.array_equal(b.get_state(), ref.get_state())
    assert b.time() == ref.time()


def test_fp32_bulk_form_tolerance(awe):
    """FP32 bulk arithmetic, FP64 update: one step within 1e-5 relative L1 of
    the FP64 oracle (a stated tolerance: FP32 rounding of fluxes ~1e-7
    relative, times the face count and the flux-difference cancellation)."""
    for dim, order, n, state in CASES:
        prob, U = make(dim, order, n, state)
        g = awe.Grid(prob, prec="fp32")
        g.set_state(U)
        orc = oracle.Oracle(prob)
        dt = 0.3 / orc.signal_max(U)
        g.step(dt)
        Uo, _, _ = orc.step(U, 0.0, dt)
        Ug = g.get_state()
        for v in range(prob.nv):
            assert rel_l1(Ug[v], Uo[v]) <= 1e-5, (dim, order, v, rel_l1(Ug[v], Uo[v]))


def test_status_codes(awe, monkeypatch):
    prob = P.uniform(dim=2, n=8, order=3)
    # invalid configuration
    bad = prob.replace(order=5)
    with pytest.raises(awe.AweError) as ei:
        awe.Grid(bad.replace(lin=(0.25, 0.25, 0.25, 0.25)))
    assert ei.value.code == awe.AWE_ERR_ARG
    # non-physical state reported, GPU context still usable
    U = prob.initial_state()
    U[3, 0, 4, 4] = 0.01
    g = awe.Grid(prob)
    g.set_state(U)
    with pytest.raises(awe.AweError) as ei:
        g.step(1e-3)
    assert ei.value.code == awe.AWE_ERR_NONPHYSICAL
    g.set_state(prob.initial_state())
    g.step(1e-3)
    # forced allocation failure
    monkeypatch.setenv("AWE_FAIL_ALLOC", "1")
    with pytest.raises(awe.AweError) as ei:
        awe.Grid(prob)
    assert ei.value.code == awe.AWE_ERR_OOM


@pytest.mark.parametrize("name", ["dmr", "blast"])
def test_positivity_fallback_matches_the_oracle(awe, name):
    """With the opt-in positivity fallback the double Mach reflection and the
    blast run; both implementations send the same zones to first order."""
    if name == "dmr":
        prob, steps = P.dmr(nx=64, ny=16).replace(fallback=True), 8
    else:
        prob, steps = P.blast3d(n=10, order=4).replace(fallback=True), 3
    U = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    t = 0.0
    dt = orc.cfl_dt(U, prob.cfl)
    for k in range(steps):
        g.step(dt)
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        dt = prob.cfl / smax
    Ug = g.get_state()
    for v in range(prob.nv):
        scale = max(np.abs(U[v]).sum(), np.abs(U[0]).sum())
        assert np.abs(Ug[v] - U[v]).sum() <= 1e-12 * steps * scale, v


def test_order2_vortex_run_matches_the_oracle(awe):
    """The paper's own second-order scheme (MC limiter, one predictor sweep,
    one mid-face mid-step Riemann solve) on the vortex for 30 steps."""
    prob = P.vortex2d(n=32, order=2)
    U = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    t, dt = 0.0, orc.cfl_dt(U, prob.cfl)
    for _ in range(30):
        g.step(dt)
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        dt = prob.cfl / smax
    Ug = g.get_state()
    for v in range(prob.nv):
        assert rel_l1(Ug[v], U[v]) <= 1e-12 * 30, v


@pytest.mark.parametrize("name", ["dmr", "blast"])
def test_fallback_count_matches_the_oracle(awe, name):
    """The number of box zones whose face states go to the positivity
    fallback in one step equals the oracle's (an integer decision taken in
    FP64 on both sides)."""
    if name == "dmr":
        prob = P.dmr(nx=96, ny=24, order=3).replace(fallback=True)
    else:
        prob = P.blast3d(n=24, order=4).replace(fallback=True)
    U = prob.initial_state()
    orc = oracle.Oracle(prob)
    dt = orc.cfl_dt(U, prob.cfl)
    g = awe.Grid(prob)
    g.set_state(U)
    g.step(dt, sync=False)
    n_gpu = g.fallback_count()
    g.close()
    n_orc = orc.fallback_count(U, 0.0, dt)
    assert n_gpu == n_orc and n_orc > 0, (n_gpu, n_orc)
