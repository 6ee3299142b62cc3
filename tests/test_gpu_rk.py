"""Parity of the Runge-Kutta variant on the GPU (Table IV's comparison
scheme: SSP(2,2), SSP(3,3), SSP(5,4)) with the FP64 oracle: whole steps on
ragged 2D/3D grids at orders 2-4 (FP64 within 1e-12 relative L1, FP32 bulk
within 1e-5), a time-dependent boundary crossed within the step, the gate
(flags recomputed at every stage), the other Riemann solvers, slab streaming
(bitwise), and sampled windows of a full-size step."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P
from test_gpu_parity import CASES, make, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


def gpu_step(awe, prob, U, dt, prec="fp64", gate=None, slab=0, t=0.0):
    g = awe.Grid(prob, prec=prec, gate=gate is not None, slab=slab)
    if gate is not None:
        g.gate_set_weights(gate)
    g.set_state(U)
    if t:
        g.set_time(t)
    dn = g.step(dt)
    out = g.get_state()
    g.close()
    return out, dn


@pytest.mark.parametrize("dim,order,n,state", CASES)
def test_step_matches_the_oracle(awe, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    prob = prob.replace(scheme="ssprk")
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Ug, dn = gpu_step(awe, prob, U, dt)
    Uo, smax, rc = orc.rk_step(U, 0.0, dt)
    assert rc == 0
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v
    assert abs(dn - prob.cfl / smax) <= 1e-13 * dn
    U32, _ = gpu_step(awe, prob, U, dt, prec="fp32")
    for v in range(prob.nv):
        assert rel_l1(U32[v], Uo[v]) <= 1e-5, v


@pytest.mark.parametrize("stages", [2, 3, 5])
def test_stage_count_and_riemann_solver(awe, stages):
    """Every stage count at order 3 (3D, shocked), with HLLEM."""
    prob, U = make(3, 3, (9, 7, 6), "shock")
    prob = prob.replace(scheme="ssprk", rk_stages=stages, riemann="hllem")
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Ug, _ = gpu_step(awe, prob, U, dt)
    Uo, _, rc = orc.rk_step(U, 0.0, dt)
    assert rc == 0
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v


@pytest.mark.parametrize("stages", [2, 3, 5])
def test_time_dependent_boundary_at_the_stage_times(awe, stages):
    """Double Mach reflection, started so that the top boundary's shock
    passes a ghost zone centre within the step (the oracle pins that the
    boundary values then differ between stages)."""
    prob = P.dmr(nx=24, ny=8, order=3).replace(fallback=True, scheme="ssprk", rk_stages=stages)
    orc = oracle.Oracle(prob)
    U = prob.initial_state()
    dt = 0.3 / orc.signal_max(U)
    xg, sq3 = 5.5 * prob.dx(0), math.sqrt(3.0)
    t = ((xg - 1.0 / 6.0 - 10.0 * dt / sq3) * sq3 - 1.0) / 20.0
    g = awe.Grid(prob)
    g.set_state(U)
    g.set_time(t)
    g.step(dt, sync=False)
    code = 0
    try:
        g.check()
    except awe.AweError as e:
        code = e.code
    Ug = g.get_state()
    g.close()
    Uo, _, rc = orc.rk_step(U, t, dt)
    assert (code != 0) == (rc != 0)
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v


def test_gate_flags_every_stage(awe):
    """Gated reconstruction with flags recomputed from each stage's state
    (smooth data: with these random weights the shocked case loses
    positivity in the oracle as well)."""
    from paper_2211_13295_gb300.gate_train import he_init
    prob, U = make(3, 4, (7, 6, 5), "smooth")
    prob = prob.replace(scheme="ssprk")
    nin, _ = awe.gate_dims(3, 4)
    params = he_init(nin, 7)
    params[-1] = -0.2
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    Ug, _ = gpu_step(awe, prob, U, dt, gate=params)
    Uo, _, rc = orc.rk_step(U, 0.0, dt, gate_params=params)
    assert rc == 0
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v
    Ufull, _, _ = orc.rk_step(U, 0.0, dt)
    assert rel_l1(Uo[0], Ufull[0]) > 1e-14       # the gate changed something


def test_slab_streaming_is_bitwise_identical(awe):
    prob = P.tgv3d(n=12, order=4).replace(scheme="ssprk")
    U = prob.initial_state()
    dt = 0.2
    a, _ = gpu_step(awe, prob, U, dt)
    b, _ = gpu_step(awe, prob, U, dt, slab=5)
    assert np.array_equal(a, b)


def test_probes_cover_ader_only(awe):
    prob, U = make(2, 3, (13, 11, 1), "smooth")
    g = awe.Grid(prob.replace(scheme="ssprk"))
    g.set_state(U)
    g.probe_modes()          # the reconstruction is shared
    with pytest.raises(awe.AweError) as e:
        g.probe_fluxes(0.01)
    assert e.value.code == awe.AWE_ERR_STATE
    g.close()


def windows_rk(prob, U0, U1, dt, centers, m):
    """The oracle's step on a window of m zones plus a margin of stages x g
    zones per side (the reach of one stage is g zones, so the margin
    isolates the m zones from the window's own boundary values)."""
    orc_full = oracle.Oracle(prob)
    s = orc_full.rk_stages()
    M = s * prob.order
    errs = []
    for c in centers:
        sl = tuple(slice(c[d] - M, c[d] + m + M) if d < prob.dim else slice(0, 1) for d in (2, 1, 0))
        win = np.ascontiguousarray(U0[(slice(None),) + sl])
        n = tuple(m + 2 * M if d < prob.dim else 1 for d in range(3))
        hi = tuple(prob.dx(d) * n[d] if d < prob.dim else 1.0 for d in range(3))
        wp = P.Problem("uniform", prob.dim, n, (0, 0, 0), hi, prob.order, gamma=prob.gamma,
                       bc=("outflow",) * 6, scheme="ssprk", rk_stages=s, riemann=prob.riemann)
        Uo, _, _ = oracle.Oracle(wp).rk_step(win, 0.0, dt)
        inner = tuple(slice(M, M + m) if d < prob.dim else slice(0, 1) for d in (2, 1, 0))
        out = tuple(slice(c[d], c[d] + m) if d < prob.dim else slice(0, 1) for d in (2, 1, 0))
        a, b = U1[(slice(None),) + out], Uo[(slice(None),) + inner]
        scale = max(np.abs(b[0]).sum(), 1e-300)
        errs.append(max(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), scale) for v in range(prob.nv)))
    return errs


@pytest.mark.parametrize("order", [3, 4])
def test_full_size_tgv_192_windows(awe, order):
    """TGV on 192^3 (the grid of Table IV's largest row), one step at full
    size; windows in the interior against the oracle."""
    prob = P.tgv3d(n=192, order=order, cfl=0.3).replace(scheme="ssprk")
    U0 = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U0)
    dt = g.cfl_dt()
    g.step(dt)
    U1 = g.get_state()
    g.close()
    centers = [[40, 60, 80], [100, 30, 150]] if order == 3 else [[60, 90, 120]]
    errs = windows_rk(prob, U0, U1, dt, centers, m=3)
    assert max(errs) <= 1e-12, errs
