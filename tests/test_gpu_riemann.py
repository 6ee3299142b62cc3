"""Parity of the corrector's other Riemann solvers (HLL, HLLEM, Rusanov; the
solvers Sec. I.1 names beside HLLC) on the GPU with the FP64 oracle: face
fluxes elementwise within 1e-10 of each variable's scale, the full step within
1e-12 relative L1, the FP32-bulk step within 1e-5, on ragged 2D and 3D grids
at orders 2-4 with smooth data and with a strong tilted jump (so that every
branch of each solver is taken)."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import CASES, make, rel_l1

pytestmark = pytest.mark.gpu

KINDS = ["hll", "hllem", "rusanov"]
SUBSET = [c for c in CASES if (c[0], c[1], c[3]) in
          {(2, 2, "shock"), (2, 4, "shock"), (3, 3, "shock"), (3, 4, "smooth"), (3, 4, "shock")}]


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dim,order,n,state", SUBSET)
def test_fluxes_and_step_match_the_oracle(awe, kind, dim, order, n, state):
    prob, U = make(dim, order, n, state)
    prob = prob.replace(riemann=kind)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    g = awe.Grid(prob)
    g.set_state(U)
    Fg = g.probe_fluxes(dt)
    Fo = orc.fluxes(U, 0.0, dt)
    for d in range(dim):
        for v in range(prob.nv):
            scale = np.abs(Fo[d][v]).max() + 1e-300
            assert np.abs(Fg[d][v] - Fo[d][v]).max() <= 1e-10 * scale, (d, v)
    dn = g.step(dt)
    Ug = g.get_state()
    g.close()
    Uo, smax, rc = orc.step(U, 0.0, dt)
    assert rc == 0
    for v in range(prob.nv):
        assert rel_l1(Ug[v], Uo[v]) <= 1e-12, v
    assert abs(dn - prob.cfl / smax) <= 1e-13 * dn
    g32 = awe.Grid(prob, prec="fp32")
    g32.set_state(U)
    g32.step(dt)
    U32 = g32.get_state()
    g32.close()
    for v in range(prob.nv):
        assert rel_l1(U32[v], Uo[v]) <= 1e-5, v


@pytest.mark.parametrize("kind", KINDS)
def test_solvers_differ_where_they_should(awe, kind):
    """Sanity of the dispatch: on the shocked 3D order-4 case each solver's
    step differs from the HLLC step (by far more than rounding)."""
    dim, order, n, state = 3, 4, (6, 7, 5), "shock"
    prob, U = make(dim, order, n, state)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    outs = {}
    for k in ("hllc", kind):
        g = awe.Grid(prob.replace(riemann=k))
        g.set_state(U)
        g.step(dt)
        outs[k] = g.get_state()
        g.close()
    assert rel_l1(outs[kind][0], outs["hllc"][0]) > 1e-8
