"""The a posteriori positivity fallback on the GPU (awe_config.fallback = 2;
not in the paper): on seeded rough states that the face-state fallback alone
leaves with negative pressure, one step must equal the oracle's (fallback 2)
within the FP64 bar, report a physical state, conserve on the periodic grid,
give the same result with slab streaming, and keep the FP32-bulk form
physical.  The configurations it is not defined for are refused."""
import numpy as np
import pytest

import oracle
from paper_2211_13295_gb300 import problems as P
from test_oracle_fallback import CASES, case, physical

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


def gpu_step(awe, prob, U, dt, prec="fp64", slab=0):
    g = awe.Grid(prob, prec=prec, slab=slab)
    g.set_state(U)
    g.step(dt, sync=False)
    code = 0
    try:
        g.check()
    except awe.AweError as e:
        code = e.code
    out = g.get_state()
    dtn = g.get_dt()
    g.close()
    return out, code, dtn


@pytest.mark.parametrize("dim,n,seed", CASES)
def test_a_posteriori_fallback_matches_the_oracle(awe, dim, n, seed):
    prob, U, dt = case(dim, n, seed)
    _, code1, _ = gpu_step(awe, prob, U, dt)
    assert code1 == awe.AWE_ERR_NONPHYSICAL
    p2 = prob.replace(fallback=2)
    Ug, code, dtn = gpu_step(awe, p2, U, dt)
    Uo, smax, rc = oracle.Oracle(p2).step(U, 0.0, dt)
    assert code == awe.AWE_OK and rc == 0 and physical(Ug, dim).all()
    sc = np.abs(Uo[0]).sum()
    for v in range(prob.nv):
        err = np.abs(Ug[v] - Uo[v]).sum() / max(np.abs(Uo[v]).sum(), sc)
        assert err <= 1e-12, (v, err)
        assert abs(Ug[v].sum() - U[v].sum()) <= 1e-13 * np.abs(U[v]).sum()
    # the next dt comes from the final state
    assert abs(dtn - prob.cfl / smax) <= 1e-13 * dtn
    if dim == 3:
        Us, code_s, _ = gpu_step(awe, p2, U, dt, slab=2)
        assert code_s == awe.AWE_OK and np.array_equal(Us, Ug)
    U32, code32, _ = gpu_step(awe, p2, U, dt, prec="fp32")
    assert code32 == awe.AWE_OK and physical(U32, dim).all()
    for v in range(prob.nv):
        assert abs(U32[v].sum() - U[v].sum()) <= 1e-12 * np.abs(U[v]).sum()


def test_a_posteriori_fallback_is_refused_where_undefined(awe):
    prob, U, dt = case(3, (6, 5, 4), 92)
    with pytest.raises(awe.AweError) as e:
        awe.Grid(prob.replace(fallback=2, scheme="ssprk"))
    assert e.value.code == awe.AWE_ERR_ARG
    sub = prob.replace(fallback=2, bc=("periodic",) * 4 + ("exchange", "exchange"))
    with pytest.raises(awe.AweError) as e:
        awe.Grid(sub)
    assert e.value.code == awe.AWE_ERR_ARG
    with pytest.raises(awe.AweError) as e:
        awe.Grid(prob.replace(fallback=3))
    assert e.value.code == awe.AWE_ERR_ARG
