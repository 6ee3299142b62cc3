"""No stage reads an intermediate element that the earlier stages of the
same slab did not write: with AWE_POISON=1 the library fills every
intermediate buffer (mode fields, modes, face states, fluxes) and the
output and stage states with NaN bit patterns before use, and two steps must
still be bit-for-bit those of a plain grid, for every order, dimension,
scheme, precision, slab split, the gate and the positivity fallback."""
import numpy as np
import pytest

from paper_2211_13295_gb300 import problems as P
from test_gpu_parity import make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


def two_steps(awe, prob, U, monkeypatch, poison, **kw):
    monkeypatch.setenv("AWE_POISON", "1" if poison else "0")
    gate = kw.pop("gate", None)
    g = awe.Grid(prob, gate=gate is not None, **kw)
    if gate is not None:
        g.gate_set_weights(gate)
    g.set_state(U)
    g.cfl_dt()
    g.step(0.0, sync=False)
    dn = g.step(0.0)
    out = g.get_state()
    g.close()
    return out, dn


CASES = [(2, 2, (13, 11, 1)), (2, 3, (13, 11, 1)), (2, 4, (12, 9, 1)),
         (3, 2, (9, 7, 6)), (3, 3, (9, 7, 6)), (3, 4, (7, 6, 5))]


@pytest.mark.parametrize("scheme", ["ader", "ssprk"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,order,n", CASES)
def test_poisoned_intermediates_change_nothing(awe, monkeypatch, dim, order, n, prec, scheme):
    prob, U = make(dim, order, n, "smooth")
    prob = prob.replace(scheme=scheme)
    slab = 2 if dim == 3 else 0
    a, da = two_steps(awe, prob, U, monkeypatch, False, prec=prec, slab=slab)
    b, db = two_steps(awe, prob, U, monkeypatch, True, prec=prec, slab=slab)
    assert np.isfinite(a).all()
    assert np.array_equal(a, b) and da == db


def test_poisoned_gate_and_fallback(awe, monkeypatch):
    from paper_2211_13295_gb300.gate_train import he_init
    prob, U = make(3, 4, (7, 6, 5), "smooth")
    nin, _ = awe.gate_dims(3, 4)
    params = he_init(nin, 5)
    a, _ = two_steps(awe, prob, U, monkeypatch, False, gate=params, slab=2)
    b, _ = two_steps(awe, prob, U, monkeypatch, True, gate=params, slab=2)
    assert np.array_equal(a, b)
    prob = P.dmr(nx=48, ny=12, order=3).replace(fallback=True)
    U = prob.initial_state()
    out = []
    for poison in (False, True):
        monkeypatch.setenv("AWE_POISON", "1" if poison else "0")
        g = awe.Grid(prob)
        g.set_state(U)
        g.step(g.cfl_dt(), sync=False)
        out.append(g.get_state())
        g.close()
    assert np.array_equal(out[0], out[1])
