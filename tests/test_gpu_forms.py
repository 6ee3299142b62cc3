"""The FP32-bulk form keeps the design order: on the isentropic vortex
(order 3, to t = 0.5) its error against the exact solution stays within 2% of
the FP64 form's at 64^2 and 128^2 (FP32 rounding, ~1e-7 relative, lies far
below the truncation error) and converges at rate > 2.5; the order-2 scheme
keeps its rate in FP32 as well.  (The gated forms' order is checked with the
trained gate in test_gpu_gate.py.)"""
import numpy as np
import pytest

from paper_2211_13295_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awe():
    from paper_2211_13295_gb300 import awe as A
    from paper_2211_13295_gb300 import build
    build.build()
    return A


def run(awe, prob, prec, t_end):
    g = awe.Grid(prob, prec=prec)
    g.set_state(prob.initial_state())
    t, dt = 0.0, g.cfl_dt()
    while t < t_end - 1e-12:
        dt = min(dt, t_end - t)
        dn = g.step(dt)
        t += dt
        dt = dn
    U = g.get_state()
    g.close()
    return np.abs(U[0] - P.vortex_exact(prob, t_end)[0]).mean(), np.abs(U[0] - P.vortex_exact(prob, t_end)[0]).max()


@pytest.mark.parametrize("order,ns,min_rate", [(3, (64, 128), 2.5), (2, (64, 128), 1.6)])
def test_fp32_form_keeps_the_order(awe, order, ns, min_rate):
    errs = {}
    for n in ns:
        prob = P.vortex2d(n=n, order=order, t_end=0.5)
        for prec in ("fp64", "fp32"):
            errs[(n, prec)] = run(awe, prob, prec, 0.5)
    for n in ns:
        l1_64, linf_64 = errs[(n, "fp64")]
        l1_32, linf_32 = errs[(n, "fp32")]
        assert abs(l1_32 - l1_64) <= 0.02 * l1_64, errs
        assert abs(linf_32 - linf_64) <= 0.02 * linf_64, errs
    rate = np.log2(errs[(ns[0], "fp32")][0] / errs[(ns[1], "fp32")][0])
    assert rate > min_rate, (rate, errs)
