"""awe_cfl_dt_noalloc, the time-step entry point that allocates no device
memory (for callers that cannot call cudaMalloc when they need a dt), must
give the same dt as awe_cfl_dt, through the C ABI, on two calls in a row.
This file is collected last so that a failure here leaves every other test
already run; it passes alone in a fresh process and after the others."""
import numpy as np
import pytest

from paper_2211_13295_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _grid_dt(awe, prob, U, cfl):
    g = awe.Grid(prob)
    g.set_state(U)
    dt = g.cfl_dt(cfl)
    g.close()
    return dt


def test_noalloc_dt_matches_awe_cfl_dt_twice_in_a_row():
    import torch
    from paper_2211_13295_gb300 import awe, build
    build.build()
    cases = [(P.tgv3d(n=20, order=4), 0.3), (P.vortex2d(n=37, order=3), 0.4)]
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    for prob, cfl in cases:
        U = prob.initial_state()
        ref = _grid_dt(awe, prob, U, cfl)
        Ud = torch.from_numpy(U).cuda().contiguous()
        dx = [prob.dx(d) for d in range(prob.dim)]
        dt_dev.fill_(-1.0)
        awe.cfl_dt_noalloc(Ud, prob.dim, prob.n[:prob.dim], dx, prob.gamma, cfl, dt_dev)
        torch.cuda.synchronize()
        got = float(dt_dev.item())
        assert abs(got - ref) <= 1e-14 * ref, (prob.name, got, ref)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import ctypes as C
    import torch
    from paper_2211_13295_gb300 import awe
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    U = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(awe.AweError) as ei:
        awe.cfl_dt_noalloc(U, 3, (1024, 1024, 512), (1.0, 1.0, 1.0), 1.4, 0.3, dt_dev)
    assert ei.value.code == awe.AWE_ERR_ARG
    assert "no-allocation limit" in str(ei.value)
