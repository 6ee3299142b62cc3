"""awe_cfl_dt_noalloc, the time-step entry point that allocates no device
memory (for callers that cannot call cudaMalloc when they need a dt), must
give the same dt as awe_cfl_dt, through the C ABI, on two calls in a row.
This file is collected last so that a failure here leaves every other test
already run; it passes alone in a fresh process and after the others."""
import ctypes as C

import numpy as np
import pytest

from paper_2211_13295_gb300 import problems as P


def _grid_dt(awe, prob, U, cfl):
    g = awe.Grid(prob)
    g.set_state(U)
    dt = g.cfl_dt(cfl)
    g.close()
    return dt


def _noalloc(awe, torch, Ud, prob, cfl, dt_dev):
    dx = [prob.dx(d) for d in range(prob.dim)]
    dt_dev.fill_(-1.0)
    awe.cfl_dt_noalloc(Ud, prob.dim, prob.n[:prob.dim], dx, prob.gamma, cfl, dt_dev)
    torch.cuda.synchronize()
    return float(dt_dev.item())


@pytest.mark.gpu
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
        first = _noalloc(awe, torch, Ud, prob, cfl, dt_dev)
        second = _noalloc(awe, torch, Ud, prob, cfl, dt_dev)
        assert abs(first - ref) <= 1e-14 * ref, (prob.name, first, ref)
        assert second == first, (prob.name, first, second)


@pytest.mark.gpu
def test_noalloc_signals_a_nonphysical_zone_with_dt_zero():
    import torch
    from paper_2211_13295_gb300 import awe
    prob = P.tgv3d(n=12, order=4)
    U = prob.initial_state()
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    bad = U.copy()
    bad[4, 3, 5, 7] = 0.0  # energy zero: negative pressure
    assert _noalloc(awe, torch, torch.from_numpy(bad).cuda(), prob, 0.3, dt_dev) == 0.0
    bad = U.copy()
    bad[0, 11, 0, 2] = np.nan
    assert _noalloc(awe, torch, torch.from_numpy(bad).cuda(), prob, 0.3, dt_dev) == 0.0
    # and the shared scratch keeps nothing of the bad calls
    good = _noalloc(awe, torch, torch.from_numpy(U).cuda(), prob, 0.3, dt_dev)
    assert abs(good - _grid_dt(awe, prob, U, 0.3)) <= 1e-14 * good


@pytest.mark.gpu
def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2211_13295_gb300 import awe
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    U = torch.zeros(5, dtype=torch.float64, device="cuda")
    n = (C.c_int * 3)(1024, 1024, 512)
    dx = (C.c_double * 3)(1.0, 1.0, 1.0)
    # the C entry point checks the zone count before it touches U
    rc = awe.lib().awe_cfl_dt_noalloc(C.c_void_p(U.data_ptr()), 3, n, dx, 1.4, 0.3,
                                      C.c_void_p(dt_dev.data_ptr()), None)
    assert rc == awe.AWE_ERR_ARG
    assert b"no-allocation limit" in awe.lib().awe_last_error(None)


def test_noalloc_wrapper_checks_its_buffers_before_the_library():
    """The binding is the only guard of the buffers' extent; these cases must be
    refused on the host (no CUDA device or library call is needed for that)."""
    import torch
    from paper_2211_13295_gb300 import awe
    cpu_state = torch.zeros(5 * 8 * 8 * 8, dtype=torch.float64)
    cpu_dt = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="float64 CUDA tensor"):
        awe.cfl_dt_noalloc(cpu_state, 3, (8, 8, 8), (0.1, 0.1, 0.1), 1.4, 0.3, cpu_dt)
    with pytest.raises(ValueError, match="dim"):
        awe.cfl_dt_noalloc(cpu_state, 3, (8, 8, 8, 1), (0.1, 0.1, 0.1), 1.4, 0.3, cpu_dt)
    with pytest.raises(ValueError, match="dim"):
        awe.cfl_dt_noalloc(cpu_state, 3, (8, 8), (0.1, 0.1), 1.4, 0.3, cpu_dt)
    with pytest.raises(ValueError, match="float64 CUDA tensor"):
        awe.cfl_dt_noalloc(cpu_state.float(), 3, (8, 8, 8), (0.1, 0.1, 0.1), 1.4, 0.3, cpu_dt)


@pytest.mark.gpu
def test_noalloc_wrapper_rejects_a_short_state_on_the_gpu():
    import torch
    from paper_2211_13295_gb300 import awe
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    short = torch.zeros(5 * 8 * 8 * 8 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="elements"):
        awe.cfl_dt_noalloc(short, 3, (8, 8, 8), (0.1, 0.1, 0.1), 1.4, 0.3, dt_dev)
    strided = torch.zeros(2 * 5 * 8 * 8 * 8, dtype=torch.float64, device="cuda")[::2]
    with pytest.raises(ValueError, match="contiguous"):
        awe.cfl_dt_noalloc(strided, 3, (8, 8, 8), (0.1, 0.1, 0.1), 1.4, 0.3, dt_dev)
