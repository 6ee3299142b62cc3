"""Host buffers of awe_set_state / awe_get_state: a page-locked buffer is read
and written directly by the scatter and gather kernels, pageable memory goes
through the staging copy; both routes must move the state bit for bit, on
ragged 2D and 3D grids, and a step started from either must agree exactly."""
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


CASES = {
    "vortex2d_37_o3": lambda: (P.vortex2d(n=37, order=3), P.vortex2d(n=37, order=3).initial_state()),
    "shock3d_7x6x5_o4": lambda: make(3, 4, (7, 6, 5), "shock"),
    "smooth3d_9x7x6_o3": lambda: make(3, 3, (9, 7, 6), "smooth"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_pinned_and_pageable_routes_agree_bitwise(awe, case):
    import torch
    prob, U = CASES[case]()
    U = np.ascontiguousarray(U, dtype=np.float64)
    pinned = torch.from_numpy(U.copy()).pin_memory()
    out_pinned = torch.zeros_like(pinned).pin_memory()
    out_pageable = np.zeros_like(U)
    results = []
    for route in ("pinned", "pageable"):
        g = awe.Grid(prob)
        g.set_state(pinned.numpy() if route == "pinned" else U.copy())
        if route == "pinned":
            g.get_state(out_pinned.numpy())
            assert np.array_equal(out_pinned.numpy(), U)
        else:
            g.get_state(out_pageable)
            assert np.array_equal(out_pageable, U)
        dt = g.cfl_dt()
        g.step(dt)
        if route == "pinned":
            out_pinned.zero_()
            g.get_state(out_pinned.numpy())
            results.append(out_pinned.numpy().copy())
        else:
            results.append(g.get_state())
        g.close()
    assert np.array_equal(results[0], results[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_large_fresh_pageable_buffers_read_the_grid_state(awe, prec):
    """States of tens of MB land in fresh anonymous mappings (np.zeros), which
    this platform's pointer attributes report as host memory although CUDA did
    not page-lock them: such a buffer must take the staging copy and read the
    grid's own state, equal to the page-locked and the touched-pageable reads,
    and different between the FP64 and FP32 forms after a step."""
    import torch
    prob = P.tgv3d(n=64, order=4, cfl=0.3)
    Uh = torch.from_numpy(prob.initial_state()).pin_memory()
    reads = {}
    for form in ("fp64", prec):
        g = awe.Grid(prob, prec=form)
        g.set_state(Uh.numpy())
        g.step(g.cfl_dt())
        fresh = g.get_state()                     # np.zeros: a fresh mapping
        touched = np.full(fresh.shape, 7.0)
        g.get_state(touched)
        pinned = torch.empty_like(Uh).pin_memory()
        g.get_state(pinned.numpy())
        g.close()
        assert np.array_equal(fresh, touched)
        assert np.array_equal(fresh, pinned.numpy())
        assert np.abs(fresh - Uh.numpy()).max() > 1e-6    # the step changed the state
        reads[form] = fresh
    if prec == "fp32":
        d = np.abs(reads["fp32"] - reads["fp64"]).max()
        assert 0 < d < 1e-3


def test_partly_registered_buffers_are_never_read_directly(awe):
    """A host buffer page-locked over only its first pages (cudaHostRegister of
    a prefix) must not be read or written by the scatter/gather kernels (both
    ends of the buffer are checked).  The staged copy of such a range is
    refused by CUDA itself (invalid argument): the call must either move the
    state bit for bit or fail with AWE_ERR_CUDA, and the grid must stay
    usable either way."""
    import torch
    cudart = torch.cuda.cudart()
    prob = P.tgv3d(n=32, order=4, cfl=0.3)
    U = np.ascontiguousarray(prob.initial_state())
    prefix = 1 << 16  # 64 KB of a 1.3 MB state
    src = np.empty_like(U)
    src[...] = U
    dst = np.full_like(U, 7.0)
    g = awe.Grid(prob)
    regs = []
    try:
        for buf in (src, dst):
            assert int(cudart.cudaHostRegister(buf.ctypes.data, prefix, 0)) == 0
            regs.append(buf)
        for call, args in ((g.set_state, (src,)), (g.get_state, (dst,))):
            try:
                call(*args)
            except awe.AweError as e:
                assert e.code == awe.AWE_ERR_CUDA, e
        if not np.array_equal(dst, np.full_like(U, 7.0)):
            assert np.array_equal(dst, U)  # a transfer that happened was exact
    finally:
        for buf in regs:
            cudart.cudaHostUnregister(buf.ctypes.data)
    # the grid works on after the refused copies
    g.set_state(U)
    dt = g.cfl_dt()
    g.step(dt)
    a = g.get_state()
    g.close()
    h = awe.Grid(prob)
    h.set_state(U)
    h.step(dt)
    assert np.array_equal(a, h.get_state())
    h.close()
