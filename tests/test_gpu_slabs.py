"""Slab decomposition on one GPU (paper Sec. II.2 and Sec. V: one ghost
exchange per step and one MIN of dt over the patches): a grid split along its
outermost dimension into subdomains whose facing ghost planes are exchanged
through the library's halo pack/unpack kernels must step exactly like the
undivided grid, bit for bit, for ADER (one exchange per step) and the
Runge-Kutta variant (one per stage), periodic and non-periodic ends, FP64 and
FP32-bulk forms, in 3D (z slabs) and 2D (y slabs, the double Mach reflection
with its wall and moving-shock boundaries), with uneven slab sizes."""
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


def run_both(awe, prob, U, parts, steps, prec="fp64"):
    from paper_2211_13295_gb300 import slabs
    g = awe.Grid(prob, prec=prec)
    g.set_state(U)
    g.cfl_dt()
    sg = slabs.SlabGrid(prob, parts, prec=prec)
    sg.set_state(U)
    sg.cfl_dt()
    assert sg.subs[0].get_dt() == g.get_dt()
    for _ in range(steps):
        g.step(0.0, sync=False)
        sg.step(0.0, sync=False)
    g.check()
    sg.check()
    a, b = g.get_state(), sg.get_state()
    da, db = g.get_dt(), sg.subs[-1].get_dt()
    ta, tb = g.time(), sg.subs[0].time()
    g.close()
    sg.close()
    return a, b, (da, db), (ta, tb)


CASES = [
    # (dim, order, n, state, bc, parts, scheme, prec)
    (3, 4, (7, 6, 13), "shock", "periodic", 2, "ader", "fp64"),
    (3, 4, (6, 7, 13), "smooth", "outflow", 3, "ader", "fp64"),
    (3, 3, (9, 7, 10), "shock", "periodic", 3, "ader", "fp64"),
    (3, 3, (9, 7, 7), "smooth", "reflect", 2, "ader", "fp64"),
    (3, 2, (9, 7, 8), "shock", "periodic", 2, "ader", "fp64"),
    (3, 4, (7, 6, 12), "smooth", "periodic", 2, "ader", "fp32"),
    (3, 3, (9, 7, 10), "smooth", "periodic", 2, "ssprk", "fp64"),
    (3, 4, (6, 5, 9), "shock", "outflow", 2, "ssprk", "fp64"),
    (2, 3, (13, 11, 1), "shock", "periodic", 2, "ader", "fp64"),
    (2, 4, (12, 13, 1), "smooth", "outflow", 3, "ssprk", "fp64"),
]


@pytest.mark.parametrize("dim,order,n,state,bc,parts,scheme,prec", CASES)
def test_slab_decomposition_equals_the_undivided_grid(awe, dim, order, n, state, bc, parts, scheme, prec):
    prob, U = make(dim, order, n, state, bc=bc)
    prob = prob.replace(scheme=scheme)
    a, b, dts, ts = run_both(awe, prob, U, parts, steps=3, prec=prec)
    assert np.array_equal(a, b), np.abs(a - b).max()
    assert dts[0] == dts[1] and ts[0] == ts[1]


def test_slab_decomposition_of_the_double_mach_reflection(awe):
    """2D, split along y: the bottom (wall / post-shock) and top (moving shock)
    boundaries stay with the first and last slab; the positivity fallback
    decides per zone from stencils that the ghost planes cover."""
    prob = P.dmr(nx=96, ny=24, order=3).replace(fallback=True)
    U = prob.initial_state()
    for prec in ("fp64", "fp32"):
        a, b, dts, ts = run_both(awe, prob, U, 3, steps=4, prec=prec)
        assert np.array_equal(a, b), (prec, np.abs(a - b).max())
        assert dts[0] == dts[1]


def test_subdomain_contract(awe):
    """exchanged faces only on the outermost dimension; no gate with them; a
    multi-stage grid with exchanged faces must be stepped stage by stage;
    stages run in order; halo buffers have the documented size"""
    prob, U = make(3, 3, (9, 7, 8), "smooth")
    bad = prob.replace(bc=("exchange", "exchange") + ("periodic",) * 4)
    with pytest.raises(awe.AweError) as e:
        awe.Grid(bad)
    assert e.value.code == awe.AWE_ERR_ARG
    sub = prob.replace(bc=("periodic",) * 4 + ("exchange", "exchange"))
    with pytest.raises(awe.AweError) as e:
        awe.Grid(sub, gate=True)
    assert e.value.code == awe.AWE_ERR_ARG
    g = awe.Grid(sub.replace(scheme="ssprk"))
    assert g.stage_count() == 3
    assert g.halo_size() == 5 * 3 * (9 + 6) * (7 + 6)
    with pytest.raises(awe.AweError) as e:
        g.step(1e-3)
    assert e.value.code == awe.AWE_ERR_STATE
    with pytest.raises(awe.AweError) as e:
        g.stage(1, 1e-3)
    assert e.value.code == awe.AWE_ERR_STATE
    # the binding refuses buffers the C entry points would overrun
    with pytest.raises(ValueError):
        g.halo_pack(0, np.zeros(g.halo_size() - 1))
    with pytest.raises(ValueError):
        g.halo_unpack(1, np.zeros(g.halo_size(), dtype=np.float32))
    g.close()


def test_halo_buffers_by_hand(awe):
    """pack into a host buffer: the planes next to each face with their inner
    ghost zones (periodic in x and y), planes in increasing z"""
    prob, U = make(3, 3, (5, 4, 6), "smooth")
    sub = prob.replace(bc=("periodic",) * 4 + ("exchange", "exchange"))
    g = awe.Grid(sub)
    g.set_state(U)
    m = g.halo_size()
    lo, hi = np.zeros(m), np.zeros(m)
    g.halo_pack(0, lo)
    g.halo_pack(1, hi)
    gw = 3
    lo = lo.reshape(5, gw, 4 + 2 * gw, 5 + 2 * gw)
    hi = hi.reshape(5, gw, 4 + 2 * gw, 5 + 2 * gw)
    # inner ghosts are the periodic images of the active zones
    ext = np.pad(U, ((0, 0), (0, 0), (gw, gw), (gw, gw)), mode="wrap")
    assert np.array_equal(lo, ext[:, :gw])
    assert np.array_equal(hi, ext[:, -gw:])
    g.close()


@pytest.mark.parametrize("bc,scheme", [("periodic", "ader"), ("outflow", "ader"), ("periodic", "ssprk")])
def test_distributed_slab_grid_on_one_rank(awe, bc, scheme):
    """slabs.DistSlabGrid with a single rank: the path the multi-GPU bench runs
    (device halo buffers, the exchange object -- a periodic self-exchange here
    -- the stage loop, the device-resident dt through get_dt/set_dt) must step
    exactly like the plain grid."""
    from paper_2211_13295_gb300 import slabs
    prob, U = make(3, 4, (7, 6, 9), "shock", bc=bc)
    prob = prob.replace(scheme=scheme)
    g = awe.Grid(prob)
    g.set_state(U)
    g.cfl_dt()
    d = slabs.DistSlabGrid(prob, 0, 1)
    d.set_state(d.local(U))
    d.cfl_dt()
    for _ in range(3):
        g.step(0.0, sync=False)
        d.step(0.0)
    g.check()
    d.check()
    assert np.array_equal(g.get_state(), d.get_state())
    assert g.get_dt() == d.sub.get_dt()
    g.close()
    d.close()
