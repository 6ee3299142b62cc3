"""Full-size parity: each workload configuration runs at its full size on the
GPU, in the launch configuration bench.py uses; the FP64 oracle then
recomputes sampled windows of the result one by one (a window of m^3 zones
plus its ghost frame cut from the full input state has exactly the inputs
those zones depend on).  Errors are relative L1 per variable, normalised by
max(sum|U_v|, sum|rho|) over the window (momentum components can start at
zero, e.g. rho*w in the Taylor-Green vortex)."""
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


def window_err(a, b):
    scale = max(np.abs(b[0]).sum(), 1e-300)
    return max(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), scale) for v in range(b.shape[0]))


def ghosted_full(prob, U, t):
    return oracle.Oracle(prob).ghosted(U, t)


def cut(Ug, prob, c, m, g, extra=0):
    """window of the ghosted full array around active zone corner c"""
    sl = []
    for d in range(3):
        if d < prob.dim:
            lo = c[d] - extra
            sl.append(slice(lo, lo + m + 2 * g + 2 * extra))   # ghosted index = active + g
        else:
            sl.append(slice(0, 1))
    return Ug[:, sl[2], sl[1], sl[0]]


def window_problem(prob, m, extra=0):
    n = tuple((m + 2 * extra) if d < prob.dim else 1 for d in range(3))
    hi = tuple(prob.dx(d) * n[d] if d < prob.dim else 1.0 for d in range(3))
    return P.Problem("uniform", prob.dim, n, (0, 0, 0), hi, prob.order, gamma=prob.gamma,
                     fallback=prob.fallback)


def sampled_windows(prob, U0, U1, dt, t, nwin, m, seed, flags_params=None, centers=None):
    g = prob.order
    N = g - 1
    Ug = ghosted_full(prob, U0, t)
    rng = np.random.default_rng(seed)
    errs = []
    for w in range(nwin):
        if centers is not None:
            c = centers[w]
        else:
            c = [int(rng.integers(0, prob.n[d] - m + 1)) if d < prob.dim else 0 for d in range(3)]
        win = np.ascontiguousarray(cut(Ug, prob, c, m, g))
        wp = window_problem(prob, m)
        wo = oracle.Oracle(wp)
        flags = None
        if flags_params is not None:
            # gate flags from a wider window so that every feature stencil of
            # the window's zones and their face neighbours is complete
            ex = N + 1
            big = np.ascontiguousarray(cut(Ug, prob, c, m, g, extra=ex))
            bp = window_problem(prob, m, extra=ex)
            bo = oracle.Oracle(bp)
            fb = bo.gate_flags_ghosted(big, flags_params)
            inner = tuple(slice(ex, ex + m + 2 * g) if d < prob.dim else slice(0, 1) for d in (2, 1, 0))
            flags = np.ascontiguousarray(fb[inner])
        Uo, _, rc = wo.step_ghosted(win, dt, flags)
        sl = [slice(c[d], c[d] + m) if d < prob.dim else slice(0, 1) for d in range(3)]
        Ugpu = U1[:, sl[2], sl[1], sl[0]]
        errs.append(window_err(Ugpu, Uo))
    return errs


def run_one(awe, prob, U0, prec="fp64", gate=None, slab=0):
    g = awe.Grid(prob, prec=prec, gate=gate is not None, slab=slab)
    if gate is not None:
        g.gate_set_weights(gate)
    g.set_state(U0)
    dt = g.cfl_dt()
    g.step(dt)
    U1 = g.get_state()
    g.close()
    return U1, dt


def test_tgv_256_order4_fp64_windows(awe):
    """The headline workload in the bench's configuration."""
    prob = P.tgv3d(n=256, order=4, cfl=0.3)
    U0 = prob.initial_state()
    U1, dt = run_one(awe, prob, U0)
    errs = sampled_windows(prob, U0, U1, dt, 0.0, nwin=4, m=4, seed=1)
    assert max(errs) <= 1e-12, errs


def test_vortex_64_order3_fp64_full_run(awe):
    """C1 in full: isentropic vortex 64^2, order 3, CFL 0.4, to t = 1, against
    the oracle's full run (same dt sequence) and the exact solution."""
    prob = P.vortex2d(n=64, order=3)
    U = prob.initial_state()
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    t, dt = 0.0, orc.cfl_dt(U, prob.cfl)
    while t < 1.0 - 1e-12:
        dt = min(dt, 1.0 - t)
        g.step(dt)
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        dt = prob.cfl / smax
    Ug = g.get_state()
    assert window_err(Ug, U) <= 1e-11
    ex = P.vortex_exact(prob, 1.0)[0]
    assert np.abs(Ug[0] - ex).mean() < 1.2e-4  # oracle: 9.09e-5


def test_dmr_4096x1024_fallback(awe):
    """DMR at full size with the positivity fallback: FP64 windows at the
    shock and the wall within 1e-12; the FP32-bulk form within 1e-5."""
    prob = P.dmr(nx=4096, ny=1024).replace(fallback=True)
    U0 = prob.initial_state()
    U1, dt = run_one(awe, prob, U0)
    # windows straddling the initial shock (x = 1/6 + y/sqrt(3)) and the wall
    xs = lambda j: int((1.0 / 6.0 + (j + 0.5) / 1024 / np.sqrt(3.0)) * 1024)
    centers = [[xs(0) - 2, 0, 0], [xs(500) - 3, 500, 0], [xs(1000) - 2, 1000, 0], [3000, 700, 0]]
    errs = sampled_windows(prob, U0, U1, dt, 0.0, nwin=4, m=6, seed=2, centers=centers)
    assert max(errs) <= 1e-12, errs
    U1f, dtf = run_one(awe, prob, U0, prec="fp32")
    assert abs(dtf - dt) <= 1e-15 * dt
    errs32 = sampled_windows(prob, U0, U1f, dt, 0.0, nwin=4, m=6, seed=2, centers=centers)
    assert max(errs32) <= 1e-5, errs32


def jump_gate(nin, N, thresh=0.5):
    """A hand-set gate: logit = 10*relu(sum of the magnitude features - thresh)
    - 0.01, i.e. troubled where the stencil differences are large relative to
    the zone value (the magnitude feature is (x/(1+x)), x = 100*max|diff|/|f|)."""
    from paper_2211_13295_gb300.gate_train import he_init
    H = 32
    p = np.zeros_like(he_init(nin, 0))
    W1 = p[:H * nin].reshape(H, nin)
    for k in range(nin // (2 * N + 1)):
        W1[0, k * (2 * N + 1) + 2 * N] = 1.0
    o = H * nin
    p[o] = -thresh                     # b1[0]
    o += H
    W2 = p[o:o + H * H].reshape(H, H)
    W2[0, 0] = 1.0
    o += H * H + H                     # skip b2
    p[o] = 10.0                        # w3[0]
    p[o + H] = -0.01                   # b3
    return p


def run_one_status(awe, prob, U0, gate=None, slab=0):
    """run_one that tolerates the non-physical status: returns (U1, dt, code)"""
    g = awe.Grid(prob, gate=gate is not None, slab=slab)
    if gate is not None:
        g.gate_set_weights(gate)
    g.set_state(U0)
    dt = g.cfl_dt()
    g.step(dt, sync=False)
    code = 0
    try:
        g.check()
    except awe.AweError as e:
        code = e.code
    U1 = g.get_state()
    g.close()
    return U1, dt, code


def nonphysical_zones(U, gamma):
    rho = U[0]
    with np.errstate(all="ignore"):
        p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho)
        return np.argwhere(~((rho > 0) & (p > 0) & np.isfinite(p)))


def test_blast_384_order4_gate_fallback_slabbed(awe):
    """Blast on 384^3, order 4, FP64 with the positivity fallback,
    slab-streamed (128 planes), first with full WENO, then with a gate that
    flags large stencil jumps (the oracle computes its own flags).

    At this size the first step leaves a few zones just outside the sphere's
    surface with negative pressure, in the oracle as on the GPU: the fallback
    keeps the face states and hence the Riemann problems physical, not the
    updated means.  The test therefore checks (a) that the GPU reports the
    non-physical status exactly when its state holds such zones, (b) windows
    around those zones against the oracle (same values, so the oracle finds
    the same zones non-physical), and (c) windows on the sphere's surface."""
    prob = P.blast3d(n=384, order=4).replace(fallback=True)
    nin, _ = awe.gate_dims(3, 4)
    U0 = prob.initial_state()
    n = 384
    r0 = int(0.5 * n + 0.2 * n) - 2
    surface = [[r0, n // 2, n // 2], [n // 2, r0, n // 2 - 3], [n // 2 - 2, n // 2, r0], [100, 120, 140]]
    params = jump_gate(nin, 3)
    for gate in (None, params):
        U1, dt, code = run_one_status(awe, prob, U0, gate=gate, slab=128)
        bad = nonphysical_zones(U1, prob.gamma)
        assert code == (awe.AWE_ERR_NONPHYSICAL if len(bad) else awe.AWE_OK), (code, len(bad))
        centers = [[min(max(int(i) - 1, 0), n - 4), min(max(int(j) - 1, 0), n - 4), min(max(int(k) - 1, 0), n - 4)]
                   for (k, j, i) in bad[:3]] + surface
        errs = sampled_windows(prob, U0, U1, dt, 0.0, nwin=len(centers), m=4, seed=3,
                               flags_params=gate, centers=centers)
        assert max(errs) <= 1e-12, (gate is not None, errs)


def test_kh_512_order4_fp32_gate_slabbed(awe):
    """Kelvin-Helmholtz on 512^3, order 4, FP32 bulk with the gate,
    slab-streamed (64 planes): windows within the FP32 tolerance of the FP64
    oracle (with its own flags)."""
    from paper_2211_13295_gb300.gate_train import he_init
    prob = P.kh3d(n=512, order=4)
    nin, _ = awe.gate_dims(3, 4)
    params = he_init(nin, 12)
    params[-1] = -0.3
    U0 = prob.initial_state()
    U1, dt = run_one(awe, prob, U0, prec="fp32", gate=params, slab=64)
    n = 512
    centers = [[10, n // 4 - 2, 30], [200, 3 * n // 4 - 2, 400], [300, n // 2, 100], [n - 10, n - 10, n - 10]]
    errs = sampled_windows(prob, U0, U1, dt, 0.0, nwin=4, m=4, seed=4, flags_params=params, centers=centers)
    assert max(errs) <= 1e-5, errs
