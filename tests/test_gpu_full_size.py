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
    # outflow: no periodic image across the window's edge (the a posteriori
    # fallback looks for flagged neighbours there); the ghosts come from the
    # full array
    return P.Problem("uniform", prob.dim, n, (0, 0, 0), hi, prob.order, gamma=prob.gamma,
                     fallback=prob.fallback, bc=("outflow",) * 6)


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


def central_windows(prob, U0, U1, dt, centers, m, inner, flags_params=None):
    """oracle windows of m^3 active zones around each centre; only the central
    inner^3 zones are compared (the a posteriori fallback of a zone depends on
    the flags of zones up to a few faces away, which the window's edge does
    not see)"""
    g = prob.order
    N = g - 1
    Ug = ghosted_full(prob, U0, 0.0)
    errs = []
    for c0 in centers:
        c = [min(max(int(c0[d]) - m // 2, 0), prob.n[d] - m) for d in range(3)]
        win = np.ascontiguousarray(cut(Ug, prob, c, m, g))
        flags = None
        if flags_params is not None:
            ex = N + 1
            big = np.ascontiguousarray(cut(Ug, prob, c, m, g, extra=ex))
            bo = oracle.Oracle(window_problem(prob, m, extra=ex))
            fb = bo.gate_flags_ghosted(big, flags_params)
            inr = tuple(slice(ex, ex + m + 2 * g) for _ in range(3))
            flags = np.ascontiguousarray(fb[inr])
        Uo, _, rc = oracle.Oracle(window_problem(prob, m)).step_ghosted(win, dt, flags)
        o = (m - inner) // 2
        sl = [slice(c[d] + o, c[d] + o + inner) for d in range(3)]
        Ugpu = U1[:, sl[2], sl[1], sl[0]]
        errs.append(window_err(Ugpu, Uo[:, o:o + inner, o:o + inner, o:o + inner]))
    return errs


def test_blast_384_order4_gate_fallback_slabbed(awe):
    """C4, the blast on 384^3, order 4, FP64, slab-streamed (128 planes), with
    full WENO and with a gate that flags large stencil jumps (the oracle
    computes its own flags).  With the face-state fallback alone the first
    step leaves a few zones just outside the sphere with negative pressure;
    with the a posteriori fallback (fallback 2) it is physical everywhere, and
    windows centred on those zones, and on the sphere's surface, match the
    oracle's fallback-2 step."""
    n = 384
    prob1 = P.blast3d(n=n, order=4).replace(fallback=1)
    prob2 = prob1.replace(fallback=2)
    nin, _ = awe.gate_dims(3, 4)
    U0 = prob1.initial_state()
    r0 = int(0.5 * n + 0.2 * n) - 2
    surface = [[r0, n // 2, n // 2], [n // 2, r0, n // 2 - 3], [n // 2 - 2, n // 2, r0]]
    params = jump_gate(nin, 3)
    for gate in (None, params):
        U1, dt, code1 = run_one_status(awe, prob1, U0, gate=gate, slab=128)
        bad = nonphysical_zones(U1, prob1.gamma)
        assert code1 == (awe.AWE_ERR_NONPHYSICAL if len(bad) else awe.AWE_OK), (code1, len(bad))
        U2, dt2, code2 = run_one_status(awe, prob2, U0, gate=gate, slab=128)
        assert dt2 == dt and code2 == awe.AWE_OK and len(nonphysical_zones(U2, prob2.gamma)) == 0
        centers = [[int(i), int(j), int(k)] for (k, j, i) in bad[:3]] + surface
        errs = central_windows(prob2, U0, U2, dt, centers, m=12, inner=4, flags_params=gate)
        assert max(errs) <= 1e-12, (gate is not None, errs)


def test_blast_384_twenty_steps_stay_physical_and_conservative(awe):
    """C4 over 20 steps (FP64, the jump gate, the a posteriori fallback,
    128-plane slabs): status OK after every step, and the totals of mass,
    momentum and energy kept to round-off (the blast wave stays far inside
    the domain, whose boundary is uniform ambient gas at rest: zero mass and
    energy flux, opposite pressure forces)."""
    n = 384
    prob = P.blast3d(n=n, order=4).replace(fallback=2)
    nin, _ = awe.gate_dims(3, 4)
    U0 = prob.initial_state()
    g = awe.Grid(prob, gate=True, slab=128)
    g.gate_set_weights(jump_gate(nin, 3))
    g.set_state(U0)
    g.cfl_dt()
    for _ in range(20):
        g.step(0.0, sync=False)
        g.check()
    U = g.get_state()
    g.close()
    assert len(nonphysical_zones(U, prob.gamma)) == 0
    for v in range(5):
        scale = np.abs(U0[v]).sum() if v in (0, 4) else np.abs(U0[0]).sum()
        assert abs(U[v].sum() - U0[v].sum()) <= 1e-12 * scale, v


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
