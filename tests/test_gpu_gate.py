"""The learned troubled-zone gate on the GPU against the oracle: features and
flags bitwise, labels, the FP32 decision forward bitwise, gradients against
the FP64 oracle, deterministic training, the gated step against the oracle's
gated step, and what the trained gate gains over full WENO."""
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


def shocky(prob, seed=4, jr=2.0, jp=3.0):
    rng = np.random.default_rng(seed)
    sh = prob.shape()
    idx = np.meshgrid(*[np.arange(n) for n in sh[1:]], indexing="ij")
    f = lambda: sum(np.sin(2 * np.pi * (x + 0.5) / n + rng.uniform(0, 6)) for x, n in zip(idx, sh[1:]))
    rho = 1.0 + 0.05 * f()
    vel = [0.2 * f() for _ in range(prob.dim)]
    p = 1.0 + 0.05 * f()
    plane = sum((0.6 + 0.2 * d) * x / n for d, (x, n) in enumerate(zip(idx, sh[1:]))) < 0.8
    rho = np.where(plane, jr * rho, rho)
    p = np.where(plane, jp * p, p)
    c = P.conserved(1.4, rho, vel, p)
    U = np.zeros(sh)
    for v in range(prob.nv):
        U[v] = c[v]
    return U


CASES = [(2, 3, (14, 11, 1)), (3, 4, (7, 6, 5))]


def random_params(nin, seed):
    from paper_2211_13295_gb300.gate_train import he_init
    p = he_init(nin, seed)
    p[-1] = -0.5
    return p


@pytest.mark.parametrize("dim,order,n", CASES)
def test_features_labels_flags_match_the_oracle(awe, dim, order, n):
    prob = P.Problem("uniform", dim, n, (0, 0, 0), (1.0, 1.2, 0.9), order)
    U = shocky(prob)
    g = awe.Grid(prob)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    Fg = g.gate_features()
    Fo = orc.features(U, 0.0)
    assert np.array_equal(Fg.reshape(Fo.shape), Fo)
    Lg = g.gate_labels(0.1)
    Lo = orc.labels(U, 0.0, 0.1)
    assert np.array_equal(Lg.reshape(Lo.shape), Lo)
    assert 0 < (Lo == 1).sum()
    nin, npar = awe.gate_dims(dim, order)
    params = random_params(nin, 7)
    g.gate_set_weights(params)
    Gg = g.gate_flags()
    Go = orc.gate_flags(U, 0.0, params)
    assert np.array_equal(Gg.reshape(Go.shape), Go)
    assert 0 < Go.sum() < Go.size


def test_mlp_forward_bitwise_and_gradient_vs_fp64(awe):
    import torch
    rng = np.random.default_rng(3)
    nin = 36
    params = random_params(nin, 11)
    X = rng.uniform(-1, 1, size=(1000, nin)).astype(np.float32)
    y = (rng.uniform(size=1000) < 0.3).astype(np.float32)
    z = torch.empty(1000, dtype=torch.float32, device="cuda")
    awe.mlp_forward(nin, torch.from_numpy(params).cuda(), torch.from_numpy(X).cuda(), z)
    assert np.array_equal(z.cpu().numpy(), oracle.mlp_forward_f32(params, X))
    grad = torch.empty(params.size, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    awe.mlp_loss_grad(nin, torch.from_numpy(params).cuda(), torch.from_numpy(X).cuda(),
                      torch.from_numpy(y).cuda(), grad, loss)
    lo, go = oracle.mlp_loss_grad_f64(params, X, y)
    gg = grad.cpu().numpy()
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    assert np.abs(gg - go).max() <= 1e-5 * np.abs(go).max()


def test_training_is_deterministic_and_learns(awe):
    from paper_2211_13295_gb300 import gate_train as T
    probs = [P.vortex2d(n=64, order=3), P.sod(nx=96, ny=8, order=3), P.vortex2d(n=32, order=3)]
    X, Y = T.collect(probs, steps=(0, 3, 8))
    nin = X.shape[1]
    p1, l1 = T.train(X, Y, nin, steps=1200, batch=2048)
    p2, l2 = T.train(X, Y, nin, steps=1200, batch=2048)
    assert np.array_equal(p1, p2) and np.array_equal(l1, l2)
    assert l1[-50:].mean() < 0.6 * l1[:50].mean()
    acc, recall, frac = T.accuracy(p1, X, Y, nin)
    assert acc > 0.85 and recall > 0.9, (acc, recall, frac)


@pytest.mark.parametrize("dim,order,n", CASES)
def test_gated_step_matches_the_oracle(awe, dim, order, n):
    prob = P.Problem("uniform", dim, n, (0, 0, 0), (1.0, 1.2, 0.9), order)
    # a mild jump: random weights may send it through linear reconstruction,
    # which must stay positive for the step to be comparable
    U = shocky(prob, jr=1.2, jp=1.3)
    nin, npar = awe.gate_dims(dim, order)
    params = random_params(nin, 5)
    g = awe.Grid(prob, gate=True)
    g.gate_set_weights(params)
    g.set_state(U)
    orc = oracle.Oracle(prob)
    dt = 0.3 / orc.signal_max(U)
    g.step(dt)
    flags = orc.gate_flags(U, 0.0, params)
    assert 0 < flags.mean() < 1
    Uo, _, rc = orc.step(U, 0.0, dt, flags=flags)
    assert rc == 0
    Ug = g.get_state()
    for v in range(prob.nv):
        assert np.abs(Ug[v] - Uo[v]).sum() <= 1e-12 * np.abs(Uo[v]).sum(), v
    fl, tot = g.gate_stats()
    assert 0 < fl < tot


def test_trained_gate_gains_over_full_weno(awe):
    """Trained on labels from the method, the gate sends most of the resolved
    smooth vortex to linear reconstruction: the gated run is at least as
    accurate as full WENO against the exact solution (the linear weights are
    the smooth-optimal ones), keeps the design order, and still flags the Sod
    shock."""
    from paper_2211_13295_gb300 import gate_train as T
    probs = [P.vortex2d(n=64, order=3), P.sod(nx=96, ny=8, order=3), P.vortex2d(n=32, order=3)]
    X, Y = T.collect(probs, steps=(0, 3, 8))
    nin = X.shape[1]
    params, _ = T.train(X, Y, nin, steps=1500, batch=4096)
    errs, frac = {}, {}
    for n in (64, 128):
        prob = P.vortex2d(n=n, order=3, t_end=0.5)
        ex = P.vortex_exact(prob, 0.5)[0]
        for gate in (False, True):
            g = awe.Grid(prob, gate=gate)
            if gate:
                g.gate_set_weights(params)
            g.set_state(prob.initial_state())
            t, dt = 0.0, g.cfl_dt()
            fl_sum = tot_sum = 0
            while t < 0.5 - 1e-12:
                dt = min(dt, 0.5 - t)
                dn = g.step(dt)
                if gate:
                    fl, tot = g.gate_stats()
                    fl_sum += fl
                    tot_sum += tot
                t += dt
                dt = dn
            if gate:
                frac[n] = fl_sum / tot_sum
            errs[(n, gate)] = np.abs(g.get_state()[0] - ex).mean()
    assert frac[128] < 0.5, frac
    for n in (64, 128):
        assert errs[(n, True)] <= 1.05 * errs[(n, False)], errs
    rate = np.log2(errs[(64, True)] / errs[(128, True)])
    assert rate > 2.5, errs
    # the shock is flagged
    prob = P.sod(nx=64, ny=8, order=3)
    g = awe.Grid(prob, gate=True)
    g.gate_set_weights(params)
    g.set_state(prob.initial_state())
    fl = g.gate_flags()
    gz = 3
    row = fl[0, gz + 4, gz:gz + 64]
    assert row[30:34].all()
