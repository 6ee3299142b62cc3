"""Steps captured in a CUDA graph (awe.StepGraph) replay bit for bit what the
same steps do eagerly, for the ADER scheme (the 64^2 order-3 vortex, a
launch-bound size), the gated form and the Runge-Kutta variant; the replay
also carries the device-resident time and time step along."""
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


def eager_and_graph(awe, prob, steps, gate=None):
    import torch
    s = torch.cuda.Stream()
    out = []
    for use_graph in (False, True):
        with torch.cuda.stream(s):
            g = awe.Grid(prob, gate=gate is not None)
            if gate is not None:
                g.gate_set_weights(gate)
            g.set_state(prob.initial_state())
            g.cfl_dt()
            g.step(0.0, sync=False)          # loads every kernel before any capture
            if use_graph:
                sg = awe.StepGraph(g, steps, s)
                sg.replay()
            else:
                for _ in range(steps):
                    g.step(0.0, sync=False)
            s.synchronize()
            g.check()
            out.append((g.get_state(), g.time()))
            g.close()
    return out


@pytest.mark.parametrize("scheme", ["ader", "ssprk"])
def test_graph_replay_is_bitwise(awe, scheme):
    prob = P.vortex2d(n=64, order=3).replace(scheme=scheme)
    (Ue, te), (Ug, tg) = eager_and_graph(awe, prob, 12)
    assert np.array_equal(Ue, Ug) and te == tg and te > 0


def test_graph_replay_gated(awe):
    from paper_2211_13295_gb300.gate_train import he_init
    prob = P.vortex2d(n=32, order=3)
    nin, _ = awe.gate_dims(2, 3)
    params = he_init(nin, 3)
    (Ue, te), (Ug, tg) = eager_and_graph(awe, prob, 6, gate=params)
    assert np.array_equal(Ue, Ug) and te == tg
