"""Host logic of the slab decomposition on CPU ranks (gloo; world sizes 2 and
3): the split of the outermost dimension, the subdomains' boundary
conditions, the neighbour topology and message order of HaloExchange, and
DistSlabGrid's step (exchange, stage, MIN of dt over the ranks).

The subdomain grid is a test double built on the FP64 oracle with host
buffers, with the same interface as the CUDA grid (halo_pack / halo_unpack /
stage / get_dt / set_dt): after the exchange every rank's ghosted array must
equal, bit for bit, the window of the undivided grid's ghosted array (the
oracle's own boundary fill), and two sharded steps must equal two steps of the
undivided oracle, bit for bit, with the same dt on every rank."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_and_subdomain_boundaries():
    from paper_2211_13295_gb300 import problems as P
    from paper_2211_13295_gb300 import slabs
    assert slabs.split_extent(10, 3, 3) == [(0, 4), (4, 3), (7, 3)]
    with pytest.raises(ValueError):
        slabs.split_extent(8, 3, 3)
    prob = P.Problem("uniform", 3, (6, 5, 12), (0, 0, 0), (1.0, 1.0, 2.0), 3,
                     bc=("periodic", "periodic", "reflect", "reflect", "outflow", "inflow"))
    first = slabs.sub_problem(prob, 0, 4, True, False)
    mid = slabs.sub_problem(prob, 4, 4, False, False)
    last = slabs.sub_problem(prob, 8, 4, False, True)
    assert first.bc[4:] == ("outflow", "exchange") and mid.bc[4:] == ("exchange", "exchange")
    assert last.bc[4:] == ("exchange", "inflow") and last.bc[:4] == prob.bc[:4]
    assert mid.n == (6, 5, 4) and abs(mid.lo[2] - 2.0 / 3.0) < 1e-15 and abs(mid.hi[2] - 4.0 / 3.0) < 1e-15
    # every subdomain's zone sizes are the undivided ones, to the bit
    for n, L in ((11, 1.8), (13, 0.8), (1000, 0.7), (37, 2 * np.pi)):
        big = prob.replace(n=(6, 5, n), hi=(1.0, 1.0, L))
        for off, size in slabs.split_extent(n, 3, 3):
            sub = slabs.sub_problem(big, off, size, off == 0, off + size == n)
            assert all(sub.dx(d) == big.dx(d) for d in range(3))
    per = slabs.sub_problem(prob.replace(bc=("periodic",) * 6), 0, 4, True, False)
    assert per.bc[4:] == ("exchange", "exchange")
    two_d = P.Problem("uniform", 2, (8, 9, 1), (0, 0, 0), (1.0, 1.0, 1.0), 3, bc=("outflow",) * 6)
    assert slabs.sub_problem(two_d, 3, 3, False, False).bc[:4] == ("outflow", "outflow", "exchange", "exchange")


def _state(prob, seed):
    """a positive state with smooth parts and a jump (seeded)"""
    from paper_2211_13295_gb300 import problems as P
    rng = np.random.default_rng(seed)
    sh = prob.shape()
    idx = np.meshgrid(*[np.arange(n) for n in sh[1:]], indexing="ij")
    f = lambda: sum(np.sin(2 * np.pi * (k + 1) * (x + 0.5) / n + rng.uniform(0, 6))  # noqa: E731
                    for k, x, n in zip(range(3), idx, sh[1:]))
    rho = 1.0 + 0.05 * f()
    rho = np.where(idx[0] < sh[1] // 2, rho, 2.0 * rho)
    vel = [0.2 * f() for _ in range(prob.dim)]
    p = 1.0 + 0.05 * f()
    c = P.conserved(prob.gamma, rho, vel, p)
    U = np.zeros(sh)
    for v in range(prob.nv):
        U[v] = c[v]
    return U


class OracleSubdomain:
    """The FP64 oracle behind the subdomain-grid interface, on host buffers:
    exchanged faces are filled from the unpacked planes, every other ghost
    zone by the oracle's own fill (a periodic placeholder stands in for the
    exchanged faces before they are overwritten)."""

    def __init__(self, sub_prob):
        import oracle
        self.prob = sub_prob
        ph = tuple("periodic" if b == "exchange" else b for b in sub_prob.bc)
        self.orc = oracle.Oracle(sub_prob.replace(bc=ph))
        # the oracle takes its zone sizes from the extent: the test's grid is
        # chosen so that they are the undivided grid's (z zones of 1/8)
        assert all((sub_prob.hi[d] - sub_prob.lo[d]) / sub_prob.n[d] == sub_prob.dx(d) for d in range(3))
        self.exch = [sub_prob.bc[4] == "exchange", sub_prob.bc[5] == "exchange"]
        self.g = sub_prob.order
        self.recv = [None, None]
        self.t, self.dt = 0.0, None
        self.last_ghosted = None

    def stage_count(self):
        return 1

    def halo_size(self):
        G = self.orc.G
        return self.orc.nv * self.g * G[0] * G[1]

    def set_state(self, U):
        self.U = np.array(U, dtype=np.float64)

    def get_state(self, out=None):
        return self.U.copy()

    def _ghosted(self):
        return self.orc.ghosted(self.U, self.t)

    def halo_pack(self, side, out):
        Ug = self._ghosted()
        g, n = self.g, self.prob.n[2]
        planes = Ug[:, g:2 * g] if side == 0 else Ug[:, n:n + g]
        out.copy_(__import__("torch").from_numpy(np.ascontiguousarray(planes).reshape(-1)))

    def halo_unpack(self, side, buf):
        G = self.orc.G
        self.recv[side] = buf.numpy().reshape(self.orc.nv, self.g, G[1], G[0]).copy()

    def stage(self, k, dt):
        assert k == 0
        Ug = self._ghosted()
        g, n = self.g, self.prob.n[2]
        if self.exch[0]:
            Ug[:, :g] = self.recv[0]
        if self.exch[1]:
            Ug[:, n + g:] = self.recv[1]
        self.last_ghosted = Ug.copy()
        dt = dt if dt > 0 else self.dt
        self.U, smax, rc = self.orc.step_ghosted(Ug, dt)
        assert rc == 0
        self.t += dt
        self.dt = self.prob.cfl / smax

    def cfl_dt(self, sync=True):
        self.dt = self.orc.cfl_dt(self.U, self.prob.cfl)

    def get_dt(self, out=None):
        if out is None:
            return self.dt
        out[0] = self.dt
        return out

    def set_dt(self, t):
        self.dt = float(t[0])

    def check(self):
        pass

    def close(self):
        pass


def _worker(rank, world, port, bc, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2211_13295_gb300 import problems as P
        from paper_2211_13295_gb300 import slabs
        prob = P.Problem("uniform", 3, (6, 5, 11), (0, 0, 0), (1.0, 0.9, 1.375), 3, cfl=0.4,
                         bc=("periodic", "periodic", "reflect", "reflect", bc, bc))
        U = _state(prob, 7)
        buf = lambda m: torch.zeros(m, dtype=torch.float64)  # noqa: E731
        dsg = slabs.DistSlabGrid(prob, rank, world, grid=OracleSubdomain, buffer=buf)
        dsg.set_state(dsg.local(U))
        dsg.cfl_dt()
        ghosted, dts = [], []
        for _ in range(2):
            dsg.step(0.0)
            ghosted.append(dsg.sub.last_ghosted)
            dts.append(dsg.sub.dt)
        q.put((rank, dsg.offset, dsg.size, dsg.get_state(), ghosted, dts))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,bc", [(2, "periodic"), (2, "outflow"), (3, "periodic")])
def test_sharded_oracle_steps_equal_the_undivided_steps(world, bc):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2211_13295_gb300 import problems as P
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bc, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, off, size, Ur, gh, dts = q.get(timeout=300)
        got[r] = (off, size, Ur, gh, dts)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the undivided grid, the same two steps
    prob = P.Problem("uniform", 3, (6, 5, 11), (0, 0, 0), (1.0, 0.9, 1.375), 3, cfl=0.4,
                     bc=("periodic", "periodic", "reflect", "reflect", bc, bc))
    orc = oracle.Oracle(prob)
    U = _state(prob, 7)
    dt, t = orc.cfl_dt(U, prob.cfl), 0.0
    g = prob.order
    for s in range(2):
        Ug = orc.ghosted(U, t)
        for r in range(world):
            off, size, _, gh, dts = got[r]
            assert np.array_equal(gh[s], Ug[:, off:off + size + 2 * g]), (r, s)
        U, smax, rc = orc.step(U, t, dt)
        assert rc == 0
        t += dt
        dt = prob.cfl / smax
        assert all(got[r][4][s] == dt for r in range(world))
    whole = np.concatenate([got[r][2] for r in range(world)], axis=1)
    assert np.array_equal(whole, U)
