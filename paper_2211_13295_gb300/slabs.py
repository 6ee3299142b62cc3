"""Slab decomposition of one grid along its outermost dimension (z in 3D, y in
2D): the paper's patch layer reduced to slabs (Sec. II.2, the MPI remarks
after Fig. 7: per step one exchange of ghost zones and one MIN reduction of
dt over all patches; Sec. V, the patch layer; Sec. I.1: ADER needs one
exchange per step, a Runge-Kutta scheme one per stage).

Every subdomain is an ordinary grid (awe.Grid) whose faces towards its
neighbours have the boundary "exchange": before each stage the planes next
to those faces are packed on the device (awe_halo_pack), moved to the
neighbour and unpacked into its ghost planes (awe_halo_unpack); every other
ghost zone is filled by the library.  The time step is the minimum of the
subdomains' device-resident dt (each cfl / max of its signal speeds), which
equals cfl / the global maximum because division is monotone.

* SlabGrid: all subdomains on the current device, in one process: the
  exchange is a device copy through two halo buffers per subdomain.
* DistSlabGrid: one subdomain per rank of a torch.distributed process group;
  HaloExchange moves the buffers with point-to-point sends (NCCL between
  GPUs, gloo between host buffers) and dt is an all-reduce MIN.

This module holds host logic only (which planes go where, in which order);
all arithmetic on the state runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def split_extent(n, parts, min_size):
    """Offsets and sizes of `parts` contiguous pieces of n zones, sizes
    differing by at most one, each at least min_size (the ghost width)."""
    if parts < 1 or n < parts * min_size:
        raise ValueError(f"{n} zones cannot be split into {parts} slabs of at least {min_size}")
    base, extra = divmod(n, parts)
    out, off = [], 0
    for p in range(parts):
        size = base + (1 if p < extra else 0)
        out.append((off, size))
        off += size
    return out


def outer_dim(prob):
    return prob.dim - 1


def sub_problem(prob, offset, size, first, last):
    """The subdomain [offset, offset + size) of prob's outermost dimension: its
    faces towards neighbours exchange; the global ends keep prob's boundary
    conditions unless they are periodic (then they exchange with the other
    end).  Its zone sizes are the undivided grid's, passed explicitly: the
    extent of a piece divided by its zone count can differ from them in the
    last bit, which would change every update of the subdomain."""
    od = outer_dim(prob)
    n = list(prob.n)
    n[od] = size
    h = prob.dx(od)
    lo, hi = list(prob.lo), list(prob.hi)
    lo[od] = prob.lo[od] + offset * h
    hi[od] = prob.lo[od] + (offset + size) * h
    dxs = tuple(prob.dx(d) if d < prob.dim else 1.0 for d in range(3))
    bc = list(prob.bc)
    periodic = prob.bc[2 * od] == "periodic"
    if periodic != (prob.bc[2 * od + 1] == "periodic"):
        raise ValueError("periodic on one outer face only")
    if periodic or not first:
        bc[2 * od] = "exchange"
    if periodic or not last:
        bc[2 * od + 1] = "exchange"
    return prob.replace(n=tuple(n), lo=tuple(lo), hi=tuple(hi), bc=tuple(bc), dxs=dxs)


def state_axis(prob):
    """axis of the outermost dimension in a [var][z][y][x] state array"""
    return 1 if prob.dim == 3 else 2


class HaloExchange:
    """Point-to-point exchange of halo buffers between the ranks of a process
    group that own consecutive slabs (rank r the r-th slab).  Two phases, each
    one batch of sends and receives: upward (every rank sends its high-side
    planes to rank r + 1 and receives its low-side ghosts from rank r - 1),
    then downward.  With two ranks and periodic ends both neighbours are the
    same rank; the phases keep the messages of the two directions apart.  A
    non-periodic end has no neighbour and its buffer is left alone."""

    def __init__(self, rank, world, periodic, group=None):
        self.rank, self.world, self.periodic, self.group = rank, world, periodic, group
        self.lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
        self.hi = rank + 1 if rank < world - 1 else (0 if periodic else None)

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        if self.world == 1:
            if self.periodic:
                recv_lo.copy_(send_hi)
                recv_hi.copy_(send_lo)
            return
        import torch.distributed as dist
        for send, to, recv, frm in ((send_hi, self.hi, recv_lo, self.lo), (send_lo, self.lo, recv_hi, self.hi)):
            ops = []
            if to is not None:
                ops.append(dist.P2POp(dist.isend, send, to, self.group))
            if frm is not None:
                ops.append(dist.P2POp(dist.irecv, recv, frm, self.group))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()

    def min_(self, t):
        """in-place MIN over the group of a one-element tensor"""
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return t


class SlabGrid:
    """A grid split into `parts` slabs along its outermost dimension, all on
    the current device and stream.  Same results as the unsplit grid, bit for
    bit, for the plain and FP32-bulk forms, ADER and Runge-Kutta."""

    def __init__(self, prob, parts, prec="fp64", gate=False, slab=0):
        import torch
        from . import awe
        self.prob = prob
        od = outer_dim(prob)
        self.pieces = split_extent(prob.n[od], parts, prob.order)
        self.subs = [awe.Grid(sub_problem(prob, off, size, p == 0, p == parts - 1), prec=prec, gate=gate, slab=slab)
                     for p, (off, size) in enumerate(self.pieces)]
        self.periodic = prob.bc[2 * od] == "periodic"
        self.stages = self.subs[0].stage_count()
        m = self.subs[0].halo_size()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.lo_buf = [torch.empty(m, dtype=torch.float64, device=dev) for _ in self.subs]
        self.hi_buf = [torch.empty(m, dtype=torch.float64, device=dev) for _ in self.subs]
        self.dts = torch.empty(len(self.subs), dtype=torch.float64, device=dev)
        self.axis = state_axis(prob)

    def close(self):
        for s in self.subs:
            s.close()

    def set_state(self, U):
        for s, (off, size) in zip(self.subs, self.pieces):
            s.set_state(np.ascontiguousarray(np.take(U, range(off, off + size), axis=self.axis)))

    def get_state(self):
        return np.concatenate([s.get_state() for s in self.subs], axis=self.axis)

    def set_time(self, t):
        for s in self.subs:
            s.set_time(t)

    def gate_set_weights(self, params):
        for s in self.subs:
            s.gate_set_weights(params)

    def exchange(self):
        """halo planes of the next stage's input: pack every slab, then unpack
        into its neighbours' ghost planes"""
        P = len(self.subs)
        for s, lo, hi in zip(self.subs, self.lo_buf, self.hi_buf):
            s.halo_pack(0, lo)
            s.halo_pack(1, hi)
        for p, s in enumerate(self.subs):
            below = p - 1 if p > 0 else (P - 1 if self.periodic else None)
            above = p + 1 if p < P - 1 else (0 if self.periodic else None)
            if below is not None:
                s.halo_unpack(0, self.hi_buf[below])
            if above is not None:
                s.halo_unpack(1, self.lo_buf[above])

    def _global_dt(self):
        for p, s in enumerate(self.subs):
            s.get_dt(self.dts[p:p + 1])
        m = self.dts.min().reshape(1)
        for s in self.subs:
            s.set_dt(m)

    def cfl_dt(self, sync=True):
        for s in self.subs:
            s.cfl_dt(sync=False)
        self._global_dt()
        return self.subs[0].get_dt() if sync else None

    def step(self, dt=0.0, sync=True):
        """one step of every slab: per stage an exchange, then the stage; then
        the global dt (minimum over the slabs) for the next step"""
        for k in range(self.stages):
            if self._spans is not None:
                a = _event()
            self.exchange()
            if self._spans is not None:
                self._spans.append((a, _event()))
            for s in self.subs:
                s.stage(k, dt if k == 0 else 0.0)
        self._global_dt()
        if sync:
            for s in self.subs:
                s.check()
            return self.subs[0].get_dt()
        return None

    def check(self):
        for s in self.subs:
            s.check()

    # timing: every slab's kernels plus the exchanges (CUDA events)
    _spans = None

    def profile(self, enable=True):
        for s in self.subs:
            s.profile(enable)
        self._spans = [] if enable else None

    def profile_read(self):
        import torch
        out = {}
        for s in self.subs:
            for k, (n, ms) in s.profile_read().items():
                a = out.get(k, (0, 0.0))
                out[k] = (a[0] + n, a[1] + ms)
        torch.cuda.synchronize()
        sp = self._spans or []
        out["halo_exchange"] = (len(sp), sum(a.elapsed_time(b) for a, b in sp))
        return out


def _event():
    import torch
    e = torch.cuda.Event(enable_timing=True)
    e.record()
    return e


class DistSlabGrid:
    """This rank's slab of a grid split over the ranks of a process group (one
    slab per rank, rank r the r-th).  `grid` makes the subdomain grid from a
    problem (default: awe.Grid on the current device); `buffer` makes a halo
    buffer of m doubles (default: a float64 tensor on the current device)."""

    def __init__(self, prob, rank, world, prec="fp64", gate=False, slab=0, group=None, grid=None, buffer=None):
        import torch
        od = outer_dim(prob)
        self.prob = prob
        self.pieces = split_extent(prob.n[od], world, prob.order)
        off, size = self.pieces[rank]
        self.offset, self.size = off, size
        self.sub_prob = sub_problem(prob, off, size, rank == 0, rank == world - 1)
        if grid is None:
            from . import awe
            self.sub = awe.Grid(self.sub_prob, prec=prec, gate=gate, slab=slab)
        else:
            self.sub = grid(self.sub_prob)
        self.comm = HaloExchange(rank, world, prob.bc[2 * od] == "periodic", group)
        self.stages = self.sub.stage_count()
        m = self.sub.halo_size()
        if buffer is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            buffer = lambda k: torch.empty(k, dtype=torch.float64, device=dev)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = (buffer(m) for _ in range(4))
        self.dt = buffer(1)
        self.axis = state_axis(prob)

    def close(self):
        self.sub.close()

    def local(self, U):
        """this rank's part of a global state array"""
        return np.ascontiguousarray(np.take(U, range(self.offset, self.offset + self.size), axis=self.axis))

    def set_state(self, U_local):
        self.sub.set_state(U_local)

    def get_state(self, out=None):
        return self.sub.get_state(out)

    def exchange(self):
        self.sub.halo_pack(0, self.send_lo)
        self.sub.halo_pack(1, self.send_hi)
        self.comm.exchange(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi)
        if self.comm.lo is not None:
            self.sub.halo_unpack(0, self.recv_lo)
        if self.comm.hi is not None:
            self.sub.halo_unpack(1, self.recv_hi)

    def _global_dt(self):
        self.sub.get_dt(self.dt)
        self.comm.min_(self.dt)
        self.sub.set_dt(self.dt)

    def cfl_dt(self, sync=True):
        self.sub.cfl_dt(sync=False)
        self._global_dt()
        return self.sub.get_dt() if sync else None

    def set_time(self, t):
        self.sub.set_time(t)

    def step(self, dt=0.0, sync=False):
        """one step: per stage the halo exchange, then the stage; then the
        global dt.  With timing on (profile), CUDA events on the current stream
        bracket the exchanges (packing, transfer, unpacking)."""
        for k in range(self.stages):
            if self._ev is not None:
                a = _event()
            self.exchange()
            if self._ev is not None:
                self._spans.append((a, _event()))
            self.sub.stage(k, dt if k == 0 else 0.0)
        self._global_dt()

    def check(self):
        self.sub.check()

    # timing: the subdomain's kernels plus the exchanges
    _ev = None

    def profile(self, enable=True):
        self.sub.profile(enable)
        self._ev = True if enable else None
        self._spans = []

    def profile_read(self):
        import torch
        out = self.sub.profile_read()
        torch.cuda.synchronize()
        out["halo_exchange"] = (len(self._spans), sum(a.elapsed_time(b) for a, b in self._spans))
        return out
