"""ctypes binding of libawe.so (include/awe.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The module-level functions carry the C names (awe_create,
awe_step, ...); :class:`Grid` is a thin convenience wrapper over them that
accepts numpy arrays (host) or CUDA torch tensors (device pointers; torch is
used only for device memory and the stream).

Loading fails loudly (RuntimeError) when the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libawe.so")

AWE_OK, AWE_ERR_ARG, AWE_ERR_CUDA, AWE_ERR_OOM, AWE_ERR_NONPHYSICAL, AWE_ERR_TIMEOUT, AWE_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
BC = {"periodic": 0, "outflow": 1, "reflect": 2, "inflow": 3, "dmr_bottom": 4, "dmr_top": 5, "exchange": 6}
PREC = {"fp64": 0, "fp32": 1}
RIEMANN = {"hllc": 0, "hll": 1, "hllem": 2, "rusanov": 3}
SCHEME = {"ader": 0, "ssprk": 1}


class AweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"awe status {code}: {msg}")
        self.code = code


class AweConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("order", C.c_int), ("gamma", C.c_double), ("bc", C.c_int * 6),
        ("inflow", (C.c_double * 5) * 6), ("pre", C.c_double * 5), ("prec", C.c_int),
        ("picard", C.c_int), ("weno_eps", C.c_double), ("lin", C.c_double * 4), ("cfl", C.c_double),
        ("gate", C.c_int), ("slab", C.c_int), ("fallback", C.c_int),
        ("riemann", C.c_int), ("scheme", C.c_int), ("rk_stages", C.c_int), ("dx", C.c_double * 3),
    ]


_lib = None


def lib():
    """Load libawe.so (raises if it is missing: build it with
    ``python -m paper_2211_13295_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libawe.so not built ({LIB_PATH}); run python -m paper_2211_13295_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, dp, fp, up = C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p
    sig = {
        "awe_create": (C.c_int, [C.POINTER(AweConfig), vp, C.POINTER(vp)]),
        "awe_destroy": (C.c_int, [vp]),
        "awe_last_error": (C.c_char_p, [vp]),
        "awe_set_state": (C.c_int, [vp, vp, C.c_int]),
        "awe_get_state": (C.c_int, [vp, vp, C.c_int]),
        "awe_set_time": (C.c_int, [vp, C.c_double]),
        "awe_get_time": (C.c_int, [vp, dp]),
        "awe_cfl_dt": (C.c_int, [vp, C.c_double, dp]),
        "awe_step": (C.c_int, [vp, C.c_double, dp]),
        "awe_check": (C.c_int, [vp]),
        "awe_fallback_count": (C.c_int, [vp, C.POINTER(C.c_longlong)]),
        "awe_probe_modes": (C.c_int, [vp, vp]),
        "awe_probe_face_states": (C.c_int, [vp, C.c_double, vp]),
        "awe_probe_fluxes": (C.c_int, [vp, C.c_double, vp]),
        "awe_profile": (C.c_int, [vp, C.c_int]),
        "awe_profile_count": (C.c_int, []),
        "awe_profile_read": (C.c_int, [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_long), dp]),
        "awe_gate_dims": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
        "awe_gate_set_weights": (C.c_int, [vp, vp, C.c_size_t]),
        "awe_gate_features": (C.c_int, [vp, vp, C.c_int]),
        "awe_gate_labels": (C.c_int, [vp, C.c_double, vp, C.c_int]),
        "awe_gate_flags": (C.c_int, [vp, vp, C.c_int]),
        "awe_gate_stats": (C.c_int, [vp, C.POINTER(C.c_long), C.POINTER(C.c_long)]),
        "awe_mlp_train": (C.c_int, [C.c_int, vp, vp, vp, vp, vp, C.c_long, C.c_int, C.c_int, C.c_long,
                                    C.c_float, C.c_ulonglong, vp, vp]),
        "awe_mlp_loss_grad": (C.c_int, [C.c_int, vp, vp, vp, C.c_long, vp, vp, vp]),
        "awe_mlp_forward": (C.c_int, [C.c_int, vp, vp, C.c_long, vp, vp]),
        "awe_measure_fma_peaks": (C.c_int, [dp, dp]),
        "awe_cfl_dt_noalloc": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), dp, C.c_double, C.c_double,
                                         vp, vp]),
        "awe_halo_size": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "awe_halo_pack": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "awe_halo_unpack": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "awe_stage_count": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "awe_stage": (C.c_int, [vp, C.c_int, C.c_double]),
        "awe_get_dt": (C.c_int, [vp, vp, C.c_int]),
        "awe_set_dt": (C.c_int, [vp, vp, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points the binding expects."""
    return [
        "awe_create", "awe_destroy", "awe_last_error", "awe_set_state", "awe_get_state", "awe_set_time",
        "awe_get_time", "awe_cfl_dt", "awe_step", "awe_check", "awe_probe_modes", "awe_probe_face_states",
        "awe_probe_fluxes", "awe_profile", "awe_profile_count", "awe_profile_read", "awe_gate_dims",
        "awe_gate_set_weights", "awe_gate_features", "awe_gate_labels", "awe_gate_flags", "awe_gate_stats",
        "awe_mlp_train", "awe_mlp_loss_grad", "awe_mlp_forward", "awe_measure_fma_peaks",
        "awe_cfl_dt_noalloc", "awe_fallback_count", "awe_halo_size", "awe_halo_pack", "awe_halo_unpack",
        "awe_stage_count", "awe_stage", "awe_get_dt", "awe_set_dt",
    ]


def _check(rc, handle=None):
    if rc != AWE_OK:
        msg = lib().awe_last_error(handle)
        raise AweError(rc, msg.decode() if msg else "")


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor"""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data_as(C.c_void_p), 0
    # torch tensor
    assert x.is_contiguous()
    return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def make_config(prob, prec="fp64", gate=False, slab=0, cfl=None, picard=None) -> AweConfig:
    c = AweConfig()
    c.dim = prob.dim
    for d in range(3):
        c.n[d] = prob.n[d] if d < prob.dim else 1
        c.lo[d] = prob.lo[d] if d < prob.dim else 0.0
        c.hi[d] = prob.hi[d] if d < prob.dim else 1.0
    c.order = prob.order
    c.gamma = prob.gamma
    for f in range(6):
        c.bc[f] = BC[prob.bc[f]]
        st = prob.inflow[f]
        if st is not None:
            for v in range(len(st)):
                c.inflow[f][v] = st[v]
    if prob.pre is not None:
        for v in range(len(prob.pre)):
            c.pre[v] = prob.pre[v]
    c.prec = PREC[prec]
    c.picard = prob.picard if picard is None else picard
    c.weno_eps = prob.eps
    for k, w in enumerate(prob.lin):
        c.lin[k] = w
    c.cfl = prob.cfl if cfl is None else cfl
    c.gate = 1 if gate else 0
    c.slab = slab
    c.fallback = int(getattr(prob, "fallback", 0) or 0)
    c.riemann = RIEMANN[getattr(prob, "riemann", "hllc")]
    c.scheme = SCHEME[getattr(prob, "scheme", "ader")]
    c.rk_stages = int(getattr(prob, "rk_stages", 0))
    for d, h in enumerate(getattr(prob, "dxs", ()) or ()):
        c.dx[d] = float(h)
    return c


class Grid:
    """A grid on the current CUDA device (wraps awe_create/awe_destroy)."""

    def __init__(self, prob, prec="fp64", gate=False, slab=0, cfl=None, picard=None, stream=None):
        self.prob = prob
        self.prec = prec
        self.cfg = make_config(prob, prec, gate, slab, cfl, picard)
        h = C.c_void_p()
        self._stream = _current_stream() if stream is None else C.c_void_p(stream)
        rc = lib().awe_create(C.byref(self.cfg), self._stream, C.byref(h))
        if rc != AWE_OK:
            raise AweError(rc, lib().awe_last_error(None).decode())
        self.h = h
        self.nv = prob.dim + 2
        self.shape = prob.shape()
        g = prob.order
        self.ghosted_shape = tuple((prob.n[d] + 2 * g) if d < prob.dim else 1 for d in (2, 1, 0))
        self.box_shape = tuple((prob.n[d] + 2) if d < prob.dim else 1 for d in (2, 1, 0))

    def close(self):
        if getattr(self, "h", None):
            lib().awe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state ---------------------------------------------------------------
    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
            assert U.shape == self.shape, (U.shape, self.shape)
        p, dev = _ptr(U)
        _check(lib().awe_set_state(self.h, p, dev), self.h)

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.shape)
        p, dev = _ptr(out)
        _check(lib().awe_get_state(self.h, p, dev), self.h)
        return out

    def set_time(self, t):
        _check(lib().awe_set_time(self.h, float(t)), self.h)

    def time(self):
        t = C.c_double()
        _check(lib().awe_get_time(self.h, C.byref(t)), self.h)
        return t.value

    def cfl_dt(self, cfl=None, sync=True):
        cfl = self.cfg.cfl if cfl is None else cfl
        dt = C.c_double()
        _check(lib().awe_cfl_dt(self.h, float(cfl), C.byref(dt) if sync else None), self.h)
        return dt.value if sync else None

    def step(self, dt=0.0, sync=True):
        """One step with dt (> 0), or the device-resident dt (dt <= 0); returns
        dt_next when sync, else None (no host round trip)."""
        dn = C.c_double()
        _check(lib().awe_step(self.h, float(dt), C.byref(dn) if sync else None), self.h)
        return dn.value if sync else None

    def check(self):
        _check(lib().awe_check(self.h), self.h)

    # stages, halos and dt of a subdomain (slab decomposition) ------------
    def stage_count(self):
        n = C.c_int()
        _check(lib().awe_stage_count(self.h, C.byref(n)), self.h)
        return n.value

    def stage(self, k, dt=0.0):
        _check(lib().awe_stage(self.h, int(k), float(dt)), self.h)

    def halo_size(self):
        n = C.c_size_t()
        _check(lib().awe_halo_size(self.h, C.byref(n)), self.h)
        return n.value

    def _buffer(self, buf, count, what):
        """pointer of a float64 buffer of at least `count` elements: a
        contiguous numpy array, or a contiguous tensor on the host or on the
        grid's device (the C entry points cannot see a buffer's extent)"""
        if isinstance(buf, np.ndarray):
            if buf.dtype != np.float64 or not buf.flags["C_CONTIGUOUS"] or buf.size < count:
                raise ValueError(f"{what}: need a contiguous float64 array of {count} elements")
        else:
            import torch
            if not isinstance(buf, torch.Tensor) or buf.dtype != torch.float64 or not buf.is_contiguous() \
                    or buf.numel() < count:
                raise ValueError(f"{what}: need a contiguous float64 tensor of {count} elements")
            if buf.is_cuda and buf.device.index != torch.cuda.current_device():
                raise ValueError(f"{what}: the tensor is not on the current device")
        return _ptr(buf)

    def halo_pack(self, side, out):
        """planes next to face `side` of the next stage's input into `out`
        (numpy array or contiguous float64 tensor of halo_size() elements)"""
        p, dev = self._buffer(out, self.halo_size(), "halo_pack")
        _check(lib().awe_halo_pack(self.h, int(side), p, dev), self.h)
        return out

    def halo_unpack(self, side, buf):
        p, dev = self._buffer(buf, self.halo_size(), "halo_unpack")
        _check(lib().awe_halo_unpack(self.h, int(side), p, dev), self.h)

    def get_dt(self, out=None):
        """device-resident dt: into `out` (a float64 tensor on the device, no
        host round trip) or returned as a float"""
        if out is None:
            v = C.c_double()
            _check(lib().awe_get_dt(self.h, C.byref(v), 0), self.h)
            return v.value
        p, dev = self._buffer(out, 1, "get_dt")
        _check(lib().awe_get_dt(self.h, p, dev), self.h)
        return out

    def set_dt(self, dt):
        """dt from a float or from a one-element float64 tensor on the device"""
        if isinstance(dt, (int, float)):
            v = C.c_double(float(dt))
            _check(lib().awe_set_dt(self.h, C.byref(v), 0), self.h)
        else:
            p, dev = self._buffer(dt, 1, "set_dt")
            _check(lib().awe_set_dt(self.h, p, dev), self.h)

    def fallback_count(self):
        """box zones sent to the positivity fallback since the last call"""
        n = C.c_longlong()
        _check(lib().awe_fallback_count(self.h, C.byref(n)), self.h)
        return n.value

    # probes --------------------------------------------------------------
    def probe_modes(self):
        from . import problems  # noqa: F401
        ns = _num_modes(self.prob.dim, self.prob.order - 1)
        W = np.zeros((self.nv, ns) + self.box_shape)
        _check(lib().awe_probe_modes(self.h, W.ctypes.data_as(C.c_void_p)), self.h)
        return W

    def probe_face_states(self, dt):
        nq = ((self.prob.order + 1) // 2) ** self.prob.dim
        FS = np.zeros((self.prob.dim, 2, nq, self.nv) + self.box_shape)
        _check(lib().awe_probe_face_states(self.h, float(dt), FS.ctypes.data_as(C.c_void_p)), self.h)
        return FS

    def probe_fluxes(self, dt):
        n = [self.prob.n[d] if d < self.prob.dim else 1 for d in range(3)]
        shapes, total = [], 0
        for d in range(self.prob.dim):
            E = list(n)
            E[d] += 1
            shapes.append(E)
            total += self.nv * E[0] * E[1] * E[2]
        F = np.zeros(total)
        _check(lib().awe_probe_fluxes(self.h, float(dt), F.ctypes.data_as(C.c_void_p)), self.h)
        out, off = [], 0
        for E in shapes:
            sz = self.nv * E[0] * E[1] * E[2]
            out.append(F[off:off + sz].reshape(self.nv, E[2], E[1], E[0]))
            off += sz
        return out

    # timing --------------------------------------------------------------
    def profile(self, enable=True):
        _check(lib().awe_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        out = {}
        for k in range(lib().awe_profile_count()):
            name, n, ms = C.c_char_p(), C.c_long(), C.c_double()
            _check(lib().awe_profile_read(self.h, k, C.byref(name), C.byref(n), C.byref(ms)), self.h)
            out[name.value.decode()] = (n.value, ms.value)
        return out

    # gate ----------------------------------------------------------------
    def gate_set_weights(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().awe_gate_set_weights(self.h, params.ctypes.data_as(C.c_void_p), params.size), self.h)

    def gate_features(self, out=None):
        nin, _ = gate_dims(self.prob.dim, self.prob.order)
        if out is None:
            out = np.zeros(self.ghosted_shape + (nin,), dtype=np.float32)
        p, dev = _ptr(out)
        _check(lib().awe_gate_features(self.h, p, dev), self.h)
        return out

    def gate_labels(self, tau, out=None):
        if out is None:
            out = np.zeros(self.ghosted_shape, dtype=np.uint8)
        p, dev = _ptr(out)
        _check(lib().awe_gate_labels(self.h, float(tau), p, dev), self.h)
        return out

    def gate_flags(self, out=None):
        if out is None:
            out = np.zeros(self.ghosted_shape, dtype=np.uint8)
        p, dev = _ptr(out)
        _check(lib().awe_gate_flags(self.h, p, dev), self.h)
        return out

    def gate_stats(self):
        a, b = C.c_long(), C.c_long()
        _check(lib().awe_gate_stats(self.h, C.byref(a), C.byref(b)), self.h)
        return a.value, b.value


def _num_modes(dim, N):
    from math import comb
    return comb(N + dim, dim)


def gate_dims(dim, order):
    nin, npar = C.c_int(), C.c_size_t()
    _check(lib().awe_gate_dims(dim, order, C.byref(nin), C.byref(npar)))
    return nin.value, npar.value


def mlp_train(nin, params, m, v, X, y, batch, steps, step0, lr, seed, loss_out=None):
    """Adam training on the GPU (all tensors CUDA float32, modified in place)."""
    rc = lib().awe_mlp_train(nin, C.c_void_p(params.data_ptr()), C.c_void_p(m.data_ptr()),
                             C.c_void_p(v.data_ptr()), C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()),
                             X.shape[0], batch, steps, step0, lr, seed,
                             C.c_void_p(loss_out.data_ptr()) if loss_out is not None else None,
                             _current_stream())
    _check(rc)


def mlp_loss_grad(nin, params, X, y, grad, loss):
    rc = lib().awe_mlp_loss_grad(nin, C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()),
                                 C.c_void_p(y.data_ptr()), X.shape[0], C.c_void_p(grad.data_ptr()),
                                 C.c_void_p(loss.data_ptr()), _current_stream())
    _check(rc)


def mlp_forward(nin, params, X, z):
    rc = lib().awe_mlp_forward(nin, C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()), X.shape[0],
                               C.c_void_p(z.data_ptr()), _current_stream())
    _check(rc)


def measure_fma_peaks():
    a, b = C.c_double(), C.c_double()
    _check(lib().awe_measure_fma_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def cfl_dt_noalloc(U, dim, n, dx, gamma, cfl, dt_out):
    """awe_cfl_dt_noalloc on CUDA tensors: U (state, float64, awe_get_state
    layout) and dt_out (one float64) on the current device; enqueues only.

    The C entry point cannot see the extent of the buffers it is given, so the
    checks that keep its kernel inside them are made here, before the call."""
    import torch
    if dim not in (2, 3) or len(n) != dim or len(dx) != dim:
        raise ValueError("cfl_dt_noalloc: dim must be 2 or 3, with dim entries in n and dx")
    for name, t in (("U", U), ("dt_out", dt_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise ValueError(f"cfl_dt_noalloc: {name} must be a float64 CUDA tensor")
    dev = torch.cuda.current_device()
    for name, t in (("U", U), ("dt_out", dt_out)):
        if not t.is_contiguous() or t.device.index != dev:
            raise ValueError(f"cfl_dt_noalloc: {name} must be contiguous and on the current device")
    zones = 1
    for v in n:
        if int(v) < 1:
            raise ValueError("cfl_dt_noalloc: zone counts must be positive")
        zones *= int(v)
    if U.numel() != (dim + 2) * zones:
        raise ValueError(f"cfl_dt_noalloc: U has {U.numel()} elements, the grid needs {(dim + 2) * zones}")
    if dt_out.numel() < 1:
        raise ValueError("cfl_dt_noalloc: dt_out needs one element")
    nn = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    dd = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    rc = lib().awe_cfl_dt_noalloc(C.c_void_p(U.data_ptr()), dim, nn, dd, float(gamma), float(cfl),
                                  C.c_void_p(dt_out.data_ptr()), _current_stream())
    _check(rc)


# C names at module level (same names as include/awe.h)
def __getattr__(name):
    if name.startswith("awe_"):
        return getattr(lib(), name)
    raise AttributeError(name)


class StepGraph:
    """`steps` steps of a grid with the device-resident time step, captured
    into one CUDA graph: replay() launches all their kernels with one call
    (for small grids, where a step is a few microseconds of work per kernel
    and launch overhead dominates).  The grid must live on `stream` (create it
    inside `with torch.cuda.stream(stream)`) and have stepped once eagerly, so
    that every kernel is loaded before the capture; awe_step makes no
    allocation and no host synchronisation when no dt_next is requested."""

    def __init__(self, grid, steps, stream):
        import torch
        if grid._stream.value != stream.cuda_stream:
            raise ValueError("the grid was created on another stream")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=stream):
            for _ in range(steps):
                grid.step(0.0, sync=False)
        self.steps = steps

    def replay(self):
        self.graph.replay()
