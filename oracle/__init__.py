"""ctypes wrapper of the FP64 CPU oracle (oracle/ora.c, oracle/ora_gate.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / --impl reference legs may import this package.  It never
imports the CUDA library and the CUDA library never imports it.

State arrays are numpy float64, conserved variables, [var][z][y][x] (2D:
[var][1][y][x]); the wrapper embeds them into the ghosted layout the C code
uses.  Problem descriptions come from paper_2211_13295_gb300.problems (seeded
input generators that hold none of the method's arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

BC_CODES = {"periodic": 0, "outflow": 1, "reflect": 2, "inflow": 3, "dmr_bottom": 4, "dmr_top": 5}


class OraCfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("order", C.c_int), ("picard", C.c_int),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("gamma", C.c_double),
        ("eps", C.c_double), ("lin", C.c_double * 4), ("bc", C.c_int * 6),
        ("inflow", (C.c_double * 5) * 6), ("pre", C.c_double * 5), ("fallback", C.c_int),
        ("riemann", C.c_int),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        up = C.POINTER(C.c_ubyte)
        cp = C.POINTER(OraCfg)
        sig = {
            "ora_gauss_legendre": (None, [C.c_int, dp, dp]),
            "ora_basis": (C.c_double, [C.c_int, C.c_double]),
            "ora_num_modes": (C.c_int, [C.c_int, C.c_int]),
            "ora_num_st_modes": (C.c_int, [C.c_int, C.c_int]),
            "ora_mode_list": (None, [C.c_int, C.c_int, C.POINTER(C.c_int)]),
            "ora_candidate": (None, [C.c_int, C.c_int, dp, dp]),
            "ora_beta": (C.c_double, [C.c_int, dp]),
            "ora_weno1d": (None, [C.c_int, dp, C.c_double, dp, C.c_int, dp, dp]),
            "ora_hllc": (None, [C.c_int, C.c_double, C.c_int, dp, dp, dp]),
            "ora_riemann": (None, [C.c_int, C.c_int, C.c_double, C.c_int, dp, dp, dp]),
            "ora_rk_coefficients": (C.c_int, [C.c_int, dp, dp]),
            "ora_rk_rhs": (C.c_int, [cp, dp, up, dp]),
            "ora_rk_step": (C.c_int, [cp, dp, C.c_double, C.c_double, C.c_int, C.c_int, fp, dp, dp]),
            "ora_mc_slope": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "ora_phys_flux": (None, [C.c_int, C.c_double, C.c_int, dp, dp]),
            "ora_ghosted_size": (C.c_size_t, [cp]),
            "ora_fill_ghosts": (C.c_int, [cp, dp, C.c_double]),
            "ora_reconstruct": (C.c_int, [cp, dp, up, dp]),
            "ora_predict_zone": (None, [cp, dp, C.c_double, dp]),
            "ora_face_states": (C.c_int, [cp, dp, up, C.c_double, dp]),
            "ora_step": (C.c_int, [cp, dp, C.c_double, up, dp, dp]),
            "ora_fluxes": (C.c_int, [cp, dp, up, C.c_double, dp]),
            "ora_signal_max": (C.c_double, [cp, dp]),
            "ora_exact_riemann": (C.c_int, [C.c_double] * 7 + [C.c_double, dp, dp, dp, dp, dp]),
            "ora_gate_num_features": (C.c_int, [C.c_int, C.c_int]),
            "ora_weno_labels": (C.c_int, [cp, dp, C.c_double, up]),
            "ora_gate_features": (C.c_int, [cp, dp, fp]),
            "ora_mlp_num_params": (C.c_size_t, [C.c_int, C.c_int]),
            "ora_mlp_forward_f64": (None, [C.c_int, C.c_int, fp, fp, C.c_int, dp]),
            "ora_mlp_loss_grad_f64": (C.c_double, [C.c_int, C.c_int, fp, fp, fp, C.c_int, dp]),
            "ora_mlp_forward_f32": (None, [C.c_int, C.c_int, fp, fp, C.c_int, fp]),
            "ora_gate_flags": (C.c_int, [cp, dp, C.c_int, fp, up]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def _up(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_ubyte))


def num_modes(dim, N):
    return lib().ora_num_modes(dim, N)


def num_st_modes(dim, N):
    return lib().ora_num_st_modes(dim, N)


def mode_list(dim, N):
    m = np.zeros((num_modes(dim, N), 3), dtype=np.int32)
    lib().ora_mode_list(dim, N, m.ctypes.data_as(C.POINTER(C.c_int)))
    return m


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().ora_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def basis(a, x):
    return lib().ora_basis(a, float(x))


def candidate(N, k, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.zeros(N)
    lib().ora_candidate(N, k, _dp(u), _dp(c))
    return c


def beta(N, coef):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    return lib().ora_beta(N, _dp(coef))


def weno1d(N, u, eps, lin, linear_only=False):
    u = np.ascontiguousarray(u, dtype=np.float64)
    lin = np.ascontiguousarray(lin, dtype=np.float64)
    c = np.zeros(N)
    om = np.zeros(N + 1)
    lib().ora_weno1d(N, _dp(u), eps, _dp(lin), int(linear_only), _dp(c), _dp(om))
    return c, om


def mc_slope(a, b, cfac):
    return lib().ora_mc_slope(float(a), float(b), float(cfac))


def hllc(dim, gamma, direction, UL, UR):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(dim + 2)
    lib().ora_hllc(dim, gamma, direction, _dp(UL), _dp(UR), _dp(F))
    return F


RIEMANN = {"hllc": 0, "hll": 1, "hllem": 2, "rusanov": 3}


def riemann(kind, dim, gamma, direction, UL, UR):
    """Numerical flux of one of the Riemann solvers ("hllc", "hll", "hllem",
    "rusanov")."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(dim + 2)
    lib().ora_riemann(RIEMANN[kind], dim, gamma, direction, _dp(UL), _dp(UR), _dp(F))
    return F


def phys_flux(dim, gamma, direction, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(dim + 2)
    lib().ora_phys_flux(dim, gamma, direction, _dp(U), _dp(F))
    return F


def exact_riemann(gamma, left, right, s):
    """Exact solution (rho, u, p) at x/t = s for primitive left/right states;
    also returns (p*, u*)."""
    r, u, p, ps, us = (C.c_double() for _ in range(5))
    rc = lib().ora_exact_riemann(gamma, *left, *right, s, C.byref(r), C.byref(u), C.byref(p),
                                 C.byref(ps), C.byref(us))
    if rc != 0:
        raise ValueError("vacuum generated; not handled")
    return (r.value, u.value, p.value), (ps.value, us.value)


class Oracle:
    """Whole-grid oracle for one problem description (a problems.Problem)."""

    def __init__(self, prob):
        self.prob = prob
        c = OraCfg()
        c.dim = prob.dim
        n = list(prob.n) + [1] * (3 - len(prob.n))
        for d in range(3):
            c.n[d] = n[d]
            c.lo[d] = prob.lo[d] if d < prob.dim else 0.0
            c.hi[d] = prob.hi[d] if d < prob.dim else 1.0
        c.order = prob.order
        c.picard = prob.picard
        c.gamma = prob.gamma
        c.eps = prob.eps
        for k, w in enumerate(prob.lin):
            c.lin[k] = w
        for f in range(6):
            c.bc[f] = BC_CODES[prob.bc[f]]
            st = prob.inflow[f] if prob.inflow[f] is not None else [0.0] * 5
            for v in range(len(st)):
                c.inflow[f][v] = st[v]
        if prob.pre is not None:
            for v in range(len(prob.pre)):
                c.pre[v] = prob.pre[v]
        c.fallback = int(getattr(prob, "fallback", 0) or 0)
        c.riemann = RIEMANN[getattr(prob, "riemann", "hllc")]
        self.cfg = c
        self.dim = prob.dim
        self.nv = prob.dim + 2
        self.N = prob.order - 1
        self.g = prob.order
        self.n = tuple(n)
        self.G = tuple(n[d] + 2 * self.g if d < self.dim else 1 for d in range(3))

    # --- layout helpers -------------------------------------------------
    def embed(self, U):
        """[nv][nz][ny][nx] active state -> ghosted array (ghosts NaN)."""
        Ug = np.full((self.nv, self.G[2], self.G[1], self.G[0]), np.nan)
        g = self.g
        zs = slice(g, g + self.n[2]) if self.dim == 3 else slice(0, 1)
        Ug[:, zs, g:g + self.n[1], g:g + self.n[0]] = U.reshape(self.nv, self.n[2], self.n[1], self.n[0])
        return Ug

    def ghosted(self, U, t):
        Ug = np.ascontiguousarray(self.embed(U))
        lib().ora_fill_ghosts(C.byref(self.cfg), _dp(Ug), float(t))
        return Ug

    # --- method ---------------------------------------------------------
    def step(self, U, t, dt, flags=None):
        """One full step from the active state U at time t; returns
        (U_new, smax, status)."""
        Ug = self.ghosted(U, t)
        out = np.zeros((self.nv, self.n[2], self.n[1], self.n[0]))
        smax = C.c_double()
        rc = lib().ora_step(C.byref(self.cfg), _dp(Ug), float(dt), _up(flags), _dp(out), C.byref(smax))
        return out, smax.value, rc

    def step_ghosted(self, Ug, dt, flags=None):
        """One step on an array whose ghost zones are already filled (for
        instance a window cut out of a larger ghost-filled state): returns
        (U_new of the active zones, smax, status)."""
        Ug = np.ascontiguousarray(Ug, dtype=np.float64)
        assert Ug.shape == (self.nv, self.G[2], self.G[1], self.G[0]), Ug.shape
        out = np.zeros((self.nv, self.n[2], self.n[1], self.n[0]))
        smax = C.c_double()
        rc = lib().ora_step(C.byref(self.cfg), _dp(Ug), float(dt), _up(flags), _dp(out), C.byref(smax))
        return out, smax.value, rc

    # --- Runge-Kutta variant -------------------------------------------
    def rk_stages(self):
        st = getattr(self.prob, "rk_stages", 0)
        return st if st else {2: 2, 3: 3, 4: 5}[self.prob.order]

    def rk_rhs(self, U, t, flags=None):
        """L(U) on the active zones (ghosts filled at time t)."""
        Ug = self.ghosted(U, t)
        L = np.zeros((self.nv, self.n[2], self.n[1], self.n[0]))
        lib().ora_rk_rhs(C.byref(self.cfg), _dp(Ug), _up(flags), _dp(L))
        return L

    def rk_step(self, U, t, dt, gate_params=None, nh=32, stages=None):
        """One SSP Runge-Kutta step: returns (U_new, smax, status)."""
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.nv, self.n[2], self.n[1], self.n[0])
        out = np.zeros_like(U)
        smax = C.c_double()
        gp = None if gate_params is None else np.ascontiguousarray(gate_params, dtype=np.float32)
        rc = lib().ora_rk_step(C.byref(self.cfg), _dp(U), float(t), float(dt), int(stages or self.rk_stages()),
                               nh, _fp(gp), _dp(out), C.byref(smax))
        return out, smax.value, rc

    def signal_max(self, U):
        Ug = self.ghosted(U, 0.0)
        return lib().ora_signal_max(C.byref(self.cfg), _dp(Ug))

    def cfl_dt(self, U, cfl):
        return cfl / self.signal_max(U)

    def box_shape(self):
        return tuple(self.n[d] + 2 if d < self.dim else 1 for d in range(3))

    def reconstruct(self, U, t, flags=None):
        """Spatial modes of the box zones: [nv][nmodes][Bz][By][Bx]."""
        Ug = self.ghosted(U, t)
        B = self.box_shape()
        ns = num_modes(self.dim, self.N)
        W = np.zeros((self.nv, ns, B[2], B[1], B[0]))
        lib().ora_reconstruct(C.byref(self.cfg), _dp(Ug), _up(flags), _dp(W))
        return W

    def face_states(self, U, t, dt, flags=None):
        """[dim][2][nq][nv][Bz][By][Bx]"""
        Ug = self.ghosted(U, t)
        B = self.box_shape()
        nq = ((self.prob.order + 1) // 2) ** self.dim
        FS = np.zeros((self.dim, 2, nq, self.nv, B[2], B[1], B[0]))
        lib().ora_face_states(C.byref(self.cfg), _dp(Ug), _up(flags), float(dt), _dp(FS))
        return FS

    def fallback_count(self, U, t, dt, flags=None):
        """box zones whose face states go to the positivity fallback"""
        Ug = self.ghosted(U, t)
        B = self.box_shape()
        nq = ((self.prob.order + 1) // 2) ** self.dim
        FS = np.zeros((self.dim, 2, nq, self.nv, B[2], B[1], B[0]))
        return lib().ora_face_states(C.byref(self.cfg), _dp(Ug), _up(flags), float(dt), _dp(FS))

    def fluxes(self, U, t, dt, flags=None):
        """List over directions of [nv][Ez][Ey][Ex] face-averaged fluxes."""
        Ug = self.ghosted(U, t)
        shapes = []
        total = 0
        for d in range(self.dim):
            E = list(self.n)
            E[d] += 1
            shapes.append(E)
            total += self.nv * E[0] * E[1] * E[2]
        F = np.zeros(total)
        lib().ora_fluxes(C.byref(self.cfg), _dp(Ug), _up(flags), float(dt), _dp(F))
        out, off = [], 0
        for E in shapes:
            sz = self.nv * E[0] * E[1] * E[2]
            out.append(F[off:off + sz].reshape(self.nv, E[2], E[1], E[0]))
            off += sz
        return out

    def predict_zone(self, w, dt):
        w = np.ascontiguousarray(w, dtype=np.float64)
        st = np.zeros((self.nv, num_st_modes(self.dim, self.N)))
        lib().ora_predict_zone(C.byref(self.cfg), _dp(w), float(dt), _dp(st))
        return st

    # --- gate -----------------------------------------------------------
    def labels(self, U, t, tau):
        Ug = self.ghosted(U, t)
        lab = np.zeros(Ug.shape[1:], dtype=np.uint8)
        lib().ora_weno_labels(C.byref(self.cfg), _dp(Ug), float(tau), _up(lab))
        return lab

    def num_features(self):
        return lib().ora_gate_num_features(self.dim, self.prob.order)

    def features(self, U, t):
        Ug = self.ghosted(U, t)
        nf = self.num_features()
        feat = np.zeros(Ug.shape[1:] + (nf,), dtype=np.float32)
        lib().ora_gate_features(C.byref(self.cfg), _dp(Ug), _fp(feat))
        return feat

    def gate_flags_ghosted(self, Ug, params, nh=32):
        """gate flags of an array whose ghost zones are already filled"""
        Ug = np.ascontiguousarray(Ug, dtype=np.float64)
        params = np.ascontiguousarray(params, dtype=np.float32)
        fl = np.zeros(Ug.shape[1:], dtype=np.uint8)
        lib().ora_gate_flags(C.byref(self.cfg), _dp(Ug), nh, _fp(params), _up(fl))
        return fl

    def gate_flags(self, U, t, params, nh=32):
        Ug = self.ghosted(U, t)
        params = np.ascontiguousarray(params, dtype=np.float32)
        fl = np.zeros(Ug.shape[1:], dtype=np.uint8)
        lib().ora_gate_flags(C.byref(self.cfg), _dp(Ug), nh, _fp(params), _up(fl))
        return fl


def rk_coefficients(stages):
    """Shu-Osher (alpha, beta), each [stages+1][stages]."""
    a = np.zeros((stages + 1) * stages)
    b = np.zeros((stages + 1) * stages)
    if lib().ora_rk_coefficients(stages, _dp(a), _dp(b)) != 0:
        raise ValueError("stages must be 2, 3 or 5")
    return a.reshape(stages + 1, stages), b.reshape(stages + 1, stages)


def mlp_num_params(nin, nh=32):
    return lib().ora_mlp_num_params(nin, nh)


def mlp_forward_f64(params, x, nh=32):
    x = np.ascontiguousarray(x, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    z = np.zeros(x.shape[0])
    lib().ora_mlp_forward_f64(x.shape[1], nh, _fp(params), _fp(x), x.shape[0], _dp(z))
    return z


def mlp_forward_f32(params, x, nh=32):
    x = np.ascontiguousarray(x, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    z = np.zeros(x.shape[0], dtype=np.float32)
    lib().ora_mlp_forward_f32(x.shape[1], nh, _fp(params), _fp(x), x.shape[0], _fp(z))
    return z


def mlp_loss_grad_f64(params, x, y, nh=32):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros(params.size)
    loss = lib().ora_mlp_loss_grad_f64(x.shape[1], nh, _fp(params), _fp(x), _fp(y), x.shape[0], _dp(g))
    return loss, g
