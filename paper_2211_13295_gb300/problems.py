"""Seeded synthetic inputs: problem descriptions and initial conditions.

This module serves both the CUDA path (tests, bench) and the CPU oracle.  It
holds none of the method's arithmetic (no reconstruction, predictor, Riemann
solver or update): only domain/BC/order descriptions and zone averages of
analytic initial states.  Zone averages are taken with a tensor Gauss-Legendre
rule (smooth states), exactly (Taylor-Green, separable trigonometric products)
or by sub-zone sampling (states with discontinuities).

The problems are the standard test problems the workloads are built on (the
paper names only the 3D isentropic vortex of its accuracy study, Sec. IV.1,
Table XII; the rest are synthetic stand-ins of the stated shapes and sizes):

* ``vortex2d``   isentropic vortex (strength 5) advected diagonally on [0,10]^2
* ``sod``        Sod shock tube along x on a thin 2D strip
* ``tgv3d``      Taylor-Green vortex on [0, 2 pi]^3, p0 = 100/gamma
* ``dmr``        double Mach reflection (Mach 10 shock at 60 degrees)
* ``blast3d``    spherical blast (Sod in a box) with a seeded density perturbation
* ``kh3d``       Kelvin-Helmholtz shear layer with a seeded velocity perturbation
* ``uniform``    free stream (any dim)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

LINEAR_WEIGHTS = {2: (0.0, 0.0),  # order 2 uses the MC limiter, not WENO
                  3: (1.0 / 102.0, 100.0 / 102.0, 1.0 / 102.0),
                  4: (1.0 / 22.0, 10.0 / 22.0, 10.0 / 22.0, 1.0 / 22.0)}


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    order: int
    gamma: float = 1.4
    bc: tuple = ("periodic",) * 6
    inflow: tuple = (None,) * 6          # conserved state per face (inflow / DMR post-shock)
    pre: Optional[tuple] = None          # DMR pre-shock conserved state
    cfl: float = 0.4
    t_end: Optional[float] = None
    steps: Optional[int] = None
    eps: float = 1e-12
    lin: tuple = ()
    picard: int = 0
    seed: Optional[int] = None
    fallback: int = 0                    # opt-in positivity fallback: 1 face states, 2 also a posteriori
    riemann: str = "hllc"                # corrector's Riemann solver: hllc, hll, hllem, rusanov
    scheme: str = "ader"                 # time stepping: ader, or ssprk (Table IV's comparison)
    rk_stages: int = 0                   # SSP-RK stages (2, 3, 5); 0: 2, 3, 5 at orders 2, 3, 4
    params: dict = dataclasses.field(default_factory=dict)
    dxs: tuple = ()                      # zone sizes, if not (hi - lo) / n (subdomains)

    def __post_init__(self):
        if not self.lin:
            self.lin = LINEAR_WEIGHTS[self.order]
        if self.picard == 0:
            self.picard = self.order - 1
        self.n = tuple(int(v) for v in self.n)

    @property
    def nv(self):
        return self.dim + 2

    @property
    def zones(self):
        return int(np.prod(self.n[: self.dim]))

    def dx(self, d):
        if self.dxs:
            return self.dxs[d]
        return (self.hi[d] - self.lo[d]) / self.n[d]

    def shape(self):
        nz = self.n[2] if self.dim == 3 else 1
        return (self.nv, nz, self.n[1], self.n[0])

    def initial_state(self) -> np.ndarray:
        return _IC[self.name](self)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# primitive -> conserved (equation of state of the inputs)
# ---------------------------------------------------------------------------
def conserved(gamma, rho, vel, p):
    """Conserved (rho, rho v..., E) from primitive values (ideal gas)."""
    kin = 0.0
    for v in vel:
        kin = kin + 0.5 * rho * v * v
    return [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + kin]


def _centers(prob, d):
    h = prob.dx(d)
    return prob.lo[d] + (np.arange(prob.n[d]) + 0.5) * h


def _gl(nq):
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * x, 0.5 * w


def _average_2d(prob, fn, nq=6):
    """Zone averages of conserved fn(x, y) -> list of arrays, tensor GL."""
    xq, wq = _gl(nq)
    xc, yc = _centers(prob, 0), _centers(prob, 1)
    hx, hy = prob.dx(0), prob.dx(1)
    out = np.zeros(prob.shape())
    for a in range(nq):
        for b in range(nq):
            X = (xc + xq[a] * hx)[None, :]
            Y = (yc + xq[b] * hy)[:, None]
            vals = fn(X, Y)
            for v in range(prob.nv):
                out[v, 0] += wq[a] * wq[b] * np.broadcast_to(vals[v], (prob.n[1], prob.n[0]))
    return out


# ---------------------------------------------------------------------------
# 2D isentropic vortex
# ---------------------------------------------------------------------------
def vortex2d(n=64, order=3, cfl=0.4, t_end=1.0, strength=5.0) -> Problem:
    """Isentropic vortex of the given strength at (5,5) in a (1,1) free stream,
    periodic [0,10]^2 (the exact solution is the initial state shifted by t*(1,1))."""
    return Problem("vortex2d", 2, (n, n, 1), (0.0, 0.0, 0.0), (10.0, 10.0, 1.0), order,
                   cfl=cfl, t_end=t_end, params={"strength": strength})


def _vortex_fn(prob, t=0.0):
    g = prob.gamma
    eps = prob.params.get("strength", 5.0)
    L = 10.0

    def fn(X, Y):
        # position relative to the advected centre, wrapped into [-5, 5)
        xr = np.mod(X - 5.0 - t + 0.5 * L, L) - 0.5 * L
        yr = np.mod(Y - 5.0 - t + 0.5 * L, L) - 0.5 * L
        r2 = xr * xr + yr * yr
        f = np.exp(0.5 * (1.0 - r2))
        du = -eps / (2.0 * math.pi) * f * yr
        dv = eps / (2.0 * math.pi) * f * xr
        T = 1.0 - (g - 1.0) * eps * eps * np.exp(1.0 - r2) / (8.0 * g * math.pi ** 2)
        rho = T ** (1.0 / (g - 1.0))
        p = rho ** g
        return conserved(g, rho, [1.0 + du, 1.0 + dv], p)

    return fn


def vortex_exact(prob, t, nq=6):
    return _average_2d(prob, _vortex_fn(prob, t), nq)


# ---------------------------------------------------------------------------
# Sod shock tube along x
# ---------------------------------------------------------------------------
SOD_LEFT = (1.0, 0.0, 1.0)     # rho, u, p
SOD_RIGHT = (0.125, 0.0, 0.1)


def sod(nx=400, ny=4, order=3, cfl=0.4, t_end=0.2) -> Problem:
    h = 1.0 / nx
    return Problem("sod", 2, (nx, ny, 1), (0.0, 0.0, 0.0), (1.0, ny * h, 1.0), order,
                   bc=("outflow", "outflow", "periodic", "periodic", "periodic", "periodic"),
                   cfl=cfl, t_end=t_end)


def _sod_ic(prob):
    g = prob.gamma
    x = _centers(prob, 0)
    out = np.zeros(prob.shape())
    left = x < 0.5
    for side, st in ((left, SOD_LEFT), (~left, SOD_RIGHT)):
        c = conserved(g, st[0], [st[1], 0.0], st[2])
        for v in range(4):
            out[v, 0, :, side] = c[v]
    return out


# ---------------------------------------------------------------------------
# 3D Taylor-Green vortex (exact zone averages: separable products)
# ---------------------------------------------------------------------------
def tgv3d(n=256, order=4, cfl=0.3, steps=100, nz=None) -> Problem:
    """Taylor-Green vortex on [0, 2 pi]^3 with n^3 zones; nz > n stacks nz / n
    periods along z (the same zone size), the grid of a z-slab decomposition
    that gives every rank an n^3 slab."""
    L = 2.0 * math.pi
    nz = n if nz is None else nz
    return Problem("tgv3d", 3, (n, n, nz), (0.0, 0.0, 0.0), (L, L, L * nz / n), order, cfl=cfl, steps=steps)


def _avg_trig(c, h, kind, k=1.0):
    """Average over [c-h/2, c+h/2] of sin(kx) / cos(kx)."""
    s = np.sinc(k * h / (2.0 * math.pi))  # sin(kh/2)/(kh/2)
    return (np.sin(k * c) if kind == "sin" else np.cos(k * c)) * s


def _tgv_ic(prob):
    g = prob.gamma
    n = prob.n
    xs = [_centers(prob, d) for d in range(3)]
    hs = [prob.dx(d) for d in range(3)]
    S = [_avg_trig(xs[d], hs[d], "sin") for d in range(3)]
    Co = [_avg_trig(xs[d], hs[d], "cos") for d in range(3)]
    C2 = [_avg_trig(xs[d], hs[d], "cos", 2.0) for d in range(3)]
    sin2 = [0.5 - 0.5 * C2[d] for d in range(3)]
    cos2 = [0.5 + 0.5 * C2[d] for d in range(3)]

    def outer(fx, fy, fz):
        return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]

    out = np.zeros(prob.shape())
    out[0] = 1.0
    out[1] = outer(S[0], Co[1], Co[2])
    out[2] = -outer(Co[0], S[1], Co[2])
    out[3] = 0.0
    p = 100.0 / g + (1.0 / 16.0) * (C2[0][None, None, :] + C2[1][None, :, None]) * (C2[2][:, None, None] + 2.0)
    kin = 0.5 * (outer(sin2[0], cos2[1], cos2[2]) + outer(cos2[0], sin2[1], cos2[2]))
    out[4] = p / (g - 1.0) + kin
    return out


# ---------------------------------------------------------------------------
# Double Mach reflection
# ---------------------------------------------------------------------------
def dmr(nx=4096, ny=1024, order=3, cfl=0.4, t_end=0.2) -> Problem:
    g = 1.4
    a = math.radians(30.0)
    post = tuple(conserved(g, 8.0, [8.25 * math.cos(a), -8.25 * math.sin(a)], 116.5))
    pre = tuple(conserved(g, 1.4, [0.0, 0.0], 1.0))
    return Problem("dmr", 2, (nx, ny, 1), (0.0, 0.0, 0.0), (4.0, 1.0, 1.0), order, gamma=g,
                   bc=("inflow", "outflow", "dmr_bottom", "dmr_top", "periodic", "periodic"),
                   inflow=(post, None, post, post, None, None), pre=pre, cfl=cfl, t_end=t_end)


def _dmr_ic(prob, nsub=8):
    post, pre = np.array(prob.inflow[0]), np.array(prob.pre)
    hx, hy = prob.dx(0), prob.dx(1)
    xc, yc = _centers(prob, 0), _centers(prob, 1)
    sub = (np.arange(nsub) + 0.5) / nsub - 0.5
    out = np.zeros(prob.shape())
    for j0 in range(0, prob.n[1], 64):
        ys = yc[j0:j0 + 64]
        frac = np.zeros((len(ys), prob.n[0]))
        for a in sub:
            for b in sub:
                X = (xc + a * hx)[None, :]
                Y = (ys + b * hy)[:, None]
                frac += (X < 1.0 / 6.0 + Y / math.sqrt(3.0))
        frac /= nsub * nsub
        for v in range(4):
            out[v, 0, j0:j0 + 64] = frac * post[v] + (1.0 - frac) * pre[v]
    return out


# ---------------------------------------------------------------------------
# seeded smooth periodic perturbation (sum of Fourier modes)
# ---------------------------------------------------------------------------
def fourier_modes(seed, nmodes=8, kmax=4):
    rng = np.random.default_rng(seed)
    ks, phases = [], []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(k != 0) and np.sqrt((k * k).sum()) <= kmax:
            ks.append(k.astype(np.float64))
            phases.append(rng.uniform(0.0, 2.0 * math.pi))
    return np.array(ks), np.array(phases)


def _perturbation_avg(prob, seed, k_axes=(0, 1, 2)):
    """Zone average on the unit box of f = sum_m sin(2 pi k_m . x + phi_m) / nmodes
    (normalised so that |f| <= 1), exact per mode (product of sinc factors)."""
    ks, ph = fourier_modes(seed)
    xs = [_centers(prob, d) for d in range(3)]
    hs = [prob.dx(d) for d in range(3)]
    f = np.zeros(prob.shape()[1:])
    for k, phi in zip(ks, ph):
        w = 2.0 * math.pi * k
        arg = (w[0] * xs[0])[None, None, :] + (w[1] * xs[1])[None, :, None] + (w[2] * xs[2])[:, None, None] + phi
        damp = np.sinc(w[0] * hs[0] / (2 * math.pi)) * np.sinc(w[1] * hs[1] / (2 * math.pi)) * \
            np.sinc(w[2] * hs[2] / (2 * math.pi))
        f += damp * np.sin(arg)
    return f / len(ks)


# ---------------------------------------------------------------------------
# 3D blast (Sod in a box)
# ---------------------------------------------------------------------------
def blast3d(n=384, order=4, cfl=0.15, steps=None, seed=2211) -> Problem:
    """Blast (Sod in a box).  CFL 0.15: below 1/6, where the first-order
    update of the positivity fallback stays positive in 3D."""
    return Problem("blast3d", 3, (n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), order,
                   bc=("outflow",) * 6, cfl=cfl, steps=steps, seed=seed)


def _blast_ic(prob, nsub=8):
    g = prob.gamma
    n = prob.n
    xs = [_centers(prob, d) for d in range(3)]
    h = prob.dx(0)
    # volume fraction inside the sphere: exact for zones wholly inside/outside,
    # nsub^3 sub-zone samples for zones cut by the surface
    X, Y, Z = xs[0][None, None, :], xs[1][None, :, None], xs[2][:, None, None]
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    half_diag = math.sqrt(3.0) * 0.5 * h
    frac = (r < 0.2).astype(np.float64)
    cut = np.abs(r - 0.2) <= half_diag
    idx = np.argwhere(cut)
    sub = (np.arange(nsub) + 0.5) / nsub - 0.5
    sx, sy, sz = np.meshgrid(sub, sub, sub, indexing="ij")
    for (k, j, i) in idx:
        px = xs[0][i] + sx * h - 0.5
        py = xs[1][j] + sy * h - 0.5
        pz = xs[2][k] + sz * h - 0.5
        frac[k, j, i] = np.mean(px * px + py * py + pz * pz < 0.04)
    rho0 = frac * 1.0 + (1.0 - frac) * 0.125
    p = frac * 10.0 + (1.0 - frac) * 0.1
    f = _perturbation_avg(prob, prob.seed)
    rho = rho0 * (1.0 + 1e-2 * f)
    out = np.zeros(prob.shape())
    out[0] = rho
    out[4] = p / (g - 1.0)
    return out


# ---------------------------------------------------------------------------
# 3D Kelvin-Helmholtz shear layer
# ---------------------------------------------------------------------------
def kh3d(n=512, order=4, cfl=0.3, steps=None, seed=2212) -> Problem:
    return Problem("kh3d", 3, (n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), order, cfl=cfl,
                   steps=steps, seed=seed)


def _kh_ic(prob, nsub=8):
    g = prob.gamma
    yc = _centers(prob, 1)
    h = prob.dx(1)
    sub = (np.arange(nsub) + 0.5) / nsub - 0.5
    inner = np.zeros_like(yc)
    for s in sub:
        inner += np.abs(yc + s * h - 0.5) < 0.25
    inner /= nsub                                   # fraction of the zone in the dense band
    rho = (inner * 2.0 + (1.0 - inner) * 1.0)[None, :, None]
    mx = (inner * 2.0 * 0.5 + (1.0 - inner) * 1.0 * -0.5)[None, :, None]
    vy = 1e-2 * _perturbation_avg(prob, prob.seed)
    out = np.zeros(prob.shape())
    out[0] = rho
    out[1] = mx
    out[2] = rho * vy
    kin = 0.5 * (mx * mx / rho + rho * vy * vy)
    out[4] = 2.5 / (g - 1.0) + kin
    return out


# ---------------------------------------------------------------------------
# 3D density wave advected along the diagonal (smooth; exact solution known)
# ---------------------------------------------------------------------------
def wave3d(n=32, order=4, cfl=0.3, t_end=0.1, amp=0.2, vel=(1.0, 1.0, 1.0)) -> Problem:
    """rho = 1 + amp sin(2 pi (x + y + z)), constant velocity and pressure p = 1 on
    the periodic unit cube: an isolated contact whose exact solution at time t
    is the initial state moved by vel * t.  Every mixed derivative of the
    density is non-zero, so all cross modes of the reconstruction take part."""
    return Problem("wave3d", 3, (n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), order, cfl=cfl,
                   t_end=t_end, params={"amp": amp, "vel": tuple(vel)})


def wave3d_exact(prob, t):
    """Zone averages of the exact state at time t (products of sinc factors)."""
    amp, vel = prob.params["amp"], prob.params["vel"]
    w = 2.0 * math.pi
    xs = [_centers(prob, d) - vel[d] * t for d in range(3)]
    hs = [prob.dx(d) for d in range(3)]
    damp = 1.0
    for d in range(3):
        damp *= np.sinc(w * hs[d] / (2.0 * math.pi))
    arg = (w * xs[0])[None, None, :] + (w * xs[1])[:, None][None] + (w * xs[2])[:, None, None]
    rho = 1.0 + amp * damp * np.sin(arg)
    out = np.zeros(prob.shape())
    out[0] = rho
    for d in range(3):
        out[1 + d] = rho * vel[d]
    kin = 0.5 * sum(v * v for v in vel)
    out[4] = 1.0 / (prob.gamma - 1.0) + kin * rho
    return out


# ---------------------------------------------------------------------------
# free stream
# ---------------------------------------------------------------------------
def uniform(dim=2, n=16, order=3, rho=1.0, vel=(0.3, -0.2, 0.1), p=1.0, bc="periodic") -> Problem:
    nn = (n, n, n if dim == 3 else 1)
    return Problem("uniform", dim, nn, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), order, bc=(bc,) * 6,
                   params={"rho": rho, "vel": tuple(vel[:dim]), "p": p})


def _uniform_ic(prob):
    c = conserved(prob.gamma, prob.params["rho"], list(prob.params["vel"]), prob.params["p"])
    out = np.zeros(prob.shape())
    for v in range(prob.nv):
        out[v] = c[v]
    return out


_IC = {
    "vortex2d": lambda p: _average_2d(p, _vortex_fn(p, 0.0)),
    "sod": _sod_ic,
    "tgv3d": _tgv_ic,
    "dmr": _dmr_ic,
    "blast3d": _blast_ic,
    "kh3d": _kh_ic,
    "uniform": _uniform_ic,
    "wave3d": lambda p: wave3d_exact(p, 0.0),
}


def by_name(name: str, **kw) -> Problem:
    return {"vortex2d": vortex2d, "sod": sod, "tgv3d": tgv3d, "dmr": dmr, "blast3d": blast3d,
            "kh3d": kh3d, "uniform": uniform, "wave3d": wave3d}[name](**kw)
