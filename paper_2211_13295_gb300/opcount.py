"""Algorithmic floating-point operation counts of one step, per zone.

Counted from the loop structure of the kernels (csrc/): an FMA counts 2
flops, an add, subtract or multiply 1; divisions and square roots are
counted apart (they are not flops of the FMA pipe).  These are the numerators
of the ALU roofline fractions; they are checked against the executed
FP64/FP32 instruction counts of an ncu capture (profiles/).

Units: the predictor and reconstruction run on the box of zones (active
zones plus one layer per side), the flux kernel on faces, the update on
active zones; :func:`step_flops_per_zone` folds these into flops per active
zone for a given grid.
"""
from __future__ import annotations

from math import comb


def _flux_node(D):
    """phys_fluxes: 1/rho (1 div), velocities D mul, m2 1 mul + (D-1) FMA,
    p = gm1*(E - 0.5*m2): 3, Ep 1, per direction D mul + 1 add + 1 mul."""
    flops = D + 1 + 2 * (D - 1) + 3 + 1 + D * (D + 2)
    return flops, 1


def _hllc(D):
    """HLLC (awe_internal.cuh::hllc), star branch (the costliest): counted
    from the source; 2 div for 1/rho, 1 for Roe denominator, 1 for S*, 1 for
    f, 1 for p/m; 4 sqrt."""
    nv = D + 2
    flops = 0
    flops += 2 * D                       # velocities
    flops += 2 * (1 + 2 * (D - 1))       # kinetic terms
    flops += 2 * 3                       # pressures
    flops += 2 * 2                       # gamma*p*irho
    flops += D * (3 + 2)                 # Roe velocities + |v|^2
    flops += 8                           # Roe enthalpy
    flops += 4                           # c~
    flops += 4                           # S_L, S_R
    flops += 4                           # m_l, m_r
    flops += 7                           # S*
    flops += 2                           # S - S*
    flops += 3                           # mass flux
    flops += D * 5                       # momentum fluxes
    flops += 1                           # + p
    flops += 9                           # energy star state + flux
    divs = 6 + 4                         # divisions + square roots
    return flops + 0 * nv, divs


def _weno(N, linear):
    """weno1d: 2N differences (counted by the caller), candidates, beta,
    FP64 weights (product form), combination.  N = 1 (order 2): the MC
    limiter of Fig. 3 (sum, three scaled magnitudes, two minima, the sign
    factor and its product)."""
    if N == 1:
        return 8, 0
    # candidate stencils: number of nonzero weights per coefficient
    terms = {2: [2, 2, 2, 2, 2, 2], 3: [3, 3, 3, 3, 2, 3, 3, 2, 3, 3, 3, 3]}[N]
    cand = sum(1 + 2 * (t - 1) for t in terms)
    if linear:
        beta = wts = 0
        divs = 0
    else:
        beta = (N + 1) * (4 if N == 2 else 8)
        wts = (N + 1) * 2 + (6 if N == 2 else 10) + N + (N + 1)
        divs = 1
    comb_ = N * (1 + 2 * N)
    return cand + beta + wts + comb_, divs


def recon_flops(D, N, gated_linear_fraction=0.0):
    """flops per box zone of the three reconstruction passes, including the
    extra zones of the pass regions (returned as (per-box-zone at the given
    region ratios, divs)); region ratios are applied by the caller."""
    nv = D + 2
    nl, dl = _weno(N, True)
    nn, dn = _weno(N, False)
    per_call = (1 - gated_linear_fraction) * nn + gated_linear_fraction * nl + 2 * N
    per_div = (1 - gated_linear_fraction) * dn
    # calls per zone and variable in each pass
    x_calls = 1
    y_calls = 1 + (N - 1)                       # recon_y(U), recon_y(X[a]) a < N
    # recon_z(U), recon_z(X[a]) and recon_z(Y[a]) for a < N, recon_z(XY[a][b])
    # for a, b >= 1 with a + b < N
    z_calls = 0 if D == 2 else 1 + 2 * (N - 1) + (N - 1) * (N - 2) // 2
    return {"x": (nv * x_calls * per_call, nv * x_calls * per_div),
            "y": (nv * y_calls * per_call, nv * y_calls * per_div),
            "z": (nv * z_calls * per_call, nv * z_calls * per_div)}


def _mass_gmode_flops(emax, D=3, N=3):
    """mass row of G from the momentum's coefficients (awe_predict.cu::
    mass_gmode, mass_gmode_direct), over the G-modes (a, b, c, e) with
    a+b+c+e <= N-1, e <= emax: per direction the derivative's one or two
    source modes (the coefficient of L_e: 2 FMA for e = 0, FMA + mul for
    e = 1, mul for e = 2; an FMA into the direction's sum), then an FMA with
    lambda_d."""
    flops = 0
    cmax = N - 1 if D == 3 else 0
    for e in range(emax + 1):
        for c in range(cmax + 1):
            for b in range(N):
                for a in range(N):
                    if a + b + c + e > N - 1:
                        continue
                    for d in range(D):
                        abc = [a, b, c]
                        for k in range(2):
                            ad = abc[d]
                            if k == 1 and ad != 0:
                                break
                            src = list(abc)
                            src[d] = ad + 1 if k == 0 else 3
                            if sum(src) + e > N:
                                continue
                            flops += (4 if e == 0 else 3 if e == 1 else 1) + 2
                        flops += 2
    return flops


def predictor_flops(D, N, picard):
    """flops and divs per box zone of the predictor kernel."""
    nv = D + 2
    fn, fd = _flux_node(D)
    if D == 3 and N == 3:
        # factorised kernel (awe_predict.cu::k_predict_fact)
        fma = 0
        fma += 4 * 5 * 20 + 16 * 5 * 10 + 64 * 5 * 4       # w at the spatial nodes
        flops = 2 * fma
        divs = 0
        # P1, P2 and P3 project the momentum and energy rows (4 variables);
        # the mass row comes from the momentum's coefficients (mass_gmode).
        # P1 runs once per distinct flux entry (9 row sets: the off-diagonal
        # momentum flux serves two directions), P2 per (direction, variable)
        if picard >= 1:
            flops += 64 * fn
            divs += 64 * fd
            flops += 2 * (9 * 16 * 3 * 4 + 12 * 4 * 6 * 4)         # P1, P2 with e = 0
            flops += 4 * 10 * 3 * 4 * 3                                # P3 (mul + FMA)
            flops += _mass_gmode_flops(0)
        for _ in range(1, picard):
            flops += 2 * (5 * 4 * 15 + 5 * 4 * 4 * 10 + 5 * 16 * 4 * 6)   # E1, E2, E3
            # nodes: q and the 9 distinct momentum and energy flux entries
            # (the momentum flux is symmetric: 24 flops and a division) at 4
            # time points, then the time contraction over the 2 symmetric
            # pairs (sum and difference: 18 adds, 27 FMA)
            flops += 64 * (4 * (2 * 5 * 3 + 24) + 2 * (18 + 2 * 27))
            divs += 64 * 4 * fd
            flops += 2 * (9 * 16 * 6 * 4 + 12 * 4 * 10 * 4)               # P1, P2
            flops += 4 * 15 * 3 * 4 * 3                                     # P3
            flops += _mass_gmode_flops(2)
        # face states (factorised): G integrated at the two face times
        # (5 x 2 x 15 FMA), then per (variable, direction, side) the normal axis,
        # the two transverse axes and the time points: 124 FMA + 8 adds
        flops += 2 * 150 + 30 * (2 * 124 + 8)
        return flops, divs
    # direct kernel (awe_predict.cu::k_predict_direct)
    NS = comb(N + D, D)
    NG = comb(N - 1 + D + 1, D + 1)
    NG0 = comb(N - 1 + D, D)
    NN = N + 1
    NSN = NN ** D
    nq = (N + 2) // 2
    NFQ = nq ** D
    flops = divs = 0
    # the node fluxes are projected for the momentum and energy rows (nv - 1);
    # the mass row comes from the momentum's coefficients (mass_gmode_direct)
    if picard >= 1:
        flops += NSN * (2 * nv * NS + fn + D * (nv - 1) * (1 + 2 * NG0))
        flops += _mass_gmode_flops(0, D, N)
        divs += NSN * fd
    npair, nmid = NN // 2, NN % 2
    for _ in range(1, picard):
        flops += NSN * 2 * nv * NS
        flops += NSN * NN * (2 * nv * NG + fn)
        # time contraction: a symmetric pair of time nodes enters through the
        # sum and the difference of its scaled fluxes (2 adds, 2 mul, NG FMA
        # per flux entry), the middle node of an odd rule alone (1 mul, NG FMA)
        flops += NSN * D * (nv - 1) * (npair * (4 + 2 * NG) + nmid * (1 + 2 * NG))
        flops += _mass_gmode_flops(N - 1, D, N)
        divs += NSN * NN * fd
    # face states: the w part once per spatial face point, the G part per
    # space-time point
    flops += D * 2 * (NFQ // nq) * nv * 2 * NS + D * 2 * NFQ * nv * 2 * NG
    return flops, divs


def flux_flops(D, N=2):
    """flops and divs+sqrt per face of the flux kernel (Gauss points per face:
    1 at order 2, 2 per transverse dimension and in time at orders 3 and 4)."""
    nfq = ((N + 2) // 2) ** D
    h, hd = _hllc(D)
    return nfq * (h + 2 * (D + 2)), nfq * hd


def update_flops(D):
    """per active zone: flux differences and the signal speed (FP64)."""
    nv = D + 2
    return nv * (3 * D) + (2 + 2 * D + 3 + 2 + 3 * D), 2


def step_flops_per_zone(prob, picard=None, gate_linear_fraction=0.0):
    """dict of (flops, divs) per active zone and stage for one step of prob."""
    D, N = prob.dim, prob.order - 1
    picard = prob.order - 1 if picard is None else picard
    n = [prob.n[d] if d < D else 1 for d in range(3)]
    nact = n[0] * n[1] * n[2]
    box = (n[0] + 2) * (n[1] + 2) * (n[2] + 2 if D == 3 else 1)
    rx = (n[0] + 2) * (n[1] + 2 + 2 * N) * ((n[2] + 2 + 2 * N) if D == 3 else 1)
    ry = (n[0] + 2) * (n[1] + 2) * ((n[2] + 2 + 2 * N) if D == 3 else 1)
    rec = recon_flops(D, N, gate_linear_fraction)
    out = {
        "recon_x": (rec["x"][0] * rx / nact, rec["x"][1] * rx / nact),
        "recon_y": (rec["y"][0] * ry / nact, rec["y"][1] * ry / nact),
        "recon_z": (rec["z"][0] * box / nact, rec["z"][1] * box / nact),
    }
    pf, pd = predictor_flops(D, N, picard)
    out["predictor"] = (pf * box / nact, pd * box / nact)
    ff, fd = flux_flops(D, N)
    nfaces = sum((n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2)) for d in range(D))
    out["riemann_flux"] = (ff * nfaces / nact, fd * nfaces / nact)
    uf, ud = update_flops(D)
    out["update_cfl"] = (uf, ud)
    return out


def predictor_flops_per_launch(prob, picard=None):
    """algorithmic flops of one predictor launch over the whole box"""
    D, N = prob.dim, prob.order - 1
    picard = prob.order - 1 if picard is None else picard
    n = [prob.n[d] if d < D else 1 for d in range(3)]
    box = (n[0] + 2) * (n[1] + 2) * (n[2] + 2 if D == 3 else 1)
    return predictor_flops(D, N, picard)[0] * box


def predictor_source_sha():
    """Short hash of the predictor kernel's sources: a DRAM-traffic figure
    measured by ncu on one version of the kernel is only reported while the
    sources it was measured on are unchanged."""
    import hashlib
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    h = hashlib.sha256()
    for name in ("awe_predict.cu", "predict_index.cuh", "awe_internal.cuh"):
        with open(os.path.join(here, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]
