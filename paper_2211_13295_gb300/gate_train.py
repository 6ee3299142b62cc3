"""Training of the troubled-zone gate on the GPU, with the library's own
kernels (features, labels, forward/backward, Adam).

Labels are produced by the method itself: a zone is troubled when the WENO
nonlinear weights of its pure-direction reconstruction deviate from the
linear weights by more than tau (awe_gate_labels).  Training states come
from short seeded runs of smooth and discontinuous problems (vortex, Sod,
blast, Kelvin-Helmholtz); every zone with a full stencil is one example.
"""
from __future__ import annotations

import numpy as np

from . import awe
from . import problems as P


def he_init(nin, seed, nh=32):
    """He-normal initial parameters in the packed layout (W1, b1, W2, b2, w3, b3)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / nin), size=(nh, nin))
    W2 = rng.normal(0.0, np.sqrt(2.0 / nh), size=(nh, nh))
    w3 = rng.normal(0.0, np.sqrt(2.0 / nh), size=nh)
    return np.concatenate([W1.ravel(), np.zeros(nh), W2.ravel(), np.zeros(nh), w3, [0.0]]).astype(np.float32)


def default_problems(dim, order, n):
    if dim == 2:
        return [P.vortex2d(n=n, order=order), P.sod(nx=n, ny=8, order=order),
                P.sod(nx=n, ny=8, order=order).replace(name="sod")]
    return [P.tgv3d(n=n, order=order, cfl=0.3), P.blast3d(n=n, order=order), P.kh3d(n=n, order=order)]


def collect(probs, steps=(0, 3, 8), tau=0.1, prec="fp64"):
    """features/labels (torch CUDA tensors) from states of short GPU runs;
    runs stop early (and keep what they have) if a state becomes non-physical."""
    import torch
    X, Y = [], []
    for prob in probs:
        g = awe.Grid(prob, prec=prec)
        g.set_state(prob.initial_state())
        g.cfl_dt()
        done = 0
        for k in range(max(steps) + 1):
            if k in steps:
                nin, _ = awe.gate_dims(prob.dim, prob.order)
                feat = torch.empty(g.ghosted_shape + (nin,), dtype=torch.float32, device="cuda")
                lab = torch.empty(g.ghosted_shape, dtype=torch.uint8, device="cuda")
                g.gate_features(feat)
                g.gate_labels(tau, lab)
                keep = lab.reshape(-1) != 255
                X.append(feat.reshape(-1, nin)[keep])
                Y.append(lab.reshape(-1)[keep].float())
                done += 1
            try:
                g.step(0.0)
            except awe.AweError:
                break
        g.close()
    return torch.cat(X), torch.cat(Y)


def train(X, Y, nin, steps=1500, batch=4096, lr=1e-3, seed=2211, balance=True):
    """Adam on the mean logistic loss; returns (params numpy, loss history).
    With balance, the rarer class is repeated so that both classes are drawn
    about equally often."""
    import torch
    if balance:
        pos = Y > 0.5
        npos, nneg = int(pos.sum()), int((~pos).sum())
        if npos and nneg:
            rep = max(1, nneg // max(npos, 1)) if npos < nneg else 1
            repn = max(1, npos // max(nneg, 1)) if nneg < npos else 1
            X = torch.cat([X[~pos]] * repn + [X[pos]] * rep)
            Y = torch.cat([Y[~pos]] * repn + [Y[pos]] * rep)
    X = X.contiguous()
    Y = Y.contiguous()
    p = torch.from_numpy(he_init(nin, seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.zeros(steps, dtype=torch.float32, device="cuda")
    awe.mlp_train(nin, p, m, v, X, Y, batch, steps, 0, lr, seed, loss)
    torch.cuda.synchronize()
    return p.cpu().numpy(), loss.cpu().numpy()


def accuracy(params, X, Y, nin):
    import torch
    z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    awe.mlp_forward(nin, torch.from_numpy(params).cuda(), X.contiguous(), z)
    pred = (z > 0).float()
    tp = float(((pred > 0.5) & (Y > 0.5)).sum())
    recall = tp / max(float((Y > 0.5).sum()), 1.0)
    acc = float((pred == Y).float().mean())
    return acc, recall, float(pred.mean())
