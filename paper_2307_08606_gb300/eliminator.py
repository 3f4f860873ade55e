"""Training of the learned elimination proposal (criterion elim = 2; an
extension of Algorithm 1, which the paper does not have).

Data come from plain SADMM runs (elim = 0) of the library's own solver: at
every learn point t (a multiple of learn_every, t >= max(Kp, 4)) the six
features of sadmm_features are recorded, and pixel i is labelled droppable
when no sensor's iterate moves by more than Kp * eps_p for the rest of the run:
    label_i(t) = [ max_q max_{t' > t} |x_qi^(t') - x_qi^(t)| <= Kp * eps_p ].
Training minimises the weighted binary cross-entropy of the network with the
library's backward kernels and Adam steps (sadmm_cnn_backward / _adam_step).
Everything here is host orchestration; the arithmetic runs in the library.
"""
from dataclasses import dataclass

import numpy as np

from . import binding


@dataclass
class Samples:
    features: np.ndarray    # (n, 6, H, W) float32
    labels: np.ndarray      # (n, H, W) float32 in {0, 1}
    ks: list                # learn point of each sample


def plain_trajectory(solver, y, iters, learn_every=10):
    """Runs `iters` plain iterations one at a time on `solver` (created with
    elim = 0).  Returns (ks, features at each learn point (n, 6, N), stacked
    iterates X^(0..iters) (iters + 1, Q, N))."""
    Kp = solver.crit.Kp
    solver.solve(y, 0)
    X = [solver.X()]
    ks, feats = [], []
    for k in range(1, iters + 1):
        solver.resume(1)
        X.append(solver.X())
        if k % learn_every == 0 and k >= max(Kp, 4):
            ks.append(k)
            feats.append(solver.features())
    return ks, np.stack(feats) if feats else np.zeros((0, 6, solver.N), np.float32), np.stack(X)


def labels(X, ks, Kp, eps_p, horizon):
    """Droppable flags (len(ks), N) for learn points with at least `horizon`
    later iterates; returns (kept indices into ks, labels)."""
    keep, out = [], []
    T = X.shape[0] - 1
    for n, k in enumerate(ks):
        if T - k < horizon:
            continue
        dev = np.max(np.abs(X[k + 1:] - X[k][None]), axis=(0, 1))
        keep.append(n)
        out.append((dev <= Kp * eps_p).astype(np.float32))
    return keep, (np.stack(out) if out else np.zeros((0, X.shape[2]), np.float32))


def collect(scenes, lam_of, H, W, iters, learn_every=10, horizon=50, rho=1.0, **criterion):
    """Samples from plain runs on `scenes` (objects with geom, A, y);
    lam_of(scene) gives each scene's lambda."""
    F, L, K = [], [], []
    for sc in scenes:
        g = sc.geom
        s = binding.Solver(g.Q, g.M, g.K, g.N, rho, lam_of(sc), elim=0, **criterion)
        for q in range(g.Q):
            s.set_operator(q, sc.A[q])
        ks, feats, X = plain_trajectory(s, sc.y, iters, learn_every)
        keep, lab = labels(X, ks, s.crit.Kp, s.crit.eps_p, horizon)
        F.append(feats[keep].reshape(len(keep), 6, H, W))
        L.append(lab.reshape(len(keep), H, W))
        K += [ks[i] for i in keep]
        s.close()
    return Samples(np.concatenate(F), np.concatenate(L), K)


def collect_on(solver, ys, lams, H, W, iters, learn_every=10, horizon=50):
    """Samples from plain runs of several scenes of one geometry on one solver
    (created with elim = 0, operators set): the factorisation is shared, each
    scene sets its own measurements y and lambda (sadmm_set_lambda)."""
    F, L, K = [], [], []
    for y, lam in zip(ys, lams):
        solver.set_lambda(lam)
        ks, feats, X = plain_trajectory(solver, y, iters, learn_every)
        keep, lab = labels(X, ks, solver.crit.Kp, solver.crit.eps_p, horizon)
        F.append(feats[keep].reshape(len(keep), 6, H, W))
        L.append(lab.reshape(len(keep), H, W))
        K += [ks[i] for i in keep]
    return Samples(np.concatenate(F), np.concatenate(L), K)


def train(net, samples, steps, lr=1e-3, batch=8, pos_weight=1.0, seed=0):
    """Adam on the network `net` (binding.CNN, max_batch >= batch) over random
    mini-batches of `samples`; returns the loss of every step."""
    import torch
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(samples.features)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(samples.labels)).to(dev)
    n = Xd.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(steps):
        idx = torch.from_numpy(rng.choice(n, size=min(batch, n), replace=False)).to(dev)
        xb, yb = Xd[idx].contiguous(), Yd[idx].contiguous()
        g, loss = net.backward(xb, yb, pos_weight=pos_weight)
        net.adam_step(g, lr)
        losses.append(loss)
    return losses
