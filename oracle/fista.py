"""Independent FISTA solver of the same objective (Eq. 2, selectors = identity).

TEST INFRASTRUCTURE.  Only the tests may import this module.  It is written
separately from the ADMM oracle (no shared helpers) so that agreement between
the two is evidence about both.

Objective over the stacked X = (x_1..x_Q), x_q real:
    F(X) = sum_q mu/2 ||y_q - A_q x_q||^2        (smooth, grad mu Re(A_q^H (A_q x_q - y_q)))
    G(X) = lambda ||S X||_1,   S X = sum_q x_q    (S S^T = Q I)
The proximal map of t G follows from the rule for a convex function composed
with a linear map whose Gram is a multiple of the identity (Parikh and Boyd,
"Proximal Algorithms", 2014, Sec. 2.2):
    prox_{tG}(V)_q = V_q + (1/Q) (soft(sum V, Q t lambda) - sum V).
FISTA is Beck and Teboulle (2009) with the function-value adaptive restart of
O'Donoghue and Candes (2015).
"""
import numpy as np


def _shrink(u, t):
    a = np.abs(u) - t
    return np.where(a > 0, np.copysign(a, u), 0.0)


def _lipschitz(A, mu):
    best = 0.0
    for Aq in A:
        M = np.asarray(Aq).astype(np.complex128).T        # KM x N
        Mr = np.concatenate([M.real, M.imag], axis=0)
        best = max(best, np.linalg.norm(Mr, 2) ** 2)
    return mu * best


def fista(A, y, lam, mu=1.0, iters=20000, tol=1e-15, X0=None):
    Ac = [np.asarray(a).astype(np.complex128).T for a in A]   # KM x N each
    yc = [np.asarray(v).astype(np.complex128) for v in y]
    Q, N = len(Ac), Ac[0].shape[1]
    L = _lipschitz(A, mu)
    t_step = 1.0 / L

    def F(X):
        return sum(0.5 * mu * np.sum(np.abs(yc[q] - Ac[q] @ X[q]) ** 2) for q in range(Q))

    def grad(X):
        return np.stack([mu * (Ac[q].conj().T @ (Ac[q] @ X[q] - yc[q])).real for q in range(Q)])

    def prox(V):
        S = V.sum(axis=0)
        return V + (_shrink(S, Q * t_step * lam) - S)[None, :] / Q

    def total(X):
        return F(X) + lam * np.sum(np.abs(X.sum(axis=0)))

    X = np.zeros((Q, N)) if X0 is None else np.array(X0, dtype=np.float64)
    Yv, t = X.copy(), 1.0
    f_prev = total(X)
    for k in range(iters):
        Xn = prox(Yv - t_step * grad(Yv))
        f_new = total(Xn)
        if f_new > f_prev:          # adaptive restart
            Yv, t = X.copy(), 1.0
            continue
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        Yv = Xn + ((t - 1.0) / tn) * (Xn - X)
        step = np.linalg.norm(Xn - X)
        X, t, f_prev = Xn, tn, f_new
        if step <= tol * max(1.0, np.linalg.norm(X)):
            break
    return X, total(X)


def fista_consensus(A, y, lam, mu=1.0, iters=20000, tol=1e-15):
    """FISTA (with the same restart) on the consensus objective, a LASSO in the
    common image z with the sensors' operators stacked:
        F(z) = sum_q mu/2 ||y_q - A_q z||^2,  G(z) = lambda ||z||_1,
    L = mu ||[B_1; ..; B_Q]||_2^2 (B_q the real form of A_q).
    Returns (z, F(z) + G(z))."""
    Ac = [np.asarray(a).astype(np.complex128).T for a in A]
    yc = [np.asarray(v).astype(np.complex128) for v in y]
    N = Ac[0].shape[1]
    stack = np.concatenate([np.concatenate([M.real, M.imag], axis=0) for M in Ac], axis=0)
    t_step = 1.0 / (mu * np.linalg.norm(stack, 2) ** 2)

    def total(z):
        return sum(0.5 * mu * np.sum(np.abs(v - M @ z) ** 2) for M, v in zip(Ac, yc)) + lam * np.sum(np.abs(z))

    def grad(z):
        return sum(mu * (M.conj().T @ (M @ z - v)).real for M, v in zip(Ac, yc))

    z = np.zeros(N)
    w, t = z.copy(), 1.0
    f_prev = total(z)
    for _ in range(iters):
        zn = _shrink(w - t_step * grad(w), t_step * lam)
        f_new = total(zn)
        if f_new > f_prev:
            w, t = z.copy(), 1.0
            continue
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        w = zn + ((t - 1.0) / tn) * (zn - z)
        step = np.linalg.norm(zn - z)
        z, t, f_prev = zn, tn, f_new
        if step <= tol * max(1.0, np.linalg.norm(z)):
            break
    return z, total(z)
