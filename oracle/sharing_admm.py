"""FP64 CPU oracle of sharing-ADMM with pixel elimination (SADMM / ASADMM).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module; the library never does.  It shares no code
with the CUDA path.

What it computes (Section III of the paper, Eq. 2, Eq. 3 and Algorithm 1), under
the readings listed below.  Notation: B_q = [Re A_q; Im A_q] is the real form of
the complex operator, so for real x, ||y - A x||^2 = ||[Re y; Im y] - B x||^2 and
Re(A^H y) = B^T [Re y; Im y].

Problem (Eq. 2 with the selectors equal to the identity):
    min_{x_1..x_Q}  sum_q mu/2 ||y_q - A_q x_q||^2 + lambda ||x_G||_1,
    x_G = sum_q x_q.
This is the sharing problem of Boyd et al. (2011, Sec. 7.3), which the paper cites
for its ADMM.  Internally the averaged variables are carried:
x_bar = (1/Q) sum_q x_q, z_bar = x_G / Q, and the scaled dual s, so that the
paper's dual is sigma = rho * s and its beta is rho.

One iteration k -> k+1:
  1. x-update (Eq. 3, x_q-update), per sensor, on the active set J_q only:
       v_J   = x_q - x_bar + z_bar - s           (restricted to J_q)
       x_q,J = (rho I + mu B_J^T B_J)^{-1} (mu B_J^T y'_q + rho v_J)
     Entries outside J_q keep their value (frozen).  y'_q is y_q minus the
     contribution of the frozen pixels.
  2. x_bar = (1/Q) sum_q x_q over all N pixels.
  3. z_bar' = soft(x_bar + s, lambda/rho)        (Eq. 3, x_G-update)
  4. s'     = s + x_bar - z_bar'                 (Eq. 3, dual update)
  5. residuals: r_pri = sqrt(Q) ||x_bar - z_bar'||,
       eps_pri  = sqrt(QN) eps_abs + eps_rel max(||X||_F, ||Z||_F),  Z_q = x_q - x_bar + z_bar',
       d        = rho ||Z^{k+1} - Z^k||_F,
       eps_dual = sqrt(QN) eps_abs + eps_rel rho sqrt(Q) ||s'||.
  6. SSC (Algorithm 1): |x_q^{k+1} - x_q^k| is pushed into a ring of the last Kp
     differences; if elimination is on, k+1 >= Kp and r_pri <= eps_pri, then
     zeta = mean of the ring and J_q <- {i in J_q : zeta_i >= eps_p}.  Newly
     removed pixels are frozen at their value and folded into y'_q
     (y'_q -= A_q,E x_q,E), or, in zero mode, set to 0.
  7. stop when k+1 = iters, or (mode 0) ||X^{k+1} - X^k||_F <= tol ||X^{k+1}||_F,
     or (mode 1) r_pri <= eps_pri and d <= eps_dual.

Readings where the paper is silent or garbled (each is a choice both this oracle
and the CUDA path make): real x_q (Eq. 1 folds the phase into A_q); x_G is the sum
of the x_q and the threshold on the averaged variable is lambda/rho; the x-update
carries Boyd's x_q^k - x_bar^k + z_bar^k term that Eq. 3's garbled x_q-update
drops; the dual enters the x_G-update with the sign that makes the fixed point the
optimum of Eq. 2; the primal/dual residuals follow Boyd Sec. 3.3.1 applied to the
sharing form; Algorithm 1's window is the last Kp differences including the newest
one and its gate uses the newest residual; ties zeta = eps_p are kept; the active
set only shrinks; all iterates start at zero; the factor is refreshed whenever an
active set changes.

Consensus formulation (Criterion.consensus; CADMM / ACADMM, the sibling
variant Section I attributes to the authors' earlier work and does not
reproduce; read here as Boyd et al. 2011, Sec. 7.1, global consensus): every
sensor images one common reflectivity z,
    min_{x_1..x_Q, z}  sum_q mu/2 ||y_q - A_q x_q||^2 + lambda ||z||_1,  x_q = z,
with scaled duals u_q (one per sensor and pixel).  One iteration:
  1. x-update on J_q with v = z - u_q (the same system as the sharing form);
  2. x_bar = mean_q x_q;
  3. z' = soft(x_bar + u_bar, lambda / (Q rho)),  u_bar = mean_q u_q;
  4. u_q' = u_q + x_q - z';
  5. r_pri = ||X - z'||_F, eps_pri = sqrt(QN) eps_abs + eps_rel max(||X||_F, sqrt(Q) ||z'||),
     d = rho sqrt(Q) ||z' - z||, eps_dual = sqrt(QN) eps_abs + eps_rel rho ||U'||_F;
  6. Algorithm 1 per sensor on |x_q^{k+1} - x_q^k|, frozen pixels folded into y'_q.
The image is z (Result.xG).  zbar holds z; xbar and s are kept for the shared
code path only.  The learned step is defined for the sharing form only.
"""
from dataclasses import dataclass, field
import numpy as np
import scipy.linalg as sla

from . import cnn as _cnn
from . import learned as _learned


@dataclass
class Criterion:
    mu: float = 1.0
    Kp: int = 5
    eps_p: float = 1e-5
    eps_abs: float = 1e-4
    eps_rel: float = 1e-2
    elim: int = 1          # 0: plain SADMM, 1: pixel elimination (Algorithm 1), 2: plus learned step
    freeze_mode: int = 0   # 0: removed pixels keep their value, 1: set to zero
    stop: int = 0          # 0: relative change of X, 1: primal and dual residuals
    learn_every: int = 10  # elim 2: period of the learned step
    learn_theta: float = 0.5   # elim 2: drop pixel i when the network's p_i > learn_theta
    readmit: float = 10.0  # elim 2: re-admit when the coordinate step exceeds readmit * eps_p
    ssc_every: int = 1     # Algorithm 1's pass after iteration k only when ssc_every divides k
    consensus: bool = False  # consensus formulation (CADMM / ACADMM, see below) instead of sharing


def soft(v, t):
    """Soft threshold: the closed-form minimiser of t|x| + 1/2 (x - v)^2 (Eq. 3, x_G-update)."""
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def real_form(Aq):
    """B_q = [Re A_q; Im A_q] (2KM x N, float64) from a pixel-major (N, KM) operator."""
    At = np.asarray(Aq).astype(np.complex128).T
    return np.vstack([At.real, At.imag])


def real_vec(y):
    y = np.asarray(y).astype(np.complex128)
    return np.concatenate([y.real, y.imag])


def forward(Aq, x):
    """A_q x for real x (Eq. 1), complex128."""
    return np.asarray(Aq).astype(np.complex128).T @ np.asarray(x, dtype=np.float64)


def adjoint_re(Aq, r):
    """Re(A_q^H r), float64: the adjoint of the real-input forward map."""
    return (np.asarray(Aq).astype(np.complex128).conj() @ np.asarray(r).astype(np.complex128)).real


class RidgeSolver:
    """Solves (rho I + mu B_J^T B_J) x = b for a fixed active set J (Eq. 3, x_q-update).

    The factor is a Cholesky decomposition of the smaller of the two Gram forms:
    the |J| x |J| matrix itself, or, when |J| > 2KM, rho I + mu B_J B_J^T, used
    through the Woodbury identity
        (rho I + mu B^T B)^{-1} = (I - mu B^T (rho I + mu B B^T)^{-1} B) / rho.
    """

    def __init__(self, BJ, mu, rho):
        self.BJ, self.mu, self.rho = BJ, mu, rho
        m, n = BJ.shape
        self.woodbury = n > m
        if self.woodbury:
            G = rho * np.eye(m) + mu * (BJ @ BJ.T)
        else:
            G = rho * np.eye(n) + mu * (BJ.T @ BJ)
        self.cf = sla.cho_factor(G, lower=True)

    def solve(self, b):
        if self.woodbury:
            t = sla.cho_solve(self.cf, self.BJ @ b)
            return (b - self.mu * (self.BJ.T @ t)) / self.rho
        return sla.cho_solve(self.cf, b)


@dataclass
class State:
    k: int                      # iterations completed
    x: np.ndarray               # (Q, N)
    xbar: np.ndarray            # (N,)
    zbar: np.ndarray            # (N,)
    s: np.ndarray               # (N,)
    ring: np.ndarray            # (Kp, Q, N) |x^{t+1} - x^t| for the last Kp iterations
    J: list                     # Q sorted int arrays
    yprime: list                # Q arrays (2KM,) real form of y'_q
    u: np.ndarray = None        # (Q, N) scaled duals of the consensus formulation (zbar then holds z)

    def copy(self):
        return State(self.k, self.x.copy(), self.xbar.copy(), self.zbar.copy(), self.s.copy(),
                     self.ring.copy(), [j.copy() for j in self.J], [v.copy() for v in self.yprime],
                     None if self.u is None else self.u.copy())


def initial_state(A, y, Kp, consensus=False):
    Q, N = len(A), A[0].shape[0]
    return State(0, np.zeros((Q, N)), np.zeros(N), np.zeros(N), np.zeros(N),
                 np.zeros((Kp, Q, N)), [np.arange(N) for _ in range(Q)],
                 [real_vec(v) for v in y], np.zeros((Q, N)) if consensus else None)


@dataclass
class Result:
    state: State
    history: list = field(default_factory=list)
    stop_reason: str = "iters"
    snapshots: dict = field(default_factory=dict)   # k -> State copy (requested k only)
    consensus: bool = False

    @property
    def xG(self):
        """The image: x_G = Q z_bar (sharing), or the consensus variable z."""
        return self.state.zbar.copy() if self.consensus else len(self.state.x) * self.state.zbar


@dataclass
class Eliminator:
    """Proposal network of the learned step: FP32 master parameters (flat layout
    of oracle.cnn) for an H x W pixel grid (pixel i at row i // W, column i % W).
    The network is evaluated with the parameters rounded to BF16."""
    params: np.ndarray
    H: int
    W: int


def sadmm(A, y, rho, lam, crit: Criterion, iters, tol=0.0, state: State = None, B=None,
          snapshots=(), eliminator: Eliminator = None):
    """Run SADMM (crit.elim = 0), ASADMM (crit.elim = 1) or ASADMM with the
    learned step (crit.elim = 2 with an eliminator) for at most `iters`
    iterations from `state` (zeros if None).  Returns a Result whose history holds,
    per iteration: r_pri, eps_pri, d, eps_dual, relchange, gate, sizes, and the
    decision margins zeta_margin (min |zeta - eps_p| over tested pixels) and
    gate_margin (|r_pri - eps_pri| / eps_pri); learned steps add learned,
    readmitted, prob_margin (min |p_i - learn_theta| over pixels active in some
    sensor) and readmit_margin (min |step - thr| / thr over frozen pixels).  A
    copy of the state after iteration k is kept in Result.snapshots for every k
    in `snapshots`.

    The learned step (an extension; the paper has no counterpart) runs after
    iteration k when k is a multiple of learn_every and k >= max(Kp, 4): the
    re-admission test (oracle.learned) marks frozen pixels against the sets
    before this pass, the network maps the features to p, Algorithm 1's pass
    also drops every pixel with p_i > learn_theta (whether or not its gate
    passed), and the marked pixels then re-enter their sets: unfolded from y',
    their last Kp updates set to 2 eps_p.  Removed pixels' window entries are
    cleared at every pass."""
    Q = len(A)
    mu = crit.mu
    B = B if B is not None else [real_form(a) for a in A]
    N = B[0].shape[1]
    cons = crit.consensus
    if cons and crit.elim == 2:
        raise ValueError("the learned step is defined for the sharing formulation only")
    st = (state.copy() if state is not None else initial_state(A, y, crit.Kp, consensus=cons))
    solvers, cvec = [None] * Q, [None] * Q

    def refresh(q):
        J = st.J[q]
        BJ = B[q] if len(J) == N else B[q][:, J]
        solvers[q] = RidgeSolver(BJ, mu, rho)
        cvec[q] = mu * (BJ.T @ st.yprime[q])

    for q in range(Q):
        refresh(q)
    pr = None
    if crit.elim == 2 and eliminator is not None:
        assert eliminator.H * eliminator.W == N and crit.eps_p > 0
        pr = _learned.round_bf16(eliminator.params)
    res = Result(st, consensus=cons)
    Zold = st.x - st.xbar[None, :] + st.zbar[None, :]
    for it in range(iters):
        x_old = st.x.copy()
        # 1. x-update per sensor on its active set
        for q in range(Q):
            J = st.J[q]
            if cons:
                v = st.zbar[J] - st.u[q, J]
            else:
                v = st.x[q, J] - st.xbar[J] + st.zbar[J] - st.s[J]
            st.x[q, J] = solvers[q].solve(cvec[q] + rho * v)
        # 2-4. average, prox, dual
        xbar_new = st.x.mean(axis=0)
        nx = np.linalg.norm(st.x)
        relchange = np.linalg.norm(st.x - x_old) / nx if nx > 0 else np.inf
        if cons:
            z_new = soft(xbar_new + st.u.mean(axis=0), lam / (Q * rho))
            u_new = st.u + st.x - z_new[None, :]
            # 5. residuals of the consensus form (Boyd Sec. 7.1)
            r_pri = np.linalg.norm(st.x - z_new[None, :])
            eps_pri = np.sqrt(Q * N) * crit.eps_abs + crit.eps_rel * max(nx, np.sqrt(Q) * np.linalg.norm(z_new))
            d = rho * np.sqrt(Q) * np.linalg.norm(z_new - st.zbar)
            eps_dual = np.sqrt(Q * N) * crit.eps_abs + crit.eps_rel * rho * np.linalg.norm(u_new)
            st.xbar, st.zbar, st.u = xbar_new, z_new, u_new
        else:
            zbar_new = soft(xbar_new + st.s, lam / rho)
            s_new = st.s + xbar_new - zbar_new
            # 5. residuals
            Z = st.x - xbar_new[None, :] + zbar_new[None, :]
            r_pri = np.sqrt(Q) * np.linalg.norm(xbar_new - zbar_new)
            eps_pri = np.sqrt(Q * N) * crit.eps_abs + crit.eps_rel * max(nx, np.linalg.norm(Z))
            d = rho * np.linalg.norm(Z - Zold)
            eps_dual = np.sqrt(Q * N) * crit.eps_abs + crit.eps_rel * rho * np.sqrt(Q) * np.linalg.norm(s_new)
            st.xbar, st.zbar, st.s = xbar_new, zbar_new, s_new
        # 6. SSC
        slot = st.k % crit.Kp
        st.ring[slot] = np.abs(st.x - x_old)
        st.k += 1
        rec = dict(k=st.k, r_pri=r_pri, eps_pri=eps_pri, d=d, eps_dual=eps_dual,
                   relchange=relchange, gate=False, zeta_margin=np.inf, gate_margin=np.inf)
        gate = False
        if crit.elim and st.k >= crit.Kp:
            rec["gate_margin"] = abs(r_pri - eps_pri) / eps_pri if eps_pri > 0 else np.inf
            gate = r_pri <= eps_pri and st.k % crit.ssc_every == 0
        rec["gate"] = gate
        learned = (pr is not None and st.k % crit.learn_every == 0 and st.k >= max(crit.Kp, 4))
        readd, prob = None, None
        if learned:
            # re-admission test against the sets before this pass
            thr = crit.readmit * crit.eps_p
            readd, rmargin = [], np.inf
            for q in range(Q):
                F, step = _learned.readmission_steps(B[q], st.yprime[q], st.x[q], st.J[q], st.s, mu, rho)
                readd.append(F[step > thr])
                if len(F) and thr > 0:
                    rmargin = min(rmargin, float(np.min(np.abs(step - thr))) / thr)
            feats = _learned.features(st.x, st.ring, st.k, crit.eps_p)
            p, _ = _cnn.forward(pr, feats.reshape(1, _learned.NFEAT, eliminator.H, eliminator.W))
            prob = p.reshape(N)
            act = np.zeros(N, dtype=bool)
            for J in st.J:
                act[J] = True
            rec["prob_margin"] = (float(np.min(np.abs(prob[act] - crit.learn_theta))) if act.any() else np.inf)
            rec["readmit_margin"] = rmargin
        rec["learned"] = learned
        if gate or learned:
            zeta = st.ring.mean(axis=0)
            changed = False
            for q in range(Q):
                J = st.J[q]
                zq = zeta[q, J]
                if gate:
                    if len(zq):
                        rec["zeta_margin"] = min(rec["zeta_margin"], float(np.min(np.abs(zq - crit.eps_p))))
                    keep = zq >= crit.eps_p
                else:
                    keep = np.ones(len(J), dtype=bool)
                if learned:
                    keep &= ~(prob[J] > crit.learn_theta)
                if keep.all():
                    continue
                E = J[~keep]
                st.J[q] = J[keep]
                st.ring[:, q, E] = 0.0
                if crit.freeze_mode == 0:
                    st.yprime[q] = st.yprime[q] - B[q][:, E] @ st.x[q, E]
                else:
                    st.x[q, E] = 0.0
                changed = True
                refresh(q)
            if changed and crit.freeze_mode == 1:
                st.xbar = st.x.mean(axis=0)
        if learned:
            total = 0
            for q in range(Q):
                R = readd[q]
                if len(R) == 0:
                    continue
                total += len(R)
                st.J[q] = np.union1d(st.J[q], R)
                st.ring[:, q, R] = 2.0 * crit.eps_p
                if crit.freeze_mode == 0:
                    st.yprime[q] = st.yprime[q] + B[q][:, R] @ st.x[q, R]
                refresh(q)
            rec["readmitted"] = total
        rec["sizes"] = [len(j) for j in st.J]
        res.history.append(rec)
        if st.k in snapshots:
            res.snapshots[st.k] = st.copy()
        Zold = st.x - st.xbar[None, :] + st.zbar[None, :]
        # 7. stop
        if crit.stop == 0 and tol > 0 and relchange <= tol:
            res.stop_reason = "tol"
            break
        if crit.stop == 1 and r_pri <= eps_pri and d <= eps_dual:
            res.stop_reason = "residuals"
            break
    return res


def sadmm_primal_inverse(A, y, rho, lam, mu=1.0, iters=1000, tol=0.0, record=None):
    """Plain SADMM (Eq. 3 with every selector the identity: no elimination)
    for problems whose sensors each resolve the grid (N <= 2KM, so the x-update
    is taken in its primal form), held in the memory of Q explicit inverses.

    Per sensor, one after another, in FP64 from the complex operator
    (pixel-major, N x KM):
        G_q = B_q^T B_q = Re(A_q^H A_q)  (two symmetric rank-KM products of the
                                          real and imaginary parts),
        H_q = (rho I + mu G_q)^{-1}       (Cholesky factor, then its inverse),
        c_q = mu B_q^T [Re y_q; Im y_q] = mu Re(A_q^H y_q).
    Each iteration is steps 1-5 of the plain iteration (see sadmm): the
    x-update x_q = H_q (c_q + rho (x_q - x_bar + z_bar - s)) for every q, then
    x_bar = mean_q x_q, z_bar = soft(x_bar + s, lam / rho), s += x_bar - z_bar,
    and the relative change of the stacked iterate.  The same iterates as
    sadmm(..., Criterion(elim=0)) up to rounding (an explicit inverse instead
    of two triangular solves).  Stops after `iters` iterations or when the
    relative change is <= tol.  record(k, x_G) is called after every
    iteration when given.  Returns a Result whose state holds X, x_bar, z_bar,
    s (J = all pixels, y' = y, the ring unused)."""
    from scipy.linalg import blas, lapack
    Q = len(A)
    N, KM = np.asarray(A[0]).shape
    if N > 2 * KM:
        raise ValueError("sadmm_primal_inverse needs N <= 2KM (the primal form)")
    H, c = [], []
    for q in range(Q):
        Ar = np.asarray(A[q]).real.astype(np.float64)
        Ai = np.asarray(A[q]).imag.astype(np.float64)
        # Ar, Ai are C-ordered N x KM: their transposes are Fortran-ordered KM x N
        G = blas.dsyrk(mu, Ar.T, trans=1, lower=0)
        G = blas.dsyrk(mu, Ai.T, beta=1.0, c=G, trans=1, lower=0, overwrite_c=1)
        yq = np.asarray(y[q]).astype(np.complex128)
        c.append(mu * (Ar @ yq.real + Ai @ yq.imag))
        del Ar, Ai
        G[np.diag_indices(N)] += rho
        L, info = lapack.dpotrf(G, lower=0, overwrite_a=1)
        if info != 0:
            raise np.linalg.LinAlgError(f"sensor {q}: rho I + mu G is not positive definite ({info})")
        Hq, info = lapack.dpotri(L, lower=0, overwrite_c=1)
        if info != 0:
            raise np.linalg.LinAlgError(f"sensor {q}: inverse failed ({info})")
        Hq = np.triu(Hq)                     # the upper triangle holds the inverse
        Hq += np.triu(Hq, 1).T
        H.append(np.ascontiguousarray(Hq))
        del L, G
    st = initial_state(A, y, 1)
    res = Result(st)
    for it in range(iters):
        x_old = st.x.copy()
        for q in range(Q):
            v = st.x[q] - st.xbar + st.zbar - st.s
            st.x[q] = H[q] @ (c[q] + rho * v)
        xb = np.mean(st.x, axis=0)
        zb = soft(xb + st.s, lam / rho)
        st.s = st.s + xb - zb
        st.xbar, st.zbar = xb, zb
        st.k += 1
        nx = np.linalg.norm(st.x)
        relchange = np.linalg.norm(st.x - x_old) / nx if nx > 0 else np.inf
        res.history.append(dict(k=st.k, relchange=relchange))
        if record is not None:
            record(st.k, Q * st.zbar)
        if tol > 0 and relchange <= tol:
            res.stop_reason = "tol"
            break
    return res


def kkt_consensus(A, y, X, U, z, rho, lam, mu=1.0, B=None):
    """Optimality conditions of the consensus problem for (X, z, nu_q = rho u_q):
      stationarity  mu B_q^T (B_q x_q - y_q) + nu_q = 0 for every q,
      subgradient   sum_q nu_q in lambda d||z||_1,
      feasibility   x_q = z for every q.
    Residuals normalised by lambda (and by max(1, ||z||_inf) for feasibility)."""
    B = B if B is not None else [real_form(a) for a in A]
    nu = rho * np.asarray(U)
    stat = max(np.max(np.abs(mu * (B[q].T @ (B[q] @ X[q] - real_vec(y[q]))) + nu[q])) for q in range(len(A)))
    tot = nu.sum(axis=0)
    sub = max(0.0, float(np.max(np.abs(tot))) - lam)
    supp = np.abs(z) > 0
    sgn = float(np.max(np.abs(tot[supp] - lam * np.sign(z[supp])))) if supp.any() else 0.0
    feas = float(np.max(np.abs(np.asarray(X) - z[None, :]))) / max(1.0, float(np.max(np.abs(z))))
    return dict(stationarity=stat / lam, subgradient=max(sub, sgn) / lam, feasibility=feas)


def objective(A, y, X, lam, mu=1.0, B=None):
    """Eq. 2 objective with the selectors equal to the identity."""
    B = B if B is not None else [real_form(a) for a in A]
    f = sum(0.5 * mu * np.sum((real_vec(y[q]) - B[q] @ X[q]) ** 2) for q in range(len(A)))
    return f + lam * np.sum(np.abs(np.sum(X, axis=0)))


def kkt(A, y, X, s, rho, lam, mu=1.0, xG=None, B=None):
    """Optimality conditions of Eq. 2 (selectors = identity) for the primal-dual
    pair (X, nu = rho s):
      stationarity  mu B_q^T (B_q x_q - y_q) + nu = 0 for every q,
      subgradient   nu in lambda d||x_G||_1 (|nu_i| <= lambda; nu_i = lambda sign(x_G,i) on the support),
      feasibility   x_G = sum_q x_q.
    Returns the residuals normalised by lambda (and by max(1, ||x_G||_inf) for feasibility)."""
    B = B if B is not None else [real_form(a) for a in A]
    nu = rho * np.asarray(s)
    xsum = np.sum(X, axis=0)
    xG = xsum if xG is None else xG
    stat = max(np.max(np.abs(mu * (B[q].T @ (B[q] @ X[q] - real_vec(y[q]))) + nu))
               for q in range(len(A)))
    sub = max(0.0, float(np.max(np.abs(nu))) - lam)
    supp = np.abs(xG) > 0
    sgn = float(np.max(np.abs(nu[supp] - lam * np.sign(xG[supp])))) if supp.any() else 0.0
    feas = float(np.max(np.abs(xG - xsum))) / max(1.0, float(np.max(np.abs(xG))))
    return dict(stationarity=stat / lam, subgradient=max(sub, sgn) / lam, feasibility=feas)
