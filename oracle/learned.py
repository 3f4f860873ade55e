"""FP64 CPU reference of the learned elimination step (an extension of
Algorithm 1; the paper has no counterpart).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module; the library never does.

Two parts, both evaluated on the state after k completed iterations:

* Features (six per-pixel channels of the proposal network):
    c0 = log(1 + sum_q |x_qi|),  c1 = log(1 + max_q |x_qi|),
    c(2+j) = log10(||x_.i^(k-j) - x_.i^(k-j-1)||_2 / eps_p + 1e-4) / 4,  j = 0..3,
  the update norms taken over the sensors from the window of Algorithm 1 (zero
  before the first iteration and beyond the window).

* Re-admission test for a frozen pixel i of sensor q.  The optimality
  condition of Eq. 2 in x_q (the augmented Lagrangian's x_q-gradient at the
  fixed point, where x_bar = z_bar) has the entry
      c_qi = mu b_i^T (B_q x_q - y_q) + rho s_i
  (b_i the real-form column of pixel i), and a single-coordinate step of the
  x-update moves x_qi by c_qi / (mu ||b_i||^2 + rho).  The pixel re-enters J_q
  when that step exceeds thr.  Because the frozen pixels are folded into y'
  (y'_q = y_q - B_F x_F in freeze mode 0; in zero mode x_F = 0 and y' = y),
  B_q x_q - y_q = -(y'_q - B_J x_J).
"""
import numpy as np

NFEAT = 6


def features(x, ring, k, eps_p):
    """(6, N) features; x (Q, N), ring (Kp, Q, N) with the update of iteration t
    (1-based) in slot (t - 1) mod Kp."""
    x = np.asarray(x, dtype=np.float64)
    Kp = ring.shape[0]
    N = x.shape[1]
    f = np.empty((NFEAT, N))
    a = np.abs(x)
    f[0] = np.log1p(a.sum(axis=0))
    f[1] = np.log1p(a.max(axis=0))
    for j in range(4):
        u = np.zeros(N)
        t = k - j                      # iteration whose update is wanted
        if j < Kp and t >= 1:
            u = np.sqrt(np.sum(np.asarray(ring[(t - 1) % Kp], dtype=np.float64) ** 2, axis=0))
        f[2 + j] = np.log10(u / eps_p + 1e-4) / 4.0
    return f


def frozen(J, N):
    """Sorted complement of the active set."""
    m = np.ones(N, dtype=bool)
    m[np.asarray(J, dtype=np.int64)] = False
    return np.nonzero(m)[0]


def readmission_steps(Bq, yprime_q, x_q, J, s, mu, rho):
    """(F, step): the frozen pixels of one sensor and |c_qi| / (mu ||b_i||^2 + rho)."""
    N = Bq.shape[1]
    F = frozen(J, N)
    r = yprime_q - Bq[:, J] @ x_q[J]                 # = y_q - B_q x_q
    BF = Bq[:, F]
    c = -mu * (BF.T @ r) + rho * s[F]
    return F, np.abs(c) / (mu * np.sum(BF * BF, axis=0) + rho)


def round_bf16(p):
    """Round-to-nearest-even of FP32 values to BF16 (kept in float64): the
    upper 16 bits of the FP32 pattern after adding 0x7fff plus the lowest kept
    bit.  Non-finite inputs are not expected (the network's parameters)."""
    bits = np.asarray(p, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    r = ((bits + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
