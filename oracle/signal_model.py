"""FP64 forward operator of the signal model from the round-trip delays.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module; the library never does.  It shares no code
with the CUDA path.

Section II, Eq. 1: y_q = A_q x_q + w_q with A_q in C^{KM x N}.  The paper takes
the entries of A_q from its reference; the reading used here is the dechirped
LFM echo: receiver m, fast-time sample k, pixel n with round-trip delay
tau[m, n] give

    A_q[(m, k), n] = exp(j 2 pi tau[m, n] (f0 + k df)),    row index m K + k,

with f0 the chirp start frequency and df = BW / K the frequency step per
sample.  Parity: pinned in tests/test_oracle_pins.py against the scene
generator's complex64 operator (an independent implementation that reduces the
phase in cycles before its cosine and sine), and by the invariants of the
formula (unit modulus, a geometric progression in k per (m, n) with ratio
exp(j 2 pi tau df), the phase at k = 0).
"""
import numpy as np


def operator_from_delays(tau, f0, df, K):
    """A_q pixel-major, shape (N, M K), complex128, from tau (M, N) in seconds."""
    tau = np.asarray(tau, dtype=np.float64)
    M, N = tau.shape
    A = np.empty((N, M * K), dtype=np.complex128)
    for m in range(M):
        for k in range(K):
            A[:, m * K + k] = np.exp(2j * np.pi * tau[m] * (f0 + k * df))
    return A
