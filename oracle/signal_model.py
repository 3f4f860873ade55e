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
exp(j 2 pi tau df), the phase at k = 0).  The back-projection image (Section
IV, Fig. 1) is pinned by the closed form at a lone noiseless target
(sum_q KM x_q at its pixel, since every entry has unit modulus) and by the
matched-filter bound (no other pixel exceeds it).
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


def backprojection(A, y):
    """Composite back-projection image sum_q |A_q^H y_q| (real, length N).

    The paper shows BP images beside SADMM and ASADMM (Section IV, Fig. 1)
    without defining them; the reading here is the matched filter of each
    sensor's own echo, A_q^H y_q, taken in magnitude (the sensors see the
    scene with different reflectivities, so their images add incoherently,
    as the composite ground truth adds the per-sensor images)."""
    out = np.zeros(np.asarray(A[0]).shape[0])
    for Aq, yq in zip(A, y):
        out += np.abs(np.asarray(Aq).astype(np.complex128).conj() @ np.asarray(yq).astype(np.complex128))
    return out


def db_image(img, dynamic_range=30.0):
    """20 log10(|img| / max |img|), clipped below at -dynamic_range dB (the
    display of Fig. 1, 30 dB dynamic range)."""
    a = np.abs(np.asarray(img, dtype=np.float64))
    peak = a.max()
    if peak <= 0:
        return np.full(a.shape, -dynamic_range)
    with np.errstate(divide="ignore"):
        d = 20.0 * np.log10(a / peak)
    return np.maximum(d, -dynamic_range)
