"""Split-precision operator of the oracle (extension a12: the operator stored
as two 16-bit planes).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module; the library never does.  It shares no
code with the CUDA path.

Each real component a of the complex64 operator is rounded to nearest (ties to
even) into the 16-bit format, hi = RN(a), and the remainder once more,
lo = RN(a - hi).  The pair operator P = hi + lo is what products that read both
planes compute with; the method run on the planes solves Eq. 2 for P instead of
A.  For BF16 (8 significant bits) |a - P| <= 2^-16 |a|; for FP16 (11 bits)
|a - P| <= 2^-22 |a| plus the subnormal spacing 2^-25 of tiny remainders."""
import numpy as np

from .learned import round_bf16

BF16, FP16 = 1, 2


def _round(x, kind):
    """RN of float32 values into the 16-bit format, as float64."""
    x = np.asarray(x, dtype=np.float32)
    if kind == BF16:
        return round_bf16(x)
    if kind == FP16:
        return x.astype(np.float16).astype(np.float64)
    raise ValueError("kind must be 1 (BF16) or 2 (FP16)")


def split_planes(A, kind):
    """(hi, lo) complex128 planes of the complex64 operator A."""
    A = np.asarray(A, dtype=np.complex64)
    out = []
    for part in (A.real, A.imag):
        h = _round(part, kind)
        r = (part.astype(np.float32) - h.astype(np.float32))   # exact in FP32
        out.append((h, _round(r, kind)))
    (hr, lr), (hi_, li) = out
    return hr + 1j * hi_, lr + 1j * li


def pair_operator(A, kind):
    """P = hi + lo as complex64 (exact: the two planes' sum needs at most 24
    significant bits per component)."""
    h, l = split_planes(A, kind)
    P = h + l
    out = P.astype(np.complex64)
    assert np.array_equal(out.astype(np.complex128), P)
    return out
