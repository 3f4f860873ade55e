"""The allocation-free forward product (sadmm_forward_noalloc) agrees with the
allocating one (sadmm_forward).

It serves callers that may not allocate device memory while running (real-time
pipelines with a fixed latency budget, processes whose device memory another
allocator rations): its partial sums use one fixed device array per GPU.  The
test calls it twice in a row, with different inputs, so that the second call
runs on the first call's leftover scratch contents.  This file sorts last so
that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_08606_gb300 import build, binding
    build()
    binding.load()
    return binding


def _bound(A, idx, v, base):
    Asel = A[idx].astype(np.complex128)
    ref = base.astype(np.complex128) - Asel.T @ v[idx].astype(np.float64)
    mag_re = np.abs(base.real) + np.abs(Asel.real).T @ np.abs(v[idx])
    mag_im = np.abs(base.imag) + np.abs(Asel.imag).T @ np.abs(v[idx])
    return ref, (len(idx) + 2) * U32 * mag_re, (len(idx) + 2) * U32 * mag_im


@pytest.mark.parametrize("KM,N,nidx", [(256, 1024, 700), (2048, 4096, 4000)])
def test_noalloc_matches_allocating_forward_twice(B, KM, N, nidx):
    dev = torch.device("cuda:0")
    s = scenegen.Stream(31, KM)
    A = ((s.normal(N * KM) + 1j * s.normal(N * KM)).reshape(N, KM) / np.sqrt(2)).astype(np.complex64)
    At = torch.from_numpy(A).to(dev)
    for call in range(2):
        idx = s.integers(nidx, N).astype(np.int32)
        v = s.normal(N).astype(np.float32)
        base = (s.normal(KM) + 1j * s.normal(KM)).astype(np.complex64)
        it, vt, bt = (torch.from_numpy(a).to(dev) for a in (idx, v, base))
        r_alloc = B.forward(At, it, vt, base=bt)
        r_fixed = B.forward_noalloc(At, it, vt, base=bt)
        torch.cuda.synchronize()
        ra = r_alloc.cpu().numpy().astype(np.complex128)
        rf = r_fixed.cpu().numpy().astype(np.complex128)
        ref, tol_re, tol_im = _bound(A, idx, v, base)
        for r in (ra, rf):
            assert np.all(np.abs(r.real - ref.real) <= tol_re), call
            assert np.all(np.abs(r.imag - ref.imag) <= tol_im), call
        assert np.all(np.abs(rf.real - ra.real) <= 2 * tol_re), call
        assert np.all(np.abs(rf.imag - ra.imag) <= 2 * tol_im), call


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    """One column of KM = 2^19 + 2 rows needs 8 MiB + 32 bytes of partial sums
    (one chunk of double-float pairs, 16 bytes per complex row), more than the
    fixed 8 MiB: the host refuses it with EINVAL and a message
    before any device work (the placeholder pointers are never dereferenced)."""
    import ctypes
    lib = B.load()
    p = ctypes.c_void_p(256)
    rc = lib.sadmm_forward_noalloc(p, (1 << 19) + 2, 1, p, 1, p, None, p, None)
    assert rc == B.EINVAL
    assert b"fixed scratch" in lib.sadmm_last_error()
    rc = lib.sadmm_forward_noalloc(None, 4096, 1, None, 0, None, None, None, None)
    assert rc == B.EINVAL
