"""Kernel-level parity of the CUDA path (called through the C ABI) against the
FP64 oracle's definitions: the Eq. 1 forward product over an index list, its
adjoint, the FP64 x-update factor (Eq. 3, x_q-update) and its SPD apply.

Floating-point bounds are derived from the arithmetic: an FP32 sum of n
products differs from the exact value by at most n u sum|terms| (u = 2^-24)."""
import numpy as np
import pytest

import oracle
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


def _operator(KM, N, seed, radar=False):
    if radar:
        g = scenegen.Geometry(Q=1, M=KM // 32, K=32, nx=int(np.sqrt(N)), cell=0.05, radius=10.0,
                              fc=77e9, bw=1e9)
        return scenegen.operator(g, 0)
    s = scenegen.Stream(seed, 500)
    re = s.normal(N * KM).reshape(N, KM)
    im = s.normal(N * KM).reshape(N, KM)
    return ((re + 1j * im) / np.sqrt(2)).astype(np.complex64)


FWD_CASES = [
    # KM, N, nidx, repeats, radar
    (2, 10, 7, False, False),
    (32, 100, 37, False, False),
    (96, 513, 300, True, False),
    (256, 1024, 1024, False, True),
    (256, 1024, 0, False, False),
    (2048, 3001, 2999, False, False),
]


@pytest.mark.parametrize("KM,N,nidx,repeats,radar", FWD_CASES)
def test_forward_matches_oracle(B, KM, N, nidx, repeats, radar):
    A = _operator(KM, N, seed=KM + N, radar=radar)
    s = scenegen.Stream(7, KM)
    if repeats:
        idx = s.integers(nidx, N).astype(np.int32)
    else:
        idx = np.sort(s.permutation(N)[:nidx]).astype(np.int32)
    v = s.normal(N).astype(np.float32)
    base = (s.normal(KM) + 1j * s.normal(KM)).astype(np.complex64)
    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev)
    r = B.forward(At, torch.from_numpy(idx).to(dev), torch.from_numpy(v).to(dev),
                  base=torch.from_numpy(base).to(dev))
    torch.cuda.synchronize()
    r = r.cpu().numpy().astype(np.complex128)
    Asel = A[idx].astype(np.complex128)                      # (nidx, KM)
    ref = base.astype(np.complex128) - (Asel.T @ v[idx].astype(np.float64) if nidx else 0.0)
    mag_re = np.abs(base.real) + (np.abs(Asel.real).T @ np.abs(v[idx]) if nidx else 0.0)
    mag_im = np.abs(base.imag) + (np.abs(Asel.imag).T @ np.abs(v[idx]) if nidx else 0.0)
    n = nidx + 2
    assert np.all(np.abs(r.real - ref.real) <= n * U32 * mag_re + 1e-30)
    assert np.all(np.abs(r.imag - ref.imag) <= n * U32 * mag_im + 1e-30)
    if nidx:
        rel = np.linalg.norm(r - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5


@pytest.mark.parametrize("KM,N,nidx", [(32, 100, 37), (96, 513, 513), (2048, 700, 650), (8192, 70, 69),
                                       (16384, 3000, 2999)])
def test_adjoint_matches_oracle(B, KM, N, nidx):
    A = _operator(KM, N, seed=3 * KM + N)
    s = scenegen.Stream(11, KM)
    idx = s.permutation(N)[:nidx].astype(np.int32)           # unsorted
    w = (s.normal(KM) + 1j * s.normal(KM)).astype(np.complex64)
    dev = torch.device("cuda:0")
    g = B.adjoint(torch.from_numpy(A).to(dev), torch.from_numpy(idx).to(dev),
                  torch.from_numpy(w).to(dev))
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    ref = oracle.adjoint_re(A[idx], w)
    mag = np.abs(A[idx].real) @ np.abs(w.real) + np.abs(A[idx].imag) @ np.abs(w.imag)
    assert np.all(np.abs(g - ref) <= (2 * KM + 2) * U32 * mag)
    # adjoint identity through the two GPU products, Re<A v, w> = <v, Re(A^H w)>
    v = s.normal(N).astype(np.float32)
    r = B.forward(torch.from_numpy(A).to(dev), torch.from_numpy(np.sort(idx)).to(dev),
                  torch.from_numpy(v).to(dev)).cpu().numpy().astype(np.complex128)
    lhs = -np.vdot(w.astype(np.complex128), r).real        # forward returns 0 - A v
    rhs = float(np.dot(v[idx].astype(np.float64), g))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(r) * np.linalg.norm(w)


def _interleaved_real_form(A, idx):
    """B[2m, p] = Re A[idx_p, m], B[2m+1, p] = Im A[idx_p, m] (float64)."""
    cols = A[idx].astype(np.complex128)                       # (nidx, KM)
    Bm = np.empty((2 * A.shape[1], len(idx)))
    Bm[0::2] = cols.real.T
    Bm[1::2] = cols.imag.T
    return Bm


@pytest.mark.parametrize("KM,N,nidx,mu,rho", [
    (32, 200, 50, 1.0, 1.0),      # primal, padded 50 -> 64
    (32, 200, 64, 0.7, 2.0),      # primal, one full tile
    (32, 200, 150, 1.0, 1.0),     # Woodbury, n = 64
    (128, 1200, 1000, 1.3, 0.5),  # Woodbury, 4 tiles
    (128, 1200, 200, 1.0, 3.0),   # primal, 200 -> 256
])
def test_factor_matches_fp64_inverse(B, KM, N, nidx, mu, rho):
    A = _operator(KM, N, seed=KM * 7 + nidx)
    idx = np.sort(scenegen.Stream(5, nidx).permutation(N)[:nidx]).astype(np.int32)
    dev = torch.device("cuda:0")
    F, form, n = B.factor(torch.from_numpy(A).to(dev), torch.from_numpy(idx).to(dev), mu, rho)
    torch.cuda.synchronize()
    F = F.cpu().numpy()
    Bm = _interleaved_real_form(A, idx)
    if nidx > 2 * KM:
        assert form == 1 and n == 2 * KM
        G = rho * np.eye(n) + mu * Bm @ Bm.T
    else:
        assert form == 0 and n == nidx
        G = rho * np.eye(n) + mu * Bm.T @ Bm
    ref = np.linalg.inv(G)
    Fn = F[:n, :n]
    assert np.array_equal(Fn, Fn.T)
    cond = np.linalg.cond(G)
    # the factor inverts the tensor-core Gram G + E (|E_ij| within _gram_bound)
    tol = _inverse_tol(ref, G, Bm, form, mu)
    assert np.max(np.abs(Fn - ref)) <= tol
    assert np.max(np.abs(Fn @ G - np.eye(n))) <= 1e-13 * cond * n + np.linalg.norm(G, 2) * tol * n


def _inverse_tol(ref, G, Bm_gram, form, mu):
    """Bound of |F - G^{-1}| for a factor computed from the tensor-core Gram
    of the columns Bm_gram (error E entrywise within _gram_bound; a downdate
    or update carries E along) and then inverted in FP64:
    ||G^{-1}||^2 ||E|| / (1 - ||G^{-1}|| ||E||) + 1e-14 cond(G) max|G^{-1}| n."""
    n = G.shape[0]
    Enorm = np.linalg.norm(_gram_bound(Bm_gram, form, mu))
    r2 = np.linalg.norm(ref, 2)
    assert r2 * Enorm < 0.5
    return 1e-14 * np.linalg.cond(G) * np.max(np.abs(ref)) * n + r2 ** 2 * Enorm / (1 - r2 * Enorm)


def _row_exponents(R):
    """Least e with max |row| <= 2^e, per row of R (0 for a zero row)."""
    m = np.max(np.abs(R), axis=1)
    e = np.zeros(len(m), dtype=np.int64)
    nz = m > 0
    e[nz] = np.frexp(m[nz])[1]
    return e


def _gram_bound(Bm, form, mu):
    """Entrywise bound of the tensor-core Gram's error against the exact Gram
    (the arithmetic of the digit method): each Gram row is scaled by 2^-e to
    [-1, 1] and cut into four 8-bit digits (the rest, at most 2^-32, is
    dropped); of the digit products, the orders 6..8 (3 + 2 + 1 pairs of
    weight 2^-32, 2^-40, 2^-48 against the leading 2^-14 scale x 2^14) are
    dropped: at most 5 x 2^-32 per term; the double-float totals add 2^-46 of
    the sum of magnitudes.  Returns mu 2^(e_i + e_j) (K 2^-29.6 + 2^-46 K)."""
    R = Bm.T if form == 0 else Bm            # Gram rows (primal: pixels; Woodbury: real rows)
    e = _row_exponents(R)
    K = R.shape[1]
    return mu * np.ldexp(1.0, (e[:, None] + e[None, :]).astype(np.int64)) * K * (5 * 2.0 ** -32 + 2.0 ** -46)


GRAM_CASES = [
    # KM, N, nidx: primal when nidx <= 2 KM (rows = pixels, k = 2KM real rows),
    # Woodbury otherwise (rows = 2KM real rows, k = pixels)
    (256, 300, 300),      # primal: 300 rows -> 3 row blocks (ragged), 2 chunks of k
    (2048, 700, 129),     # primal: 16 chunks of k, one row past a block
    (64, 300, 300),       # Woodbury: 128 rows, 300 pixels -> 2 chunks (ragged)
    (32, 2000, 1500),     # Woodbury: 64 rows (one partial block), 6 chunks
    (96, 1000, 999),      # Woodbury: 192 rows (ragged second block)
]


@pytest.mark.parametrize("KM,N,nidx", GRAM_CASES)
def test_tensor_core_gram_is_exact_on_16_bit_entries(B, KM, N, nidx):
    """Operator entries that are multiples of 2^-15 in (-1, 1) have only two
    nonzero digits, so no digit product is dropped and every chunk sum is an
    exact integer: the tensor-core Gram (method 0) must equal the FP64 Gram
    bit for bit, padding (identity) included, for any active subset."""
    s = scenegen.Stream(41, KM + nidx)
    re = s.integers(N * KM, 65535).reshape(N, KM) - 32767
    im = s.integers(N * KM, 65535).reshape(N, KM) - 32767
    A = ((re + 1j * im) / 32768.0).astype(np.complex64)
    idx = np.sort(s.permutation(N)[:nidx]).astype(np.int32)
    dev = torch.device("cuda:0")
    mu, rho = 1.0, 0.5
    F, form, n = B.gram(torch.from_numpy(A).to(dev), torch.from_numpy(idx).to(dev), mu, rho, method=0)
    F = F.cpu().numpy()
    Bm = _interleaved_real_form(A, idx)
    G = Bm @ Bm.T if form == 1 else Bm.T @ Bm
    assert form == (1 if nidx > 2 * KM else 0) and n == G.shape[0]
    npad = F.shape[0]
    ref = np.eye(npad)
    ref[:n, :n] = mu * G + rho * np.eye(n)
    assert np.array_equal(F, ref)


@pytest.mark.parametrize("KM,N,nidx", GRAM_CASES + [(256, 1024, 1024), (4096, 4096, 4096)])
def test_tensor_core_gram_matches_fp64(B, KM, N, nidx):
    """General FP32 operators (Gaussian and, in the last case, the radar
    signal model): the tensor-core Gram is within the entrywise bound of its
    arithmetic (_gram_bound) of the exact FP64 Gram, and so is the SIMT FP64
    method (method 1) to 2^-40 relative."""
    A = _operator(KM, N, seed=3 * KM + nidx, radar=(N == 1024))
    idx = np.sort(scenegen.Stream(43, nidx).permutation(N)[:nidx]).astype(np.int32)
    dev = torch.device("cuda:0")
    mu, rho = 1.3, 0.7
    At, it = torch.from_numpy(A).to(dev), torch.from_numpy(idx).to(dev)
    F0, form, n = B.gram(At, it, mu, rho, method=0)
    F0 = F0.cpu().numpy()[:n, :n]
    Bm = _interleaved_real_form(A, idx)
    G = mu * (Bm @ Bm.T if form == 1 else Bm.T @ Bm) + rho * np.eye(n)
    assert np.all(np.abs(F0 - G) <= _gram_bound(Bm, form, mu))
    assert np.array_equal(F0, F0.T)
    if KM % 8 == 0:
        F1 = B.gram(At, it, mu, rho, method=1)[0].cpu().numpy()[:n, :n]
        assert np.max(np.abs(F1 - G)) <= 2.0 ** -40 * np.max(np.abs(G))


@pytest.mark.parametrize("n,ld", [(1, 2), (37, 64), (101, 102), (4096, 4096)])
def test_spd_apply_matches_fp64(B, n, ld):
    s = scenegen.Stream(9, n)
    M = s.normal(n * n).reshape(n, n)
    F = np.zeros((ld, ld))
    F[:n, :n] = M + M.T
    u = s.normal(n).astype(np.float32)
    dev = torch.device("cuda:0")
    out = B.spd_apply(torch.from_numpy(F).to(dev), n, torch.from_numpy(u).to(dev))
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    ref = F[:n, :n] @ u.astype(np.float64)
    mag = np.abs(F[:n, :n]) @ np.abs(u.astype(np.float64))
    # exact products summed as FP32 pairs (about 48 bits), rounded once to FP32;
    # the pair split of F itself costs 2^-48 relative per element
    assert np.all(np.abs(out - ref) <= U32 * np.abs(ref) + (2 * n + 8) * 2.0 ** -47 * mag)


def test_bounded_wait_runs_out_and_the_next_call_succeeds(B):
    """The factor apply's tile-copy wait is bounded: with its limit set to
    zero polls every wait gives up at once, the CTA waits (with the full
    limit) for its copy in flight and the call reports SADMM_ETIMEOUT, with
    the context still usable; with the limit restored the same call succeeds
    and is correct.  Also through the solver: a solve under the zero limit
    reports SADMM_ETIMEOUT, and the next solve matches a clean run."""
    n, ld = 300, 320
    s = scenegen.Stream(19, n)
    M = s.normal(n * n).reshape(n, n)
    F = np.zeros((ld, ld))
    F[:n, :n] = M + M.T
    u = s.normal(n).astype(np.float32)
    dev = torch.device("cuda:0")
    Ft, ut = torch.from_numpy(F).to(dev), torch.from_numpy(u).to(dev)
    try:
        B.set_wait_limit(0)
        with pytest.raises(B.SadmmError) as ei:
            B.spd_apply(Ft, n, ut)
        assert ei.value.status == B.ETIMEOUT
    finally:
        B.set_wait_limit(-1)
    out = B.spd_apply(Ft, n, ut).cpu().numpy().astype(np.float64)
    ref = F[:n, :n] @ u.astype(np.float64)
    mag = np.abs(F[:n, :n]) @ np.abs(u.astype(np.float64))
    assert np.all(np.abs(out - ref) <= U32 * np.abs(ref) + (2 * n + 8) * 2.0 ** -47 * mag)

    sc = scenegen.build_scene("small_point", seed=3)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    g = sc.geom
    sol = B.Solver(g.Q, g.M, g.K, g.N, 1.0, lam, elim=0)
    try:
        for q in range(g.Q):
            sol.set_operator(q, sc.A[q])
        sol.prepare()
        xg_ref, _ = sol.solve(sc.y, 10)
        X_ref = sol.X()
        try:
            B.set_wait_limit(0)
            with pytest.raises(B.SadmmError) as ei:
                sol.solve(sc.y, 10)
            assert ei.value.status == B.ETIMEOUT
        finally:
            B.set_wait_limit(-1)
        sol.solve(sc.y, 10)
        assert np.array_equal(sol.X(), X_ref)
    finally:
        sol.close()


@pytest.mark.parametrize("KM,N,e", [(32, 300, 1), (32, 300, 7), (128, 700, 40), (256, 1024, 3)])
def test_factor_downdate_matches_fresh_inverse(B, KM, N, e):
    """Rank-e downdate of the Woodbury factor equals the FP64 inverse of the
    Gram without the removed columns."""
    A = _operator(KM, N, seed=KM + 3 * N + e, radar=(KM == 256))
    mu, rho = 1.0, 1.0
    s = scenegen.Stream(13, e)
    J = np.arange(N, dtype=np.int32)
    E = np.sort(s.permutation(N)[:e]).astype(np.int32)
    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev)
    W, form, n = B.factor(At, torch.from_numpy(J).to(dev), mu, rho)
    assert form == 1
    B.factor_downdate(At, torch.from_numpy(E).to(dev), mu, W)
    torch.cuda.synchronize()
    Wd = W.cpu().numpy()[:n, :n]
    keep = np.setdiff1d(J, E)
    Bm = _interleaved_real_form(A, keep)
    G = rho * np.eye(n) + mu * Bm @ Bm.T
    ref = np.linalg.inv(G)
    assert np.max(np.abs(Wd - ref)) <= _inverse_tol(ref, G, _interleaved_real_form(A, J), 1, mu)
    assert np.array_equal(Wd, Wd.T)


@pytest.mark.parametrize("KM,N,e", [(32, 300, 5), (128, 700, 40), (256, 1024, 33)])
def test_factor_rank_update_adds_columns(B, KM, N, e):
    """Rank-e update with sign -1 (columns re-admitted) of the Woodbury factor of
    a reduced set equals the FP64 inverse of the Gram of the enlarged set."""
    A = _operator(KM, N, seed=KM + 5 * N + e, radar=(KM == 256))
    mu, rho = 0.8, 1.3
    s = scenegen.Stream(17, e)
    R = np.sort(s.permutation(N)[:e]).astype(np.int32)
    J = np.setdiff1d(np.arange(N), R).astype(np.int32)
    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev)
    W, form, n = B.factor(At, torch.from_numpy(J).to(dev), mu, rho)
    assert form == 1
    B.factor_update(At, torch.from_numpy(R).to(dev), mu, -1, W)
    torch.cuda.synchronize()
    Wu = W.cpu().numpy()[:n, :n]
    Bm = _interleaved_real_form(A, np.arange(N))
    G = rho * np.eye(n) + mu * Bm @ Bm.T
    ref = np.linalg.inv(G)
    assert np.max(np.abs(Wu - ref)) <= _inverse_tol(ref, G, _interleaved_real_form(A, J), 1, mu)
    assert np.array_equal(Wu, Wu.T)


@pytest.mark.parametrize("KM,N", [(16, 128), (32, 200), (256, 1024), (2048, 300), (4096, 8192)])
def test_tensor_core_adjoint16_matches_fp64(B, KM, N):
    """Batched adjoint on tcgen05 (3xTF32 split, FP32 accumulation) against the
    FP64 product: each of the 2KM terms is within 2^-21 of its exact value and
    the FP32 accumulation adds at most 2KM roundings (or truncations, 2^-23) of
    the running magnitude, so |G - G64| <= (2KM 2^-23 + 2^-20) sum |a||w|."""
    A = _operator(KM, N, seed=KM + N, radar=(KM == 256))
    s = scenegen.Stream(31, N)
    W = (s.normal(KM * 16) + 1j * s.normal(KM * 16)).reshape(KM, 16).astype(np.complex64)
    dev = torch.device("cuda:0")
    G = B.adjoint16_tc(torch.from_numpy(A).to(dev), torch.from_numpy(W).to(dev)).cpu().numpy().astype(np.float64)
    A64, W64 = A.astype(np.complex128), W.astype(np.complex128)
    ref = (A64.conj() @ W64).real
    mag = np.abs(A64.real) @ np.abs(W64.real) + np.abs(A64.imag) @ np.abs(W64.imag)
    bound = (2 * KM * 2.0 ** -23 + 2.0 ** -20) * mag
    err = np.abs(G - ref)
    print(f"KM={KM} N={N}: max |G - G64| / bound = {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("KM,N", [(8, 100), (72, 200), (256, 1024), (2048, 9216), (4096, 8192)])
def test_tensor_core_forward16_matches_fp64(B, KM, N):
    """Batched forward on tcgen05 (transposing 3xTF32 split, FP32
    accumulation over the N pixels) against the FP64 product A^T V: each term
    within 2^-21 of its exact value and at most N FP32 roundings (or
    truncations, 2^-23) of the running magnitude, so |R - R64| <= (N 2^-23 +
    2^-20) sum |a||v| per real and imaginary part (ragged N and 2KM/128)."""
    A = _operator(KM, N, seed=7 * KM + N, radar=(KM == 256))
    s = scenegen.Stream(37, N)
    V = s.normal(N * 16).reshape(N, 16).astype(np.float32)
    V[:, 3] = 0.0
    dev = torch.device("cuda:0")
    R = B.forward16_tc(torch.from_numpy(A).to(dev), torch.from_numpy(V).to(dev)).cpu().numpy().astype(np.complex128)
    A64, V64 = A.astype(np.complex128), V.astype(np.float64)
    ref = A64.T @ V64
    for part in (np.real, np.imag):
        mag = np.abs(part(A64)).T @ np.abs(V64)
        bound = (N * 2.0 ** -23 + 2.0 ** -20) * mag
        err = np.abs(part(R) - part(ref))
        print(f"KM={KM} N={N}: max |R - R64| / bound = {np.max(err / np.maximum(bound, 1e-300)):.3f}")
        assert np.all(err <= bound)
    assert np.all(R[:, 3] == 0)


# ------------------------------------------- batched factor apply (digits)
def _digit_entries(s, rows, cols, ndig):
    """Values that are exactly ndig balanced 8-bit digits below 2^7: d_0 +
    2^-8 d_1 + ..., |d_a| <= 127, and one entry of 100 per row (so that the
    row scale 2^-e_i is 2^-7 and the digits are the ones drawn)."""
    D = [s.integers(rows * cols, 255).reshape(rows, cols).astype(np.int64) - 127 for _ in range(ndig)]
    D[0][np.arange(rows), s.integers(rows, cols)] = 100
    v = sum(D[a].astype(np.float64) * 2.0 ** (-8 * a) for a in range(ndig))
    return v, D


@pytest.mark.parametrize("n", [1, 200, 1000, 4133])
def test_digit_apply_is_exact_on_integers(B, n):
    """Integer F and U with |entries| <= 128: every digit but the first is
    zero and the chunk sums are exact, so the tensor-core apply equals the
    integer product exactly (ragged n, several 256-chunks and row blocks)."""
    s = scenegen.Stream(71, n)
    F = s.integers(n * n, 257).reshape(n, n).astype(np.float64) - 128
    U = (s.integers(n * 16, 257).reshape(n, 16) - 128).astype(np.float32)
    U[:, 5] = 0.0                                     # a zero right-hand side
    F[n // 2, :] = 0.0                                # a zero row
    dev = torch.device("cuda:0")
    out = B.digit_apply16(torch.from_numpy(F).to(dev), torch.from_numpy(U).to(dev)).cpu().numpy()
    ref = F.astype(np.int64) @ U.astype(np.int64)
    assert np.array_equal(out, ref.astype(np.float64))


@pytest.mark.parametrize("n", [300, 2000])
def test_digit_apply_keeps_orders_zero_to_three(B, n):
    """F with four exact digits per entry, U with three: the apply forms the
    digit products of orders 0..3 exactly (orders 4..6 are dropped by
    design), so its result equals that truncated sum, computed here in exact
    integer arithmetic, to the double-float totals' rounding: four additions
    per 256-chunk, each within 2^-48 of the running total, one or two chunks
    per work item at these sizes (2^-44 of sum |F||U|)."""
    s = scenegen.Stream(72, n)
    F, DF = _digit_entries(s, n, n, 4)
    Ut, DU = _digit_entries(s, 16, n, 3)               # columns of U as rows
    U = Ut.T.astype(np.float32)
    assert np.array_equal(U.astype(np.float64), Ut.T)
    DU = [d.T for d in DU] + [np.zeros((n, 16), np.int64)]
    dev = torch.device("cuda:0")
    out = B.digit_apply16(torch.from_numpy(F).to(dev), torch.from_numpy(U).to(dev)).cpu().numpy()
    # sum_{a+b<=3} 2^(-8(a+b)) D_a E_b, scaled by 2^24 to integers
    T = sum((DF[a] @ DU[b]) * (1 << (8 * (3 - a - b))) for a in range(4) for b in range(4) if a + b <= 3)
    ref = T.astype(np.float64) * 2.0 ** -24
    full = F @ Ut.T
    mag = np.abs(F) @ np.abs(Ut.T)
    assert np.all(np.abs(out - ref) <= 2.0 ** -44 * mag)
    # and the dropped orders are visible: the exact product differs
    assert np.max(np.abs(full - ref)) > 2.0 ** -40 * np.max(mag)


@pytest.mark.parametrize("n", [129, 3000, 16384])
def test_digit_apply_matches_fp64(B, n):
    """General FP64 F (rows scaled over six decades) and FP32 U (columns over
    four, one zero): within the apply's entrywise bound 5 * 2^-32 * n *
    2^(e_i + f_s) of the FP64 product (the three slicing and truncation
    terms), at the batched form's full primal size among others."""
    s = scenegen.Stream(73, n)
    w = min(n, 512)                                   # a drawn panel, tiled and rescaled per column
    F = np.tile(s.normal(n * w).reshape(n, w), (1, -(-n // w)))[:, :n]
    F *= s.uniform(n, 0.5, 1.5)[None, :] * (10.0 ** s.uniform(n, -3, 3))[:, None]
    U = (s.normal(n * 16).reshape(n, 16) * (10.0 ** s.uniform(16, -2, 2))[None, :]).astype(np.float32)
    U[:, 11] = 0.0
    dev = torch.device("cuda:0")
    out = B.digit_apply16(torch.from_numpy(F).to(dev), torch.from_numpy(U).to(dev)).cpu().numpy()
    ref = F @ U.astype(np.float64)
    ei = np.frexp(np.max(np.abs(F), axis=1))[1].astype(np.float64)
    fs = np.frexp(np.max(np.abs(U.astype(np.float64)), axis=0))[1].astype(np.float64)
    bound = 5.0 * 2.0 ** -32 * n * np.exp2(ei[:, None] + fs[None, :])
    assert np.all(np.abs(out - ref) <= bound)
    assert np.all(out[:, 11] == 0.0)
    # typical error far inside the bound (random rounding, not a lost order)
    scale = np.exp2(ei[:, None] + fs[None, :]) * np.sqrt(n)
    assert np.sqrt(np.mean(((out - ref) / scale) ** 2)) <= 2.0 ** -30
