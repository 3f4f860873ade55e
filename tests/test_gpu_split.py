"""Split-precision operator (A = A_hi + A_lo in BF16 or FP16 planes): kernel
parity of the plane conversion and the split GEMVs, and solver accuracy of the
precision forms against the FP64 oracle (which uses the complex64 operator).

Bounds: round-to-nearest into a format with unit roundoff u gives
|a - hi| <= u|a| and |a - hi - lo| <= u^2|a| (BF16 u = 2^-8, FP16 u = 2^-11; FP16
lo values below 2^-14 are subnormal, absolute spacing 2^-24)."""
import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
BF16, FP16 = 1, 2


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_08606_gb300 import build, binding
    build()
    binding.load()
    return binding


def _decode(plane, kind):
    """16-bit plane (int16 tensor, (..., 2)) -> complex128 numpy."""
    bits = plane.cpu().numpy().view(np.uint16)
    if kind == FP16:
        f = bits.view(np.float16).astype(np.float64)
    else:
        f = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


def _radar(KM=256, nx=32):
    g = scenegen.Geometry(Q=1, M=KM // 32, K=32, nx=nx, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    return scenegen.operator(g, 0)


@pytest.mark.parametrize("kind", [BF16, FP16])
def test_planes_reconstruct_the_operator(B, kind):
    A = _radar()
    dev = torch.device("cuda:0")
    hi, lo = B.split_operator(torch.from_numpy(A).to(dev), kind)
    torch.cuda.synchronize()
    h, l = _decode(hi, kind), _decode(lo, kind)
    a = A.astype(np.complex128)
    u = 2.0 ** -8 if kind == BF16 else 2.0 ** -11
    sub = 0.0 if kind == BF16 else 2.0 ** -25     # half spacing of FP16 subnormals
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(a) - part(h)) <= u * np.abs(part(a)) + sub)
        assert np.all(np.abs(part(a) - part(h) - part(l)) <= u * u * np.abs(part(a)) + sub)


@pytest.mark.parametrize("kind", [BF16, FP16])
@pytest.mark.parametrize("planes", [1, 2, 3])
def test_split_products_match_fp64(B, kind, planes):
    A = _radar()
    N, KM = A.shape
    dev = torch.device("cuda:0")
    hi, lo = B.split_operator(torch.from_numpy(A).to(dev), kind)
    P = (_decode(hi, kind) if planes & 1 else 0) + (_decode(lo, kind) if planes & 2 else 0)
    s = scenegen.Stream(17, planes)
    idx = np.sort(s.permutation(N)[:777]).astype(np.int32)
    v = s.normal(N).astype(np.float32)
    w = (s.normal(KM) + 1j * s.normal(KM)).astype(np.complex64)
    it = torch.from_numpy(idx).to(dev)
    r = B.forward_split(hi, lo, kind, planes, it, torch.from_numpy(v).to(dev)).cpu().numpy()
    g = B.adjoint_split(hi, lo, kind, planes, it, torch.from_numpy(w).to(dev)).cpu().numpy()
    Ps = P[idx]
    ref_r = -(Ps.T @ v[idx].astype(np.float64))
    mag_r = np.abs(Ps.real).T @ np.abs(v[idx]) + 1j * (np.abs(Ps.imag).T @ np.abs(v[idx]))
    n = len(idx) + 2
    assert np.all(np.abs(r.real - ref_r.real) <= n * U32 * mag_r.real)
    assert np.all(np.abs(r.imag - ref_r.imag) <= n * U32 * mag_r.imag)
    ref_g = (Ps.conj() @ w.astype(np.complex128)).real
    mag_g = np.abs(Ps.real) @ np.abs(w.real) + np.abs(Ps.imag) @ np.abs(w.imag)
    assert np.all(np.abs(g - ref_g) <= (2 * KM + 4) * U32 * mag_g)


def _run(B, sc, lam, iters, **crit):
    g = sc.geom
    s = B.Solver(g.Q, g.M, g.K, g.N, 1.0, lam, **crit)
    for q in range(g.Q):
        s.set_operator(q, sc.A[q])
    xg, st = s.solve(sc.y, iters)
    X = s.X()
    s.close()
    return xg, X, st


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair_scene(sc, kind):
    """The scene with each operator replaced by its pair operator hi + lo
    (oracle.precision, rounded on the oracle side): what the split forms solve."""
    import dataclasses
    return dataclasses.replace(sc, A=[oracle.precision.pair_operator(a, kind) for a in sc.A])


@pytest.mark.parametrize("precision", [1, 2])
def test_pair_forms_match_the_oracle_on_the_pair_operator(B, precision):
    """BF16 (1) and FP16 (2) hi/lo pairs, 300 plain SADMM iterations on the
    32x32 scene: the split form solves Eq. 2 for the pair operator P = hi + lo
    (products, factor and fold all use P), so at equal k its stacked iterate
    matches the FP64 oracle run on P to the FP32 path's bar, 1e-4.  Against
    the oracle on the complex64 operator the difference is the problem's own
    sensitivity to the 2^-16 / 2^-22 operator change (printed)."""
    sc = scenegen.build_scene("small_point", seed=0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    scp = _pair_scene(sc, precision)
    ref_p = oracle.sadmm(scp.A, scp.y, 1.0, lam, oracle.Criterion(elim=0), iters=300)
    ref_a = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=300)
    _, X, st = _run(B, sc, lam, 300, elim=0, precision=precision)
    err_p, err_a = _rel(X, ref_p.state.x), _rel(X, ref_a.state.x)
    print(f"precision {precision}: vs oracle on P {err_p:.3e}, vs oracle on A {err_a:.3e}")
    assert err_p <= 1e-4


@pytest.mark.parametrize("precision", [1, 3, 4])
def test_hi_plane_with_periodic_correction_reaches_the_limit(B, precision):
    """hi plane every iteration, lo-plane products refreshed every 4 iterations:
    at a fixed point the refreshed products are exact, so the limit on a
    well-posed scene is the oracle's limit (x_G within 1e-3)."""
    sc = scenegen.build_scene("resolved_tiny", seed=1, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=20000, tol=1e-15)
    xg, X, st = _run(B, sc, lam, 6000, elim=0, precision=precision, correct_every=4)
    err = _rel(xg, ref.xG)
    print(f"precision {precision}: |xG - xG_oracle_limit| / |xG_oracle_limit| = {err:.3e}")
    assert err <= 1e-3
    assert st["bytes_iter"] > 0


@pytest.fixture(scope="module")
def twin():
    sc = scenegen.build_scene("precision_twin", seed=0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=20)
    B0 = oracle.real_form(sc.A[0])
    ev = np.linalg.eigvalsh(B0.T @ B0)
    cond_h = (1.0 + ev[-1]) / (1.0 + max(ev[0], 0.0))        # rho = mu = 1
    return sc, lam, ref, cond_h


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4])
def test_precision_workload_twin_matches_the_oracle(B, twin, precision):
    """The precision workload's sensors (Q=8, M=16, K=512: KM=8192) on its
    64x64 twin, 20 plain SADMM iterations against the FP64 oracle at equal k,
    bar 1e-4 for every form.  Here 2KM > N, so the x-update is the primal
    x = v + mu H g, and B^T B is rank-deficient: cond(H) = cond(rho I + mu B^T B)
    is about 3.5e5, and any error in g outside the range of B^T is amplified by
    up to that factor.  Every form therefore forms g from exact products in
    double-float and passes it to the factor apply as a pair, and the split
    forms (1, 2: pairs; 3, 4: hi plane with the lo-plane products refreshed
    every iteration here, correct_every = 1) factor the pair operator P they
    read, so each is compared with the oracle run on its own operator (A for
    FP32, P for the planes).  The distance to the oracle on A -- the
    problem's sensitivity to the 2^-16 (BF16) or 2^-22 (FP16) operator change,
    amplified by cond(H) -- is printed."""
    sc, lam, ref, cond_h = twin
    kind = {0: 0, 1: BF16, 2: FP16, 3: BF16, 4: FP16}[precision]
    if kind:
        scp = _pair_scene(sc, kind)
        ref_p = oracle.sadmm(scp.A, scp.y, 1.0, lam, oracle.Criterion(elim=0), iters=20)
    else:
        ref_p = ref
    _, X, st = _run(B, sc, lam, 20, elim=0, precision=precision, correct_every=1)
    err_p, err_a = _rel(X, ref_p.state.x), _rel(X, ref.state.x)
    print(f"precision twin, precision {precision}: vs oracle on its operator {err_p:.3e}, "
          f"vs oracle on A {err_a:.3e} (cond(H) {cond_h:.2e})")
    assert st["iters"] == 20
    assert err_p <= 1e-4
