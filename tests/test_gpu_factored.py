"""Factored (matrix-free) operator: the tables built from the round-trip delays
and the products that read them, against the FP64 oracle's signal-model
operator (Section II, Eq. 1), and the solver running on them against the
oracle iterates (Eq. 3 with Algorithm 1).

Bars, from the arithmetic (u = 2^-24):
* stored entries: FP64 phases rounded once to complex64, |A - A64| <= u per
  component; the factors C and D likewise, and the factored entry C D within
  3u of A64;
* forward r = base - A_J v: each term within 3u (factored entry) + u (v C),
  FP32 sums over at most 32 pixels of a stage (<= 32u of their sum of |terms|),
  double-float across stages and chunks, one final rounding:
  |r - r64| <= 40u sum|A||v| + 2u (|base| + |r64|);
* adjoint g = Re(A_J^H w): 16-term FP32 sums t_a (<= 16u), the C product and
  its double-float sum over (m, a): |g - g64| <= 24u sum|A||w| + u|g64|;
* solver: stacked iterate within 1e-4 of the oracle at equal k, active sets
  bit-identical while the decision margins stay above delta (as the stored
  operator's solver tests)."""
import numpy as np
import pytest

import oracle
import scenegen
from scenegen import radar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_08606_gb300 import build, binding
    build()
    binding.load()
    return binding


def _geom(M, K, nx, Q=2):
    return scenegen.Geometry(Q=Q, M=M, K=K, nx=nx, cell=0.05, radius=10.0, fc=77e9, bw=1e9)


def _tables(B, g, q):
    dev = torch.device("cuda:0")
    tau = radar.delays(g, q)
    A, Ct, Dt = B.operator_tables(torch.from_numpy(tau).to(dev), g.M, g.K, g.N, g.fc, g.bw / g.K)
    torch.cuda.synchronize()
    return tau, A, Ct, Dt


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


@pytest.mark.parametrize("M,K,nx", [(4, 64, 16), (2, 512, 8), (16, 16, 8)])
def test_tables_match_signal_model(B, M, K, nx):
    g = _geom(M, K, nx)
    tau, A, Ct, Dt = _tables(B, g, 1)
    A64 = oracle.operator_from_delays(tau, g.fc, g.bw / g.K, g.K)
    Ah = A.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(Ah.real - A64.real)) <= U + 1e-12
    assert np.max(np.abs(Ah.imag - A64.imag)) <= U + 1e-12
    # the scene generator's complex64 operator: the same values but for rounding ties
    assert np.max(np.abs(Ah - radar.operator(g, 1).astype(np.complex128))) <= 2 * U
    Ch = Ct.cpu().numpy().astype(np.complex128)          # (M, K/16, N)
    Dh = Dt.cpu().numpy().astype(np.complex128)          # (M, 16, N)
    Ar = Ah.reshape(g.N, M, K)
    for a in range(K // 16):
        assert np.array_equal(Ch[:, a, :], Ar[:, :, 16 * a].T)
    b = np.arange(16)
    Dexact = np.exp(2j * np.pi * tau[:, None, :] * (b[None, :, None] * (g.bw / g.K)))
    assert np.max(np.abs(Dh - Dexact)) <= 2 * U
    prod = (Ch[:, :, None, :] * Dh[:, None, :, :]).reshape(M, K, g.N)        # entry k = 16 a + b
    A64r = A64.reshape(g.N, M, K).transpose(1, 2, 0)
    assert np.max(np.abs(prod - A64r)) <= 3 * U


@pytest.mark.parametrize("M,K,nx,nidx", [(4, 64, 32, 700), (8, 256, 64, 3000), (2, 16, 24, 577),
                                         (3, 512, 16, 256), (4, 64, 32, 0), (32, 32, 16, 200)])
def test_factored_forward_matches_oracle(B, M, K, nx, nidx):
    g = _geom(M, K, nx)
    dev = torch.device("cuda:0")
    tau, _, Ct, Dt = _tables(B, g, 0)
    A64 = oracle.operator_from_delays(tau, g.fc, g.bw / g.K, g.K)
    s = scenegen.Stream(71, M * K + nidx)
    idx = s.permutation(g.N)[:nidx].astype(np.int32)
    v = s.normal(g.N).astype(np.float32)
    base = (s.normal(g.KM) + 1j * s.normal(g.KM)).astype(np.complex64)
    r = B.forward_factored(Ct, Dt, K, torch.from_numpy(idx).to(dev), torch.from_numpy(v).to(dev),
                           base=torch.from_numpy(base).to(dev))
    torch.cuda.synchronize()
    got = r.cpu().numpy().astype(np.complex128)
    Asel = A64[idx]
    ref = base.astype(np.complex128) - Asel.T @ v[idx].astype(np.float64)
    mag = np.abs(Asel).T @ np.abs(v[idx].astype(np.float64))
    tol = 40 * U * mag + 2 * U * (np.abs(base) + np.abs(ref))
    assert np.all(np.abs(got.real - ref.real) <= tol)
    assert np.all(np.abs(got.imag - ref.imag) <= tol)
    if nidx == 0:
        assert np.array_equal(r.cpu().numpy(), base)


@pytest.mark.parametrize("M,K,nx,nidx", [(4, 64, 32, 700), (8, 256, 64, 4096), (16, 16, 12, 100),
                                         (2, 512, 16, 33), (32, 32, 16, 200)])
def test_factored_adjoint_matches_oracle(B, M, K, nx, nidx):
    g = _geom(M, K, nx)
    dev = torch.device("cuda:0")
    tau, _, Ct, Dt = _tables(B, g, 1)
    A64 = oracle.operator_from_delays(tau, g.fc, g.bw / g.K, g.K)
    s = scenegen.Stream(72, M * K + nidx)
    idx = s.permutation(g.N)[:nidx].astype(np.int32)
    w = (s.normal(g.KM) + 1j * s.normal(g.KM)).astype(np.complex64)
    out = B.adjoint_factored(Ct, Dt, K, torch.from_numpy(idx).to(dev), torch.from_numpy(w).to(dev))
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    Asel = A64[idx]
    ref = oracle.adjoint_re(Asel, w.astype(np.complex128))
    mag = np.abs(Asel) @ np.abs(w.astype(np.complex128))
    assert np.all(np.abs(got - ref) <= 24 * U * mag + U * np.abs(ref))


def _delay_solver(B, sc, rho, lam, **crit):
    g = sc.geom
    s = B.Solver(g.Q, g.M, g.K, g.N, rho, lam, **crit)
    for q in range(g.Q):
        s.set_operator_delays(q, radar.delays(g, q), g.fc, g.bw / g.K)
    return s


def test_solver_on_factored_operator_matches_oracle(B):
    """small_point (Q=4, M=4, K=64, N=32x32): the solver with every operator set
    from its delays runs the factored products and matches the oracle's
    iterate (on the scene generator's complex64 operator) within 1e-4; the
    same solver forced to the stored operator differs from it only by the
    entry rounding (2e-4), and asking for factored products while a sensor has
    no delays is refused."""
    sc = scenegen.build_scene("small_point", seed=0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    iters = 80
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=iters)
    s = _delay_solver(B, sc, 1.0, lam, elim=0)
    xg, st = s.solve(sc.y, iters)
    Xf = s.X()
    assert st["iters"] == iters
    assert _rel(Xf, ref.state.x) <= 1e-4
    if np.any(ref.xG != 0):
        assert _rel(xg, ref.xG) <= 1e-4
    s.set_products(1)
    s.solve(sc.y, iters)
    Xs = s.X()
    assert _rel(Xs, ref.state.x) <= 1e-4
    assert _rel(Xf, Xs) <= 2e-4
    assert not np.array_equal(Xf, Xs)           # the two representations really ran
    s.close()
    t = B.Solver(sc.geom.Q, sc.geom.M, sc.geom.K, sc.geom.N, 1.0, lam, elim=0)
    for q in range(sc.geom.Q):
        if q == 0:
            t.set_operator(q, sc.A[q])
        else:
            t.set_operator_delays(q, radar.delays(sc.geom, q), sc.geom.fc, sc.geom.bw / sc.geom.K)
    t.set_products(2)
    with pytest.raises(B.SadmmError) as e:
        t.solve(sc.y, 1)
    assert e.value.status == B.ENOTREADY
    t.close()


def test_solver_on_factored_operator_with_elimination(B):
    """resolved_tiny (Q=3, M=16, K=16: one C factor per antenna; N < 2KM, so
    the primal x-update, where factored products run only when asked for) with
    Algorithm 1 on: iterate within 1e-4 of the oracle and the same active sets
    while the decision margins allow (this geometry is well conditioned)."""
    sc = scenegen.build_scene("resolved_tiny", seed=2, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    crit = oracle.Criterion(elim=1, Kp=4)
    iters = 150
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=iters)
    s = _delay_solver(B, sc, 1.0, lam, elim=1, Kp=4)
    s.set_products(2)           # the primal form: automatic selection would take the stored operator
    s.solve(sc.y, iters)
    assert _rel(s.X(), ref.state.x) <= 1e-4
    ok = all(h["gate_margin"] >= 1e-3 and (not h["gate"] or h["zeta_margin"] >= 0.1 * crit.eps_p)
             for h in ref.history)
    if ok:
        for q in range(sc.geom.Q):
            assert np.array_equal(s.active(q), ref.state.J[q])
    s.close()


@pytest.mark.parametrize("representation", ["stored", "factored"])
def test_backprojection_matches_oracle(B, representation):
    """Composite BP image sum_q |A_q^H y_q| (sadmm_backprojection) on the
    small_point scene against the oracle's, with the operator the library
    reads (the scene generator's complex64 entries for the stored form; the
    exact signal-model operator for the factored tables).  Per pixel:
    each real adjoint is within c u sum_r |a_r||y_r| (c = 8 stored: FP32
    partials of four products and a double-float sum; c = 24 factored, as
    the factored adjoint test), the magnitude within the sum of the two, and
    the FP32 sum over sensors adds 4u |bp|.  The solver state is left alone:
    a solve after the back-projection equals one before it."""
    sc = scenegen.build_scene("small_point", seed=0)
    g = sc.geom
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    if representation == "stored":
        s = B.Solver(g.Q, g.M, g.K, g.N, 1.0, lam, elim=0)
        for q in range(g.Q):
            s.set_operator(q, sc.A[q])
        A_ref = [a.astype(np.complex128) for a in sc.A]
        c = 8
    else:
        s = _delay_solver(B, sc, 1.0, lam, elim=0)
        A_ref = [oracle.operator_from_delays(radar.delays(g, q), g.fc, g.bw / g.K, g.K) for q in range(g.Q)]
        c = 24
    x0, _ = s.solve(sc.y, 20)
    X0 = s.X()
    got = s.backprojection(sc.y).astype(np.float64)
    ref = oracle.backprojection(A_ref, sc.y)
    mag = sum(np.abs(A_ref[q]) @ np.abs(sc.y[q].astype(np.complex128)) for q in range(g.Q))
    assert np.all(np.abs(got - ref) <= 2 * c * U * mag + 4 * U * ref)
    x1, _ = s.solve(sc.y, 20)
    assert np.array_equal(s.X(), X0) and np.array_equal(x1, x0)
    s.close()
