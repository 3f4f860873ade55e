"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an identity,
a closed form, an independent solver, brute force, or an invariant of
Algorithm 1.  The mutation tests at the end plant plausible mistakes in a copy of
the oracle and check that the pins catch them.
"""
import inspect
import sys
import types

import numpy as np
import pytest

import oracle
import oracle.sharing_admm as osadmm
import scenegen
from scenegen import radar


# ---------------------------------------------------------------- Eq. 1 products
def test_forward_matches_elementwise_sum():
    """A x computed one entry at a time (Eq. 1, with the pixel-major layout)."""
    sc = scenegen.random_problem(1, 6, 5, seed=3)
    A = sc.A[0]                       # (N, KM) pixel-major
    x = scenegen.Stream(9, 1).normal(5)
    ref = np.zeros(6, dtype=np.complex128)
    for r in range(6):
        for n in range(5):
            ref[r] += complex(A[n, r]) * x[n]
    assert np.allclose(oracle.forward(A, x), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_identity(seed):
    """Re<A x, r> = <x, Re(A^H r)> for real x, complex r (Eq. 1 operator)."""
    g = scenegen.GEOMS["small_point"]
    A = radar.operator(g, seed % g.Q)
    s = scenegen.Stream(seed, 7)
    x = s.normal(g.N)
    r = s.normal(g.KM) + 1j * s.normal(g.KM)
    lhs = np.vdot(r, oracle.forward(A, x)).real
    rhs = np.dot(x, oracle.adjoint_re(A, r))
    scale = np.linalg.norm(oracle.forward(A, x)) * np.linalg.norm(r)
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_real_form_consistent_with_complex_products():
    """B = [Re A; Im A]: ||y - A x||^2 = ||[Re y; Im y] - B x||^2 and
    Re(A^H y) = B^T [Re y; Im y] for real x."""
    sc = scenegen.random_problem(1, 16, 12, seed=5)
    A, y = sc.A[0], sc.y[0]
    B = oracle.real_form(A)
    x = scenegen.Stream(2, 2).normal(12)
    lhs = np.sum(np.abs(y.astype(np.complex128) - oracle.forward(A, x)) ** 2)
    rhs = np.sum((oracle.real_vec(y) - B @ x) ** 2)
    assert abs(lhs - rhs) <= 1e-12 * lhs
    assert np.allclose(B.T @ oracle.real_vec(y), oracle.adjoint_re(A, y), rtol=1e-13, atol=1e-12)


# ------------------------------------------------------------ Eq. 3 ingredients
def test_soft_threshold_is_the_prox():
    """soft(v, t) minimises t|x| + (x - v)^2 / 2: brute force on a fine grid,
    and the subgradient condition v - x in t d|x|."""
    s = scenegen.Stream(4, 4)
    v = s.uniform(200, -3, 3)
    t = s.uniform(200, 0, 2)
    x = oracle.soft(v, t)
    grid = np.linspace(-4, 4, 80001)
    for vi, ti, xi in zip(v[:40], t[:40], x[:40]):
        f = ti * np.abs(grid) + 0.5 * (grid - vi) ** 2
        assert abs(grid[np.argmin(f)] - xi) <= 1e-4
    nz = x != 0
    assert np.allclose(v[nz] - x[nz], t[nz] * np.sign(x[nz]), atol=1e-12)
    assert np.all(np.abs(v[~nz]) <= t[~nz] + 1e-15)


@pytest.mark.parametrize("nJ", [20, 200])
def test_ridge_solver_residual_and_forms_agree(nJ):
    """The x-update solve of Eq. 3: residual of (rho I + mu B_J^T B_J) x = b, for
    the primal Cholesky (|J| <= 2KM) and the Woodbury form (|J| > 2KM)."""
    sc = scenegen.random_problem(1, 32, 256, seed=11)
    B = oracle.real_form(sc.A[0])                        # 64 x 256
    J = np.sort(scenegen.Stream(1, 5).permutation(256)[:nJ])
    BJ = B[:, J]
    b = scenegen.Stream(2, 5).normal(nJ)
    mu, rho = 0.7, 1.3
    Hm = rho * np.eye(nJ) + mu * BJ.T @ BJ
    solver = oracle.RidgeSolver(BJ, mu, rho)
    assert solver.woodbury == (nJ > 64)
    x = solver.solve(b)
    assert np.linalg.norm(Hm @ x - b) <= 1e-12 * np.linalg.norm(b) * np.linalg.norm(Hm, 2)
    # the other form of the same solve
    x2 = np.linalg.solve(Hm, b)
    assert np.allclose(x, x2, rtol=1e-10, atol=1e-12 * np.linalg.norm(x2))


# ------------------------------------------------------- the whole iteration
def _resolved(seed=1, snr=30.0):
    sc = scenegen.build_scene("resolved_tiny", seed=seed, snr_db=snr)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    return sc, lam


@pytest.fixture(scope="module")
def converged_plain():
    sc, lam = _resolved()
    res = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=20000, tol=1e-15)
    return sc, lam, res


def test_kkt_at_the_limit(converged_plain):
    """With elimination off the limit satisfies Eq. 2's optimality conditions to 1e-8."""
    sc, lam, res = converged_plain
    k = oracle.kkt(sc.A, sc.y, res.state.x, res.state.s, 1.0, lam, xG=res.xG)
    assert k["stationarity"] <= 1e-8
    assert k["subgradient"] <= 1e-8
    assert k["feasibility"] <= 1e-8


def test_fista_agrees(converged_plain):
    """An independent proximal-gradient solve of Eq. 2 reaches the same minimiser
    (unique here: every sensor resolves the grid, 2KM > N)."""
    sc, lam, res = converged_plain
    Xf, fval = oracle.fista(sc.A, sc.y, lam, iters=6000, tol=1e-14)
    fa = oracle.objective(sc.A, sc.y, res.state.x, lam)
    assert abs(fa - fval) <= 1e-10 * abs(fval)
    assert np.max(np.abs(res.state.x - Xf)) <= 1e-6
    assert np.max(np.abs(res.xG - Xf.sum(axis=0))) <= 1e-6


@pytest.mark.parametrize("rho", [0.5, 4.0])
def test_kkt_other_rho_random_operator(rho):
    """Same optimality pin on unstructured operators and rho != 1, so that a
    rho-scaling slip in the prox threshold or the dual cannot hide."""
    sc = scenegen.random_problem(2, 24, 32, seed=21)
    lam = 0.1 * scenegen.lambda_max(sc.A, sc.y)
    res = oracle.sadmm(sc.A, sc.y, rho, lam, oracle.Criterion(elim=0, mu=0.8), iters=20000,
                       tol=1e-15)
    k = oracle.kkt(sc.A, sc.y, res.state.x, res.state.s, rho, lam, mu=0.8, xG=res.xG)
    assert max(k.values()) <= 1e-8
    Xf, fval = oracle.fista(sc.A, sc.y, lam, mu=0.8, iters=6000, tol=1e-14)
    assert abs(oracle.objective(sc.A, sc.y, res.state.x, lam, mu=0.8) - fval) <= 1e-10 * abs(fval)


def test_lasso_zero_above_lambda_max():
    """Q = 1 is the LASSO; for lambda >= mu ||Re(A^H y)||_inf the minimiser is 0,
    and the oracle stays at exactly zero."""
    sc = scenegen.random_problem(1, 24, 40, seed=8)
    lam = 1.0001 * scenegen.lambda_max(sc.A, sc.y)
    res = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=3000, tol=1e-14)
    assert np.all(res.xG == 0.0)
    k = oracle.kkt(sc.A, sc.y, res.state.x, res.state.s, 1.0, lam, xG=res.xG)
    assert max(k.values()) <= 1e-8


@pytest.mark.parametrize("name,sensors", [("resolved_tiny", None), ("small_point", [0])])
def test_single_point_target_recovered(name, sensors):
    """A noiseless single point target: argmax |x_G| is its pixel, and its value
    is the composite magnitude up to the l1 shrinkage bias."""
    g = scenegen.GEOMS[name]
    A = [radar.operator(g, q) for q in range(g.Q)]
    n0 = g.N // 2 + g.nx // 3
    x = np.zeros((g.Q, g.N))
    x[:, n0] = 0.8
    if sensors:
        A, x = [A[q] for q in sensors], x[sensors]
    y = radar.measure(A, x, None, 0)
    lam = 0.01 * scenegen.lambda_max(A, y)
    res = oracle.sadmm(A, y, 1.0, lam, oracle.Criterion(elim=0), iters=3000, tol=1e-12)
    xG = res.xG
    assert int(np.argmax(np.abs(xG))) == n0
    truth = x.sum(axis=0)[n0]
    assert truth * 0.95 <= xG[n0] <= truth
    assert np.linalg.norm(np.delete(xG, n0)) <= 0.05 * truth


# ------------------------------------------------------------- Algorithm 1
def _elim_scene():
    """A scene on which the gate opens near iteration 187 (rho = 1) and
    Algorithm 1 then removes most pixels."""
    sc, lam = _resolved(seed=2)
    return sc, lam


def test_eps_p_zero_is_plain_sadmm():
    """zeta >= 0 always, so eps_p = 0 keeps every pixel: identical to SADMM."""
    sc, lam = _elim_scene()
    a = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=60)
    b = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=1, eps_p=0.0), iters=60)
    assert np.array_equal(a.state.x, b.state.x)
    assert np.array_equal(a.state.s, b.state.s)
    assert all(len(j) == sc.geom.N for j in b.state.J)


def _trajectory(sc, lam, crit, iters):
    st = None
    xs, Js, recs = [], [], []
    for _ in range(iters):
        r = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=1, state=st)
        st = r.state
        xs.append(st.x.copy())
        Js.append([j.copy() for j in st.J])
        recs.append(r.history[-1])
    return xs, Js, recs, st


@pytest.mark.parametrize("ssc_every", [1, 3])
def test_ssc_window_and_monotone_sets(ssc_every):
    """Recompute Algorithm 1 from the stored trajectory: at every gated
    iteration J_q = {i in previous J_q : mean_{last Kp} |x^{t+1} - x^t| >= eps_p}.
    Active sets only shrink, and frozen entries are bit-constant afterwards.
    With the batched removal policy the test runs only when ssc_every divides k."""
    sc, lam = _elim_scene()
    crit = oracle.Criterion(elim=1, eps_p=1e-5, Kp=4, ssc_every=ssc_every)
    x0 = np.zeros((sc.geom.Q, sc.geom.N))
    xs, Js, recs, _ = _trajectory(sc, lam, crit, 200)
    traj = [x0] + xs
    prevJ = [np.arange(sc.geom.N)] * sc.geom.Q
    removed_any = False
    frozen_at = {}
    for t, (J, rec) in enumerate(zip(Js, recs)):
        k = t + 1
        if k % ssc_every:
            assert not rec["gate"]
        for q in range(sc.geom.Q):
            assert set(J[q]) <= set(prevJ[q])
            if rec["gate"]:
                zeta = np.mean([np.abs(traj[u + 1][q] - traj[u][q]) for u in range(k - crit.Kp, k)],
                               axis=0)
                expect = prevJ[q][zeta[prevJ[q]] >= crit.eps_p]
                assert np.array_equal(J[q], expect)
            else:
                assert np.array_equal(J[q], prevJ[q])
            for i in set(prevJ[q]) - set(J[q]):
                frozen_at[(q, i)] = (t, xs[t][q, i])
                removed_any = True
        prevJ = J
    assert removed_any
    for (q, i), (t, val) in frozen_at.items():
        for u in range(t, len(xs)):
            assert xs[u][q, i] == val


def test_frozen_fold_is_the_restricted_problem():
    """After elimination, y'_q = y_q - A_q,E x_q,E, and the next x-update equals the
    minimiser of mu/2||y_q - A_q x||^2 + rho/2||x_J - v_J||^2 over x_J with the
    frozen x_E held fixed (solved here by least squares on the stacked system)."""
    sc, lam = _elim_scene()
    crit = oracle.Criterion(elim=1, eps_p=1e-5, Kp=4)
    r = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=190)
    st = r.state
    q = int(np.argmin([len(j) for j in st.J]))
    J = st.J[q]
    E = np.setdiff1d(np.arange(sc.geom.N), J)
    assert len(E) > 0
    B = oracle.real_form(sc.A[q])
    yq = oracle.real_vec(sc.y[q])
    assert np.allclose(st.yprime[q], yq - B[:, E] @ st.x[q, E], rtol=0, atol=1e-12 * np.linalg.norm(yq))
    nxt = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=1, state=st).state
    v = st.x[q, J] - st.xbar[J] + st.zbar[J] - st.s[J]
    M = np.vstack([np.sqrt(crit.mu) * B[:, J], np.sqrt(1.0) * np.eye(len(J))])
    rhs = np.concatenate([np.sqrt(crit.mu) * (yq - B[:, E] @ st.x[q, E]), np.sqrt(1.0) * v])
    xJ = np.linalg.lstsq(M, rhs, rcond=None)[0]
    assert np.allclose(nxt.x[q, J], xJ, rtol=1e-9, atol=1e-10)


def test_residuals_follow_the_stacked_definitions():
    """Residuals of Boyd Sec. 3.3.1 for the sharing problem written with copies
    z_q (x_q - z_q = 0, z_q = x_q - x_bar + z_bar): recompute r_pri, eps_pri, d and
    eps_dual from two consecutive states through the stacked vectors."""
    sc, lam = _elim_scene()
    crit = oracle.Criterion(elim=0)
    rho = 1.0
    a = oracle.sadmm(sc.A, sc.y, rho, lam, crit, iters=12).state
    r = oracle.sadmm(sc.A, sc.y, rho, lam, crit, iters=1, state=a)
    b, rec = r.state, r.history[-1]
    Q, N = b.x.shape
    Za = np.stack([a.x[q] - a.xbar + a.zbar for q in range(Q)]).ravel()
    Zb = np.stack([b.x[q] - b.xbar + b.zbar for q in range(Q)]).ravel()
    Xb = b.x.ravel()
    assert np.isclose(rec["r_pri"], np.linalg.norm(Xb - Zb), rtol=1e-12)
    assert np.isclose(rec["eps_pri"], np.sqrt(Xb.size) * crit.eps_abs
                      + crit.eps_rel * max(np.linalg.norm(Xb), np.linalg.norm(Zb)), rtol=1e-12)
    assert np.isclose(rec["d"], rho * np.linalg.norm(Zb - Za), rtol=1e-12)
    U = np.tile(rho * b.s, Q)
    assert np.isclose(rec["eps_dual"], np.sqrt(Xb.size) * crit.eps_abs
                      + crit.eps_rel * np.linalg.norm(U), rtol=1e-12)
    assert np.isclose(rec["relchange"], np.linalg.norm(b.x - a.x) / np.linalg.norm(b.x), rtol=1e-12)


def test_resume_is_bit_exact():
    """Running k1 then k2 iterations from the saved state equals k1 + k2 at once."""
    sc, lam = _elim_scene()
    crit = oracle.Criterion(elim=1, eps_p=1e-5, Kp=4)
    full = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=200)
    half = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=183)
    rest = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=17, state=half.state)
    assert np.array_equal(full.state.x, rest.state.x)
    assert [list(j) for j in full.state.J] == [list(j) for j in rest.state.J]


def test_degenerate_sharing_certificate():
    """When the per-sensor null spaces together span R^N (here: the 32x32 grid
    seen by four 4-antenna sensors, 2KM = 512 < N = 1024), Eq. 2 is minimised with
    x_G = 0: build a point with sum_q x_q = 0 that fits every sensor's data, and
    check that its objective is far below that of the ground truth and below the
    oracle's iterates."""
    sc = scenegen.build_scene("small_point", seed=0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    B = [oracle.real_form(a) for a in sc.A]
    ys = [oracle.real_vec(v) for v in sc.y]
    X0, nulls = [], []
    for b, v in zip(B, ys):
        U, S, Vt = np.linalg.svd(b)
        r = int(np.sum(S > 1e-9 * S[0]))
        X0.append(Vt[:r].T @ ((U[:, :r].T @ v) / S[:r]))
        nulls.append(Vt[r:].T)
    Nall = np.hstack(nulls)
    c = np.linalg.lstsq(Nall, -np.sum(X0, axis=0), rcond=None)[0]
    X, o = [], 0
    for x0, nb in zip(X0, nulls):
        X.append(x0 + nb @ c[o:o + nb.shape[1]])
        o += nb.shape[1]
    X = np.array(X)
    assert np.max(np.abs(X.sum(axis=0))) <= 1e-8 * np.max(np.abs(X))
    f_cert = oracle.objective(sc.A, sc.y, X, lam, B=B)
    f_true = oracle.objective(sc.A, sc.y, sc.x_true, lam, B=B)
    assert f_cert <= 1e-6 * f_true
    it = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=50, B=B)
    assert np.all(it.xG == 0.0)
    assert oracle.objective(sc.A, sc.y, it.state.x, lam, B=B) >= f_cert


# ------------------------------------------------------------ planted mistakes
MUTANTS = {
    "dual_sign": ("s_new = st.s + xbar_new - zbar_new", "s_new = st.s - xbar_new + zbar_new"),
    "threshold_lambda": ("soft(xbar_new + st.s, lam / rho)", "soft(xbar_new + st.s, lam)"),
    "paper_literal_x_update": ("v = st.x[q, J] - st.xbar[J] + st.zbar[J] - st.s[J]",
                               "v = - st.xbar[J] * len(A) + st.zbar[J] - st.s[J]"),
    "drop_rho_in_rhs": ("solvers[q].solve(cvec[q] + rho * v)", "solvers[q].solve(cvec[q] + v)"),
    "mean_without_frozen": ("xbar_new = st.x.mean(axis=0)", "xbar_new = st.x.sum(axis=0)"),
}


def _mutant(name):
    old, new = MUTANTS[name]
    src = inspect.getsource(osadmm)
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_mutant_" + name)
    mod.__package__ = "oracle"               # its relative imports resolve in the oracle package
    sys.modules[mod.__name__] = mod          # dataclasses look their module up here
    try:
        exec(compile(src.replace(old, new), osadmm.__file__, "exec"), mod.__dict__)
    finally:
        sys.modules.pop(mod.__name__, None)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name):
    sc = scenegen.random_problem(2, 24, 32, seed=21)
    lam = 0.1 * scenegen.lambda_max(sc.A, sc.y)
    rho = 2.0
    m = _mutant(name)
    with np.errstate(all="ignore"):
        try:
            res = m.sadmm(sc.A, sc.y, rho, lam, m.Criterion(elim=0), iters=3000, tol=1e-15)
        except Exception:
            return                     # blowing up is also caught
        x, s = res.state.x, res.state.s
        if not np.all(np.isfinite(x)):
            return
        k = oracle.kkt(sc.A, sc.y, x, s, rho, lam, xG=res.xG)
        Xf, fval = oracle.fista(sc.A, sc.y, lam, iters=3000, tol=1e-13)
        fa = oracle.objective(sc.A, sc.y, x, lam)
    caught = (max(k.values()) > 1e-6) or abs(fa - fval) > 1e-8 * abs(fval)
    assert caught, name


def test_batch_geometries_draw_distinct_combinations():
    """The mixed-geometry batched workload draws distinct (Q, M, K, N)
    combinations from the 48 of its grid, the same ones for the same seed."""
    gs = scenegen.batch_geometries(3, 32)
    keys = {(g.Q, g.M, g.K, g.N) for g in gs}
    assert len(keys) == 32
    assert all(g.Q in (2, 4, 6, 8) and g.M in (4, 8) and g.K in (128, 256) and g.N in (48 ** 2, 64 ** 2, 96 ** 2)
               for g in gs)
    assert [(g.Q, g.M, g.K, g.N) for g in scenegen.batch_geometries(3, 32)] == [(g.Q, g.M, g.K, g.N) for g in gs]
    assert len({(g.Q, g.M, g.K, g.N) for g in scenegen.batch_geometries(0, 48)}) == 48
    with pytest.raises(ValueError):
        scenegen.batch_geometries(0, 49)


def test_signal_model_operator_pins():
    """The oracle's signal-model operator (Section II, Eq. 1, entries from the
    round-trip delays) against the scene generator's complex64 operator, an
    independent implementation: equal within the FP32 rounding of the
    generator; unit modulus; a geometric progression in k for every (m, n)
    with ratio exp(j 2 pi tau df); the k = 0 phase is 2 pi tau f0 (mod 2 pi)."""
    g = scenegen.Geometry(Q=3, M=4, K=32, nx=12, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    for q in (0, 2):
        tau = radar.delays(g, q)
        A = oracle.operator_from_delays(tau, g.fc, g.bw / g.K, g.K)
        A32 = radar.operator(g, q)
        assert A.shape == A32.shape == (g.N, g.KM)
        assert np.max(np.abs(A - A32.astype(np.complex128))) <= 2.0 ** -23
        assert np.allclose(np.abs(A), 1.0, atol=1e-12)
        Ar = A.reshape(g.N, g.M, g.K)
        ratio = Ar[:, :, 1:] / Ar[:, :, :-1]
        want = np.exp(2j * np.pi * tau.T * (g.bw / g.K))
        assert np.max(np.abs(ratio - want[:, :, None])) <= 1e-9
        ph0 = np.angle(Ar[:, :, 0])
        cyc = (tau.T * g.fc) % 1.0
        assert np.max(np.abs(np.angle(np.exp(1j * (ph0 - 2 * np.pi * cyc))))) <= 1e-7


def test_backprojection_pins():
    """Composite BP image (Section IV, Fig. 1 reading): at a lone noiseless
    target of per-sensor magnitudes x_q at pixel n0 it equals sum_q KM x_q
    there (unit-modulus entries) and nowhere exceeds it (Cauchy-Schwarz: the
    matched filter peaks on its own column); it is the magnitude of the
    complex adjoint, i.e. of Re(A^H y) and Re(A^H (-i y)) together; the dB
    display is 0 at the peak and clipped at -30."""
    g = scenegen.Geometry(Q=3, M=4, K=32, nx=12, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    A = [oracle.operator_from_delays(radar.delays(g, q), g.fc, g.bw / g.K, g.K) for q in range(g.Q)]
    n0 = 77
    xq = np.array([0.3, 0.9, 0.6])
    y = [xq[q] * A[q][n0] for q in range(g.Q)]
    bp = oracle.backprojection(A, y)
    assert bp[n0] == pytest.approx(g.KM * xq.sum(), rel=1e-12)
    assert np.all(bp <= bp[n0] * (1 + 1e-12))
    assert int(np.argmax(bp)) == n0
    s = scenegen.Stream(5, 9)
    yr = [(s.normal(g.KM) + 1j * s.normal(g.KM)) for _ in range(g.Q)]
    two = sum(np.hypot(oracle.adjoint_re(A[q], yr[q]), oracle.adjoint_re(A[q], -1j * yr[q])) for q in range(g.Q))
    assert np.allclose(oracle.backprojection(A, yr), two, rtol=1e-12)
    d = oracle.db_image(bp)
    assert d[n0] == 0.0 and d.min() >= -30.0


def test_golden_limit_is_optimal():
    """The stored limit x_G* (tests/golden/resolved_32_limit.json, written by
    tests/golden/make_limits.py from the oracle) certified from x_G* alone,
    independently of the iteration that produced it: on this well-posed
    workload every B_q^T B_q is invertible, so the stationarity conditions of
    Eq. 2 give x_q = H_q (mu B_q^T y_q - nu) with H_q = (mu B_q^T B_q)^{-1}, and
    sum_q x_q = x_G* fixes nu = (sum_q H_q)^{-1} (sum_q H_q mu B_q^T y_q - x_G*);
    x_G* is optimal iff that nu is a subgradient of lambda ||.||_1 at x_G*."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "resolved_32_limit.json")) as f:
        d = json.load(f)
    sc = scenegen.build_scene(d["scene"], seed=d["seed"])
    lam, mu = d["lam"], d["mu"]
    assert lam == pytest.approx(d["lam_frac"] * scenegen.lambda_max(sc.A, sc.y), rel=1e-12)
    xg = np.array(d["xG"])
    B = [oracle.real_form(a) for a in sc.A]
    Hs = [np.linalg.inv(mu * (Bq.T @ Bq)) for Bq in B]
    rhs = sum(H @ (mu * (Bq.T @ oracle.real_vec(yq))) for H, Bq, yq in zip(Hs, B, sc.y)) - xg
    nu = np.linalg.solve(sum(Hs), rhs)
    supp = xg != 0
    assert supp.any() and not supp.all()
    assert np.max(np.abs(nu)) <= lam * (1 + 1e-6)
    assert np.max(np.abs(nu[supp] - lam * np.sign(xg[supp]))) <= 1e-6 * lam


def test_asadmm_limit_deviation_from_the_minimiser():
    """What the ASADMM limit is (parity of elimination runs is otherwise
    unpinned: the paper prints no worked example).  On the well-posed 32x32
    workload (the certified minimiser of test_golden_limit_is_optimal) with
    the paper's eps_p = 1e-5, Algorithm 1 freezes every (sensor, pixel) pair
    within 3000 iterations; frozen coordinates keep the stationarity
    violations they had when frozen (up to about lambda), so the limit is
    not a KKT point of Eq. 2, but its image x_G stays within 1e-3 of the
    minimiser (4.0e-4 measured; with eps_p = 1e-4 it is 6.4e-3)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "resolved_32_limit.json")) as f:
        d = json.load(f)
    sc = scenegen.build_scene(d["scene"], seed=d["seed"])
    B = [oracle.real_form(a) for a in sc.A]
    r = oracle.sadmm(sc.A, sc.y, d["rho"], d["lam"], oracle.Criterion(elim=1), iters=3000, B=B)
    xs = np.array(d["xG"])
    rel = np.linalg.norm(r.xG - xs) / np.linalg.norm(xs)
    k = oracle.kkt(sc.A, sc.y, r.state.x, r.state.s, d["rho"], d["lam"], xG=r.xG, B=B)
    print(f"ASADMM limit: |xG - xG*|/|xG*| = {rel:.2e}, stationarity {k['stationarity']:.2f} lambda, "
          f"active pairs {sum(len(j) for j in r.state.J)}")
    assert sum(len(j) for j in r.state.J) == 0
    assert k["stationarity"] > 0.1                   # not a KKT point of Eq. 2
    assert rel <= 1e-3


def test_batch_scenes_follow_their_recipe():
    """The mixed-geometry batch scenes: 16 scenes per geometry drawn by seed
    (the same draws for the same seed), complex64 measurements of shape
    (S, Q, KM), and per-scene lambda = 0.05 lambda_max of that scene."""
    g = scenegen.Geometry(Q=2, M=4, K=16, nx=8, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    A = [radar.operator(g, q) for q in range(g.Q)]
    Y, lams = scenegen.batch_scenes(g, A, seed=4)
    Y2, lams2 = scenegen.batch_scenes(g, A, seed=4)
    assert Y.shape == (16, g.Q, g.KM) and Y.dtype == np.complex64
    assert np.array_equal(Y, Y2) and lams == lams2
    for s in (0, 7, 15):
        ys = [Y[s, q] for q in range(g.Q)]
        assert lams[s] == pytest.approx(0.05 * scenegen.lambda_max(A, ys), rel=1e-6)
    Y3, _ = scenegen.batch_scenes(g, A, seed=5)
    assert not np.array_equal(Y, Y3)


# planted mistakes in the signal-model oracle: every one must fail its pins
SM_MUTANTS = {
    "row_index_swapped": ("A[:, m * K + k] =", "A[:, k * M + m] ="),
    "phase_sign": ("np.exp(2j * np.pi * tau[m] * (f0 + k * df))", "np.exp(-2j * np.pi * tau[m] * (f0 + k * df))"),
    "start_frequency_dropped": ("tau[m] * (f0 + k * df)", "tau[m] * (k * df)"),
    "bp_coherent_sum": ("out += np.abs(np.asarray(Aq).astype(np.complex128).conj() @ np.asarray(yq).astype(np.complex128))",
                        "out = out + (np.asarray(Aq).astype(np.complex128).conj() @ np.asarray(yq).astype(np.complex128)).real"),
}


def _sm_module(name=None):
    import oracle.signal_model as osm
    src = inspect.getsource(osm)
    if name is not None:
        old, new = SM_MUTANTS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_sm_" + (name or "original"))
    exec(compile(src, osm.__file__, "exec"), mod.__dict__)
    return mod


def _sm_pins_hold(m):
    g = scenegen.Geometry(Q=2, M=3, K=16, nx=8, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    ok = True
    A = []
    for q in range(g.Q):
        tau = radar.delays(g, q)
        Aq = m.operator_from_delays(tau, g.fc, g.bw / g.K, g.K)
        A.append(Aq)
        ok &= Aq.shape == (g.N, g.KM)
        ok &= bool(np.max(np.abs(Aq - radar.operator(g, q).astype(np.complex128))) <= 2.0 ** -23)
    n0, xq = 21, np.array([0.4, 0.7])
    y = [xq[q] * A[q][n0] for q in range(g.Q)]
    bp = m.backprojection(A, y)
    ok &= bool(abs(bp[n0] - g.KM * xq.sum()) <= 1e-9 * g.KM)
    ok &= int(np.argmax(bp)) == n0
    st = scenegen.Stream(6, 1)
    yr = [st.normal(g.KM) + 1j * st.normal(g.KM) for _ in range(g.Q)]
    two = sum(np.hypot(oracle.adjoint_re(A[q], yr[q]), oracle.adjoint_re(A[q], -1j * yr[q])) for q in range(g.Q))
    ok &= bool(np.allclose(m.backprojection(A, yr), two, rtol=1e-12))
    return bool(ok)


def test_signal_model_pins_hold_for_the_oracle():
    assert _sm_pins_hold(_sm_module())


@pytest.mark.parametrize("name", sorted(SM_MUTANTS))
def test_signal_model_pins_catch_planted_mistakes(name):
    with np.errstate(all="ignore"):
        assert not _sm_pins_hold(_sm_module(name)), name


@pytest.mark.parametrize("kind", [1, 2])
def test_pair_operator_is_two_nearest_roundings(kind):
    """oracle.precision: hi = RN(a) and lo = RN(a - hi) per real component,
    checked against torch's round-to-nearest-even conversions (independent
    code), the bounds |a - hi| <= u |a| and |a - P| <= u^2 |a| (BF16 u = 2^-8,
    FP16 u = 2^-11, plus FP16's subnormal half-spacing 2^-25), and exactness
    of P = hi + lo in complex64."""
    torch = pytest.importorskip("torch")
    g = scenegen.Geometry(Q=1, M=4, K=32, nx=8, cell=0.05, radius=10.0, fc=77e9, bw=1e9)
    A = radar.operator(g, 0)
    A[0, :4] = [1.0 + 0j, 2.0 ** -20 + 0.5j, -3.0e-9 + 0j, 1.0 + 2.0 ** -9 * 1j]   # edge values
    h, l = oracle.precision.split_planes(A, kind)
    dt = torch.bfloat16 if kind == 1 else torch.float16
    for part, hp, lp in ((A.real, h.real, l.real), (A.imag, h.imag, l.imag)):
        t = torch.from_numpy(np.ascontiguousarray(part, dtype=np.float32))
        th = t.to(dt)
        assert np.array_equal(hp, th.to(torch.float64).numpy())
        tl = (t - th.to(torch.float32)).to(dt)
        assert np.array_equal(lp, tl.to(torch.float64).numpy())
    u = 2.0 ** -8 if kind == 1 else 2.0 ** -11
    sub = 0.0 if kind == 1 else 2.0 ** -25
    P = oracle.precision.pair_operator(A, kind).astype(np.complex128)
    a = A.astype(np.complex128)
    for f in (np.real, np.imag):
        assert np.all(np.abs(f(a) - f(h)) <= u * np.abs(f(a)) + sub)
        assert np.all(np.abs(f(a) - f(P)) <= u * u * np.abs(f(a)) + sub)
    assert np.array_equal(P, h + l)


def _kkt_stationarity_chunked(Aq, yq, xq, nu, mu, chunk=2048):
    """max_i |mu Re(a_i^H (A_q x_q - y_q)) + nu_i| with the FP64 products of
    oracle.forward / oracle.adjoint_re taken over pixel chunks (the operator is
    never held in complex128 as a whole)."""
    N = Aq.shape[0]
    r = -np.asarray(yq).astype(np.complex128)
    for n0 in range(0, N, chunk):
        r += oracle.forward(Aq[n0:n0 + chunk], xq[n0:n0 + chunk])
    g = np.concatenate([oracle.adjoint_re(Aq[n0:n0 + chunk], r) for n0 in range(0, N, chunk)])
    return float(np.max(np.abs(mu * g + nu)))


def test_golden_limit_128_is_optimal():
    """The stored limit of the well-posed paper-size workload
    (tests/golden/resolved_128_limit.npz, written by tests/golden/make_limits.py
    from the oracle) certified by the KKT conditions of Eq. 2 alone: for the
    stored per-sensor images X* and dual nu = rho s*, stationarity
    mu Re(A_q^H (A_q x_q - y_q)) + nu = 0 for every sensor, nu a subgradient of
    lambda ||.||_1 at x_G* (|nu| <= lambda, nu = lambda sign(x_G*) on its
    support) and x_G* = sum_q x_q.  The scene and lambda are regenerated from
    the scene generator and must match the stored measurements."""
    import json
    import os
    from concurrent.futures import ThreadPoolExecutor
    here = os.path.join(os.path.dirname(__file__), "golden")
    with open(os.path.join(here, "resolved_128_limit.json")) as f:
        meta = json.load(f)
    d = np.load(os.path.join(here, "resolved_128_limit.npz"))
    sc = scenegen.build_scene(meta["scene"], seed=meta["seed"])
    assert np.array_equal(np.stack(sc.y).astype(np.complex64), d["y"])
    lam, mu, rho = meta["lam"], meta["mu"], meta["rho"]
    assert lam == pytest.approx(meta["lam_frac"] * scenegen.lambda_max(sc.A, sc.y), rel=1e-12)
    X, s, xg = d["X"], d["s"], d["xG"]
    nu = rho * s
    with ThreadPoolExecutor(max_workers=4) as pool:
        stat = list(pool.map(lambda q: _kkt_stationarity_chunked(sc.A[q], sc.y[q], X[q], nu, mu),
                             range(sc.geom.Q)))
    supp = xg != 0
    assert 0 < supp.sum() < len(xg)
    assert max(stat) <= 1e-6 * lam
    assert np.max(np.abs(nu)) <= lam * (1 + 1e-6)
    assert np.max(np.abs(nu[supp] - lam * np.sign(xg[supp]))) <= 1e-6 * lam
    assert np.max(np.abs(xg - X.sum(axis=0))) <= 1e-6 * max(1.0, np.max(np.abs(xg)))


# ------------------------------------------------- consensus form (ACADMM)
@pytest.mark.parametrize("seed,rho", [(31, 2.0), (32, 0.5)])
def test_consensus_limit_satisfies_kkt_and_matches_fista(seed, rho):
    """Consensus ADMM (Criterion.consensus, Boyd Sec. 7.1 read for the CADMM
    form of Section I), elimination off: at the limit the KKT conditions of
    min sum_q mu/2 ||y_q - A_q z||^2 + lambda ||z||_1 hold to 1e-8 and z
    agrees with an independent FISTA on the stacked LASSO (objective to 1e-10,
    iterate to 1e-6)."""
    sc = scenegen.random_problem(3, 24, 20, seed=seed)
    lam = 0.2 * scenegen.lambda_max(sc.A, sc.y)
    r = oracle.sadmm(sc.A, sc.y, rho, lam, oracle.Criterion(elim=0, consensus=True), iters=20000, tol=1e-15)
    k = oracle.kkt_consensus(sc.A, sc.y, r.state.x, r.state.u, r.xG, rho, lam)
    assert max(k.values()) <= 1e-8, k
    z, fz = oracle.fista_consensus(sc.A, sc.y, lam, iters=30000, tol=1e-14)
    Bs = [oracle.real_form(a) for a in sc.A]
    fa = sum(0.5 * np.sum((oracle.real_vec(v) - Bq @ r.xG) ** 2) for Bq, v in zip(Bs, sc.y)) + lam * np.sum(
        np.abs(r.xG))
    assert abs(fa - fz) <= 1e-10 * abs(fz)
    assert np.linalg.norm(r.xG - z) <= 1e-6 * np.linalg.norm(z)
    assert np.count_nonzero(r.xG) < len(r.xG)


def test_consensus_limit_matches_a_library_lasso():
    """The consensus problem is a LASSO in z with the real forms stacked:
    scikit-learn's coordinate-descent Lasso (its objective
    1/(2n) ||b - B z||^2 + alpha ||z||_1 with alpha = lambda / (mu n)) gives
    the same minimiser."""
    lm = pytest.importorskip("sklearn.linear_model")
    sc = scenegen.random_problem(2, 24, 16, seed=33)
    lam = 0.2 * scenegen.lambda_max(sc.A, sc.y)
    r = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0, consensus=True), iters=20000, tol=1e-15)
    Bst = np.concatenate([oracle.real_form(a) for a in sc.A], axis=0)
    b = np.concatenate([oracle.real_vec(v) for v in sc.y])
    n = Bst.shape[0]
    las = lm.Lasso(alpha=lam / n, fit_intercept=False, tol=1e-14, max_iter=1000000).fit(Bst, b)
    assert np.linalg.norm(r.xG - las.coef_) <= 1e-6 * np.linalg.norm(las.coef_)


def test_consensus_elimination_invariants():
    """ACADMM (consensus with Algorithm 1): eps_p = 0 reproduces plain CADMM
    bit for bit; with the paper's eps_p the active sets only shrink, frozen
    entries keep their value, and the result stays near the plain limit."""
    sc = scenegen.build_scene("resolved_tiny", seed=1)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    plain = oracle.sadmm(sc.A, sc.y, 2.0, lam, oracle.Criterion(elim=0, consensus=True), iters=300)
    zero = oracle.sadmm(sc.A, sc.y, 2.0, lam, oracle.Criterion(elim=1, eps_p=0.0, consensus=True), iters=300)
    assert np.array_equal(plain.state.x, zero.state.x) and np.array_equal(plain.xG, zero.xG)
    r = oracle.sadmm(sc.A, sc.y, 2.0, lam, oracle.Criterion(elim=1, consensus=True), iters=600,
                     snapshots=set(range(1, 601)))
    prev = [set(range(sc.geom.N))] * sc.geom.Q
    for k in range(1, 601):
        st = r.snapshots[k]
        for q in range(sc.geom.Q):
            cur = set(st.J[q].tolist())
            assert cur <= prev[q]
            frozen = np.setdiff1d(np.arange(sc.geom.N), st.J[q])
            if k > 1 and len(frozen):
                before = r.snapshots[k - 1]
                was = np.setdiff1d(np.arange(sc.geom.N), before.J[q])
                assert np.array_equal(st.x[q, was], before.x[q, was])
        prev = [set(j.tolist()) for j in st.J]
    assert sum(len(j) for j in r.state.J) < sc.geom.Q * sc.geom.N
    lim = oracle.sadmm(sc.A, sc.y, 2.0, lam, oracle.Criterion(elim=0, consensus=True), iters=4000)
    assert np.linalg.norm(r.xG - lim.xG) <= 1e-2 * np.linalg.norm(lim.xG)


CONSENSUS_MUTANTS = {
    "threshold_without_Q": ("soft(xbar_new + st.u.mean(axis=0), lam / (Q * rho))",
                            "soft(xbar_new + st.u.mean(axis=0), lam / rho)"),
    "dual_sign": ("u_new = st.u + st.x - z_new[None, :]", "u_new = st.u - st.x + z_new[None, :]"),
    "v_without_dual": ("v = st.zbar[J] - st.u[q, J]", "v = st.zbar[J]"),
}


@pytest.mark.parametrize("name", sorted(CONSENSUS_MUTANTS))
def test_consensus_pins_catch_planted_mistakes(name):
    old, new = CONSENSUS_MUTANTS[name]
    src = inspect.getsource(osadmm)
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_cmutant_" + name)
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src.replace(old, new), osadmm.__file__, "exec"), mod.__dict__)
    finally:
        sys.modules.pop(mod.__name__, None)
    sc = scenegen.random_problem(3, 24, 20, seed=31)
    lam = 0.2 * scenegen.lambda_max(sc.A, sc.y)
    with np.errstate(all="ignore"):
        try:
            r = mod.sadmm(sc.A, sc.y, 2.0, lam, mod.Criterion(elim=0, consensus=True), iters=5000, tol=1e-15)
        except Exception:
            return
        if not np.all(np.isfinite(r.state.x)):
            return
        k = oracle.kkt_consensus(sc.A, sc.y, r.state.x, r.state.u, r.xG, 2.0, lam)
        z, _ = oracle.fista_consensus(sc.A, sc.y, lam, iters=30000, tol=1e-14)
    caught = max(k.values()) > 1e-6 or np.linalg.norm(r.xG - z) > 1e-4 * np.linalg.norm(z)
    assert caught, name
