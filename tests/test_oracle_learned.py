"""Pins of the oracle's learned elimination step (oracle/learned.py and the
elim = 2 branch of oracle.sadmm), checked against facts fixed independently of
its code: BF16 rounding against torch's round-to-nearest-even conversion, the
update channels against differences of stored iterates, the re-admission step
against the exact minimiser of the one-coordinate problem and against the
optimality of a converged solution, and the learned step's reductions to
Algorithm 1 alone."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle
import oracle.cnn as ocnn
import oracle.learned as ol
import scenegen


def test_round_bf16_matches_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    s = scenegen.Stream(3, 1)
    v = (s.normal(20000) * np.exp(s.normal(20000) * 4)).astype(np.float32)
    # exact ties: mantissas ending in 0x8000 (round half to even, both parities)
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32) * np.float32(1.0)
    v = np.concatenate([v, ties, -ties, np.float32([0.0, -0.0, 1.0, 3.0e38, 1e-40])])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = ol.round_bf16(v)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    assert ol.round_bf16(np.float32([1.0 + 2.0 ** -8]))[0] == 1.0                 # tie to even (down)
    assert ol.round_bf16(np.float32([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie to even (up)


def test_update_channels_are_norms_of_stored_iterate_differences():
    sc = scenegen.build_scene("resolved_tiny", seed=1)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    eps_p = 1e-5
    for Kp in (5, 3):
        crit = oracle.Criterion(elim=0, Kp=Kp, eps_p=eps_p)
        ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=12, snapshots=range(1, 13))
        snap = ref.snapshots
        snap[0] = oracle.initial_state(sc.A, sc.y, Kp)
        for k in (1, 2, 7, 12):
            st = snap[k]
            f = ol.features(st.x, st.ring, k, eps_p)
            assert np.allclose(f[0], np.log1p(np.abs(st.x).sum(axis=0)), rtol=0, atol=1e-15)
            assert np.allclose(f[1], np.log1p(np.abs(st.x).max(axis=0)), rtol=0, atol=1e-15)
            for j in range(4):
                if j < Kp and k - j >= 1:
                    d = np.linalg.norm(snap[k - j].x - snap[k - j - 1].x, axis=0)
                else:
                    d = np.zeros(sc.geom.N)
                assert np.allclose(f[2 + j], np.log10(d / eps_p + 1e-4) / 4, rtol=0, atol=1e-12), (Kp, k, j)


def _problem(seed=5, Q=2, KM=64, N=40):
    sc = scenegen.random_problem(Q, KM, N, seed=seed)
    B = [oracle.real_form(a) for a in sc.A]
    return sc, B


def test_readmission_step_is_the_exact_one_coordinate_minimiser():
    """For pixel i frozen in sensor q, phi(t) = mu/2 ||y_q - B_q (x_q + t e_i)||^2
    + rho s_i t + rho/2 t^2 is the x-update's objective along e_i at the fixed
    point; its minimiser has magnitude equal to the re-admission step.  y' is
    the folded measurement (frozen pixels subtracted), as in the solver."""
    sc, B = _problem()
    s = scenegen.Stream(9, 2)
    mu, rho = 0.7, 1.6
    N = sc.geom.N
    for q in range(2):
        x = s.normal(N)
        sv = s.normal(N) * 0.1
        J = np.sort(s.permutation(N)[:25])
        F_true = np.setdiff1d(np.arange(N), J)
        y = oracle.real_vec(sc.y[q])
        yprime = y - B[q][:, F_true] @ x[F_true]
        F, step = ol.readmission_steps(B[q], yprime, x, J, sv, mu, rho)
        assert np.array_equal(F, F_true)
        for i, st in zip(F, step):
            def phi(t):
                xt = x.copy()
                xt[i] += t
                return 0.5 * mu * np.sum((y - B[q] @ xt) ** 2) + rho * sv[i] * t + 0.5 * rho * t * t
            t = minimize_scalar(phi, bracket=(-1.0, 1.0), tol=1e-12).x
            assert abs(abs(t) - st) <= 1e-6 * max(1.0, st), (q, i)


def test_no_readmission_at_the_optimum():
    """At a converged plain SADMM solution the optimality condition of Eq. 2
    holds for every (sensor, pixel), so every pixel, viewed as frozen at its
    optimal value, has a vanishing re-admission step."""
    sc = scenegen.build_scene("resolved_tiny", seed=1, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=20000, tol=1e-14)
    st = ref.state
    B = [oracle.real_form(a) for a in sc.A]
    empty = np.zeros(0, dtype=np.int64)
    scale = np.max(np.abs(st.x))
    for q in range(sc.geom.Q):
        # every pixel frozen: y' = y - B x
        yprime = oracle.real_vec(sc.y[q]) - B[q] @ st.x[q]
        F, step = ol.readmission_steps(B[q], yprime, st.x[q], empty, st.s, 1.0, 1.0)
        assert len(F) == sc.geom.N
        assert np.max(step) <= 1e-7 * scale
    # ... while a support pixel frozen at zero has a step of its own size
    q = 0
    i = int(np.argmax(np.abs(st.x[q])))
    x = st.x[q].copy()
    x[i] = 0.0
    yprime = oracle.real_vec(sc.y[q]) - B[q] @ x
    F, step = ol.readmission_steps(B[q], yprime, x, empty, st.s, 1.0, 1.0)
    assert step[i] >= 0.1 * abs(st.x[q, i])


def _eliminator(geom, seed=4, head_bias=0.0):
    return oracle.Eliminator(scenegen.cnn_init(seed, head_bias=head_bias), geom.ny or geom.nx, geom.nx)


def test_unreachable_threshold_reduces_to_algorithm_1():
    """learn_theta = 1 (p > 1 never holds) and an infinite re-admission
    threshold: the learned steps run but change nothing, so elim = 2 is elim = 1."""
    sc = scenegen.build_scene("resolved_tiny", seed=2, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    c1 = oracle.Criterion(elim=1, Kp=4)
    c2 = oracle.Criterion(elim=2, Kp=4, learn_every=5, learn_theta=1.0, readmit=np.inf)
    r1 = oracle.sadmm(sc.A, sc.y, 1.0, lam, c1, iters=200)
    r2 = oracle.sadmm(sc.A, sc.y, 1.0, lam, c2, iters=200, eliminator=_eliminator(sc.geom))
    assert sum(h["learned"] for h in r2.history) == 40
    assert np.array_equal(r1.state.x, r2.state.x)
    assert all(np.array_equal(a, b) for a, b in zip(r1.state.J, r2.state.J))
    assert sum(len(j) for j in r1.state.J) < sc.geom.Q * sc.geom.N     # Algorithm 1 did act


@pytest.mark.parametrize("freeze_mode", [0, 1])
def test_proposal_of_every_pixel_freezes_everything(freeze_mode):
    """A network whose output is ~1 everywhere drops every pixel at the first
    learned step (k = 10, gate closed): all sets empty, y' = y - B_q x_q
    (freeze mode 0) or x = 0 (zero mode), and the iterates stop moving."""
    sc = scenegen.build_scene("resolved_tiny", seed=2, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    crit = oracle.Criterion(elim=2, Kp=4, learn_every=10, readmit=np.inf, freeze_mode=freeze_mode)
    el = _eliminator(sc.geom, head_bias=60.0)
    r = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=15, eliminator=el, snapshots=(9, 10, 15))
    assert not r.history[9]["gate"] and r.history[9]["learned"]
    s10, s15 = r.snapshots[10], r.snapshots[15]
    assert all(len(j) == 0 for j in s10.J)
    B = [oracle.real_form(a) for a in sc.A]
    for q in range(sc.geom.Q):
        if freeze_mode == 0:
            assert np.allclose(s10.yprime[q], oracle.real_vec(sc.y[q]) - B[q] @ s10.x[q], rtol=0, atol=1e-12)
        else:
            assert np.all(s10.x[q] == 0.0)
    assert np.array_equal(s10.x, s15.x)
    assert np.all(s10.ring == 0.0)


def test_readmission_restores_wrongly_frozen_pixels():
    """Start from the converged plain solution with sensor 0's largest pixels
    frozen at zero (folded, freeze mode 0).  Without proposals (learn_theta = 1)
    and with Algorithm 1's gate closed, the first learned step re-admits exactly
    those pixels and the run returns to the optimum."""
    sc = scenegen.build_scene("resolved_tiny", seed=1, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    ref = oracle.sadmm(sc.A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=20000, tol=1e-14)
    st = ref.state.copy()
    B = [oracle.real_form(a) for a in sc.A]
    q = 0
    wrong = np.sort(np.argsort(-np.abs(st.x[q]))[:3])
    st.x[q, wrong] = 0.0
    st.J[q] = np.setdiff1d(np.arange(sc.geom.N), wrong)
    st.yprime[q] = oracle.real_vec(sc.y[q]) - B[q][:, wrong] @ st.x[q, wrong]
    st.k = 40
    # eps_abs = eps_rel = 0 keeps Algorithm 1's gate closed (r_pri > 0)
    crit = oracle.Criterion(elim=2, Kp=4, learn_every=10, learn_theta=1.0, eps_abs=0.0, eps_rel=0.0)
    r = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=3000, state=st, eliminator=_eliminator(sc.geom))
    first = [h for h in r.history if h["learned"]][0]
    assert first["readmitted"] == len(wrong)
    assert np.array_equal(r.state.J[q], np.arange(sc.geom.N))
    assert np.linalg.norm(r.xG - ref.xG) <= 1e-5 * np.linalg.norm(ref.xG)


def test_eliminator_network_uses_rounded_parameters():
    """The oracle evaluates the network with BF16-rounded parameters: a
    network built from already-rounded parameters gives the same run."""
    sc = scenegen.build_scene("resolved_tiny", seed=2, snr_db=30.0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    el = _eliminator(sc.geom, seed=8, head_bias=-1.0)
    el2 = oracle.Eliminator(ol.round_bf16(el.params).astype(np.float32), el.H, el.W)
    crit = oracle.Criterion(elim=2, Kp=4, learn_every=5, learn_theta=0.4)
    r1 = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=30, eliminator=el)
    r2 = oracle.sadmm(sc.A, sc.y, 1.0, lam, crit, iters=30, eliminator=el2)
    assert np.array_equal(r1.state.x, r2.state.x)
    assert ocnn.num_params() == el.params.size


def test_readmission_brings_the_limit_near_a_kkt_point():
    """The learned mode's limit with a network that never proposes (learn_theta
    = 1): Algorithm 1 plus re-admission.  On the well-posed 32x32 workload
    (certified minimiser in tests/golden/resolved_32_limit.json), re-admission
    returns the pairs whose one-coordinate step is still large, so after 3000
    iterations the limit is close to a KKT point of Eq. 2 (stationarity
    violation 0.0033 lambda measured, against 0.98 lambda for Algorithm 1
    alone: test_asadmm_limit_deviation_from_the_minimiser), its image is
    within 5e-4 of the minimiser (1.6e-4 measured) with the same support."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "resolved_32_limit.json")) as f:
        d = json.load(f)
    sc = scenegen.build_scene(d["scene"], seed=d["seed"])
    B = [oracle.real_form(a) for a in sc.A]
    crit = oracle.Criterion(elim=2, learn_theta=1.0, learn_every=10)
    r = oracle.sadmm(sc.A, sc.y, d["rho"], d["lam"], crit, iters=3000, B=B, eliminator=_eliminator(sc.geom))
    xs = np.array(d["xG"])
    k = oracle.kkt(sc.A, sc.y, r.state.x, r.state.s, d["rho"], d["lam"], xG=r.xG, B=B)
    rel = np.linalg.norm(r.xG - xs) / np.linalg.norm(xs)
    print(f"learned mode (no proposals) limit: |xG - xG*|/|xG*| = {rel:.2e}, "
          f"stationarity {k['stationarity']:.4f} lambda")
    assert sum(h.get("readmitted", 0) or 0 for h in r.history) > 0
    assert k["stationarity"] <= 0.02
    assert rel <= 5e-4
    assert np.array_equal(r.xG != 0, xs != 0)
