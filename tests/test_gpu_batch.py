"""Batched form: 16 scenes sharing one geometry iterate together (GEMMs with
16 right-hand sides).  Each scene must match the FP64 oracle run on that
scene alone at equal iteration count (stacked iterate within 1e-4, the bar of
the single-scene path), and therefore the single-scene CUDA solver within
2e-4 (both sit within 1e-4 of the same oracle iterate; their FP32 sums run in
different orders)."""
import numpy as np
import pytest

import oracle
import scenegen
from scenegen import radar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_08606_gb300 import build, binding
    build()
    binding.load()
    return binding


def _scenes(name, S=16):
    g = scenegen.GEOMS[name]
    A = [radar.operator(g, q) for q in range(g.Q)]
    ys, lams, xs = [], [], []
    for s in range(S):
        x = radar.point_targets(g, 100 + s, 3 + s % 5, p_vis=0.8)
        y = radar.measure(A, x, 25.0, 100 + s)
        ys.append(y)
        xs.append(x)
        lams.append(0.05 * scenegen.lambda_max(A, y))
    return g, A, ys, lams


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


@pytest.mark.parametrize("name,iters", [("small_point", 60), ("resolved_tiny", 150)])
def test_batch_matches_oracle_and_single_solver(B, name, iters):
    g, A, ys, lams = _scenes(name)
    bs = B.BatchSolver(g.Q, g.M, g.K, g.N, 1.0, lams)
    for q in range(g.Q):
        bs.set_operator(q, A[q])
    Y = np.stack([np.stack(y) for y in ys])              # (S, Q, KM)
    xg, st = bs.solve(Y, iters)
    assert st["iters"] == iters
    for s in range(16):
        Xb = np.stack([bs.xq(s, q) for q in range(g.Q)])
        one = B.Solver(g.Q, g.M, g.K, g.N, 1.0, lams[s], elim=0)
        for q in range(g.Q):
            one.set_operator(q, A[q])
        x1, _ = one.solve(ys[s], iters)
        X1 = one.X()
        one.close()
        assert _rel(Xb, X1) <= 2e-4, s
        if np.any(x1 != 0):
            assert _rel(xg[s], x1) <= 2e-4, s
        ref = oracle.sadmm(A, ys[s], 1.0, lams[s], oracle.Criterion(elim=0), iters=iters)
        assert _rel(Xb, ref.state.x) <= 1e-4, s
        if np.any(ref.xG != 0):
            assert _rel(xg[s], ref.xG) <= 1e-4, s
    bs.close()


def _batch(B, g, A, lams):
    bs = B.BatchSolver(g.Q, g.M, g.K, g.N, 1.0, lams)
    for q in range(g.Q):
        bs.set_operator(q, A[q])
    return bs


def _stack_x(bs, g):
    return np.stack([np.stack([bs.xq(s, q) for q in range(g.Q)]) for s in range(16)])


def test_tuner_picks_fastest_candidate_and_keeps_results(B):
    """sadmm_batch_tune times every candidate split of the two tensor-core
    products and keeps the fastest; the solve after tuning still matches the
    oracle (1e-4) and the untuned solve (2e-4: a different split changes only
    the order of FP32 sums)."""
    g, A, ys, lams = _scenes("small_point")
    Y = np.stack([np.stack(y) for y in ys])
    bs = _batch(B, g, A, lams)
    iters = 60
    xg0, _ = bs.solve(Y, iters)
    X0 = _stack_x(bs, g)
    t = bs.tune(reps=2)
    for part, key in (("forward", "forward_splits"), ("adjoint", "adjoint_splits")):
        times = t[part]
        assert len(times) >= 2 and all(k >= 1 for k in times)
        assert all(v > 0 for v in times.values())
        assert t[key] == min(times, key=times.get)
    xg1, _ = bs.solve(Y, iters)
    X1 = _stack_x(bs, g)
    for s in range(16):
        assert _rel(X1[s], X0[s]) <= 2e-4, s
    ref = oracle.sadmm(A, ys[0], 1.0, lams[0], oracle.Criterion(elim=0), iters=iters)
    assert _rel(X1[0], ref.state.x) <= 1e-4
    bs.close()


def test_group_of_geometries_matches_separate_solves(B):
    """Three geometries of different Q, KM and N (one with the primal factor,
    N < 2KM, two with the Woodbury factor) iterate together as one batch
    group: every scene's iterates equal those of its batch solved alone, bit
    for bit (same kernels, same splits, fixed summation orders), scene 0 of
    each geometry matches the oracle (1e-4), a second group solve resets the
    state, and re-tuning one batch makes the group rebuild its graph."""
    third = scenegen.Geometry(Q=2, M=4, K=32, nx=16, cell=0.1, radius=5.0, fc=77e9, bw=1e9)
    specs = []
    for name in ("small_point", "resolved_tiny", None):
        if name is None:
            g = third
            A = [radar.operator(g, q) for q in range(g.Q)]
            Y, lams = scenegen.batch_scenes(g, A, seed=7)
            ys = [list(Y[s]) for s in range(16)]
        else:
            g, A, ys, lams = _scenes(name)
            Y = np.stack([np.stack(y) for y in ys])
        specs.append((g, A, ys, lams, Y))
    iters = 40
    sep = []
    batches = []
    for g, A, ys, lams, Y in specs:
        bs = _batch(B, g, A, lams)
        xg, _ = bs.solve(Y, iters)
        sep.append((xg.copy(), _stack_x(bs, g)))
        batches.append(bs)
    grp = B.BatchGroup(batches)
    for rep in range(2):
        outs, stats = grp.solve([sp[4] for sp in specs], iters)
        for i, (g, A, ys, lams, Y) in enumerate(specs):
            assert stats[i]["iters"] == iters
            assert np.array_equal(outs[i], sep[i][0]), (rep, i)
            assert np.array_equal(_stack_x(batches[i], g), sep[i][1]), (rep, i)
    for i, (g, A, ys, lams, Y) in enumerate(specs):
        ref = oracle.sadmm(A, ys[0], 1.0, lams[0], oracle.Criterion(elim=0), iters=iters)
        assert _rel(sep[i][1][0], ref.state.x) <= 1e-4, i
    batches[0].tune(reps=1)
    xg_alone, _ = batches[0].solve(specs[0][4], iters)
    outs, _ = grp.solve([sp[4] for sp in specs], iters)
    assert np.array_equal(outs[0], xg_alone)
    assert np.array_equal(outs[1], sep[1][0])
    grp.close()
    for bs in batches:
        bs.close()
