"""Writes the FP64 oracle's limits x_G* of plain SADMM on the well-posed
workloads, the references of the time-to-accuracy measurements (relative
error ||x_G^k - x_G*|| / ||x_G*|| <= 1e-3):

* resolved_32_limit.json: scene resolved_32 (Q=4, N=32x32), seed 20,
  rho = 100, lambda = 0.05 lambda_max, mu = 1; 1000 iterations of
  oracle.sadmm.
* resolved_128_limit.npz (+ .json with the parameters and KKT residuals):
  scene resolved_128 (Q=8, M=256, K=64, N=128x128), seed 0, lambda = 0.05
  lambda_max, mu = 1; oracle.sadmm_primal_inverse (the same iteration through
  explicit inverses) until the relative change of the stacked iterate is
  below 1e-13.  The .npz holds x_G*, the per-sensor limits X* and the scaled
  dual s* (so that the KKT conditions of Eq. 2 can be checked without
  iterating) and the measurements y (complex64) that the benchmark reuses.

* precision_twin_oracle.npz: the precision workload's oracle-sized twin
  (scene precision_twin, seed 0: Q=8, M=16, K=512, N=64x64; rho = 1,
  lambda = 0.05 lambda_max), 20 plain SADMM iterations of oracle.sadmm on the
  complex64 operator A and on its BF16 and FP16 pair operators
  (oracle.precision): the stacked iterates X that the benchmark compares its
  split-precision runs with, and the measurements y.

Calls only the oracle and the scene generator.  The stored limits are checked
independently of the iteration by tests/test_oracle_pins.py
(test_golden_limit_is_optimal, test_golden_limit_128_is_optimal).
Run: python tests/golden/make_limits.py [resolved_32|resolved_128|precision_twin]"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import scenegen    # noqa: E402

R32 = dict(scene="resolved_32", seed=20, rho=100.0, lam_frac=0.05, iters=1000)
R128 = dict(scene="resolved_128", seed=0, rho=1000.0, lam_frac=0.05, iters=3000, tol=1e-13)


def resolved_32():
    p = R32
    sc = scenegen.build_scene(p["scene"], seed=p["seed"])
    lam = p["lam_frac"] * scenegen.lambda_max(sc.A, sc.y)
    B = [oracle.real_form(a) for a in sc.A]
    r = oracle.sadmm(sc.A, sc.y, p["rho"], lam, oracle.Criterion(elim=0), iters=p["iters"], B=B)
    k = oracle.kkt(sc.A, sc.y, r.state.x, r.state.s, p["rho"], lam, xG=r.xG, B=B)
    out = {"scene": p["scene"], "seed": p["seed"], "rho": p["rho"], "lam_frac": p["lam_frac"], "lam": lam,
           "mu": 1.0, "iterations": p["iters"], "kkt": {k_: float(v) for k_, v in k.items()},
           "xG": [float(v) for v in r.xG]}
    with open(os.path.join(HERE, "resolved_32_limit.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(k, float(np.linalg.norm(r.xG)))


def kkt_per_sensor(A, y, X, s, rho, lam, xG, mu=1.0):
    """oracle.kkt's residuals, one sensor's FP64 operator at a time."""
    nu = rho * s
    stat = 0.0
    for q in range(len(A)):
        r = oracle.forward(A[q], X[q]) - np.asarray(y[q]).astype(np.complex128)
        stat = max(stat, float(np.max(np.abs(mu * oracle.adjoint_re(A[q], r) + nu))))
    sub = max(0.0, float(np.max(np.abs(nu))) - lam)
    supp = np.abs(xG) > 0
    sgn = float(np.max(np.abs(nu[supp] - lam * np.sign(xG[supp])))) if supp.any() else 0.0
    feas = float(np.max(np.abs(xG - X.sum(axis=0)))) / max(1.0, float(np.max(np.abs(xG))))
    return dict(stationarity=stat / lam, subgradient=max(sub, sgn) / lam, feasibility=feas)


def resolved_128():
    p = R128
    t0 = time.time()
    sc = scenegen.build_scene(p["scene"], seed=p["seed"])
    lam = p["lam_frac"] * scenegen.lambda_max(sc.A, sc.y)
    print(f"scene {time.time() - t0:.0f} s, lambda {lam:.6g}", flush=True)
    log = []

    def record(k, xg):
        if k % 50 == 0:
            log.append((k, float(np.linalg.norm(xg))))
            print(f"k {k} |x_G| {log[-1][1]:.12g} ({time.time() - t0:.0f} s)", flush=True)

    r = oracle.sadmm_primal_inverse(sc.A, sc.y, p["rho"], lam, iters=p["iters"], tol=p["tol"], record=record)
    xg = r.xG
    k = kkt_per_sensor(sc.A, sc.y, r.state.x, r.state.s, p["rho"], lam, xg)
    print(k, r.state.k, float(np.linalg.norm(xg)), int(np.count_nonzero(xg)), flush=True)
    np.savez_compressed(os.path.join(HERE, "resolved_128_limit.npz"), xG=xg, X=r.state.x, s=r.state.s,
                        y=np.stack(sc.y).astype(np.complex64))
    meta = {"scene": p["scene"], "seed": p["seed"], "rho": p["rho"], "lam_frac": p["lam_frac"], "lam": lam,
            "mu": 1.0, "iterations": r.state.k, "final_relchange": r.history[-1]["relchange"],
            "kkt": {k_: float(v) for k_, v in k.items()}, "support": int(np.count_nonzero(xg)),
            "norm_xG": float(np.linalg.norm(xg))}
    with open(os.path.join(HERE, "resolved_128_limit.json"), "w") as f:
        json.dump(meta, f, indent=1)


def precision_twin(iters=20):
    sc = scenegen.build_scene("precision_twin", seed=0)
    lam = 0.05 * scenegen.lambda_max(sc.A, sc.y)
    out = {"y": np.stack(sc.y).astype(np.complex64), "lam": np.float64(lam), "iters": np.int64(iters)}
    for name, A in (("X_fp32", sc.A), ("X_bf16_pairs", [oracle.precision.pair_operator(a, 1) for a in sc.A]),
                    ("X_fp16_pairs", [oracle.precision.pair_operator(a, 2) for a in sc.A])):
        r = oracle.sadmm(A, sc.y, 1.0, lam, oracle.Criterion(elim=0), iters=iters)
        out[name] = r.state.x
        print(name, float(np.linalg.norm(r.state.x)), flush=True)
    np.savez_compressed(os.path.join(HERE, "precision_twin_oracle.npz"), **out)


if __name__ == "__main__":
    which = sys.argv[1:] or ["resolved_32"]
    for w in which:
        {"resolved_32": resolved_32, "resolved_128": resolved_128, "precision_twin": precision_twin}[w]()
