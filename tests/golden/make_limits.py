"""Writes resolved_32_limit.json: the FP64 oracle's limit x_G* of plain SADMM
on the well-posed 32x32 workload (scene resolved_32, seed 20, rho = 100,
lambda = 0.05 lambda_max, mu = 1), the reference of the time-to-accuracy
measurement (relative error ||x_G^k - x_G*|| / ||x_G*|| <= 1e-3).

Calls only the oracle and the scene generator.  The stored limit is checked
independently of the iteration by tests/test_oracle_pins.py
(test_golden_limit_is_optimal: the dual implied by x_G* satisfies the
subgradient condition of Eq. 2).  Run: python tests/golden/make_limits.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import scenegen    # noqa: E402

SCENE, SEED, RHO, LAM_FRAC, ITERS = "resolved_32", 20, 100.0, 0.05, 1000


def main():
    sc = scenegen.build_scene(SCENE, seed=SEED)
    lam = LAM_FRAC * scenegen.lambda_max(sc.A, sc.y)
    B = [oracle.real_form(a) for a in sc.A]
    r = oracle.sadmm(sc.A, sc.y, RHO, lam, oracle.Criterion(elim=0), iters=ITERS, B=B)
    k = oracle.kkt(sc.A, sc.y, r.state.x, r.state.s, RHO, lam, xG=r.xG, B=B)
    out = {"scene": SCENE, "seed": SEED, "rho": RHO, "lam_frac": LAM_FRAC, "lam": lam, "mu": 1.0,
           "iterations": ITERS, "kkt": {k_: float(v) for k_, v in k.items()},
           "xG": [float(v) for v in r.xG]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "resolved_32_limit.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(k, float(np.linalg.norm(r.xG)))


if __name__ == "__main__":
    main()
