"""Write the stored expected values of the GPU solve tests.

Runs only the FP64 CPU oracle (oracle/hallar_oracle.py) on the seeded
instances below and writes tests/golden/solve_values.json.  Usage:
    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402

CASES = {
    # Max-Cut SDP on Erdos-Renyi G(1000, 0.01), unit weights, r0 = 10, U0 seed 1001
    "maxcut_er_n1000_p0.01": (lambda: I.maxcut_er_1000(seed=1), 10, 1001),
    # Max-Cut SDP on the 24 x 24 torus with +-1 weights (seed 2), r0 = 8, U0 seed 1002
    "maxcut_torus_24x24_pm1": (lambda: I.maxcut_torus(24, "pm1", seed=2), 8, 1002),
    # Lovasz theta on G(300, 1500) (seed 3) with the trace row, r0 = 4, U0 seed 1003
    "theta_gnm_n300_m1500": (lambda: I.theta_gnm(300, 1500, seed=3), 4, 1003),
}


def main():
    out = {}
    for name, (make, r0, useed) in CASES.items():
        inst = make()
        t = time.time()
        res = O.hallar_solve(inst, I.initial_factor(inst.n, r0, useed),
                             opt=O.Options(tol=1e-7, r_cap=32))
        out[name] = {"pval": res.pval, "dval": res.dval, "user_value": res.user_value,
                     "kkt": res.kkt, "rank": res.rank, "converged": bool(res.converged),
                     "oracle_seconds": round(time.time() - t, 1), "tol": 1e-7, "r0": r0,
                     "u0_seed": useed}
        print(name, out[name], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
