"""Write the stored expected values of the GPU solve tests.

Runs only the FP64 CPU oracle (oracle/hallar_oracle.py) on the seeded
instances below and writes tests/golden/solve_values.json, one entry per
instance, keeping entries already present.  Usage:
    python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve_values.json")

# name: (instance, r0, U0 seed, r_cap)
CASES = {
    # Max-Cut SDP on Erdos-Renyi G(1000, 0.01), unit weights
    "maxcut_er_n1000_p0.01": (lambda: I.maxcut_er_1000(seed=1), 10, 1001, 32),
    # Max-Cut SDP on the 16 x 16 torus with +-1 weights (seed 2)
    "maxcut_torus_16x16_pm1": (lambda: I.maxcut_torus(16, "pm1", seed=2), 8, 1002, 64),
    # Lovasz theta on G(40, 80) (seed 3) with the trace row: a random graph
    # the oracle solves to 1e-7 in under half an hour (about 2.8e6 gradients;
    # G(60, 150) did not finish within an hour)
    "theta_gnm_n40_m80": (lambda: I.theta_gnm(40, 80, seed=3), 4, 1003, 64),
}


def main(names):
    out = json.load(open(PATH)) if os.path.exists(PATH) else {}
    for name in names or list(CASES):
        if name in out:
            continue
        make, r0, useed, rcap = CASES[name]
        inst = make()
        t = time.time()
        res = O.hallar_solve(inst, I.initial_factor(inst.n, r0, useed),
                             opt=O.Options(tol=1e-7, r_cap=rcap))
        out[name] = {"pval": res.pval, "dval": res.dval, "user_value": res.user_value,
                     "kkt": res.kkt, "rank": res.rank, "converged": bool(res.converged),
                     "oracle_seconds": round(time.time() - t, 1), "tol": 1e-7, "r0": r0,
                     "u0_seed": useed, "r_cap": rcap}
        print(name, out[name], flush=True)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
