"""Writes tests/golden/bench_cycles.json: the number of cycles (plain FP64,
V(2,1), lambda = 5, junction relaxation at its defaults) the FP64 oracle needs to bring each
benchmark workload to its relative-residual target.  Calls only the oracle;
bench.py uses the counts to scale the oracle's seconds per cycle into its
unknowns/s baseline.

    python tests/golden/make_bench_cycles.py [workload ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1111_0983_gb300 import inputs  # noqa: E402

TARGETS = {"flower1025": (inputs.flower, 1025, 33, 1e-10), "disk65": (inputs.disk, 65, 17, 1e-10),
           "flower4097": (inputs.flower, 4097, 33, 1e-9), "torus257": (inputs.torus, 257, 17, 1e-10),
           "torus513": (inputs.torus, 513, 17, 5e-10)}
# torus513 and flower4097: the FP64 oracle stalls above 1e-10 there (the
# rounding of u in its smoother times 2d/h^2), so their targets are the
# floors the plain FP64 solves reach


def main(names):
    path = os.path.join(HERE, "bench_cycles.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        fac, n, nc, rtol = TARGETS[name]
        P = fac()
        O = oracle.Oracle(P.phi_grid(n), nc)
        for l in range(O.nlev):
            O.set_bc(l, P.bc_types(O.ghosts(l)["B"]))
        G = O.ghosts(0)
        O.set_rhs(P.f_grid(n), P.g_values(G["B"], G["nu"], P.bc_types(G["B"])))
        threads = oracle.set_threads(os.cpu_count() or 1)   # the count does not change the iterates
        t = time.perf_counter()
        _, norms, ok = O.solve(rtol=rtol, max_cycles=200)
        out[name] = {"cycles": len(norms) - 1, "converged": bool(ok), "rtol": rtol,
                     "rel": float(norms[-1] / norms[0]), "oracle_seconds": time.perf_counter() - t,
                     "threads": threads}
        print(name, out[name], flush=True)
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["disk65", "flower1025"])
