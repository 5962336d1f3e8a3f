"""Offline driver of the oracle's kappa search (test infrastructure only; CPU, scipy).

Runs ``oracle.kappa.search_m0`` on the field recipe of one workload and prints a JSON record that
``synth/kappa.json`` stores.  The sparse LU behind sigma_min is affordable on lattices up to 6^4,
so larger workloads are searched on a 6^4 lattice of the same recipe (same eps, seed, c_sw,
boundary) and the record says so.

    python -m oracle.kappa_search NAME LX,LY,LZ,T EPS SEED CSW TARGET
"""
from __future__ import annotations

import json
import sys
import time

from . import dirac, kappa


def main(argv):
    name, dims, eps, seed, csw, target = argv
    dims = tuple(int(v) for v in dims.split(","))
    eps, seed, csw, target = float(eps), int(seed), float(csw), float(target)
    from synth import fields
    U = fields.gauge_field(dims, eps, seed)
    log = []
    t0 = time.time()
    prog = lambda m, v: print(f"m0 {m:+.5f} sigma_min {v:.6e} ({time.time() - t0:.0f} s)", file=sys.stderr, flush=True)
    m0, smin, reached = kappa.search_m0(U, csw, -1, target, log=log, progress=prog)
    rec = {"m0": m0, "kappa": dirac.kappa_from_m0(m0), "sigma_min": smin, "reached_target": reached,
           "search_lattice": list(dims),
           "eps": eps, "seed": seed, "csw": csw, "target": target, "evaluations": len(log),
           "cpu_s": round(time.time() - t0, 1), "log": log}
    print(json.dumps({name: rec}))


if __name__ == "__main__":
    main(sys.argv[1:])
