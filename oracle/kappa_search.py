"""Offline driver of the oracle's kappa search (test infrastructure only; CPU, scipy).

Runs ``oracle.kappa.search_m0`` on the field recipe of one workload and prints a JSON record that
``synth/kappa.json`` stores.  The sparse LU behind sigma_min is affordable on lattices up to 6^4,
so larger workloads are searched on a 6^4 lattice of the same recipe (same eps, seed, c_sw,
boundary) and the record says so.

    python -m oracle.kappa_search NAME LX,LY,LZ,T EPS SEED CSW TARGET

On the synthetic fields of the workloads (uncorrelated link noise, far rougher than a physical
ensemble) the target is not reached on the physical branch of a 6^4 lattice, and near the
strong-coupling critical point the two-level method stops converging (the oracle and the GPU both
stall at the same residual).  The workloads therefore take kappa from the convergence edge:

    python -m oracle.kappa_search --edge NAME EPS SEED CSW MU NV TARGET [--write synth/kappa.json]
    python -m oracle.kappa_search --merge synth/kappa.json RECORD.json ...
    python -m oracle.kappa_search --select synth/kappa.json NAME ...

The edge itself is too close to breakdown to carry over to the workloads' lattices (at the edge m0
of the 16^3 x 32 recipe the GPU needs 481 outer steps against 39 on the 8^4 search lattice), so
--select moves each record to the most critical m0 of the recorded walk whose step count is at
most twice the count at m0 = 0.

walks m0 down with the oracle's two-level DD-alpha-AMG on an 8^4 lattice of the workload's recipe
(4^4 blocks and aggregates, N_v test vectors, Gaussian right-hand side), keeps the most critical m0
that still converges within 50 outer steps (step 0.1, two bisections), and records sigma_min(D_W)
there on the 6^4 lattice of the same recipe.
"""
from __future__ import annotations

import json
import sys
import time

from . import dirac, kappa


def edge(argv):
    write = None
    if "--write" in argv:
        i = argv.index("--write")
        write = argv[i + 1]
        argv = argv[:i] + argv[i + 2:]
    name, eps, seed, csw, mu, nv, target = argv
    eps, seed, csw, mu, nv, target = float(eps), int(seed), float(csw), float(mu), int(nv), float(target)
    from synth import fields
    d8, d6 = (8, 8, 8, 8), (6, 6, 6, 6)
    U8 = fields.gauge_field(d8, eps, seed)
    b = fields.gaussian_spinor(d8, seed + 1)
    v0 = fields.gaussian_spinor(d8, seed + 100, n=nv)
    log = []
    t0 = time.time()
    prog = lambda m, n: print(f"m0 {m:+.5f} mg_steps {n} ({time.time() - t0:.0f} s)", file=sys.stderr, flush=True)
    m0 = kappa.search_m0_mg(U8, csw, mu, (4, 4, 4, 4), nv, b, v0, log=log, progress=prog)
    U6 = fields.gauge_field(d6, eps, seed)
    smin = kappa.sigma_min(U6, dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, tbc=-1))
    rec = {"m0": m0, "kappa": dirac.kappa_from_m0(m0), "sigma_min": smin, "reached_target": bool(smin <= target),
           "target": target, "rule": "convergence edge of the oracle two-level DD-alpha-AMG (50 outer steps)",
           "mg_lattice": list(d8), "sigma_lattice": list(d6), "eps": eps, "seed": seed, "csw": csw, "mu": mu,
           "nv": nv, "cpu_s": round(time.time() - t0, 1), "mg_log": log,
           "source": f"oracle kappa_search --edge: m0 = {m0:.4f}, sigma_min(D_W, 6^4) = {smin:.3e}"}
    print(json.dumps({name: rec}))
    if write:
        try:
            with open(write) as f:
                table = json.load(f)
        except FileNotFoundError:
            table = {}
        table[name] = rec
        with open(write, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")


def merge(argv):
    """--merge TABLE RECORD...: store the records printed by --edge runs into TABLE."""
    table_path, records = argv[0], argv[1:]
    try:
        with open(table_path) as f:
            table = json.load(f)
    except FileNotFoundError:
        table = {}
    for path in records:
        with open(path) as f:
            table.update(json.loads(f.read().strip().splitlines()[-1]))
    with open(table_path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def select(argv):
    """--select TABLE NAME...: move each named record of TABLE from the convergence edge to the
    margin rule of kappa.select_m0 (recorded walk, ratio 2) and recompute sigma_min there."""
    table_path, names = argv[0], argv[1:]
    with open(table_path) as f:
        table = json.load(f)
    from synth import fields
    for name in names:
        rec = table[name]
        m0 = kappa.select_m0([tuple(e) for e in rec["mg_log"]], 2.0)
        U6 = fields.gauge_field(tuple(rec["sigma_lattice"]), rec["eps"], rec["seed"])
        smin = kappa.sigma_min(U6, dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=rec["csw"], tbc=-1))
        rec.update({"edge_m0": rec.get("edge_m0", rec["m0"]), "m0": m0, "kappa": dirac.kappa_from_m0(m0), "sigma_min": smin,
                    "reached_target": bool(smin <= rec["target"]),
                    "rule": "most critical m0 of the walk whose oracle two-level steps are at most twice those at m0 = 0",
                    "source": f"oracle kappa_search --select: m0 = {m0:.4f}, sigma_min(D_W, 6^4) = {smin:.3e}"})
        with open(table_path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")
        print(name, m0, smin, flush=True)


def main(argv):
    if argv and argv[0] == "--select":
        return select(argv[1:])
    if argv and argv[0] == "--edge":
        return edge(argv[1:])
    if argv and argv[0] == "--merge":
        return merge(argv[1:])
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
