"""Tune kappa so that sigma_min(D_W) at mu = 0 hits a target on a given gauge field.

The workloads define kappa this way ("kappa tuned so that sigma_min(D_W) ~ target"); sigma_min is
measured on the workload's own lattice with ``tmg_sigma_min`` (Lanczos on (D(mu_s)^dag D(mu_s))^-1,
every product two multigrid solves in the library).  The search walks m0 = 1/(2 kappa) - 4 down
from a start value in fixed steps until sigma_min falls below the target, then bisects the last
step until sigma_min is within a relative band of the target: the first crossing from above (the
largest m0), i.e. the physical branch closest to the free theory.

    python -m paper_1710_06198_gb300.tune_kappa WORKLOAD [--start M0] [--step S] [--mu-s MU] [--out FILE]

Only argument marshalling and the one-dimensional search happen here; every solve runs in libtmg.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import PREC_F32, SOLVE_MG_MIXED, Context


def kappa_of(m0):
    return 1.0 / (2.0 * (m0 + 4.0))


def sigma_at(ctx, U, w, m0, mu_s, start, v0, prm, log, t0):
    ctx.set_params(kappa_of(m0), w["csw"], mu_s)
    ctx.load_gauge(U, -1)
    ctx.setup(v0, prm)
    sigma, rr, ns = ctx.sigma_min(start, mu_s, max_steps=48, rtol=1e-4, solve_tol=1e-9, method=SOLVE_MG_MIXED,
                                  check=False)
    log.append({"m0": m0, "sigma_min": sigma, "ritz_res": rr, "solves": ns, "t_s": round(time.time() - t0, 1)})
    print(json.dumps(log[-1]), file=sys.stderr, flush=True)
    return sigma


def search(name, start_m0=-0.5, step=0.1, band=0.02, mu_s=None, m0_min=-2.0, n_bisect=12):
    from synth import fields, workloads
    w = workloads.WORKLOADS[name]
    target = w["sigma_target"]
    mu_s = mu_s if mu_s is not None else 2.0 * target
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    ctx = Context(dims, w["block"])
    prm = Context.mg_defaults()
    prm.nv, prm.restart = w["nv"], w["restart"]
    prm.prec_fine, prm.prec_coarse = PREC_F32, PREC_F32
    v0 = fields.gaussian_spinor(dims, w["seed"] + 100, n=w["nv"])
    start = fields.gaussian_spinor(dims, w["seed"] + 300)
    log, t0 = [], time.time()
    hi, s_hi = start_m0, sigma_at(ctx, U, w, start_m0, mu_s, start, v0, prm, log, t0)
    lo = None
    m = hi
    while lo is None and m - step >= m0_min - 1e-12:
        m = round(m - step, 10)
        s = sigma_at(ctx, U, w, m, mu_s, start, v0, prm, log, t0)
        if s < target:
            lo = m
        else:
            hi, s_hi = m, s
    best = min(log, key=lambda e: abs(e["sigma_min"] - target))
    if lo is not None:
        for _ in range(n_bisect):
            if abs(best["sigma_min"] - target) <= band * target:
                break
            mid = 0.5 * (hi + lo)
            s = sigma_at(ctx, U, w, mid, mu_s, start, v0, prm, log, t0)
            if s < target:
                lo = mid
            else:
                hi = mid
            best = min(log, key=lambda e: abs(e["sigma_min"] - target))
    ctx.close()
    m0 = best["m0"]
    return {"m0": m0, "kappa": kappa_of(m0), "sigma_min": best["sigma_min"], "target": target,
            "reached_target": abs(best["sigma_min"] - target) <= band * target, "mu_s": mu_s,
            "sigma_lattice": list(dims), "eps": w["eps"], "seed": w["seed"], "csw": w["csw"],
            "rule": "first crossing from above of sigma_min(D_W) = target on the workload lattice (band %g)" % band,
            "log": log, "gpu_s": round(time.time() - t0, 1),
            "source": "tmg_sigma_min on %s: m0 = %.5f, sigma_min(D_W) = %.3e" % ("x".join(map(str, dims)), m0,
                                                                                best["sigma_min"])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--start", type=float, default=-0.5)
    ap.add_argument("--step", type=float, default=0.1)
    ap.add_argument("--mu-s", type=float, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rec = search(a.workload, a.start, a.step, mu_s=a.mu_s)
    line = json.dumps({a.workload: rec})
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
