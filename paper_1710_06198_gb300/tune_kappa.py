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


def find_crossing(sig, target, start_m0=-0.5, step=0.05, band=0.02, m0_min=-2.0, n_bisect=14, n_golden=14):
    """The first crossing from above of sigma(m0) = target, with sigma(m0) evaluated by `sig`.

    Walks m0 down from start_m0 in steps; stops at the first value below the target, or once sigma
    has risen twice after a minimum: sigma_min of the Wilson operator moves with m0 like |m0 - m_c|
    near a real eigenvalue m_c, so a walk can step over the dip.  A passed dip is searched by golden
    sections for a point below the target.  The last interval (sigma above the target at its upper
    end, below at its lower end) is then bisected until sigma is within the relative band of the
    target.  Returns (m0 of the evaluation closest to the target, {m0: sigma} of all evaluations)."""
    ev = {}

    def f(m):
        m = round(m, 10)
        if m not in ev:
            ev[m] = sig(m)
        return ev[m]

    lo = None
    m, best_m, rises = start_m0, start_m0, 0
    f(m)
    while m - step >= m0_min - 1e-12:
        m = round(m - step, 10)
        if f(m) < target:
            lo = m
            break
        if ev[m] < ev[round(best_m, 10)]:
            best_m, rises = m, 0
        else:
            rises += 1
            if rises >= 2:
                break
    if lo is None:
        a, b = best_m - step, best_m + step
        gr = 0.5 * (5.0 ** 0.5 - 1.0)
        c, d = b - gr * (b - a), a + gr * (b - a)
        for _ in range(n_golden):
            if f(c) < target:
                lo = c
                break
            if f(d) < target:
                lo = d
                break
            if ev[round(c, 10)] < ev[round(d, 10)]:
                b, d = d, c
                c = b - gr * (b - a)
            else:
                a, c = c, d
                d = a + gr * (b - a)
    if lo is None:
        return min(ev, key=lambda mm: abs(ev[mm] - target)), ev
    # bisect the bracket [lo, hi] (sigma below the target at lo, at or above it at hi) onto the
    # crossing nearest hi, i.e. the upper branch of the dip: every point strictly inside the dip has
    # sigma below the target, so a midpoint at or above it lies on the upper branch
    ups = [mm for mm, v in ev.items() if mm > lo and v >= target]
    hi = min(ups) if ups else lo + step
    for _ in range(n_bisect):
        if abs(f(hi) - target) <= band * target:
            break
        mid = 0.5 * (hi + lo)
        v = f(mid)
        if v < target:
            lo = mid
        else:
            hi = mid
        if abs(v - target) <= band * target:
            break
    bracket = [mm for mm in ev if lo - 1e-9 <= mm <= hi + 1e-9]
    return min(bracket, key=lambda mm: abs(ev[mm] - target)), ev


def search(name, start_m0=-0.5, step=0.05, band=0.02, mu_s=None, m0_min=-2.0):
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
    m0, ev = find_crossing(lambda m: sigma_at(ctx, U, w, m, mu_s, start, v0, prm, log, t0), target, start_m0, step,
                           band, m0_min)
    ctx.close()
    return {"m0": m0, "kappa": kappa_of(m0), "sigma_min": ev[m0], "target": target,
            "reached_target": abs(ev[m0] - target) <= band * target, "mu_s": mu_s,
            "sigma_lattice": list(dims), "eps": w["eps"], "seed": w["seed"], "csw": w["csw"],
            "rule": "first crossing from above of sigma_min(D_W) = target on the workload lattice (band %g)" % band,
            "log": log, "gpu_s": round(time.time() - t0, 1),
            "source": "tmg_sigma_min on %s: m0 = %.6f, sigma_min(D_W) = %.3e" % ("x".join(map(str, dims)), m0, ev[m0])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--start", type=float, default=-0.5)
    ap.add_argument("--step", type=float, default=0.05)
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
