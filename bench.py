#!/usr/bin/env python
"""Benchmark of the twisted-mass DD-alpha-AMG solve on one GB300 (arXiv:1710.06198 hot path).

Workload (the mixed-precision fine-level configuration): a 16^3 x 32 lattice, SU(3) links
U = exp(i 0.35 H) from seed 3, c_sw = 1.5, mu = 0.003, antiperiodic time, kappa from the
oracle's sigma_min search (synth/kappa.json), two-level DD-alpha-AMG with 4^4 SAP blocks and
aggregates, N_v = 16 test vectors (setup: 5 SAP passes + 3 cycle iterations, untimed), one
Gaussian right-hand side (seed 4), solved to a true FP64 relative residual of 1e-10.

One timed step = one mixed-precision solve (FP64 defect correction around FP32 FGMRES with the
FP32 / FP16-link multigrid cycle), inputs already resident in HBM.  L2 (129 MB) is flushed
between steps by writing a 512 MB buffer.  The JSON line also carries:
  * e2e: the same solve through the public API with pinned host buffers (H2D + D2H timed);
  * roofline: the kernel class with the largest share of the solve's device time (CUDA events
    around each of its launches in one instrumented solve), its algorithmic bytes per launch
    against the measured HBM copy peak, with the other classes listed beside it;
  * fp64_solve_s, cg_fp64: the plain FP64 multigrid and FP64 CG solves of the same system;
  * cpu_baseline: the FP64 numpy oracle timed on the host cores: its whole 8^4 solve, its
    operator on the timed lattice, and a labelled estimate for the timed solve.
`--impl reference` times the oracle itself (the CPU reference arm) on the timed lattice.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import workloads  # noqa: E402

WORKLOAD = dict(name="tm_clover_16x16x16x32_mixed_2lvl", tol=1e-10,
                **workloads.WORKLOADS["tm_clover_16x16x16x32_mixed_2lvl"])
METRIC = "DD-alphaAMG solve s to 1e-10 (mixed+batched vs FP64) ; dslash GB/s vs HBM peak"


def workload_kappa(w):
    return workloads.kappa(w["name"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# FP32 flops per site (conventional counts): Wilson-clover operator = 1320 hopping + 504 clover
# + 48 twist and combination; SAP colour launch per site of the colour = residual (D + 24) and
# n_MR = 4 minimal-residual steps of (block operator + 3 dot products + 2 axpys = D + 144)
D_FLOPS = 1872
SAP_FLOPS = (D_FLOPS + 24) + 4 * (D_FLOPS + 144)


def algorithmic_flops(kind, V):
    if kind.startswith("sap"):
        return (V // 2) * SAP_FLOPS
    if kind.startswith("dslash"):
        return V * D_FLOPS
    return None


def coarse_step_bytes(nc, nd, ncol=1, es=8, eo=False):
    """Bytes one coarse GMRES step must move at least: the coarse operator once in its 5-block form
    (self + 4 forward hops; the backward hops follow from G5_c-hermiticity), for the odd-even reduced
    system also the even sites' inverse blocks, and one coarse vector read and written per column
    (FP32 complex: 8 bytes)."""
    return nc * (5 * nd * nd * es + 2 * ncol * nd * es) + (nc // 2) * nd * nd * es * int(eo)


def kernel_sha(kind):
    """Hash of the source file that holds a kernel class (a stored ncu traffic figure is used only
    while the kernel it was taken from is unchanged)."""
    import hashlib
    src = {"coarse_solve": "k_coarse_gmres.cu", "sap_f32": "k_mg.cu", "sap_f16": "k_mg.cu", "restrict": "k_mg.cu",
           "prolong": "k_mg.cu", "dslash_f32": "k_dslash.cu", "dslash_f64": "k_dslash.cu"}.get(kind)
    if not src:
        return None
    with open(os.path.join(ROOT, "paper_1710_06198_gb300", "csrc", src), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def run_config3(dev):
    """The 24^3 x 48 three-level workload: 12 point sources D(mu) x = b and the first solves
    D(-mu_k) y = g5 phi of the 8 shifted systems, all 20 in one lock-step mixed-precision solve
    (setup untimed), against the same 20 systems solved one after another by the FP64 multigrid and
    by the mixed single-column solve."""
    import torch

    import paper_1710_06198_gb300 as tmg
    from synth import fields
    name = "tm_clover_24x24x24x48_batched_3lvl"
    w = workloads.WORKLOADS[name]
    kappa, _ = workloads.kappa(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    ctx = tmg.Context(dims, w["block"], device=dev.index or 0)
    try:
        ctx.set_params(kappa, w["csw"], w["mu"])
        ctx.load_gauge(U, -1)
        prm = tmg.Context.mg_defaults()
        prm.nv, prm.restart = w["nv"], w["restart"]
        t0 = time.time()
        ctx.setup(fields.gaussian_spinor(dims, w["seed"] + 100, n=w["nv"]), prm)
        q = workloads.level2_params(w, tmg.Context.level2_defaults())
        c1 = ctx.coarse_lat
        ctx.setup_level2(fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * w["nv"], w["seed"] + 200, n=w["nv2"]), q)
        torch.cuda.synchronize()
        setup_s = time.time() - t0
        sig = workloads.shifts(w["n_shifts"])
        mu_k = [float(np.sqrt(w["mu"] ** 2 + s_)) for s_ in sig]
        ps = fields.point_sources(dims)
        g5phi = fields.gaussian_spinor(dims, w["phi_seed"])
        g5phi[..., 2:, :] *= -1.0          # gamma5 = diag(1, 1, -1, -1) in the chiral spin basis
        b = torch.from_numpy(np.ascontiguousarray(np.concatenate([ps, np.broadcast_to(g5phi, (len(sig),) + g5phi.shape)]))).to(dev)
        mus = [w["mu"]] * len(ps) + [-m for m in mu_k]
        x = torch.empty_like(b)

        def timed(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3, r

        ctx.solve(b, tol=w.get("tol", 1e-10), method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus, out=x)   # warm-up
        tb, (_, stb) = timed(lambda: ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus, out=x))
        rb = ctx.apply(x, tmg.OP_D, tmg.PREC_F64, mu_per_col=mus) - b
        worst = max(float(torch.linalg.vector_norm(rb[j]) / torch.linalg.vector_norm(b[j])) for j in range(len(mus)))
        x1 = torch.empty_like(b[0])
        t64, it64, tmx, itmx = 0.0, 0, 0.0, 0
        for j in range(len(mus)):
            t, (_, s1) = timed(lambda: ctx.solve(b[j], tol=1e-10, method=tmg.SOLVE_MG_F64, mu_per_col=[mus[j]], out=x1))
            t64 += t
            it64 += s1["iterations"]
            t, (_, s2) = timed(lambda: ctx.solve(b[j], tol=1e-10, method=tmg.SOLVE_MG_MIXED, mu_per_col=[mus[j]], out=x1))
            tmx += t
            itmx += s2["iterations"]
        return {"lattice": list(dims), "levels": 3, "rhs": len(mus), "kinds": "12 point sources + 8 shifted systems",
                "kcycle": {"smooth_m": q.smooth_m, "k_rtol": q.k_rtol, "level2_gmres_m": q.coarse_m, "form": "lock-step, tensor-core applies"},
                "setup_s_untimed": round(setup_s, 2), "batched_mixed_s": round(tb, 4), "batched_iterations": stb["iterations"],
                "batched_true_residual_max": worst, "sequential_fp64_multigrid_s": round(t64, 4),
                "sequential_fp64_iterations_total": it64, "sequential_mixed_s": round(tmx, 4),
                "sequential_mixed_iterations_total": itmx, "speedup_batched_vs_sequential_fp64": round(t64 / tb, 2),
                "speedup_batched_vs_sequential_mixed": round(tmx / tb, 2)}
    finally:
        ctx.close()


def stored_traffic(kind):
    """DRAM bytes per launch of a kernel class from an ncu capture summarised under profiles/ (a line
    'traffic: <kind> <bytes> bytes per launch, source sha <sha>'), or None when no summary has one
    or the kernel's source changed since the capture."""
    import glob
    import re
    pat = re.compile(r"^traffic: (\S+) (\d+) bytes per launch, source sha (\w+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = pat.match(line.strip())
                if m and m.group(1) == kind and m.group(3) == kernel_sha(kind):
                    return int(m.group(2))
    return None


def algorithmic_bytes(kind, V, nv, nc, nd):
    """Bytes one launch of a kernel class must move at least (each input read once, each output
    written once); per-site figures are listed in the design notes."""
    spinor32, spinor64 = 96, 192
    if kind == "dslash_f32":
        return V * (2 * spinor32 + 4 * 48 + 288)
    if kind == "dslash_f16":     # FP32 spinors, FP16 links and clover (the F16 mode of the solve)
        return V * (2 * spinor32 + 4 * 24 + 144 + 4)
    if kind == "dslash_h16":     # all FP16: fixed-point spinors with per-site norms (52 B), links, clover
        return V * (2 * 52 + 4 * 24 + 144 + 4)
    if kind == "dslash_f64":
        return V * (2 * spinor64 + 4 * 144 + 576)
    if kind == "sap_f32":       # one colour: b, x read, x written, 4 links and clover of the colour's sites
        return (V // 2) * (3 * spinor32 + 4 * 48 + 288)
    if kind == "sap_f16":
        return (V // 2) * (3 * spinor32 + 4 * 24 + 144 + 4)
    if kind == "sap_f64":
        return (V // 2) * (3 * spinor64 + 4 * 144 + 576)
    if kind == "schur_f32":      # one Dhat application, both half-lattice kernels, per lattice site:
        # links read twice (2 x 4 x 32 B, 8-real), five half-lattice spinor passes (x_o twice, t_e
        # written and read, y_o written: 5 x 96 / 2), the even sites' inverse (576 / 2) and the odd
        # sites' clover (288 / 2)
        return V * (256 + 240 + 288 + 144)
    if kind == "schur_f64":      # the same with 12-real FP64 links (96 B), FP64 spinors and blocks
        return V * (768 + 480 + 576 + 288)
    if kind == "restrict":
        return V * spinor32 * (1 + nv) + nc * nd * 8
    if kind == "prolong":
        return V * spinor32 * (1 + nv) + nc * nd * 8
    if kind == "coarse_apply":
        return nc * (9 * nd * nd * 8 + 2 * nd * 8)
    return None


def run_kernel_case(args):
    """A single kernel class on a 24^3 x 48 lattice (working set above the 129 MB L2), for ncu."""
    import torch
    import paper_1710_06198_gb300 as tmg
    from synth import fields
    dims = (24, 24, 24, 48)
    U = fields.gauge_field(dims, 0.3, 4)
    ctx = tmg.Context(dims, (4, 4, 4, 4))
    ctx.set_params(1.0 / (2.0 * (4.0 - 0.4)), 1.6, 0.002)
    ctx.load_gauge(U, -1)
    for kv in args.tune:
        k, v = kv.split("=")
        ctx.tune(k, float(v))
    if args.kernel_case == "dslash":
        ms = ctx.bench_dslash(tmg.PREC_F32, 3)
        print(json.dumps({"kernel_case": "dslash", "ms": ms}))
    elif args.kernel_case == "coarse_tc":
        prm = tmg.Context.mg_defaults()
        prm.nv, prm.n_init, prm.n_iter = 16, 0, 0
        ctx.setup(fields.gaussian_spinor(dims, 5, n=16), prm)
        clat = ctx.coarse_lat
        xc = torch.from_numpy(fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 32, 7, n=20)).cuda()
        mus = np.linspace(0.001, 0.01, 20)
        yc = ctx.coarse_apply_multi(xc, mus)
        tmg.profile(ctx, True)
        for _ in range(5):
            yc = ctx.coarse_apply_multi(xc, mus)
        prof = tmg.profile_read(ctx)
        tmg.profile(ctx, False)
        torch.cuda.synchronize()
        n_l, ms = prof["coarse_apply"]
        nc, nd = int(np.prod(clat)), 32
        algo = nc * 9 * nd * nd * 8 + 2 * 20 * nc * nd * 8
        us = 1e3 * ms / max(1, n_l)
        print(json.dumps({"kernel_case": "coarse_tc", "norm": float(torch.linalg.vector_norm(yc)), "us_per_launch": round(us, 2),
                          "algo_bytes": algo, "gbs": round(algo / (us * 1e-6) / 1e9, 1),
                          "tflops": round(nc * 9 * (2 * nd) ** 2 * 2 * 20 / (us * 1e-6) / 1e12, 2)}))
    elif args.kernel_case == "schur":
        # the even-odd reduced operator, staged (eo_stage 1) then direct (eo_stage 0): two applications each
        for stage in (1, 0):
            ctx.tune("eo_stage", stage)
            ms = ctx.bench_schur(tmg.PREC_F32, 1)
        print(json.dumps({"kernel_case": "schur", "ms": ms}))
    elif args.kernel_case == "sap":
        prm = tmg.Context.mg_defaults()
        prm.nv, prm.n_init, prm.n_iter, prm.sap_sweeps = 2, 0, 0, 1
        ctx.setup(fields.gaussian_spinor(dims, 5, n=2), prm)
        b = torch.from_numpy(fields.gaussian_spinor(dims, 6)).cuda()
        x = torch.zeros_like(b)
        y = ctx.sap(b, x, tmg.PREC_F32)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": "sap", "norm": float(torch.linalg.vector_norm(y))}))


def run_ours(args):
    import torch
    import paper_1710_06198_gb300 as tmg
    from synth import fields

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = WORKLOAD
    kappa, kinfo = workload_kappa(w)
    U = fields.gauge_field(w["dims"], w["eps"], w["seed"])
    b_host = fields.gaussian_spinor(w["dims"], w["rhs_seed"])
    v0 = fields.gaussian_spinor(w["dims"], w["setup_seed"], n=w["nv"])
    ctx = tmg.Context(w["dims"], w["block"], device=local)
    ctx.set_params(kappa, w["csw"], w["mu"])
    ctx.load_gauge(U, -1)
    for kv in args.tune:
        k, v = kv.split("=")
        ctx.tune(k, float(v))
    prm = tmg.Context.mg_defaults()
    prm.nv = w["nv"]
    prm.sap_mr = w.get("sap_mr", prm.sap_mr)
    prm.coarse_m = w.get("coarse_m", prm.coarse_m)
    ctx.tune("coarse_eo", w.get("coarse_eo", 0))
    ctx.tune("batched_coarse_m", w.get("batched_coarse_m", 0))
    prm.prec_fine = tmg.PREC_F16 if args.fine == "f16" else tmg.PREC_F32
    prm.prec_coarse = tmg.PREC_F32
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.setup(v0, prm)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    autotune_ms = None if args.no_autotune else ctx.autotune()

    dev = torch.device("cuda", local)
    b = torch.from_numpy(b_host).to(dev)
    x = torch.empty_like(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(method=tmg.SOLVE_MG_MIXED):
        _, st = ctx.solve(b, tol=w["tol"], method=method, out=x)
        return st

    if args.ncu_solve:
        # one warm solve, then exactly one solve inside the profiler range (for ncu --profile-from-start off)
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        st = step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_solve": True, "iterations": st["iterations"], "launches_total": tmg.launch_count(ctx)}))
        return
    if args.ncu_batched:
        # the lock-step solve of the point sources: one warm solve, then one inside the profiler range
        bb = torch.from_numpy(np.ascontiguousarray(fields.point_sources(w["dims"])[:args.batch])).to(dev)
        xb = torch.empty_like(bb)
        ctx.solve(bb, tol=w["tol"], method=tmg.SOLVE_MG_BATCHED, out=xb)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, stb = ctx.solve(bb, tol=w["tol"], method=tmg.SOLVE_MG_BATCHED, out=xb)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_batched": True, "rhs": args.batch, "iterations": stb["iterations"]}))
        return

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local)
    sampler.start()
    times, iters, stats = [], [], None
    n0 = tmg.launch_count(ctx)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        stats = step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters.append(stats["iterations"])
    torch.cuda.synchronize()
    launches = (tmg.launch_count(ctx) - n0) // max(1, args.steps)
    clocks = sampler.stop()
    t_step = max_over_ranks(sum(times) / len(times), world, dev)
    # the same solves with the cycle launched kernel by kernel instead of replayed as a CUDA graph
    ctx.tune("cycle_graph", 0)
    t_eager = []
    for _ in range(max(1, args.steps // 2)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        t_eager.append(e0.elapsed_time(e1) / 1e3)
    ctx.tune("cycle_graph", 1)
    step()
    graphs = {"cycle_graphs": tmg.graph_count(ctx), "s_with_graphs": round(t_step, 6),
              "s_kernel_by_kernel": round(sum(t_eager) / len(t_eager), 6)}
    # verify the last solve in FP64 on the device (true residual through the FP64 operator)
    r = (ctx.apply(x, tmg.OP_D, tmg.PREC_F64) - b)
    true_res = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))

    # end to end through the public API with pinned host buffers
    bp = torch.from_numpy(b_host).pin_memory()
    xp = torch.empty_like(bp).pin_memory()
    bnp, xnp = bp.numpy(), xp.numpy()
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve(bnp, tol=w["tol"], method=tmg.SOLVE_MG_MIXED, out=xnp)
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e) / len(e2e), world, dev)

    # comparators: plain FP64 multigrid and FP64 CG on the same system
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st64 = ctx.solve(b, tol=w["tol"], method=tmg.SOLVE_MG_F64, out=x)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t0
    cg = None
    if not args.no_cg:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, stcg = ctx.solve(b, tol=w["tol"], method=tmg.SOLVE_CG_F64, out=x, maxiter=args.cg_maxiter, check=False)
        torch.cuda.synchronize()
        cg = {"s": time.perf_counter() - t0, "iterations": stcg["iterations"], "true_residual": stcg["true_residual"]}

    # the odd-even CG on the Schur operator (Fig. 1's comparator) on the same system
    cg_eo = None
    if not args.no_cg:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, steo = ctx.solve(b, tol=w["tol"], method=tmg.SOLVE_CG_EO, out=x, maxiter=args.cg_maxiter, check=False)
        torch.cuda.synchronize()
        cg_eo = {"s": time.perf_counter() - t0, "iterations": steo["iterations"], "true_residual": steo["true_residual"]}

    # shifted systems (D^dag D + sigma_k) as twists mu_k = sqrt(mu^2 + sigma_k), solved one after
    # another from zero and with first-order Taylor initial guesses (Sec. 3)
    shifts = None
    if args.shifts > 0:
        sig = workloads.shifts(args.shifts)
        mus = [float(np.sqrt(w["mu"] ** 2 + sg)) for sg in sig]
        res = {}
        for guess in (0, 1, 2):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, its, sts = ctx.solve_shifts(b, mus, tol=w["tol"], guess=guess, taylor_tol=1e-2)
            torch.cuda.synchronize()
            res[guess] = {"s": round(time.perf_counter() - t0, 5), "iterations_per_system": its,
                          "iterations_total": sts["iterations"]}
        shifts = {"sigma": sig, "mu_k": mus, "zero_guess": res[0], "previous_solution_guess": res[1],
                  "taylor_guess": res[2], "time_saved_frac_taylor": round(1.0 - res[2]["s"] / res[0]["s"], 3),
                  "time_saved_frac_previous": round(1.0 - res[1]["s"] / res[0]["s"], 3)}

    # batched: the 12 spin-colour point sources in one lock-step solve (mixed precision)
    batched = None
    if args.batch > 0:
        nb = args.batch
        bb = torch.from_numpy(np.ascontiguousarray(fields.point_sources(w["dims"])[:nb])).to(dev)
        xb = torch.empty_like(bb)
        ctx.solve(bb, tol=w["tol"], method=tmg.SOLVE_MG_BATCHED, out=xb)   # warm-up
        tb = []
        for _ in range(max(1, args.steps // 2)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, stb = ctx.solve(bb, tol=w["tol"], method=tmg.SOLVE_MG_BATCHED, out=xb)
            e1.record()
            e1.synchronize()
            tb.append(e0.elapsed_time(e1) / 1e3)
        tbm = sum(tb) / len(tb)
        rb = ctx.apply(xb, tmg.OP_D, tmg.PREC_F64) - bb
        worst = max(float(torch.linalg.vector_norm(rb[j]) / torch.linalg.vector_norm(bb[j])) for j in range(nb))
        tmg.profile(ctx, True)
        ctx.solve(bb, tol=w["tol"], method=tmg.SOLVE_MG_BATCHED, out=xb)
        bprof = {k: {"launches": n_, "ms_total": round(ms_, 3)} for k, (n_, ms_) in tmg.profile_read(ctx).items() if n_}
        tmg.profile(ctx, False)
        batched = {"rhs": nb, "kind": "point sources", "s_total": round(tbm, 5), "s_per_rhs": round(tbm / nb, 6),
                   "iterations": stb["iterations"], "coarse_iterations": stb["coarse_iterations"],
                   "true_residual_max": worst, "per_rhs_over_single": round(tbm / nb / t_step, 3),
                   "kernels_one_solve": bprof}

    # the 24^3 x 48 three-level workload: 12 point sources and 8 shifted systems in one lock-step
    # mixed-precision solve, against the same 20 systems solved one at a time by the FP64 multigrid
    config3 = None
    if args.config3 and world == 1:
        config3 = run_config3(dev)

    # one instrumented solve: device time of every kernel class
    flush.zero_()
    tmg.profile(ctx, True)
    step()
    prof = tmg.profile_read(ctx)
    tmg.profile(ctx, False)
    V = int(np.prod(w["dims"]))
    nd = 2 * w["nv"]
    nc = V // int(np.prod(w["block"]))
    kernels = {}
    for k, (n, ms) in prof.items():
        if n:
            ab = algorithmic_bytes(k, V, w["nv"], nc, nd)
            kernels[k] = {"launches": n, "ms_total": round(ms, 4), "us_per_launch": round(1e3 * ms / n, 3),
                          "algo_bytes_per_launch": ab,
                          "gbs": round(ab / (ms / n * 1e-3) / 1e9, 1) if ab else None}
    for k, v in kernels.items():
        fl = algorithmic_flops(k, V)
        if fl:
            v["tflops"] = round(fl / (v["us_per_launch"] * 1e-6) / 1e12, 2)
    if "coarse_solve" in kernels and stats.get("coarse_iterations"):
        # one launch = one whole coarse GMRES; per GMRES step it must read the coarse operator once
        # in its 5-block form (self + 4 forward hops; the backward hops follow from G5_c-hermiticity)
        # and read/write one coarse vector
        kc = kernels["coarse_solve"]
        ksteps = stats["coarse_iterations"] / max(1, kc["launches"])
        kc["gmres_steps_per_launch"] = round(ksteps, 2)
        kc["us_per_gmres_step"] = round(kc["us_per_launch"] / max(ksteps, 1e-9), 2)
        kc["algo_bytes_per_launch"] = int(round(ksteps * coarse_step_bytes(nc, nd, eo=bool(w.get("coarse_eo", 0)))))
        kc["gbs"] = round(kc["algo_bytes_per_launch"] / (kc["us_per_launch"] * 1e-6) / 1e9, 1)
        kc["bound"] = "latency: grid-wide barriers and the Hessenberg update per GMRES step; the 9-block stencil stays in L2"
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    peak, peak_src = peaks()
    # dslash bandwidth of the FP32 operator alone: average of launches with L2 flushed in between
    dsl = []
    for _ in range(20):
        flush.zero_()
        dsl.append(ctx.bench_dslash(tmg.PREC_F32, 1))
    dsl_ms = statistics.median(dsl)
    dsl_gbs = algorithmic_bytes("dslash_f32", V, 0, 0, 0) / (dsl_ms * 1e-3) / 1e9
    traffic = stored_traffic(dom)
    # the kernel class with the largest share of the solve's device time, against the measured HBM
    # copy peak with its algorithmic bytes per launch
    roof = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": round(kernels[dom]["gbs"] / peak, 3) if kernels[dom]["gbs"] else None,
            "peak_source": peak_src, "traffic": traffic,
            "time_share": round(kernels[dom]["ms_total"] / sum(v["ms_total"] for v in kernels.values()), 3)}
    others = {}
    for k in ("sap_f32", "sap_f16", "dslash_f32", "dslash_f64", "restrict", "prolong"):
        if k in kernels and k != dom and kernels[k]["gbs"]:
            others[k] = {"achieved_gbs": kernels[k]["gbs"], "frac": round(kernels[k]["gbs"] / peak, 3),
                         "time_share": round(kernels[k]["ms_total"] / sum(v["ms_total"] for v in kernels.values()), 3)}
            if kernels[k].get("tflops"):
                others[k]["tflops"] = kernels[k]["tflops"]
    roof["other_kernels"] = others
    # the operator alone on a lattice whose working set (446 MB) exceeds L2
    dsl_large = None
    if not args.no_large_dslash:
        dl = (24, 24, 24, 48)
        cl = tmg.Context(dl, (4, 4, 4, 4), device=local)
        cl.set_params(kappa, w["csw"], w["mu"])
        cl.load_gauge(fields.gauge_field(dl, 0.3, 4), -1)
        Vl = int(np.prod(dl))
        ms_l = cl.bench_dslash(tmg.PREC_F32, 50)
        gbs_l = algorithmic_bytes("dslash_f32", Vl, 0, 0, 0) / (ms_l * 1e-3) / 1e9
        ms_h = cl.bench_dslash(tmg.PREC_F16, 50)
        gbs_h = algorithmic_bytes("dslash_h16", Vl, 0, 0, 0) / (ms_h * 1e-3) / 1e9
        schur = {}
        for stage in (1, 0):
            cl.tune("eo_stage", stage)
            ms_s = cl.bench_schur(tmg.PREC_F32, 50)
            gbs_s = algorithmic_bytes("schur_f32", Vl, 0, 0, 0) / (ms_s * 1e-3) / 1e9
            schur["staged" if stage else "direct"] = {"us": round(ms_s * 1e3, 2), "gbs": round(gbs_s, 1),
                                                      "frac_measured_peak": round(gbs_s / peak, 3),
                                                      "frac_nominal_8tbs": round(gbs_s / 8000.0, 3)}
        cl.tune("eo_stage", 1)
        schur["bytes_per_site"] = 928
        schur["form"] = "Dhat = M_o - H_oe M_e^-1 H_eo, FP32, 8-real links, two half-lattice kernels"
        dsl_large = {"lattice": list(dl), "f32_us": round(ms_l * 1e3, 2), "f32_gbs": round(gbs_l, 1),
                     "f32_frac_measured_peak": round(gbs_l / peak, 3), "f32_frac_nominal_8tbs": round(gbs_l / 8000.0, 3),
                     "f16_storage": "spinors, links and clover in FP16 fixed point (348 B per site)",
                     "f16_us": round(ms_h * 1e3, 2), "f16_gbs": round(gbs_h, 1),
                     "f16_frac_measured_peak": round(gbs_h / peak, 3), "schur_f32": schur}
        cl.close()

    line = {
        # replicas: every rank solves its own system in each step, so the whole job finishes one
        # solve per t_step / world seconds
        "metric": METRIC, "value": round(t_step / world, 6), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.fine == "f32" else "f32+f16",
        "data": "synthetic",
        "config": workload_config(w, kappa, kinfo, args, world),
        "iterations": iters[-1], "refinements": stats["refinements"], "coarse_iterations": stats["coarse_iterations"],
        "true_residual": true_res, "setup_s": round(setup_s, 3),
        "autotune_coarse_ms": None if autotune_ms is None else round(autotune_ms, 4), "graphs": graphs,
        "fp64_solve_s": round(fp64_s, 4), "fp64_iterations": st64["iterations"],
        "batched": batched,
        "batched_three_level_24x24x24x48": config3,
        "speedup_vs_fp64": {"mixed_single": round(fp64_s / t_step, 2),
                            "mixed_batched_per_rhs": round(fp64_s / batched["s_per_rhs"], 2) if batched else None},
        "cg_fp64": cg,
        "cg_eo_fp64": cg_eo,
        "speedup_vs_cg": {"vs_cg": round(cg["s"] / t_step, 1) if cg else None,
                          "vs_cg_eo": round(cg_eo["s"] / t_step, 1) if cg_eo else None},
        "shifted_solves": shifts,
        "dslash_f32": {"us": round(dsl_ms * 1e3, 2), "gbs": round(dsl_gbs, 1), "frac_measured_peak": round(dsl_gbs / peak, 3),
                       "frac_nominal_8tbs": round(dsl_gbs / 8000.0, 3)},
        "dslash_f32_large": dsl_large,
        "kernels": kernels,
        "roofline": roof,
        "e2e": {"value": round(e2e_s / world, 6), "unit": "s", "h2d_bytes_per_step": int(b_host.nbytes),
                "d2h_bytes_per_step": int(b_host.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, kappa, float(np.mean(iters)), gpu_small_solve(tmg, local))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def workload_config(w, kappa, kinfo, args, world):
    """The workload description both arms print (the same dict for the same arguments)."""
    return {"workload": w["name"], "lattice": list(w["dims"]), "kappa": kappa,
            "kappa_source": kinfo.get("source"), "sigma_min_DW": kinfo.get("sigma_min"),
            "sigma_min_lattice": kinfo.get("sigma_lattice"), "sigma_target": w["sigma_target"], "csw": w["csw"],
            "mu": w["mu"], "levels": 2, "sap_block": list(w["block"]), "aggregate": list(w["block"]), "nv": w["nv"], "sap_mr": w.get("sap_mr", 4),
            "coarse_m": w.get("coarse_m", 30), "coarse_eo": bool(w.get("coarse_eo", 0)),
            "batched_coarse_m": w.get("batched_coarse_m", w.get("coarse_m", 30)),
            "fine_precision": args.fine, "tol": w["tol"], "rhs": 1, "rhs_per_step": world, "tune": args.tune,
            "l2": "flushed (512 MB write) between steps", "parallelism": "replicas" if world > 1 else "single"}


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks of the default process group (x itself for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def d_equivalents_per_outer_iteration(k=3, n_mr=4):
    """Fine-operator applications (D-equivalents) in one outer FGMRES iteration of the two-level
    method: the cycle's k SAP sweeps (two colours, each a residual on half the lattice and n_mr
    block-operator applications) and the outer operator application; P, P^dag and the coarse solve
    are counted as one more D-equivalent."""
    return k * (1 + n_mr) + 1 + 1


def oracle_d_apply(w, kappa, reps=2):
    """Seconds per FP64 application of D(mu) by the oracle on the workload's own lattice (measured)."""
    from oracle import dirac
    from synth import fields
    U = fields.gauge_field(w["dims"], w["eps"], w["seed"])
    p = dirac.Params(kappa=kappa, csw=w["csw"], mu=w["mu"], tbc=-1)
    C = dirac.clover_term(U, p.csw)
    x = fields.gaussian_spinor(w["dims"], w.get("rhs_seed", 4))
    dirac.apply_D(U, x, p, clover=C)
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        dirac.apply_D(U, x, p, clover=C)
        t.append(time.perf_counter() - t0)
    return min(t)


def oracle_small_solve():
    """The oracle's whole two-level DD-alpha-AMG solve of the 8^4 FP64 workload to 1e-10 (setup
    untimed, solve timed end to end): the configuration the oracle finishes in seconds."""
    from oracle import dirac, mg
    from synth import fields
    name = "tm_clover_8x8x8x8_fp64_2lvl"
    w1 = workloads.WORKLOADS[name]
    k1, _ = workloads.kappa(name)
    U = fields.gauge_field(w1["dims"], w1["eps"], w1["seed"])
    p = dirac.Params(kappa=k1, csw=w1["csw"], mu=w1["mu"], tbc=-1)
    H = mg.Hierarchy(U, p, mg.MGParams(block=w1["block"], agg=w1["block"], nv=w1["nv"], restart=w1["restart"]))
    H.setup(fields.gaussian_spinor(w1["dims"], w1["seed"] + 100, n=w1["nv"]))
    b = fields.gaussian_spinor(w1["dims"], w1["rhs_seed"])
    t0 = time.perf_counter()
    x, it, res = H.solve(b, tol=1e-10)
    return {"workload": name, "s": round(time.perf_counter() - t0, 3), "iterations": it, "true_residual": res}


def gpu_small_solve(tmg, local):
    """The same 8^4 FP64 two-level solve on the GPU (setup untimed), for a like-for-like ratio."""
    import torch
    from synth import fields
    name = "tm_clover_8x8x8x8_fp64_2lvl"
    w1 = workloads.WORKLOADS[name]
    k1, _ = workloads.kappa(name)
    ctx = tmg.Context(w1["dims"], w1["block"], device=local)
    ctx.set_params(k1, w1["csw"], w1["mu"])
    ctx.load_gauge(fields.gauge_field(w1["dims"], w1["eps"], w1["seed"]), -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.restart = w1["nv"], w1["restart"]
    prm.prec_fine, prm.prec_coarse = tmg.PREC_F64, tmg.PREC_F64
    ctx.setup(fields.gaussian_spinor(w1["dims"], w1["seed"] + 100, n=w1["nv"]), prm)
    b = torch.from_numpy(fields.gaussian_spinor(w1["dims"], w1["rhs_seed"])).cuda(local)
    x = torch.empty_like(b)
    ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_F64, out=x)
    t = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_F64, out=x)
        torch.cuda.synchronize()
        t.append(time.perf_counter() - t0)
    ctx.close()
    return {"s": round(min(t), 5), "iterations": st["iterations"]}


def cpu_baseline(w, kappa, gpu_iters, gpu_small=None):
    """The oracle as it stands on the host cores: (1) its whole FP64 two-level solve of the 8^4
    workload, timed end to end (the value: seconds per solve, like the metric, on the configuration
    the oracle finishes); (2) its FP64 operator application on the timed workload's own lattice,
    timed; (3) a separately labelled estimate for the timed workload, (2) times the D-equivalents of
    the GPU solve's outer iterations."""
    cores = len(os.sched_getaffinity(0))
    small = oracle_small_solve()
    t_d = oracle_d_apply(w, kappa)
    per_it = d_equivalents_per_outer_iteration()
    out = {"value": small["s"], "unit": "s", "cores": cores, "kind": "oracle",
           "sample": f"whole FP64 two-level solve of {small['workload']} to 1e-10 ({small['iterations']} outer "
                     f"iterations, setup untimed); numpy FP64 (elementwise work on one thread)",
           "oracle_small_solve": small,
           "oracle_d_apply_s": {"lattice": list(w["dims"]), "s": round(t_d, 3)},
           "estimate_timed_workload_s": {"value": round(t_d * per_it * gpu_iters, 2),
                                         "how": f"oracle D application on {'x'.join(map(str, w['dims']))} x "
                                                f"{per_it} D-equivalents per outer iteration x {gpu_iters:.0f} outer "
                                                f"iterations of the GPU solve (an estimate, not a run)"}}
    if gpu_small:
        out["gpu_same_small_solve"] = gpu_small
        out["small_solve_ratio_cpu_over_gpu"] = round(small["s"] / max(gpu_small["s"], 1e-9), 1)
    return out


def run_reference(args):
    """The oracle arm: each step is a bounded sample of the timed workload, the oracle's FP64
    application of D(mu) on the full lattice; the line's value converts it to seconds per solve
    with the D-equivalents of one outer iteration and the outer iteration count given by
    --ref-outer-iterations (the GPU solve's count; an estimate, labelled as such)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    kappa, kinfo = workload_kappa(w)
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_d_apply(w, kappa, reps=1)
        if i >= args.warmup:
            times.append(t)
    t_d = sum(times) / len(times)
    per_it = d_equivalents_per_outer_iteration()
    v = round(t_d * per_it * args.ref_outer_iterations, 3)
    sample = (f"per step one FP64 oracle application of D(mu) on the full {'x'.join(map(str, w['dims']))} lattice "
              f"({t_d:.3f} s); value = that x {per_it} D-equivalents per outer iteration x "
              f"{args.ref_outer_iterations} outer iterations (estimate)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t_d, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, kappa, kinfo, args, 1),
            "cpu_baseline": {"kind": "oracle", "cores": len(os.sched_getaffinity(0)), "sample": sample, "value": v,
                             "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fine", default="f32", choices=["f32", "f16"])
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-large-dslash", action="store_true")
    ap.add_argument("--batch", type=int, default=12, help="right-hand sides of the batched solve (0: skip)")
    ap.add_argument("--no-config3", dest="config3", action="store_false",
                    help="skip the 24^3 x 48 three-level batched comparison")
    ap.add_argument("--cg-maxiter", type=int, default=50000)
    ap.add_argument("--shifts", type=int, default=8, help="shifted systems solved with and without Taylor guesses (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-outer-iterations", type=int, default=14,
                    help="outer iterations the reference arm's per-solve estimate assumes")
    ap.add_argument("--ncu-solve", action="store_true", help="profile one solve only (for ncu)")
    ap.add_argument("--ncu-batched", action="store_true", help="profile one batched solve only (for ncu)")
    ap.add_argument("--tune", action="append", default=[], help="launch-shape knob key=value (tmg_tune)")
    ap.add_argument("--kernel-case", choices=["dslash", "sap", "coarse_tc", "schur"], default=None,
                    help="run one kernel class on a 24^3 x 48 lattice (for ncu --set full)")
    args = ap.parse_args()
    if args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
