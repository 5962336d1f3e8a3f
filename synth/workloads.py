"""The five synthetic workloads (lattice, field recipe, operator and multigrid parameters, right-hand
sides) shared by bench.py and the full-size tests.  Data only: no arithmetic of the method.

kappa comes from ``synth/kappa.json``, which the oracle's kappa search writes
(``python -m oracle.kappa_search``); a workload without a search record uses the provisional
m0 = -0.4 and says so.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))

PROVISIONAL_M0 = -0.4

WORKLOADS = {
    # plain method, FP64: CG on D D^dag against 2-level DD-alpha-AMG
    "tm_clover_8x8x8x8_fp64_2lvl": dict(
        dims=(8, 8, 8, 8), eps=0.4, seed=1, csw=1.0, mu=0.01, sigma_target=1e-3, block=(4, 4, 4, 4), nv=8,
        restart=10, rhs_seed=2, levels=2),
    # mixed-precision fine level with FP64 refinement (the timed workload)
    "tm_clover_16x16x16x32_mixed_2lvl": dict(
        dims=(16, 16, 16, 32), eps=0.35, seed=3, csw=1.5, mu=0.003, sigma_target=5e-4, block=(4, 4, 4, 4), nv=16,
        restart=10, rhs_seed=4, setup_seed=103, levels=2, sap_mr=6, coarse_eo=1, coarse_m=15,
        batched_coarse_m=30),
    # batched: 12 point sources + 8 shifted pseudofermion systems, three levels
    "tm_clover_24x24x24x48_batched_3lvl": dict(
        dims=(24, 24, 24, 48), eps=0.3, seed=4, csw=1.6, mu=0.002, sigma_target=5e-4, block=(4, 4, 4, 4), nv=24,
        agg2=(2, 2, 2, 2), nv2=32, restart=10, phi_seed=1004, n_shifts=8, levels=3,
        smooth_m=4, k_rtol=0.2, coarse_m2=20),
    # pseudofermion action and force
    "tm_clover_16x16x16x16_force": dict(
        dims=(16, 16, 16, 16), eps=0.3, seed=5, csw=1.0, mu=0.005, sigma_target=1e-3, block=(4, 4, 4, 4), nv=16,
        restart=10, phi_seed=6, levels=2),
    # non-degenerate doublet (Eq. 2), three levels
    "nd_clover_48x48x48x96_3lvl": dict(
        dims=(48, 48, 48, 96), eps=0.3, seed=6, csw=1.7, mu=0.0, mubar=0.12, epsbar=0.13, sigma_target=2e-4,
        block=(4, 4, 4, 4), nv=24, agg2=(2, 2, 2, 2), nv2=24, restart=10, rhs_seeds=tuple(range(7, 15)), levels=3),
}


def level2_params(w, q):
    """Copy a three-level workload's K-cycle parameters (smoother steps, K-cycle residual target,
    level-2 GMRES steps) into a level-2 parameter struct; the others keep their defaults."""
    q.agg[:] = w["agg2"]
    q.nv = w["nv2"]
    q.smooth_m = w.get("smooth_m", q.smooth_m)
    q.k_rtol = w.get("k_rtol", q.k_rtol)
    q.coarse_m = w.get("coarse_m2", q.coarse_m)
    return q


def shifts(n):
    """Multi-shift pseudofermion shifts sigma_k = 10^(-5 + 4 k / (n - 1)), log-spaced 1e-5 .. 1e-1."""
    return [10.0 ** (-5.0 + 4.0 * k / (n - 1)) for k in range(n)]


def kappa(name):
    """(kappa, record) of a workload; the record's "source" says where kappa came from."""
    with open(os.path.join(HERE, "kappa.json")) as f:
        table = json.load(f)
    if name in table:
        e = table[name]
        return e["kappa"], e
    m0 = PROVISIONAL_M0
    return 1.0 / (2.0 * (m0 + 4.0)), {"m0": m0, "source": f"provisional m0 = {m0} (no search record)"}
