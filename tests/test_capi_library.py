"""Host-side checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every
entry point declared in include/tmg.h, and rejects bad arguments without touching a device."""
import ctypes
import os
import re

import pytest

import paper_1710_06198_gb300 as tmg
from paper_1710_06198_gb300 import build as tmg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    tmg_build.build()
    return tmg.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tmg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(tmg._SIGS), "binding lacks a declared entry point"


def test_version_without_device(L):
    assert "sm_103a" in tmg.version()


def test_create_rejects_bad_geometry(L):
    h = ctypes.c_void_p()
    bad = [((8, 4, 4, 4), (4, 2, 2, 3)),    # block does not divide
           ((8, 4, 4, 6), (4, 2, 2, 2)),    # odd number of blocks in t
           ((4, 4, 4, 4), (4, 2, 2, 2)),    # a single block in x
           ((8, 8, 4, 4), (2, 2, 2, 2))]    # block volume not a multiple of 32
    for dims, block in bad:
        d = (ctypes.c_int * 4)(*dims)
        b = (ctypes.c_int * 4)(*block)
        assert L.tmg_create(ctypes.byref(h), d, b, 0, None) == -1
    assert L.tmg_create(None, None, None, 0, None) == -1


def test_null_context_calls_fail_cleanly(L):
    assert L.tmg_destroy(None) == -1
    assert L.tmg_load_gauge(None, None, 0, -1) == -1
    assert L.tmg_apply(None, 0, None, None, 1, None, 0, 0) == -1
    assert L.tmg_solve(None, None, None, 1, None, 1e-10, 0, 10, None, 0) == -1
    p = tmg.MGParams()
    assert L.tmg_mg_defaults(ctypes.byref(p)) == 0
    assert p.nv == 8 and p.sap_sweeps == 3 and p.restart == 10


def test_level2_defaults_and_null_context(L):
    q = tmg.Level2Params()
    assert L.tmg_level2_defaults(ctypes.byref(q)) == 0
    assert list(q.agg) == [2, 2, 2, 2] and q.nv == 8 and q.smooth_m == 3
    assert q.k_restart == 10 and abs(q.k_rtol - 0.1) < 1e-15 and q.coarse_m == 30
    assert L.tmg_level2_defaults(None) == -1
    assert L.tmg_setup_level2(None, ctypes.byref(q), None, 0) == -1
    assert L.tmg_kcycle(None, None, None, 0.0, 0, 0, 0) == -1
    assert L.tmg_kcycle_multi(None, None, None, 1, None, 0, 0) == -1
    assert L.tmg_coarse_solve_multi(None, None, None, 1, None, 0) == -1
    assert L.tmg_coarse_apply2(None, None, None, 0.0, 0, 0) == -1


def test_doublet_tuning_and_graph_entries_reject_null_context(L):
    assert L.tmg_sap_nd(None, None, None, 0, 0) == -1
    assert L.tmg_coarse_apply_nd(None, None, None, 0, 0) == -1
    assert L.tmg_coarse_solve_nd(None, None, None, 0, 0) == -1
    assert L.tmg_kcycle_nd(None, None, None, 0, 0, 0) == -1
    assert L.tmg_cycle_nd(None, None, None, 0) == -1
    assert L.tmg_autotune(None, None) == -1
    assert L.tmg_graph_count(None, None) == -1
    assert L.tmg_tune(None, b"cycle_graph", 1.0) == -1
    assert L.tmg_coarse_solve_noalloc(None, None, None, 0.0, 0) == -1


def test_check_links_accepts_su3_and_names_the_bad_link(L):
    """tmg_check_links (the host-side check behind tmg_load_gauge): the synthetic SU(3) fields pass;
    a link scaled by 1.001, one with a unit-modulus phase on the whole matrix (unitary but det != 1),
    and one with a NaN each fail, with the index of the bad link reported."""
    import numpy as np
    from synth import fields
    U = fields.gauge_field((4, 4, 4, 4), 0.4, 120)
    ok, w, _ = tmg.check_links(U)
    assert ok and w < 1e-12
    flat = U.reshape(-1, 3, 3)
    for k, spoil in ((17, lambda u: 1.001 * u), (203, lambda u: np.exp(0.3j) * u), (511, lambda u: u * np.nan)):
        V = flat.copy()
        V[k] = spoil(V[k])
        ok, w, i = tmg.check_links(V.reshape(U.shape))
        assert not ok and i == k and not (w <= 1e-8)
    h = ctypes.c_double()
    assert L.tmg_check_links(None, 4, ctypes.byref(h), None) != 0
