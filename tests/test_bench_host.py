"""Host-side pieces of bench.py's roofline line, on the CPU: the algorithmic bytes of the coarse
solve (the 5-block stencil of D_c and, for the odd-even reduced system, the even sites' inverse
blocks), and the DRAM traffic figure read from the committed ncu summary, which is used only while
the source it was taken from is unchanged."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_coarse_step_bytes_of_the_timed_workload():
    b = _bench()
    nc, nd = 512, 32                       # 16^3 x 32 with 4^4 aggregates, N_v = 16
    per_site = 5 * nd * nd * 8 + 2 * nd * 8
    assert per_site == 41472
    assert b.coarse_step_bytes(nc, nd) == nc * per_site
    # odd-even reduced system: the even sites' (A_ee + i mu G5_c)^-1 blocks once more per step
    assert b.coarse_step_bytes(nc, nd, eo=True) == nc * per_site + (nc // 2) * nd * nd * 8
    # twelve columns: the vectors scale, the stencil does not
    assert b.coarse_step_bytes(nc, nd, ncol=12) - b.coarse_step_bytes(nc, nd) == nc * 2 * 11 * nd * 8


def test_stored_traffic_matches_the_current_coarse_gmres_source():
    """The committed summary of the dominant kernel carries a traffic line for the current source:
    a changed k_coarse_gmres.cu without a new capture would leave the bench's traffic field empty."""
    b = _bench()
    t = b.stored_traffic("coarse_solve")
    assert t is not None
    assert 20e6 < t < 60e6                 # one launch reads the L2-resident stencil (~38 MB) once
    assert b.stored_traffic("no_such_kernel") is None
