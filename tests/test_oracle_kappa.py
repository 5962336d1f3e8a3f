

def test_convergence_edge_walk_and_bisection(monkeypatch):
    """search_m0_mg keeps the most critical converging m0: walk in steps of 0.1, then bisect."""
    from oracle import kappa
    edge = -1.23
    monkeypatch.setattr(kappa, "mg_steps", lambda U, m0, *a, **k: 20 if m0 > edge else 51)
    log = []
    m0 = kappa.search_m0_mg(None, 1.0, 0.01, (4, 4, 4, 4), 8, None, None, log=log)
    assert -1.25 <= m0 <= -1.2 + 1e-12
    assert [m for m, _ in log][:3] == [0.0, -0.1, -0.2]
    assert all(n == 20 for m, n in log if m > edge) and all(n == 51 for m, n in log if m <= edge)
