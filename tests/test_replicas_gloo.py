"""Host-side logic of the multi-GPU replica runs of bench.py, exercised with two gloo ranks on the
CPU: the step time is the maximum over the ranks, and the reference arm runs on rank 0 only."""
import contextlib
import importlib.util
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        got = bench.max_over_ranks(1.5 + rank, world)
        # the reference arm: every rank but 0 returns at once, printing nothing
        printed = ""
        if rank != 0:
            buf = io.StringIO()
            with contextlib.redirect_stdout(buf):
                bench.run_reference(None)
            printed = buf.getvalue()
        out.put((rank, got, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_step_time_and_keep_rank0_output():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(abs(v - 2.5) < 1e-15 for _, v, _ in res)
    assert res[1][2] == ""


def test_single_rank_is_identity():
    assert _bench().max_over_ranks(3.25, 1) == 3.25
