"""The N > 1 path of bench.py on CPU: the method does not shard (one problem
per GPU, replicas only), so the only multi-rank logic is the timing
aggregation (barrier, MAX of the per-rank times over ranks, units of all ranks
over that time) and the rule that only rank 0 runs the reference arm and
prints.  Two gloo ranks on 127.0.0.1."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds for 64 x 5 units
        rate, t = bench.job_rate(float(rank + 1), 64 * 5, world, dist, "cpu")
        q.put((rank, rate, t))
    finally:
        dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, rate, t in got:
        assert t == 2.0                       # the slowest rank's time on every rank
        assert rate == pytest.approx(64 * 5 * 2 / 2.0)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    rate, t = bench.job_rate(0.5, 100, 1, None, "cpu")
    assert (rate, t) == (200.0, 0.5)


def test_reference_arm_nonzero_rank_is_silent(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    out = io.StringIO()
    with redirect_stdout(out):
        bench.main()
    assert out.getvalue() == ""
