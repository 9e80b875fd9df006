"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own timing; the job's time is the slowest rank's and the rate counts
the work of all ranks.  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank, world)       # rank 1 is the slow one
        rate = bench.whole_job_rate(1000, 4, 10, t, world)
        dist.barrier()
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, t, rate in got:
        assert t == 2.0                                    # the slowest rank's time
        assert rate == 2 * 1000 * 4 * 10 / 2.0             # both ranks' work


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(131072, 1, 200, 0.4, 1) == 131072 * 200 / 0.4


def test_stored_accuracy_uses_only_matching_draws(monkeypatch):
    """bench.py's accuracy of the r = 49 workloads: the stored oracle values
    are used only for calls whose theta they hold and only when the data's
    fingerprint matches the one stored with them."""
    import numpy as np
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    import golden_values
    rng = np.random.default_rng(5)
    d = {"x": rng.random(50), "y": rng.random(50), "z": rng.standard_normal(50)}
    fp = (50, float(np.sum(d["x"])), float(np.sum(d["y"])), float(np.sum(d["z"])), float(np.sum(np.abs(d["z"]))))
    th = np.array([[1.0, 0.05, 0.01], [1.2, 0.06, 0.012]])[:, None, :]
    ll = np.array([[-10.0], [-12.0]])
    monkeypatch.setattr(golden_values, "golden", lambda name: [(np.array([1.2, 0.06, 0.012]), -12.5, 50, fp)])
    acc = bench.stored_accuracy("swaths", d, th, ll, 50, "mixed")
    assert acc["calls_checked"] == 1 and abs(acc["mixed"] - 0.5 / 50) < 1e-15
    other = (51,) + fp[1:]
    monkeypatch.setattr(golden_values, "golden", lambda name: [(np.array([1.2, 0.06, 0.012]), -12.5, 50, other)])
    assert bench.stored_accuracy("swaths", d, th, ll, 50, "mixed")["against"] is None
