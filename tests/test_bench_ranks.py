"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2).

The hot path does not shard: with several GPUs every rank runs an
independent replica, and bench.py only aggregates timings (max over ranks)
and work (sum over ranks).  That aggregation, and the rule that only rank 0
runs the reference arm, are exercised here without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.reduce_max_sum(1.0 + rank, 100.0 * (rank + 1), world)
    bench.barrier(world)
    w, r, lr = bench.dist_env()
    dist.destroy_process_group()
    q.put((rank, t, u, w, r, lr))


def test_max_time_sum_units_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, w, r, lr in res:
        assert t == 2.0          # max over ranks of the timed span
        assert u == 300.0        # sum over ranks of the work
        assert (w, r, lr) == (world, rank, rank)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out == ""


def test_sweep_block_allocation():
    """Blocks of the several-problem launch: every problem at least one, all
    blocks used, the rest in proportion to the ratings."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import synth
    assert bench.sweep_blocks([5, 1, 1], 3) == [1, 1, 1]
    assert bench.sweep_blocks([100, 1], 152) == [150, 2]
    assert bench.sweep_blocks([1, 1, 1, 1], 8) == [2, 2, 2, 2]
    specs = synth.sweep_specs(64, seed=5)
    assert specs == synth.sweep_specs(64, seed=5)  # seeded
    nnz = [int(s["m"] * s["n"] * s["density"]) for s in specs]
    b = bench.sweep_blocks(nnz, 152)
    assert sum(b) == 152 and min(b) >= 1
    share = [x / sum(nnz) * 152 for x in nnz]
    assert all(abs(bi - si) < 1.0 or bi == 1 for bi, si in zip(b, share))
    for s in specs:
        assert 2000 <= s["m"] <= 200000 and 1000 <= s["n"] <= 50000
        assert 0.001 <= s["density"] <= 0.02
        assert s["k"] in (16, 32, 64, 128) and s["lam"] in (0.01, 0.05, 0.1, 0.5)

