"""bench.py under torchrun runs one independent replica per GPU (a single scene does not shard) and times the
job by the slowest rank: every rank's timed total is reduced with MAX after a barrier.  Checked with two
CPU ranks over gloo (127.0.0.1)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, local_values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    got = [bench.slowest_rank(v, device="cpu") for v in local_values[rank]]
    out.put((rank, got))
    dist.destroy_process_group()


def test_slowest_rank_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    local_values = {0: [120.0, 3.5], 1: [95.25, 4.75]}  # ms of the timed steps, e2e seconds
    procs = [ctx.Process(target=_rank, args=(r, 2, port, local_values, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [120.0, 4.75]


def _shard_rank(rank, world, port, n_items, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    mine = bench.shard_scenes(list(range(n_items)), dist.get_rank(), dist.get_world_size())
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, gathered))
    dist.destroy_process_group()


def test_batched_scenes_partition_across_two_gloo_ranks():
    """Independent scenes shard across ranks with no data-path collective: every scene on exactly one rank."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, 5, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = res[0]
    assert res[1] == parts
    assert sorted(parts[0] + parts[1]) == list(range(5)) and not set(parts[0]) & set(parts[1])
    assert abs(len(parts[0]) - len(parts[1])) <= 1


def test_timed_steps_span_the_trajectory():
    sys.path.insert(0, ROOT)
    import bench
    idx = bench.timed_indices(400, 5, 20, "trajectory")
    assert len(idx) == 20 and idx[0] == 5 and idx[-1] >= 380 and all(b > a for a, b in zip(idx, idx[1:]))
    assert bench.timed_indices(400, 5, 20, "consecutive") == list(range(5, 25))


def test_slowest_rank_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(42.5, device="cpu") == 42.5
