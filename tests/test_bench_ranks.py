"""The bench's host logic on CPU: its multi-rank path (gloo, world size 2),
the size of its host-side oracle sample, and its clock record.

Instances are independent, so `bench.py --gpus N` runs replicas: each rank
solves its own seeded instances and the only collectives are the barrier and
the max over ranks of the timed region.  These tests run that host logic in
two processes on the gloo backend: disjoint instance seeds per rank, the max
over ranks seen identically by both, and the whole-job rate (every rank's
steps over the slowest rank's time)."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    seeds = [bench.step_seed(s, r) for s in range(16)]
    gathered = [None] * w
    dist.all_gather_object(gathered, seeds)
    # rank r's timed region took 1.5 + r seconds
    t = bench.max_over_ranks(1.5 + r, torch.device("cpu"))
    dist.barrier()
    out.put((r, w, lr, gathered, t, bench.job_rate(w, 10, t)))
    dist.destroy_process_group()


def test_two_ranks_solve_disjoint_instances_and_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, (rank, world, local, gathered, t, rate) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t == 2.5                      # the slower rank's time, on both
        assert rate == pytest.approx(2 * 10 / 2.5)
        s0, s1 = gathered
        assert len(set(s0)) == 16 and len(set(s1)) == 16
        assert not set(s0) & set(s1)         # disjoint instances
        assert s0[0] == 1                    # rank 0 starts from the canonical field


def test_single_process_needs_no_group():
    import torch
    import bench
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25
    assert bench.job_rate(1, 4, 2.0) == 2.0


def test_reference_sample_is_bounded_whatever_the_step_count():
    import bench
    assert bench.ref_chunk(20) == 15
    assert bench.ref_chunk(100) == 3
    assert bench.ref_chunk(1000) == 1                  # at least one per step
    assert bench.ref_chunk(0) == 300
    for k in (1, 7, 20, 64, 299):                      # about 300 iterations in all
        assert 300 <= k * bench.ref_chunk(k) < 300 + k


def test_batches_of_ranks_and_of_training_are_disjoint():
    import bench
    # a rank's test batch: 64 consecutive seeds; its training instances:
    # TRAIN_BATCHES x 64 consecutive seeds from the training base
    spans = sorted((bench.batch_seed(r, t), 64 * (bench.TRAIN_BATCHES if t else 1))
                   for r in range(8) for t in (False, True))
    assert len({a for a, _ in spans}) == 16
    assert all(a + n <= b for (a, n), (b, _) in zip(spans, spans[1:]))


def test_clock_summary_reads_the_timed_region_and_flags_throttling():
    import bench
    c = bench.ClockSampler(0)
    idle = ["345", "2070", "90.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    busy = ["2070", "2070", "1100.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["1800", "2070", "1300.0", "0x40", "Not Active", "Active", "Not Active", "Not Active"]
    c.rows = [idle, busy, busy, hot, ["garbage"]]
    c.start = 1  # the idle sample came before the timed region
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    # a region too short for a sample of its own: the last one before it
    c.rows, c.start = [idle, busy], 2
    assert c.summary()["samples"] == 1 and c.summary()["sm_mhz"] == 2070.0
