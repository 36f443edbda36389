"""The multi-GPU path of bench.py runs independent replicas (the lattice Boltzmann step
needs no exchange between them): the job time is the maximum over ranks and the value
counts every rank's updates. Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, _ = bench.dist_info()
    assert (w, r) == (world, rank)
    seconds = [2.0, 3.0][rank]  # rank 1 is the slow replica
    lups, t = bench.job_throughput(1000, 10, seconds, world, device="cpu")
    out[rank] = (lups, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(2):
        lups, t = out[r]
        assert t == pytest.approx(3.0)
        assert lups == pytest.approx(2 * 1000 * 10 / 3.0)


def _rank_retry(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # only rank 0's first clock record is rejected; both ranks must take the region again
    records = [{"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown"] if rank == 0 else []},
               {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}]

    class _Sampler:
        def __init__(self, gpu_index):
            self.rec = records.pop(0)

        def wait_first_sample(self):
            pass

        def stop(self, window=None):
            return dict(self.rec)

    class _Lat:
        def launch_count(self):
            return 0

    bench.ClockSampler = _Sampler
    # the ranks' K-step regions take different times; the repeat count follows the slowest
    bench.time_steps = lambda lat, k, stream: [0.1, 0.3][rank]
    t, clocks, _ = bench.timed_region(_Lat(), 5, None, 0, world, device="cpu")
    out[rank] = (clocks["remeasured"], len(records), clocks["repeats"])
    dist.barrier()
    dist.destroy_process_group()


def test_a_rejected_clock_record_on_one_rank_retakes_the_region_on_all():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_retry, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    reps = max(3, -(-0.8 // 0.3))  # ceil(MIN_TIMED_SECONDS / slowest region), at least three
    assert out[0] == (True, 0, reps) and out[1] == (True, 0, reps)
