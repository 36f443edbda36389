"""Host side of the slab partitioning, on the CPU: the exchange schedule over torch.distributed
(gloo, two and three ranks: every face buffer reaches the right neighbour's ghost buffer), the
FP64 all-reduce of the global sums and of a parameter gradient, and the layer bookkeeping."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2106_12929_gb300.slab import DistTransport, allreduce_gradient, normalise_sums
    t = DistTransport()
    # face buffers tagged with the sender and face; two rounds (the schedule is reused)
    got = []
    for rnd in range(2):
        send_lo = torch.full((5,), 1000.0 * rnd + 10 * rank + 1)
        send_hi = torch.full((5,), 1000.0 * rnd + 10 * rank + 2)
        recv_lo, recv_hi = torch.zeros(5), torch.zeros(5)
        t.exchange(send_lo, send_hi, recv_lo, recv_hi)
        got.append((float(recv_lo[0]), float(recv_hi[0])))
    sums = t.allreduce_sum(torch.tensor([1.0, rank, 2.0 * rank, 0.0, 4.0, 8.0], dtype=torch.float64))
    g = torch.full((793,), float(rank + 1), dtype=torch.float32)
    allreduce_gradient(g)
    out[rank] = (got, sums.tolist(), float(g[0]), float(g[-1]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_schedule_and_allreduces_over_gloo(world):
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        got, sums, g0, g1 = out[r]
        lo, hi = (r - 1) % world, (r + 1) % world
        for rnd, (rl, rh) in enumerate(got):
            assert rl == 1000.0 * rnd + 10 * lo + 2  # the lower neighbour's high face
            assert rh == 1000.0 * rnd + 10 * hi + 1  # the upper neighbour's low face
        assert sums == [float(world), sum(range(world)), 2.0 * sum(range(world)), 0.0, 4.0 * world, 8.0 * world]
        assert g0 == g1 == sum(range(1, world + 1))


def test_single_rank_transport_sends_to_itself():
    sys.path.insert(0, ROOT)
    from paper_2106_12929_gb300.slab import DistTransport
    t = DistTransport.__new__(DistTransport)
    t.world, t.rank = 1, 0
    send_lo, send_hi, recv_lo, recv_hi = torch.tensor([1.0]), torch.tensor([2.0]), torch.zeros(1), torch.zeros(1)
    t.exchange(send_lo, send_hi, recv_lo, recv_hi)
    assert float(recv_lo[0]) == 2.0 and float(recv_hi[0]) == 1.0


def test_layer_bookkeeping():
    sys.path.insert(0, ROOT)
    from paper_2106_12929_gb300.slab import interior, normalise_sums, slab_bounds, with_ghosts
    assert slab_bounds(20, 4, 3) == (15, 5)
    with pytest.raises(ValueError):
        slab_bounds(18, 4, 0)
    # a [2][N] field of a 3 x 2 x 6 grid (z slowest): rank 1 of 3 owns z = 2, 3
    z = np.repeat(np.arange(6), 3 * 2)
    a = np.stack([z, 10 * z]).astype(float)
    g = with_ghosts(a, 2, 2, 6, 3)
    assert g.shape == (2, 4 * 6) and list(np.unique(g[0])) == [1, 2, 3, 4]
    assert list(g[0].reshape(4, 6)[:, 0]) == [1, 2, 3, 4]
    np.testing.assert_array_equal(interior(g, 2), a[:, 2 * 6:4 * 6])
    # the periodic wrap at both ends
    assert list(with_ghosts(a, 0, 2, 6, 3)[0].reshape(4, 6)[:, 0]) == [5, 0, 1, 2]
    assert list(with_ghosts(a, 4, 2, 6, 3)[0].reshape(4, 6)[:, 0]) == [3, 4, 5, 0]
    t = torch.tensor(a)
    assert torch.equal(with_ghosts(t, 4, 2, 6, 3), torch.tensor(with_ghosts(a, 4, 2, 6, 3)))
    s = normalise_sums([10.0, 1.0, 2.0, 3.0, 8.0, 16.0], 4)
    assert list(s) == [10.0, 1.0, 2.0, 3.0, 1.0, 2.0]


def _fake_rollout(j, g):
    """Stand-in for one rollout + adjoint: adds an item-dependent gradient, returns its loss."""
    if g is not None:
        g += (j + 1) * torch.arange(793, dtype=torch.float32) / 793.0
    return float(j) ** 2


BATCH = [5, 2, 7, 0, 3]  # five rollouts: the ranks' shares differ in size


def _dp_rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2106_12929_gb300.training import rank_world, sharded_mean
    group = dist.group.WORLD
    calls = []
    g = torch.zeros(793, dtype=torch.float32)
    L = sharded_mean(lambda j, gr: calls.append(j) or _fake_rollout(j, gr), BATCH, group, g, device="cpu")
    Lv = sharded_mean(_fake_rollout, BATCH, group, device="cpu")  # evaluation: no gradient
    out[rank] = (rank_world(group), calls, L, Lv, g.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_data_parallel_batch_matches_one_process(world):
    """training.sharded_mean over gloo ranks: each rank runs only its share of the batch, and
    every rank ends with the one-process batch loss and summed parameter gradient."""
    sys.path.insert(0, ROOT)
    from paper_2106_12929_gb300.training import rank_world, sharded_mean
    assert rank_world(None) == (0, 1)
    g1 = torch.zeros(793, dtype=torch.float32)
    L1 = sharded_mean(_fake_rollout, BATCH, None, g1, device="cpu")
    assert L1 == np.mean([j * j for j in BATCH])
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_dp_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    seen = []
    for r in range(world):
        rw, calls, L, Lv, g = out[r]
        assert rw == (r, world)
        assert calls == BATCH[r::world]
        seen += calls
        assert L == pytest.approx(L1, rel=1e-15) and Lv == pytest.approx(L1, rel=1e-15)
        np.testing.assert_allclose(g, g1.numpy(), rtol=1e-6, atol=0)
    assert sorted(seen) == sorted(BATCH)  # every rollout ran exactly once
