"""Slab partitioning (the multi-GPU layout) on one GPU: slabs of a periodic grid, each in its
own context with a ghost layer at each end, exchanging the crossing populations by device
copies after every step, reproduce the whole grid's state bit for bit (same launch shape), and
their FP64 sums add up to the whole grid's."""
import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_12929_gb300 import build
    build.build()


CASES = [("D3Q19", (24, 16, 20), "bgk"), ("D2Q9", (40, 36, 1), "bgk"), ("D3Q27", (16, 12, 16), "regularized")]


@pytest.mark.parametrize("name,dims,coll", CASES)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("world", [2, 4])
def test_slabs_reproduce_the_whole_grid_bit_exactly(name, dims, coll, storage, world):
    from paper_2106_12929_gb300 import Lattice
    from paper_2106_12929_gb300.slab import LocalTransport, SlabLattice, interior, step_local
    d = 2 if name == "D2Q9" else 3
    rho, u = lbinputs.random_moments(dims, seed=5, u_amp=0.05)
    tau = 0.6
    whole = Lattice(name, dims, tau, coll, storage=storage, nodes_per_thread=1, graphs=False)
    whole.init_from_moments(rho, u)
    hub = LocalTransport(world)
    slabs = [SlabLattice(name, dims, tau, coll, hub.endpoint(r), storage=storage, nodes_per_thread=1)
             for r in range(world)]
    for sl in slabs:
        sl.init_from_moments(rho, u)
    Q = oracle.stencil(name)[2].size
    for n in range(10):
        whole.step(1)
        step_local(slabs, 1)
        ref = whole.get_populations(torch.float64, "cpu").numpy().reshape(Q, dims[d - 1], -1)
        got = np.concatenate([sl.get_populations(torch.float64, "cpu").numpy().reshape(Q, sl.count, -1)
                              for sl in slabs], axis=1)
        np.testing.assert_array_equal(got, ref, err_msg=f"step {n + 1}")
    # the slabs' FP64 sums add up to the whole grid's
    s = sum(sl.local_sums() for sl in slabs)
    from paper_2106_12929_gb300.slab import normalise_sums
    np.testing.assert_allclose(normalise_sums(s, int(np.prod(dims))), whole.reduce(), rtol=1e-12, atol=1e-13)
    for sl in slabs:
        sl.close()
    whole.close()


def test_three_slabs_and_a_force_free_flow_in_2d():
    """Three y-slabs of a 2D Taylor-Green vortex over 25 steps, FP32, the default launch shape
    of the slab contexts forced to the whole grid's."""
    from paper_2106_12929_gb300 import Lattice
    from paper_2106_12929_gb300.slab import LocalTransport, SlabLattice, step_local
    dims, rho, u = lbinputs.taylor_green_2d(48, u0=0.05)
    whole = Lattice("D2Q9", dims, 0.8, "bgk", storage="f32", nodes_per_thread=2, graphs=False)
    whole.init_from_moments(rho, u)
    hub = LocalTransport(3)
    slabs = [SlabLattice("D2Q9", dims, 0.8, "bgk", hub.endpoint(r), storage="f32", nodes_per_thread=2)
             for r in range(3)]
    for sl in slabs:
        sl.init_from_moments(rho, u)
    whole.step(25)
    step_local(slabs, 25)
    ref = whole.get_populations(torch.float64, "cpu").numpy()
    got = np.concatenate([sl.get_populations(torch.float64, "cpu").numpy() for sl in slabs], axis=1)
    np.testing.assert_array_equal(got, ref)
    for sl in slabs:
        sl.close()
    whole.close()


def test_halo_calls_reject_what_they_do_not_support():
    from paper_2106_12929_gb300 import Lattice, _lib
    lat = Lattice("D3Q19", (8, 8, 2), 0.6, "bgk", storage="f32")  # no interior layer
    buf = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    assert lat._lib.lb_halo_pack(lat.handle, 0, buf.data_ptr()) == 1
    lat.close()
    lat = Lattice("D3Q19", (8, 8, 6), 0.6, "bgk", storage="f32", layout="aa")
    assert lat._lib.lb_halo_pack(lat.handle, 1, buf.data_ptr()) == 6  # LB_ERR_UNSUPPORTED
    assert lat._lib.lb_halo_pack(lat.handle, 2, buf.data_ptr()) == 1
    lat.close()


def test_one_rank_over_nccl():
    """The torch.distributed transport on an NCCL group of one rank: the exchange (a local copy)
    keeps the slab equal to the whole grid, and the all-reduce of host sums goes through the
    device, as NCCL needs."""
    import os
    import socket

    import torch.distributed as dist
    from paper_2106_12929_gb300 import Lattice
    from paper_2106_12929_gb300.slab import DistTransport, SlabLattice
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        t = DistTransport()
        host = torch.tensor([1.0, 2.5, -3.0], dtype=torch.float64)
        assert t.allreduce_sum(host).tolist() == [1.0, 2.5, -3.0]
        dims = (24, 16, 20)
        rho, u = lbinputs.random_moments(dims, seed=6, u_amp=0.05)
        whole = Lattice("D3Q19", dims, 0.6, "bgk", storage="f32", nodes_per_thread=1, graphs=False)
        whole.init_from_moments(rho, u)
        slab = SlabLattice("D3Q19", dims, 0.6, "bgk", t, storage="f32", nodes_per_thread=1)
        slab.init_from_moments(rho, u)
        whole.step(5)
        slab.step(5)
        np.testing.assert_array_equal(slab.get_populations(torch.float64, "cpu").numpy(),
                                      whole.get_populations(torch.float64, "cpu").numpy())
        np.testing.assert_allclose(slab.reduce(), whole.reduce(), rtol=1e-12, atol=1e-13)
        slab.close()
        whole.close()
    finally:
        dist.destroy_process_group()
