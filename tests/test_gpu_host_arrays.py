"""Host arrays through the C ABI: page-locked host arrays are read and written in place by the
kernels, pageable ones go through a staging buffer; both must give identical results, and an
output the adjoint accumulates into (grad_F) keeps its prior contents in either kind of memory."""
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
    oracle.build()


def L(*a, **k):
    from paper_2106_12929_gb300 import Lattice
    return Lattice(*a, **k)


def host(x, pinned):
    t = torch.tensor(np.ascontiguousarray(x))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_page_locked_and_pageable_host_arrays_agree(dtype):
    dims = (96, 40, 1)
    N = dims[0] * dims[1]
    rho = 1.0 + 0.01 * lbinputs.random_field(N, seed=11)
    u = 0.03 * lbinputs.random_field((2, N), seed=12)
    outs = {}
    for pinned in (False, True):
        lat = L("D2Q9", dims, 0.6, "bgk", storage="f32")
        r_in, u_in = torch.tensor(rho, dtype=dtype), torch.tensor(u, dtype=dtype)
        if pinned:
            r_in, u_in = r_in.pin_memory(), u_in.pin_memory()
        assert r_in.is_pinned() == pinned and u_in.is_pinned() == pinned
        lat.init_from_moments(r_in, u_in)
        lat.step(7)
        r_out = torch.empty(N, dtype=dtype, pin_memory=pinned)
        u_out = torch.empty((2, N), dtype=dtype, pin_memory=pinned)
        lat.moments(out=(r_out, u_out))
        f = torch.empty((9, N), dtype=torch.float64, pin_memory=pinned)
        assert lat._lib.lb_get_populations(lat.handle, f.data_ptr(), 0) == 0  # LB_HOST_F64
        r_dev, u_dev = lat.moments(dtype, "cuda")
        outs[pinned] = (r_out.clone(), u_out.clone(), f.clone(), r_dev.cpu(), u_dev.cpu())
        lat.close()
    for a, b in zip(outs[False], outs[True]):
        assert torch.equal(a, b)
    # host outputs equal the device outputs of the same state
    assert torch.equal(outs[True][0], outs[True][3]) and torch.equal(outs[True][1], outs[True][4])


@pytest.mark.parametrize("pinned", [False, True])
def test_adjoint_adds_to_a_host_gradient_in_either_memory(pinned):
    dims = (32, 32, 1)
    N = 32 * 32
    _, rho, u = lbinputs.taylor_green_2d(32, u0=0.05)
    F = lbinputs.smooth_force(dims, 1e-4, seed=1)
    lamT = lbinputs.random_field((9, N), seed=2)
    lat = L("D2Q9", dims, 0.8, "bgk", storage="f64", record_every=2)
    lat.set_force(F)
    lat.init_from_moments(rho, u)
    lat.step(4)
    g0 = torch.zeros((2, N), dtype=torch.float64)
    lam_h = host(lamT, pinned)
    lat.step_adjoint(lam_h, 4, grad_F=g0)
    lat.init_from_moments(rho, u)
    lat.step(4)
    g1 = host(np.full((2, N), 0.25), pinned)
    lat.step_adjoint(lam_h, 4, grad_F=g1)
    lat.close()
    assert torch.allclose(g1 - 0.25, g0, rtol=0, atol=1e-15)
    assert float(g0.abs().max()) > 0
