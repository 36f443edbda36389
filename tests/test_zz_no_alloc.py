"""The allocation-free global sums (lb_reduce_noalloc) against lb_reduce.

lb_reduce_noalloc serves callers that cannot allocate device memory where they
need the sums (for instance when another framework's caching allocator owns the
device memory, or in a loop where a cudaMalloc/cudaFree would stall the device):
it takes a caller-owned population array and keeps its partial sums in a fixed
static device array of the library. This file is collected after the parity tests of the
hot path so that a run stopping at the first failure has already run them.
"""
import ctypes

import numpy as np
import pytest
import torch

import lbinputs

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2106_12929_gb300 import _lib, build
    build.build()
    return _lib


def _noalloc(stencil, dims, f, F=None):
    lib = _lib()
    lb = lib.load()
    mem = lib.MEM["device_f64"] if f.dtype == torch.float64 else lib.MEM["device_f32"]
    out = (ctypes.c_double * 6)()
    d = (ctypes.c_int64 * 3)(*dims)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lb.lb_reduce_noalloc(lib.STENCIL[stencil], d, f.data_ptr(), None if F is None else F.data_ptr(), mem, out,
                              ctypes.c_void_p(stream))
    return rc, np.array(list(out))


def _with_context(stencil, dims, f, F=None, storage="f64"):
    from paper_2106_12929_gb300 import Lattice
    lat = Lattice(stencil, dims, 0.7, "bgk", storage=storage)
    if F is not None:
        lat.set_force(F)
    lat.set_populations(f)
    r = lat.reduce()
    lat.close()
    return r


@pytest.mark.parametrize("stencil,dims,forced", [("D2Q9", (257, 129, 1), False), ("D3Q19", (33, 30, 17), True),
                                                 ("D3Q27", (16, 16, 16), False)])
def test_noalloc_matches_lb_reduce_on_two_calls(stencil, dims, forced):
    Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[stencil]
    d = 2 if stencil == "D2Q9" else 3
    N = int(np.prod(dims))
    for call, seed in enumerate((1, 2)):  # two calls in a row, different inputs
        f = torch.tensor(lbinputs.random_populations(np.full(Q, 1.0 / Q), N, seed=seed + 10), device="cuda")
        F = torch.tensor(lbinputs.random_field((d, N), seed + 20, amp=1e-3), device="cuda") if forced else None
        rc, got = _noalloc(stencil, dims, f, F)
        assert rc == 0, call
        ref = _with_context(stencil, dims, f, F)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
        # FP32 arrays: against lb_reduce of an FP32 context given the same values; the context
        # stores f - w in FP32 (its own rounding of the same numbers), so the two agree to FP32
        # rounding per node: 1e-6 relative, and 1e-9 N absolute for the near-cancelling momenta
        f32, F32 = f.float(), None if F is None else F.float()
        rc32, got32 = _noalloc(stencil, dims, f32, F32)
        assert rc32 == 0
        ref32 = _with_context(stencil, dims, f32, F32, storage="f32")
        np.testing.assert_allclose(got32, ref32, rtol=1e-6, atol=1e-9 * N)


def test_noalloc_rejects_oversized_grids_and_host_arrays():
    lib = _lib()
    lb = lib.load()
    f = torch.zeros(9 * 16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 6)()
    too_big = (ctypes.c_int64 * 3)(8192, 4097, 1)  # 33,562,624 nodes: beyond the fixed scratch capacity
    rc = lb.lb_reduce_noalloc(0, too_big, f.data_ptr(), None, lib.MEM["device_f64"], out, None)
    assert rc == 1
    assert b"33,554,432" in lb.lb_last_error()
    host = np.zeros(9 * 16)
    ok_dims = (ctypes.c_int64 * 3)(4, 4, 1)
    assert lb.lb_reduce_noalloc(0, ok_dims, host.ctypes.data, None, lib.MEM["host_f64"], out, None) == 1


@pytest.mark.parametrize("dims", [(2048, 1200, 1), (8192, 4096, 1)])
def test_noalloc_matches_lb_reduce_at_many_blocks_and_at_capacity(dims):
    """600 partial blocks (the final pass loops over more slots than it has threads) and exactly
    the 33,554,432-node capacity (all 8192 slots), FP32 D2Q9 populations made on the device."""
    N = int(np.prod(dims))
    w = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=torch.float32, device="cuda")
    for seed in (5, 6):  # two calls in a row
        gen = torch.Generator(device="cuda").manual_seed(seed)
        f = w[:, None] * (1.0 + 0.05 * torch.randn((9, N), generator=gen, device="cuda", dtype=torch.float32))
        rc, got = _noalloc("D2Q9", dims, f)
        assert rc == 0
        ref = _with_context("D2Q9", dims, f, storage="f32")  # holds f - w in FP32: see above
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * N)
        del f
    torch.cuda.empty_cache()


def test_noalloc_rejects_a_host_pointer_passed_as_device_memory():
    """A host array with a device memory code is refused before any launch (the kernel would
    otherwise read memory the GPU cannot address)."""
    lib = _lib()
    lb = lib.load()
    out = (ctypes.c_double * 6)()
    dims = (ctypes.c_int64 * 3)(4, 4, 1)
    host = np.full(9 * 16, 1.0 / 9.0)
    assert lb.lb_reduce_noalloc(0, dims, host.ctypes.data, None, lib.MEM["device_f64"], out, None) == 1
    assert b"device" in lb.lb_last_error()
    f = torch.full((9 * 16,), 1.0 / 9.0, dtype=torch.float64, device="cuda")
    assert lb.lb_reduce_noalloc(0, dims, f.data_ptr(), host.ctypes.data, lib.MEM["device_f64"], out, None) == 1
    rc = lb.lb_reduce_noalloc(0, dims, f.data_ptr(), None, lib.MEM["device_f64"], out, None)
    assert rc == 0 and out[0] == pytest.approx(16.0, rel=1e-15)
