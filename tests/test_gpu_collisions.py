"""Parity of the TRT, KBC and fixed-rate MRT collisions (CUDA path through the C ABI)
with the FP64 oracle. Same error measure and bars as the BGK / regularized parity
tests: max over i, x of |f_gpu - f_oracle| / w_i; FP64 <= 1e-12 (1 and 10 steps);
FP32 <= 1e-5 after 100 steps; half storage relative to the stored deviation."""
import math

import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

# grids with odd and even nx, one and several blocks per row; the launch shape (nodes per
# thread) is forced by the tests' npt parameter
TINY = {"D2Q9": [(5, 4, 1), (6, 5, 1), (33, 5, 1), (2, 3, 1), (8, 3, 1)],
        "D3Q19": [(5, 4, 3), (6, 5, 3), (2, 3, 3)],
        "D3Q27": [(5, 4, 3), (4, 5, 3), (7, 6, 5), (2, 2, 3)]}

# (stencil, collision, parameters for lb_set_relaxation or None for the defaults, forced)
CASES = [("D2Q9", "trt", None, False), ("D2Q9", "trt", [3.0 / 16.0], True), ("D3Q19", "trt", [0.25], True),
         ("D3Q27", "trt", [1.0 / 12.0], False), ("D2Q9", "kbc", None, False), ("D3Q27", "kbc", None, False),
         ("D2Q9", "mrt", None, False), ("D2Q9", "mrt", [0.9, 1.3, 0.55], False)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_12929_gb300 import build
    build.build()
    oracle.build()


def L(*a, **k):
    from paper_2106_12929_gb300 import Lattice
    return Lattice(*a, **k)


def werr(a, b, w):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / w[:, None]))


def gpu_pops(lat):
    return lat.get_populations(torch.float64, "cpu").numpy()


def near_eq(name, dims, seed, eps=0.05):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    rho, u = lbinputs.random_moments(dims, seed=seed, u_amp=0.05)
    return oracle.init_eq(name, dims, rho, u) + eps * 0.1 * w[:, None] * lbinputs.random_field((len(w), N), seed + 1)


def make(name, dims, tau, coll, params, storage, layout="ab", npt=0):
    lat = L(name, dims, tau, coll, storage=storage, layout=layout, nodes_per_thread=npt)
    if params is not None:
        lat.set_relaxation(params)
    return lat


@pytest.mark.parametrize("name,coll,params,forced", CASES)
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("npt", [1, 2])
def test_fp64_matches_oracle(name, coll, params, forced, layout, npt):
    d, c, w, _ = oracle.stencil(name)
    for dims in TINY[name]:
        N = oracle.n_nodes(dims)
        f0 = near_eq(name, dims, seed=71)
        F = lbinputs.random_field((d, N), seed=72, amp=1e-3) if forced else None
        lat = make(name, dims, 0.62, coll, params, "f64", layout, npt)
        if forced:
            lat.set_force(F)
        lat.set_populations(f0)
        lat.step(1)
        ref1 = oracle.step(name, dims, 0.62, coll, f0, nsteps=1, F=F, params=params)
        assert werr(gpu_pops(lat), ref1, w) <= 1e-12, dims
        lat.step(9)
        ref10 = oracle.step(name, dims, 0.62, coll, ref1, nsteps=9, F=F, params=params)
        assert werr(gpu_pops(lat), ref10, w) <= 1e-12, dims
        lat.close()


@pytest.mark.parametrize("name,n,coll,params,tau", [
    ("D2Q9", 64, "trt", None, 0.8), ("D2Q9", 64, "kbc", None, 0.8), ("D2Q9", 64, "mrt", [0.7, 0.7, 1.1], 0.8),
    ("D2Q9", 64, "kbc", None, 0.52), ("D3Q19", 48, "trt", [3.0 / 16.0], None), ("D3Q27", 24, "kbc", None, 0.55),
    ("D3Q27", 24, "trt", None, 0.55)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("npt", [1, 2])
def test_fp32_100_steps_within_1e_5(name, n, coll, params, tau, layout, npt):
    d, c, w, _ = oracle.stencil(name)
    if name == "D2Q9":
        dims, rho, u = lbinputs.taylor_green_2d(n, u0=0.05)
    else:
        u0 = 0.1 / math.sqrt(3.0)
        dims, rho, u = lbinputs.taylor_green_3d(n, u0=u0)
        if tau is None:
            tau = lbinputs.tau_from_reynolds(1600.0, u0, n)
    lat = make(name, dims, tau, coll, params, "f32", layout, npt)
    lat.init_from_moments(rho, u)
    lat.step(100)
    ref = oracle.step(name, dims, tau, coll, oracle.init_eq(name, dims, rho, u), nsteps=100, params=params)
    assert werr(gpu_pops(lat), ref, w) <= 1e-5


@pytest.mark.parametrize("coll,params", [("trt", None), ("kbc", None), ("mrt", [0.9, 0.9, 1.2])])
@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("npt", [1, 4])
def test_half_storage_tracks_oracle(coll, params, storage, tol, npt):
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims, rho, u = lbinputs.taylor_green_2d(64, u0=0.05)
    lat = make(name, dims, 0.8, coll, params, storage, npt=npt)
    lat.init_from_moments(rho, u)
    lat.step(50)
    ref = oracle.step(name, dims, 0.8, coll, oracle.init_eq(name, dims, rho, u), nsteps=50, params=params)
    dev = np.max(np.abs(ref - w[:, None]) / w[:, None])
    assert werr(gpu_pops(lat), ref, w) <= tol * dev


@pytest.mark.parametrize("name,coll", [("D2Q9", "trt"), ("D3Q27", "kbc"), ("D2Q9", "mrt"), ("D3Q19", "trt")])
def test_aa_matches_ab_bit_exact(name, coll):
    dims = TINY[name][1]
    f0 = near_eq(name, dims, seed=81)
    for storage in ["f32", "f16"]:
        a = L(name, dims, 0.6, coll, storage=storage, layout="ab")
        b = L(name, dims, 0.6, coll, storage=storage, layout="aa")
        a.set_populations(f0)
        b.set_populations(f0)
        for _ in range(3):
            a.step(1)
            b.step(1)
            np.testing.assert_array_equal(gpu_pops(a), gpu_pops(b))


def test_new_relaxation_applies_to_later_steps():
    # lb_set_relaxation between runs of graph-replayed steps takes effect at once
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims = (16, 6, 1)
    f0 = near_eq(name, dims, seed=91)
    lat = L(name, dims, 0.7, "trt", storage="f64")
    lat.set_populations(f0)
    lat.step(4)
    lat.set_relaxation([0.1])
    lat.step(4)
    ref = oracle.step(name, dims, 0.7, "trt", f0, nsteps=4, params=[0.25])
    ref = oracle.step(name, dims, 0.7, "trt", ref, nsteps=4, params=[0.1])
    assert werr(gpu_pops(lat), ref, w) <= 1e-12


def test_relaxation_arguments_are_checked():
    from paper_2106_12929_gb300._lib import LBError
    lat = L("D2Q9", (8, 8, 1), 0.7, "trt", storage="f32")
    with pytest.raises(LBError):
        lat.set_relaxation([0.0])
    with pytest.raises(LBError):
        lat.set_relaxation([0.25, 0.25])
    m = L("D2Q9", (8, 8, 1), 0.7, "mrt", storage="f32")
    with pytest.raises(LBError):
        m.set_relaxation([0.5, 1.0, 1.0])
    k = L("D2Q9", (8, 8, 1), 0.7, "kbc", storage="f32")
    with pytest.raises(LBError):
        k.set_relaxation([1.0])
    with pytest.raises(LBError):
        k.set_force(np.zeros((2, 64)))
    with pytest.raises(LBError):
        m.set_force(np.zeros((2, 64)))
