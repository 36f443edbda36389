"""Halfway bounce-back walls through the C ABI against the oracle: random obstacle fields,
moving walls, every collision that supports walls, FP64 / FP32 / half storage; plus the
exact Poiseuille profile and mass conservation in a closed box on the GPU."""
import math

import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


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


CASES = [("D2Q9", (9, 7, 1), "bgk", True, False), ("D2Q9", (8, 6, 1), "regularized", False, True),
         ("D2Q9", (33, 5, 1), "trt", True, True), ("D2Q9", (10, 6, 1), "kbc", False, False),
         ("D2Q9", (7, 8, 1), "mrt", False, True), ("D3Q19", (5, 4, 3), "bgk", True, True),
         ("D3Q19", (6, 5, 3), "trt", False, False), ("D3Q27", (4, 5, 3), "regularized", True, False),
         ("D3Q27", (5, 4, 4), "kbc", False, True), ("D2Q9", (9, 7, 1), "none", False, True)]


@pytest.mark.parametrize("name,dims,coll,forced,moving", CASES)
def test_fp64_matches_oracle(name, dims, coll, forced, moving):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    mask = lbinputs.random_solid_mask(dims, seed=17, fraction=0.25)
    f0 = near_eq(name, dims, seed=18)
    F = lbinputs.random_field((d, N), seed=19, amp=1e-3) if forced else None
    wall_u = lbinputs.random_field((d, N), seed=20, amp=0.02) * mask if moving else None
    lat = L(name, dims, 0.64, coll, storage="f64")
    if forced:
        lat.set_force(F)
    lat.set_populations(f0)
    lat.set_solid(mask, wall_u)
    lat.step(1)
    ref1 = oracle.step_walls(name, dims, 0.64, coll, f0, mask, nsteps=1, F=F, wall_u=wall_u)
    assert werr(gpu_pops(lat), ref1, w) <= 1e-12
    lat.step(9)
    ref10 = oracle.step_walls(name, dims, 0.64, coll, ref1, mask, nsteps=9, F=F, wall_u=wall_u)
    assert werr(gpu_pops(lat), ref10, w) <= 1e-12
    # moments and sums of the walled state (solid nodes: rho = 1, u = F/2)
    r_o, u_o = oracle.moments(name, dims, ref10, F=F)
    r_g, u_g = lat.moments(torch.float64, "cpu")
    np.testing.assert_allclose(r_g.numpy(), r_o, rtol=0, atol=1e-13)
    np.testing.assert_allclose(u_g.numpy(), u_o, rtol=0, atol=1e-14)
    np.testing.assert_allclose(lat.reduce(), oracle.reduce(name, dims, ref10, F=F), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f16", 0.0)])
def test_changing_and_removing_walls(storage, tol):
    # the exposed state carries over a change of geometry: solid nodes at rest, fluid nodes kept
    name, dims = "D2Q9", (8, 6, 1)
    d, c, w, _ = oracle.stencil(name)
    f0 = near_eq(name, dims, seed=21)
    m1 = lbinputs.random_solid_mask(dims, seed=22)
    m2 = lbinputs.random_solid_mask(dims, seed=25)
    lat = L(name, dims, 0.7, "bgk", storage=storage)
    lat.set_populations(f0)
    lat.set_solid(m1)
    lat.step(3)
    before = gpu_pops(lat)
    lat.set_solid(m2)
    after = gpu_pops(lat)
    keep = m2 == 0
    np.testing.assert_array_equal(after[:, keep], before[:, keep])
    np.testing.assert_array_equal(after[:, ~keep], np.repeat(w[:, None], int((~keep).sum()), axis=1))
    lat.step(2)
    lat.set_solid(None)
    lat.step(3)
    if storage == "f64":
        ref = oracle.step_walls(name, dims, 0.7, "bgk", f0, m1, nsteps=3)
        ref[:, ~keep] = w[:, None]
        ref = oracle.step_walls(name, dims, 0.7, "bgk", ref, m2, nsteps=2)
        ref = oracle.step(name, dims, 0.7, "bgk", ref, nsteps=3)
        assert werr(gpu_pops(lat), ref, w) <= tol


@pytest.mark.parametrize("coll,tau", [("bgk", 0.6), ("trt", 0.9)])
def test_fp32_100_steps_duct_with_cylinder(coll, tau):
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims = (64, 34, 1)
    N = oracle.n_nodes(dims)
    mask = lbinputs.duct_with_obstacle(dims, radius=5.0)
    F = np.zeros((2, N))
    F[0] = 2e-5
    f0 = oracle.init_eq(name, dims, np.ones(N), np.zeros((2, N)))
    lat = L(name, dims, tau, coll, storage="f32")
    lat.set_force(F)
    lat.set_populations(f0)
    lat.set_solid(mask)
    lat.step(100)
    ref = oracle.step_walls(name, dims, tau, coll, f0, mask, nsteps=100, F=F)
    assert werr(gpu_pops(lat), ref, w) <= 1e-5


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_half_storage_with_walls(storage, tol):
    name = "D3Q19"
    d, c, w, _ = oracle.stencil(name)
    dims = (16, 12, 10)
    N = oracle.n_nodes(dims)
    mask = lbinputs.duct_with_obstacle(dims, radius=2.5)
    rho, u = lbinputs.random_moments(dims, seed=23, u_amp=0.03)
    f0 = oracle.init_eq(name, dims, rho, u)
    lat = L(name, dims, 0.6, "bgk", storage=storage)
    lat.set_populations(f0)
    lat.set_solid(mask)
    lat.step(30)
    ref = oracle.step_walls(name, dims, 0.6, "bgk", f0, mask, nsteps=30)
    dev = np.max(np.abs(ref - w[:, None]) / w[:, None])
    assert werr(gpu_pops(lat), ref, w) <= tol * dev


def test_poiseuille_profile_on_the_gpu():
    # TRT with Lambda = 3/16 and halfway walls: the parabola is exact (FP64)
    H = 16
    name = "D2Q9"
    dims = (8, H + 2, 1)
    N = oracle.n_nodes(dims)
    m = np.zeros((H + 2, 8), dtype=np.uint8)
    m[0] = m[-1] = 1
    mask = m.reshape(-1)
    tau, Fx = 0.8, 1e-6
    F = np.zeros((2, N))
    F[0] = Fx
    lat = L(name, dims, tau, "trt", storage="f64")
    lat.set_relaxation([3.0 / 16.0])
    lat.set_force(F)
    lat.init_from_moments(np.ones(N), np.zeros((2, N)))
    lat.set_solid(mask)
    nu = CS2 * (tau - 0.5)
    lat.step(int(40.0 * H * H / (nu * math.pi ** 2)))
    _, u = lat.moments(torch.float64, "cpu")
    ux = u[0].numpy().reshape(H + 2, 8)[1:-1, 3]
    y = np.arange(1, H + 1, dtype=float)
    exact = Fx / (2.0 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.max(np.abs(ux - exact)) < 1e-9 * exact.max()


def test_closed_box_conserves_mass_fp32():
    name = "D3Q19"
    dims = (32, 32, 32)
    N = oracle.n_nodes(dims)
    m = np.ones((32, 32, 32), dtype=np.uint8)
    m[1:-1, 1:-1, 1:-1] = 0
    rho, u = lbinputs.random_moments(dims, seed=24, u_amp=0.03)
    lat = L(name, dims, 0.6, "bgk", storage="f32")
    lat.init_from_moments(rho, u)
    lat.set_solid(m.reshape(-1))
    lat.step(1)
    m0 = lat.reduce()[0]
    lat.step(1000)
    lat.check()
    assert abs(lat.reduce()[0] - m0) < 2e-6 * m0


def test_walls_argument_checks():
    from paper_2106_12929_gb300._lib import LBError
    mask = np.zeros(64, dtype=np.uint8)
    with pytest.raises(LBError):
        L("D2Q9", (8, 8, 1), 0.7, "bgk", storage="f32", layout="aa").set_solid(mask)
    with pytest.raises(LBError):
        L("D2Q9", (8, 8, 1), 0.7, "learned", storage="f32").set_solid(mask)
    with pytest.raises(LBError):
        L("D2Q9", (8, 8, 1), 0.7, "bgk", storage="f32", record_every=2).set_solid(mask)


# ------------------------------------------------------------------ walls in the vector kernels
SHAPE_CASES = [("D2Q9", (16, 6, 1)), ("D3Q19", (8, 5, 4)), ("D3Q27", (12, 4, 3))]


def _wall_colls(name):
    colls = [("bgk", True), ("regularized", False), ("trt", True)]
    if name != "D3Q19":
        colls.append(("kbc", False))
    if name == "D2Q9":
        colls.append(("mrt", False))
    return colls


@pytest.mark.parametrize("name,dims", SHAPE_CASES)
def test_two_nodes_per_thread_with_walls_fp64(name, dims):
    """Two nodes per thread with walls (a solid node inside a vector access keeps its slots for
    the reflections; the fluid one is stored alone), 30 % solid, moving walls: the oracle."""
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    mask = lbinputs.random_solid_mask(dims, seed=31, fraction=0.3)
    f0 = near_eq(name, dims, seed=32)
    F = lbinputs.random_field((d, N), seed=33, amp=1e-3)
    wall_u = lbinputs.random_field((d, N), seed=34, amp=0.02) * mask
    for coll, forced in _wall_colls(name):
        lat = L(name, dims, 0.64, coll, storage="f64", nodes_per_thread=2)
        if forced:
            lat.set_force(F)
        lat.set_populations(f0)
        lat.set_solid(mask, wall_u)
        lat.step(5)
        ref = oracle.step_walls(name, dims, 0.64, coll, f0, mask, nsteps=5, F=F if forced else None, wall_u=wall_u)
        assert werr(gpu_pops(lat), ref, w) <= 1e-12, coll


@pytest.mark.parametrize("name,dims", SHAPE_CASES)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_wall_launch_shapes_agree(name, dims, storage):
    """One, two and four nodes per thread with walls run the same per-node arithmetic: the
    states agree to the last bits of the arithmetic type (FP32 1e-6) or one quantisation step
    of the stored deviation (half, 1e-4), relative to w_i; half storage also tracks the oracle."""
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    mask = lbinputs.random_solid_mask(dims, seed=35, fraction=0.3)
    f0 = near_eq(name, dims, seed=36)
    F = lbinputs.random_field((d, N), seed=37, amp=1e-3)
    wall_u = lbinputs.random_field((d, N), seed=38, amp=0.02) * mask
    for coll, forced in _wall_colls(name):
        out = []
        for npt in (1, 2, 4):
            lat = L(name, dims, 0.64, coll, storage=storage, nodes_per_thread=npt)
            if forced:
                lat.set_force(F)
            lat.set_populations(f0)
            lat.set_solid(mask, wall_u)
            lat.step(4)
            out.append(gpu_pops(lat))
            lat.close()
        tol = 1e-6 if storage == "f32" else 1e-4
        for o in out[1:]:
            assert werr(o, out[0], w) <= tol, coll
        if storage != "f32":
            ref = oracle.step_walls(name, dims, 0.64, coll, f0, mask, nsteps=4, F=F if forced else None,
                                    wall_u=wall_u)
            dev = np.max(np.abs(ref - w[:, None]) / w[:, None])
            assert werr(out[2], ref, w) <= {"f16": 2e-3, "bf16": 2e-2}[storage] * dev, coll
