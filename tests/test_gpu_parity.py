"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error measure for populations: max over i, x of |f_gpu - f_oracle| / w_i (the
populations scale with w_i). Bars: streaming (collision "none") bit-exact in
FP64/FP32; FP64 collisions <= 1e-12; FP32 <= 1e-5 after 100 steps.
"""
import math

import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

STENCILS = ["D2Q9", "D3Q19", "D3Q27"]
# odd and even nx, ragged rows; the stream-collide launch shape is forced by the npt
# parameter where a test has one (the default picks one node per thread on grids this small)
TINY = {"D2Q9": [(5, 4, 1), (6, 5, 1), (33, 5, 1), (2, 3, 1), (258, 3, 1)],
        "D3Q19": [(5, 4, 3), (6, 5, 3), (7, 6, 5), (2, 3, 3)],
        "D3Q27": [(5, 4, 3), (4, 5, 3), (7, 6, 5), (2, 2, 3)]}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_12929_gb300 import build
    build.build()
    oracle.build()


def L(*a, **k):
    from paper_2106_12929_gb300 import Lattice
    return Lattice(*a, **k)


def werr(a, b, w):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / w[:, None]))


def gpu_pops(lat):
    return lat.get_populations(torch.float64, "cpu").numpy()


def near_eq(name, dims, seed, eps=0.05):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    rho, u = lbinputs.random_moments(dims, seed=seed, u_amp=0.05)
    return oracle.init_eq(name, dims, rho, u) + eps * 0.1 * w[:, None] * lbinputs.random_field((len(w), N), seed + 1)


# ------------------------------------------------------------------ streaming
@pytest.mark.parametrize("name", STENCILS)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_streaming_bit_exact(name, storage, layout):
    d, c, w, _ = oracle.stencil(name)
    for dims in TINY[name]:
        N = oracle.n_nodes(dims)
        f0 = lbinputs.random_populations(w, N, seed=3)
        if storage == "f32":
            # FP32 storage holds f - w: values whose deviation is an FP32 number (f = w + that
            # deviation is then exact in FP64) move through it unchanged
            f0 = w[:, None] + (f0 - w[:, None]).astype(np.float32).astype(np.float64)
        lat = L(name, dims, 0.8, "none", storage=storage, layout=layout)
        lat.set_populations(f0)
        np.testing.assert_array_equal(gpu_pops(lat), f0)
        for n in (1, 2, 3):
            lat.step(1)
            np.testing.assert_array_equal(gpu_pops(lat), oracle.step(name, dims, 0.8, "none", f0, nsteps=n))
        lat.close()


@pytest.mark.parametrize("name", STENCILS)
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_streaming_half_storage_moves_values_unchanged(name, storage):
    d, c, w, _ = oracle.stencil(name)
    dims = TINY[name][0]
    N = oracle.n_nodes(dims)
    lat = L(name, dims, 0.8, "none", storage=storage)
    lat.set_populations(lbinputs.random_populations(w, N, seed=4))
    q0 = gpu_pops(lat)  # the quantised state
    lat.step(3)
    # streaming moves the stored values untouched
    np.testing.assert_array_equal(gpu_pops(lat), oracle.step(name, dims, 0.8, "none", q0, nsteps=3))


# ------------------------------------------------------------------ FP64 collision parity
@pytest.mark.parametrize("name", STENCILS)
@pytest.mark.parametrize("coll", ["bgk", "regularized"])
@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("npt", [1, 2])
def test_collision_fp64_matches_oracle(name, coll, forced, layout, npt):
    d, c, w, _ = oracle.stencil(name)
    for dims in TINY[name][:4]:
        N = oracle.n_nodes(dims)
        f0 = near_eq(name, dims, seed=11)
        F = lbinputs.random_field((d, N), seed=12, amp=1e-3) if forced else None
        lat = L(name, dims, 0.67, coll, storage="f64", layout=layout, nodes_per_thread=npt)
        if forced:
            lat.set_force(F)
        lat.set_populations(f0)
        lat.step(1)
        ref1 = oracle.step(name, dims, 0.67, coll, f0, nsteps=1, F=F)
        assert werr(gpu_pops(lat), ref1, w) <= 1e-12
        lat.step(9)
        ref10 = oracle.step(name, dims, 0.67, coll, ref1, nsteps=9, F=F)
        assert werr(gpu_pops(lat), ref10, w) <= 1e-12
        lat.close()


@pytest.mark.parametrize("name", STENCILS)
@pytest.mark.parametrize("which", [0, 1, 3])
def test_aa_matches_ab_bit_exact(name, which):
    d, c, w, _ = oracle.stencil(name)
    dims = TINY[name][which]
    f0 = near_eq(name, dims, seed=21)
    for storage in ["f64", "f32", "f16"]:
        a = L(name, dims, 0.6, "bgk", storage=storage, layout="ab")
        b = L(name, dims, 0.6, "bgk", storage=storage, layout="aa")
        a.set_populations(f0)
        b.set_populations(f0)
        for _ in range(4):
            a.step(1)
            b.step(1)
            np.testing.assert_array_equal(gpu_pops(a), gpu_pops(b))
            ra, ua = a.moments()
            rb, ub = b.moments()
            assert torch.equal(ra, rb) and torch.equal(ua, ub)


# ------------------------------------------------------------------ FP32, 100 steps
@pytest.mark.parametrize("name,n,coll,tau", [("D2Q9", 64, "bgk", 0.8), ("D3Q19", 64, "bgk", None),
                                             ("D3Q27", 24, "regularized", 0.55)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("npt", [1, 2])
def test_fp32_100_steps_within_1e_5(name, n, coll, tau, layout, npt):
    d, c, w, _ = oracle.stencil(name)
    if name == "D2Q9":
        dims, rho, u = lbinputs.taylor_green_2d(n, u0=0.05)
    else:
        u0 = 0.1 / math.sqrt(3.0)
        dims, rho, u = lbinputs.taylor_green_3d(n, u0=u0)
        if tau is None:
            tau = lbinputs.tau_from_reynolds(1600.0, u0, n)
    lat = L(name, dims, tau, coll, storage="f32", layout=layout, nodes_per_thread=npt)
    lat.init_from_moments(rho, u)
    lat.step(100)
    ref = oracle.step(name, dims, tau, coll, oracle.init_eq(name, dims, rho, u), nsteps=100)
    assert werr(gpu_pops(lat), ref, w) <= 1e-5
    r_o, u_o = oracle.moments(name, dims, ref)
    r_g, u_g = lat.moments(torch.float64, "cpu")
    assert np.max(np.abs(r_g.numpy() - r_o)) <= 1e-5
    assert np.max(np.abs(u_g.numpy() - u_o)) <= 1e-5 * 0.1


# ------------------------------------------------------------------ moments and sums
@pytest.mark.parametrize("name", STENCILS)
@pytest.mark.parametrize("forced", [False, True])
def test_moments_and_reduce_fp64(name, forced):
    d, c, w, _ = oracle.stencil(name)
    dims = TINY[name][1]
    N = oracle.n_nodes(dims)
    f0 = near_eq(name, dims, seed=31)
    F = lbinputs.random_field((d, N), seed=32, amp=1e-3) if forced else None
    for layout in ["ab", "aa"]:
        lat = L(name, dims, 0.7, "bgk", storage="f64", layout=layout)
        if forced:
            lat.set_force(F)
        lat.set_populations(f0)
        lat.step(3)
        ref = oracle.step(name, dims, 0.7, "bgk", f0, nsteps=3, F=F)
        r_o, u_o = oracle.moments(name, dims, ref, F=F)
        r_g, u_g = lat.moments(torch.float64, "cpu")
        np.testing.assert_allclose(r_g.numpy(), r_o, rtol=0, atol=1e-13)
        np.testing.assert_allclose(u_g.numpy(), u_o, rtol=0, atol=1e-14)
        np.testing.assert_allclose(lat.reduce(), oracle.reduce(name, dims, ref, F=F), rtol=1e-12, atol=1e-15)
        # device outputs, FP32
        r32, u32 = lat.moments(torch.float32, "cuda")
        np.testing.assert_allclose(r32.cpu().numpy(), r_o, rtol=1e-6)


def test_reduce_is_deterministic():
    dims, rho, u = lbinputs.taylor_green_3d(48)
    lat = L("D3Q19", dims, 0.6, "bgk", storage="f32")
    lat.init_from_moments(rho, u)
    lat.step(5)
    a = lat.reduce()
    b = lat.reduce()
    np.testing.assert_array_equal(a, b)


def test_init_from_device_fp32_arrays():
    dims, rho, u = lbinputs.taylor_green_2d(32)
    lat = L("D2Q9", dims, 0.8, "bgk", storage="f64")
    lat.init_from_moments(torch.tensor(rho, dtype=torch.float32, device="cuda"),
                          torch.tensor(u, dtype=torch.float32, device="cuda"))
    ref = oracle.init_eq("D2Q9", dims, rho.astype(np.float32).astype(np.float64),
                         u.astype(np.float32).astype(np.float64))
    assert werr(gpu_pops(lat), ref, oracle.stencil("D2Q9")[2]) <= 1e-14


# ------------------------------------------------------------------ half-precision storage
@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("npt", [1, 2, 4])
def test_half_storage_tracks_oracle(storage, tol, npt):
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims, rho, u = lbinputs.taylor_green_2d(64, u0=0.05)
    lat = L(name, dims, 0.8, "bgk", storage=storage, nodes_per_thread=npt)
    lat.init_from_moments(rho, u)
    lat.step(50)
    ref = oracle.step(name, dims, 0.8, "bgk", oracle.init_eq(name, dims, rho, u), nsteps=50)
    # error relative to the largest deviation from rest, which is what the shifted format stores
    dev = np.max(np.abs(ref - w[:, None]) / w[:, None])
    assert werr(gpu_pops(lat), ref, w) <= tol * dev


# ------------------------------------------------------------------ learned collision
def _net(tau, seed=5, out_scale=0.5):
    th = lbinputs.random_mlp_params(seed, out_bias=math.log(tau - 0.5), out_scale=out_scale)
    return np.concatenate([th, np.zeros(6), np.array([50.0, 100.0, 300.0, 1e5, 1e5, 1e5])])


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_learned_fp64_matches_oracle(layout):
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims = (33, 7, 1)
    tau = 0.6
    net = _net(tau)
    f0 = near_eq(name, dims, seed=41)
    lat = L(name, dims, tau, "learned", storage="f64", layout=layout)
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(5)
    ref = oracle.step(name, dims, tau, "learned", f0, nsteps=5, mlp=net)
    assert werr(gpu_pops(lat), ref, w) <= 1e-12


def test_learned_fp32_100_steps():
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims, rho, u = lbinputs.shear_layer(64, u0=0.05)
    tau = 0.55
    net = _net(tau, seed=6)
    lat = L(name, dims, tau, "learned", storage="f32")
    lat.set_mlp(net)
    lat.init_from_moments(rho, u)
    lat.step(100)
    ref = oracle.step(name, dims, tau, "learned", oracle.init_eq(name, dims, rho, u), nsteps=100, mlp=net)
    assert werr(gpu_pops(lat), ref, w) <= 1e-5


def test_learned_with_bgk_network_equals_bgk():
    name = "D2Q9"
    dims, rho, u = lbinputs.shear_layer(32)
    tau = 0.6
    net = _net(tau, out_scale=0.0)
    a = L(name, dims, tau, "learned", storage="f64")
    a.set_mlp(net)
    b = L(name, dims, tau, "bgk", storage="f64")
    for lat in (a, b):
        lat.init_from_moments(rho, u)
        lat.step(20)
    assert werr(gpu_pops(a), gpu_pops(b), oracle.stencil(name)[2]) <= 1e-13


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("name,dims,coll,forced", [
    ("D2Q9", (9, 7, 1), "bgk", True), ("D2Q9", (9, 7, 1), "regularized", True),
    ("D3Q19", (5, 4, 3), "bgk", True), ("D3Q27", (5, 4, 3), "regularized", False),
    ("D2Q9", (9, 7, 1), "none", False),
    # even nx: the two-nodes-per-thread adjoint kernel
    ("D2Q9", (8, 7, 1), "bgk", True), ("D2Q9", (2, 3, 1), "regularized", True),
    ("D3Q19", (6, 4, 3), "regularized", True), ("D3Q27", (4, 4, 3), "bgk", True),
    ("D2Q9", (10, 3, 1), "none", False)])
def test_adjoint_fp64_matches_oracle(name, dims, coll, forced):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    f0 = near_eq(name, dims, seed=51)
    F = lbinputs.random_field((d, N), seed=52, amp=1e-3) if forced else None
    lamT = lbinputs.random_field((len(w), N), seed=53)
    n = 7
    lat = L(name, dims, 0.7, coll, storage="f64", record_every=3)
    if forced:
        lat.set_force(F)
    lat.set_populations(f0)
    lat.step(n)
    gF = torch.zeros((d, N), dtype=torch.float64) if forced else None
    lam0 = lat.step_adjoint(torch.tensor(lamT), n, grad_F=gF)
    ref_lam, ref_gF, _ = oracle.adjoint(name, dims, 0.7, coll, f0, n, lamT, F=F)
    scale = np.max(np.abs(ref_lam))
    assert np.max(np.abs(lam0.numpy() - ref_lam)) <= 1e-12 * scale
    if forced:
        assert np.max(np.abs(gF.numpy() - ref_gF)) <= 1e-12 * np.max(np.abs(ref_gF))
    # the state is left at f^n
    assert werr(gpu_pops(lat), oracle.step(name, dims, 0.7, coll, f0, nsteps=n, F=F), w) <= 1e-12


def test_learned_adjoint_fp64_matches_oracle():
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims = (131, 3, 1)  # more than one block of the parameter-gradient reduction, ragged tail
    N = oracle.n_nodes(dims)
    tau = 0.6
    net = _net(tau, seed=8)
    f0 = near_eq(name, dims, seed=61)
    lamT = lbinputs.random_field((9, N), seed=62)
    lat = L(name, dims, tau, "learned", storage="f64", record_every=2)
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(5)
    gth = torch.zeros(793, dtype=torch.float64)
    lam0 = lat.step_adjoint(torch.tensor(lamT), 5, grad_theta=gth)
    ref_lam, _, ref_th = oracle.adjoint(name, dims, tau, "learned", f0, 5, lamT, mlp=net)
    assert np.max(np.abs(lam0.numpy() - ref_lam)) <= 1e-11 * np.max(np.abs(ref_lam))
    assert np.max(np.abs(gth.numpy() - ref_th)) <= 1e-10 * np.max(np.abs(ref_th))


@pytest.mark.parametrize("dims", [(131, 24, 1), (1100, 40, 1)])
def test_learned_adjoint_fp32_matches_oracle(dims):
    """The FP32 adjoint of the 6-24-24-1 network (the one training runs: network products on the
    tensor cores with split BF16 operands, FP32 tanh) against the FP64 oracle, element by element
    on lambda_0 and the parameter gradient. Both grids end in a ragged warp tile; the second has
    more warp tiles than the persistent grid has warps, so warps sum several tiles."""
    name = "D2Q9"
    N = oracle.n_nodes(dims)
    tau = 0.6
    net = _net(tau, seed=8)
    f0 = near_eq(name, dims, seed=71)
    lamT = lbinputs.random_field((9, N), seed=72)
    n = 6
    lat = L(name, dims, tau, "learned", storage="f32", record_every=4)  # a partial last segment
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(n)
    gth = torch.zeros(793, dtype=torch.float32, device="cuda")
    lam0 = lat.step_adjoint(torch.tensor(lamT, dtype=torch.float32, device="cuda"), n, grad_theta=gth)
    f0_32 = f0.astype(np.float32).astype(np.float64)  # the FP32 state starts from f0 rounded
    ref_lam, _, ref_th = oracle.adjoint(name, dims, tau, "learned", f0_32, n, lamT.astype(np.float32).astype(np.float64),
                                        mlp=net)
    got_th, got_lam = gth.cpu().numpy().astype(np.float64), lam0.cpu().numpy().astype(np.float64)
    err_th = np.max(np.abs(got_th - ref_th)) / np.max(np.abs(ref_th))
    err_lam = np.max(np.abs(got_lam - ref_lam)) / np.max(np.abs(ref_lam))
    rel_l2 = np.linalg.norm(got_th - ref_th) / np.linalg.norm(ref_th)
    print(f"learned FP32 adjoint {dims}: theta max {err_th:.2e} L2 {rel_l2:.2e}, lambda {err_lam:.2e}")
    assert err_th <= 1e-4 and rel_l2 <= 1e-4 and err_lam <= 1e-4
    for lo, hi in ((0, 144), (144, 168), (168, 744), (744, 768), (768, 792), (792, 793)):
        assert np.max(np.abs(got_th[lo:hi])) > 0.0  # every parameter group carries gradient


def test_adjoint_fp32_gradient_within_1e_4_of_fp64_reference():
    # energy-field loss of a forced D2Q9 run: the FP32 GPU gradient w.r.t. F against
    # the oracle's FP64 adjoint, which itself matches finite differences
    name = "D2Q9"
    d, c, w, _ = oracle.stencil(name)
    dims, rho, u = lbinputs.shear_layer(64, u0=0.05)
    N = oracle.n_nodes(dims)
    tau = 0.6
    F = lbinputs.smooth_force(dims, 1e-5, seed=12929)
    et = lbinputs.random_field(N, 7, amp=1e-4) + 1e-3
    n = 50
    lat = L(name, dims, tau, "bgk", storage="f32", record_every=10)
    lat.set_force(torch.tensor(F, dtype=torch.float32, device="cuda"))
    lat.init_from_moments(rho, u)
    lat.step(n)
    gF = torch.zeros((2, N), dtype=torch.float32, device="cuda")
    loss, lamT = lat.loss_energy(torch.tensor(et, dtype=torch.float32, device="cuda"), grad_F=gF)
    lat.step_adjoint(lamT, n, grad_F=gF, want_lambda0=False)
    f0 = oracle.init_eq(name, dims, rho, u)
    fN = oracle.step(name, dims, tau, "bgk", f0, nsteps=n, F=F)
    L_o, lam_o, gF_o = oracle.loss_energy(name, dims, fN, et, F=F)
    _, gF_adj, _ = oracle.adjoint(name, dims, tau, "bgk", f0, n, lam_o, F=F)
    ref = gF_o + gF_adj
    assert abs(loss - L_o) <= 1e-4 * abs(L_o)
    rel = np.linalg.norm(gF.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4


def test_adjoint_requires_matching_recording():
    from paper_2106_12929_gb300 import LBError
    dims = (8, 8, 1)
    lat = L("D2Q9", dims, 0.7, "bgk", storage="f64", record_every=4)
    lat.init_from_moments(np.ones(64), np.zeros((2, 64)))
    lat.step(6)
    with pytest.raises(LBError) as e:
        lat.step_adjoint(torch.zeros((9, 64), dtype=torch.float64), 5)
    assert e.value.code == "LB_ERR_STATE"
    plain = L("D2Q9", dims, 0.7, "bgk", storage="f64")
    plain.init_from_moments(np.ones(64), np.zeros((2, 64)))
    plain.step(2)
    with pytest.raises(LBError):
        plain.step_adjoint(torch.zeros((9, 64), dtype=torch.float64), 2)


# ------------------------------------------------------------------ loss seeds
def test_energy_loss_and_moment_seed_fp64():
    name = "D3Q19"
    d, c, w, _ = oracle.stencil(name)
    dims = (5, 4, 3)
    N = 60
    f0 = near_eq(name, dims, seed=71)
    F = lbinputs.random_field((3, N), seed=72, amp=1e-3)
    et = lbinputs.random_field(N, 73, amp=1e-3) + 2e-3
    lat = L(name, dims, 0.7, "bgk", storage="f64")
    lat.set_force(F)
    lat.set_populations(f0)
    gF = torch.zeros((3, N), dtype=torch.float64)
    loss, lam = lat.loss_energy(torch.tensor(et), grad_F=gF)
    L_o, lam_o, gF_o = oracle.loss_energy(name, dims, f0, et, F=F)
    assert abs(loss - L_o) <= 1e-13 * abs(L_o)
    np.testing.assert_allclose(lam.numpy(), lam_o, rtol=0, atol=1e-13 * np.abs(lam_o).max())
    np.testing.assert_allclose(gF.numpy(), gF_o, rtol=0, atol=1e-13 * np.abs(gF_o).max())
    gr = lbinputs.random_field(N, 74)
    gu = lbinputs.random_field((3, N), 75)
    gF2 = torch.zeros((3, N), dtype=torch.float64)
    lam2 = lat.adjoint_seed_moments(torch.tensor(gr), torch.tensor(gu), grad_F=gF2)
    lam2_o, gF2_o = oracle.seed_moments(name, dims, f0, gr, gu, F=F)
    np.testing.assert_allclose(lam2.numpy(), lam2_o, rtol=0, atol=1e-13)
    np.testing.assert_allclose(gF2.numpy(), gF2_o, rtol=0, atol=1e-13)


def test_eq6_loss_fp64():
    dims = (17, 13, 1)
    N = 17 * 13
    f0 = near_eq("D2Q9", dims, seed=81)
    uref = lbinputs.random_field((2, N), 82, amp=0.05)
    wref = lbinputs.random_field(N, 83, amp=0.01)
    lat = L("D2Q9", dims, 0.7, "bgk", storage="f64")
    lat.set_populations(f0)
    loss, lam = lat.loss_eq6(torch.tensor(uref), torch.tensor(wref), 1e-3)
    L_o, lam_o = oracle.loss_eq6(dims, f0, uref, wref, 1e-3)
    assert abs(loss - L_o) <= 1e-13 * abs(L_o)
    np.testing.assert_allclose(lam.numpy(), lam_o, rtol=0, atol=1e-13 * np.abs(lam_o).max())


# ------------------------------------------------------------------ failure detection
def test_unstable_state_is_reported_not_trapped():
    from paper_2106_12929_gb300 import LBError
    name = "D2Q9"
    dims = (16, 8, 1)
    d, c, w, _ = oracle.stencil(name)
    f0 = near_eq(name, dims, seed=91)
    f0[3, 17] = float("nan")  # fault injected from the host
    lat = L(name, dims, 0.7, "bgk", storage="f32", check_every=2)
    lat.set_populations(f0)
    with pytest.raises(LBError) as e:
        lat.step(4)
    assert e.value.code == "LB_ERR_UNSTABLE"
    # the flag is cleared and the context stays usable
    lat.set_populations(near_eq(name, dims, seed=92))
    lat.step(4)
    lat.check()


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_full_size_d3q19_256_sampled(layout):
    """The benchmark's workload (D3Q19 BGK FP32, 256^3 TGV, Re 1600, Ma 0.1) in its
    launch configuration: one step, 64 sampled nodes recomputed by the oracle one by one."""
    name = "D3Q19"
    d, c, w, _ = oracle.stencil(name)
    n = 256
    u0 = 0.1 / math.sqrt(3.0)
    tau = lbinputs.tau_from_reynolds(1600.0, u0, n)
    dims, rho, u = lbinputs.taylor_green_3d(n, u0=u0)
    lat = L(name, dims, tau, "bgk", storage="f32", layout=layout)
    lat.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    lat.step(1)
    f1 = lat.get_populations(torch.float64, "cuda")
    rng = np.random.default_rng(256)
    xs = rng.integers(0, n, size=(64, 3))
    xs[:4] = [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 7], [n - 1, 0, 0]]
    # the FP32 state after init is f^eq rounded to FP32: the oracle starts from that
    worst = 0.0
    for x, y, z in xs:
        node = x + n * (y + n * z)
        got = f1[:, node].cpu().numpy()
        for i in range(len(w)):
            sx, sy, sz = (x - c[i, 0]) % n, (y - c[i, 1]) % n, (z - c[i, 2]) % n
            src = sx + n * (sy + n * sz)
            fsrc = oracle.init_eq(name, (1, 1, 1), [rho[src]], u[:, src].reshape(3, 1))[:, 0]
            fsrc = fsrc.astype(np.float32).astype(np.float64)
            post = oracle.collide_node(name, tau, "bgk", fsrc)
            worst = max(worst, abs(got[i] - post[i]) / w[i])
    assert worst <= 1e-6
    # properties at full size: mass conserved, momentum zero
    r = lat.reduce()
    assert abs(r[0] / n ** 3 - rho.mean()) <= 1e-6
    assert np.max(np.abs(r[1:4])) / n ** 3 <= 1e-7


# ------------------------------------------------------------------ torch.autograd
def test_autograd_force_gradient_matches_oracle():
    from paper_2106_12929_gb300 import Lattice, lb_run
    name = "D2Q9"
    dims, rho, u = lbinputs.shear_layer(32, u0=0.05)
    N = 32 * 32
    tau = 0.6
    F0 = lbinputs.smooth_force(dims, 1e-4, seed=3)
    et = lbinputs.random_field(N, 4, amp=1e-4) + 1e-3
    lat = Lattice(name, dims, tau, "bgk", storage="f64", record_every=4)
    F = torch.tensor(F0, device="cuda", requires_grad=True)
    r, v = lb_run(lat, torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"), 10, F=F)
    e = 0.5 * r * (v * v).sum(0)
    loss = ((e - torch.tensor(et, device="cuda")) ** 2).sum()
    loss.backward()
    f0 = oracle.init_eq(name, dims, rho, u)
    fN = oracle.step(name, dims, tau, "bgk", f0, nsteps=10, F=F0)
    L_o, lam_o, gF_o = oracle.loss_energy(name, dims, fN, et, F=F0)
    _, gF_adj, _ = oracle.adjoint(name, dims, tau, "bgk", f0, 10, lam_o, F=F0)
    ref = gF_o + gF_adj
    assert abs(loss.item() - L_o) <= 1e-12 * L_o
    assert np.max(np.abs(F.grad.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_autograd_network_gradient_matches_oracle():
    from paper_2106_12929_gb300 import Lattice, lb_run
    dims, rho, u = lbinputs.shear_layer(24, u0=0.05)
    N = 24 * 24
    tau = 0.6
    net = _net(tau, seed=9)
    lat = Lattice("D2Q9", dims, tau, "learned", storage="f64", record_every=3)
    theta = torch.tensor(net[:793], device="cuda", requires_grad=True)
    extra = torch.tensor(net[793:], device="cuda")
    wu = lbinputs.random_field((2, N), 5)
    r, v = lb_run(lat, torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"), 7, theta=theta,
                  net_extra=extra)
    loss = (v * torch.tensor(wu, device="cuda")).sum()
    loss.backward()
    f0 = oracle.init_eq("D2Q9", dims, rho, u)
    fN = oracle.step("D2Q9", dims, tau, "learned", f0, nsteps=7, mlp=net)
    lamN, _ = oracle.seed_moments("D2Q9", dims, fN, None, wu)
    _, _, gth = oracle.adjoint("D2Q9", dims, tau, "learned", f0, 7, lamN, mlp=net)
    assert np.max(np.abs(theta.grad.cpu().numpy() - gth)) <= 1e-10 * np.max(np.abs(gth))


def test_autograd_backward_after_another_run_raises():
    """The lattice keeps one recorded run: a second lb_run with the same step count replaces it,
    so the first result's backward pass must fail instead of returning the second run's gradient."""
    from paper_2106_12929_gb300 import Lattice, lb_run
    dims, rho, u = lbinputs.shear_layer(16, u0=0.05)
    lat = Lattice("D2Q9", dims, 0.6, "bgk", storage="f64", record_every=2)
    F1 = torch.tensor(lbinputs.smooth_force(dims, 1e-4, seed=3), device="cuda", requires_grad=True)
    F2 = torch.tensor(lbinputs.smooth_force(dims, 1e-4, seed=4), device="cuda", requires_grad=True)
    r0, v0 = torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda")
    _, v1 = lb_run(lat, r0, v0, 5, F=F1)
    _, v2 = lb_run(lat, r0, v0, 5, F=F2)
    with pytest.raises(RuntimeError, match="recorded run is gone"):
        (v1 ** 2).sum().backward()
    (v2 ** 2).sum().backward()  # the latest run still differentiates
    assert torch.isfinite(F2.grad).all() and F2.grad.abs().max() > 0
    _, v3 = lb_run(lat, r0, v0, 5, F=F1)
    lat.set_force(F2.detach())
    with pytest.raises(RuntimeError, match="recorded run is gone"):
        (v3 ** 2).sum().backward()
    lat.close()


@pytest.mark.parametrize("name,dims", [("D2Q9", (8, 3, 1)), ("D2Q9", (4, 5, 1)), ("D3Q19", (4, 3, 3)),
                                       ("D3Q19", (12, 2, 2)), ("D3Q27", (4, 5, 3))])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_half_storage_four_node_kernel(name, dims, storage):
    """nx % 4 == 0 runs the four-nodes-per-thread half kernel: AA == AB bit-exact, and close
    to the oracle started from the same quantised state."""
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    f0 = near_eq(name, dims, seed=101)
    F = lbinputs.random_field((d, N), seed=102, amp=1e-3)
    for coll, forced in (("bgk", False), ("bgk", True), ("regularized", False)):
        a = L(name, dims, 0.7, coll, storage=storage, layout="ab")
        b = L(name, dims, 0.7, coll, storage=storage, layout="aa")
        for lat in (a, b):
            if forced:
                lat.set_force(F)
            lat.set_populations(f0)
        q0 = gpu_pops(a)
        for _ in range(3):
            a.step(1)
            b.step(1)
            np.testing.assert_array_equal(gpu_pops(a), gpu_pops(b))
        ref = oracle.step(name, dims, 0.7, coll, q0, nsteps=3, F=F if forced else None)
        dev = np.max(np.abs(ref - w[:, None]) / w[:, None])
        tol = (2e-3 if storage == "f16" else 2e-2) * dev
        assert werr(gpu_pops(a), ref, w) <= tol


# ------------------------------------------------------------------ learned collision on tensor cores
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_learned_tensor_core_option(storage):
    name = "D2Q9"
    dims = (130, 40, 1)  # five 32-node warp tiles per row, the last one ragged
    rho, u = lbinputs.random_moments(dims, seed=7, u_amp=0.05)
    d, c, w, _ = oracle.stencil(name)
    tau = 0.6
    # zero output layer: z = b3 in both paths, so they differ only by FP32 rounding (which can
    # flip a half-precision rounding: a few FP16 ulps); random network: FP16 activations
    # change the higher-moment rate by ~1e-3 relative
    same_tol = 1e-6 if storage == "f32" else 2e-4
    for net, tol in ((_net(tau, out_scale=0.0), same_tol), (_net(tau, seed=12, out_scale=0.5), 1e-3)):
        a = L(name, dims, tau, "learned", storage=storage)
        b = L(name, dims, tau, "learned", storage=storage, learned_tc=True)
        for lat in (a, b):
            lat.set_mlp(net)
            lat.init_from_moments(rho, u)
            lat.step(10)
        fa, fb = gpu_pops(a), gpu_pops(b)
        assert werr(fa, fb, w) <= tol
        if tol == 1e-3:
            assert werr(fa, fb, w) > 0.0  # the BF16 network really ran


# ------------------------------------------------------------------ graph replay of step pairs
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("coll,storage", [("bgk", "f32"), ("regularized", "f16"), ("learned", "f32")])
def test_graph_replay_equals_single_steps(layout, coll, storage):
    """lb_step(n) replays a captured two-step graph; lb_step(1) launches directly. Same bits."""
    name = "D2Q9"
    dims = (48, 20, 1)
    rho, u = lbinputs.random_moments(dims, seed=3, u_amp=0.05)
    F = lbinputs.random_field((2, 960), seed=4, amp=1e-4)
    a = L(name, dims, 0.6, coll, storage=storage, layout=layout)
    b = L(name, dims, 0.6, coll, storage=storage, layout=layout)
    for lat in (a, b):
        if coll == "learned":
            lat.set_mlp(_net(0.6, seed=3))
        else:
            lat.set_force(F)
        lat.init_from_moments(rho, u)
    a.step(7)           # 3 graph replays + 1 direct step
    for _ in range(7):
        b.step(1)
    np.testing.assert_array_equal(gpu_pops(a), gpu_pops(b))
    assert a.launch_count() - b.launch_count() == 0
    # changing the force (or the network) must not replay a stale graph
    if coll == "learned":
        a.set_mlp(_net(0.6, seed=4))
        b.set_mlp(_net(0.6, seed=4))
    else:
        a.set_force(2 * F)
        b.set_force(2 * F)
    a.step(4)
    for _ in range(4):
        b.step(1)
    np.testing.assert_array_equal(gpu_pops(a), gpu_pops(b))


# ------------------------------------------------------------------ launch shapes
@pytest.mark.parametrize("name,dims", [("D2Q9", (12, 5, 1)), ("D3Q19", (8, 5, 3)), ("D3Q27", (8, 3, 4))])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_launch_shapes_are_bit_identical(name, dims, storage, layout):
    """One, two and four nodes per thread (and the automatic choice) run the same per-node
    arithmetic. The compiler may contract a multiply and an add into one FMA differently in
    the three kernels, so the states agree to the last bits of the arithmetic type after a
    few steps: FP64 1e-14, FP32 1e-6, half storage one quantisation step of the stored
    deviation (1e-4), all relative to w_i."""
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    f0 = near_eq(name, dims, seed=101)
    F = lbinputs.random_field((d, N), seed=102, amp=1e-3)
    colls = [("bgk", True), ("regularized", True), ("trt", True), ("none", False)]
    if name != "D3Q19":
        colls.append(("kbc", False))
    if name == "D2Q9":
        colls.append(("mrt", False))
    for coll, forced in colls:
        out = []
        for npt in (0, 1, 2, 4):
            lat = L(name, dims, 0.6, coll, storage=storage, layout=layout, nodes_per_thread=npt)
            if forced:
                lat.set_force(F)
            lat.set_populations(f0)
            lat.step(3)
            out.append(gpu_pops(lat))
            lat.close()
        tol = {"f64": 1e-14, "f32": 1e-6}.get(storage, 1e-4)
        for o in out[1:]:
            assert werr(o, out[0], w) <= tol, coll


# ------------------------------------------------------------------ bandwidth reference
def test_stream_copy_copies_bytes_and_rejects_host_memory():
    """lb_stream_copy (the benchmark's bandwidth reference) moves every byte, including a tail
    shorter than one four-vector round, and refuses host memory before any launch."""
    from paper_2106_12929_gb300 import _lib
    lib = _lib.load()
    nbytes = 16 * (3 * 1024 * 1024 + 5)
    src = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device="cuda")
    dst = torch.zeros(nbytes + 16, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    assert lib.lb_stream_copy(src.data_ptr(), dst.data_ptr(), nbytes, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(dst[:nbytes], src)
    assert int(dst[nbytes:].abs().sum()) == 0  # nothing past the end
    host = np.zeros(1024, dtype=np.uint8)
    assert lib.lb_stream_copy(host.ctypes.data, dst.data_ptr(), 1024, None) == 1
