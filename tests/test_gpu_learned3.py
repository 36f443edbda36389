"""Parity of the one-hidden-layer, three-output learned collision (collision "learned3": the
network shape Sec. 3.1 describes, one relaxation time exp(z) + 1/2 per higher moment) with
the FP64 oracle, through the C ABI: the forward step in every storage and layout, the limits
that fix which output drives which moment, the adjoint with its parameter gradient (also
through torch.autograd), graph replay and the argument checks.

Error measure for populations: max over i, x of |f_gpu - f_oracle| / w_i. Bars as for the
other collisions: FP64 <= 1e-12, FP32 <= 1e-5 after 100 steps; half storage relative to the
largest stored deviation from rest.
"""
import math

import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

NAME = "D2Q9"
SCALE = np.array([50.0, 100.0, 300.0, 1e5, 1e5, 1e5])  # input standardisation (shift 0)


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


def pops(lat):
    return lat.get_populations(torch.float64, "cpu").numpy()


def near_eq(dims, seed, eps=0.05):
    d, c, w, _ = oracle.stencil(NAME)
    rho, u = lbinputs.random_moments(dims, seed=seed, u_amp=0.05)
    N = oracle.n_nodes(dims)
    return oracle.init_eq(NAME, dims, rho, u) + eps * 0.1 * w[:, None] * lbinputs.random_field((9, N), seed + 1)


def net3(tau, seed=5, out_scale=0.5, taus=None):
    """545 values; output biases ln(tau_o - 1/2) (all tau unless taus = (tau_N, tau_J0, tau_J1))."""
    bias = math.log(tau - 0.5) if taus is None else np.log(np.asarray(taus, dtype=np.float64) - 0.5)
    th = lbinputs.random_mlp3_params(seed, out_bias=bias, out_scale=out_scale)
    return np.concatenate([th, np.zeros(6), SCALE])


W = oracle.stencil(NAME)[2]


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_fp64_matches_oracle(layout):
    dims = (131, 5, 1)  # two blocks per row, the second ragged
    tau = 0.6
    net = net3(tau, taus=(0.9, 0.7, 1.3))
    f0 = near_eq(dims, seed=41)
    lat = L(NAME, dims, tau, "learned3", storage="f64", layout=layout)
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(5)
    ref = oracle.step(NAME, dims, tau, "learned3", f0, nsteps=5, mlp=net)
    assert werr(pops(lat), ref, W) <= 1e-12


def test_fp32_100_steps():
    dims, rho, u = lbinputs.shear_layer(64, u0=0.05)
    tau = 0.55
    net = net3(tau, seed=6, taus=(0.8, 0.6, 0.7))
    lat = L(NAME, dims, tau, "learned3", storage="f32")
    lat.set_mlp(net)
    lat.init_from_moments(rho, u)
    lat.step(100)
    ref = oracle.step(NAME, dims, tau, "learned3", oracle.init_eq(NAME, dims, rho, u), nsteps=100, mlp=net)
    assert werr(pops(lat), ref, W) <= 1e-5


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_half_storage_tracks_oracle(storage, tol):
    dims, rho, u = lbinputs.taylor_green_2d(64, u0=0.05)
    tau = 0.8
    net = net3(tau, seed=7, taus=(1.0, 0.9, 1.1))
    lat = L(NAME, dims, tau, "learned3", storage=storage)
    lat.set_mlp(net)
    lat.init_from_moments(rho, u)
    lat.step(50)
    ref = oracle.step(NAME, dims, tau, "learned3", oracle.init_eq(NAME, dims, rho, u), nsteps=50, mlp=net)
    dev = np.max(np.abs(ref - W[:, None]) / W[:, None])
    assert werr(pops(lat), ref, W) <= tol * dev


def test_constant_outputs_are_the_fixed_rate_mrt_and_bgk():
    """Zero output weights: the rates are the biases, so the step is the GPU's own MRT with
    (tau_6, tau_7, tau_8) = (tau_J0, tau_J1, tau_N), and BGK when all equal tau."""
    dims, rho, u = lbinputs.shear_layer(32)
    tau = 0.6
    tN, tJ0, tJ1 = 1.3, 0.8, 2.1
    a = L(NAME, dims, tau, "learned3", storage="f64")
    a.set_mlp(net3(tau, out_scale=0.0, taus=(tN, tJ0, tJ1)))
    b = L(NAME, dims, tau, "mrt", storage="f64")
    b.set_relaxation([tJ0, tJ1, tN])
    c = L(NAME, dims, tau, "learned3", storage="f64")
    c.set_mlp(net3(tau, out_scale=0.0))
    d = L(NAME, dims, tau, "bgk", storage="f64")
    for lat in (a, b, c, d):
        lat.init_from_moments(rho, u)
        lat.step(20)
    assert werr(pops(a), pops(b), W) <= 1e-13
    assert werr(pops(c), pops(d), W) <= 1e-13
    assert werr(pops(a), pops(d), W) > 1e-8  # the three times really differ from BGK


def test_adjoint_fp64_matches_oracle():
    dims = (131, 3, 1)  # more than one block of the parameter-gradient reduction, ragged tail
    N = oracle.n_nodes(dims)
    tau = 0.6
    net = net3(tau, seed=8, taus=(0.9, 0.7, 1.3))
    f0 = near_eq(dims, seed=61)
    lamT = lbinputs.random_field((9, N), seed=62)
    lat = L(NAME, dims, tau, "learned3", storage="f64", record_every=2)
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(5)
    gth = torch.zeros(533, dtype=torch.float64)
    lam0 = lat.step_adjoint(torch.tensor(lamT), 5, grad_theta=gth)
    ref_lam, _, ref_th = oracle.adjoint(NAME, dims, tau, "learned3", f0, 5, lamT, mlp=net)
    assert np.max(np.abs(lam0.numpy() - ref_lam)) <= 1e-11 * np.max(np.abs(ref_lam))
    assert np.max(np.abs(gth.numpy() - ref_th)) <= 1e-10 * np.max(np.abs(ref_th))
    # every parameter group carries gradient (no block of the reduction was dropped)
    for lo, hi in ((0, 318), (318, 371), (371, 530), (530, 533)):
        assert np.max(np.abs(gth.numpy()[lo:hi])) > 0.0


def test_adjoint_fp32_parameter_gradient():
    """FP32 arithmetic (network products on the tensor cores with split BF16 operands, FP32 tanh)
    against the FP64 oracle on a 64^2 shear layer: relative L2 error of the parameter gradient
    within the 1e-4 gradient bar."""
    dims, rho, u = lbinputs.shear_layer(64, u0=0.05)
    N = oracle.n_nodes(dims)
    tau = 0.55
    net = net3(tau, seed=9, taus=(0.8, 0.6, 0.7))
    lamT = lbinputs.random_field((9, N), seed=63)
    n = 20
    lat = L(NAME, dims, tau, "learned3", storage="f32", record_every=5)
    lat.set_mlp(net)
    lat.init_from_moments(rho, u)
    lat.step(n)
    gth = torch.zeros(533, dtype=torch.float32, device="cuda")
    lat.step_adjoint(torch.tensor(lamT, dtype=torch.float32, device="cuda"), n, grad_theta=gth,
                     want_lambda0=False)
    f0 = oracle.init_eq(NAME, dims, rho, u)
    _, _, ref = oracle.adjoint(NAME, dims, tau, "learned3", f0, n, lamT, mlp=net)
    rel = np.linalg.norm(gth.cpu().numpy() - ref) / np.linalg.norm(ref)
    print("learned3 FP32 parameter-gradient relative error", rel)
    assert rel <= 1e-4


def test_adjoint_fp32_matches_oracle_elementwise():
    """lambda_0 and every parameter-gradient entry of the FP32 adjoint against the FP64 oracle,
    on a grid with more warp tiles than the persistent grid has warps and a ragged last tile."""
    dims = (1100, 40, 1)
    N = oracle.n_nodes(dims)
    tau = 0.6
    net = net3(tau, seed=8, taus=(0.9, 0.7, 1.3))
    f0 = near_eq(dims, seed=81)
    lamT = lbinputs.random_field((9, N), seed=82)
    n = 6
    lat = L(NAME, dims, tau, "learned3", storage="f32", record_every=4)
    lat.set_mlp(net)
    lat.set_populations(f0)
    lat.step(n)
    gth = torch.zeros(533, dtype=torch.float32, device="cuda")
    lam0 = lat.step_adjoint(torch.tensor(lamT, dtype=torch.float32, device="cuda"), n, grad_theta=gth)
    f0_32 = f0.astype(np.float32).astype(np.float64)
    ref_lam, _, ref_th = oracle.adjoint(NAME, dims, tau, "learned3", f0_32, n,
                                        lamT.astype(np.float32).astype(np.float64), mlp=net)
    got_th, got_lam = gth.cpu().numpy().astype(np.float64), lam0.cpu().numpy().astype(np.float64)
    err_th = np.max(np.abs(got_th - ref_th)) / np.max(np.abs(ref_th))
    err_lam = np.max(np.abs(got_lam - ref_lam)) / np.max(np.abs(ref_lam))
    print(f"learned3 FP32 adjoint: theta {err_th:.2e}, lambda {err_lam:.2e}")
    assert err_th <= 1e-4 and err_lam <= 1e-4
    for lo, hi in ((0, 318), (318, 371), (371, 530), (530, 533)):
        assert np.max(np.abs(got_th[lo:hi])) > 0.0


def test_autograd_parameter_gradient_matches_oracle():
    from paper_2106_12929_gb300 import Lattice, lb_run
    dims, rho, u = lbinputs.shear_layer(24, u0=0.05)
    N = 24 * 24
    tau = 0.6
    net = net3(tau, seed=10, taus=(0.9, 0.7, 1.3))
    lat = Lattice(NAME, dims, tau, "learned3", storage="f64", record_every=3)
    theta = torch.tensor(net[:533], device="cuda", requires_grad=True)
    extra = torch.tensor(net[533:], device="cuda")
    wu = lbinputs.random_field((2, N), 5)
    r, v = lb_run(lat, torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"), 7, theta=theta,
                  net_extra=extra)
    (v * torch.tensor(wu, device="cuda")).sum().backward()
    f0 = oracle.init_eq(NAME, dims, rho, u)
    fN = oracle.step(NAME, dims, tau, "learned3", f0, nsteps=7, mlp=net)
    lamN, _ = oracle.seed_moments(NAME, dims, fN, None, wu)
    _, _, gth = oracle.adjoint(NAME, dims, tau, "learned3", f0, 7, lamN, mlp=net)
    assert np.max(np.abs(theta.grad.cpu().numpy() - gth)) <= 1e-10 * np.max(np.abs(gth))


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_tensor_core_option(storage, layout):
    """The network in half precision on the tensor cores (FP16 operands and hidden-layer
    accumulation, hardware tanh) against the FP32 kernel: with zero output weights both give
    z = the output biases (they differ by FP32 rounding elsewhere, which can flip an FP16
    rounding); with a random network the FP16 activations move the rates by ~1e-3 relative."""
    dims = (130, 40, 1)  # five 32-node warp tiles per row, the last one ragged
    rho, u = lbinputs.random_moments(dims, seed=7, u_amp=0.05)
    tau = 0.6
    same_tol = 1e-6 if storage == "f32" else 2e-4
    for net, tol in ((net3(tau, out_scale=0.0, taus=(0.9, 0.7, 1.3)), same_tol),
                     (net3(tau, seed=12, taus=(0.9, 0.7, 1.3)), 1e-3)):
        a = L(NAME, dims, tau, "learned3", storage=storage, layout=layout)
        b = L(NAME, dims, tau, "learned3", storage=storage, layout=layout, learned_tc=True)
        for lat in (a, b):
            lat.set_mlp(net)
            lat.init_from_moments(rho, u)
            lat.step(10)
        fa, fb = pops(a), pops(b)
        assert werr(fa, fb, W) <= tol
        if tol == 1e-3:
            assert werr(fa, fb, W) > 0.0  # the BF16 network really ran


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_graph_replay_equals_single_steps(layout):
    dims = (48, 20, 1)
    rho, u = lbinputs.random_moments(dims, seed=3, u_amp=0.05)
    a = L(NAME, dims, 0.6, "learned3", storage="f32", layout=layout)
    b = L(NAME, dims, 0.6, "learned3", storage="f32", layout=layout)
    for lat in (a, b):
        lat.set_mlp(net3(0.6, seed=3))
        lat.init_from_moments(rho, u)
    a.step(7)
    for _ in range(7):
        b.step(1)
    np.testing.assert_array_equal(pops(a), pops(b))
    for lat in (a, b):  # a new network must not replay a stale graph
        lat.set_mlp(net3(0.6, seed=4))
    a.step(4)
    for _ in range(4):
        b.step(1)
    np.testing.assert_array_equal(pops(a), pops(b))


def test_argument_checks():
    from paper_2106_12929_gb300 import LBError
    dims = (16, 8, 1)
    lat = L(NAME, dims, 0.6, "learned3", storage="f32")
    with pytest.raises(LBError, match="LB_ERR_ARG"):
        lat.set_mlp(np.zeros(805))  # the other network's size
    with pytest.raises(LBError, match="LB_ERR_STATE"):
        lat.step(1)  # no network yet
    with pytest.raises(LBError, match="LB_ERR_UNSUPPORTED"):
        lat.set_force(np.zeros((2, 128)))
    with pytest.raises(LBError, match="LB_ERR_UNSUPPORTED"):
        L(NAME, dims, 0.6, "learned3", storage="f64", learned_tc=True)
    with pytest.raises(LBError, match="LB_ERR_UNSUPPORTED"):
        L("D3Q19", (8, 8, 8), 0.6, "learned3")
    lat.set_mlp(net3(0.6))
    lat.init_from_moments(np.ones(128), np.zeros((2, 128)))
    lat.step(2)
    lat.check()
