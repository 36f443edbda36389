"""Parity at the workloads' full sizes, in the launch configuration the benchmark uses, on
sampled nodes the oracle recomputes one by one: D3Q27 regularized on 384^3 decaying
turbulence, D2Q9 BGK with a Guo force on the 1024^2 shear layer, and the learned collisions
on 2048^2 decaying turbulence. After the initialisation the FP32 state is f^eq rounded to
FP32; the oracle starts from the same rounded values, pulls them along c_i and collides.
Error measure: |f_gpu - f_oracle| / w_i."""
import math

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


def _sample(dims, seed, count=48):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    xs = np.stack([rng.integers(0, nx, count), rng.integers(0, ny, count), rng.integers(0, nz, count)], axis=1)
    xs[0] = [0, 0, 0]
    xs[1] = [nx - 1, ny - 1, nz - 1]
    return xs


def _check_one_step(name, dims, tau, coll, rho, u, F=None, mlp=None, tol=1e-6, seed=0):
    """One GPU step from f^eq(rho, u) against the oracle on sampled nodes; returns the lattice."""
    d, c, w, _ = oracle.stencil(name)
    nx, ny, nz = dims
    lat = L(name, dims, tau, coll, storage="f32")
    if mlp is not None:
        lat.set_mlp(mlp)
    if F is not None:
        lat.set_force(torch.tensor(F, dtype=torch.float32, device="cuda"))
    lat.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    lat.step(1)
    f1 = lat.get_populations(torch.float64, "cuda")
    worst = 0.0
    for x, y, z in _sample(dims, seed):
        node = x + nx * (y + ny * z)
        fl = np.empty(len(w))
        for i in range(len(w)):  # pull: f_i(x) = f*_i(x - c_i) of the previous state
            src = (x - c[i, 0]) % nx + nx * ((y - c[i, 1]) % ny + ny * ((z - c[i, 2]) % nz))
            feq = oracle.init_eq(name, (1, 1, 1), [rho[src]], u[:, src].reshape(d, 1))[:, 0]
            fsrc = feq.astype(np.float32).astype(np.float64)
            Fs = None if F is None else F[:, src]
            fl[i] = oracle.collide_node(name, tau, coll, fsrc, F=Fs, mlp=mlp)[i]
        got = f1[:, node].cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - fl) / w)))
    assert worst <= tol, worst
    return lat


def test_d3q27_regularized_384_turbulence():
    """The precision-sweep workload (D3Q27 regularized, 384^3 random-phase turbulence, k0 = 8,
    u_rms = 0.04, Re 3000), FP32 storage, two nodes per thread."""
    n = 384
    dims = (n, n, n)
    rho, u = lbinputs.random_spectrum_velocity(dims, 8.0, 0.04, 2106)
    tau = 0.5 + 3.0 * 0.04 * (n / (2.0 * math.pi)) / 3000.0
    lat = _check_one_step("D3Q27", dims, tau, "regularized", rho, u, seed=384)
    r = lat.reduce()
    assert abs(r[0] / n ** 3 - 1.0) <= 1e-6
    lat.close()


def test_d2q9_guo_1024_shear_layer():
    """The adjoint workload's forward step (D2Q9 BGK + Guo force, 1024^2 shear layer, tau 0.51,
    the smooth seeded force field), FP32 storage, two nodes per thread."""
    dims, rho, u = lbinputs.shear_layer(1024, u0=0.05)
    F = lbinputs.smooth_force(dims, 1e-5, seed=12929)
    _check_one_step("D2Q9", dims, 0.51, "bgk", rho, u, F=F, seed=1024).close()


@pytest.mark.parametrize("coll", ["learned", "learned3"])
def test_learned_2048_turbulence(coll):
    """The learned collisions on the evaluation workload (2048^2 decaying turbulence, k0 = 12,
    u_rms = 0.05) with a random network, FP32 network (hardware tanh: 1e-5 bar)."""
    n = 2048
    dims = (n, n, 1)
    rho, u = lbinputs.random_spectrum_velocity(dims, 12.0, 0.05, 30000)
    tau = 0.5 + 3.0 * 0.05 * (n / (2.0 * math.pi)) / 30000.0
    gen = lbinputs.random_mlp3_params if coll == "learned3" else lbinputs.random_mlp_params
    th = gen(7, out_bias=math.log(tau - 0.5), out_scale=0.5)
    mlp = np.concatenate([th, np.zeros(6), np.array([400.0, 100.0, 1e3, 1e6, 1e6, 1e6])])
    _check_one_step("D2Q9", dims, tau, coll, rho, u, mlp=mlp, tol=1e-5, seed=2048).close()
