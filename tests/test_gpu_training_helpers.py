"""Parity of the training helpers of Sec. 3.1, each on its own: the 2 x 2 coarse-graining of a
fine state (lb_coarsen_into), the Eq. 6 vorticity (lb_vorticity), the network's six inputs
(lb_learned_inputs) against the oracle, and one Adam update (lb_adam_update) against its
definition. The training driver runs all four; its tests check the resulting gain."""
import numpy as np
import pytest
import torch

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

NAME = "D2Q9"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_12929_gb300 import build
    build.build()
    oracle.build()


def L(*a, **k):
    from paper_2106_12929_gb300 import Lattice
    return Lattice(*a, **k)


def _stored_state(lat, dims, seed):
    """Seeded populations away from equilibrium (f = w (1 + 0.05 r)), set into the lattice; returns
    the state as stored (FP32 storage rounds it) and the weights."""
    d, c, w, _ = oracle.stencil(NAME)
    lat.set_populations(lbinputs.random_populations(w, oracle.n_nodes(dims), seed, eps=0.05))
    return lat.get_populations(torch.float64, "cpu").numpy(), w


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 3e-6)])
def test_coarsen_is_equilibrium_of_block_means(storage, tol):
    # coarse state = f^eq(rho_c, u_c), rho_c and rho_c u_c the means of rho and rho u over 2 x 2
    # blocks of the fine state (an odd coarse edge: 9 x 7)
    fine_dims, coarse_dims = (18, 14, 1), (9, 7, 1)
    fine = L(NAME, fine_dims, 0.51, "bgk", storage=storage)
    fs, w = _stored_state(fine, fine_dims, 70)
    coarse = L(NAME, coarse_dims, 0.505, "bgk", storage=storage)
    _stored_state(coarse, coarse_dims, 71)
    coarse.step(2)
    coarse.coarsen_from(fine)
    assert coarse.steps_taken() == 0
    got = coarse.get_populations(torch.float64, "cpu").numpy()
    rho, u = oracle.moments(NAME, fine_dims, fs)
    ny, nx = fine_dims[1], fine_dims[0]

    def block_mean(a):
        return a.reshape(ny // 2, 2, nx // 2, 2).mean(axis=(1, 3)).reshape(-1)

    rho_c = block_mean(rho)
    u_c = np.stack([block_mean(rho * u[k]) for k in range(2)]) / rho_c
    ref = oracle.init_eq(NAME, coarse_dims, rho_c, u_c)
    assert np.max(np.abs(got - ref) / w[:, None]) <= tol
    fine.close()
    coarse.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 5e-6)])
def test_vorticity_matches_oracle(storage, tol):
    dims = (17, 12, 1)  # ragged: 17 is odd
    lat = L(NAME, dims, 0.6, "bgk", storage=storage)
    fs, _ = _stored_state(lat, dims, 80)
    ref, _ = oracle.vorticity(dims, fs)
    scale = np.max(np.abs(ref))
    assert scale > 1e-3
    for dt, out_tol in ((torch.float64, tol), (torch.float32, max(tol, 2e-7))):  # FP32 output rounds
        got = lat.vorticity(dt, "cuda").double().cpu().numpy()
        assert np.max(np.abs(got - ref)) <= out_tol * scale, dt
    lat.close()


@pytest.mark.parametrize("storage,rtol", [("f64", 1e-11), ("f32", 5e-4)])
def test_learned_inputs_match_oracle(storage, rtol):
    # the six invariants of every node, before standardisation; error relative to each input's
    # largest magnitude over the grid
    dims = (13, 6, 1)
    N = oracle.n_nodes(dims)
    lat = L(NAME, dims, 0.6, "bgk", storage=storage)
    fs, _ = _stored_state(lat, dims, 90)
    ref = np.stack([oracle.invariants(fs[:, n]) for n in range(N)], axis=1)
    got = lat.learned_inputs(torch.float64, "cuda").cpu().numpy()
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.all(scale > 0)
    assert np.all(np.abs(got - ref) <= rtol * scale)
    lat.close()


def test_adam_update_matches_its_definition():
    # m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    # theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); FP32 on the device
    from paper_2106_12929_gb300 import adam_update
    n, t, lr, b1, b2, eps = 1000, 3, 1e-2, 0.9, 0.999, 1e-8  # 1000: a ragged last block
    rng = np.random.default_rng(5)
    th = rng.standard_normal(n).astype(np.float32)
    m = (0.01 * rng.standard_normal(n)).astype(np.float32)
    v = (1e-4 * (0.5 + rng.random(n))).astype(np.float32)
    g = (0.1 * rng.standard_normal(n)).astype(np.float32)
    T = [torch.tensor(a, device="cuda") for a in (th, m, v, g)]
    adam_update(T[0], T[1], T[2], T[3], t, lr=lr, betas=(b1, b2), eps=eps)
    th64, m64, v64, g64 = (a.astype(np.float64) for a in (th, m, v, g))
    m1 = b1 * m64 + (1 - b1) * g64
    v1 = b2 * v64 + (1 - b2) * g64 * g64
    th1 = th64 - lr * (m1 / (1 - b1 ** t)) / (np.sqrt(v1 / (1 - b2 ** t)) + eps)
    np.testing.assert_allclose(T[1].cpu().numpy(), m1, rtol=1e-5, atol=2e-8)  # FP32 of terms up to 0.05
    np.testing.assert_allclose(T[2].cpu().numpy(), v1, rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(T[0].cpu().numpy(), th1, rtol=0, atol=1e-5)
    assert np.max(np.abs(th1 - th64)) > 1e-3  # the update is not negligible
