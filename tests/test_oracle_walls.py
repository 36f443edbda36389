"""Pins of the oracle's halfway bounce-back walls: exact mass conservation in a closed box,
the Poiseuille profile that halfway bounce-back reproduces exactly when
(tau - 1/2)(tau_minus - 1/2) = 3/16 (Ginzburg's TRT result; BGK at tau = 1/2 + sqrt(3/16)),
the exact linear Couette profile under a moving wall, and an all-fluid mask that reduces to
the periodic step."""
from __future__ import annotations

import math

import numpy as np
import pytest

import lbinputs
import oracle

CS2 = 1.0 / 3.0


def _box_mask(dims, d):
    nx, ny, nz = dims
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[:, 0, :] = m[:, -1, :] = 1
    m[:, :, 0] = m[:, :, -1] = 1
    if d == 3:
        m[0] = m[-1] = 1
    return m.reshape(-1)


@pytest.mark.parametrize("name,dims", [("D2Q9", (12, 10, 1)), ("D3Q19", (7, 6, 5)), ("D3Q27", (6, 6, 5))])
@pytest.mark.parametrize("coll", ["bgk", "trt", "regularized"])
def test_closed_box_conserves_mass(name, dims, coll):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    mask = _box_mask(dims, d)
    f = lbinputs.random_populations(w, N, seed=5, eps=0.05)
    f[:, mask == 1] = w[:, None]
    m0 = f[:, mask == 0].sum()
    g = oracle.step_walls(name, dims, 0.7, coll, f, mask, nsteps=60)
    assert abs(g[:, mask == 0].sum() - m0) < 1e-13 * m0
    # solid nodes hold the rest equilibrium
    np.testing.assert_array_equal(g[:, mask == 1], np.repeat(w[:, None], int(mask.sum()), axis=1))


def test_all_fluid_mask_is_the_periodic_step():
    name, dims = "D2Q9", (6, 5, 1)
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    f = lbinputs.random_populations(w, N, seed=6)
    F = lbinputs.random_field((2, N), seed=7, amp=1e-3)
    a = oracle.step_walls(name, dims, 0.66, "bgk", f, np.zeros(N), nsteps=4, F=F)
    b = oracle.step(name, dims, 0.66, "bgk", f, nsteps=4, F=F)
    np.testing.assert_array_equal(a, b)


def _channel(name, H, nx=4, nz=2):
    d, c, w, _ = oracle.stencil(name)
    dims = (nx, H + 2, nz if d == 3 else 1)
    N = oracle.n_nodes(dims)
    m = np.zeros((dims[2], dims[1], dims[0]), dtype=np.uint8)
    m[:, 0, :] = m[:, -1, :] = 1
    return dims, N, m.reshape(-1), d, w


def _row_velocity(name, dims, f, F):
    _, u = oracle.moments(name, dims, f, F=F)
    ux = u[0].reshape(dims[2], dims[1], dims[0])
    return ux[0, 1:-1, 0], ux


@pytest.mark.parametrize("name,coll,tau,params", [
    ("D2Q9", "trt", 0.8, [3.0 / 16.0]), ("D2Q9", "bgk", 0.5 + math.sqrt(3.0 / 16.0), None),
    ("D3Q19", "trt", 0.7, [3.0 / 16.0])])
def test_poiseuille_profile_exact_at_magic_parameter(name, coll, tau, params):
    H = 8
    dims, N, mask, d, w = _channel(name, H)
    Fx = 1e-6
    F = np.zeros((d, N))
    F[0] = Fx
    f = oracle.init_eq(name, dims, np.ones(N), np.zeros((d, N)))
    nu = CS2 * (tau - 0.5)
    steps = int(40.0 * H * H / (nu * math.pi ** 2))  # exp(-40) of the slowest mode left
    f = oracle.step_walls(name, dims, tau, coll, f, mask, nsteps=steps, F=F, params=params)
    u, ux = _row_velocity(name, dims, f, F)
    y = np.arange(1, H + 1, dtype=float)
    exact = Fx / (2.0 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.max(np.abs(u - exact)) < 1e-9 * exact.max()
    # uniform along the channel
    assert np.allclose(ux[:, 1:-1, :], ux[0:1, 1:-1, 0:1], rtol=0, atol=1e-15)


def test_poiseuille_with_bgk_off_the_magic_value_slips():
    # away from the magic combination the halfway wall is off by a slip of order (tau - 1/2)^2
    H = 8
    name, tau = "D2Q9", 1.2
    dims, N, mask, d, w = _channel(name, H)
    Fx = 1e-6
    F = np.zeros((d, N))
    F[0] = Fx
    f = oracle.init_eq(name, dims, np.ones(N), np.zeros((d, N)))
    nu = CS2 * (tau - 0.5)
    f = oracle.step_walls(name, dims, tau, "bgk", f, mask, nsteps=int(40.0 * H * H / (nu * math.pi ** 2)), F=F)
    u, _ = _row_velocity(name, dims, f, F)
    y = np.arange(1, H + 1, dtype=float)
    exact = Fx / (2.0 * nu) * (y - 0.5) * (H + 0.5 - y)
    err = np.max(np.abs(u - exact)) / exact.max()
    assert 1e-4 < err < 0.2


@pytest.mark.parametrize("name,coll,tau", [("D2Q9", "bgk", 0.7), ("D2Q9", "regularized", 0.9),
                                           ("D3Q27", "bgk", 0.8)])
def test_couette_profile_with_moving_wall(name, coll, tau):
    # top wall moves with U along x, bottom wall rests: u(y) = U (y - 1/2) / H exactly
    H = 6
    dims, N, mask, d, w = _channel(name, H)
    U = 0.01
    wall_u = np.zeros((d, N))
    top = np.zeros((dims[2], dims[1], dims[0]), dtype=bool)
    top[:, -1, :] = True
    wall_u[0, top.reshape(-1)] = U
    f = oracle.init_eq(name, dims, np.ones(N), np.zeros((d, N)))
    nu = CS2 * (tau - 0.5)
    f = oracle.step_walls(name, dims, tau, coll, f, mask, nsteps=int(40.0 * H * H / (nu * math.pi ** 2)),
                          wall_u=wall_u)
    u, _ = _row_velocity(name, dims, f, None)
    y = np.arange(1, H + 1, dtype=float)
    np.testing.assert_allclose(u, U * (y - 0.5) / H, rtol=0, atol=1e-9 * U)


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
@pytest.mark.parametrize("wall_axis,flow_axis", [(2, 1), (0, 2), (1, 0)])
def test_couette_in_every_orientation(name, wall_axis, flow_axis):
    # walls normal to wall_axis (solid planes at index 0 and H + 1), the upper one moving with U
    # along flow_axis: the steady profile is U (s - 1/2) / H across the channel, zero elsewhere
    H, U, tau = 5, 0.01, 0.8
    d, c, w, _ = oracle.stencil(name)
    dims = [3, 3, 3]
    dims[wall_axis] = H + 2
    dims = tuple(dims)
    N = oracle.n_nodes(dims)
    idx = np.indices((dims[2], dims[1], dims[0])).reshape(3, -1)[::-1]  # x, y, z of each node
    s = idx[wall_axis]
    mask = ((s == 0) | (s == H + 1)).astype(np.uint8)
    wall_u = np.zeros((d, N))
    wall_u[flow_axis, s == H + 1] = U
    f = oracle.init_eq(name, dims, np.ones(N), np.zeros((d, N)))
    nu = CS2 * (tau - 0.5)
    f = oracle.step_walls(name, dims, tau, "bgk", f, mask, nsteps=int(40.0 * H * H / (nu * math.pi ** 2)),
                          wall_u=wall_u)
    _, u = oracle.moments(name, dims, f)
    fluid = mask == 0
    np.testing.assert_allclose(u[flow_axis, fluid], U * (s[fluid] - 0.5) / H, rtol=0, atol=1e-9 * U)
    for a in range(d):
        if a != flow_axis:
            np.testing.assert_allclose(u[a, fluid], 0.0, rtol=0, atol=1e-12 * U)
