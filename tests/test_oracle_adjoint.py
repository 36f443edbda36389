"""Pins of the oracle's hand-written discrete adjoint against the oracle's forward map.

The adjoint is checked by central finite differences of the forward solver (a
different computation: only forward steps), and for the linear streaming-only case
by the exact dot-product identity <S^n a, b> = <a, (S^n)^T b>.
"""
import math

import numpy as np
import pytest

import lbinputs
import oracle


def _linear_loss(a, f):
    return float((a * f).sum())


def _fd_check(name, dims, tau, coll, nsteps, F=None, mlp=None, seed=0, rtol=1e-6):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    rho, u = lbinputs.random_moments(dims, seed=seed, u_amp=0.06)
    f0 = oracle.init_eq(name, dims, rho, u) + 2e-3 * lbinputs.random_populations(w, N, seed + 1)
    a = lbinputs.random_field((len(w), N), seed + 2)
    lam0, gF, gth = oracle.adjoint(name, dims, tau, coll, f0, nsteps, a, F=F, mlp=mlp)

    def L(f0_, F_=F, mlp_=mlp):
        return _linear_loss(a, oracle.step(name, dims, tau, coll, f0_, nsteps=nsteps, F=F_, mlp=mlp_))

    # direction in population space
    df = lbinputs.random_field(f0.shape, seed + 3) * w[:, None]
    h = 1e-6
    fd = (L(f0 + h * df) - L(f0 - h * df)) / (2 * h)
    an = float((lam0 * df).sum())
    assert abs(fd - an) <= rtol * max(abs(fd), 1e-12), (fd, an)
    if F is not None:
        dF = lbinputs.random_field(F.shape, seed + 4)
        hF = 1e-3 * max(np.abs(F).max(), 1e-6)
        fd = (L(f0, F + hF * dF) - L(f0, F - hF * dF)) / (2 * hF)
        an = float((gF * dF).sum())
        assert abs(fd - an) <= rtol * max(abs(fd), 1e-12), (fd, an)
    if mlp is not None:
        nth = len(gth)  # trained parameters (the input shift / scale follow them)
        dth = lbinputs.random_field(nth, seed + 5)
        ht = 1e-5
        mp = mlp.copy(); mp[:nth] += ht * dth
        mm = mlp.copy(); mm[:nth] -= ht * dth
        fd = (L(f0, F, mp) - L(f0, F, mm)) / (2 * ht)
        an = float((gth * dth).sum())
        assert abs(fd - an) <= 1e2 * rtol * max(abs(fd), 1e-12), (fd, an)


@pytest.mark.parametrize("name,dims", [("D2Q9", (5, 4, 1)), ("D3Q19", (3, 4, 3)), ("D3Q27", (3, 3, 2))])
@pytest.mark.parametrize("coll", ["bgk", "regularized"])
def test_adjoint_matches_finite_differences(name, dims, coll):
    _fd_check(name, dims, 0.7, coll, nsteps=4, seed=100)


@pytest.mark.parametrize("name,dims", [("D2Q9", (5, 4, 1)), ("D3Q19", (3, 4, 3)), ("D3Q27", (3, 3, 2))])
@pytest.mark.parametrize("coll", ["bgk", "regularized"])
def test_adjoint_with_force_matches_finite_differences(name, dims, coll):
    d = 2 if dims[2] == 1 else 3
    F = lbinputs.random_field((d, oracle.n_nodes(dims)), seed=200, amp=1e-3)
    _fd_check(name, dims, 0.66, coll, nsteps=4, F=F, seed=210)


def _mlp(seed, tau):
    th = lbinputs.random_mlp_params(seed, out_bias=math.log(tau - 0.5), out_scale=0.5)
    # shifts/scales chosen so the inputs are O(1) for a near-equilibrium state
    shift = np.zeros(6)
    scale = np.array([50.0, 100.0, 300.0, 1e5, 1e5, 1e5])
    return np.concatenate([th, shift, scale])


def test_learned_adjoint_matches_finite_differences():
    _fd_check("D2Q9", (5, 4, 1), 0.6, "learned", nsteps=3, mlp=_mlp(7, 0.6), seed=300, rtol=2e-6)


def _mlp3(seed, tau):
    th = lbinputs.random_mlp3_params(seed, out_bias=math.log(tau - 0.5), out_scale=0.5)
    return np.concatenate([th, np.zeros(6), np.array([50.0, 100.0, 300.0, 1e5, 1e5, 1e5])])


def test_learned3_adjoint_matches_finite_differences():
    _fd_check("D2Q9", (5, 4, 1), 0.6, "learned3", nsteps=3, mlp=_mlp3(9, 0.6), seed=310, rtol=2e-6)


@pytest.mark.parametrize("name,dims", [("D2Q9", (5, 4, 1)), ("D3Q27", (3, 2, 3))])
def test_streaming_adjoint_dot_product_exact(name, dims):
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    a = lbinputs.random_field((len(w), N), 1)
    b = lbinputs.random_field((len(w), N), 2)
    Sa = oracle.step(name, dims, 0.8, "none", a, nsteps=3)
    STb, _, _ = oracle.adjoint(name, dims, 0.8, "none", a, 3, b)
    assert abs(float((Sa * b).sum()) - float((a * STb).sum())) < 1e-12


@pytest.mark.parametrize("name,dims", [("D2Q9", (5, 4, 1)), ("D3Q19", (3, 2, 2))])
@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("with_rho", [False, True])
def test_moment_seed_is_the_derivative_of_the_moments(name, dims, forced, with_rho):
    # L = sum_x grho rho + gu . u with (rho, u) of Eq. 4 (u = (j + F/2)/rho): lambda = dL/df and
    # the direct dL/dF, both against central differences of the oracle's moments
    d, c, w, _ = oracle.stencil(name)
    N = oracle.n_nodes(dims)
    rho, u = lbinputs.random_moments(dims, seed=40, u_amp=0.08)
    f = oracle.init_eq(name, dims, rho, u) + 2e-3 * lbinputs.random_populations(w, N, 41)
    F = lbinputs.random_field((d, N), 42, amp=1e-3) if forced else None
    grho = lbinputs.random_field(N, 43) if with_rho else None
    gu = lbinputs.random_field((d, N), 44)
    lam, gF = oracle.seed_moments(name, dims, f, grho, gu, F=F)

    def L(f_, F_=F):
        r, uu = oracle.moments(name, dims, f_, F=F_)
        return float((gu * uu).sum()) + (float((grho * r).sum()) if with_rho else 0.0)

    df = lbinputs.random_field(f.shape, 45) * w[:, None]
    h = 1e-6
    fd = (L(f + h * df) - L(f - h * df)) / (2 * h)
    assert abs(fd - float((lam * df).sum())) <= 1e-8 * abs(fd)
    if forced:
        dF = lbinputs.random_field(F.shape, 46)
        hF = 1e-6
        fd = (L(f, F + hF * dF) - L(f, F - hF * dF)) / (2 * hF)
        assert abs(fd - float((gF * dF).sum())) <= 1e-8 * abs(fd)
    else:
        assert gF is None


def test_energy_loss_seed_matches_finite_differences():
    dims = (6, 5, 1)
    N = 30
    d, c, w, _ = oracle.stencil("D2Q9")
    rho, u = lbinputs.random_moments(dims, seed=5)
    f = oracle.init_eq("D2Q9", dims, rho, u) + 1e-3 * lbinputs.random_populations(w, N, 6)
    F = lbinputs.random_field((2, N), 7, amp=1e-3)
    et = lbinputs.random_field(N, 8, amp=1e-3) + 1e-3
    L0, lam, gF = oracle.loss_energy("D2Q9", dims, f, et, F=F)
    df = lbinputs.random_field(f.shape, 9) * w[:, None]
    h = 1e-6
    fd = (oracle.loss_energy("D2Q9", dims, f + h * df, et, F=F)[0]
          - oracle.loss_energy("D2Q9", dims, f - h * df, et, F=F)[0]) / (2 * h)
    assert abs(fd - float((lam * df).sum())) < 1e-6 * abs(fd)
    dF = lbinputs.random_field(F.shape, 10)
    hF = 1e-9
    fd = (oracle.loss_energy("D2Q9", dims, f, et, F=F + hF * dF)[0]
          - oracle.loss_energy("D2Q9", dims, f, et, F=F - hF * dF)[0]) / (2 * hF)
    assert abs(fd - float((gF * dF).sum())) < 1e-5 * abs(fd)
    # closed form: L = sum (rho |u|^2 / 2 - e*)^2 with u = (j + F/2)/rho
    r, uu = oracle.moments("D2Q9", dims, f, F=F)
    assert abs(L0 - float(((0.5 * r * (uu * uu).sum(0) - et) ** 2).sum())) < 1e-15


def test_eq6_loss_seed_matches_finite_differences():
    dims = (7, 6, 1)
    N = 42
    d, c, w, _ = oracle.stencil("D2Q9")
    rho, u = lbinputs.random_moments(dims, seed=11)
    f = oracle.init_eq("D2Q9", dims, rho, u)
    uref = lbinputs.random_field((2, N), 12, amp=0.05)
    wref = lbinputs.random_field(N, 13, amp=0.02)
    L0, lam = oracle.loss_eq6(dims, f, uref, wref, 1e-3)
    df = lbinputs.random_field(f.shape, 14) * w[:, None]
    h = 1e-6
    fd = (oracle.loss_eq6(dims, f + h * df, uref, wref, 1e-3)[0]
          - oracle.loss_eq6(dims, f - h * df, uref, wref, 1e-3)[0]) / (2 * h)
    assert abs(fd - float((lam * df).sum())) < 1e-6 * abs(fd)
    # closed form of the loss with the paper's weights 0.6 / 0.2 / 0.2
    r, uu = oracle.moments("D2Q9", dims, f)
    ug = uu.reshape(2, 6, 7)
    vort = (0.5 * (np.roll(ug[1], -1, 1) - np.roll(ug[1], 1, 1))
            - 0.5 * (np.roll(ug[0], -1, 0) - np.roll(ug[0], 1, 0))).ravel()
    E = 0.5 * (uu * uu).sum() / N
    expect = 0.6 * ((uu - uref) ** 2).sum() / N + 0.2 * ((vort - wref) ** 2).sum() / N + 0.2 * (E - 1e-3) ** 2
    assert abs(L0 - expect) < 1e-15
    w2, E2 = oracle.vorticity(dims, f)
    np.testing.assert_allclose(w2, vort, atol=1e-17)


def test_vorticity_of_single_modes():
    # second-order central differences of sin(2 pi k x / n) give sin(2 pi k / n) cos(2 pi k x / n),
    # and w = dv/dx - du/dy; E = (1/2N) sum |u|^2 = (A^2 + B^2)/4 over whole periods
    nx, ny = 12, 10
    dims = (nx, ny, 1)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A, B, k, m = 0.03, 0.02, 2, 3
    u = np.stack([(B * np.sin(2 * np.pi * m * y / ny)).ravel(), (A * np.sin(2 * np.pi * k * x / nx)).ravel()])
    f = oracle.init_eq("D2Q9", dims, np.ones(nx * ny), u)
    w, E = oracle.vorticity(dims, f)
    expect = (A * math.sin(2 * math.pi * k / nx) * np.cos(2 * np.pi * k * x / nx)
              - B * math.sin(2 * math.pi * m / ny) * np.cos(2 * np.pi * m * y / ny)).ravel()
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-15)
    assert E == pytest.approx((A * A + B * B) / 4, rel=1e-13)
