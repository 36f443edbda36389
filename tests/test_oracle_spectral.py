"""Pins of the oracle's spectral flow control (Sec. 3.2): the spectrum against closed forms
of single Fourier modes and Parseval's identity, the cost gradient against finite
differences, and the velocity-shift step against BGK and its exact momentum change."""
import math

import numpy as np
import pytest

import lbinputs
import oracle
from oracle import spectral


def _mode_field(n, comps):
    """u[2][n*n] = sum of A cos(2 pi (kx x + ky y)/n + phase) per component."""
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((2, n, n))
    for a, kx, ky, A, ph in comps:
        u[a] += A * np.cos(2 * np.pi * (kx * x + ky * y) / n + ph)
    return u.reshape(2, n * n)


def _bandlimited(n, seed, amp=0.05, kmax=None):
    rng = np.random.default_rng(seed)
    kmax = kmax or n // 2 - 1
    k = np.fft.fftfreq(n, 1.0 / n)
    keep = (k[:, None] ** 2 + k[None, :] ** 2) < (kmax - 0.5) ** 2
    u = np.zeros((2, n, n))
    for a in range(2):
        c = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * keep
        u[a] = np.real(np.fft.ifft2(c))
    u *= amp / np.sqrt(np.mean(u ** 2))
    return u.reshape(2, n * n)


def test_shells_are_rounded_wavenumber_magnitudes():
    for n in (4, 8, 64, 256):
        k = np.fft.fftfreq(n, 1.0 / n)
        r = np.hypot(k[:, None], k[None, :])
        sh = spectral.shells(n)
        np.testing.assert_array_equal(sh, np.floor(r + 0.5).astype(np.int64))
        # every kept shell is closed under k -> -k (real fields give real gradients)
        kept = sh < n // 2
        np.testing.assert_array_equal(kept, np.roll(np.flip(kept, (0, 1)), 1, (0, 1)))


def test_single_modes_have_closed_form_spectra():
    n = 32
    A, B = 0.03, 0.02
    # |k| = 5 for (3, 4); |k| = 7 for (7, 0): sigma_s = 2 modes x (A/2)^2 / 2 = A^2 / 4
    u = _mode_field(n, [(0, 3, 4, A, 0.3), (1, 7, 0, B, -1.1)])
    s = spectral.spectrum(u, n)
    expect = np.zeros(n // 2)
    expect[5] = A * A / 4
    expect[7] = B * B / 4
    np.testing.assert_allclose(s, expect, rtol=0, atol=1e-18)


def test_parseval_for_band_limited_fields():
    n = 64
    u = _bandlimited(n, seed=3)
    s = spectral.spectrum(u, n)
    assert math.isclose(s.sum(), 0.5 * np.mean(np.sum(u ** 2, axis=0)), rel_tol=1e-13)


def test_zero_cost_and_gradient_at_the_target():
    n = 32
    u = _bandlimited(n, seed=4)
    s0 = spectral.spectrum(u, n)
    assert spectral.cost(u, n, s0) == 0.0
    assert np.max(np.abs(spectral.cost_gradient(u, n, s0))) == 0.0


@pytest.mark.parametrize("c", [1e-12, spectral.CUTOFF])
def test_gradient_matches_central_differences(c):
    n = 16
    u = _bandlimited(n, seed=5, amp=0.05)
    s = spectral.spectrum(u, n)
    if c == spectral.CUTOFF:
        # shells well below the cutoff (no gradient) and well above it; none near it
        live = s > c
        assert live.any() and (~live).any()
        assert np.all(np.abs(np.log(s[s > 0] / c)) > 0.05)
    s0 = s * np.exp(0.3 * lbinputs.random_field(n // 2, seed=6))
    g = spectral.cost_gradient(u, n, s0, c)
    rng = np.random.default_rng(7)
    h = 1e-7
    for _ in range(12):
        a, x = int(rng.integers(2)), int(rng.integers(n * n))
        up, um = u.copy(), u.copy()
        up[a, x] += h
        um[a, x] -= h
        fd = (spectral.cost(up, n, s0, c) - spectral.cost(um, n, s0, c)) / (2 * h)
        assert fd == pytest.approx(g[a, x], rel=1e-5, abs=1e-9 * np.max(np.abs(g)))


def test_shift_step_with_zero_shift_is_bgk():
    n = 16
    dims = (n, n, 1)
    rho, u = lbinputs.random_moments(dims, seed=8, u_amp=0.05)
    f = oracle.init_eq("D2Q9", dims, rho, u)
    a = oracle.step_ushift("D2Q9", dims, 0.7, f, np.zeros((2, n * n)), nsteps=3)
    b = oracle.step("D2Q9", dims, 0.7, "bgk", f, nsteps=3)
    np.testing.assert_array_equal(a, b)


def test_shift_step_changes_momentum_by_omega_rho_du():
    n = 16
    dims = (n, n, 1)
    d, c, w, _ = oracle.stencil("D2Q9")
    rho, u = lbinputs.random_moments(dims, seed=9, u_amp=0.05)
    f = oracle.init_eq("D2Q9", dims, rho, u) * (1 + 0.01 * lbinputs.random_field((9, n * n), 10))
    du = 1e-3 * lbinputs.random_field((2, n * n), 11)
    tau = 0.8
    r0, u0 = oracle.moments("D2Q9", dims, f)
    g = oracle.step_ushift("D2Q9", dims, tau, f, du)
    r1, u1 = oracle.moments("D2Q9", dims, g)
    assert abs(r1.sum() - r0.sum()) <= 1e-13 * r0.sum()
    dP = (r1 * u1).sum(axis=1) - (r0 * u0).sum(axis=1)
    np.testing.assert_allclose(dP, (r0 * du).sum(axis=1) / tau, rtol=1e-9, atol=1e-16)


def test_control_keeps_the_spectrum_closer_than_the_free_flow():
    """The sign and scale of du: after 150 steps the controlled flow's cost is below the
    free (plain BGK) flow's, started from the same decaying field with sigma_0 = sigma(u_0)."""
    n = 32
    dims = (n, n, 1)
    rho, u = lbinputs.random_spectrum_velocity(dims, 4.0, 0.05, 2000)
    tau = 0.5 + 3.0 * 0.05 * (n / (2 * np.pi)) / 2000.0
    f0 = oracle.init_eq("D2Q9", dims, rho, u)
    s0 = spectral.spectrum(u, n)
    free = oracle.step("D2Q9", dims, tau, "bgk", f0, nsteps=150)
    ctrl = spectral.run(n, tau, f0, s0, 150, kappa=1e-3)
    Rf = spectral.cost(oracle.moments("D2Q9", dims, free)[1], n, s0)
    Rc = spectral.cost(oracle.moments("D2Q9", dims, ctrl)[1], n, s0)
    assert Rc < 0.5 * Rf, (Rc, Rf)


def test_constants_are_the_papers():
    import os
    const = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                const[k] = float(v)
    assert spectral.CUTOFF == const["spectrum_cutoff"]
    assert spectral.KAPPA == const["force_constant"]
    # the paper-shaped network: one hidden layer, parameter count within 1 % of the paper's
    assert const["net_hidden_layers"] == 1
    assert abs(oracle.N_THETA3 - const["net_parameters"]) <= 0.01 * const["net_parameters"]
