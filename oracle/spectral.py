"""FP64 oracle of the spectral flow control of Sec. 3.2 (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module; the product library never loads it.

Sec. 3.2 keeps a 2D flow's energy spectrum sigma(u) near a target sigma_0 by the cost
    R(u) = || ln max(sigma(u), c) - ln max(sigma_0, c) ||_2^2     (elementwise max and log)
and a velocity-shift forcing: every step the equilibrium is taken at u + du with
du = -kappa grad_u R (c = 2e-5, kappa = 5e-5 in the paper). Written out here, with numpy's
FFT as a library step and everything else in plain numpy:

  - u_hat_a(k) = (1/N) sum_x u_a(x) exp(-2 pi i k.x / n), the normalised DFT of each
    velocity component on the periodic n x n grid (k in numpy's signed frequency order);
  - the shell of a mode is round(|k|), computed in exact integer arithmetic; shells
    0 .. n/2 - 1 are kept (the corner modes with |k| >= n/2 - 1/2 are not part of sigma);
  - sigma_s = sum over the modes of shell s of (|u_hat_x|^2 + |u_hat_y|^2) / 2;
  - grad_u R by the chain rule: dR/dsigma_s = 2 (ln sigma_s - ln max(sigma0_s, c)) / sigma_s
    where sigma_s > c, else 0 (max is flat there); d sigma_s / d(Re, Im) u_hat = (Re, Im) u_hat;
    and back through the DFT (the transpose of (1/N) exp(-i theta) on real input), which is
    Re(ifft2(G u_hat)) with G(k) = dR/dsigma of k's shell (0 outside the kept shells).

Readings (the paper defines neither the spectrum's normalisation nor its shells): the
spectrum is the shell sum of the normalised modal energy (Parseval: the sum over all modes
is (1/2N) sum_x |u|^2), shells by rounding |k|, and the target is the initial spectrum.
Parity is pinned by closed forms (single Fourier modes), Parseval, finite differences of R
and the zero-cost special case (tests/test_oracle_spectral.py).
"""
from __future__ import annotations

import numpy as np

from . import moments, step_ushift

CUTOFF = 2e-5   # c of Sec. 3.2
KAPPA = 5e-5    # kappa of Sec. 3.2


def _freq(n: int) -> np.ndarray:
    return np.fft.fftfreq(n, 1.0 / n).astype(np.int64)


def shells(n: int) -> np.ndarray:
    """Shell index round(|k|) of every mode [ky][kx] of an n x n grid (exact integers)."""
    k = _freq(n)
    m = k[:, None] ** 2 + k[None, :] ** 2
    r = np.floor(np.sqrt(m.astype(np.float64))).astype(np.int64)
    r = np.where(r * r > m, r - 1, r)
    r = np.where((r + 1) * (r + 1) <= m, r + 1, r)   # r = floor(sqrt(m)) exactly
    return np.where(4 * m >= (2 * r + 1) ** 2, r + 1, r)  # round half up never ties for integer m


def _uhat(u: np.ndarray, n: int) -> np.ndarray:
    u = np.asarray(u, dtype=np.float64).reshape(2, n, n)
    return np.fft.fft2(u, axes=(1, 2)) / (n * n)


def spectrum(u: np.ndarray, n: int) -> np.ndarray:
    """sigma[n/2]: shell sums of (|u_hat_x|^2 + |u_hat_y|^2)/2 of a velocity field u[2][n*n]."""
    uh = _uhat(u, n)
    e = 0.5 * (np.abs(uh[0]) ** 2 + np.abs(uh[1]) ** 2)
    sh = shells(n)
    K = n // 2
    keep = sh < K
    return np.bincount(sh[keep], weights=e[keep], minlength=K)[:K]


def cost(u: np.ndarray, n: int, sigma0: np.ndarray, c: float = CUTOFF) -> float:
    s = spectrum(u, n)
    return float(np.sum((np.log(np.maximum(s, c)) - np.log(np.maximum(sigma0, c))) ** 2))


def cost_gradient(u: np.ndarray, n: int, sigma0: np.ndarray, c: float = CUTOFF) -> np.ndarray:
    """dR/du[2][n*n] by the chain rule through sigma and the DFT."""
    uh = _uhat(u, n)
    s = spectrum(u, n)
    K = n // 2
    live = s > c
    dRds = np.zeros(K)
    dRds[live] = 2.0 * (np.log(s[live]) - np.log(np.maximum(sigma0[live], c))) / s[live]
    sh = shells(n)
    G = np.where(sh < K, dRds[np.minimum(sh, K - 1)], 0.0)
    # d sigma / d(Re u_hat, Im u_hat) = (Re u_hat, Im u_hat); the transpose of u -> fft2(u)/N
    # maps a complex cotangent Y to Re(sum_k Y(k) exp(+i theta)) / N = Re(ifft2(Y))
    g = np.real(np.fft.ifft2(G[None] * uh, axes=(1, 2)))
    return g.reshape(2, n * n)


def velocity_shift(u, n, sigma0, c=CUTOFF, kappa=KAPPA):
    """du = -kappa grad_u R."""
    return -kappa * cost_gradient(u, n, sigma0, c)


def run(n: int, tau: float, f: np.ndarray, sigma0: np.ndarray, nsteps: int, c: float = CUTOFF,
        kappa: float = KAPPA) -> np.ndarray:
    """nsteps controlled BGK steps of a D2Q9 state f[9][n*n]: each step takes du from the
    current pre-collision velocity and collides with f^eq(rho, u + du)."""
    dims = (n, n, 1)
    for _ in range(nsteps):
        _, u = moments("D2Q9", dims, f)
        f = step_ushift("D2Q9", dims, tau, f, velocity_shift(u, n, sigma0, c, kappa))
    return f


__all__ = ["CUTOFF", "KAPPA", "shells", "spectrum", "cost", "cost_gradient", "velocity_shift", "run"]
