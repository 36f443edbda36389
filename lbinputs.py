"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module only builds initial fields, force fields and random arrays. It holds
none of the lattice Boltzmann arithmetic (no equilibrium, collision, streaming or
moment sums), so both solvers can be fed the same FP64 arrays without sharing
method code. All arrays use the node order x fastest, then y, then z, i.e. a flat
index ``n = x + nx*(y + ny*z)``; a vector field is stored component-major,
``u[a][n]``.

Workloads (the paper runs analytic or seeded flows only; Sec. 2.2, 3.1, 3.3):
  * 2D Taylor-Green vortex with its pressure perturbation (Sec. 3.3 benchmark flow);
  * 3D Taylor-Green vortex in Brachet's form (Sec. 2.2 code example, Fig. 2);
  * doubly periodic shear layer (Sec. 3.1 training flow);
  * random-phase decaying isotropic turbulence with E(k) ~ k^4 exp(-2 (k/k0)^2)
    (Sec. 3.1 transfer flow, Sec. 3.2 flow-control flow);
  * a smooth seeded body-force field and near-equilibrium random populations;
  * solid masks for walls: a seeded random obstacle field and a duct with a cylinder or
    sphere.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared, used only for unit conversion


def _grid(dims):
    nx, ny, nz = (int(d) for d in dims)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64).ravel(), y.astype(np.float64).ravel(), z.astype(np.float64).ravel()


def tau_from_nu(nu: float) -> float:
    """Relaxation time for kinematic viscosity nu (lattice units, c_s^2 = 1/3)."""
    return nu / CS2 + 0.5


def tau_from_reynolds(re: float, u0: float, n: int) -> float:
    """Relaxation time of a periodic box of n nodes per side at Reynolds number re.

    The length scale is n/(2 pi): the box is read as a 2 pi-periodic domain, the
    convention of the Taylor-Green benchmark (Sec. 2.2). nu = u0 L / Re.
    """
    length = n / (2.0 * math.pi)
    return tau_from_nu(u0 * length / re)


def taylor_green_2d(n: int, u0: float = 0.05, ny: int | None = None):
    """2D Taylor-Green vortex on an n x ny periodic grid (node coordinates x = i).

    u = u0 sin(kx) cos(ky), v = -u0 cos(kx) sin(ky), k = 2 pi / n,
    p = (u0^2/4) (cos 2kx + cos 2ky), rho = 1 + p / c_s^2: the pressure in balance with this
    field (lap p = -d_i d_j (u_i u_j); highest at the stagnation points x = y = 0).
    Returns (dims, rho[N], u[2][N]) in FP64.
    """
    ny = n if ny is None else ny
    dims = (n, ny, 1)
    x, y, _ = _grid(dims)
    kx = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    u = np.empty((2, x.size))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y)
    p = (u0 * u0 / 4.0) * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    rho = 1.0 + p / CS2
    return dims, rho, u


def taylor_green_3d(n: int, u0: float = 0.1 * math.sqrt(CS2)):
    """3D Taylor-Green vortex (Brachet form) on an n^3 periodic grid.

    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0,
    p = (u0^2/16)(cos 2kx + cos 2ky)(cos 2kz + 2), rho = 1 + p / c_s^2.
    """
    dims = (n, n, n)
    x, y, z = _grid(dims)
    k = 2.0 * math.pi / n
    u = np.empty((3, x.size))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    u[2] = 0.0
    p = (u0 * u0 / 16.0) * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
    rho = 1.0 + p / CS2
    return dims, rho, u


def shear_layer(n: int, u0: float = 0.05, ny: int | None = None):
    """Doubly periodic shear layer (the Sec. 3.1 training flow, thin-layer form).

    With node coordinates x = i/n, y = j/ny:
    u = u0 tanh(80 (y - 0.25)) for y <= 0.5, u0 tanh(80 (0.75 - y)) above;
    v = 0.05 u0 sin(2 pi (x + 0.25)); rho = 1.
    """
    ny = n if ny is None else ny
    dims = (n, ny, 1)
    xi, yi, _ = _grid(dims)
    x = xi / n
    y = yi / ny
    u = np.empty((2, xi.size))
    u[0] = np.where(y <= 0.5, u0 * np.tanh(80.0 * (y - 0.25)), u0 * np.tanh(80.0 * (0.75 - y)))
    u[1] = 0.05 * u0 * np.sin(2.0 * math.pi * (x + 0.25))
    rho = np.ones(xi.size)
    return dims, rho, u


def random_spectrum_velocity(dims, k0: float, u_rms: float, seed: int):
    """Random-phase solenoidal velocity field with E(k) ~ k^4 exp(-2 (k/k0)^2).

    Each integer wavevector kappa gets amplitude sqrt(E(|kappa|) / shell count)
    and a uniform random phase (numpy PCG64 from ``seed``); the field is projected
    onto its divergence-free part, transformed back to real space and scaled so
    that the rms of a component, averaged over the components (sqrt(mean |u|^2 / d)),
    equals u_rms. rho = 1.
    """
    nx, ny, nz = (int(d) for d in dims)
    d = 2 if nz == 1 else 3
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx) if d == 3 else (ny, nx)
    ks = [np.fft.fftfreq(s, 1.0 / s) for s in shape]
    kk = np.meshgrid(*ks, indexing="ij")
    kmag = np.sqrt(sum(k * k for k in kk))
    shell = np.rint(kmag).astype(np.int64)
    counts = np.bincount(shell.ravel())
    with np.errstate(divide="ignore", invalid="ignore"):
        spec = kmag ** 4 * np.exp(-2.0 * (kmag / k0) ** 2)
        amp = np.sqrt(spec / np.maximum(counts[shell], 1))
    amp[kmag == 0] = 0.0
    comps = []
    for _ in range(d):
        phase = rng.uniform(0.0, 2.0 * math.pi, size=shape)
        comps.append(amp * np.exp(1j * phase))
    # kk is ordered like `shape` (slowest axis first); velocity components are (x, y[, z])
    kvec = list(reversed(kk))
    k2 = np.where(kmag == 0, 1.0, kmag * kmag)
    div = sum(kvec[a] * comps[a] for a in range(d))
    comps = [comps[a] - kvec[a] * div / k2 for a in range(d)]
    fields = [np.fft.ifftn(c).real for c in comps]
    rms = math.sqrt(sum(float(np.mean(f * f)) for f in fields) / d)
    u = np.empty((3 if d == 3 else 2, nx * ny * nz))
    for a in range(d):
        u[a] = (fields[a] * (u_rms / rms)).ravel()
    rho = np.ones(nx * ny * nz)
    return rho, u


def balanced_density(dims, u):
    """rho = 1 + p / c_s^2 (c_s^2 = 1/3) with p the incompressible pressure of the periodic
    velocity field u[d][N]: lap p = -d_i d_j (u_i u_j), solved spectrally (p has zero mean).
    A field started at this density is in pressure balance, so it does not launch the
    acoustic waves that rho = 1 does."""
    nx, ny, nz = (int(d) for d in dims)
    d = 2 if nz == 1 else 3
    shape = (nz, ny, nx) if d == 3 else (ny, nx)
    ks = [np.fft.fftfreq(s, 1.0 / s) * (2.0 * math.pi / s) for s in shape]
    kk = np.meshgrid(*ks, indexing="ij")
    kvec = list(reversed(kk))  # components (x, y[, z])
    uf = [np.asarray(u[a]).reshape(shape) for a in range(d)]
    rhs = np.zeros(shape, dtype=np.complex128)
    for i in range(d):
        for j in range(d):
            rhs += kvec[i] * kvec[j] * np.fft.fftn(uf[i] * uf[j])  # FFT of -d_i d_j (u_i u_j)
    k2 = sum(k * k for k in kvec)
    k2[(0,) * d] = 1.0
    ph = -rhs / k2  # -k^2 p_hat = FFT(-d_i d_j u_i u_j)
    ph[(0,) * d] = 0.0
    p = np.fft.ifftn(ph).real
    return (1.0 + 3.0 * p).ravel()


def smooth_force(dims, amplitude: float, seed: int, modes: int = 4):
    """Seeded smooth body-force field F[d][N]: a sum of the lowest Fourier modes.

    Each component is sum_{m=1..modes} a_m sin(2 pi m x/nx + p_m) cos(2 pi m y/ny + q_m)
    (times a z factor in 3D) with seeded a_m in [-1, 1] and phases, scaled so that
    max |F| = amplitude.
    """
    nx, ny, nz = (int(v) for v in dims)
    d = 2 if nz == 1 else 3
    x, y, z = _grid(dims)
    rng = np.random.default_rng(seed)
    F = np.zeros((d, x.size))
    for a in range(d):
        for m in range(1, modes + 1):
            c, p, q, r = rng.uniform(-1, 1), rng.uniform(0, 6.28), rng.uniform(0, 6.28), rng.uniform(0, 6.28)
            term = c * np.sin(2 * math.pi * m * x / nx + p) * np.cos(2 * math.pi * m * y / ny + q)
            if d == 3:
                term = term * np.cos(2 * math.pi * m * z / nz + r)
            F[a] += term
        F[a] *= amplitude / max(np.abs(F[a]).max(), 1e-300)
    return F


def smooth_scalar(dims, mean: float, rel_amp: float, seed: int, modes: int = 4):
    """Seeded smooth positive scalar field mean * (1 + rel_amp * s(x)), s a sum of the lowest
    Fourier modes scaled to max |s| = 1 (used as a target field of a loss)."""
    s = smooth_force(dims, 1.0, seed, modes)[0]
    return mean * (1.0 + rel_amp * s)


def random_moments(dims, seed: int, u_amp: float = 0.05, rho_amp: float = 0.02):
    """Seeded random (rho, u) fields: rho = 1 + rho_amp r, u = u_amp r', r uniform in [-1, 1]."""
    nx, ny, nz = (int(v) for v in dims)
    d = 2 if nz == 1 else 3
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, size=n)
    u = u_amp * rng.uniform(-1, 1, size=(d, n))
    return rho, u


def random_populations(scale, n_nodes: int, seed: int, eps: float = 0.05):
    """Seeded positive populations f[i][n] = scale[i] (1 + eps r), r uniform in [-1, 1].

    ``scale`` is a per-direction magnitude supplied by the caller (the weights of a
    velocity set); passing it in keeps this module free of stencil tables.
    """
    scale = np.asarray(scale, dtype=np.float64)
    rng = np.random.default_rng(seed)
    return scale[:, None] * (1.0 + eps * rng.uniform(-1, 1, size=(scale.size, n_nodes)))


def random_field(shape, seed: int, amp: float = 1.0):
    """Seeded uniform random FP64 array in [-amp, amp]."""
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1, 1, size=shape)


def random_mlp_params(seed: int, n_in: int = 6, n_hidden: int = 24, out_bias: float = 0.0,
                      out_scale: float = 0.0):
    """Seeded Xavier-uniform parameters of an n_in -> n_hidden -> n_hidden -> 1 tanh MLP.

    Flat layout: W1[n_hidden][n_in], b1[n_hidden], W2[n_hidden][n_hidden], b2[n_hidden],
    W3[n_hidden], b3. The output layer is scaled by ``out_scale`` (0 gives a network
    whose output is exactly ``out_bias``) and its bias set to ``out_bias``.
    """
    rng = np.random.default_rng(seed)

    def xavier(fan_out, fan_in):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    w1 = xavier(n_hidden, n_in)
    b1 = np.zeros(n_hidden)
    w2 = xavier(n_hidden, n_hidden)
    b2 = np.zeros(n_hidden)
    w3 = xavier(1, n_hidden).ravel() * out_scale
    b3 = np.array([out_bias])
    return np.concatenate([w1.ravel(), b1, w2.ravel(), b2, w3, b3])


def random_solid_mask(dims, seed: int, fraction: float = 0.2):
    """Seeded random solid mask (uint8 [N], x fastest): each node solid with the given
    probability (obstacle fields for tests)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    return (rng.uniform(0.0, 1.0, size=n) < fraction).astype(np.uint8)


def duct_with_obstacle(dims, radius: float, center=None):
    """Solid mask (uint8 [N], x fastest) of a duct: walls on the planes y = 0, y = ny - 1 (and
    z = 0, z = nz - 1 in 3D), periodic along x, plus a cylinder (2D) or sphere (3D) of the
    given radius centred at `center` (default: a quarter of the length, mid-section)."""
    nx, ny, nz = (int(v) for v in dims)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = center if center is not None else (nx / 4.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    m = (y == 0) | (y == ny - 1)
    if nz > 1:
        m |= (z == 0) | (z == nz - 1)
        m |= (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius ** 2
    else:
        m |= (x - cx) ** 2 + (y - cy) ** 2 <= radius ** 2
    return m.reshape(-1).astype(np.uint8)


def random_mlp3_params(seed: int, n_in: int = 6, n_hidden: int = 53, out_bias=0.0, out_scale: float = 0.0):
    """Seeded Xavier-uniform parameters of an n_in -> n_hidden (tanh) -> 3 network.

    Flat layout: W1[n_hidden][n_in], b1[n_hidden], W2[3][n_hidden], b2[3]. The output layer
    is scaled by ``out_scale`` and its biases set to ``out_bias`` (a scalar or three values).
    """
    rng = np.random.default_rng(seed)

    def xavier(fan_out, fan_in):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    w1 = xavier(n_hidden, n_in)
    b1 = np.zeros(n_hidden)
    w2 = xavier(3, n_hidden) * out_scale
    b2 = np.broadcast_to(np.asarray(out_bias, dtype=np.float64), (3,)).copy()
    return np.concatenate([w1.ravel(), b1, w2.ravel(), b2])
