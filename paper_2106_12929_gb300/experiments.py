"""Workload drivers for the paper's flows, run through liblb on one GPU.

Each function runs one experiment and returns a dict of numbers; the tests call
them at small sizes, and ``python -m paper_2106_12929_gb300.experiments <name>``
runs them at the full sizes and prints one JSON line.

  tgv2d_decay        2D Taylor-Green vortex: fitted energy decay rate vs exp(-4 nu k^2 t)
  tgv3d_precision    3D Taylor-Green vortex: kinetic-energy error of FP32 / FP16 / BF16
                     storage against the FP64 run of the same lattice
  turbulence_precision  D3Q27 regularized decaying isotropic turbulence: energy and
                     dissipation (-dE/dt) error of each storage type against FP64
  adjoint_fd         gradient of the energy-field loss w.r.t. the body force: FP32 adjoint
                     against central finite differences of the FP64 forward run
  spectral_control   Sec. 3.2: decaying 2D turbulence with and without the spectral flow
                     control that holds the initial spectrum (cost R and energy over time)
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

import lbinputs

from .lattice import Lattice


def _energy_history(lat: Lattice, steps: int, every: int):
    ts, Es, Erho = [], [], []
    t = 0
    while True:
        r = lat.reduce()
        ts.append(t)
        Es.append(r[4])
        Erho.append(r[5])
        if t >= steps:
            break
        k = min(every, steps - t)
        lat.step(k)
        t += k
    lat.check()
    return np.array(ts, dtype=np.float64), np.array(Es), np.array(Erho)


def tgv2d_decay(n: int = 64, tau: float = 0.8, u0: float = 0.05, steps: int = 1000, storage: str = "f64",
                fit_from: int = 100, every: int = 10):
    """Least-squares slope of ln E over [fit_from, steps] against -4 nu k^2 with
    nu = c_s^2 (tau - 1/2) and k = 2 pi / n (the BGK viscosity of Sec. 2.1)."""
    dims, rho, u = lbinputs.taylor_green_2d(n, u0=u0)
    lat = Lattice("D2Q9", dims, tau, "bgk", storage=storage)
    lat.init_from_moments(rho, u)
    ts, Es, _ = _energy_history(lat, steps, every)
    lat.close()
    sel = ts >= fit_from
    slope = float(np.polyfit(ts[sel], np.log(Es[sel]), 1)[0])
    nu = (tau - 0.5) / 3.0
    k = 2.0 * math.pi / n
    theory = -4.0 * nu * k * k
    return {"n": n, "tau": tau, "steps": steps, "storage": storage, "slope": slope, "theory": theory,
            "rel_err": abs(slope / theory - 1.0), "E0": float(Es[0]), "E_end": float(Es[-1])}


def tgv3d_precision(n: int = 64, steps: int = 1000, storages=("f32", "f16", "bf16"), re: float = 1600.0,
                    every: int = 20, layout: str = "ab"):
    """Max over t of |E_s(t) - E_64(t)| / E_64(t) for the 3D TGV at Re 1600, Ma 0.1."""
    u0 = 0.1 / math.sqrt(3.0)
    tau = lbinputs.tau_from_reynolds(re, u0, n)
    dims, rho, u = lbinputs.taylor_green_3d(n, u0=u0)
    rho_d = torch.tensor(rho, device="cuda")
    u_d = torch.tensor(u, device="cuda")
    hist = {}
    for st in ("f64",) + tuple(storages):
        lat = Lattice("D3Q19", dims, tau, "bgk", storage=st, layout=layout)
        lat.init_from_moments(rho_d, u_d)
        ts, Es, _ = _energy_history(lat, steps, every)
        hist[st] = Es
        lat.close()
    out = {"n": n, "steps": steps, "tau": tau, "E0": float(hist["f64"][0]), "E_end_f64": float(hist["f64"][-1])}
    for st in storages:
        out[f"energy_rel_err_{st}"] = float(np.max(np.abs(hist[st] - hist["f64"]) / hist["f64"]))
    return out


def turbulence_precision(n: int = 384, steps: int = 1000, storages=("f32", "f16", "bf16"), k0: float = 8.0,
                         u_rms: float = 0.04, seed: int = 2106, re: float = 3000.0, every: int = 20):
    """D3Q27 regularized decaying isotropic turbulence (random-phase field with
    E(k) ~ k^4 exp(-2 (k/k0)^2)): per storage type the max relative error of E(t) and of
    the dissipation -dE/dt (central differences of E) against the FP64 run, and GLUPS."""
    tau = 0.5 + 3.0 * u_rms * (n / (2.0 * math.pi)) / re
    dims = (n, n, n)
    rho, u = lbinputs.random_spectrum_velocity(dims, k0, u_rms, seed)
    rho_d = torch.tensor(rho, device="cuda")
    u_d = torch.tensor(u, device="cuda")
    hist, glups = {}, {}
    for st in ("f64",) + tuple(storages):
        lat = Lattice("D3Q27", dims, tau, "regularized", storage=st)
        lat.init_from_moments(rho_d, u_d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ts, Es, _ = _energy_history(lat, steps, every)
        torch.cuda.synchronize()
        glups[st] = n ** 3 * steps / (time.perf_counter() - t0) / 1e9
        hist[st] = Es
        lat.close()
    ref = hist["f64"]
    diss_ref = -np.gradient(ref, every)
    out = {"n": n, "steps": steps, "tau": tau, "E0": float(ref[0]), "E_end_f64": float(ref[-1]),
           "glups_with_reductions": {k: round(v, 3) for k, v in glups.items()}}
    for st in storages:
        out[f"energy_rel_err_{st}"] = float(np.max(np.abs(hist[st] - ref) / ref))
        diss = -np.gradient(hist[st], every)
        out[f"dissipation_rel_err_{st}"] = float(np.max(np.abs(diss - diss_ref)) / np.max(np.abs(diss_ref)))
    return out


def adjoint_fd(n: int = 64, steps: int = 50, k: int = 10, tau: float = 0.51, u0: float = 0.05,
               seed: int = 12929, h_rel: float = 1e-3):
    """Energy-field loss L = sum_x (e(x) - e*(x))^2 of a forced D2Q9 shear layer after
    `steps` steps, e* a seeded smooth target field. dL/dF by the adjoint (checkpoints every
    k) in FP32 and in FP64, against central differences of the FP64 forward run along three
    smooth seeded directions and one random direction."""
    dims, rho, u = lbinputs.shear_layer(n, u0=u0)
    N = n * n
    F0 = lbinputs.smooth_force(dims, 1e-5, seed=seed)
    et = torch.tensor(lbinputs.smooth_scalar(dims, 0.5 * u0 * u0, 0.5, seed + 1), device="cuda")

    def gradient(storage):
        rdt = torch.float64 if storage == "f64" else torch.float32
        lat = Lattice("D2Q9", dims, tau, "bgk", storage=storage, record_every=k)
        lat.set_force(torch.tensor(F0, dtype=rdt, device="cuda"))
        lat.init_from_moments(rho, u)
        lat.step(steps)
        gF = torch.zeros((2, N), dtype=rdt, device="cuda")
        L, lamT = lat.loss_energy(et.to(rdt), grad_F=gF)
        lat.step_adjoint(lamT, steps, grad_F=gF, want_lambda0=False)
        lat.close()
        return L, gF.double().cpu().numpy()

    L32, g32 = gradient("f32")
    L64, g64 = gradient("f64")
    fwd = Lattice("D2Q9", dims, tau, "bgk", storage="f64")

    def loss(F):
        fwd.set_force(F)
        fwd.init_from_moments(rho, u)
        fwd.step(steps)
        return fwd.loss_energy(et)[0]

    dirs = [lbinputs.smooth_force(dims, 1.0, seed=seed + 10 + j) for j in range(3)]
    dirs.append(np.random.default_rng(seed).uniform(-1, 1, size=(2, N)))
    h = h_rel * np.abs(F0).max()
    err32, err64 = [], []
    for d in dirs:
        fd = (loss(F0 + h * d) - loss(F0 - h * d)) / (2 * h)
        err32.append(abs(float((g32 * d).sum()) - fd) / abs(fd))
        err64.append(abs(float((g64 * d).sum()) - fd) / abs(fd))
    fwd.close()
    return {"n": n, "steps": steps, "k": k, "tau": tau, "loss_f64": L64, "loss_f32": L32,
            "fd_rel_err_f32": float(max(err32)), "fd_rel_err_f64": float(max(err64)),
            "f32_vs_f64_adjoint_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
            "dir_errs_f32": err32, "dir_errs_f64": err64}


def spectral_control(n: int = 128, steps: int = 2000, kappa: float = 5e-4, cutoff: float = 2e-5,
                     re: float = 2000.0, k0: float = 8.0, seed: int = 2000, storage: str = "f32", every: int = 250):
    """Sec. 3.2's flow control on random-phase 2D turbulence (n^2, Ma 0.1, tau from Re on the
    length n / (2 pi)): a free BGK run and a controlled run whose target is the initial
    spectrum. Reports the cost R and the kinetic energy (1/2N) sum |u|^2 every ``every`` steps
    and the final spectra. The free run's R is read by switching the control on with kappa = 0
    for the report only, so its steps stay plain BGK."""
    u0 = 0.1 / math.sqrt(3.0)
    dims = (n, n, 1)
    rho, u = lbinputs.random_spectrum_velocity(dims, k0, u0, seed)
    tau = lbinputs.tau_from_reynolds(re, u0, n)
    out = {"n": n, "steps": steps, "tau": tau, "kappa": kappa, "cutoff": cutoff, "storage": storage}
    sigma0 = None
    for name in ("free", "controlled"):
        lat = Lattice("D2Q9", dims, tau, "bgk", storage=storage, check_every=500)
        lat.init_from_moments(rho, u)
        if sigma0 is None:
            sigma0 = lat.spectrum()
        if name == "controlled":
            lat.set_spectral_control(sigma0, cutoff=cutoff, kappa=kappa)
        ts, Es, Rs = [], [], []
        t = 0
        while True:
            if name == "free":
                lat.set_spectral_control(sigma0, cutoff=cutoff, kappa=0.0)
            sig, R = lat.spectrum(with_cost=True)
            if name == "free":
                lat.set_spectral_control(None)
            ts.append(t)
            Es.append(float(lat.reduce()[4]))
            Rs.append(float(R))
            if t >= steps:
                break
            k = min(every, steps - t)
            lat.step(k)
            t += k
        lat.check()
        out[name] = {"t": ts, "E": Es, "R": Rs, "sigma_final": sig.tolist()}
        lat.close()
    out["sigma0"] = sigma0.tolist()
    out["E0"] = out["free"]["E"][0]
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("name", choices=["tgv2d_decay", "tgv3d_precision", "turbulence_precision", "adjoint_fd",
                                     "spectral_control"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    a = ap.parse_args()
    kw = {}
    if a.n is not None:
        kw["n"] = a.n
    if a.steps is not None:
        kw["steps"] = a.steps
    fn = globals()[a.name]
    t0 = time.perf_counter()
    res = fn(**kw)
    res["experiment"] = a.name
    res["wall_s"] = round(time.perf_counter() - t0, 2)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
