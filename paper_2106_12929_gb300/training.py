"""Training and evaluation of the learned collision (Sec. 3.1), driven through liblb.

Training (Sec. 3.1): a fine BGK run of the doubly periodic shear layer produces
snapshots; each snapshot is mapped onto a grid of half the resolution
(``lb_coarsen_into``: block means of rho and rho u, equilibrium populations) and
a coarse run with the learned collision is started from it. After ``horizon``
coarse steps (2 x horizon fine steps) its velocity, vorticity and energy are
compared with the coarsened fine state by the Eq. 6 loss (``lb_loss_eq6``); the
gradient w.r.t. the network parameters comes from the checkpointed adjoint
(``lb_step_adjoint``) and Adam (``lb_adam_update``) updates them. Two networks:
``"learned"`` (6-24-24-1, one rate shared by the higher moments, 793 parameters) and
``"learned3"`` (the shape Sec. 3.1 describes: one hidden layer of 53 units and one rate
per higher moment, 533 parameters). Every step of
this runs in liblb's kernels; this module only orders the calls.

The network starts as BGK exactly (output weights 0, output bias ln(tau - 1/2)),
so the untrained model is the plain method and any gain is measured against it.

Evaluation (Sec. 3.1, transfer): decaying 2D turbulence with
E(k) ~ k^4 exp(-2 (k/k0)^2) on the coarse grid with the learned collision and
with BGK, against the coarsened run of the fine grid with BGK: Eq. 6 loss,
energy and enstrophy over time, and the high-wavenumber energy spectrum.

Scale conventions (acoustic scaling, lattice velocity fixed): coarse
tau_c = 1/2 + (tau_f - 1/2) / 2; one coarse step spans two fine steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import asdict, dataclass, field

import numpy as np
import torch

import lbinputs

from . import _lib
from .lattice import Lattice, adam_update
from .slab import allreduce_gradient


def coarse_tau(tau_f: float) -> float:
    return 0.5 + (tau_f - 0.5) / 2.0


@dataclass
class TrainConfig:
    n_fine: int = 1024          # fine shear-layer grid (coarse = n_fine / 2)
    tau_fine: float = 0.503     # low viscosity: the coarse grid under-resolves the layer
    u0: float = 0.05
    spinup: int = 4000          # fine steps before the first snapshot
    snap_every: int = 400       # fine steps between snapshots
    n_snap: int = 16
    holdout: int = 4            # last snapshots: test set; the `holdout` before them: validation
    horizon: int = 100          # coarse steps per rollout
    batch: int = 4
    iters: int = 300
    lr: float = 0.05
    record_every: int = 10
    seed: int = 5
    storage: str = "f32"
    net: str = "learned"        # "learned" (6-24-24-1) or "learned3" (6-53-3)


@dataclass
class Sample:
    rho0: torch.Tensor
    u0: torch.Tensor
    u_ref: torch.Tensor
    w_ref: torch.Tensor
    E_ref: float


def make_shear_data(cfg: TrainConfig):
    """Fine BGK shear-layer trajectory -> list of (coarse initial state, coarse target)."""
    n, nc = cfg.n_fine, cfg.n_fine // 2
    dims, rho, u = lbinputs.shear_layer(n, u0=cfg.u0)
    fine = Lattice("D2Q9", dims, cfg.tau_fine, "bgk", storage=cfg.storage)
    fine.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    fine.step(cfg.spinup)
    tmp = Lattice("D2Q9", (nc, nc, 1), coarse_tau(cfg.tau_fine), "bgk", storage="f64")
    samples = []
    for _ in range(cfg.n_snap):
        tmp.coarsen_from(fine)
        r0, v0 = tmp.moments(torch.float32, "cuda")
        fine.step(2 * cfg.horizon)
        tmp.coarsen_from(fine)
        _, vt = tmp.moments(torch.float32, "cuda")
        wt = tmp.vorticity(torch.float32, "cuda")
        Et = float(tmp.reduce()[4])
        samples.append(Sample(r0, v0, vt, wt, Et))
        fine.step(cfg.snap_every - 2 * cfg.horizon)
    fine.check()
    # standardisation of the network inputs from the coarse snapshots
    stats = []
    for s in samples[: cfg.n_snap - 2 * cfg.holdout]:
        tmp.init_from_moments(s.rho0.double(), s.u0.double())
        tmp.step(5)
        stats.append(tmp.learned_inputs(torch.float64, "cuda"))
    I = torch.cat(stats, dim=1)
    shift = I.mean(dim=1)
    scale = 1.0 / torch.clamp(I.std(dim=1), min=1e-30)
    fine.close()
    tmp.close()
    return samples, torch.cat([shift, scale]).float()


def init_theta(tau_c: float, seed: int, net: str = "learned") -> torch.Tensor:
    """Xavier hidden layers, zero output weights, output bias ln(tau_c - 1/2): exactly BGK."""
    gen = lbinputs.random_mlp3_params if net == "learned3" else lbinputs.random_mlp_params
    th = gen(seed, out_bias=math.log(tau_c - 0.5), out_scale=0.0)
    return torch.tensor(th, dtype=torch.float32, device="cuda")


def rollout_loss(lat: Lattice, s: Sample, horizon: int, grad=None):
    """Eq. 6 loss of one coarse rollout; if grad is given, add dL/dtheta to it."""
    lat.init_from_moments(s.rho0, s.u0)
    lat.step(horizon)
    L, lam = lat.loss_eq6(s.u_ref, s.w_ref, s.E_ref, want_lambda=grad is not None)
    if grad is not None:
        lat.step_adjoint(lam, horizon, grad_theta=grad, want_lambda0=False)
    return L


def rank_world(group) -> tuple[int, int]:
    """(rank, world size) of a torch.distributed group; (0, 1) for group None (one process)."""
    if group is None:
        return 0, 1
    import torch.distributed as dist
    return dist.get_rank(group), dist.get_world_size(group)


def sharded_mean(loss_of, items, group=None, g=None, device="cuda"):
    """Data-parallel batch: rank r of `group` evaluates loss_of(item, g) for items r, r + world, ...
    (every rank holds the same list), and every rank gets back the mean over all items. If g is
    given, each call adds its item's dL/dtheta to g and g ends as the sum over all items on every
    rank (FP64 all-reduce), so the update that follows is the same on every rank as in one process."""
    rank, world = rank_world(group)
    mine = items[rank::world]
    Ls = [loss_of(it, g) for it in mine]
    if world == 1:
        return float(np.mean(Ls))
    import torch.distributed as dist
    if g is not None:
        allreduce_gradient(g, group)
    tot = torch.tensor([float(sum(Ls)), float(len(Ls))], dtype=torch.float64, device=device)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    return float(tot[0] / tot[1])


def mean_loss(lat: Lattice, samples, horizon: int, group=None):
    return sharded_mean(lambda s, _: rollout_loss(lat, s, horizon), samples, group)


def train(cfg: TrainConfig, samples=None, extra=None, log=None, group=None):
    """Train the network on the shear-layer samples; returns theta, extra and a history.

    group: a torch.distributed process group for data-parallel training, or None for one
    process. Every rank builds the same samples and draws the same batches (same seed); each
    runs its share of a batch's rollouts and adjoints on its own GPU, the parameter gradients
    are summed across the ranks, and every rank then takes the same Adam step. Held-out and
    validation rollouts are shared out the same way."""
    if samples is None:
        samples, extra = make_shear_data(cfg)
    nc = cfg.n_fine // 2
    tau_c = coarse_tau(cfg.tau_fine)
    n = len(samples)
    train_set = samples[: n - 2 * cfg.holdout]
    val = samples[n - 2 * cfg.holdout: n - cfg.holdout]   # early stopping
    hold = samples[n - cfg.holdout:]                       # reported gain, never used for choices
    theta = init_theta(tau_c, cfg.seed, cfg.net)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    lat = Lattice("D2Q9", (nc, nc, 1), tau_c, cfg.net, storage=cfg.storage, record_every=cfg.record_every)
    rng = np.random.default_rng(cfg.seed)
    hist = {"train_loss": [], "holdout_loss": []}
    lat.set_mlp(torch.cat([theta, extra]))
    base_hold = mean_loss(lat, hold, cfg.horizon, group)
    base_val = mean_loss(lat, val, cfg.horizon, group)
    hist["holdout_loss"].append((0, base_hold))
    hist["val_loss"] = [(0, base_val)]
    best = (base_val, 0, theta.clone())  # early stopping on the validation loss
    t0 = time.perf_counter()
    for it in range(1, cfg.iters + 1):
        lat.set_mlp(torch.cat([theta, extra]))
        g = torch.zeros(_lib.n_theta(cfg.net), dtype=torch.float32, device="cuda")
        pick = rng.choice(len(train_set), size=min(cfg.batch, len(train_set)), replace=False)
        L = sharded_mean(lambda j, gr: rollout_loss(lat, train_set[j], cfg.horizon, grad=gr), list(pick), group, g)
        if not torch.isfinite(g).all():
            raise FloatingPointError(f"non-finite gradient at iteration {it}")
        adam_update(theta, m, v, g, it, lr=cfg.lr)
        hist["train_loss"].append(L)
        if it % max(1, cfg.iters // 20) == 0 or it == cfg.iters:
            lat.set_mlp(torch.cat([theta, extra]))
            hl = mean_loss(lat, hold, cfg.horizon, group)
            vl = mean_loss(lat, val, cfg.horizon, group)
            hist["holdout_loss"].append((it, hl))
            hist["val_loss"].append((it, vl))
            if vl < best[0]:
                best = (vl, it, theta.clone())
            if log:
                log(f"iter {it}: train {hist['train_loss'][-1]:.4e} val {vl:.4e} test {hl:.4e} (BGK {base_hold:.4e})")
    torch.cuda.synchronize()
    hist["train_seconds"] = time.perf_counter() - t0
    theta = best[2]
    hist["best_iter"] = best[1]
    lat.set_mlp(torch.cat([theta, extra]))
    final_hold = mean_loss(lat, hold, cfg.horizon, group)
    lat.close()
    # the same held-out rollouts with the plain BGK operator (the method without the network)
    bgk = Lattice("D2Q9", (nc, nc, 1), tau_c, "bgk", storage=cfg.storage)
    bgk_hold = mean_loss(bgk, hold, cfg.horizon, group)
    bgk.close()
    hist.update({"holdout_loss_bgk": bgk_hold, "holdout_loss_learned": final_hold,
                 "holdout_gain": 1.0 - final_hold / bgk_hold})
    return theta, extra, hist


def spectrum_2d(u: np.ndarray, n: int):
    """Shell-averaged kinetic-energy spectrum E(k) of a periodic n x n velocity field u[2][N]."""
    uh = [np.fft.fft2(u[a].reshape(n, n)) / (n * n) for a in range(2)]
    e = 0.5 * (np.abs(uh[0]) ** 2 + np.abs(uh[1]) ** 2)
    k = np.fft.fftfreq(n, 1.0 / n)
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    shell = np.rint(kk).astype(np.int64)
    return np.bincount(shell.ravel(), weights=e.ravel())[: n // 2]


def evaluate_turbulence(theta, extra, n_coarse: int = 2048, k0: float = 12.0, u_rms: float = 0.05,
                        seed: int = 30000, re: float = 30000.0, steps: int = 4000, every: int = 250,
                        storage: str = "f32", reference: str = "bgk", net: str = "learned",
                        balanced: bool = False):
    """Learned vs BGK on coarse decaying turbulence against the coarsened fine run (BGK on
    the grid of twice the resolution). If the fine reference itself goes unstable the
    result records when (the caller then lowers Re). balanced: start from the density of the
    field's incompressible pressure instead of rho = 1 (no initial acoustic waves)."""
    nf = 2 * n_coarse
    tau_f = 0.5 + 3.0 * u_rms * (nf / (2.0 * math.pi)) / re
    tau_c = coarse_tau(tau_f)
    rho, u = lbinputs.random_spectrum_velocity((nf, nf, 1), k0, u_rms, seed)  # k0 counts modes per domain
    if balanced:
        rho = lbinputs.balanced_density((nf, nf, 1), u)
    fine = Lattice("D2Q9", (nf, nf, 1), tau_f, reference, storage=storage)
    fine.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    ref = Lattice("D2Q9", (n_coarse, n_coarse, 1), tau_c, "bgk", storage="f64")
    learned = Lattice("D2Q9", (n_coarse, n_coarse, 1), tau_c, net, storage=storage)
    learned.set_mlp(torch.cat([theta.float(), extra.float()]))
    bgk = Lattice("D2Q9", (n_coarse, n_coarse, 1), tau_c, "bgk", storage=storage)
    for lat in (learned, bgk):
        lat.coarsen_from(fine)
    out = {"n_coarse": n_coarse, "re": re, "tau_fine": tau_f, "tau_coarse": tau_c, "reference": reference,
           "times": [],
           "loss_learned": [],
           "loss_bgk": [], "E_ref": [], "E_learned": [], "E_bgk": [], "Z_ref": [], "Z_learned": [], "Z_bgk": []}
    alive = {"learned": True, "bgk": True}
    t = 0
    while t < steps:
        fine.step(2 * every)
        try:
            fine.check()
        except Exception:
            out["reference_unstable_at"] = t + every
            break
        t += every
        ref.coarsen_from(fine)
        _, ur = ref.moments(torch.float32, "cuda")
        wr = ref.vorticity(torch.float32, "cuda")
        Er = float(ref.reduce()[4])
        out["times"].append(t)
        out["E_ref"].append(Er)
        out["Z_ref"].append(0.5 * float((wr.double() ** 2).mean()))
        for name, lat in (("learned", learned), ("bgk", bgk)):
            if not alive[name]:
                for key in ("loss_", "E_", "Z_"):
                    out[key + name].append(None)
                continue
            lat.step(every)
            try:
                lat.check()
            except Exception:
                alive[name] = False
                for key in ("loss_", "E_", "Z_"):
                    out[key + name].append(None)
                out[f"unstable_{name}_at"] = t
                continue
            L, _ = lat.loss_eq6(ur, wr, Er, want_lambda=False)
            w = lat.vorticity(torch.float64, "cuda")
            out["loss_" + name].append(L)
            out["E_" + name].append(float(lat.reduce()[4]))
            out["Z_" + name].append(0.5 * float((w ** 2).mean()))
    # high-wavenumber spectrum error of the final states against the reference
    _, ur = ref.moments(torch.float64, "cpu")
    sr = spectrum_2d(ur.numpy(), n_coarse)
    hi = slice(n_coarse // 8, n_coarse // 2)
    for name, lat in (("learned", learned), ("bgk", bgk)):
        if alive[name] and "reference_unstable_at" not in out and out["times"]:
            _, ul = lat.moments(torch.float64, "cpu")
            sl = spectrum_2d(ul.numpy(), n_coarse)
            out[f"spectrum_hi_log_err_{name}"] = float(np.mean(np.abs(np.log(sl[hi] + 1e-300) - np.log(sr[hi] + 1e-300))))
    for lat in (fine, ref, learned, bgk):
        lat.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n-fine", type=int, default=1024)
    ap.add_argument("--tau-fine", type=float, default=0.503)
    ap.add_argument("--horizon", type=int, default=100)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--eval-n", type=int, default=2048)
    ap.add_argument("--eval-steps", type=int, default=2000)
    ap.add_argument("--net", choices=["learned", "learned3"], default="learned")
    ap.add_argument("--save", type=str, default=None, help="write theta + input scaling (805 / 545 floats) here")
    a = ap.parse_args()
    group = None
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # launched by torchrun: one rank per GPU, data-parallel over the batch's rollouts
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        group = dist.group.WORLD
    rank0 = group is None or rank_world(group)[0] == 0
    cfg = TrainConfig(n_fine=a.n_fine, iters=a.iters, tau_fine=a.tau_fine, horizon=a.horizon,
                      spinup=max(1000, 4 * a.n_fine), snap_every=max(2 * a.horizon + 50, a.n_fine // 2), net=a.net)
    t0 = time.perf_counter()
    theta, extra, hist = train(cfg, log=(lambda s: print(s, flush=True)) if rank0 else None, group=group)
    if not rank0:
        return
    res = {"train": {k: v for k, v in hist.items() if k != "train_loss"}, "config": asdict(cfg)}
    res["train"]["train_loss_first_last"] = [hist["train_loss"][0], hist["train_loss"][-1]]
    if a.save:
        np.save(a.save, torch.cat([theta, extra]).cpu().numpy())
    if a.eval_n > 0:
        # Re 30000 first (Sec. 3.1); if the fine reference itself goes unstable there, halve Re
        for re in (30000.0, 15000.0, 7500.0, 3750.0):
            ev = evaluate_turbulence(theta, extra, n_coarse=a.eval_n, steps=a.eval_steps, re=re, net=a.net)
            ev["re"] = re
            res.setdefault("eval_attempts", []).append({"re": re, "reference_unstable_at": ev.get("reference_unstable_at")})
            if "reference_unstable_at" not in ev:
                res["eval"] = ev
                break
    res["wall_s"] = round(time.perf_counter() - t0, 1)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
