"""Differentiable lattice Boltzmann runs for torch.autograd (gradients through the
solver, Sec. 3.2), backed by liblb's hand-written discrete adjoint.

``lb_run(lattice, rho0, u0, nsteps, F=None, theta=None)`` initialises the lattice
from (rho0, u0), advances ``nsteps`` steps and returns the moments (rho, u) of the
final state. Its backward pass seeds the adjoint from the moment cotangents
(``lb_adjoint_seed_moments``) and runs ``lb_step_adjoint`` over the recorded run
(checkpoints every ``record_every`` steps, recomputation in between), returning
dL/dF for the body force and dL/dtheta for a learned collision's network parameters
(793 for "learned", 533 for "learned3"). rho0 and u0 are treated as constants. The
lattice keeps only its last recorded run: a backward pass after the lattice was
stepped, re-initialised or given a new force or network raises instead of returning
another run's gradient.
"""
from __future__ import annotations

import torch

from . import _lib
from .lattice import Lattice


class _LBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, theta, lattice: Lattice, rho0, u0, nsteps: int, net_extra):
        if F is not None:
            lattice.set_force(F.detach())
        if theta is not None:
            lattice.set_mlp(torch.cat([theta.detach().to(net_extra.dtype), net_extra]))
        lattice.init_from_moments(rho0, u0)
        lattice.step(nsteps)
        dtype = (F if F is not None else theta if theta is not None else rho0).dtype
        rho, u = lattice.moments(dtype=torch.float64 if lattice.storage == "f64" else torch.float32,
                                 device=lattice.device)
        ctx.lattice = lattice
        ctx.version = lattice.version
        ctx.nsteps = nsteps
        ctx.has_F = F is not None
        ctx.has_theta = theta is not None
        ctx.F_dtype = None if F is None else F.dtype
        ctx.theta_dtype = None if theta is None else theta.dtype
        return rho.to(dtype), u.to(dtype)

    @staticmethod
    def backward(ctx, g_rho, g_u):
        lat: Lattice = ctx.lattice
        if lat.version != ctx.version:
            # lb_step_adjoint differentiates whatever run the lattice recorded last; after another
            # run, a new initial state, force or network it would return that run's gradient
            raise RuntimeError("lb_run backward: the lattice was re-initialised, stepped or given a new force or "
                               "network since this run's forward pass; its recorded run is gone")
        rdt = torch.float64 if lat.storage == "f64" else torch.float32
        dev = lat.device
        g_u = torch.zeros((lat.D, lat.N), dtype=rdt, device=dev) if g_u is None else g_u.to(device=dev, dtype=rdt)
        g_rho = None if g_rho is None else g_rho.to(device=dev, dtype=rdt).contiguous()
        gF = torch.zeros((lat.D, lat.N), dtype=rdt, device=dev) if ctx.has_F else None
        gth = torch.zeros(_lib.n_theta(lat.collision), dtype=rdt, device=dev) if ctx.has_theta else None
        lam = lat.adjoint_seed_moments(g_rho, g_u.contiguous(), grad_F=gF)
        lat.step_adjoint(lam, ctx.nsteps, grad_F=gF, grad_theta=gth, want_lambda0=False)
        return (None if gF is None else gF.to(ctx.F_dtype), None if gth is None else gth.to(ctx.theta_dtype),
                None, None, None, None, None)


def lb_run(lattice: Lattice, rho0, u0, nsteps: int, F: torch.Tensor | None = None,
           theta: torch.Tensor | None = None, net_extra: torch.Tensor | None = None):
    """Differentiable run: returns (rho, u) after ``nsteps`` steps from f^eq(rho0, u0).

    F: body force [d, N] (CUDA tensor) or None. theta: the trained network parameters of a
    learned-collision lattice (793 or 533), with ``net_extra`` its fixed 12 input
    shift/scale values. The lattice must have been created with record_every > 0.
    """
    if theta is not None and net_extra is None:
        raise ValueError("theta needs net_extra (input shift[6] and scale[6])")
    if net_extra is not None:
        net_extra = net_extra.to(device=lattice.device, dtype=torch.float64).contiguous()
    return _LBRun.apply(F, theta, lattice, rho0, u0, int(nsteps), net_extra)
