"""Python face of liblb: a ``Lattice`` handle over one C context.

Argument marshalling only. Every step of the method runs in liblb's CUDA kernels;
torch supplies device memory, the CUDA stream and tensors for results. Arrays may
be torch tensors (CUDA or CPU, float32/float64) or numpy arrays (host); all arrays
of one call are brought to the location and dtype of the first one.

Layouts: populations ``[Q, N]``, vectors ``[d, N]``, scalars ``[N]``, nodes in
x-fastest order (``n = x + nx*(y + ny*z)``), i.e. a numpy array of shape
``(nz, ny, nx)`` flattened in C order.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _mem_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return _lib.MEM["device_f64" if t.is_cuda else "host_f64"]
    if t.dtype == torch.float32:
        return _lib.MEM["device_f32" if t.is_cuda else "host_f32"]
    raise TypeError(f"arrays must be float32 or float64, got {t.dtype}")


def _to_tensor(x, like: torch.Tensor | None = None) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x
    else:
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float64)))
    if t.dtype not in (torch.float32, torch.float64):
        t = t.double()
    if like is not None:
        t = t.to(device=like.device, dtype=like.dtype)
    return t.contiguous()


class Lattice:
    """One periodic lattice advanced by liblb on one GPU.

    stencil: "D2Q9" | "D3Q19" | "D3Q27"; dims: (nx, ny, nz) with nz = 1 in 2D;
    tau > 1/2; collision: "bgk" | "regularized" | "learned" (6-24-24-1 network, one higher-moment
    rate) | "learned3" (6-53-3 network, one rate per higher moment) | "none" | "trt" | "kbc" | "mrt";
    storage: "f64" | "f32" | "f16" | "bf16" (the half types store f_i - w_i);
    layout: "ab" (two buffers) | "aa" (in place); record_every > 0 keeps
    checkpoints for ``step_adjoint``; learned_tc runs the learned collision's network
    in half precision on the tensor cores (FP16 operands and hidden-layer accumulation, the
    hardware tanh; forward only); graphs
    replays ``step(n)`` as captured two-step CUDA graphs (off: one launch per kernel);
    nodes_per_thread forces the stream-collide launch shape (0: chosen from the grid).
    The context runs on torch's current CUDA stream at construction time.
    """

    def __init__(self, stencil: str, dims, tau: float, collision: str = "bgk", storage: str = "f32",
                 layout: str = "ab", device: int | None = None, stream=None, check_every: int = 0,
                 record_every: int = 0, learned_tc: bool = False, graphs: bool = True,
                 nodes_per_thread: int = 0):
        self._lib = _lib.load()
        self.stencil = stencil
        self.dims = tuple(int(v) for v in dims)
        if len(self.dims) == 2:
            self.dims = (*self.dims, 1)
        self.tau = float(tau)
        self.collision = collision
        self.storage = storage
        self.layout = layout
        self.Q = _lib.Q_OF[stencil]
        self.D = _lib.D_OF[stencil]
        self.N = int(np.prod(self.dims))
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        opt = _lib.Options()
        self._lib.lb_default_options(ctypes.byref(opt))
        opt.storage = _lib.STORAGE[storage]
        opt.layout = _lib.LAYOUT[layout]
        opt.cuda_stream = ctypes.c_void_p(stream.cuda_stream)
        opt.device = device
        opt.check_every = check_every
        opt.record_every = record_every
        opt.learned_tc = int(bool(learned_tc))
        opt.graphs = int(bool(graphs))
        opt.nodes_per_thread = int(nodes_per_thread)
        dims_arr = (ctypes.c_int64 * 3)(*self.dims)
        h = ctypes.c_void_p()
        _lib.check(self._lib.lb_create(ctypes.byref(h), _lib.STENCIL[stencil], dims_arr, ctypes.c_double(tau),
                                       _lib.COLLISION[collision], ctypes.byref(opt)), "lb_create")
        self._h = h
        # bumped by every call that changes the state, the force, the collision's parameters
        # or the recording, so that a pending backward pass can tell that its run is gone
        self.version = 0

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ helpers
    def _out(self, shape, dtype, device):
        dev = self.device if device in (None, "cuda") else torch.device(device)
        pin = dev.type == "cpu"
        return torch.empty(shape, dtype=dtype, device=dev, pin_memory=pin and torch.cuda.is_available())

    @property
    def handle(self):
        return self._h

    def launch_count(self) -> int:
        return int(self._lib.lb_launch_count(self._h))

    def steps_taken(self) -> int:
        return int(self._lib.lb_steps_taken(self._h))

    # ------------------------------------------------------------------ state
    def init_from_moments(self, rho, u):
        self.version += 1
        r = _to_tensor(rho)
        v = _to_tensor(u, like=r)
        _lib.check(self._lib.lb_init_from_moments(self._h, r.data_ptr(), v.data_ptr(), _mem_code(r)),
                   "lb_init_from_moments")
        self._keep = (r, v)
        return self

    def set_force(self, F):
        self.version += 1
        if F is None:
            _lib.check(self._lib.lb_set_force(self._h, None, 0), "lb_set_force")
            return self
        t = _to_tensor(F)
        _lib.check(self._lib.lb_set_force(self._h, t.data_ptr(), _mem_code(t)), "lb_set_force")
        self._keep = (t,)
        return self

    def set_mlp(self, params):
        self.version += 1
        t = _to_tensor(params)
        _lib.check(self._lib.lb_set_mlp(self._h, t.data_ptr(), t.numel(), _mem_code(t)), "lb_set_mlp")
        return self

    def set_relaxation(self, params):
        """TRT: [Lambda]; MRT: [tau_6, tau_7, tau_8] (see lb_set_relaxation)."""
        self.version += 1
        v = (ctypes.c_double * len(params))(*[float(x) for x in params])
        _lib.check(self._lib.lb_set_relaxation(self._h, v, len(params)), "lb_set_relaxation")
        return self

    def set_solid(self, mask, wall_u=None):
        """Solid nodes (mask[N] nonzero) with halfway bounce-back; wall_u[d][N] moves them
        (float32/float64, like the other arrays); mask None removes all walls."""
        self.version += 1
        if mask is None:
            _lib.check(self._lib.lb_set_solid(self._h, None, None, _lib.MEM["host_f64"]), "lb_set_solid")
            return self
        if isinstance(mask, torch.Tensor):
            mt = (mask != 0).to(torch.uint8).contiguous()
        else:
            mt = torch.from_numpy(np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0).astype(np.uint8))
        if mt.numel() != self.N:
            raise ValueError(f"mask needs {self.N} entries")
        if wall_u is not None:
            wu = _to_tensor(wall_u).to(mt.device)
            code = _mem_code(wu)
        else:
            wu = None
            code = _lib.MEM["device_f64" if mt.is_cuda else "host_f64"]
        _lib.check(self._lib.lb_set_solid(self._h, mt.data_ptr(), None if wu is None else wu.data_ptr(), code),
                   "lb_set_solid")
        self._keep = (mt, wu)
        return self

    def set_populations(self, f):
        self.version += 1
        t = _to_tensor(f)
        _lib.check(self._lib.lb_set_populations(self._h, t.data_ptr(), _mem_code(t)), "lb_set_populations")
        self._keep = (t,)
        return self

    def step(self, n: int = 1):
        self.version += 1
        _lib.check(self._lib.lb_step(self._h, int(n)), "lb_step")
        return self

    def check(self):
        _lib.check(self._lib.lb_check(self._h), "lb_check")

    def get_populations(self, dtype=torch.float64, device=None) -> torch.Tensor:
        out = self._out((self.Q, self.N), dtype, device)
        _lib.check(self._lib.lb_get_populations(self._h, out.data_ptr(), _mem_code(out)), "lb_get_populations")
        return out

    def moments(self, dtype=torch.float64, device=None, out=None):
        """(rho[N], u[D][N]) of the pre-collision state; out = (rho, u): contiguous tensors of one
        dtype to fill instead (e.g. page-locked host buffers kept across calls)."""
        if out is None:
            rho = self._out((self.N,), dtype, device)
            u = self._out((self.D, self.N), dtype, device)
        else:
            rho, u = out
            if (rho.numel() != self.N or u.numel() != self.D * self.N or rho.dtype != u.dtype
                    or rho.device != u.device or not (rho.is_contiguous() and u.is_contiguous())):
                raise ValueError("out must be contiguous (rho[N], u[D][N]) of one dtype and device")
        _lib.check(self._lib.lb_moments(self._h, rho.data_ptr(), u.data_ptr(), _mem_code(rho)), "lb_moments")
        return rho, u

    def reduce(self) -> np.ndarray:
        out = (ctypes.c_double * 6)()
        _lib.check(self._lib.lb_reduce(self._h, out), "lb_reduce")
        return np.array(list(out))

    def coarsen_from(self, fine: "Lattice"):
        """This (coarse) lattice's state <- f^eq of the 2x block-averaged moments of `fine`."""
        self.version += 1
        _lib.check(self._lib.lb_coarsen_into(fine._h, self._h), "lb_coarsen_into")
        return self

    def vorticity(self, dtype=torch.float64, device=None) -> torch.Tensor:
        w = self._out((self.N,), dtype, device)
        _lib.check(self._lib.lb_vorticity(self._h, w.data_ptr(), _mem_code(w)), "lb_vorticity")
        return w

    def learned_inputs(self, dtype=torch.float64, device=None) -> torch.Tensor:
        """The six (unstandardised) network inputs of every node, [6, N]."""
        out = self._out((6, self.N), dtype, device)
        _lib.check(self._lib.lb_learned_inputs(self._h, out.data_ptr(), _mem_code(out)), "lb_learned_inputs")
        return out

    # ------------------------------------------------------------------ spectral flow control
    def set_spectral_control(self, sigma0, cutoff: float = 2e-5, kappa: float = 5e-5):
        """Sec. 3.2: every later step collides at u + du, du = -kappa grad_u R, R the log-spectrum
        mismatch to sigma0 (n/2 shells) with cutoff c; sigma0 None turns it off."""
        self.version += 1
        if sigma0 is None:
            _lib.check(self._lib.lb_set_spectral_control(self._h, None, 0, 0.0, 0.0), "lb_set_spectral_control")
            return self
        s0 = np.ascontiguousarray(np.asarray(sigma0, dtype=np.float64).reshape(-1))
        _lib.check(self._lib.lb_set_spectral_control(self._h, s0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                     s0.size, float(cutoff), float(kappa)),
                   "lb_set_spectral_control")
        return self

    def spectrum(self, with_cost: bool = False):
        """Energy spectrum sigma[n/2] of the current state (and the cost R if with_cost)."""
        K = self.dims[0] // 2
        sig = np.zeros(K)
        cost = ctypes.c_double()
        _lib.check(self._lib.lb_spectrum(self._h, sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(cost) if with_cost else None), "lb_spectrum")
        return (sig, cost.value) if with_cost else sig

    def spectral_shift(self, dtype=torch.float64, device=None) -> torch.Tensor:
        """The velocity shift du[2][N] the next controlled step applies."""
        out = self._out((self.D, self.N), dtype, device)
        _lib.check(self._lib.lb_spectral_shift(self._h, out.data_ptr(), _mem_code(out)), "lb_spectral_shift")
        return out

    # ------------------------------------------------------------------ adjoint
    def adjoint_seed_moments(self, grad_rho, grad_u, grad_F=None, dtype=None, device=None):
        gu = _to_tensor(grad_u)
        gr = None if grad_rho is None else _to_tensor(grad_rho, like=gu)
        lam = torch.empty((self.Q, self.N), dtype=gu.dtype, device=gu.device)
        gF = None if grad_F is None else grad_F
        if gF is not None:
            assert gF.dtype == gu.dtype and gF.device == gu.device and gF.is_contiguous()
        _lib.check(self._lib.lb_adjoint_seed_moments(self._h, None if gr is None else gr.data_ptr(), gu.data_ptr(),
                                                     lam.data_ptr(), None if gF is None else gF.data_ptr(),
                                                     _mem_code(gu)), "lb_adjoint_seed_moments")
        return lam

    def loss_energy(self, e_target, grad_F=None):
        et = _to_tensor(e_target)
        lam = torch.empty((self.Q, self.N), dtype=et.dtype, device=et.device)
        if grad_F is not None:
            assert grad_F.dtype == et.dtype and grad_F.device == et.device and grad_F.is_contiguous()
        L = ctypes.c_double()
        _lib.check(self._lib.lb_loss_energy(self._h, et.data_ptr(), ctypes.byref(L), lam.data_ptr(),
                                            None if grad_F is None else grad_F.data_ptr(), _mem_code(et)),
                   "lb_loss_energy")
        return L.value, lam

    def loss_eq6(self, u_ref, w_ref, E_ref: float, want_lambda: bool = True):
        ur = _to_tensor(u_ref)
        wr = _to_tensor(w_ref, like=ur)
        lam = torch.empty((self.Q, self.N), dtype=ur.dtype, device=ur.device) if want_lambda else None
        L = ctypes.c_double()
        _lib.check(self._lib.lb_loss_eq6(self._h, ur.data_ptr(), wr.data_ptr(), ctypes.c_double(E_ref),
                                         ctypes.byref(L), None if lam is None else lam.data_ptr(), _mem_code(ur)),
                   "lb_loss_eq6")
        return L.value, lam

    def step_adjoint(self, lambda_T, n: int, grad_F=None, grad_theta=None, want_lambda0: bool = True):
        lt = _to_tensor(lambda_T)
        lam0 = torch.empty_like(lt) if want_lambda0 else None
        for g in (grad_F, grad_theta):
            if g is not None:
                assert g.dtype == lt.dtype and g.device == lt.device and g.is_contiguous()
        _lib.check(self._lib.lb_step_adjoint(self._h, lt.data_ptr(), int(n),
                                             None if lam0 is None else lam0.data_ptr(),
                                             None if grad_F is None else grad_F.data_ptr(),
                                             None if grad_theta is None else grad_theta.data_ptr(), _mem_code(lt)),
                   "lb_step_adjoint")
        return lam0


def adam_update(theta: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, step: int,
                lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8):
    """One Adam step on FP32 CUDA tensors, in liblb's kernel, on torch's current stream."""
    lib = _lib.load()
    for t in (theta, m, v, grad):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    s = torch.cuda.current_stream(theta.device).cuda_stream
    _lib.check(lib.lb_adam_update(theta.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), theta.numel(),
                                  lr, betas[0], betas[1], eps, int(step), ctypes.c_void_p(s)), "lb_adam_update")
