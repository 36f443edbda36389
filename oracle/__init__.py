"""FP64 CPU oracle of the lattice Boltzmann hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never loads it and has
no CPU fallback. The arithmetic lives in ``lb_oracle.c`` (plain C, FP64, no fused
multiply-add); this module only compiles it and marshals numpy arrays.

Conventions: a population array is ``f[Q][N]`` (FP64, natural layout, the
pre-collision state of Eq. 1), a vector field ``u[d][N]``, nodes ordered x fastest.
Collision kinds: ``"bgk"`` (Eq. 2), ``"regularized"``, ``"learned"`` (Eq. 5, D2Q9),
``"none"`` (streaming only), ``"trt"`` (two relaxation times), ``"kbc"`` (entropic,
D2Q9 and D3Q27), ``"mrt"`` (Eq. 5 with fixed rates, D2Q9), ``"learned3"`` (Eq. 5 with a
one-hidden-layer network giving three higher-moment rates, D2Q9). ``params``: TRT
``[Lambda]`` (default 1/4), MRT ``[tau_6, tau_7, tau_8]`` (default 1, 1, 1). Stencils: ``"D2Q9"``, ``"D3Q19"``, ``"D3Q27"``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblb_oracle.so")
_lock = threading.Lock()
_lib = None

STENCILS = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"bgk": 0, "regularized": 1, "learned": 2, "none": 3, "trt": 4, "kbc": 5, "mrt": 6, "learned3": 7}
N_PARAMS = {"trt": 1, "mrt": 3}
N_THETA = 793
N_MLP = N_THETA + 12
N_THETA3 = 533  # one hidden layer of 53 units, three outputs
N_MLP3 = N_THETA3 + 12

_dbl_p = ctypes.POINTER(ctypes.c_double)
_i64_p = ctypes.POINTER(ctypes.c_int64)
_int_p = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off -fopenmp) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c99",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for name in ("ora_stencil", "ora_init_eq", "ora_step", "ora_step_walls", "ora_step_ushift", "ora_collide_node", "ora_moments",
                         "ora_reduce", "ora_adjoint", "ora_seed_moments", "ora_loss_energy",
                         "ora_loss_eq6", "ora_vorticity", "ora_mlp_omega", "ora_invariants",
                         "ora_guo_source", "ora_num_threads"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dbl_p)


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _dims(dims):
    d = np.zeros(3, dtype=np.int64)
    d[:] = [int(v) for v in dims]
    return d


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def stencil(name: str):
    """(d, c[Q][3] int, w[Q], opp[Q]) of a velocity set."""
    lib = _load()
    d = ctypes.c_int()
    q = ctypes.c_int()
    c = np.zeros(27 * 3, dtype=np.intc)
    w = np.zeros(27)
    opp = np.zeros(27, dtype=np.intc)
    _check(lib.ora_stencil(STENCILS[name], ctypes.byref(d), ctypes.byref(q), c.ctypes.data_as(_int_p),
                           _p(w), opp.ctypes.data_as(_int_p)), "stencil")
    Q = q.value
    return d.value, c[: 3 * Q].reshape(Q, 3).astype(np.int64), w[:Q].copy(), opp[:Q].astype(np.int64)


def n_nodes(dims) -> int:
    return int(np.prod([int(v) for v in dims]))


def init_eq(name, dims, rho, u):
    """f = f^eq(rho, u) (Eq. 3) at every node."""
    d, c, w, _ = stencil(name)
    N = n_nodes(dims)
    rho = _arr(rho, (N,))
    u = _arr(u, (d, N))
    f = np.zeros((len(w), N))
    _check(_load().ora_init_eq(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), _p(rho), _p(u), _p(f)),
           "init_eq")
    return f


def _cpar(collision, mlp, params):
    if collision == "learned":
        return None if mlp is None else _arr(mlp, (N_MLP,))
    if collision == "learned3":
        return None if mlp is None else _arr(mlp, (N_MLP3,))
    if params is None:
        return None
    return _arr(params, (N_PARAMS[collision],))


def step(name, dims, tau, collision, f, nsteps=1, F=None, mlp=None, params=None):
    """Return f^{n+nsteps} from f^n by iterating Eq. 1 (collide, then push-stream)."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    out = _arr(f, (len(w), N)).copy()
    F = None if F is None else _arr(F, (d, N))
    mlp = _cpar(collision, mlp, params)
    _check(_load().ora_step(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), ctypes.c_double(tau),
                            COLLISIONS[collision], _p(F), _p(mlp), _p(out), ctypes.c_int64(nsteps)), "step")
    return out


def step_ushift(name, dims, tau, f, du, nsteps=1):
    """Return the state after ``nsteps`` BGK steps whose equilibrium is taken at u + du
    (the velocity-shift forcing of Sec. 3.2), du[d][N] held fixed."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    out = _arr(f, (len(w), N)).copy()
    _check(_load().ora_step_ushift(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), ctypes.c_double(tau),
                                   _p(_arr(du, (d, N))), _p(out), ctypes.c_int64(nsteps)), "step_ushift")
    return out


def step_walls(name, dims, tau, collision, f, mask, nsteps=1, F=None, wall_u=None, params=None, mlp=None):
    """Like ``step`` with solid nodes (mask[N] nonzero) and halfway bounce-back; wall_u[d][N]
    is the velocity of each solid node (moving walls) or None."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    out = _arr(f, (len(w), N)).copy()
    F = None if F is None else _arr(F, (d, N))
    m = np.ascontiguousarray(np.asarray(mask).reshape(N) != 0, dtype=np.uint8)
    wu = None
    if wall_u is not None:
        wu = np.zeros((3, N))
        wu[:d] = _arr(wall_u, (d, N))
    _check(_load().ora_step_walls(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), ctypes.c_double(tau),
                                  COLLISIONS[collision], _p(F), _p(_cpar(collision, mlp, params)),
                                  m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _p(wu), _p(out),
                                  ctypes.c_int64(nsteps)), "step_walls")
    return out


def collide_node(name, tau, collision, f, F=None, mlp=None, params=None):
    """Post-collision populations of a single node (f[Q] -> f*[Q])."""
    d, _, w, _ = stencil(name)
    f = _arr(f, (len(w),))
    out = np.zeros(len(w))
    F = None if F is None else _arr(F, (d,))
    mlp = _cpar(collision, mlp, params)
    _check(_load().ora_collide_node(STENCILS[name], ctypes.c_double(tau), COLLISIONS[collision], _p(f), _p(F),
                                    _p(mlp), _p(out)), "collide_node")
    return out


def guo_source(name, tau, u, F):
    d, _, w, _ = stencil(name)
    S = np.zeros(len(w))
    _check(_load().ora_guo_source(STENCILS[name], ctypes.c_double(tau), _p(_arr(u, (d,))), _p(_arr(F, (d,))),
                                  _p(S)), "guo_source")
    return S


def moments(name, dims, f, F=None):
    """(rho[N], u[d][N]) of the state f (u = (sum c f + F/2)/rho)."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    f = _arr(f, (len(w), N))
    F = None if F is None else _arr(F, (d, N))
    rho = np.zeros(N)
    u = np.zeros((d, N))
    _check(_load().ora_moments(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), _p(F), _p(f), _p(rho), _p(u)),
           "moments")
    return rho, u


def reduce(name, dims, f, F=None):
    """[sum rho, sum rho u_x, sum rho u_y, sum rho u_z, (1/2N) sum |u|^2, (1/2N) sum rho |u|^2]."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    f = _arr(f, (len(w), N))
    F = None if F is None else _arr(F, (d, N))
    out = np.zeros(6)
    _check(_load().ora_reduce(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), _p(F), _p(f), _p(out)), "reduce")
    return out


def adjoint(name, dims, tau, collision, f0, nsteps, lam_T, F=None, mlp=None, want_theta=False):
    """Discrete adjoint of nsteps steps from f0.

    Returns (lambda_0 = dL/df^0, dL/dF or None, dL/dtheta or None) given lam_T = dL/df^N.
    """
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    f0 = _arr(f0, (len(w), N))
    lam = _arr(lam_T, (len(w), N)).copy()
    F = None if F is None else _arr(F, (d, N))
    mlp = _cpar(collision, mlp, None)
    gF = np.zeros((d, N)) if F is not None else None
    gth = None
    if want_theta or collision in ("learned", "learned3"):
        gth = np.zeros(N_THETA3 if collision == "learned3" else N_THETA)
    _check(_load().ora_adjoint(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), ctypes.c_double(tau),
                               COLLISIONS[collision], _p(F), _p(mlp), _p(f0), ctypes.c_int64(nsteps), _p(lam),
                               _p(gF), _p(gth)), "adjoint")
    return lam, gF, gth


def seed_moments(name, dims, f, grho, gu, F=None):
    """lambda = dL/df and the direct dL/dF from moment cotangents (dL/drho, dL/du)."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    f = _arr(f, (len(w), N))
    F = None if F is None else _arr(F, (d, N))
    grho = None if grho is None else _arr(grho, (N,))
    gu = _arr(gu, (d, N))
    lam = np.zeros((len(w), N))
    gF = np.zeros((d, N)) if F is not None else None
    _check(_load().ora_seed_moments(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), _p(F), _p(f), _p(grho),
                                    _p(gu), _p(lam), _p(gF)), "seed_moments")
    return lam, gF


def loss_energy(name, dims, f, e_target, F=None):
    """(L, lambda^N, direct dL/dF) for L = sum_x (rho|u|^2/2 - e*)^2."""
    d, _, w, _ = stencil(name)
    N = n_nodes(dims)
    f = _arr(f, (len(w), N))
    F = None if F is None else _arr(F, (d, N))
    e_target = _arr(e_target, (N,))
    lam = np.zeros((len(w), N))
    gF = np.zeros((d, N)) if F is not None else None
    L = ctypes.c_double()
    _check(_load().ora_loss_energy(STENCILS[name], _dims(dims).ctypes.data_as(_i64_p), _p(F), _p(f), _p(e_target),
                                   ctypes.byref(L), _p(lam), _p(gF)), "loss_energy")
    return L.value, lam, gF


def loss_eq6(dims, f, u_ref, w_ref, E_ref):
    """(L, lambda) of the Eq. 6 training loss on a D2Q9 state."""
    N = n_nodes(dims)
    f = _arr(f, (9, N))
    lam = np.zeros((9, N))
    L = ctypes.c_double()
    _check(_load().ora_loss_eq6(_dims(dims).ctypes.data_as(_i64_p), _p(f), _p(_arr(u_ref, (2, N))),
                                _p(_arr(w_ref, (N,))), ctypes.c_double(E_ref), ctypes.byref(L), _p(lam)),
           "loss_eq6")
    return L.value, lam


def vorticity(dims, f):
    """(w[N], E) of a D2Q9 state: central-difference vorticity and (1/2N) sum |u|^2."""
    N = n_nodes(dims)
    w = np.zeros(N)
    E = ctypes.c_double()
    _check(_load().ora_vorticity(_dims(dims).ctypes.data_as(_i64_p), _p(_arr(f, (9, N))), _p(w), ctypes.byref(E)),
           "vorticity")
    return w, E.value


def mlp_omega(mlp, I):
    om = ctypes.c_double()
    _check(_load().ora_mlp_omega(_p(_arr(mlp, (N_MLP,))), _p(_arr(I, (6,))), ctypes.byref(om)), "mlp_omega")
    return om.value


def invariants(f):
    I = np.zeros(6)
    _check(_load().ora_invariants(_p(_arr(f, (9,))), _p(I)), "invariants")
    return I


def num_threads() -> int:
    """Threads the oracle's node loops run on (OpenMP)."""
    return int(_load().ora_num_threads())
