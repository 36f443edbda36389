"""ctypes loader of liblb.so and the C signatures of include/lb.h.

There is no fallback: if the library is missing or cannot be loaded, every call
raises. Build it with ``python -m paper_2106_12929_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblb.so")

# enums of include/lb.h
STENCIL = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISION = {"bgk": 0, "regularized": 1, "learned": 2, "none": 3, "trt": 4, "kbc": 5, "mrt": 6, "learned3": 7}
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
LAYOUT = {"ab": 0, "aa": 1}
MEM = {"host_f64": 0, "device_f64": 1, "host_f32": 2, "device_f32": 3}
STATUS = {0: "LB_OK", 1: "LB_ERR_ARG", 2: "LB_ERR_OOM", 3: "LB_ERR_CUDA", 4: "LB_ERR_UNSTABLE",
          5: "LB_ERR_STATE", 6: "LB_ERR_UNSUPPORTED"}
Q_OF = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
D_OF = {"D2Q9": 2, "D3Q19": 3, "D3Q27": 3}
N_NET = 805
N_THETA = 793
# the one-hidden-layer, three-output network (collision "learned3")
N_NET3 = 545
N_THETA3 = 533


def n_theta(collision: str) -> int:
    """Trained parameters of a learned collision's network (the length of its gradient)."""
    return {"learned": N_THETA, "learned3": N_THETA3}[collision]


class LBError(RuntimeError):
    """A liblb call returned a status other than LB_OK."""

    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.code}: {message}")


class Options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("layout", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("check_every", ctypes.c_int), ("record_every", ctypes.c_int),
                ("learned_tc", ctypes.c_int), ("graphs", ctypes.c_int), ("nodes_per_thread", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_D = ctypes.c_double

_SIGNATURES = {
    "lb_default_options": (None, [ctypes.POINTER(Options)]),
    "lb_create": (_INT, [ctypes.POINTER(_P), _INT, ctypes.POINTER(_I64), _D, _INT, ctypes.POINTER(Options)]),
    "lb_destroy": (None, [_P]),
    "lb_init_from_moments": (_INT, [_P, _P, _P, _INT]),
    "lb_set_force": (_INT, [_P, _P, _INT]),
    "lb_set_mlp": (_INT, [_P, _P, _I64, _INT]),
    "lb_set_relaxation": (_INT, [_P, _P, _INT]),
    "lb_set_solid": (_INT, [_P, _P, _P, _INT]),
    "lb_step": (_INT, [_P, _I64]),
    "lb_moments": (_INT, [_P, _P, _P, _INT]),
    "lb_reduce": (_INT, [_P, ctypes.POINTER(_D)]),
    "lb_get_populations": (_INT, [_P, _P, _INT]),
    "lb_set_populations": (_INT, [_P, _P, _INT]),
    "lb_check": (_INT, [_P]),
    "lb_steps_taken": (_I64, [_P]),
    "lb_adjoint_seed_moments": (_INT, [_P, _P, _P, _P, _P, _INT]),
    "lb_loss_energy": (_INT, [_P, _P, ctypes.POINTER(_D), _P, _P, _INT]),
    "lb_loss_eq6": (_INT, [_P, _P, _P, _D, ctypes.POINTER(_D), _P, _INT]),
    "lb_step_adjoint": (_INT, [_P, _P, _I64, _P, _P, _P, _INT]),
    "lb_coarsen_into": (_INT, [_P, _P]),
    "lb_learned_inputs": (_INT, [_P, _P, _INT]),
    "lb_vorticity": (_INT, [_P, _P, _INT]),
    "lb_adam_update": (_INT, [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I64, _P]),
    "lb_set_spectral_control": (_INT, [_P, ctypes.POINTER(_D), _I64, _D, _D]),
    "lb_spectrum": (_INT, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "lb_spectral_shift": (_INT, [_P, _P, _INT]),
    "lb_reduce_noalloc": (_INT, [_INT, ctypes.POINTER(_I64), _P, _P, _INT, ctypes.POINTER(_D), _P]),
    "lb_stream_copy": (_INT, [_P, _P, _I64, _P]),
    "lb_halo_bytes": (_INT, [_P, ctypes.POINTER(_I64)]),
    "lb_halo_pack": (_INT, [_P, _INT, _P]),
    "lb_halo_unpack": (_INT, [_P, _INT, _P]),
    "lb_reduce_slab": (_INT, [_P, _I64, _I64, ctypes.POINTER(_D)]),
    "lb_num_nodes": (_I64, [_P]),
    "lb_q": (_INT, [_P]),
    "lb_d": (_INT, [_P]),
    "lb_launch_count": (_I64, [_P]),
    "lb_status_string": (ctypes.c_char_p, [_INT]),
    "lb_last_error": (ctypes.c_char_p, []),
}


def declared_symbols():
    """Names of every function declared in include/lb.h."""
    return sorted(_SIGNATURES)


def load():
    """Load liblb.so (once) and attach the C signatures. Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"liblb.so not built ({LIB_PATH}); run python -m paper_2106_12929_gb300.build")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, where: str):
    if status != 0:
        msg = load().lb_last_error()
        raise LBError(status, where, msg.decode() if msg else "")
