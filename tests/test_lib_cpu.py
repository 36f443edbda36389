"""CPU-side checks of the C-ABI library: it builds, loads, exports every declared
symbol, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_12929_gb300 import _lib, build
    build.build()
    return _lib.load()


def _header_functions():
    with open(os.path.join(ROOT, "include", "lb.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^LB_API\s+[\w\s\*]+?\b(lb_\w+)\(", text, flags=re.M)))


def test_header_declares_the_boundary_calls():
    names = _header_functions()
    for required in ["lb_create", "lb_init_from_moments", "lb_step", "lb_moments", "lb_step_adjoint",
                     "lb_reduce", "lb_get_populations", "lb_set_populations", "lb_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2106_12929_gb300 import _lib
    names = _header_functions()
    assert names == _lib.declared_symbols()
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(7):
        assert lib.lb_status_string(code)
    assert lib.lb_status_string(99) == b"unknown status"


def _create(lib, stencil=0, dims=(8, 8, 1), tau=0.8, coll=0, **opt_kw):
    from paper_2106_12929_gb300 import _lib
    opt = _lib.Options()
    lib.lb_default_options(ctypes.byref(opt))
    for k, v in opt_kw.items():
        setattr(opt, k, v)
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 3)(*dims)
    rc = lib.lb_create(ctypes.byref(h), stencil, d, ctypes.c_double(tau), coll, ctypes.byref(opt))
    return rc, h


@pytest.mark.parametrize("kw,expect", [
    (dict(tau=0.5), 1),                     # tau must exceed 1/2
    (dict(tau=float("nan")), 1),
    (dict(dims=(8, 8, 2)), 1),              # 2D stencil needs nz = 1
    (dict(dims=(0, 8, 1)), 1),
    (dict(stencil=7), 1),
    (dict(coll=9), 1),
    (dict(stencil=1, dims=(4, 4, 4), coll=2), 6),   # learned collision is D2Q9 only
    (dict(storage=5), 1),
    (dict(layout=1, record_every=5), 6),    # recording needs the AB layout
    (dict(graphs=2), 1),
    (dict(nodes_per_thread=3), 1),
    (dict(coll=8), 1),
    (dict(stencil=1, dims=(4, 4, 4), coll=7), 6),   # the three-output network is D2Q9 only too
    (dict(coll=7, learned_tc=1, storage=0), 6),     # its tensor-core option needs FP32 or half storage
    (dict(stencil=1, dims=(4, 4, 4), coll=5), 6),  # KBC needs D2Q9 or D3Q27
    (dict(stencil=2, dims=(4, 4, 4), coll=6), 6),  # MRT is D2Q9 only
    (dict(coll=4, record_every=3), 6),             # no adjoint of TRT / KBC / MRT
    (dict(learned_tc=1), 6),                # tensor-core network needs the learned collision
    (dict(dims=(-4, 8, 1)), 1),
    (dict(dims=(65536, 1, 1)), 1),          # every edge at most 65535 (launch-grid limit)
    (dict(dims=(50000, 50000, 1)), 1),      # N = 2.5e9 nodes: beyond N < 2^31
    (dict(stencil=1, dims=(2048, 2048, 600)), 1),
    (dict(check_every=-1), 1),
    (dict(record_every=-2), 1),
])
def test_create_rejects_bad_arguments_without_gpu(lib, kw, expect):
    opt_keys = {"storage", "layout", "record_every", "check_every", "graphs", "learned_tc", "nodes_per_thread"}
    opt = {k: v for k, v in kw.items() if k in opt_keys}
    args = {k: v for k, v in kw.items() if k not in opt_keys}
    rc, h = _create(lib, **args, **opt)
    assert rc == expect
    assert not h.value
    assert lib.lb_last_error()


def test_null_context_calls_fail_cleanly(lib):
    assert lib.lb_step(None, 1) == 1
    assert lib.lb_check(None) == 1
    assert lib.lb_num_nodes(None) == -1
    sig = (ctypes.c_double * 4)()
    assert lib.lb_set_spectral_control(None, sig, 4, 2e-5, 5e-5) == 1
    assert lib.lb_spectrum(None, sig, None) == 1
    assert lib.lb_spectral_shift(None, None, 0) == 1
    assert lib.lb_set_mlp(None, None, 545, 0) == 1
    nbytes = ctypes.c_int64()
    assert lib.lb_halo_bytes(None, ctypes.byref(nbytes)) == 1
    assert lib.lb_halo_pack(None, 0, None) == 1
    assert lib.lb_halo_unpack(None, 1, None) == 1
    assert lib.lb_reduce_slab(None, 1, 1, (ctypes.c_double * 6)()) == 1
    lib.lb_destroy(None)


def test_adam_rejects_bad_arguments(lib):
    assert lib.lb_adam_update(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == 1


def test_product_path_has_no_cpu_fallback():
    # the package must not import the oracle, and must raise if the library is missing
    import paper_2106_12929_gb300 as pkg
    pkg_dir = os.path.dirname(pkg.__file__)
    for fn in os.listdir(pkg_dir):
        if fn.endswith(".py"):
            with open(os.path.join(pkg_dir, fn)) as fh:
                src = fh.read()
            assert "import oracle" not in src and "from oracle" not in src, fn


@pytest.mark.parametrize("stencil,dims,mem,null_f", [
    (0, (8, 8, 1), 1, True),              # f is required
    (5, (8, 8, 1), 1, False),             # unknown stencil
    (0, (8, 8, 1), 0, False),             # host arrays are not accepted
    (0, (65536, 1, 1), 1, False),         # edge beyond 65535
    (0, (8, 8, 2), 1, False),             # 2D stencil needs nz = 1
    (1, (8192, 4097, 1), 1, False),       # more nodes than its fixed scratch array serves
])
def test_noalloc_sums_reject_bad_arguments_before_any_device_work(lib, stencil, dims, mem, null_f):
    # every case fails argument validation, which runs before any CUDA call, so the host buffer
    # passed as f is never dereferenced
    buf = (ctypes.c_double * 8)()
    out = (ctypes.c_double * 6)()
    d = (ctypes.c_int64 * 3)(*dims)
    f = None if null_f else ctypes.cast(buf, ctypes.c_void_p)
    assert lib.lb_reduce_noalloc(stencil, d, f, None, mem, out, None) == 1
    assert lib.lb_last_error()


def test_stream_copy_rejects_bad_arguments_before_any_device_work(lib):
    """The bandwidth reference checks pointers, size and alignment before it touches a device."""
    buf = (ctypes.c_uint8 * 64)()
    base = ctypes.addressof(buf)
    aligned = base + (-base) % 16
    assert lib.lb_stream_copy(None, aligned, 16, None) == 1
    assert lib.lb_stream_copy(aligned, None, 16, None) == 1
    assert lib.lb_stream_copy(aligned, aligned + 16, 0, None) == 1
    assert lib.lb_stream_copy(aligned, aligned + 16, 24, None) == 1        # not a multiple of 16
    assert lib.lb_stream_copy(aligned + 4, aligned + 16, 16, None) == 1    # misaligned source
    assert b"16" in lib.lb_last_error()
