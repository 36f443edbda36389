"""The paper's flows through liblb at reduced sizes: the decay rate of the 2D
Taylor-Green vortex, the energy error of the storage types against the FP64 GPU run,
and the FP32 adjoint against finite differences of the FP64 forward run."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_12929_gb300 import build
    build.build()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_tgv2d_decay_rate_within_1_percent(storage):
    from paper_2106_12929_gb300 import experiments
    r = experiments.tgv2d_decay(n=64, tau=0.8, steps=1000, storage=storage)
    assert r["rel_err"] < 0.01, r


def test_tgv3d_half_storage_energy_error():
    from paper_2106_12929_gb300 import experiments
    r = experiments.tgv3d_precision(n=64, steps=600)
    # measured on GB300: FP32 2.3e-5, FP16 ~5e-5, BF16 ~1e-2 over 600 steps at tau = 0.5011
    assert r["energy_rel_err_f32"] < 5e-5, r
    assert r["energy_rel_err_f16"] < 1e-3, r    # the half-precision target
    assert r["energy_rel_err_bf16"] < 5e-2, r   # BF16 (8-bit mantissa) is reported, not held to 1e-3


def test_turbulence_precision_sweep_small():
    from paper_2106_12929_gb300 import experiments
    r = experiments.turbulence_precision(n=48, steps=200, every=10)
    assert r["energy_rel_err_f32"] < 1e-5, r
    assert r["energy_rel_err_f16"] < 1e-2, r


def test_fp32_adjoint_within_1e_4_of_finite_differences():
    from paper_2106_12929_gb300 import experiments
    r = experiments.adjoint_fd(n=64, steps=50, k=10)
    # the FP64 adjoint is the exact discrete gradient: it matches central differences
    assert r["fd_rel_err_f64"] < 1e-6, r
    # the FP32 gradient field is within 1e-4 (relative L2) of it
    assert r["f32_vs_f64_adjoint_rel_l2"] < 1e-4, r


def test_tgv3d_half_storage_energy_error_at_the_full_size():
    """The precision sweep of the 256^3 Taylor-Green workload over its 2000 steps: relative
    energy error of each storage type against the FP64 GPU run of the same lattice, held to the
    1e-3 bar for FP16. BF16 (8-bit significand of f - w) does not reach that bar; its figure is
    checked here against what DESIGN and BASELINE report."""
    from paper_2106_12929_gb300 import experiments
    r = experiments.tgv3d_precision(n=256, steps=2000)
    print({k: v for k, v in r.items() if k.startswith("energy")})
    assert r["energy_rel_err_f32"] < 1e-4, r
    assert r["energy_rel_err_f16"] < 1e-3, r
    assert 1e-3 < r["energy_rel_err_bf16"] < 3e-2, r


def test_spectral_control_driver_holds_the_spectrum():
    """experiments.spectral_control (Sec. 3.2) at 128^2 over 1000 steps: the controlled run
    stays closer to the initial spectrum (cost R) and keeps more of its energy than the free
    BGK run from the same state; both runs stay finite."""
    import math

    from paper_2106_12929_gb300 import experiments
    r = experiments.spectral_control(n=128, steps=1000, every=250)
    free, ctrl = r["free"], r["controlled"]
    assert free["t"] == ctrl["t"] == [0, 250, 500, 750, 1000]
    assert all(math.isfinite(v) for v in free["E"] + ctrl["E"] + free["R"] + ctrl["R"])
    assert free["R"][0] == ctrl["R"][0] <= 1e-9  # both start at the target (up to FP32 logarithms)
    assert ctrl["R"][-1] < 0.5 * free["R"][-1], (ctrl["R"], free["R"])
    assert ctrl["E"][-1] > free["E"][-1], (ctrl["E"], free["E"])
