"""Host-side logic that needs no GPU: the training driver's scale conventions and spectrum
diagnostic, the workload generators' closed forms, and the benchmark's bookkeeping."""
import math
import statistics
import os
import sys

import numpy as np
import pytest

import lbinputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_coarse_relaxation_time_keeps_the_viscosity_in_acoustic_scaling():
    from paper_2106_12929_gb300 import training
    # nu_c dt_c / dx_c^2 = nu_f dt_f / dx_f^2 with dx_c = 2 dx_f, dt_c = 2 dt_f: nu_lu halves
    for tau_f in (0.503, 0.51, 0.8):
        tau_c = training.coarse_tau(tau_f)
        assert (tau_c - 0.5) == pytest.approx((tau_f - 0.5) / 2.0, rel=1e-15)


def test_training_spectrum_of_single_modes():
    from paper_2106_12929_gb300 import training
    n = 32
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    A, B = 0.02, 0.03
    u = np.zeros((2, n * n))
    u[0] = (A * np.cos(2 * np.pi * (3 * x + 4 * y) / n)).ravel()  # |k| = 5
    u[1] = (B * np.sin(2 * np.pi * 7 * y / n)).ravel()            # |k| = 7
    e = training.spectrum_2d(u, n)
    expect = np.zeros(n // 2)
    expect[5] = A * A / 4
    expect[7] = B * B / 4
    np.testing.assert_allclose(e, expect, rtol=0, atol=1e-18)


def test_init_theta_is_exactly_bgk_for_both_networks():
    pytest.importorskip("torch")
    from paper_2106_12929_gb300 import _lib
    for net, gen in (("learned", lbinputs.random_mlp_params), ("learned3", lbinputs.random_mlp3_params)):
        th = gen(5, out_bias=math.log(0.01), out_scale=0.0)
        assert th.size == _lib.n_theta(net)
        # output weights are zero, so the output is the bias ln(tau_c - 1/2) for every input
        n_out = 1 if net == "learned" else 3
        n_w = 24 if net == "learned" else 3 * 53
        w_out = th[-(n_w + n_out):-n_out]
        assert np.all(w_out == 0.0)
        assert np.all(th[-n_out:] == math.log(0.01))


def test_relaxation_time_from_reynolds_number():
    # nu = u0 (n / 2 pi) / Re, tau = 3 nu + 1/2 (c_s^2 = 1/3)
    u0, n, re = 0.1 / math.sqrt(3.0), 256, 1600.0
    tau = lbinputs.tau_from_reynolds(re, u0, n)
    assert tau == pytest.approx(0.5 + 3.0 * u0 * n / (2 * math.pi) / re, rel=1e-14)
    assert tau == pytest.approx(0.504411, abs=1e-6)  # the 256^3 benchmark's value


def test_random_spectrum_velocity_is_solenoidal_with_the_requested_rms():
    dims = (32, 32, 1)
    rho, u = lbinputs.random_spectrum_velocity(dims, 4.0, 0.05, 7)
    assert np.all(rho == 1.0)
    ux, uy = (c.reshape(32, 32) for c in u)
    k = np.fft.fftfreq(32, 1.0 / 32)
    div = 1j * k[None, :] * np.fft.fft2(ux) + 1j * k[:, None] * np.fft.fft2(uy)
    inner = (np.abs(k) < 16)[:, None] & (np.abs(k) < 16)[None, :]  # the Nyquist lines have no sign
    assert np.max(np.abs(div[inner])) <= 1e-12 * np.max(np.abs(np.fft.fft2(ux)))
    # the rms per component, averaged over the components, is u_rms
    assert np.sqrt(0.5 * (np.mean(ux ** 2) + np.mean(uy ** 2))) == pytest.approx(0.05, rel=1e-12)


def test_job_throughput_of_a_single_replica():
    sys.path.insert(0, ROOT)
    import bench
    lups, t = bench.job_throughput(1000, 10, 2.0, world=1)
    assert t == 2.0 and lups == pytest.approx(5000.0)
    assert bench.BYTES_PER_LU[("D3Q19", "f32")] == 152
    assert bench.BYTES_PER_LU[("D3Q27", "f16")] == 108
    assert bench.LEARNED_FLOP_PER_LU["learned3"] == 2 * (6 * 53 + 53 * 3) + 200


def test_both_benchmark_arms_name_the_same_workload():
    sys.path.insert(0, ROOT)
    import bench
    cfg = bench.workload_config(2)
    n = bench.N_GRID
    assert cfg["grid"] == [n, n, n] and cfg["nodes"] == n ** 3 and cfg["parallelism"] == "replicas x2"
    tau = lbinputs.tau_from_reynolds(bench.RE, bench.U0, n)
    assert f"tau = {tau:.6f}" in cfg["workload"] and f"{n}^3" in cfg["workload"]
    assert bench.workload_config(1) == {**cfg, "parallelism": "replicas x1"}


def test_every_experiment_is_reachable_from_the_command_line():
    import inspect
    from paper_2106_12929_gb300 import experiments
    src = inspect.getsource(experiments.main)
    for name in ("tgv2d_decay", "tgv3d_precision", "turbulence_precision", "adjoint_fd", "spectral_control"):
        assert callable(getattr(experiments, name)) and f'"{name}"' in src and name in experiments.__doc__


def test_clock_sampler_keeps_the_samples_inside_the_timed_region():
    sys.path.insert(0, ROOT)
    import bench

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc, s.thread = _Proc(), None
    s.lines = [(1.0, "210, 2070, 90.0, 0x1, Not Active, Not Active, Not Active, Not Active\n"),  # idle, before
               (2.0, "1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"),
               (2.2, "2070, 2070, 1100.5, 0x4, Not Active, Not Active, Not Active, Active\n"),
               (2.4, "2070, 2070, 1180.0, 0x4, Not Active, Not Active, Not Active, Active\n"),
               (2.6, "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n"),
               (9.0, "300, 2070, 95.0, 0x1, Active, Not Active, Not Active, Not Active\n")]  # after
    got = s.stop(window=(1.5, 3.0))
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                   "in_timed_region": True}
    # no sample inside the window: the summary of all samples, marked as such
    got = s.stop(window=(5.0, 6.0))
    assert got["samples"] == 5 and got["in_timed_region"] is False and "hw_slowdown" in got["reasons"]


def test_clock_record_rejection_rule():
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected({**ok, "sm_mhz": 1500.0, "reasons": ["sw_power_cap"]})  # kept, noted
    assert bench.clocks_rejected({**ok, "reasons": ["hw_slowdown"]})
    assert bench.clocks_rejected({**ok, "reasons": ["sw_power_cap", "sw_thermal_slowdown"]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 1200.0})  # well below max with no reason: a clock lock


@pytest.mark.parametrize("first_bad", [False, True])
@pytest.mark.parametrize("region_s", [2.0, 0.05])
def test_timed_region_repeats_and_is_taken_once_more_after_a_rejected_clock_record(monkeypatch, first_bad,
                                                                                   region_s):
    sys.path.insert(0, ROOT)
    import bench
    records = [{"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown"] if first_bad else []},
               {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}]
    # a K-step region of region_s seconds is repeated max(3, ceil(0.8 s / region_s)) times
    reps = max(3, math.ceil(bench.MIN_TIMED_SECONDS / region_s))
    first = [region_s * (1.0 + 0.01 * j) for j in range(reps)]  # median = the middle one
    second = [t + 0.001 * region_s for t in first]  # the same repeat count, distinguishable times
    times = first + second
    windows = []

    class _Sampler:
        def __init__(self, gpu_index):
            self.rec = records.pop(0)

        def wait_first_sample(self):
            pass

        def stop(self, window=None):
            windows.append(window)
            return self.rec

    class _Lat:
        launches = 0

        def launch_count(self):
            return self.launches

    lat = _Lat()

    def _time_steps(lat_, k, stream):
        lat_.launches += k
        return times.pop(0)

    monkeypatch.setattr(bench, "ClockSampler", _Sampler)
    monkeypatch.setattr(bench, "time_steps", _time_steps)
    t, clocks, launches = bench.timed_region(lat, 10, None, 0, world=1)
    assert launches == 10 and clocks["remeasured"] is first_bad and clocks["repeats"] == reps
    assert t == pytest.approx(statistics.median(second if first_bad else first)) and clocks["reasons"] == []
    assert len(records) == (0 if first_bad else 1)
    assert all(w[0] <= w[1] for w in windows)
    assert len(times) == (0 if first_bad else reps)


def test_reference_arm_grid_fits_its_budget():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reference_grid(20, 5) == bench.N_GRID  # a 20 + 5 step run times the 256^3 grid itself
    assert bench.reference_grid(2000, 10) == 128
    assert bench.reference_grid(20000, 10) == 64
    for k in (1, 20, 200, 2000, 20000):
        n = bench.reference_grid(k, 10)
        assert (k + 10) * n ** 3 <= bench.REFERENCE_LU_BUDGET or n == 32
    cfg = bench.workload_config(1, 128)
    assert cfg["grid"] == [128, 128, 128] and "128^3" in cfg["workload"] and cfg["nodes"] == 128 ** 3


def test_lb_run_backward_refuses_a_replaced_run():
    """The autograd wrapper's guard, with a stand-in lattice (no GPU): any state change after
    the forward pass makes its backward pass raise instead of differentiating another run."""
    import torch
    from paper_2106_12929_gb300 import autograd

    class _Lat:
        storage, D, N, collision, device = "f64", 2, 4, "bgk", torch.device("cpu")

        def __init__(self):
            self.version = 0
            self.adjoint_calls = 0

        def set_force(self, F):
            self.version += 1

        def init_from_moments(self, r, u):
            self.version += 1

        def step(self, n):
            self.version += 1

        def moments(self, dtype, device):
            return torch.ones(4, dtype=dtype), torch.zeros((2, 4), dtype=dtype)

        def adjoint_seed_moments(self, g_rho, g_u, grad_F=None):
            return torch.zeros((9, 4), dtype=torch.float64)

        def step_adjoint(self, lam, n, grad_F=None, grad_theta=None, want_lambda0=True):
            self.adjoint_calls += 1

    lat = _Lat()
    F = torch.zeros((2, 4), dtype=torch.float64, requires_grad=True)
    _, u1 = autograd.lb_run(lat, torch.ones(4), torch.zeros((2, 4)), 3, F=F)
    u1.sum().backward()  # nothing changed: the adjoint runs
    assert lat.adjoint_calls == 1
    _, u2 = autograd.lb_run(lat, torch.ones(4), torch.zeros((2, 4)), 3, F=F)
    lat.step(1)
    with pytest.raises(RuntimeError, match="recorded run is gone"):
        u2.sum().backward()
    assert lat.adjoint_calls == 1


def test_build_rebuilds_an_object_only_when_a_dependency_is_newer(tmp_path):
    from paper_2106_12929_gb300 import build
    src, hdr, obj = (tmp_path / n for n in ("a.cu", "a.cuh", "a.o"))
    for p in (src, hdr, obj):
        p.write_text("x")
    os.utime(src, (100, 100))
    os.utime(hdr, (100, 100))
    os.utime(obj, (200, 200))
    assert not build._stale(str(obj), [str(src), str(hdr)])
    os.utime(hdr, (300, 300))  # a header edited after the object was built
    assert build._stale(str(obj), [str(src), str(hdr)])
    assert build._stale(str(tmp_path / "missing.o"), [str(src)])


def test_balanced_density_is_the_taylor_green_pressure():
    """The spectral pressure solve against the closed-form pressures of the 2D and 3D
    Taylor-Green vortices (each highest at the stagnation points); the decaying-turbulence
    field it balances has the same mean density."""
    for dims, rho, u in (lbinputs.taylor_green_2d(48, u0=0.05), lbinputs.taylor_green_3d(24)):
        got = lbinputs.balanced_density(dims, u)
        assert np.max(np.abs(got - rho)) <= 1e-15
        assert rho[0] == np.max(rho)  # node 0 is a stagnation point
    rho, u = lbinputs.random_spectrum_velocity((64, 64, 1), 6.0, 0.05, 7)
    got = lbinputs.balanced_density((64, 64, 1), u)
    assert abs(np.mean(got) - 1.0) <= 1e-15 and np.std(got) > 1e-4
