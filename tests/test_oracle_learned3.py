"""Pins of the oracle's one-hidden-layer, three-output network collision (the network shape
Sec. 3.1 describes: one relaxation time exp(z_n) + 1/2 per higher moment): its BGK and
fixed-rate MRT limits, which fix the assignment of outputs to moments, and conservation.
Its adjoint is checked against finite differences in test_oracle_adjoint.py."""
import math

import numpy as np

import lbinputs
import oracle


def _node(seed, eps=0.05):
    d, c, w, _ = oracle.stencil("D2Q9")
    return lbinputs.random_populations(w, 1, seed, eps)[:, 0]


def _net(out_bias, out_scale=0.0, seed=3):
    th = lbinputs.random_mlp3_params(seed, out_bias=out_bias, out_scale=out_scale)
    return np.concatenate([th, np.zeros(6), np.array([50.0, 100.0, 300.0, 1e5, 1e5, 1e5])])


def test_parameter_count():
    assert oracle.N_THETA3 == 6 * 53 + 53 + 3 * 53 + 3 == 533
    assert len(_net(0.0)) == oracle.N_MLP3


def test_constant_outputs_at_the_shear_time_give_bgk():
    tau = 0.62
    f = _node(11)
    a = oracle.collide_node("D2Q9", tau, "learned3", f, mlp=_net(math.log(tau - 0.5)))
    b = oracle.collide_node("D2Q9", tau, "bgk", f)
    np.testing.assert_allclose(a, b, rtol=0, atol=2e-16)


def test_constant_outputs_give_fixed_rate_mrt_in_the_paper_order():
    # outputs (z0, z1, z2) set the times of N (4th order) and J0, J1 (3rd order), the order in
    # which the paper lists the higher moments; the MRT takes (tau_6, tau_7, tau_8) for the
    # Hermite rows (cx^2 - 1/3) cy, cx (cy^2 - 1/3), (cx^2 - 1/3)(cy^2 - 1/3)
    tau = 0.7
    tN, tJ0, tJ1 = 1.3, 0.8, 2.1
    f = _node(12)
    net = _net(np.log(np.array([tN, tJ0, tJ1]) - 0.5))
    a = oracle.collide_node("D2Q9", tau, "learned3", f, mlp=net)
    b = oracle.collide_node("D2Q9", tau, "mrt", f, params=[tJ0, tJ1, tN])
    np.testing.assert_allclose(a, b, rtol=0, atol=2e-16)
    # and the assignment matters: a permuted one differs
    c = oracle.collide_node("D2Q9", tau, "mrt", f, params=[tN, tJ0, tJ1])
    assert np.max(np.abs(a - c)) > 1e-6


def test_conserves_mass_and_momentum():
    d, c, w, _ = oracle.stencil("D2Q9")
    f = _node(13, eps=0.1)
    out = oracle.collide_node("D2Q9", 0.55, "learned3", f, mlp=_net(0.0, out_scale=0.7, seed=4))
    assert abs(out.sum() - f.sum()) < 1e-15
    np.testing.assert_allclose(c.T @ out, c.T @ f, atol=1e-16)


def _rotation_perm():
    d, c, w, _ = oracle.stencil("D2Q9")
    # rotation by 90 degrees: (cx, cy) -> (-cy, cx); perm[i] = index of R c_i
    rc = np.stack([-c[:, 1], c[:, 0], c[:, 2]], 1)
    return np.array([np.where((c == v).all(1))[0][0] for v in rc])


def test_rotation_equivariance_needs_equal_third_order_times():
    """A 90-degree rotation maps the third-order moments J0, J1 onto each other (and keeps the
    network inputs, which are invariants), so the collision commutes with it exactly when
    the J0 and J1 outputs agree; with different times it does not. The shared-rate network
    is always equivariant (test_oracle_pins.py)."""
    perm = _rotation_perm()
    tau = 0.6
    f = _node(14, eps=0.3)
    fr = np.empty_like(f)
    fr[perm] = f  # population of direction i moves to direction R c_i
    same = _net(np.log(np.array([1.3, 0.8, 0.8]) - 0.5))
    a = oracle.collide_node("D2Q9", tau, "learned3", f, mlp=same)
    b = oracle.collide_node("D2Q9", tau, "learned3", fr, mlp=same)
    np.testing.assert_allclose(b[perm], a, atol=2e-16)
    differ = _net(np.log(np.array([1.3, 0.8, 2.1]) - 0.5))
    a = oracle.collide_node("D2Q9", tau, "learned3", f, mlp=differ)
    b = oracle.collide_node("D2Q9", tau, "learned3", fr, mlp=differ)
    assert np.max(np.abs(b[perm] - a)) > 1e-6
