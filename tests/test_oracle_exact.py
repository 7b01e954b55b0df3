"""Pins of the closed-form Gaussian-pulse solutions (oracle/exact.py), CPU only.

* The per-mode Strang factors equal the iterated product of the three exact sub-flows of one step (a velocity
  half step, a full pressure step, a velocity half step), built here as 2 x 2 matrices.
* The time-discrete solution tends to the continuous one at second order as dt shrinks at a fixed time.
* The grid evaluation, which integrates once per distinct radius, equals the pointwise evaluation.
* At t = 0 both solutions reproduce the initial pulse exp(-5 r^2) with zero velocity.
"""
import numpy as np

from oracle.exact import pulse_on_grid, pulse_solution, strang_mode_factors


def test_strang_mode_factors_equal_the_iterated_split_step():
    rng = np.random.default_rng(11)
    for w_tau in np.concatenate([rng.uniform(0.01, 1.99, 6), [0.2, 1.0]]):
        half_kick = np.array([[1.0, 0.0], [0.5 * w_tau, 1.0]])   # (S, U): U += (tau/2) w S
        drift = np.array([[1.0, -w_tau], [0.0, 1.0]])            # S -= tau w U
        step = half_kick @ drift @ half_kick
        state = np.array([1.0, 0.0])
        for n in range(60):
            S, U = strang_mode_factors(w_tau, n)
            assert abs(S - state[0]) < 1e-12 and abs(U - state[1]) < 1e-12, (w_tau, n)
            state = step @ state


def test_time_discrete_solution_tends_to_the_continuous_one_at_second_order():
    x = np.linspace(0.0, 4.0, 41)
    ref_s, ref_v = pulse_solution(x, 0.7 * x, 1, 0.04, discrete=False)
    diffs = []
    for k in (200, 400, 800):
        s, v = pulse_solution(x, 0.7 * x, k, 0.04 / k)
        diffs.append(max(np.abs(s - ref_s).max(), np.abs(v - ref_v).max()))
    assert diffs[0] > 1e-6
    for a, b in zip(diffs, diffs[1:]):
        assert 3.8 < a / b < 4.2, diffs


def test_grid_evaluation_equals_pointwise_evaluation():
    n = 16
    x = -5.0 + (10.0 / n) * np.arange(n + 1)
    for discrete in (True, False):
        sg, vg = pulse_on_grid(n, 300, 1e-4, discrete)
        sp, vp = pulse_solution(x[None, :], x[:, None], 300, 1e-4, discrete)
        assert np.abs(sg - sp).max() < 1e-13 and np.abs(vg - vp).max() < 1e-13
        assert np.abs(vg).max() > 1e-3
        np.testing.assert_allclose(vg[::-1, :], -vg, atol=1e-15)  # v3 is odd in z
        np.testing.assert_allclose(sg[:, ::-1], sg, atol=1e-15)


def test_initial_pulse_is_reproduced_at_time_zero():
    x = np.linspace(-5, 5, 21)
    for discrete in (True, False):
        s, v = pulse_solution(x[None, :], x[:, None], 0, 1e-4, discrete)
        assert np.abs(s - np.exp(-5 * (x[None, :] ** 2 + x[:, None] ** 2))).max() < 1e-12
        assert np.abs(v).max() == 0.0
