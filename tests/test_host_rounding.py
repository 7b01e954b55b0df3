"""Host-side FP32 storage of model coefficients (loss_round_fp32_unbiased; no GPU needed).

FP32 grids store kappa (lambda, mu) and b by unbiased rounding: with round-to-nearest, a layer of constant
coefficients carries one common relative error of up to 2^-24, a systematic wave-speed bias whose phase error
grows with the travel time (about 1e-5 over 1500 steps of a 20 Hz survey shot)."""
import numpy as np
import pytest

import paper_2301_05127_gb300 as loss

M64 = (1 << 64) - 1


def _splitmix64(z: int) -> int:
    """SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014), written from its definition."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _neighbours(x):
    f = np.float32(x)
    g = np.nextafter(f, np.float32(np.inf) if float(f) < x else np.float32(-np.inf))
    return min(f, g), max(f, g)


def test_every_value_rounds_to_one_of_its_two_fp32_neighbours():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(1e8, 2e10, 500), rng.uniform(1e-4, 1e-3, 500), -rng.uniform(1, 10, 500)])
    out = loss.round_fp32_unbiased(x)
    for xi, oi in zip(x, out):
        lo, hi = _neighbours(xi)
        assert oi == lo or oi == hi


def test_exact_and_non_finite_values_convert_as_by_a_cast():
    x = np.array([0.0, 1.0, -2.5, 0.125, 3.0e9 - 3.0e9 % 256, np.inf, -np.inf, np.nan])
    out = loss.round_fp32_unbiased(x, key0=12345)
    ref = x.astype(np.float32)
    assert np.array_equal(out[:-1], ref[:-1]) and np.isnan(out[-1])


def test_decisions_follow_the_documented_variate():
    """Element i rounds up exactly when (splitmix64(key0 + i) >> 11) * 2^-53 < (x - lo) / (hi - lo)."""
    rng = np.random.default_rng(2)
    x = 1000.0 * rng.uniform(1500.0, 4000.0, 400) ** 2
    key0 = 987654321
    out = loss.round_fp32_unbiased(x, key0=key0)
    for i, (xi, oi) in enumerate(zip(x, out)):
        lo, hi = _neighbours(xi)
        if float(lo) == xi:
            continue
        up = (xi - float(lo)) / (float(hi) - float(lo))
        u = (_splitmix64(key0 + i) >> 11) * 2.0**-53
        assert oi == (hi if u < up else lo)


def test_a_constant_layer_carries_no_common_bias():
    """A million copies of a layer's kappa: the mean stored value equals kappa to well within one ulp / 100, while
    round-to-nearest is off by a fixed fraction of an ulp."""
    kappa = 1000.0 * 2226.3**2
    lo, hi = _neighbours(kappa)
    ulp = float(hi) - float(lo)
    n = 1 << 20
    out = loss.round_fp32_unbiased(np.full(n, kappa))
    mean_err = (out.astype(np.float64) - kappa).mean() / ulp
    assert abs(mean_err) < 5 * 0.5 / np.sqrt(n)  # 5 standard deviations of the mean
    nearest_err = (float(np.float32(kappa)) - kappa) / ulp
    assert abs(nearest_err) > 0.05  # the bias the unbiased rounding removes
    frac_up = float((out == hi).mean())
    assert abs(frac_up - (kappa - float(lo)) / ulp) < 5 * 0.5 / np.sqrt(n)


def test_deterministic_and_keyed_by_position():
    x = np.full(64, 1.0e-3 / 3.0)
    a = loss.round_fp32_unbiased(x, key0=7)
    b = loss.round_fp32_unbiased(x, key0=7)
    c = loss.round_fp32_unbiased(x, key0=0)
    assert np.array_equal(a, b)
    assert np.array_equal(a[:-7], c[7:])


def test_bad_arguments():
    L = loss.lib()
    assert L.loss_round_fp32_unbiased(None, None, -1, 0) == loss.LOSS_E_ARG
    assert L.loss_round_fp32_unbiased(None, None, 4, 0) == loss.LOSS_E_ARG
    assert L.loss_round_fp32_unbiased(None, None, 0, 0) == loss.LOSS_OK


@pytest.mark.parametrize("key0", [0, 2**63 + 5])
def test_large_keys_wrap_modulo_2_64(key0):
    x = np.full(3, 0.1)
    out = loss.round_fp32_unbiased(x, key0=key0)
    for i in range(3):
        lo, hi = _neighbours(0.1)
        up = (0.1 - float(lo)) / (float(hi) - float(lo))
        u = (_splitmix64((key0 + i) & M64) >> 11) * 2.0**-53
        assert out[i] == (hi if u < up else lo)
