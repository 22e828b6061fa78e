"""Accuracy of the table-driven FP64 elementary functions against the C library.

The node right-hand sides use these routines instead of CUDA's sin/cos/exp to
save FP64 instructions; here they are checked, through the C ABI
(sim_math_eval), against numpy's libm on dense samples of the argument ranges
the models use, plus the edges of each reduction and the fallback paths.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _eval(fn, x):
    from paper_2410_19075_gb300.sim import math_eval
    return math_eval(fn, x)


def test_sin_cos_absolute_error_within_two_ulp_of_one():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-200, 200, 2_000_000), rng.uniform(-1, 1, 100_000),
                        np.arange(-2048, 2048) * (math.pi / 512),            # table points
                        (np.arange(-2048, 2048) + 0.5) * (math.pi / 512),    # reduction edges
                        [0.0, -0.0, 1e-300, 5e-324, 16383.9, 16384.5, 1e6, -3e7]])
    s, c = _eval(0, x), _eval(1, x)
    assert np.abs(s - np.sin(x)).max() <= 4.5e-16
    assert np.abs(c - np.cos(x)).max() <= 4.5e-16


def test_exp_relative_error_within_four_ulp():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-30, 30, 2_000_000), rng.uniform(-1e-3, 1e-3, 10_000),
                        np.arange(-640, 640) * (math.log(2) / 64), [0.0, 699.0, -699.0, 705.0, -705.0]])
    ref = np.exp(x)
    got = _eval(2, x)
    assert (np.abs(got - ref) / ref).max() <= 4 * 2.2205e-16
    # outside the table range the library routine takes over: overflow and underflow
    edge = _eval(2, np.array([710.0, -746.0, np.inf, -np.inf]))
    assert edge[0] == np.inf and edge[1] == 0.0 and edge[2] == np.inf and edge[3] == 0.0


def test_reciprocal_relative_error_within_one_ulp():
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(-40, 40, 1_000_000)) * rng.choice([-1.0, 1.0], 1_000_000)
    x = np.concatenate([x, [1.0, -1.0, 3.0, 1e-40, 1e40, 2.0 ** -126]])
    got = _eval(3, x)
    assert (np.abs(got * x - 1.0)).max() <= 2 * 2.2205e-16


def test_hh_rate_form_x_over_one_minus_exp():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-16, 16, 1_000_000), rng.uniform(-0.2, 0.2, 100_000),
                        [0.0, 1e-12, -1e-12, 0.0999999, 0.1, 0.1000001, -0.1, 1e-300]])
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.where(x == 0, 1.0, x / -np.expm1(-x))
    ref = np.where(np.abs(x) < 1e-300, 1.0, ref)
    got = _eval(4, x)
    assert (np.abs(got - ref) / np.abs(ref)).max() <= 4e-15
