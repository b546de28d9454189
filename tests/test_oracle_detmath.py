"""Pins for the oracle's deterministic exp/log against 60-digit mpmath values."""
import math
import random

import mpmath
import numpy as np


def _ulp_err(got: float, x, fn):
    with mpmath.workdps(60):
        ref = fn(mpmath.mpf(x))
        if ref == 0:
            return 0.0 if got == 0 else math.inf
        return float(abs(mpmath.mpf(got) - ref) / mpmath.mpf(math.ulp(float(ref))))


def test_det_exp_accuracy(orc):
    rng = random.Random(7)
    xs = [rng.uniform(-23.0, 0.0) for _ in range(3000)]           # threshold range
    xs += [rng.uniform(-700.0, 700.0) for _ in range(1000)]
    xs += [rng.uniform(-1e-6, 1e-6) for _ in range(200)] + [0.0, -1.0, 1.0, -0.5 * math.log(2)]
    worst = max(_ulp_err(orc.det_exp(x), x, mpmath.exp) for x in xs)
    assert worst <= 2.0, worst
    assert orc.det_exp(0.0) == 1.0
    assert orc.det_exp(-800.0) == 0.0
    # monotone on a fine grid
    g = np.linspace(-23, 0, 20001)
    v = np.array([orc.det_exp(x) for x in g])
    assert np.all(np.diff(v) >= 0)


def test_det_exp_subnormal(orc):
    for x in (-708.5, -720.0, -740.0, -744.0):
        got = orc.det_exp(x)
        ref = float(mpmath.exp(mpmath.mpf(x)))
        assert abs(got - ref) <= 2 * math.ulp(ref) + 5e-324


def test_det_log_accuracy(orc):
    rng = random.Random(11)
    xs = [float(rng.randint(1, 10**15)) for _ in range(2000)]     # histogram counts
    xs += [10.0 ** rng.uniform(-300, 300) for _ in range(2000)]
    xs += [1.0 + rng.uniform(-0.3, 0.4) for _ in range(1000)]
    xs += [2.0 ** k for k in range(-1074, 1024, 37)]
    worst = max(_ulp_err(orc.det_log(x), x, mpmath.log) for x in xs if x != 1.0)
    # s = (m-1)/(m+1) carries up to ~1 ulp before the series; measured worst 2.2 ulp
    assert worst <= 3.0, worst
    assert orc.det_log(1.0) == 0.0
    assert orc.det_log(0.0) == -math.inf
    assert math.isnan(orc.det_log(-1.0))


def test_det_log_exp_roundtrip(orc):
    rng = random.Random(3)
    for _ in range(2000):
        x = rng.uniform(-20, 20)
        assert abs(orc.det_log(orc.det_exp(x)) - x) <= 4 * math.ulp(max(abs(x), 1.0))
