"""The seeded recorder's own single-precision elementary functions (used so
that the GPU recorder can reproduce its paths bit for bit) against the C
library's double-precision ones."""
import math

import numpy as np

import pgrec

ULP1 = 2.0 ** -23  # float32 spacing at 1


def _f32(x):
    return float(np.float32(x))


def test_log_within_three_float_ulp():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(0, 1, 5000), 2.0 ** rng.uniform(-60, 60, 5000),
                         [0.5, 2.0, 1 - 2 ** -24, 2 ** -24, 0.70710677, 1.4142135]]).astype(np.float32)
    for x in xs:
        got, want = pgrec.elementary("log", float(x)), math.log(float(x))
        assert abs(got - want) <= 3 * float(np.spacing(np.float32(abs(want)))) + 1e-45, x
    assert pgrec.elementary("log", 1.0) == 0.0


def test_sincos_2pi():
    rng = np.random.default_rng(2)
    us = np.concatenate([rng.uniform(0, 1, 5000), [0.0, 0.125, 0.25, 0.5, 0.75, 1 - 2 ** -24]]).astype(np.float32)
    for u in us:
        s, c = pgrec.elementary("sincos_2pi", float(u))
        a = 2 * math.pi * float(u)
        assert abs(s - math.sin(a)) <= 4 * ULP1 and abs(c - math.cos(a)) <= 4 * ULP1, u
        assert abs(s * s + c * c - 1.0) <= 4 * ULP1
    assert pgrec.elementary("sincos_2pi", 0.0) == (0.0, 1.0)
    assert pgrec.elementary("sincos_2pi", 0.25) == (1.0, -0.0)
