"""The FP32 real-space kernels evaluate erfc(x) as exp(-x^2) t R(t), t = 1 / (1 + a x), with
the polynomial R of paper_2210_01255_gb300/csrc/se_erfc_fit.h. Pin it to scipy's erfc and
erfcx (independent implementations) over the whole range a real-space sum can reach."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2210_01255_gb300", "csrc", "se_erfc_fit.h")


def _fit():
    txt = open(HDR).read()
    a = float(re.search(r"#define SE_ERFC_FIT_A (\S+)", txt).group(1))
    deg = int(re.search(r"#define SE_ERFC_FIT_DEG (\d+)", txt).group(1))
    c = [float(re.search(r"#define SE_ERFC_FIT_C%d (\S+)\n" % k, txt).group(1)) for k in range(deg + 1)]
    return a, np.array(c)


def test_fit_relative_error_exact_arithmetic():
    special = pytest.importorskip("scipy.special")
    a, c = _fit()
    x = np.concatenate([np.linspace(0.0, 10.0, 200001), np.geomspace(10.0, 1e4, 2001)])
    t = 1.0 / (1.0 + a * x)
    approx = t * np.polyval(c[::-1], t)
    assert np.abs(approx / special.erfcx(x) - 1.0).max() < 2e-8
    # erfc itself where it is representable in double
    m = x < 25.0
    e = np.exp(-x[m] ** 2) * approx[m]
    assert np.abs(e / special.erfc(x[m]) - 1.0).max() < 1e-7


def test_fit_float32_rounding():
    """Horner in FP32 with a rounded reciprocal stays within 8 FP32 ulp of erfcx."""
    special = pytest.importorskip("scipy.special")
    a, c = _fit()
    x = np.linspace(0.0, 12.0, 100001).astype(np.float32)
    t = (np.float32(1.0) / (np.float32(a) * x + np.float32(1.0))).astype(np.float32)
    r = np.full_like(t, np.float32(c[-1]))
    for ck in c[-2::-1]:
        r = (r * t + np.float32(ck)).astype(np.float32)
    v = (t * r).astype(np.float32).astype(np.float64)
    assert np.abs(v / special.erfcx(x.astype(np.float64)) - 1.0).max() < 8 * 2.0**-24 * 8


def test_limits():
    a, c = _fit()
    assert abs(c[0] - a / np.sqrt(np.pi)) < 1e-8  # erfcx(x) ~ 1/(sqrt(pi) x) as x -> infinity
    assert abs(c.sum() - 1.0) < 1e-8  # erfcx(0) = 1 (t = 1)
