"""Write se_erfc_fit.h: the polynomial used by the FP32 real-space kernels for erfc.

erfc(x) = exp(-x^2) erfcx(x), and exp(-x^2) is already computed for the Gaussian terms of
the real-space kernels. With t = 1 / (1 + a x), x >= 0, the scaled function erfcx(x) / t is
smooth on t in [0, 1] (it tends to a / sqrt(pi) as x -> infinity), so a degree-10 polynomial
R(t), obtained by Chebyshev interpolation on [0, 1], gives erfc(x) = exp(-x^2) t R(t) with a
relative error below 1e-8 for every x >= 0 (far below FP32 rounding).

Run from this directory: python gen_erfc_fit.py  (needs numpy and scipy).
"""
import os

import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as Pm
from scipy.special import erfcx

A = 0.4
DEG = 10


def scaled(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.full_like(t, A / np.sqrt(np.pi))
    m = t > 0
    x = (1.0 / t[m] - 1.0) / A
    out[m] = erfcx(x) / t[m]
    return out


def coefficients():
    k = np.arange(DEG + 1)
    tn = 0.5 * (1.0 - np.cos(np.pi * (k + 0.5) / (DEG + 1)))
    cc = C.chebfit(2.0 * tn - 1.0, scaled(tn), DEG)
    # Chebyshev series in s = 2t - 1 -> monomials in t
    return Pm.Polynomial(C.cheb2poly(cc))(Pm.Polynomial([-1.0, 2.0])).coef


def main():
    c = coefficients()
    tt = np.linspace(1e-7, 1.0, 200001)
    err = np.abs(Pm.polyval(tt, c) / scaled(tt) - 1.0).max()
    lines = [
        "// Generated by gen_erfc_fit.py: erfc(x) = exp(-x^2) t R(t), t = 1 / (1 + a x),",
        "// R(t) = sum_k c_k t^k (Chebyshev interpolation of erfcx(x) / t on t in [0, 1]).",
        f"// max relative error of the polynomial (exact arithmetic): {err:.2e}",
        "#pragma once",
        f"#define SE_ERFC_FIT_A {A!r}",
        f"#define SE_ERFC_FIT_DEG {DEG}",
    ]
    lines += [f"#define SE_ERFC_FIT_C{k} {float(v)!r}" for k, v in enumerate(c)]
    lines += [""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "se_erfc_fit.h")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print(out, err)


if __name__ == "__main__":
    main()
