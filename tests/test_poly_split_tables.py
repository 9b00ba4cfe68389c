"""The tables of paper_2210_01255_gb300/csrc/se_poly_split.h (written by gen_poly_split.py)
that add back the potential of the polynomial c_n r^(2n) taken out of the free-space
biharmonic: rebuilt here from the header text and checked against a direct sum over sources of
the closed forms of the two operators applied to r^(2n) (derived by hand, an independent route
from the generator's symbolic expansion): with r = x - y,
  stokeslet (delta lap - grad grad) r^(2n) = 4 n^2 delta r^(2n-2) - 4 n (n-1) r r^T r^(2n-4),
  stresslet ((delta_jl d_m + delta_mj d_l + delta_lm d_j) lap - 2 d_j d_l d_m) r^(2n)
            = 2n (2n-2)(2n-1) (delta_jl r_m + delta_mj r_l + delta_lm r_j) r^(2n-4)
              - 4n (2n-2)(2n-4) r_j r_l r_m r^(2n-6)."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2210_01255_gb300", "csrc", "se_poly_split.h")


def _tables():
    with open(HDR) as fh:
        txt = fh.read()
    mono = np.array([[int(v) for v in m] for m in re.findall(r"\{(-?\d+), (-?\d+), (-?\d+)\}",
                                                              txt.split("se_ps_mono")[1].split(";")[0])])

    def rows(name):
        body = txt.split("se_ps_%s[" % name)[1].split("};")[0]
        return [(int(n), int(j), int(a), int(b), int(k), float(c)) for n, j, a, b, k, c in
                re.findall(r"\{(\d+), (\d+), (\d+), (\d+), (\d+), ([-0-9.e+]+)\}", body)]
    return mono, rows("stokeslet"), rows("stresslet")


def _stokeslet_closed(r, n):
    r2 = r @ r
    return 4 * n * n * np.eye(3) * r2 ** (n - 1) - (4 * n * (n - 1) * np.outer(r, r) * r2 ** (n - 2) if n > 1 else 0)


def _stresslet_closed(r, n):
    r2 = r @ r
    d = np.eye(3)
    t1 = (np.einsum("jl,m->jlm", d, r) + np.einsum("mj,l->jlm", d, r) + np.einsum("lm,j->jlm", d, r))
    out = np.zeros((3, 3, 3))
    if n >= 2:
        out += 2 * n * (2 * n - 2) * (2 * n - 1) * t1 * r2 ** (n - 2)
    if n >= 3:
        out -= 4 * n * (2 * n - 2) * (2 * n - 4) * np.einsum("j,l,m->jlm", r, r, r) * r2 ** (n - 3)
    return out


def test_tables_reproduce_direct_sums():
    mono, ts, tt = _tables()
    rng = np.random.default_rng(1)
    y = rng.random((7, 3))
    fs = rng.standard_normal((7, 3))
    q = rng.standard_normal((7, 3))
    nu = rng.standard_normal((7, 3))
    x = rng.random(3)
    for n in (1, 2, 3):
        us = np.zeros(3)
        ut = np.zeros(3)
        for s_ in range(7):
            r = x - y[s_]
            us += _stokeslet_closed(r, n) @ fs[s_]
            ut += np.einsum("jlm,l,m->j", _stresslet_closed(r, n), q[s_], nu[s_])
        # from the tables
        xm = np.prod(x[None, :] ** mono, axis=1)
        ym = np.prod(y[:, None, :] ** mono[None, :, :], axis=2)       # (sources, monomials)
        Ms = ym.T @ fs                                                 # (monomials, 3)
        Mt = ym.T @ (q[:, :, None] * nu[:, None, :]).reshape(7, 9)     # (monomials, 9)
        vs = np.zeros(3)
        vt = np.zeros(3)
        for nn, j, a, b, k, c in ts:
            if nn == n:
                vs[j] += c * xm[a] * Ms[b, k]
        for nn, j, a, b, k, c in tt:
            if nn == n:
                vt[j] += c * xm[a] * Mt[b, k]
        assert np.allclose(vs, us, rtol=1e-12, atol=1e-12 * (np.abs(us).max() + 1.0)), (n, vs, us)
        assert np.allclose(vt, ut, rtol=1e-12, atol=1e-12 * (np.abs(ut).max() + 1.0)), (n, vt, ut)


def _screened_power(n, r, xi):
    """(gamma * |.|^(2n))(x) at |x| = r by quadrature, gamma the Hasimoto screening function
    xi^3 / pi^(3/2) exp(-xi^2 s^2) (5/2 - xi^2 s^2), whose transform is
    (1 + k^2/4xi^2) exp(-k^2/4xi^2): the angular integral of (r^2 + s^2 - 2 r s mu)^n over
    mu in [-1, 1] exactly (polynomial), the radial one numerically."""
    from numpy.polynomial import polynomial as Pn
    from scipy.integrate import quad

    def radial(s):
        # coefficients in mu of (r^2 + s^2 - 2 r s mu)^n, integrated over [-1, 1]
        c = Pn.polypow([r * r + s * s, -2 * r * s], n)
        ci = Pn.polyint(c)
        ang = Pn.polyval(1.0, ci) - Pn.polyval(-1.0, ci)
        g = xi ** 3 / np.pi ** 1.5 * np.exp(-xi * xi * s * s) * (2.5 - xi * xi * s * s)
        return 2 * np.pi * g * s * s * ang

    return quad(radial, 0, 12 / xi, epsabs=0, epsrel=1e-11, limit=200)[0]


@pytest.mark.parametrize("n,extra", [(1, 0.0), (2, 0.0), (3, -840.0 / 32.0)])
def test_screening_of_the_split_powers(n, extra):
    """The Fourier part sees r^(2n) through the Hasimoto screening: r^2 and r^4 come out
    unchanged up to a constant, r^6 gains -840/(32 xi^4) r^2 (plus a constant): the
    screened power minus r^(2n) + 840/(32 xi^4) r^2 is the same at every r."""
    xi = 3.0
    rs = [0.1, 0.35, 0.8, 1.3]
    d = [_screened_power(n, r, xi) - r ** (2 * n) - extra / xi ** 4 * r * r for r in rs]
    scale = max(abs(_screened_power(n, r, xi)) for r in rs)
    assert max(d) - min(d) < 1e-9 * scale, d
