"""Pins of the numpy Algorithm 1 oracle (oracle/se_steps.py).

The SE method approximates the exact Ewald sum to the tolerance its parameters were chosen
for (Sec. 4). With generous parameters (k_inf = pi/h far beyond the screening, wide window,
ample padding and upsampling) Alg. 1 plus the real-space sum, the self term and the gauge
constants must reproduce the exact Ewald sums of oracle/ewald_oracle.c (direct k-sum for
3P, App. A/B closed forms for 2P/1P, direct sum for 0P) to ~1e-9 -- an independent check of
every step, including the modified kernels, the adaptive FFT and the 0P precomputation.
"""
import math

import numpy as np
import pytest

from oracle import ewald as E
from oracle import se_steps as S

KERNELS = ["stokeslet", "rotlet", "stresslet"]


def _strengths(rng, kernel, n):
    if kernel == "stresslet":
        nu = rng.standard_normal((n, 3))
        nu /= np.linalg.norm(nu, axis=1, keepdims=True)
        return np.hstack([rng.standard_normal((n, 3)), nu])
    return rng.standard_normal((n, 3))


def test_window_transforms_match_quadrature():
    """w^_0 of Eq. (KB-window) and of the untruncated Gaussian against quadrature of w_0."""
    h, P = 0.05, 10
    for kind in ("kb", "gaussian"):
        w = S.Window(kind, P, h)
        xg, wg = np.polynomial.legendre.leggauss(400)
        a = w.aw if kind == "kb" else 6 * w.aw
        r = a * xg
        for k in (0.0, 7.0, 31.0):
            vals = (np.where(np.abs(r) <= w.aw, np.exp(-w.alpha * (r / w.aw) ** 2), 0.0)
                    if kind == "gaussian" else w(r))
            if kind == "gaussian":   # the transform of the UNtruncated Gaussian
                vals = np.exp(-w.alpha * (r / w.aw) ** 2)
            q = np.sum(a * wg * vals * np.cos(k * r))
            assert abs(q - w.hat(k)) < 1e-10 * abs(w.hat(0.0))


def test_window_error_follows_estimate_and_pkb_adds_none():
    """Eq. (approximation-estimate): with the exact KB window (beta = 2.5 P) the Fourier-part
    error is ~10 e^{-2.5 P} relative; the PKB window with nu of Eq. (PKB-parameters) adds no
    further error (Sec. 4.3); the truncated Gaussian needs a larger P for the same error."""
    rng = np.random.default_rng(2)
    N = 120
    x = rng.random((N, 3))
    f = rng.standard_normal((N, 3))
    xi = 8.0
    ref = E.parts(3, [1, 1, 1], "stokeslet", x, f, xi=xi)["fourier"]
    for P in (4, 6, 8, 10):
        e = {w: E.rms_rel(S.fourier_part_3p("stokeslet", x, f, [1, 1, 1], (48, 48, 48), xi, w, P), ref)
             for w in ("kb", "pkb", "gaussian")}
        est = 10 * math.exp(-2.5 * P)
        assert est / 4 < e["kb"] < 4 * est, (P, e)
        assert e["pkb"] < 1.3 * e["kb"], (P, e)
        assert e["gaussian"] > 3 * e["kb"], (P, e)


def test_modified_kernel_limits():
    """Printed k -> 0 limits: Eqs. (optimal-biharmonic-0p-limit), (optimal-1p-*-limit), the
    2P limits below Eq. (2p-vico-H-kernel), and continuity of the series branches."""
    R = 1.7
    assert abs(S.hat_B0p(np.array([0.0]), R)[0] + math.pi * R ** 4 / 15) < 1e-12 * R ** 4
    assert abs(S.hat_H0p(np.array([0.0]), R)[0] - 2 * math.pi * R ** 2) < 1e-12
    assert abs(S.hat_H1p(np.array([0.0]), R)[0] - math.pi * R ** 2) < 1e-12
    assert abs(S.hat_B1p(np.array([0.0]), R)[0] + math.pi * R ** 4 / 8) < 1e-12 * R ** 4
    assert abs(S.hat_H2p(np.array([0.0]), R)[0] + 2 * math.pi * R ** 2) < 1e-12
    assert S.hat_Z2p(np.array([0.0]), R)[0] == 0
    for fn, tsw in ((S.hat_B0p, 1.0), (S.hat_H1p, 2.0), (S.hat_B1p, 2.0), (S.hat_H2p, 0.5)):
        k = np.array([tsw / R * (1 - 1e-9), tsw / R * (1 + 1e-9)])
        v = fn(k, R)
        assert abs(v[0] - v[1]) < 1e-7 * abs(v[0])  # no jump between the two branches


@pytest.mark.parametrize("kernel", KERNELS)
def test_alg1_3p_reproduces_ewald(kernel):
    rng = np.random.default_rng(2)
    N = 40
    x = rng.random((N, 3))
    f = _strengths(rng, kernel, N)
    xi = 8.0
    u = S.fourier_part_3p(kernel, x, f, [1, 1, 1], (48, 48, 48), xi, "pkb", 16)
    p = E.parts(3, [1, 1, 1], kernel, x, f, xi=xi)
    tot = u + p["real"] + p["self"] + p["k0"]
    assert E.rms_rel(tot, E.potential(3, [1, 1, 1], kernel, x, f)) < 1e-11


def _reduced_case(D, kernel, seed):
    rng = np.random.default_rng(seed)
    L = np.array([1.0, 1.0, 1.0])
    N = 24
    x = rng.random((N, 3)) * L
    f = _strengths(rng, kernel, N)
    xi, M, P = 6.0, 40, 16
    h = 1.0 / M
    lam = 2.4 if D > 0 else {"stokeslet": 2.2, "stresslet": 2.4, "rotlet": 1.5}[kernel]
    theta = 0 if kernel == "rotlet" else 8
    me = 4 * math.ceil((M + P + (lam - 1) * max(P, theta)) / 4)
    Mext = [0, 0, 0]
    for d in range(D, 3):
        Mext[d] = me
    u = S.fourier_part(D, kernel, x, f, L, h, P, xi, "pkb", Mext=Mext, s_star=3.0, kbar_star=6)
    p = E.parts(D, L, kernel, x, f, xi=xi) if D > 0 else None
    return L, x, f, xi, u, p


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("D", [2, 1])
def test_alg1_aft_reproduces_app_ab(D, kernel):
    """D = 2, 1: modified kernels (Sec. 3.1) + adaptive FFT (Sec. 3.4) + gauge constant vs the
    App. A / App. B sums."""
    L, x, f, xi, u, _ = _reduced_case(D, kernel, 10 + D)
    ur = np.zeros((x.shape[0], 3))
    E.lib().orc_real(D, E._p(L), xi, 7.0 / xi, E.kernel_id(kernel), x.shape[0], E._p(np.ascontiguousarray(x)),
                     E._p(np.ascontiguousarray(f)), x.shape[0], None, E._p(ur))
    tot = u + ur + S.self_term(kernel, xi, f)
    ref = E.potential(D, L, kernel, x, f)
    assert E.rms_rel(tot, ref) < 1e-9


@pytest.mark.parametrize("kernel", KERNELS)
def test_alg1_0p_with_precomputation_reproduces_direct_sum(kernel):
    """D = 0: precomputed truncated kernel (Sec. 3.5, mollified for the biharmonic) + gauge
    constant vs the direct sum."""
    L, x, f, xi, u, _ = _reduced_case(0, kernel, 20)
    ur = np.zeros((x.shape[0], 3))
    E.lib().orc_real(0, E._p(L), xi, 7.0 / xi, E.kernel_id(kernel), x.shape[0], E._p(np.ascontiguousarray(x)),
                     E._p(np.ascontiguousarray(f)), x.shape[0], None, E._p(ur))
    tot = u + ur + S.self_term(kernel, xi, f)
    ref = E.potential(0, L, kernel, x, f)
    assert E.rms_rel(tot, ref) < 1e-9


# ----------------------------------------------------------------- harmonic field

def _field_real(D, L, xi, x, q):
    """Real-space part of the harmonic field with splitting xi: the rotlet's real-space sums
    with torques along the axes (E_1 = (Omega q e_3)_2, E_2 = (Omega q e_1)_3,
    E_3 = (Omega q e_2)_1; the identity holds term by term, both real-space kernels being
    derivatives of erfc(xi r)/r)."""
    N = x.shape[0]
    out = np.zeros((N, 3))
    for comp, axis, row in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        f = np.zeros((N, 3))
        f[:, axis] = q
        ur = np.zeros((N, 3))
        E.lib().orc_real(D, E._p(np.asarray(L, dtype=float)), xi, 7.0 / xi, E.kernel_id("rotlet"), N,
                         E._p(np.ascontiguousarray(x)), E._p(f), N, None, E._p(ur))
        out[:, comp] = ur[:, row]
    return out


def test_alg1_harmonic_field_3p():
    rng = np.random.default_rng(31)
    N = 40
    x = rng.random((N, 3))
    q = rng.standard_normal(N)
    xi = 8.0
    u = S.fourier_part_3p("harmonic_field", x, q[:, None], [1, 1, 1], (48, 48, 48), xi, "pkb", 16)
    tot = u + _field_real(3, [1, 1, 1], xi, x, q)
    assert E.rms_rel(tot, E.harmonic_field(3, [1, 1, 1], x, q)) < 1e-11


@pytest.mark.parametrize("D", [2, 1, 0])
def test_alg1_harmonic_field_free_directions(D):
    """D = 2, 1: the harmonic modified kernels on the k^P = 0 class with the adaptive FFT;
    D = 0: the precomputed truncated harmonic kernel (no mollifier); vs the exact field."""
    rng = np.random.default_rng(40 + D)
    L = np.array([1.0, 1.0, 1.0])
    N = 24
    x = rng.random((N, 3))
    q = rng.standard_normal(N)
    xi, M, P = 6.0, 40, 16
    lam = 2.4 if D > 0 else 1.5          # Table 4, rotlet column (the field takes its rules)
    me = 4 * math.ceil((M + P + (lam - 1) * P) / 4)
    Mext = [0, 0, 0]
    for d in range(D, 3):
        Mext[d] = me
    u = S.fourier_part(D, "harmonic_field", x, q[:, None], L, 1.0 / M, P, xi, "pkb", Mext=Mext, s_star=3.0,
                       kbar_star=6)
    tot = u + _field_real(D, L, xi, x, q)
    assert E.rms_rel(tot, E.harmonic_field(D, L, x, q)) < 1e-9


# ------------------------------------------------------------ harmonic potential (scalar)

def _potential_real(D, L, xi, x, q):
    ur = np.zeros(x.shape[0])
    E.lib().orc_h_real(D, E._p(np.asarray(L, dtype=float)), xi, 7.0 / xi, x.shape[0],
                       E._p(np.ascontiguousarray(x)), E._p(np.ascontiguousarray(q)), x.shape[0], None, E._p(ur))
    return ur


def test_alg1_harmonic_potential_3p():
    """A charged system: Alg. 1 + real space + self term + the zero-mean constant."""
    rng = np.random.default_rng(51)
    N = 40
    x = rng.random((N, 3))
    q = rng.standard_normal(N) + 0.3
    xi = 8.0
    u = S.fourier_part_3p("harmonic", x, q[:, None], [1, 1, 1], (48, 48, 48), xi, "pkb", 16)[:, 0]
    tot = u + _potential_real(3, [1, 1, 1], xi, x, q) + S.self_term("harmonic", xi, q)[:, 0] \
        + S.k0_harmonic_3p([1, 1, 1], xi, q)
    ref = E.harmonic(3, [1, 1, 1], x, q)
    assert np.sqrt(np.mean((tot - ref) ** 2) / np.mean(ref ** 2)) < 1e-11


@pytest.mark.parametrize("D", [2, 1, 0])
def test_alg1_harmonic_potential_free_directions(D):
    """D = 2, 1: the truncated harmonic kernels on the k^P = 0 class with the adaptive FFT (and
    the 1P gauge change from l_H = R to 1); D = 0: the precomputed truncated harmonic kernel;
    a charged system against the exact sums."""
    rng = np.random.default_rng(60 + D)
    L = np.array([1.0, 1.0, 1.0])
    N = 24
    x = rng.random((N, 3))
    q = rng.standard_normal(N) + 0.3
    xi, M, P = 6.0, 40, 16
    lam = 2.4 if D > 0 else 1.5
    me = 4 * math.ceil((M + P + (lam - 1) * P) / 4)
    Mext = [0, 0, 0]
    for d in range(D, 3):
        Mext[d] = me
    u = S.fourier_part(D, "harmonic", x, q[:, None], L, 1.0 / M, P, xi, "pkb", Mext=Mext, s_star=3.0,
                       kbar_star=6)[:, 0]
    tot = u + _potential_real(D, L, xi, x, q) + S.self_term("harmonic", xi, q)[:, 0]
    ref = E.harmonic(D, L, x, q)
    assert np.sqrt(np.mean((tot - ref) ** 2) / np.mean(ref ** 2)) < 1e-9
