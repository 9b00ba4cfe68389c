"""Pins of the exact-Ewald oracle (oracle/ewald_oracle.c) to things other than itself.

Every check here compares the oracle with an independent fact fixed by the paper or by
mathematics (Sec. 2 and Apps. A-B of Bagge & Tornberg 2022):
  * xi-independence of the total u^R + u^F (+ k0, self)       -- Sec. 2.4, Eq. Dp-ewald-decomp
  * App. A / App. B tensors vs quadrature of their defining integrals
  * absolutely convergent 1P rotlet / stresslet image sums      -- Sec. 2 (convergence remark)
  * the stresslet integral identity (0 inside, 8 pi q outside)  -- Eq. stresslet-identity
  * special functions (K_nu identities, E_n) and printed limits -- Eqs. Knu-def, 1p-*-limit
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import ewald as E

KERNELS = ["stokeslet", "rotlet", "stresslet"]


def _strengths(rng, kernel, n):
    if kernel == "stresslet":
        q = rng.standard_normal((n, 3))
        nu = rng.standard_normal((n, 3))
        nu /= np.linalg.norm(nu, axis=1, keepdims=True)
        return np.hstack([q, nu])
    return rng.standard_normal((n, 3))


def _gf_numpy(kernel, xi, k):
    """G^F(k; xi) for an array of wave vectors k (..., 3), Eqs. (stokeslet-fourier) -
    (stresslet-fourier); used only as the integrand of the quadrature checks below."""
    k = np.asarray(k, dtype=float)
    k2 = np.sum(k * k, axis=-1)
    gE = np.exp(-k2 / (4 * xi * xi))
    gH = gE * (1 + k2 / (4 * xi * xi))
    d = np.eye(3)
    if kernel == "stokeslet":
        K = -d * k2[..., None, None] + k[..., :, None] * k[..., None, :]
        return (K * (-8 * np.pi / k2 ** 2 * gH)[..., None, None]).astype(complex)
    if kernel == "rotlet":
        eps = np.zeros((3, 3, 3))
        eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
        eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
        K = -1j * np.einsum("jlm,...m->...jl", eps, k)
        return K * (4 * np.pi / k2 * gE)[..., None, None]
    K = (-1j * (np.einsum("jl,...m->...jlm", d, k) + np.einsum("mj,...l->...jlm", d, k)
                + np.einsum("lm,...j->...jlm", d, k)) * k2[..., None, None, None]
         + 2j * k[..., :, None, None] * k[..., None, :, None] * k[..., None, None, :])
    return K * (-8 * np.pi / k2 ** 2 * gH)[..., None, None, None]


# ----------------------------------------------------------------- special functions

def test_En_matches_scipy():
    for x in [1e-3, 0.2, 0.9, 1.0, 1.1, 3.0, 12.0, 40.0]:
        assert abs(E.En(1, x) / sp.exp1(x) - 1) < 1e-14
        assert abs(E.En(2, x) / sp.expn(2, x) - 1) < 1e-12
    assert abs(E.En(0, 2.0) - math.exp(-2.0) / 2.0) < 1e-16


@pytest.mark.parametrize("a,b", [(0.7, 1.3), (0.05, 4.0), (6.0, 0.3), (2.0, 20.0)])
def test_Knu_bessel_identity(a, b):
    # K_nu(a,b) + K_{-nu}(b,a) = 2 (a/b)^{nu/2} K_nu(2 sqrt(ab))   [App. B, Harris 2008]
    for nu in (0, 1):
        lhs = E.Knu(nu, a, b) + E.Knu(-nu, b, a)
        rhs = 2 * (a / b) ** (nu / 2) * sp.kv(nu, 2 * math.sqrt(a * b))
        assert abs(lhs / rhs - 1) < 1e-13


@pytest.mark.parametrize("a,b", [(0.7, 1.3), (9.0, 0.2), (0.1, 2.0)])
def test_Knu_recurrences(a, b):
    # a K_{-1}(a,b) - b K_1(a,b) = e^{-a-b}     [App. B]
    assert abs(a * E.Knu(-1, a, b) - b * E.Knu(1, a, b) - math.exp(-a - b)) < 1e-14 * math.exp(-a - b) * 50
    # K_nu(a,0) = E_{nu+1}(a)                    [below Eq. 1p-rotlet-Q]
    for nu in (-1, 0, 1, 2):
        assert abs(E.Knu(nu, a, 0.0) / sp.expn(nu + 1, a) - 1) < 1e-13
    # d/db K_nu = -K_{nu+1}: central difference
    h = 1e-5 * max(b, 1)
    for nu in (-1, 0, 1):
        d = (E.Knu(nu, a, b + h) - E.Knu(nu, a, b - h)) / (2 * h)
        assert abs(d + E.Knu(nu + 1, a, b)) < 1e-8 * abs(E.Knu(nu + 1, a, b))


# ------------------------------------------------------------- App. A / B tensors

@pytest.mark.parametrize("kernel", KERNELS)
def test_Q2p_matches_quadrature(kernel):
    """App. A closed forms vs (1/2pi) int G^F(k1,k2,kappa3) e^{i kappa3 r3} d kappa3."""
    xi = 3.0
    K = 2 * xi * 7.5
    xg, wg = np.polynomial.legendre.leggauss(600)
    kap = K * xg
    w = K * wg
    for k1, k2, r3 in [(2 * np.pi, 0.0, 0.3), (2 * np.pi, 4 * np.pi, -0.2), (-2 * np.pi, 2 * np.pi, 0.45)]:
        kv = np.stack([np.full_like(kap, k1), np.full_like(kap, k2), kap], axis=-1)
        G = _gf_numpy(kernel, xi, kv)
        ph = np.exp(1j * kap * r3) * w / (2 * np.pi)
        q = np.tensordot(ph, G, axes=(0, 0))
        c = E.Q2p(kernel, xi, k1, k2, r3)
        assert np.abs(q - c).max() < 1e-12 * np.abs(q).max()


@pytest.mark.parametrize("kernel", KERNELS)
def test_Q1p_matches_quadrature(kernel):
    """App. B closed forms vs (1/(2pi)^2) iint G^F(k1,kap2,kap3) e^{i(kap2 r2+kap3 r3)}."""
    xi = 2.0
    K = 2 * xi * 7.0
    xg, wg = np.polynomial.legendre.leggauss(220)
    kap = K * xg
    w = K * wg
    K2, K3 = np.meshgrid(kap, kap, indexing="ij")
    W = np.outer(w, w)
    for k1, r2, r3 in [(2 * np.pi, 0.3, -0.2), (-4 * np.pi, 0.05, 0.4), (np.pi, 0.0, 0.0)]:
        kv = np.stack([np.full_like(K2, k1), K2, K3], axis=-1)
        G = _gf_numpy(kernel, xi, kv)
        ph = np.exp(1j * (K2 * r2 + K3 * r3)) * W / (2 * np.pi) ** 2
        q = np.tensordot(ph, G, axes=([0, 1], [0, 1]))
        c = E.Q1p(kernel, xi, k1, r2, r3)
        assert np.abs(q - c).max() < 1e-11 * np.abs(q).max()


def test_zero_mode_limits_are_continuous():
    # Eq. (1p-stokeslet-Q0-limit) and the zero limits of rotlet/stresslet
    xi = 3.0
    for kernel in KERNELS:
        lim = E.Q1p0(kernel, xi, 0.0, 0.0)
        near = E.Q1p0(kernel, xi, 1e-7, -0.7e-7)
        assert np.abs(lim - near).max() < 200 * 1.22e-7  # approaches the limit like O(rho)
    # Q^{2P,(0)} is smooth at r3 = 0 and odd/even as printed
    for kernel in KERNELS:
        a = E.Q2p0(kernel, xi, 0.2)
        b = E.Q2p0(kernel, xi, -0.2)
        if kernel == "stokeslet":
            assert np.allclose(a, b, rtol=0, atol=1e-14)
        else:
            assert np.allclose(a, -b, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- whole-sum pins

@pytest.mark.parametrize("D,L", [(3, [1, 1, 1]), (3, [1.0, 0.8, 1.3]), (2, [1, 1, 1]), (2, [1, 1, 0.5]),
                                 (1, [1, 1, 1]), (1, [2, 1, 1])])
@pytest.mark.parametrize("kernel", KERNELS)
def test_total_is_xi_independent(D, L, kernel):
    """u = u^R + u^F (+k0 +self) does not depend on xi (Sec. 2.4)."""
    rng = np.random.default_rng(7 + D)
    n = 10
    x = rng.random((n, 3)) * np.asarray(L)
    f = _strengths(rng, kernel, n)
    xi0 = E.default_xi(D, L)
    u1 = E.potential(D, L, kernel, x, f, xi=xi0)
    u2 = E.potential(D, L, kernel, x, f, xi=1.6 * xi0)
    # explicit, distinct targets too
    t = rng.random((4, 3)) * np.asarray(L)
    v1 = E.potential(D, L, kernel, x, f, targets=t, xi=xi0)
    v2 = E.potential(D, L, kernel, x, f, targets=t, xi=1.6 * xi0)
    assert E.rms_rel(u1, u2) < 1e-12
    assert E.rms_rel(v1, v2) < 1e-12


def test_star_form_equals_explicit_coincident_targets():
    rng = np.random.default_rng(3)
    x = rng.random((8, 3))
    for kernel in KERNELS:
        f = _strengths(rng, kernel, 8)
        a = E.potential(3, [1, 1, 1], kernel, x, f)
        b = E.potential(3, [1, 1, 1], kernel, x, f, targets=x.copy())
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("kernel", ["rotlet", "stresslet"])
def test_1p_rotlet_stresslet_equal_image_sum(kernel):
    """D = 1 rotlet and stresslet sums converge absolutely (Sec. 2): brute-force image sum
    with Richardson extrapolation in the image count."""
    rng = np.random.default_rng(11)
    L = np.array([1.5, 1.0, 1.0])
    n = 5
    x = rng.random((n, 3)) * L
    f = _strengths(rng, kernel, n)

    def image_sum(P):
        u = np.zeros((n, 3))
        p = np.arange(-P, P + 1)
        for m in range(n):
            for j in range(n):
                r = x[m] - x[j] + np.outer(p, [L[0], 0, 0])
                if m == j:
                    r = r[p != 0]
                r2 = np.sum(r * r, axis=1)
                rr = np.sqrt(r2)
                if kernel == "rotlet":   # Omega_jl f_l = (f x r)_j / r^3
                    u[m] += np.sum(np.cross(f[j], r) / (rr ** 3)[:, None], axis=0)
                else:                    # T_jlm q_l nu_m = -6 r_j (r.q)(r.nu) / r^5
                    q, nu = f[j, :3], f[j, 3:]
                    u[m] += np.sum(-6 * r * ((r @ q) * (r @ nu) / rr ** 5)[:, None], axis=0)
        return u

    s1 = image_sum(4000)
    s2 = image_sum(8000)
    brute = (4 * s2 - s1) / 3
    ref = E.potential(1, L, kernel, x, f)
    assert E.rms_rel(ref, brute) < 1e-10


def _sphere(center, a, nth=24, nph=48):
    ct, wt = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C ** 2)
    nrm = np.stack([S * np.cos(P), S * np.sin(P), C], axis=-1).reshape(-1, 3)
    w = (np.outer(wt, np.full(nph, 2 * np.pi / nph)) * a * a).reshape(-1)
    return center + a * nrm, nrm, w


@pytest.mark.parametrize("D", [0, 1, 2, 3])
def test_stresslet_integral_identity(D):
    """Eq. (stresslet-identity) for every D (Sec. 2.5).

    With T_jlm = -6 r_j r_l r_m / r^5, r = x - y and nu the OUTWARD normal, the divergence
    theorem gives 8 pi q0 at points enclosed by the surface and 0 outside (div_y T = 0 away
    from y = x; the excised ball gives 6 * (4 pi / 3) delta_jl). The printed equation lists
    the two regions the other way round, which is the inward-normal form."""
    L = np.array([1.0, 1.0, 1.0])
    c = np.array([0.5, 0.5, 0.5])
    y, nrm, w = _sphere(c, 0.2)
    q0 = np.array([0.3, -1.1, 0.7])
    f = np.hstack([q0[None, :] * w[:, None], nrm])
    inside = np.array([[0.5, 0.5, 0.5], [0.55, 0.45, 0.52]])
    outside = np.array([[0.1, 0.1, 0.1], [0.9, 0.2, 0.6]])
    ui = E.potential(D, L, "stresslet", y, f, targets=inside)
    uo = E.potential(D, L, "stresslet", y, f, targets=outside)
    assert np.abs(uo).max() < 1e-8
    assert np.abs(ui - 8 * np.pi * q0).max() < 1e-8


def test_free_space_kernels_special_values():
    """Eq. (stokes-kernels) at r = (1,0,0): S = diag(2,1,1), Omega f = f x r, T = -6 e1e1e1."""
    x = np.zeros((1, 3))
    t = np.array([[1.0, 0.0, 0.0]])
    us = E.potential(0, [1, 1, 1], "stokeslet", x, np.array([[1.0, 2.0, 3.0]]), targets=t)
    assert np.allclose(us, [[2.0, 2.0, 3.0]], atol=1e-15)
    ur = E.potential(0, [1, 1, 1], "rotlet", x, np.array([[1.0, 2.0, 3.0]]), targets=t)
    assert np.allclose(ur, [np.cross([1.0, 2.0, 3.0], [1.0, 0, 0])], atol=1e-15)
    ut = E.potential(0, [1, 1, 1], "stresslet", x, np.array([[2.0, 1.0, 0.0, 3.0, 0.0, 1.0]]), targets=t)
    assert np.allclose(ut, [[-36.0, 0.0, 0.0]], atol=1e-14)


def test_3p_self_term_and_magnitudes():
    """Self term Eq. (3p-stokeslet-self-term); Fourier-part rms near the values printed for
    N = 1000, L = 1, Q = 1, xi = 10 (Sec. 4.6: about 2, 20 and 7 for S, T, Omega)."""
    rng = np.random.default_rng(5)
    n = 1000
    x = rng.random((n, 3))
    for kernel, printed in [("stokeslet", 2.0), ("stresslet", 20.0), ("rotlet", 7.0)]:
        f = rng.uniform(-1, 1, (n, 6 if kernel == "stresslet" else 3))
        if kernel == "stresslet":
            Q = np.sum((f[:, :3, None] * f[:, None, 3:]) ** 2)
        else:
            Q = np.sum(f ** 2)
        f = f / math.sqrt(Q) if kernel != "stresslet" else np.hstack([f[:, :3] / Q ** 0.25, f[:, 3:] / Q ** 0.25])
        p = E.parts(3, [1, 1, 1], kernel, x, f, xi=10.0)
        rms = math.sqrt(np.mean(np.sum(p["fourier"] ** 2, axis=1)))
        assert printed / 3 < rms < printed * 3
        if kernel == "stokeslet":
            assert np.allclose(p["self"], -4 * 10.0 / math.sqrt(math.pi) * f, atol=1e-15)
        else:
            assert np.abs(p["self"]).max() == 0.0


# ------------------------------------------------------------- harmonic field

def test_harmonic_field_free_space_is_the_direct_sum():
    """E_j = sum_n q_n (x - x_n)_j / |x - x_n|^3 (star form: n != m), from the rotlet identity,
    against a direct numpy sum; also at explicit targets."""
    rng = np.random.default_rng(11)
    x = rng.random((40, 3))
    q = rng.standard_normal(40)
    e = E.harmonic_field(0, [1, 1, 1], x, q)
    r = x[:, None, :] - x[None, :, :]
    d = np.linalg.norm(r, axis=-1)
    np.fill_diagonal(d, np.inf)
    ref = np.einsum("mnj,n->mj", r / d[..., None] ** 3, q)
    assert np.abs(e - ref).max() < 1e-12 * np.abs(ref).max()
    t = rng.random((7, 3))
    r = t[:, None, :] - x[None, :, :]
    ref_t = np.einsum("mnj,n->mj", r / np.linalg.norm(r, axis=-1)[..., None] ** 3, q)
    assert np.abs(E.harmonic_field(0, [1, 1, 1], x, q, targets=t) - ref_t).max() < 1e-12 * np.abs(ref_t).max()


@pytest.mark.parametrize("D", [1, 2, 3])
def test_harmonic_field_periodic_is_xi_independent(D):
    rng = np.random.default_rng(12 + D)
    x = rng.random((30, 3))
    q = rng.standard_normal(30)
    a = E.harmonic_field(D, [1, 1, 1], x, q, xi=4.0)
    b = E.harmonic_field(D, [1, 1, 1], x, q, xi=7.0)
    assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()


# ------------------------------------------------ harmonic potential phi = sum q / r (scalar)

def _madelung():
    vals = {}
    path = __file__.rsplit("/", 1)[0] + "/golden/madelung.txt"
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, value = line.split()[:2]
        vals[name] = float(value)
    return vals


def _evjen_2d(n):
    """Checkerboard Madelung constant by Evjen's method: the square of side 2n around the
    ion, edge charges halved and corner charges quartered (so each shell is neutral)."""
    i = np.arange(-n, n + 1)
    I, J = np.meshgrid(i, i, indexing="ij")
    w = np.where(np.abs(I) == n, 0.5, 1.0) * np.where(np.abs(J) == n, 0.5, 1.0)
    r = np.hypot(I, J)
    r[n, n] = 1.0
    s = w * (-1.0) ** (I + J) / r
    s[n, n] = 0.0
    return -s.sum()


def test_harmonic_madelung_constants():
    """Ionic crystals of alternating unit charges: the 3P rock salt (cube of side 1, d = 1/2),
    the 2P checkerboard (d = 1/2, the free direction at any height) and the 1P alternating
    chain (d = 1/2); the potential at each ion is -+M / d, for two values of xi."""
    M = _madelung()
    # the 2-D constant also by brute force (Evjen sums, Richardson over n with error ~ n^-3)
    a, b = _evjen_2d(200), _evjen_2d(400)
    assert abs((8 * b - a) / 7 - M["square_checkerboard_2d"]) < 1e-10
    g = np.array([(i, j, k) for i in range(2) for j in range(2) for k in range(2)], dtype=float)
    x3 = 0.5 * g
    q3 = np.where(g.sum(axis=1) % 2 == 0, 1.0, -1.0)
    x2 = np.array([[0, 0, 0.3], [0.5, 0, 0.3], [0, 0.5, 0.3], [0.5, 0.5, 0.3]])
    q2 = np.array([1.0, -1.0, -1.0, 1.0])
    x1 = np.array([[0.0, 0.4, 0.6], [0.5, 0.4, 0.6]])
    q1 = np.array([1.0, -1.0])
    for D, x, q, name in ((3, x3, q3, "rock_salt_3d"), (2, x2, q2, "square_checkerboard_2d"),
                          (1, x1, q1, "alternating_chain_1d")):
        for s in (1.0, 1.8):
            phi = E.harmonic(D, [1.0, 1.0, 1.0], x, q, xi=s * E.default_xi(D, [1.0, 1.0, 1.0]))
            assert np.abs(phi * 0.5 + q * M[name]).max() < 1e-12, (D, s)


@pytest.mark.parametrize("D,L", [(3, (1.0, 1.2, 0.8)), (2, (1.0, 1.3, 1.0)), (1, (1.2, 1.0, 1.0))])
def test_harmonic_xi_independence_non_neutral(D, L):
    """A charged (non-neutral) system: the total is independent of xi, including the 3P
    zero-mean constant; star form and explicit targets (some on sources)."""
    rng = np.random.default_rng(11 + D)
    x = rng.random((14, 3)) * L
    q = rng.standard_normal(14) + 0.4
    t = np.vstack([rng.random((5, 3)) * L, x[:2]])
    xi0 = E.default_xi(D, L)
    for tg in (None, t):
        a = E.harmonic(D, L, x, q, targets=tg, xi=xi0)
        b = E.harmonic(D, L, x, q, targets=tg, xi=1.7 * xi0)
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    # explicit targets on the sources give the star values
    star = E.harmonic(D, L, x, q, xi=xi0)
    assert np.abs(E.harmonic(D, L, x, q, targets=x[:2], xi=xi0) - star[:2]).max() < 1e-12 * np.abs(star).max()


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_harmonic_gradient_is_the_field(D):
    """-grad phi (5-point central differences, h = 1e-3) equals the harmonic field of the
    same charges, which the oracle computes independently from the rotlet tensors."""
    rng = np.random.default_rng(20 + D)
    L = [1.0, 1.0, 1.0]
    x = rng.random((15, 3))
    q = rng.standard_normal(15)
    t = rng.random((4, 3))
    h = 1e-3
    g = np.zeros((4, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        f = [E.harmonic(D, L, x, q, targets=t + s * e) for s in (2, 1, -1, -2)]
        g[:, j] = -(-f[0] + 8 * f[1] - 8 * f[2] + f[3]) / (12 * h)
    F = E.harmonic_field(D, L, x, q, targets=t)
    assert np.abs(g - F).max() < 1e-7 * np.abs(F).max()


def test_harmonic_gauges_far_field():
    """The k^P = 0 conventions seen from far away, where every k^P != 0 mode has decayed:
    2P tends to -(2 pi / A) sum q |z - z_n| and 1P to -(2 / L_1) sum q log(rho_n) (l_H = 1)."""
    rng = np.random.default_rng(30)
    L = [1.0, 1.0, 1.0]
    x = rng.random((10, 3))
    q = rng.standard_normal(10)
    t = np.array([[0.3, 0.7, 7.0], [0.1, 0.2, -6.0]])
    ff = np.array([-2 * np.pi * (q * np.abs(p[2] - x[:, 2])).sum() for p in t])
    assert np.abs(E.harmonic(2, L, x, q, targets=t) - ff).max() < 1e-12 * np.abs(ff).max()
    t = np.array([[0.3, 7.0, 0.5], [0.1, -3.0, 6.0]])
    ff = np.array([-2 * (q * np.log(np.hypot(p[1] - x[:, 1], p[2] - x[:, 2]))).sum() for p in t])
    assert np.abs(E.harmonic(1, L, x, q, targets=t) - ff).max() < 1e-12 * np.abs(ff).max()


def test_harmonic_3p_zero_mean():
    """The 3P potential of a charged system has zero mean over the cell: the midpoint rule on
    32^3 targets (error from the 1/r singularities ~ h^2) against the constant -pi Q/(xi^2 V)
    that the convention adds (0.27 here)."""
    rng = np.random.default_rng(5)
    x = rng.random((6, 3))
    q = rng.standard_normal(6) + 0.5
    n = 32
    g = (np.arange(n) + 0.5) / n
    t = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    phi = E.harmonic(3, [1.0, 1.0, 1.0], x, q, targets=t, xi=3.5)
    assert abs(phi.mean()) < 0.01 * np.pi * abs(q.sum()) / 3.5 ** 2


def test_harmonic_direct_0p_by_hand():
    """Two charges at distance 2 and a target between them."""
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    q = np.array([3.0, -1.0])
    phi = E.harmonic(0, [1.0, 1.0, 1.0], x, q, targets=np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]))
    assert np.allclose(phi, [3.0 - 1.0, -0.5], rtol=0, atol=1e-15)
    assert np.allclose(E.harmonic(0, [1.0, 1.0, 1.0], x, q), [-0.5, 1.5], rtol=0, atol=1e-15)
