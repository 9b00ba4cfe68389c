"""Algorithm 1 of the paper (Spectral Ewald, Fourier-space part), step by step in plain
numpy FP64.  TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it; the library never does.

Steps, in the paper's order and notation (Sec. 3.2-3.4, Alg. 1):
  (i)   gridding   Phi(x_j) = sum_n sum_p w(x_j - x_n + p) f(x_n)          Eq. SE-gridding-disc
  (ii)  FFT        F_h = FFT(Phi)                                            Eq. SE-FFT-disc
  (iii) scaling    Phi~ = G_R^{DP}(k) gamma^(k) / w^(k)^2 . F_h              Eq. SE-scaling-disc
  (iv)  IFFT       F~ = IFFT(Phi~)                                           Eq. SE-IFFT-disc
  (v)   gathering  u(x_m) = h^3 sum_j F~(x_j) sum_p w(x_m - x_j + p)        Eq. SE-gathering-disc
followed by the self term (Eq. self-term) and, for the 3P stresslet, the k = 0 term
(Eq. k0-stresslet-3p).

Readings of the paper taken here:
  * window taps: for a coordinate u = (x - o)/h in grid units, the P taps are
    j = floor(u) - P/2 + 1, ..., floor(u) + P/2 (so |jh - x| <= a_w = Ph/2);
  * FFT normalisation: the continuous transforms are replaced by the trapezoidal rule,
    F = h^3 sum_j Phi_j e^{-ik x_j}, F^{-1} = (1/|B|) sum_k; the h^3 and 1/|B| cancel
    against the grid size, so Phi~ -> F~ is numpy's fftn / ifftn pair;
  * every mode whose index lies on a Nyquist plane (kbar_i = -M_i/2) is set to zero, which
    keeps the inverse transform exactly real (the dropped content is at the truncation
    level gamma^(pi/h));
  * the truncated Gaussian uses alpha = 0.91 (pi/2) P as printed (Eq. TG-window) and the
    untruncated Gaussian's transform in the scaling step;
  * PKB: on each of the P unit subintervals the exact KB window is interpolated in nu + 1
    Chebyshev points of the first kind, beta = 2.5 P, nu = min(P/2 + 2, 10)
    (Eq. PKB-parameters); the scaling step uses the exact KB transform (Eq. KB-window).
"""
import math

import numpy as np
import scipy.special as sp

STOKESLET, ROTLET, STRESSLET, HARMONIC_FIELD, HARMONIC = 1, 2, 4, 8, 16
_NAMES = {"stokeslet": STOKESLET, "rotlet": ROTLET, "stresslet": STRESSLET, "harmonic_field": HARMONIC_FIELD,
          "harmonic": HARMONIC}
# the harmonic field E = -grad H q (H = 1/r) is a first derivative of H like the rotlet
# (Omega_jl = -eps_jlm d_m H), the harmonic potential H q itself: Ewald screening and the
# harmonic modified kernels for all three
_HARMONIC = (ROTLET, HARMONIC_FIELD, HARMONIC)


def n_out(kernel):
    """Output components per target: 1 for the harmonic potential, 3 otherwise."""
    return 1 if kernel_id(kernel) == HARMONIC else 3


def kernel_id(kernel):
    return _NAMES[kernel] if isinstance(kernel, str) else int(kernel)


# ------------------------------------------------------------------------ windows

class Window:
    """One-dimensional window w_0 with support [-a_w, a_w], a_w = P h / 2 (Sec. 3.3)."""

    def __init__(self, kind, P, h):
        assert P % 2 == 0 and P >= 2
        self.kind, self.P, self.h = kind, P, h
        self.aw = P * h / 2.0
        if kind == "gaussian":
            self.alpha = 0.91 * (math.pi / 2.0) * P          # Eq. (TG-window)
        elif kind in ("kb", "pkb"):
            self.beta = 2.5 * P                                 # Eq. (PKB-parameters)
            self.nu = min(P // 2 + 2, 10)
            if kind == "pkb":
                self._pkb_setup()
        else:
            raise ValueError(kind)

    def _kb(self, r):
        r = np.asarray(r, dtype=float)
        t = 1.0 - (r / self.aw) ** 2
        out = np.where(t >= 0, sp.i0(self.beta * np.sqrt(np.maximum(t, 0.0))) / sp.i0(self.beta), 0.0)
        return out

    def _pkb_setup(self):
        # Chebyshev points of the first kind on [-1, 1]
        n = self.nu + 1
        s = np.cos((2 * np.arange(n) + 1) * math.pi / (2 * n))
        self.coef = []
        for l in range(-self.P // 2, self.P // 2):               # subinterval [l h, (l+1) h]
            r = (l + 0.5 + 0.5 * s) * self.h
            self.coef.append(np.polynomial.chebyshev.chebfit(s, self._kb(r), self.nu))

    def __call__(self, r):
        """w_0(r) for an array of offsets r (same length unit as h)."""
        r = np.asarray(r, dtype=float)
        if self.kind == "gaussian":
            return np.where(np.abs(r) <= self.aw, np.exp(-self.alpha * (r / self.aw) ** 2), 0.0)
        if self.kind == "kb":
            return self._kb(r)
        out = np.zeros_like(r)
        v = r / self.h
        for i, l in enumerate(range(-self.P // 2, self.P // 2)):
            # subintervals (l, l+1], closed on the right: a tap at offset exactly l+1 takes
            # the interpolant of subinterval l at its right end
            m = (v > l) & (v <= l + 1)
            s = 2.0 * (v[m] - l) - 1.0
            out[m] = np.polynomial.chebyshev.chebval(s, self.coef[i])
        return out

    def hat(self, k):
        """Fourier transform w^_0(k) used in the scaling step."""
        k = np.asarray(k, dtype=float)
        if self.kind == "gaussian":                                  # untruncated Gaussian
            return math.sqrt(math.pi / self.alpha) * self.aw * np.exp(-k * k * self.aw ** 2 / (4 * self.alpha))
        z2 = self.beta ** 2 - (k * self.aw) ** 2                     # Eq. (KB-window)
        z = np.sqrt(np.abs(z2))
        with np.errstate(invalid="ignore", divide="ignore"):
            val = np.where(z2 > 0, np.sinh(z) / np.where(z > 0, z, 1.0),
                           np.where(z > 0, np.sin(z) / np.where(z > 0, z, 1.0), 1.0))
        return 2 * self.aw * val / sp.i0(self.beta)


def taps(u, P):
    """First tap index floor(u) - P/2 + 1 for coordinates u in grid units."""
    return np.floor(u).astype(np.int64) - P // 2 + 1


# ---------------------------------------------------------------- Fourier kernels

def _Khat(kernel, k):
    """Operator symbols K^(k) of Eqs. (diffop-rel-fourier-1..3), shape (..., 3, 3[, 3]);
    the harmonic field's gradient -i k, shape (..., 3, 1); the identity for the harmonic
    potential, shape (..., 1, 1)."""
    d = np.eye(3)
    k2 = np.sum(k * k, axis=-1)
    if kernel == HARMONIC:
        return np.ones(k.shape[:-1] + (1, 1), dtype=complex)
    if kernel == HARMONIC_FIELD:
        return (-1j * k)[..., :, None]
    if kernel == STOKESLET:
        return (-d * k2[..., None, None] + k[..., :, None] * k[..., None, :]).astype(complex)
    if kernel == ROTLET:
        eps = np.zeros((3, 3, 3))
        eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
        eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
        return -1j * np.einsum("jlm,...m->...jl", eps, k)
    return (-1j * (np.einsum("jl,...m->...jlm", d, k) + np.einsum("mj,...l->...jlm", d, k)
                   + np.einsum("lm,...j->...jlm", d, k)) * k2[..., None, None, None]
            + 2j * k[..., :, None, None] * k[..., None, :, None] * k[..., None, None, :])


def _screen(kernel, k2, xi):
    gE = np.exp(-k2 / (4 * xi * xi))                                  # Eq. (ewald-screening)
    return gE if kernel in _HARMONIC else gE * (1 + k2 / (4 * xi * xi))   # Eq. (hasimoto-screening)


def kernel_3p(kernel, k, xi):
    """G_R^{3P}(k) gamma^(k; xi), Eq. (mod-kernel-3p) times the screening; zero at k = 0."""
    k2 = np.sum(k * k, axis=-1)
    safe = np.where(k2 > 0, k2, 1.0)
    A = np.where(k2 > 0, (-8 * np.pi / safe ** 2) if kernel not in _HARMONIC else (4 * np.pi / safe), 0.0)
    s = A * _screen(kernel, k2, xi)
    K = _Khat(kernel, k)
    return K * s.reshape(s.shape + (1,) * (K.ndim - s.ndim))


# ------------------------------------------------------------------ the five steps

def _components(kernel, f):
    """Source components spread on the grid: f_l (S, Omega) or f_lm = q_l nu_m (T)."""
    if kernel == STRESSLET:
        q, nu = f[:, :3], f[:, 3:]
        return (q[:, :, None] * nu[:, None, :]).reshape(-1, 9)
    return f


def gridding_3p(x, comps, L, M, win):
    """Step (i), Eq. (SE-gridding-disc) with the periodic wrap of all three directions."""
    h = win.h
    C = comps.shape[1]
    grid = np.zeros((C,) + tuple(M))
    P = win.P
    for n in range(x.shape[0]):
        idx, wts = [], []
        for d in range(3):
            j = taps(x[n, d] / h, P) + np.arange(P)
            wts.append(win(j * h - x[n, d]))
            idx.append(np.mod(j, M[d]))
        w3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        ix = np.ix_(idx[0], idx[1], idx[2])
        for c in range(C):
            grid[c][ix] += w3 * comps[n, c]
    return grid


def gathering_3p(t, Ft, L, M, win):
    """Step (v), Eq. (SE-gathering-disc)."""
    h = win.h
    P = win.P
    u = np.zeros((t.shape[0], Ft.shape[0]))
    for m in range(t.shape[0]):
        idx, wts = [], []
        for d in range(3):
            j = taps(t[m, d] / h, P) + np.arange(P)
            wts.append(win(t[m, d] - j * h))
            idx.append(np.mod(j, M[d]))
        w3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        ix = np.ix_(idx[0], idx[1], idx[2])
        for c in range(Ft.shape[0]):
            u[m, c] = h ** 3 * np.sum(Ft[c][ix] * w3)
    return u


def wavenumbers(M, L):
    """k_i = 2 pi kbar_i / L_i, kbar_i in [-M_i/2, M_i/2 - 1] (Eq. periodic-disc-wavenumbers),
    in FFT order, and the mask of modes off the Nyquist planes."""
    ks, nyq = [], []
    for d in range(3):
        kb = np.fft.fftfreq(M[d]) * M[d]
        ks.append(2 * np.pi * kb / L[d])
        nyq.append(kb == -M[d] // 2)
    K = np.stack(np.meshgrid(*ks, indexing="ij"), axis=-1)
    keep = ~(nyq[0][:, None, None] | nyq[1][None, :, None] | nyq[2][None, None, :])
    return K, keep


def scaling_3p(kernel, F, L, M, xi, win):
    """Step (iii), Eq. (SE-scaling-disc) with G_R^{3P} (Eq. mod-kernel-3p)."""
    K, keep = wavenumbers(M, L)
    what = win.hat(K[..., 0]) * win.hat(K[..., 1]) * win.hat(K[..., 2])
    G = kernel_3p(kernel, K, xi)
    G = G / (what ** 2).reshape(what.shape + (1,) * (G.ndim - 3))
    G = G * keep.reshape(keep.shape + (1,) * (G.ndim - 3))
    if kernel == STRESSLET:
        Fc = F.reshape((3, 3) + F.shape[1:])
        return np.einsum("xyzjlm,lmxyz->jxyz", G, Fc)
    return np.einsum("xyzjl,lxyz->jxyz", G, F)


def fourier_part_3p(kernel, x, f, L, M, xi, window, P, targets=None, return_steps=False):
    """u_h^{3P,F} at the targets (sources if None): steps (i)-(v) of Alg. 1 for D = 3."""
    kernel = kernel_id(kernel)
    L = np.asarray(L, dtype=float)
    M = tuple(int(m) for m in M)
    h = L[0] / M[0]
    assert all(abs(L[d] / M[d] - h) < 1e-12 * h for d in range(3)), "isotropic h"
    win = Window(window, P, h)
    x = np.asarray(x, dtype=float)
    t = x if targets is None else np.asarray(targets, dtype=float)
    comps = _components(kernel, np.asarray(f, dtype=float))
    grid = gridding_3p(x, comps, L, M, win)                     # (i)
    F = np.fft.fftn(grid, axes=(1, 2, 3))                       # (ii)
    Phit = scaling_3p(kernel, F, L, M, xi, win)                 # (iii)
    Ft = np.fft.ifftn(Phit, axes=(1, 2, 3))                     # (iv)
    assert np.abs(Ft.imag).max() <= 1e-9 * max(np.abs(Ft.real).max(), 1e-300)
    Ft = Ft.real
    u = gathering_3p(t, Ft, L, M, win)                          # (v)
    if return_steps:
        return u, dict(grid=grid, F=F, Phit=Phit, Ft=Ft)
    return u


def self_term(kernel, xi, f):
    """Eq. (self-term): -4 xi / sqrt(pi) f for the stokeslet, 0 for the rotlet, stresslet
    and harmonic field; -2 xi / sqrt(pi) q for the harmonic potential (the r -> 0 limit of
    its Fourier-space kernel erf(xi r) / r)."""
    kernel = kernel_id(kernel)
    f = np.asarray(f, dtype=float)
    if kernel == STOKESLET:
        return -4 * xi / math.sqrt(math.pi) * f
    if kernel == HARMONIC:
        return -2 * xi / math.sqrt(math.pi) * f.reshape(-1, 1)
    return np.zeros((f.shape[0], 3))


def k0_harmonic_3p(L, xi, q):
    """The constant -pi Q / (xi^2 V) (Q = sum q) that makes the 3P harmonic potential of
    real + Fourier (k != 0) + self parts the zero-mean one: minus the k -> 0 limit of the
    real-space kernel's transform, pi / xi^2, over the cell volume."""
    return -math.pi * float(np.sum(q)) / (xi * xi * float(np.prod(np.asarray(L, dtype=float))))


def k0_stresslet_3p(L, x, f, targets=None):
    """Eq. (k0-stresslet-3p)."""
    L = np.asarray(L, dtype=float)
    x = np.asarray(x, dtype=float)
    t = x if targets is None else np.asarray(targets, dtype=float)
    qn = np.sum(f[:, :3] * f[:, 3:], axis=1)
    vol = np.prod(L)
    return -8 * np.pi / vol * (t * qn.sum() - np.sum(x * qn[:, None], axis=0)[None, :])


# ============================================================ reduced periodicity (D < 3)
#
# Sec. 3.1 modified kernels, Sec. 3.2 extended grid, Sec. 3.4 adaptive FFT (D = 2, 1),
# Sec. 3.5 precomputation (D = 0). The grid has M_i = L_i / h points in the periodic
# directions and M'_i points in the free ones, origin o_i = -(M'_i h - L_i) / 2.

def _series_1mcos_tsin(t):
    """1 - cos t - t sin t, power series for small t (direct form cancels)."""
    out = np.zeros_like(t)
    term_c = np.ones_like(t)   # t^{2m} / (2m)!
    for m in range(1, 20):
        term_c = term_c * (-t * t) / ((2 * m - 1) * (2 * m))
        # -cos contributes -(-1)^m t^{2m}/(2m)! ; -t sin t contributes -(-1)^{m-1} t^{2m}/(2m-1)!
        out = out - term_c + term_c * (2 * m)
    return out


def hat_H2p(kap, R):
    """H^_R^{2P}(kappa) = 4 pi / kappa^2 (1 - cos R kappa - R kappa sin R kappa); -2 pi R^2 at 0."""
    kap = np.asarray(kap, dtype=float)
    t = R * np.abs(kap)
    small = t < 0.5
    safe = np.where(small, 1.0, kap)
    direct = 4 * np.pi / safe ** 2 * (1 - np.cos(t) - t * np.sin(t))
    ser = 4 * np.pi * R * R * _series_1mcos_tsin(np.where(small, t, 0.0)) / np.where(small & (t > 0), t * t, 1.0)
    ser = np.where(t > 0, ser, -2 * np.pi * R * R)
    return np.where(small, ser, direct)


def hat_Z2p(kap, R):
    """Z^_R^{2P}(kappa) = -4 pi i / kappa (1 - cos R kappa) = -8 pi i sin^2(R kappa/2) / kappa; 0 at 0."""
    kap = np.asarray(kap, dtype=float)
    safe = np.where(kap != 0, kap, 1.0)
    return np.where(kap != 0, -8j * np.pi * np.sin(R * kap / 2) ** 2 / safe, 0.0)


def _j_series(t, which):
    """1 - J0(t) (which=0) or 1 - J0(t) - t J1(t)/2 (which=1) by their power series."""
    out = np.zeros_like(t)
    q = (t / 2) ** 2
    term = np.ones_like(t)           # (t/2)^{2m} / (m!)^2
    for m in range(1, 30):
        term = term * q / (m * m)
        sgn = -1.0 if m % 2 == 0 else 1.0   # (-1)^{m+1}
        out = out + (sgn * term if which == 0 else sgn * term * (1 - m))
    return out


def hat_H1p(kap, R):
    """H^_R^{1P}(kappa) = 4 pi / kappa^2 (1 - J0(R kappa)), Eq. (optimal-1p-harmonic); pi R^2 at 0."""
    kap = np.asarray(kap, dtype=float)
    t = R * kap
    small = t < 2.0
    safe = np.where(small, 1.0, kap)
    direct = 4 * np.pi / safe ** 2 * (1 - sp.j0(t))
    ts = np.where(small & (t > 0), t, 1.0)
    ser = 4 * np.pi * R * R * _j_series(ts, 0) / ts ** 2
    ser = np.where(t > 0, ser, np.pi * R * R)
    return np.where(small, ser, direct)


def hat_B1p(kap, R):
    """B^_R^{1P}(kappa) = -8 pi / kappa^4 (1 - J0(R kappa) - R kappa J1(R kappa)/2),
    Eq. (optimal-1p-biharmonic); -pi R^4 / 8 at 0."""
    kap = np.asarray(kap, dtype=float)
    t = R * kap
    small = t < 2.0
    safe = np.where(small, 1.0, kap)
    direct = -8 * np.pi / safe ** 4 * (1 - sp.j0(t) - t * sp.j1(t) / 2)
    ts = np.where(small & (t > 0), t, 1.0)
    ser = -8 * np.pi * R ** 4 * _j_series(ts, 1) / ts ** 4
    ser = np.where(t > 0, ser, -np.pi * R ** 4 / 8)
    return np.where(small, ser, direct)


def hat_H0p(kap, R):
    """H^_R^{0P}(kappa) = 4 pi / kappa^2 (1 - cos R kappa), Eq. (vico-harmonic-0p); 2 pi R^2 at 0."""
    kap = np.asarray(kap, dtype=float)
    safe = np.where(kap > 0, kap, 1.0)
    return np.where(kap > 0, 8 * np.pi * np.sin(R * kap / 2) ** 2 / safe ** 2, 2 * np.pi * R * R)


def hat_B0p(kap, R):
    """B^_R^{0P}(kappa) = -8 pi / kappa^4 (1 + cos(R kappa)/2 - 3 sin(R kappa)/(2 R kappa)),
    Eq. (optimal-biharmonic-0p); -pi R^4 / 15 at 0 (Eq. optimal-biharmonic-0p-limit)."""
    kap = np.asarray(kap, dtype=float)
    t = R * kap
    small = t < 1.0
    safe = np.where(small, 1.0, kap)
    ts = np.where(small, t, 1.0)
    direct = -8 * np.pi / safe ** 4 * (1 + np.cos(np.where(small, 1.0, t)) / 2
                                       - 3 * np.sin(np.where(small, 1.0, t)) / (2 * np.where(small, 1.0, t)))
    # series: sum_{m>=2} (-1)^m (m-1) t^{2m} / (2m+1)!, divided by t^4
    ser = np.zeros_like(ts)
    for m in range(2, 20):
        ser = ser + (-1) ** m * (m - 1) * ts ** (2 * m - 4) / math.factorial(2 * m + 1)
    ser = -8 * np.pi * R ** 4 * ser
    return np.where(small, ser, direct)


def mollifier(n2):
    """mu of Sec. 3.5 for a (2M')-point direction with the origin at 0-based index M'."""
    a = 2.0 / 7.0 * math.sqrt(math.log(100.0))
    f = lambda t: math.exp(-a * a * t * t) + math.exp(-a * a * (t - 7) ** 2)
    mu = np.ones(n2)
    mu[:4] = [f(3), f(2), f(1), f(0)]
    mu[-4:] = [f(0), f(1), f(2), f(3)]
    return mu


class FreeGrid:
    """Extended grid of Eq. (extended-box): geometry shared by the D < 3 steps."""

    def __init__(self, D, L, h, Mext):
        self.D, self.L, self.h = D, np.asarray(L, dtype=float), h
        self.m = [int(round(L[d] / h)) if d < D else int(Mext[d]) for d in range(3)]
        for d in range(D):
            assert abs(self.m[d] * h - L[d]) < 1e-9 * L[d]
        self.origin = np.array([0.0 if d < D else -(self.m[d] * h - L[d]) / 2 for d in range(3)])
        Lp = np.array([self.m[d] * h for d in range(3)])
        self.Lext = Lp
        # truncation radius, Eq. (truncation-radius)
        self.R = float(np.sqrt(np.sum(Lp[D:] ** 2))) if D < 3 else 0.0


def gridding(fg, x, comps, win):
    """Step (i) on the (extended) grid; periodic wrap only in the first D directions."""
    h, P = win.h, win.P
    C = comps.shape[1]
    grid = np.zeros((C,) + tuple(fg.m))
    for n in range(x.shape[0]):
        idx, wts = [], []
        for d in range(3):
            u = (x[n, d] - fg.origin[d]) / h
            j = taps(u, P) + np.arange(P)
            wts.append(win(j * h + fg.origin[d] - x[n, d]))
            if d < fg.D:
                idx.append(np.mod(j, fg.m[d]))
            else:
                assert j[0] >= 0 and j[-1] < fg.m[d], "window outside the extended grid"
                idx.append(j)
        w3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        ix = np.ix_(idx[0], idx[1], idx[2])
        for c in range(C):
            grid[c][ix] += w3 * comps[n, c]
    return grid


def gathering(fg, t, Ft, win):
    """Step (v) on the (extended) grid."""
    h, P = win.h, win.P
    u = np.zeros((t.shape[0], Ft.shape[0]))
    for m in range(t.shape[0]):
        idx, wts = [], []
        for d in range(3):
            uu = (t[m, d] - fg.origin[d]) / h
            j = taps(uu, P) + np.arange(P)
            wts.append(win(t[m, d] - j * h - fg.origin[d]))
            idx.append(np.mod(j, fg.m[d]) if d < fg.D else j)
        w3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        ix = np.ix_(idx[0], idx[1], idx[2])
        for c in range(Ft.shape[0]):
            u[m, c] = h ** 3 * np.sum(Ft[c][ix] * w3)
    return u


def _apply(kernel, G, F):
    """Contract the multiplier G (..., 3, 3[, 3]) with the transformed components F."""
    if kernel == STRESSLET:
        Fc = F.reshape((3, 3) + F.shape[1:])
        return np.einsum("...jlm,lm...->j...", G, Fc)
    return np.einsum("...jl,l...->j...", G, F)


def _regular(kernel, K, xi, win):
    """G^(k) gamma^(k) / w^(k)^2 with the unmodified kernel (k^P != 0 modes)."""
    what = win.hat(K[..., 0]) * win.hat(K[..., 1]) * win.hat(K[..., 2])
    G = kernel_3p(kernel, K, xi)
    return G / (what ** 2).reshape(what.shape + (1,) * (G.ndim - K.ndim + 1))


def _pad_len(s, m, fM):
    return int(fM * math.ceil(s * m / fM - 1e-9))


def _kvec(kb, n, h):
    return 2 * np.pi * kb / (n * h)


def modified_2p_column(kernel, kap, xi, R):
    """G_R^{2P}(0,0,kappa3) gamma^ (Eqs. mod-stokeslet-2p, mod-rotlet-2p, mod-stresslet-2p)."""
    k2 = kap ** 2
    if kernel == STOKESLET:
        D = np.diag([2.0, 2.0, 0.0])
        s = hat_H2p(kap, R) * _screen(kernel, k2, xi)
        return s[:, None, None] * D
    if kernel == ROTLET:
        D = np.array([[0, 1.0, 0], [-1.0, 0, 0], [0, 0, 0]])
        s = hat_Z2p(kap, R) * _screen(kernel, k2, xi)
        return s[:, None, None] * D
    if kernel == HARMONIC:
        # the truncated harmonic kernel itself (its free-direction kernel is -2 pi |r_3|)
        return (hat_H2p(kap, R) * _screen(kernel, k2, xi))[:, None, None] * np.ones((1, 1))
    if kernel == HARMONIC_FIELD:
        # only the direction-3 derivative survives at k^P = 0: the rotlet's scalar (the same
        # derivative of the modified harmonic kernel) on (0, 0, q)
        D = np.array([[0.0], [0.0], [1.0]])
        s = hat_Z2p(kap, R) * _screen(kernel, k2, xi)
        return s[:, None, None] * D
    D = np.zeros((3, 3, 3))
    D[0, 0, 2] = D[0, 2, 0] = -2
    D[1, 1, 2] = D[1, 2, 1] = -2
    D[2, 0, 0] = D[2, 1, 1] = D[2, 2, 2] = -2
    s = hat_Z2p(kap, R) * _screen(kernel, k2, xi)
    return s[:, None, None, None] * D


def modified_1p_plane(kernel, k2v, k3v, xi, R):
    """G_R^{1P}(0,kappa2,kappa3) gamma^ (Eqs. mod-rotlet-1p, mod-stokeslet-1p, mod-stresslet-1p)."""
    kap = np.sqrt(k2v ** 2 + k3v ** 2)
    H = hat_H1p(kap, R)
    B = hat_B1p(kap, R)
    scr = _screen(kernel, kap ** 2, xi)
    z = np.zeros_like(kap)
    if kernel in _HARMONIC:
        K = np.stack([np.zeros_like(k2v), k2v, k3v], axis=-1)
        return _Khat(kernel, K) * (H * scr)[..., None, None]
    if kernel == STOKESLET:
        G = np.zeros(kap.shape + (3, 3), dtype=complex)
        G[..., 0, 0] = 2 * H
        G[..., 1, 1] = -k3v ** 2 * B
        G[..., 1, 2] = G[..., 2, 1] = k2v * k3v * B
        G[..., 2, 2] = -k2v ** 2 * B
        return G * scr[..., None, None]
    kk = kap ** 2
    CH = np.zeros(kap.shape + (3, 3, 3))
    CH[..., 0, 0, 1] = CH[..., 0, 1, 0] = k2v
    CH[..., 0, 0, 2] = CH[..., 0, 2, 0] = k3v
    CH[..., 1, 0, 0] = k2v
    CH[..., 2, 0, 0] = k3v
    CB = np.zeros(kap.shape + (3, 3, 3))
    CB[..., 1, 1, 1] = k2v * (3 * kk - 2 * k2v ** 2)
    CB[..., 1, 1, 2] = CB[..., 1, 2, 1] = k3v * (kk - 2 * k2v ** 2)
    CB[..., 1, 2, 2] = k2v * (kk - 2 * k3v ** 2)
    CB[..., 2, 1, 1] = k3v * (kk - 2 * k2v ** 2)
    CB[..., 2, 1, 2] = CB[..., 2, 2, 1] = k2v * (kk - 2 * k3v ** 2)
    CB[..., 2, 2, 2] = k3v * (3 * kk - 2 * k3v ** 2)
    del z
    G = 2j * CH * H[..., None, None, None] - 1j * CB * B[..., None, None, None]
    return G * scr[..., None, None, None]


def scaling_aft(D, kernel, grid, fg, xi, win, s0, s_star, kbar_star, fM):
    """Steps (ii)-(iv) for D = 2, 1: the adaptive FFT of Sec. 3.4 with the modified kernels
    for k^P = 0, the upsampling s_* on K_* and none on K_infinity; returns F~ on the grid."""
    h = win.h
    M = fg.m
    per = tuple(range(1, D + 1))                  # periodic axes of the [C, x, y, z] array
    free = tuple(range(D + 1, 4))
    Fp = np.fft.fftn(grid, axes=per)              # FFT in the periodic directions
    no = n_out(kernel)
    out = np.zeros((max(Fp.shape[0], no),) + Fp.shape[1:], dtype=complex)  # no outputs
    kbs = [np.fft.fftfreq(M[d]) * M[d] for d in range(D)]
    for idx in np.ndindex(*[M[d] for d in range(D)]):
        kb = [kbs[d][idx[d]] for d in range(D)]
        if any(kb[d] == -M[d] // 2 for d in range(D)):
            continue                              # Nyquist planes set to zero
        if all(k == 0 for k in kb):
            s, cls = s0, 0
        elif all(abs(k) <= kbar_star for k in kb):
            s, cls = s_star, 1
        else:
            s, cls = 1.0, 2
        n = [M[d] if cls == 2 else _pad_len(s, M[d], fM) for d in range(D, 3)]
        col = Fp[(slice(None),) + idx]            # [C, free dims...]
        pad = np.zeros((col.shape[0],) + tuple(n), dtype=complex)
        pad[(slice(None),) + tuple(slice(0, M[d]) for d in range(D, 3))] = col
        Fk = np.fft.fftn(pad, axes=tuple(range(1, 1 + 3 - D)))
        kf = [_kvec(np.fft.fftfreq(n[i]) * n[i], n[i], h) for i in range(3 - D)]
        nyqf = [np.fft.fftfreq(n[i]) * n[i] == -n[i] // 2 for i in range(3 - D)]
        kper = [_kvec(kb[d], M[d], h) for d in range(D)]
        if D == 2:
            k3 = kf[0]
            if cls == 0:
                G = modified_2p_column(kernel, k3, xi, fg.R)
                what = win.hat(0.0) ** 2 * win.hat(k3)
                G = G / (what ** 2).reshape((-1,) + (1,) * (G.ndim - 1))
            else:
                K = np.stack([np.full_like(k3, kper[0]), np.full_like(k3, kper[1]), k3], axis=-1)
                G = _regular(kernel, K, xi, win)
            keep = ~nyqf[0]
            G = G * keep.reshape((-1,) + (1,) * (G.ndim - 1))
        else:
            K2, K3 = np.meshgrid(kf[0], kf[1], indexing="ij")
            if cls == 0:
                G = modified_1p_plane(kernel, K2, K3, xi, fg.R)
                what = win.hat(0.0) * win.hat(K2) * win.hat(K3)
                G = G / (what ** 2).reshape(what.shape + (1,) * (G.ndim - 2))
            else:
                K = np.stack([np.full_like(K2, kper[0]), K2, K3], axis=-1)
                G = _regular(kernel, K, xi, win)
            keep = ~(nyqf[0][:, None] | nyqf[1][None, :])
            G = G * keep.reshape(keep.shape + (1,) * (G.ndim - 2))
        Phit = _apply(kernel, G, Fk)
        back = np.fft.ifftn(Phit, axes=tuple(range(1, 1 + 3 - D)))
        out[(slice(None, no),) + idx] = back[(slice(None),) + tuple(slice(0, M[d]) for d in range(D, 3))]
    Ft = np.fft.ifftn(out[:no], axes=per)
    assert np.abs(Ft.imag).max() <= 1e-9 * max(np.abs(Ft.real).max(), 1e-300)
    return Ft.real


def precompute_0p(kernel, fg, s0, fM):
    """Sec. 3.5: A^_{R,tr} on the 2M' grid from A^_R on the s0-upsampled grid (mollified for
    the biharmonic). Returned in FFT order, real."""
    h = fg.h
    M = fg.m
    nup = [_pad_len(s0, M[d], fM) for d in range(3)]
    kv = [_kvec(np.fft.fftfreq(nup[d]) * nup[d], nup[d], h) for d in range(3)]
    K0, K1, K2 = np.meshgrid(*kv, indexing="ij")
    kap = np.sqrt(K0 ** 2 + K1 ** 2 + K2 ** 2)
    Ahat = hat_H0p(kap, fg.R) if kernel in _HARMONIC else hat_B0p(kap, fg.R)
    A = np.fft.ifftn(Ahat).real                              # (ii) A_R on the grid (times 1/h^3)
    # (iii) truncate to the 2M' offsets -M' .. M'-1 around the origin, in FFT order
    At = np.zeros((2 * M[0], 2 * M[1], 2 * M[2]))
    offs = [np.concatenate([np.arange(0, M[d]), np.arange(-M[d], 0)]) for d in range(3)]
    At[...] = A[np.ix_(np.mod(offs[0], nup[0]), np.mod(offs[1], nup[1]), np.mod(offs[2], nup[2]))]
    if kernel not in _HARMONIC:
        # mollifier in natural order (origin at index M'), mapped to FFT order
        for d in range(3):
            mu = mollifier(2 * M[d])
            mu_fft = mu[np.mod(offs[d] + M[d], 2 * M[d])]
            shape = [1, 1, 1]
            shape[d] = -1
            At = At * mu_fft.reshape(shape)
    return np.fft.fftn(At).real                              # (iv)


def scaling_0p(kernel, grid, fg, xi, win, Atr):
    """Steps (ii)-(iv) for D = 0 on the 2M' grid with the precomputed kernel."""
    h = win.h
    M = fg.m
    n = [2 * M[d] for d in range(3)]
    pad = np.zeros((grid.shape[0],) + tuple(n))
    pad[:, :M[0], :M[1], :M[2]] = grid
    F = np.fft.fftn(pad, axes=(1, 2, 3))
    kv = [_kvec(np.fft.fftfreq(n[d]) * n[d], n[d], h) for d in range(3)]
    nyq = [np.fft.fftfreq(n[d]) * n[d] == -n[d] // 2 for d in range(3)]
    K = np.stack(np.meshgrid(*kv, indexing="ij"), axis=-1)
    k2 = np.sum(K * K, axis=-1)
    what = win.hat(K[..., 0]) * win.hat(K[..., 1]) * win.hat(K[..., 2])
    s = Atr * _screen(kernel, k2, xi) / what ** 2
    keep = ~(nyq[0][:, None, None] | nyq[1][None, :, None] | nyq[2][None, None, :])
    Kop = _Khat(kernel, K)
    G = Kop * (s * keep).reshape(s.shape + (1,) * (Kop.ndim - 3))
    Phit = _apply(kernel, G, F)
    Ft = np.fft.ifftn(Phit, axes=(1, 2, 3))
    assert np.abs(Ft.imag).max() <= 1e-9 * max(np.abs(Ft.real).max(), 1e-300)
    return Ft.real[:, :M[0], :M[1], :M[2]]


def fourier_part(D, kernel, x, f, L, h, P, xi, window, Mext=(0, 0, 0), s0=None, s_star=1.0,
                 kbar_star=0, fM=4, targets=None):
    """u_h^{DP,F} (Alg. 1) for any D, plus the 0P / 1P stokeslet gauge constants of
    Eqs. (0p-stokeslet-extra-contribution) and (1p-stokeslet-extra-contribution), so that
    the output follows the conventions of the exact sums (0P: zero at infinity; 1P: l_B = 1,
    l_H = 1/e)."""
    kernel = kernel_id(kernel)
    L = np.asarray(L, dtype=float)
    if D == 3:
        M = tuple(int(round(L[d] / h)) for d in range(3))
        return fourier_part_3p(kernel, x, f, L, M, xi, window, P, targets)
    fg = FreeGrid(D, L, h, Mext)
    win = Window(window, P, h)
    x = np.asarray(x, dtype=float)
    t = x if targets is None else np.asarray(targets, dtype=float)
    comps = _components(kernel, np.asarray(f, dtype=float))
    grid = gridding(fg, x, comps, win)
    if s0 is None:
        s0 = math.ceil(10 * (1 + fg.R / min(fg.Lext[D:]))) / 10
    if D == 0:
        Ft = scaling_0p(kernel, grid, fg, xi, win, precompute_0p(kernel, fg, s0, fM))
    else:
        Ft = scaling_aft(D, kernel, grid, fg, xi, win, s0, s_star, kbar_star, fM)
    u = gathering(fg, t, Ft, win)
    if kernel == HARMONIC and D == 1:
        # the k_1 = 0 class used -2 log(rho / R) (l_H = R, Eq. optimal-1p-harmonic); the output
        # convention is l_H = 1: subtract 2 log(R) / L_1 sum q
        u = u - 2.0 * math.log(fg.R) / L[0] * float(np.sum(f))
    if kernel == STOKESLET:
        fs = np.asarray(f, dtype=float).sum(axis=0)
        if D == 0:     # subtract 4 b_B sum f with b_B = -1/(2R)
            u = u + 2.0 / fg.R * fs[None, :]
        elif D == 1:   # subtract Eq. (1p-stokeslet-extra-contribution) at l_H = R, l_B = R sqrt(e)
            lr = math.log(fg.R)
            u = u - np.array([4 * (lr + 1), 2 * lr + 1, 2 * lr + 1]) * fs[None, :] / L[0]
    return u
