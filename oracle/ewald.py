"""Exact Ewald sum of the Stokes potentials (TEST INFRASTRUCTURE ONLY).

ctypes binding of oracle/ewald_oracle.c plus the choice of the oracle's own splitting
parameter.  The total potential of Eqs. (Dp-ewald-decomp) / (Dp-ewald-decomp-self) does
not depend on xi (Sec. 2.4), so the oracle picks its own xi, cut-off rc = 7/xi
(erfc and exp tails below 1e-21) and wavenumber cut-off kmax = 13.6 xi
(exp(-kmax^2/4xi^2) < 1e-20), independently of whatever the library under test uses.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import this module.
"""
import ctypes
import math

import numpy as np

from . import build as _build

STOKESLET, ROTLET, STRESSLET = 1, 2, 4
_NAMES = {"stokeslet": STOKESLET, "rotlet": ROTLET, "stresslet": STRESSLET}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("orc_real",):
            fn = getattr(L, name)
            fn.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                           ctypes.c_long, dp, dp, ctypes.c_long, dp, dp]
            fn.restype = ctypes.c_int
        for name in ("orc_fourier3p", "orc_fourier2p", "orc_fourier1p"):
            fn = getattr(L, name)
            fn.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_long,
                           dp, dp, ctypes.c_long, dp, dp]
            fn.restype = ctypes.c_int
        L.orc_k0_stresslet3p.argtypes = [dp, ctypes.c_long, dp, dp, ctypes.c_long, dp, dp]
        L.orc_direct0p.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, ctypes.c_long, dp, dp]
        L.orc_self.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_long, dp, dp,
                               ctypes.c_long, dp, dp]
        L.orc_Knu.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_Knu.restype = ctypes.c_double
        L.orc_En.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_En.restype = ctypes.c_double
        L.orc_Q2p.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, dp, dp]
        L.orc_Q2p0.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        L.orc_Q1p.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, dp, dp]
        L.orc_Q1p0.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_GF.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
        L.orc_h_real.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                 dp, dp, ctypes.c_long, dp, dp]
        for name in ("orc_h_fourier3p", "orc_h_fourier2p", "orc_h_fourier1p"):
            getattr(L, name).argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_long, dp, dp,
                                         ctypes.c_long, dp, dp]
        L.orc_h_k0_3p.argtypes = [dp, ctypes.c_double, ctypes.c_long, dp, ctypes.c_long, dp]
        L.orc_h_direct0p.argtypes = [ctypes.c_long, dp, dp, ctypes.c_long, dp, dp]
        L.orc_h_self.argtypes = [ctypes.c_double, ctypes.c_long, dp, dp, ctypes.c_long, dp, dp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def kernel_id(kernel):
    return _NAMES[kernel] if isinstance(kernel, str) else int(kernel)


def _prep(L, x, f, targets, kernel):
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    nc = 6 if kernel == STRESSLET else 3
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, nc)
    assert f.shape[0] == x.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    nt = x.shape[0] if t is None else t.shape[0]
    return L, x, f, t, nt


def default_xi(D, L):
    """The oracle's own splitting parameter (any value gives the same total)."""
    L = np.asarray(L, dtype=float)
    if D == 3:
        return 7.0 / L.min()
    if D == 2:
        return 4.0 / min(L[0], L[1])
    if D == 1:
        return 1.5 / L[0]
    return None


def parts(D, L, kernel, x, f, targets=None, xi=None, rc=None, kmax=None):
    """Return the dict of parts {real, fourier, k0, self} (each (Nt,3)) of the Ewald sum.

    For D = 0 only 'direct' is returned (the direct sum, Eq. periodic-potential)."""
    kernel = kernel_id(kernel)
    L, x, f, t, nt = _prep(L, x, f, targets, kernel)
    N = x.shape[0]
    tp = None if t is None else _p(t)
    out = {}
    lb = lib()
    if D == 0:
        u = np.zeros((nt, 3))
        rc_ = lb.orc_direct0p(kernel, N, _p(x), _p(f), nt, tp, _p(u))
        assert rc_ == 0
        out["direct"] = u
        return out
    if xi is None:
        xi = default_xi(D, L)
    if rc is None:
        rc = 7.0 / xi
    if kmax is None:
        kmax = 13.6 * xi
    ur = np.zeros((nt, 3))
    assert lb.orc_real(D, _p(L), xi, rc, kernel, N, _p(x), _p(f), nt, tp, _p(ur)) == 0
    out["real"] = ur
    uf = np.zeros((nt, 3))
    fn = {3: lb.orc_fourier3p, 2: lb.orc_fourier2p, 1: lb.orc_fourier1p}[D]
    assert fn(_p(L), xi, kmax, kernel, N, _p(x), _p(f), nt, tp, _p(uf)) == 0
    out["fourier"] = uf
    uk = np.zeros((nt, 3))
    if D == 3 and kernel == STRESSLET:
        assert lb.orc_k0_stresslet3p(_p(L), N, _p(x), _p(f), nt, tp, _p(uk)) == 0
    out["k0"] = uk
    us = np.zeros((nt, 3))
    assert lb.orc_self(xi, kernel, N, _p(x), _p(f), nt, tp, _p(us)) == 0
    out["self"] = us
    out["xi"] = xi
    return out


def potential(D, L, kernel, x, f, targets=None, xi=None):
    """The D-periodic potential u^{DP} (star form when targets is None), FP64, (Nt,3); the
    harmonic potential ("harmonic", 16) as (Nt,1)."""
    if kernel in ("harmonic", 16):
        return harmonic(D, L, x, f, targets, xi)[:, None]
    if kernel in ("harmonic_field", 8):
        return harmonic_field(D, L, x, f, targets, xi)
    p = parts(D, L, kernel, x, f, targets, xi)
    if D == 0:
        return p["direct"]
    return p["real"] + p["fourier"] + p["k0"] + p["self"]


def harmonic_field(D, L, x, q, targets=None, xi=None):
    """The D-periodic field E_j = sum q (x - y)_j / |x - y|^3 of charges q ((N,) or (N,1)).

    With H = 1/r the rotlet is Omega_jl = -eps_jlm d_m H and the field is E_j = -d_j H q, so
    E_1 = (Omega (q e_3))_2, E_2 = (Omega (q e_1))_3, E_3 = (Omega (q e_2))_1: the field is
    three rotlet sums with torques along the axes. Periodisation is linear, so the identity
    holds for the D-periodic sums with the rotlet's conventions (3P zero mode dropped; no self
    term in the star form)."""
    q = np.asarray(q, dtype=float).reshape(-1)
    out = None
    for comp, axis, row in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        f = np.zeros((q.shape[0], 3))
        f[:, axis] = q
        u = potential(D, L, "rotlet", x, f, targets, xi)
        if out is None:
            out = np.zeros_like(u)
        out[:, comp] = u[:, row]
    return out


def harmonic_parts(D, L, x, q, targets=None, xi=None, rc=None, kmax=None):
    """Parts {real, fourier, k0, self} (each (Nt,)) of the Ewald sum of the harmonic
    potential phi(x) = sum q / |x - y| (charges q, (N,) or (N,1)); for D = 0 only 'direct'.
    Zero-mode conventions as in ewald_oracle.h: 3P zero mean over the cell, 2P the k^P = 0
    kernel -2 pi |r_3| (App. A), 1P the k_1 = 0 kernel -2 log(rho) (App. B, l_H = 1)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    assert q.shape[0] == x.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    N = x.shape[0]
    nt = N if t is None else t.shape[0]
    tp = None if t is None else _p(t)
    lb = lib()
    out = {}
    if D == 0:
        u = np.zeros(nt)
        assert lb.orc_h_direct0p(N, _p(x), _p(q), nt, tp, _p(u)) == 0
        out["direct"] = u
        return out
    if xi is None:
        xi = default_xi(D, L)
    if rc is None:
        rc = 7.0 / xi
    if kmax is None:
        kmax = 13.6 * xi
    ur = np.zeros(nt)
    assert lb.orc_h_real(D, _p(L), xi, rc, N, _p(x), _p(q), nt, tp, _p(ur)) == 0
    out["real"] = ur
    uf = np.zeros(nt)
    fn = {3: lb.orc_h_fourier3p, 2: lb.orc_h_fourier2p, 1: lb.orc_h_fourier1p}[D]
    assert fn(_p(L), xi, kmax, N, _p(x), _p(q), nt, tp, _p(uf)) == 0
    out["fourier"] = uf
    uk = np.zeros(nt)
    if D == 3:
        assert lb.orc_h_k0_3p(_p(L), xi, N, _p(q), nt, _p(uk)) == 0
    out["k0"] = uk
    us = np.zeros(nt)
    assert lb.orc_h_self(xi, N, _p(x), _p(q), nt, tp, _p(us)) == 0
    out["self"] = us
    out["xi"] = xi
    return out


def harmonic(D, L, x, q, targets=None, xi=None):
    """The D-periodic harmonic potential phi (star form when targets is None), FP64, (Nt,)."""
    p = harmonic_parts(D, L, x, q, targets, xi)
    if D == 0:
        return p["direct"]
    return p["real"] + p["fourier"] + p["k0"] + p["self"]


def Knu(nu, a, b):
    return lib().orc_Knu(int(nu), float(a), float(b))


def En(n, x):
    return lib().orc_En(int(n), float(x))


def _tensor(kernel, fn, *args, cplx=True):
    n = 27 if kernel == STRESSLET else 9
    re = np.zeros(n)
    im = np.zeros(n)
    if cplx:
        assert fn(kernel, *args, _p(re), _p(im)) == 0
        v = re + 1j * im
    else:
        assert fn(kernel, *args, _p(re)) == 0
        v = re
    return v.reshape((3, 3, 3) if kernel == STRESSLET else (3, 3))


def Q2p(kernel, xi, k1, k2, r3):
    return _tensor(kernel_id(kernel), lib().orc_Q2p, float(xi), float(k1), float(k2), float(r3))


def Q2p0(kernel, xi, r3):
    return _tensor(kernel_id(kernel), lib().orc_Q2p0, float(xi), float(r3), cplx=False)


def Q1p(kernel, xi, k1, r2, r3):
    return _tensor(kernel_id(kernel), lib().orc_Q1p, float(xi), float(k1), float(r2), float(r3))


def Q1p0(kernel, xi, r2, r3):
    return _tensor(kernel_id(kernel), lib().orc_Q1p0, float(xi), float(r2), float(r3), cplx=False)


def GF(kernel, xi, k):
    kernel = kernel_id(kernel)
    k = np.ascontiguousarray(k, dtype=np.float64)
    n = 27 if kernel == STRESSLET else 9
    re = np.zeros(n)
    im = np.zeros(n)
    assert lib().orc_GF(kernel, float(xi), _p(k), _p(re), _p(im)) == 0
    return (re + 1j * im).reshape((3, 3, 3) if kernel == STRESSLET else (3, 3))


def rms_rel(u, uref):
    """E_rms,rel of Eq. (rel-rms-error)."""
    u = np.asarray(u, dtype=float).reshape(-1, 3)
    uref = np.asarray(uref, dtype=float).reshape(-1, 3)
    return math.sqrt(np.mean(np.sum((u - uref) ** 2, axis=1)) / np.mean(np.sum(uref ** 2, axis=1)))
