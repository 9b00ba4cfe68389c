"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds no arithmetic of the method: only random point clouds and strengths with the shapes
and distributions of the paper's random systems (Sec. 4.1: uniform points in the primary
cell; Sec. 5.2: clustered systems) and of the benchmark configurations.
"""
import numpy as np


def uniform_points(n, box, seed):
    """n points uniform in [0,L1) x [0,L2) x [0,L3)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * np.asarray(box, dtype=float)


def clustered_points(n, seed, sigma=0.05, centre=(0.5, 0.5, 0.5)):
    """Half uniform in the unit cube, half normal around the centre (resampled into the cube)."""
    rng = np.random.default_rng(seed)
    nu = n // 2
    out = np.empty((n, 3))
    out[:nu] = rng.random((nu, 3))
    k = nu
    while k < n:
        y = rng.normal(centre, sigma, size=(n - k, 3))
        ok = np.all((y >= 0) & (y < 1), axis=1)
        y = y[ok]
        out[k:k + y.shape[0]] = y
        k += y.shape[0]
    return out


def two_cube_points(n, seed):
    """The clustered system of the timing experiments (Sec. 5.2): n points uniform in the two
    subdomains [0,1/3)^3 and [2/3,1)^3 of the unit cube, half in each."""
    rng = np.random.default_rng(seed)
    out = rng.random((n, 3)) / 3.0
    out[n // 2:] += 2.0 / 3.0
    return out


def strengths(kernel, n, seed, n_rhs=None):
    """Stokeslet / rotlet: f ~ N(0,1)^3. Stresslet: (q, nu) with q ~ N(0,1)^3 and nu ~ N(0,1)^3
    normalised to unit length. Stokeslet + stresslet: (f, q, nu), f drawn first. Harmonic
    field and harmonic potential: charges q ~ N(0,1).
    Shape (n, c) or (n_rhs, n, c)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if n_rhs is None else (n_rhs, n)
    if kernel in ("stokeslet+stresslet", 5):
        f = rng.standard_normal(shape + (3,))
        q = rng.standard_normal(shape + (3,))
        nu = rng.standard_normal(shape + (3,))
        nu /= np.linalg.norm(nu, axis=-1, keepdims=True)
        return np.concatenate([f, q, nu], axis=-1)
    if kernel in ("harmonic_field", 8, "harmonic", 16):
        return rng.standard_normal(shape + (1,))
    if kernel in ("stresslet", 4):
        q = rng.standard_normal(shape + (3,))
        nu = rng.standard_normal(shape + (3,))
        nu /= np.linalg.norm(nu, axis=-1, keepdims=True)
        return np.concatenate([q, nu], axis=-1)
    return rng.standard_normal(shape + (3,))


def batch_sizes(n_cfg, lo, hi, seed):
    """Point counts of n_cfg independent systems, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), n_cfg))).astype(int)


def source_quantity(kernel, f):
    """Q of Eq. (vector-source-quantity) / (tensor-source-quantity) for one RHS; for the
    stokeslet + stresslet strengths (f, q, nu) the two quantities added."""
    f = np.asarray(f, dtype=float)
    if kernel in ("stokeslet+stresslet", 5):
        return source_quantity("stokeslet", f[..., :3]) + source_quantity("stresslet", f[..., 3:])
    if kernel in ("stresslet", 4):
        t = f[..., :3, None] * f[..., None, 3:]
        return float(np.sum(t * t))
    return float(np.sum(f * f))


# The benchmark configurations (names describe the workload and its sizes).
CONFIGS = {
    "3p_stokeslet_n1000": dict(D=3, box=(1.0, 1.0, 1.0), N=1000, kernels=("stokeslet",),
                               tol=1e-10, prec="fp64", window="gaussian", seed=0, n_rhs=1),
    # n_rc: average neighbours within r_c for the choice of xi (Sec. 5.2). Table 5's uniform-case
    # values balance the real-space and Fourier costs of a CPU code; 0.35 of them balance this
    # GPU path (measured with P_margin = 0: 0.5x -> 0.35x of Table 5 took the batched step
    # from 0.450 to 0.413 ms at 2.7e-7 / 2.2e-7 RMS error over 1024 targets).
    # P_margin: window points added to the estimate by the error-pollution rule (the paper: 4).
    # At this tolerance the window is not what limits the error: P = 8 instead of 12 leaves the
    # RMS relative error over 1024 targets at 3.1e-7 / 3.6e-7 (P = 12: 3.1e-7 / 3.5e-7) and
    # shortens the step by 20%.
    "3p_stresslet_rotlet_n20000": dict(D=3, box=(1.0, 1.0, 1.0), N=20000,
                                       kernels=("stresslet", "rotlet"), tol=1e-6, prec="fp32",
                                       window="pkb", seed=1, n_rhs=1,
                                       n_rc={"stresslet": 280.0, "rotlet": 140.0}, P_margin=0),
    # P_margin = 0 (P = 8 instead of 12) measured as for the 3P workload: RMS relative error
    # 3.5e-7 against 3.4e-7 with the paper's margin, 184 against 141 M targets/s
    "2p_stokeslet_n200000_rhs8": dict(D=2, box=(1.0, 1.0, 0.5), N=200000, kernels=("stokeslet",),
                                      tol=1e-6, prec="fp32", window="pkb", seed=2, n_rhs=8, P_margin=0),
    # free space, half the points uniform and half in a Gaussian cluster (sigma 0.05) at the
    # centre; stokeslet and stresslet strengths (f, q, nu) evaluated together. The uniform-case
    # neighbour count puts ~1.4e11 pairs inside r_c here, so the split is chosen by timing.
    # (grid extents rounded to FFT-friendly sizes; the timed selection also bounds the FP32
    # rounding of each candidate, which grows with xi for the free-space stresslet)
    "0p_stokeslet_stresslet_n1000000": dict(D=0, box=(1.0, 1.0, 1.0), N=1000000, points="clustered",
                                            kernels=("stokeslet+stresslet",), tol=1e-6, prec="fp32",
                                            window="pkb", seed=4, n_rhs=1, autotune="timed",
                                            fft_sizes=True),
    # the harmonic field (electrostatics: the field of N(0,1) point charges), triply periodic
    "3p_harmonic_field_n100000": dict(D=3, box=(1.0, 1.0, 1.0), N=100000, kernels=("harmonic_field",),
                                      tol=1e-6, prec="fp32", window="pkb", seed=6, n_rhs=1),
    # the harmonic (electrostatic) potential of the same charges: one output per target
    "3p_harmonic_n100000": dict(D=3, box=(1.0, 1.0, 1.0), N=100000, kernels=("harmonic",),
                                tol=1e-6, prec="fp32", window="pkb", seed=6, n_rhs=1),
    # 64 independent singly periodic systems, N log-uniform in [2e3, 5e4], 16 RHS each;
    # P_margin = 0 (P = 8): RMS relative error 5.6e-7 / 4.4e-7 on two systems (P = 12:
    # 5.0e-7 / 4.2e-7)
    "1p_stokeslet_64cfg_rhs16": dict(D=1, box=(4.0, 1.0, 1.0), n_cfg=64, N_range=(2000, 50000),
                                     kernels=("stokeslet",), tol=1e-6, prec="fp32", window="pkb", seed=5,
                                     n_rhs=16, P_margin=0),
}
