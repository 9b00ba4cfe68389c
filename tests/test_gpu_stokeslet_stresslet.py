"""Stokeslet and stresslet in one evaluation (kernel mask STOKESLET|STRESSLET, strengths
(f, q, nu) per point), through the C ABI: one gridding of 3 + 6 components, both operator
symbols applied and summed in the scaling step, one inverse transform and gathering of 3
components, one real-space pass evaluating both kernels per pair, and the corrections of
both (self term, 3P stresslet zero mode, 0P/1P stokeslet gauge constants).

The result is the sum of the two flows (each Eq. Dp-ewald-decomp-self), so it is checked
against the sum of the oracle's two potentials at the tolerance the parameters were chosen
for, and against the sum of the two single-kernel evaluations of the same plan (equal up to
the rounding order)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ST = "stokeslet+stresslet"


def plan_for(D, box, N, tol, f, prec, window="pkb"):
    Q = W.source_quantity(ST, f[0] if f.ndim == 3 else f)
    t = se.se_autotune(D, box, se.KERNELS[ST], Q, N, tol)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[ST]
    o.Q = Q
    return se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], window, prec, opts=o)


def ev(plan, kernel, x, f, targets=None, parts=se.PART_ALL):
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.ascontiguousarray(f), dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(np.asarray(targets), dtype=torch.float64, device="cuda")
    u = plan.evaluate(kernel, xt, ft, tt, parts=parts)
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


def oracle_sum(D, box, x, f, targets=None):
    return (E.potential(D, box, "stokeslet", x, f[..., :3], targets=targets)
            + E.potential(D, box, "stresslet", x, f[..., 3:], targets=targets))


@pytest.mark.parametrize("parts", [se.PART_ALL, se.PART_REAL, se.PART_FOURIER, se.PART_CORR])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_fused_equals_sum_of_single_kernels_fp64(D, parts):
    """Every part of the fused evaluation equals the sum of the stokeslet and stresslet parts."""
    box = (1.0, 1.0, 1.0)
    N = 400
    x = W.uniform_points(N, box, seed=1100 + D)
    f = W.strengths(ST, N, seed=1200 + D)
    plan = plan_for(D, box, N, 1e-10, f, "fp64")
    u = ev(plan, ST, x, f, parts=parts)
    us = ev(plan, "stokeslet", x, f[:, :3], parts=parts) + ev(plan, "stresslet", x, f[:, 3:], parts=parts)
    assert np.abs(u - us).max() <= 1e-12 * np.abs(us).max()


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-11, 1e-10), ("fp32", 1e-6, 1e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_fused_matches_oracle(D, prec, tol, bar):
    """E_rms,rel of the summed flow vs the oracle at every target (N = 300)."""
    box = (1.0, 1.0, 1.0)
    N = 300
    x = W.uniform_points(N, box, seed=1300 + D)
    f = W.strengths(ST, N, seed=1400 + D)
    u = ev(plan_for(D, box, N, tol, f, prec), ST, x, f)
    err = E.rms_rel(u, oracle_sum(D, box, x, f))
    assert 0 < err < bar, err


@pytest.mark.parametrize("D", [3, 1])
def test_fused_multi_rhs_explicit_targets(D):
    """3 RHS (27 spread components, two gridding groups in FP32) at explicit targets, one of
    them on a source (skipped pair, self term): the 3P zero mode and the 1P gauge constants
    read f and (q, nu) at stride 9."""
    box = (1.0, 1.0, 1.0)
    N, R = 300, 3
    x = W.uniform_points(N, box, seed=1500 + D)
    f = W.strengths(ST, N, seed=1600 + D, n_rhs=R)
    t = W.uniform_points(120, box, seed=1700 + D)
    t[7] = x[11]
    for prec, tol, bar in (("fp64", 1e-11, 1e-10), ("fp32", 1e-6, 1e-5)):
        plan = plan_for(D, box, N, tol, f, prec)
        u = ev(plan, ST, x, f, targets=t)
        for r in range(R):
            ref = oracle_sum(D, box, x, f[r], targets=t)
            assert E.rms_rel(u[r], ref) < bar, (prec, r)


def test_fused_tensor_core_gridding():
    """The fused 9 components through the tcgen05 gridding (FP32)."""
    box = (1.0, 1.0, 1.0)
    N = 300
    x = W.uniform_points(N, box, seed=1801)
    f = W.strengths(ST, N, seed=1802)
    Q = W.source_quantity(ST, f)
    t = se.se_autotune(3, box, se.KERNELS[ST], Q, N, 1e-6)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[ST]
    o.flags = se.FLAG_TC_GRIDDING
    plan = se.Plan(3, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", "fp32", opts=o)
    assert E.rms_rel(ev(plan, ST, x, f), oracle_sum(3, box, x, f)) < 1e-5


def config4_plan(x, f, tol, prec, fac):
    """The 0P workload's plan: the tolerance rules of Sec. 4.6 with the neighbour count of the
    uniform-case rule scaled by fac^3 (r_c by fac), FFT-friendly grid sizes (the fastest
    transforms among them), the dense-block real-space path and, in FP32, the polynomial split
    of the free-space biharmonic, as the timed selection of the benchmark chooses them."""
    box = (1.0, 1.0, 1.0)
    N = x.shape[0]
    Q = W.source_quantity(ST, f)
    o = se.se_opts_default()
    o.flags = se.FLAG_FFT_SIZES
    t = se.se_autotune(0, box, se.KERNELS[ST], Q, N, tol, opts=o)
    o = se.se_opts_default()
    o.flags = se.FLAG_FFT_SIZES
    o.n_rc = 4.0 / 3.0 * math.pi * t["rc"] ** 3 * N * fac ** 3
    t = se.se_autotune(0, box, se.KERNELS[ST], Q, N, tol, opts=o)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[ST]
    o.Q = Q
    o.flags = (se.FLAG_FFT_SIZES | se.FLAG_REAL_BLOCKS | se.FLAG_FFT_TIMED
               | (se.FLAG_SPLIT_POLY if prec == "fp32" else 0))
    return se.Plan(0, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def test_config4_0p_fused_clustered_sampled():
    """0P stokeslet + stresslet, N = 1e6 (half uniform, half a Gaussian cluster of width
    0.05), FP32, one fused evaluation at the benchmark's parameters (tolerance 1e-7 requested,
    r_c at 0.8^4 of the uniform-case rule): 256 sampled targets vs the direct sums within the
    benchmark's bar of 1e-6."""
    box = (1.0, 1.0, 1.0)
    N = 1000000
    x = W.clustered_points(N, seed=4)
    f = W.strengths(ST, N, seed=4)
    u = ev(config4_plan(x, f, 1e-7, "fp32", 0.8 ** 4), ST, x, f)
    idx = np.random.default_rng(12).choice(N, 256, replace=False)
    assert E.rms_rel(u[idx], oracle_sum(0, box, x, f, targets=x[idx])) < 1e-6


def test_config4_0p_fused_clustered_fp64_sampled():
    """The same workload in FP64 at the FP64 bar: tolerance 1e-11 requested, r_c at 0.8^3 of
    the uniform-case rule (grids of ~100 GB for the 800^3 transform, 3e10 pairs), 128 sampled
    targets within 1e-10."""
    box = (1.0, 1.0, 1.0)
    N = 1000000
    x = W.clustered_points(N, seed=4)
    f = W.strengths(ST, N, seed=4)
    u = ev(config4_plan(x, f, 1e-11, "fp64", 0.8 ** 3), ST, x, f)
    idx = np.random.default_rng(13).choice(N, 128, replace=False)
    assert E.rms_rel(u[idx], oracle_sum(0, box, x, f, targets=x[idx])) < 1e-10
