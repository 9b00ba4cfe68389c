"""SE_FLAG_SPLIT_POLY: the free-space truncated biharmonic with a fitted polynomial
c0 + c1 r^2 + c2 r^4 + c3 r^6 taken out before its transform, the polynomial's potential (as
the Hasimoto screening passes it on) added back from moment sums of the sources. Through the C
ABI:
  * FP64: the whole potential against the exact direct sums (1e-10) for the stokeslet, the
    stresslet and both fused, several RHS and explicit targets; and against the same plan
    without the flag (the two differ by the method's truncation error only);
  * FP32: the rounding of the Fourier part (FP32 against FP64, same parameters) shrinks on a
    fine grid, where the large low-wavenumber values of the truncated biharmonic amplify it;
  * rotlet and harmonic kernels are unaffected (same results to rounding; the order of the
    atomic additions of split gridding tiles may differ between runs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def rms_rel(u, ref):
    u = np.asarray(u, dtype=float).reshape(-1)
    ref = np.asarray(ref, dtype=float).reshape(-1)
    return float(np.sqrt(np.mean((u - ref) ** 2) / np.mean(ref ** 2)))


def plan(kernel, N, tol, f, prec, flags, xi=0.0, M=None):
    Q = W.source_quantity(kernel, f[0] if f.ndim == 3 else f)
    t = se.se_autotune(0, (1, 1, 1), se.KERNELS[kernel], Q, N, tol, xi=xi)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[kernel]
    o.Q = Q
    o.flags = flags
    return se.Plan(0, (1, 1, 1), t["xi"], t["rc"], M or t["M"], t["P"], "pkb", prec, opts=o)


def ev(p, kernel, x, f, targets=None, parts=se.PART_ALL):
    xt = torch.tensor(x, device="cuda")
    ft = torch.tensor(np.ascontiguousarray(f), dtype=p.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(targets, device="cuda")
    u = p.evaluate(kernel, xt, ft, tt, parts=parts)
    p.sync()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet", "stokeslet+stresslet"])
def test_fp64_against_direct_sum(kernel):
    N = 2000
    x = W.clustered_points(N, seed=5100)
    f = W.strengths(kernel, N, seed=5200)
    u = ev(plan(kernel, N, 1e-11, f, "fp64", se.FLAG_SPLIT_POLY), kernel, x, f)
    idx = np.arange(0, N, 5)
    if kernel == "stokeslet+stresslet":
        ref = (E.potential(0, [1, 1, 1], "stokeslet", x, f[:, :3], targets=x[idx])
               + E.potential(0, [1, 1, 1], "stresslet", x, f[:, 3:], targets=x[idx]))
    else:
        ref = E.potential(0, [1, 1, 1], kernel, x, f, targets=x[idx])
    assert E.rms_rel(u[idx], ref) < 1e-10


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_fp64_multi_rhs_explicit_targets_same_as_without(kernel):
    """3 RHS at explicit targets (one on a source): with and without the split, and against the
    direct sums."""
    N, R = 1500, 3
    x = W.uniform_points(N, (1, 1, 1), seed=5300)
    f = W.strengths(kernel, N, seed=5400, n_rhs=R)
    t = W.uniform_points(200, (1, 1, 1), seed=5500)
    t[3] = x[11]
    a = ev(plan(kernel, N, 1e-11, f, "fp64", se.FLAG_SPLIT_POLY), kernel, x, f, targets=t)
    b = ev(plan(kernel, N, 1e-11, f, "fp64", 0), kernel, x, f, targets=t)
    for r in range(R):
        ref = E.potential(0, [1, 1, 1], kernel, x, f[r], targets=t)
        assert E.rms_rel(a[r], ref) < 1e-10
        assert E.rms_rel(a[r], b[r]) < 1e-10


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_fp32_rounding_shrinks_on_a_fine_grid(kernel):
    """Fourier part, clustered points, M = 160, xi = 50: FP32 against FP64 of the same plan
    parameters, with and without the split."""
    N = 100000
    x = W.clustered_points(N, seed=5600)
    f = W.strengths(kernel, N, seed=5700)
    err = {}
    for flags in (0, se.FLAG_SPLIT_POLY):
        u = {}
        for prec in ("fp64", "fp32"):
            p = plan(kernel, N, 1e-8, f, prec, flags, xi=50.0, M=(160, 160, 160))
            u[prec] = ev(p, kernel, x, f, parts=se.PART_FOURIER)
            del p
        err[flags] = rms_rel(u["fp32"], u["fp64"])
    print(kernel, "fp32 Fourier-part rounding without / with the split: %.3g / %.3g" % (err[0], err[se.FLAG_SPLIT_POLY]))
    assert err[se.FLAG_SPLIT_POLY] < 0.5 * err[0]


@pytest.mark.parametrize("kernel", ["rotlet", "harmonic_field", "harmonic"])
def test_harmonic_kernels_unaffected(kernel):
    N = 1000
    x = W.uniform_points(N, (1, 1, 1), seed=5800)
    f = W.strengths(kernel, N, seed=5900)
    a = ev(plan(kernel, N, 1e-10, f, "fp64", se.FLAG_SPLIT_POLY), kernel, x, f)
    b = ev(plan(kernel, N, 1e-10, f, "fp64", 0), kernel, x, f)
    assert rms_rel(a, b) < 1e-14


def test_fft_timed_extents():
    """SE_FLAG_FFT_TIMED: the extended grid is at least the rule's, FFT-friendly, and the
    potential matches the direct sums as with the rule's grid."""
    kernel = "stokeslet+stresslet"
    N = 1500
    x = W.clustered_points(N, seed=6100)
    f = W.strengths(kernel, N, seed=6200)
    a_plan = plan(kernel, N, 1e-10, f, "fp64", se.FLAG_FFT_SIZES)
    b_plan = plan(kernel, N, 1e-10, f, "fp64", se.FLAG_FFT_SIZES | se.FLAG_FFT_TIMED)
    ma, mb = list(a_plan.info().m), list(b_plan.info().m)
    for d in range(3):
        assert ma[d] <= mb[d] <= ma[d] + ma[d] // 4 and mb[d] % 2 == 0
        v = 2 * mb[d]
        for q in (2, 3, 5, 7):
            while v % q == 0:
                v //= q
        assert v == 1
    idx = np.arange(0, N, 4)
    ref = (E.potential(0, [1, 1, 1], "stokeslet", x, f[:, :3], targets=x[idx])
           + E.potential(0, [1, 1, 1], "stresslet", x, f[:, 3:], targets=x[idx]))
    for p in (a_plan, b_plan):
        assert E.rms_rel(ev(p, kernel, x, f)[idx], ref) < 1e-9


def test_fft_timed_extents_non_cubic_box():
    """SE_FLAG_FFT_TIMED on a box (1, 0.75, 0.5): the directions are searched one at a time;
    every extent is at least the rule's and FFT-friendly, and the potential meets the direct
    sums."""
    kernel = "stokeslet"
    box = (1.0, 0.75, 0.5)
    N = 800
    rng = np.random.default_rng(6300)
    x = rng.random((N, 3)) * np.array(box)
    f = W.strengths(kernel, N, seed=6400)
    Q = W.source_quantity(kernel, f)
    plans = []
    for flags in (se.FLAG_FFT_SIZES, se.FLAG_FFT_SIZES | se.FLAG_FFT_TIMED):
        o = se.se_opts_default()
        o.flags = flags
        t = se.se_autotune(0, box, se.KERNELS[kernel], Q, N, 1e-10, opts=o)
        o = t["opts"]
        o.kernel_mask = se.KERNELS[kernel]
        o.Q = Q
        o.flags = flags
        plans.append(se.Plan(0, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", "fp64", opts=o))
    ma, mb = list(plans[0].info().m), list(plans[1].info().m)
    for d in range(3):
        assert ma[d] <= mb[d] <= ma[d] + ma[d] // 4 and mb[d] % 2 == 0
        v = 2 * mb[d]
        for q in (2, 3, 5, 7):
            while v % q == 0:
                v //= q
        assert v == 1
    idx = np.arange(0, N, 4)
    ref = E.potential(0, list(box), kernel, x, f, targets=x[idx])
    for p in plans:
        assert E.rms_rel(ev(p, kernel, x, f)[idx], ref) < 1e-9
