"""GPU parity of the reduced-periodicity paths (D = 2, 1: adaptive FFT with the modified
kernels; D = 0: precomputed truncated kernel) against the oracles, through the C ABI.

* Fourier part + gauge constants vs Alg. 1 in numpy (oracle/se_steps.py) with the plan's
  own extended grid, upsampling factors and kbar_* (read back with se_get_info).
* Whole potential vs the exact sums (App. A / App. B closed forms, direct sum) at the
  tolerance the parameters were selected for (Sec. 4.6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402
from oracle import se_steps as S  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

KERNELS = ["stokeslet", "rotlet", "stresslet"]


def tuned(D, box, kernel, N, tol, f):
    Q = W.source_quantity(kernel, f[0] if f.ndim == 3 else f)
    t = se.se_autotune(D, box, se.KERNELS[kernel], Q, N, tol / 10.0)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[kernel]
    o.Q = Q
    return t["xi"], t["rc"], t["M"], t["P"], o


def run(D, box, kernel, x, f, xi, rc, M, P, window, prec, opts=None, targets=None, parts=se.PART_ALL):
    plan = se.Plan(D, box, xi, rc, M, P, window, prec, opts=opts)
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.asarray(f), dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(np.asarray(targets), dtype=torch.float64, device="cuda")
    u = plan.evaluate(kernel, xt, ft, tt, parts=parts)
    plan.sync()
    return u.cpu().numpy().astype(np.float64), plan.info()


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-11), ("fp32", 2e-5)])
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("D", [2, 1, 0])
def test_fourier_part_matches_alg1(D, kernel, prec, bar):
    box = (1.0, 1.0, 1.0)
    N = 150
    x = W.uniform_points(N, box, seed=100 + D)
    f = W.strengths(kernel, N, seed=200 + D)
    xi, P, M = 7.0, 10, (24, 24, 24)
    o = se.se_opts_default()
    o.kernel_mask = se.KERNELS[kernel]
    o.tol_abs = 1e-9
    u, info = run(D, box, kernel, x, f, xi, 0.3, M, P, "pkb", prec, opts=o,
                  parts=se.PART_FOURIER | se.PART_CORR)
    Mext = list(info.m)
    ref = S.fourier_part(D, kernel, x, f, np.array(box), 1.0 / M[0], P, xi, "pkb", Mext=Mext, s0=info.s0,
                         s_star=info.s_star, kbar_star=info.kbar_star, fM=4)
    assert E.rms_rel(u, ref) < bar


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("D", [2, 1, 0])
def test_full_potential_fp64_1e10(D, kernel):
    box = (1.0, 1.0, 1.0)
    N = 300
    x = W.uniform_points(N, box, seed=300 + D)
    f = W.strengths(kernel, N, seed=400 + D)
    xi, rc, M, P, o = tuned(D, box, kernel, N, 1e-10, f)
    u, _ = run(D, box, kernel, x, f, xi, rc, M, P, "pkb", "fp64", opts=o)
    idx = np.arange(0, N, 3)
    ref = E.potential(D, box, kernel, x, f, targets=x[idx])
    assert E.rms_rel(u[idx], ref) < 1e-10


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("D", [2, 1])
def test_noncubic_boxes(D, kernel):
    box = (1.0, 1.0, 0.5) if D == 2 else (2.0, 1.0, 1.0)
    N = 200
    x = W.uniform_points(N, box, seed=500 + D)
    f = W.strengths(kernel, N, seed=600 + D)
    xi, rc, M, P, o = tuned(D, box, kernel, N, 1e-8, f)
    u, _ = run(D, box, kernel, x, f, xi, rc, M, P, "pkb", "fp64", opts=o)
    idx = np.arange(0, N, 4)
    ref = E.potential(D, box, kernel, x, f, targets=x[idx])
    assert E.rms_rel(u[idx], ref) < 1e-8


def test_config3_2p_stokeslet_fp32_8rhs_sampled():
    """2P stokeslet, N = 200,000 in (1,1,0.5), 8 RHS in one batched spread, FP32 at 1e-6:
    every RHS at 16 sampled targets vs the App. A sums (bar 1e-5)."""
    box = (1.0, 1.0, 0.5)
    N, R = 200000, 8
    x = W.uniform_points(N, box, seed=2)
    f = W.strengths("stokeslet", N, seed=2, n_rhs=R)
    xi, rc, M, P, o = tuned(2, box, "stokeslet", N, 1e-6, f)
    u, _ = run(2, box, "stokeslet", x, f, xi, rc, M, P, "pkb", "fp32", opts=o)
    idx = np.random.default_rng(9).choice(N, 16, replace=False)
    for r in (0, 5):
        ref = E.potential(2, box, "stokeslet", x, f[r], targets=x[idx])
        assert E.rms_rel(u[r][idx], ref) < 1e-5


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_config4_0p_clustered_sampled(kernel):
    """0P, N = 1e6 (half uniform, half a Gaussian cluster of width 0.05), FP32 at 1e-6:
    64 sampled targets vs the direct sum (bar 1e-5)."""
    box = (1.0, 1.0, 1.0)
    N = 1000000
    x = W.clustered_points(N, seed=4)
    f = W.strengths(kernel, N, seed=4)
    xi, rc, M, P, o = tuned(0, box, kernel, N, 1e-6, f)
    u, _ = run(0, box, kernel, x, f, xi, rc, M, P, "pkb", "fp32", opts=o)
    idx = np.random.default_rng(11).choice(N, 64, replace=False)
    ref = E.potential(0, box, kernel, x, f, targets=x[idx])
    assert E.rms_rel(u[idx], ref) < 1e-5


def test_free_direction_range_error():
    """A free coordinate outside [0, L) is reported as SE_ERR_RANGE (no out-of-range access)."""
    box = (1.0, 1.0, 1.0)
    x = W.uniform_points(50, box, seed=7)
    x[3, 2] = 1.5
    f = W.strengths("stokeslet", 50, seed=8)
    plan = se.Plan(2, box, 6.0, 0.4, (24, 24, 24), 8, "pkb", "fp64")
    plan.evaluate("stokeslet", torch.tensor(x, device="cuda"), torch.tensor(f, device="cuda"))
    with pytest.raises(se.SeError) as e:
        plan.sync()
    assert e.value.code == -2
