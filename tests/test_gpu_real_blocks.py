"""The dense-block real-space path (se_opts.flags = FLAG_REAL_BLOCKS, kernel k_real_blk) against
the per-target path (k_real) and the oracle, through the C ABI.

The block path computes the same real-space sum, Eq. (real-space-potential-Dp) with the
kernels of Eqs. (stokeslet-real), (rotlet-real), (stresslet-real) and the self term of
Eq. (self-term), for targets grouped in blocks of 32: only the order of summation and the
coordinates the separations are formed from differ. Bars: FP64 1e-13 relative (rounding),
FP32 2e-6 (the per-target path forms exact hi + lo separations, the block path block-relative
ones; both sum in FP32); FP32 against FP64 on a cluster with ~1e4 neighbours per target
within 3e-7 (the block path folds 32-pair chunks with compensated sums).
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


def cluster(n, box, seed, sigma=0.03):
    """Half uniform in the box, half in a Gaussian cluster at its centre (resampled inside)."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=float)
    x = rng.random((n, 3)) * box
    k = n // 2
    while k < n:
        y = rng.normal(box / 2, sigma, size=(n - k, 3))
        y = y[np.all((y >= 0) & (y < box), axis=1)]
        x[k:k + len(y)] = y
        k += len(y)
    return x


def real_part(D, box, kernel, x, f, xi, rc, prec, flags, targets=None, M=(32, 32, 32)):
    o = se.se_opts_default()
    o.flags = flags
    plan = se.Plan(D, box, xi, rc, M, 8, "pkb", prec, opts=o)
    xt = torch.tensor(x, device="cuda")
    ft = torch.tensor(f, dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(targets, device="cuda")
    u = plan.evaluate(kernel, xt, ft, targets=tt, parts=se.PART_REAL)
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


def rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


CASES = [(3, (1.0, 1.0, 1.0), (32, 32, 32)), (2, (1.0, 1.0, 0.5), (32, 32, 16)),
         (1, (2.0, 1.0, 1.0), (64, 32, 32)), (0, (1.0, 1.0, 1.0), (32, 32, 32))]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("kernel", ["stokeslet", "rotlet", "stresslet", "stokeslet+stresslet", "harmonic_field",
                                    "harmonic"])
@pytest.mark.parametrize("prec,bar", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_blocks_equal_per_target_path(case, kernel, prec, bar):
    D, box, M = CASES[case]
    N = 6000
    x = cluster(N, box, seed=40 + case)
    f = W.strengths(kernel, N, seed=41)
    xi, rc = 12.0, 0.2
    a = real_part(D, box, kernel, x, f, xi, rc, prec, 0, M=M)
    b = real_part(D, box, kernel, x, f, xi, rc, prec, se.FLAG_REAL_BLOCKS, M=M)
    assert rel(b, a) < bar


@pytest.mark.parametrize("n_rhs", [1, 3, 6])
def test_blocks_multi_rhs_and_explicit_targets(n_rhs):
    """Several RHS (the block kernel takes up to 4, more go to the per-target path) and explicit
    targets, some of them coinciding with sources (the self term, as in the star form)."""
    box = (1.0, 1.0, 1.0)
    N, NT = 5000, 3000
    x = cluster(N, box, seed=50)
    tg = cluster(NT, box, seed=51)
    tg[:100] = x[:100]
    f = W.strengths("stokeslet", N, seed=52, n_rhs=n_rhs)
    a = real_part(3, box, "stokeslet", x, f, 12.0, 0.2, "fp64", 0, targets=tg)
    b = real_part(3, box, "stokeslet", x, f, 12.0, 0.2, "fp64", se.FLAG_REAL_BLOCKS, targets=tg)
    assert rel(b, a) < 1e-13


def test_blocks_fp32_accuracy_on_a_dense_cluster():
    """~1e4 neighbours per cluster target: the FP32 block sums against FP64."""
    box = (1.0, 1.0, 1.0)
    N = 200000
    x = cluster(N, box, seed=60, sigma=0.02)
    f = W.strengths("stokeslet+stresslet", N, seed=61)
    xi, rc = 60.0, 0.06
    u64 = real_part(0, box, "stokeslet+stresslet", x, f, xi, rc, "fp64", se.FLAG_REAL_BLOCKS)
    u32 = real_part(0, box, "stokeslet+stresslet", x, f, xi, rc, "fp32", se.FLAG_REAL_BLOCKS)
    assert rel(u32, u64) < 3e-7


@pytest.mark.parametrize("D", [3, 0])
def test_blocks_whole_potential_against_oracle(D):
    """The whole FP64 potential with the block path against the exact Ewald sums (1e-10)."""
    box = (1.0, 1.0, 1.0)
    N = 3000
    x = cluster(N, box, seed=70 + D)
    f = W.strengths("stresslet", N, seed=71)
    Q = W.source_quantity("stresslet", f)
    t = se.se_autotune(D, box, se.STRESSLET, Q, N, 1e-11)
    o = t["opts"]
    o.kernel_mask = se.STRESSLET
    o.flags = se.FLAG_REAL_BLOCKS
    plan = se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", "fp64", opts=o)
    u = plan.evaluate("stresslet", torch.tensor(x, device="cuda"), torch.tensor(f, device="cuda"))
    plan.sync()
    idx = np.random.default_rng(3).choice(N, 300, replace=False)
    ref = E.potential(D, list(box), "stresslet", x, f, targets=x[idx])
    assert E.rms_rel(u.cpu().numpy()[idx], ref) < 1e-10
