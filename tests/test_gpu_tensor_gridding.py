"""FP32 gridding, Eq. (SE-gridding-disc), on the tensor cores (tcgen05, se_opts.flags =
FLAG_TC_GRIDDING) against the numpy gridding of Algorithm 1 (oracle/se_steps.py) and against
the FP32 CUDA-core gridding (the default), through the C ABI.

Bars: the TF32 hi/lo split keeps every product within ~2^-21 relative, and the FP32
accumulation of <= a few thousand terms per grid value adds ~1e-7 relative to the largest
grid values, so the grids must agree to 2e-6 of the largest |value| (FP32 itself is 6e-8).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import se_steps as S  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BAR = 2e-6


def grid_of(D, box, kernel, x, f, xi, M, P, window, flags, prec="fp32"):
    o = se.se_opts_default()
    o.flags = flags
    o.kernel_mask = se.KERNELS[kernel]
    plan = se.Plan(D, box, xi, 0.3, M, P, window, prec, opts=o)
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.asarray(f), dtype=plan.dtype, device="cuda")
    plan.evaluate(kernel, xt, ft, parts=se.PART_FOURIER)
    plan.sync()
    info = plan.info()
    nr = 1 if np.asarray(f).ndim == 2 else np.asarray(f).shape[0]
    C = (6 if kernel == "stresslet" else 3) * nr
    g = np.zeros((C,) + tuple(info.n), dtype=np.float32 if prec == "fp32" else np.float64)
    se.se_debug_grid(plan.handle, g)
    return g.astype(np.float64)


def oracle_grid(kernel, x, f, M, P, window):
    win = S.Window(window, P, 1.0 / M)
    fs = f if f.ndim == 3 else f[None]
    out = []
    for fr in fs:
        comps = S._components(S.kernel_id(kernel), fr)
        ref = S.gridding_3p(x, comps, np.ones(3), (M, M, M), win)
        if kernel == "stresslet":
            r = ref.reshape((3, 3) + ref.shape[1:])
            sym = 0.5 * (r + r.transpose(1, 0, 2, 3, 4))
            ref = np.stack([sym[0, 0], sym[1, 1], sym[2, 2], sym[0, 1], sym[0, 2], sym[1, 2]])
        out.append(ref)
    return np.concatenate(out)


def maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


FLAGS = [pytest.param(0, id="cuda_cores"), pytest.param(se.FLAG_TC_GRIDDING, id="tcgen05")]


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("P", [4, 12, 16])
@pytest.mark.parametrize("kernel", ["stokeslet", "rotlet", "stresslet"])
def test_fp32_gridding_matches_oracle(kernel, P, flags):
    """M = 36: ragged 16 x 8 x 8 (or 16 x 8 x 16) tiles, few tiles -> bins split over CTAs."""
    M = 36
    x = W.uniform_points(300, (1, 1, 1), seed=21)
    f = W.strengths(kernel, 300, seed=22)
    g = grid_of(3, (1, 1, 1), kernel, x, f, 9.0, (M, M, M), P, "pkb", flags)
    assert maxrel(g, oracle_grid(kernel, x, f, M, P, "pkb")) < BAR


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_fp32_gridding_many_tiles_no_split(kernel, flags):
    """M = 136: enough tiles that each is owned by one CTA (plain stores, no atomics)."""
    M, P = 136, 8
    x = W.uniform_points(400, (1, 1, 1), seed=23)
    f = W.strengths(kernel, 400, seed=24)
    g = grid_of(3, (1, 1, 1), kernel, x, f, 30.0, (M, M, M), P, "gaussian", flags)
    assert maxrel(g, oracle_grid(kernel, x, f, M, P, "gaussian")) < BAR


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("kernel,nr", [("stokeslet", 3), ("stresslet", 4), ("rotlet", 16)])
def test_fp32_gridding_multi_rhs_component_groups(kernel, nr, flags):
    """C = 9 (groups 6 + 3), 24 (4 x 6) and 48 components."""
    M, P = 36, 10
    x = W.uniform_points(200, (1, 1, 1), seed=25)
    f = W.strengths(kernel, 200, seed=26, n_rhs=nr)
    g = grid_of(3, (1, 1, 1), kernel, x, f, 9.0, (M, M, M), P, "pkb", flags)
    assert maxrel(g, oracle_grid(kernel, x, f, M, P, "pkb")) < BAR


def test_fp32_gridding_wide_window_uses_cuda_cores():
    """P = 20 > 16: the tensor-core request falls back to the CUDA-core gridding."""
    M, P = 40, 20
    x = W.uniform_points(150, (1, 1, 1), seed=27)
    f = W.strengths("stokeslet", 150, seed=28)
    g = grid_of(3, (1, 1, 1), "stokeslet", x, f, 6.0, (M, M, M), P, "gaussian", se.FLAG_TC_GRIDDING)
    assert maxrel(g, oracle_grid("stokeslet", x, f, M, P, "gaussian")) < BAR


@pytest.mark.parametrize("D", [3, 2, 1, 0])
@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_tensor_equals_cuda_core_gridding(D, kernel):
    """Both FP32 gridding paths on the same plan geometry, including the extended grids of
    the free directions (zero-padded for D = 0)."""
    box = (1.0, 1.0, 1.0)
    x = W.uniform_points(500, box, seed=30 + D)
    f = W.strengths(kernel, 500, seed=40 + D)
    args = (D, box, kernel, x, f, 8.0, (32, 32, 32), 12, "pkb")
    g_tc = grid_of(*args, se.FLAG_TC_GRIDDING)
    g_cc = grid_of(*args, 0)
    assert g_tc.shape == g_cc.shape
    assert maxrel(g_tc, g_cc) < BAR


def test_tensor_gridding_clustered_full_size():
    """N = 20000 clustered points (a dense Gaussian blob: ~1e4 points reach each central grid
    value, many 32-point stages per tile) on a 56^3 grid: both FP32 grids against the FP64
    grid (itself pinned to the oracle at 1e-12 by the FP64 gridding test). An FP32 sum of
    n ~ 1e4 terms is good to ~sqrt(n) 2^-24 ~ 6e-6 relative, so both grids must be within
    6e-6 of max (an accumulator rounding bias would grow like n 2^-24 ~ 6e-4 and fail this;
    the CUDA-core gridding folds 32-point chunks with compensated sums and is well inside)."""
    x = W.clustered_points(20000, seed=5)
    f = W.strengths("stresslet", 20000, seed=6)
    args = (3, (1.0, 1.0, 1.0), "stresslet", x, f, 19.7, (56, 56, 56), 12, "pkb")
    ref = grid_of(*args, 0, prec="fp64")
    e_tc = maxrel(grid_of(*args, se.FLAG_TC_GRIDDING), ref)
    e_cc = maxrel(grid_of(*args, 0), ref)
    assert e_cc < 6e-6, e_cc
    assert e_tc < 6e-6, (e_tc, e_cc)


def test_bounded_wait_timeout_is_reported_and_context_stays_usable():
    """The tensor-core gridding's bounded waits: with the testing flag SE_FLAG_TEST_TIMEOUT
    they give up at their first poll. The evaluation must then report SE_ERR_TIMEOUT at
    se_sync (no hang, no fault), and the same process must evaluate correctly afterwards."""
    N, M, P = 4000, 32, 8
    x = W.uniform_points(N, (1, 1, 1), seed=31)
    f = W.strengths("stokeslet", N, seed=32)
    o = se.se_opts_default()
    o.flags = se.FLAG_TC_GRIDDING | se.FLAG_TEST_TIMEOUT
    o.kernel_mask = se.STOKESLET
    plan = se.Plan(3, (1, 1, 1), 8.0, 0.3, (M, M, M), P, "pkb", "fp32", opts=o)
    xt = torch.tensor(x, device="cuda")
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    plan.evaluate("stokeslet", xt, ft, parts=se.PART_FOURIER)
    with pytest.raises(se.SeError) as e:
        plan.sync()
    assert e.value.code == -6
    del plan
    g_tc = grid_of(3, (1, 1, 1), "stokeslet", x, f, 8.0, (M, M, M), P, "pkb", se.FLAG_TC_GRIDDING)
    g_cu = grid_of(3, (1, 1, 1), "stokeslet", x, f, 8.0, (M, M, M), P, "pkb", 0)
    assert maxrel(g_tc, g_cu) < BAR
