"""The CUDA-core gridding (k_grid), Eq. (SE-gridding-disc), on clustered points, through the C ABI.

The tile work is split into queued items when a tile has more than 8192 candidate points; a
tight cluster makes the tiles around it far larger than that, so these cases run the split
path (first item stored, the others added atomically) next to the plain one. The FP64 grid
must equal the numpy gridding of Algorithm 1 (oracle/se_steps.py) to rounding (1e-12 of the
largest value); the FP32 grid, which sums each 32-point chunk in FP32 and folds the chunks
with Kahan compensation, must stay within 1e-6 of the largest value of the FP64 grid even
where a grid value sums ~1e4 points.
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


def tight_cluster(n, seed, sigma=0.01, centre=(0.5, 0.5, 0.5)):
    rng = np.random.default_rng(seed)
    x = rng.normal(centre, sigma, size=(n, 3))
    return np.mod(x, 1.0)


def gpu_grid(x, f, kernel, M, P, prec):
    o = se.se_opts_default()
    o.kernel_mask = se.KERNELS[kernel]
    plan = se.Plan(3, (1, 1, 1), 8.0, 0.3, (M, M, M), P, "pkb", prec, opts=o)
    xt = torch.tensor(x, device="cuda")
    ft = torch.tensor(f, dtype=plan.dtype, device="cuda")
    plan.evaluate(kernel, xt, ft, parts=se.PART_FOURIER)
    plan.sync()
    nr = 1 if f.ndim == 2 else f.shape[0]
    C = (6 if kernel == "stresslet" else 3) * nr
    g = np.zeros((C, M, M, M), dtype=np.float32 if prec == "fp32" else np.float64)
    se.se_debug_grid(plan.handle, g)
    return g.astype(np.float64)


def oracle_grid(x, f, kernel, M, P):
    win = S.Window("pkb", P, 1.0 / M)
    fs = f if f.ndim == 3 else f[None]
    out = []
    for fr in fs:
        ref = S.gridding_3p(x, S._components(S.kernel_id(kernel), fr), np.ones(3), (M, M, M), win)
        if kernel == "stresslet":
            r = ref.reshape((3, 3) + ref.shape[1:])
            sym = 0.5 * (r + r.transpose(1, 0, 2, 3, 4))
            ref = np.stack([sym[0, 0], sym[1, 1], sym[2, 2], sym[0, 1], sym[0, 2], sym[1, 2]])
        out.append(ref)
    return np.concatenate(out)


@pytest.mark.parametrize("kernel,n_rhs", [("stokeslet", 1), ("stresslet", 1), ("stokeslet", 4)])
def test_split_tiles_match_oracle(kernel, n_rhs):
    """A cluster of 20,000 points (sigma = 1/3 cell) plus 2,000 uniform ones on a 34^3 grid
    (ragged tiles): the tiles at the cluster have ~2e4 candidates (split into 3 items)."""
    M, P = 34, 8
    x = np.concatenate([tight_cluster(20000, seed=3), W.uniform_points(2000, (1, 1, 1), seed=4)])
    f = W.strengths(kernel, x.shape[0], seed=5, n_rhs=None if n_rhs == 1 else n_rhs)
    g = gpu_grid(x, f, kernel, M, P, "fp64")
    ref = oracle_grid(x, f, kernel, M, P)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fp32_grid_keeps_fp32_accuracy_on_a_dense_cluster():
    """200,000 points in a cluster of sigma = one cell: the densest grid values sum ~1e4
    points; the FP32 grid against the FP64 grid of the same evaluation."""
    M, P = 64, 12
    x = tight_cluster(200000, seed=6, sigma=1.0 / 64)
    f = W.strengths("stokeslet", x.shape[0], seed=7)
    g64 = gpu_grid(x, f, "stokeslet", M, P, "fp64")
    g32 = gpu_grid(x, f, "stokeslet", M, P, "fp32")
    assert np.abs(g32 - g64).max() <= 1e-6 * np.abs(g64).max()


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("kernel,n_rhs", [("harmonic_field", 1), ("stokeslet", 1), ("stresslet", 1),
                                          ("stokeslet+stresslet", 1), ("stokeslet", 4)])
def test_tile_depths_give_the_same_grid(kernel, n_rhs, prec, bar):
    """se_opts.tile = 4 and 8 (4 x 4 x TZ tiles) against the default choice, for 1, 3, 6, 9 and
    12 components per launch (12: always TZ = 4), on clustered points with split tiles."""
    M, P = 34, 8
    x = np.concatenate([tight_cluster(20000, seed=8), W.uniform_points(4000, (1, 1, 1), seed=9)])
    f = W.strengths(kernel, x.shape[0], seed=10, n_rhs=None if n_rhs == 1 else n_rhs)
    grids = []
    for tile in (0, 4, 8):
        o = se.se_opts_default()
        o.kernel_mask = se.KERNELS[kernel]
        o.tile = tile
        plan = se.Plan(3, (1, 1, 1), 8.0, 0.3, (M, M, M), P, "pkb", prec, opts=o)
        plan.evaluate(kernel, torch.tensor(x, device="cuda"), torch.tensor(f, dtype=plan.dtype, device="cuda"),
                      parts=se.PART_FOURIER)
        plan.sync()
        C = (1 if kernel == "harmonic_field" else 3 if kernel == "stokeslet" else 6 if kernel == "stresslet" else 9)
        g = np.zeros((C * n_rhs, M, M, M), dtype=np.float32 if prec == "fp32" else np.float64)
        se.se_debug_grid(plan.handle, g)
        grids.append(g.astype(np.float64))
    scale = np.abs(grids[0]).max()
    assert np.abs(grids[1] - grids[0]).max() <= bar * scale
    assert np.abs(grids[2] - grids[0]).max() <= bar * scale
