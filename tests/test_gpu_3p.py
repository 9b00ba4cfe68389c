"""GPU parity of the triply periodic path (libse through its C ABI) against the oracles.

Stage checks compare each CUDA stage with Algorithm 1 run step by step in numpy
(oracle/se_steps.py) on the same seeded inputs and parameters; the whole-potential checks
compare with the exact Ewald sum (oracle/ewald_oracle.c) at the tolerance the parameters
were selected for. Bars: FP64 1e-10 and FP32 1e-5 RMS relative unless stated.
"""
import math

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


def run(D, box, kernel, x, f, xi, rc, M, P, window, prec, targets=None, parts=se.PART_ALL, grid=False):
    plan = se.Plan(D, box, xi, rc, M, P, window, prec)
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.asarray(f), dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(np.asarray(targets), dtype=torch.float64, device="cuda")
    u = plan.evaluate(kernel, xt, ft, tt, parts=parts)
    plan.sync()
    out = u.cpu().numpy().astype(np.float64)
    g = None
    if grid:
        info = plan.info()
        C = (6 if kernel == "stresslet" else 3) * (1 if np.asarray(f).ndim == 2 else np.asarray(f).shape[0])
        g = np.zeros((C,) + tuple(info.n), dtype=np.float32 if prec == "fp32" else np.float64)
        se.se_debug_grid(plan.handle, g)
    return out, g


def rel(a, b):
    return E.rms_rel(a, b)


@pytest.mark.parametrize("window", ["gaussian", "kb", "pkb"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_gridding_matches_oracle(kernel, window):
    """Step (i), Eq. (SE-gridding-disc): the spread grid equals the numpy gridding."""
    x = W.uniform_points(300, (1, 1, 1), seed=11)
    f = W.strengths(kernel, 300, seed=12)
    M, P = 36, 12                    # 36 is not a multiple of the 8-point tile: ragged tiles
    _, g = run(3, (1, 1, 1), kernel, x, f, 9.0, 0.3, (M, M, M), P, window, "fp64",
               parts=se.PART_FOURIER, grid=True)
    win = S.Window(window, P, 1.0 / M)
    comps = S._components(S.kernel_id(kernel), f)
    ref = S.gridding_3p(x, comps, np.ones(3), (M, M, M), win)
    if kernel == "stresslet":
        r = ref.reshape((3, 3) + ref.shape[1:])
        sym = 0.5 * (r + r.transpose(1, 0, 2, 3, 4))
        ref = np.stack([sym[0, 0], sym[1, 1], sym[2, 2], sym[0, 1], sym[0, 2], sym[1, 2]])
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-11), ("fp32", 1e-5)])
@pytest.mark.parametrize("window", ["gaussian", "pkb"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_fourier_part_matches_alg1(kernel, window, prec, bar):
    """Steps (i)-(v) of Alg. 1 against the numpy run of the same steps."""
    N = 500
    x = W.uniform_points(N, (1, 1, 1), seed=21)
    f = W.strengths(kernel, N, seed=22)
    M, P, xi = 40, 14, 10.0
    u, _ = run(3, (1, 1, 1), kernel, x, f, xi, 0.3, (M, M, M), P, window, prec, parts=se.PART_FOURIER)
    ref = S.fourier_part_3p(kernel, x, f, [1, 1, 1], (M, M, M), xi, window, P)
    assert rel(u, ref) < bar


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_real_space_and_self_match_oracle(kernel, prec, bar):
    """Eq. (real-space-potential-Dp) with the star rule and the self term (Eq. self-term)."""
    N = 800
    x = W.uniform_points(N, (1, 1, 1), seed=31)
    f = W.strengths(kernel, N, seed=32)
    xi, rc = 9.0, 0.37        # rc > L/3: two cells per direction, images handled explicitly
    u, _ = run(3, (1, 1, 1), kernel, x, f, xi, rc, (32, 32, 32), 8, "pkb", prec, parts=se.PART_REAL)
    p = E.parts(3, [1, 1, 1], kernel, x, f, xi=xi, rc=rc)
    assert rel(u, p["real"] + p["self"]) < bar


def test_stresslet_zero_mode_matches_oracle():
    """Eq. (k0-stresslet-3p)."""
    N = 400
    x = W.uniform_points(N, (1, 1, 1), seed=41)
    f = W.strengths("stresslet", N, seed=42)
    u, _ = run(3, (1, 1, 1), "stresslet", x, f, 8.0, 0.3, (24, 24, 24), 8, "pkb", "fp64", parts=se.PART_CORR)
    ref = np.zeros((N, 3))
    E.lib().orc_k0_stresslet3p(E._p(np.ones(3)), N, E._p(np.ascontiguousarray(x)),
                               E._p(np.ascontiguousarray(f)), N, None, E._p(ref))
    assert rel(u, ref) < 1e-13


def _tuned(D, box, kernel, N, tol, f):
    Q = W.source_quantity(kernel, f)
    t = se.se_autotune(D, box, se.KERNELS[kernel], Q, N, tol / 10.0)
    return t["xi"], t["rc"], t["M"], t["P"]


def test_config1_stokeslet_fp64_full_potential():
    """3P stokeslet, plain FP64, N = 1000, sources = targets: 1e-10 RMS relative vs the
    exact Ewald sum, parameters from the selection procedure of Sec. 4.6."""
    N = 1000
    x = W.uniform_points(N, (1, 1, 1), seed=0)
    f = W.strengths("stokeslet", N, seed=0)
    xi, rc, M, P = _tuned(3, (1, 1, 1), "stokeslet", N, 1e-10, f)
    for window in ("gaussian", "pkb"):
        Pw = P if window == "pkb" else min(32, 2 * math.ceil(P / (2 * 0.6)))
        u, _ = run(3, (1, 1, 1), "stokeslet", x, f, xi, rc, M, Pw, window, "fp64")
        ref = E.potential(3, [1, 1, 1], "stokeslet", x, f)
        assert rel(u, ref) < 1e-10, window


@pytest.mark.parametrize("kernel", ["stresslet", "rotlet"])
def test_config2_fp32_full_size_sampled(kernel):
    """3P stresslet / rotlet, N = 20000, FP32 at 1e-6: whole potential at 256 sampled
    targets against the exact Ewald sum (bar 1e-5)."""
    N = 20000
    x = W.uniform_points(N, (1, 1, 1), seed=1)
    f = W.strengths(kernel, N, seed=1)
    xi, rc, M, P = _tuned(3, (1, 1, 1), kernel, N, 1e-6, f)
    u, _ = run(3, (1, 1, 1), kernel, x, f, xi, rc, M, P, "pkb", "fp32")
    idx = np.random.default_rng(5).choice(N, 256, replace=False)
    ref = E.potential(3, [1, 1, 1], kernel, x, f, targets=x[idx])
    assert rel(u[idx], ref) < 1e-5


@pytest.mark.parametrize("kernel", KERNELS)
def test_config2_fp64_1e10(kernel):
    """3P stresslet / rotlet (and stokeslet) FP64 at 1e-10 on a reduced N (oracle time)."""
    N = 2000
    x = W.uniform_points(N, (1, 1, 1), seed=3)
    f = W.strengths(kernel, N, seed=3)
    xi, rc, M, P = _tuned(3, (1, 1, 1), kernel, N, 1e-10, f)
    u, _ = run(3, (1, 1, 1), kernel, x, f, xi, rc, M, P, "kb", "fp64")
    idx = np.arange(0, N, 7)
    ref = E.potential(3, [1, 1, 1], kernel, x, f, targets=x[idx])
    assert rel(u[idx], ref) < 1e-10


@pytest.mark.parametrize("kernel", KERNELS)
def test_explicit_targets_and_coincident(kernel):
    N = 400
    x = W.uniform_points(N, (1, 1, 1), seed=51)
    f = W.strengths(kernel, N, seed=52)
    t = np.vstack([W.uniform_points(50, (1, 1, 1), seed=53), x[:10]])   # 10 coincide with sources
    xi, rc, M, P = _tuned(3, (1, 1, 1), kernel, N, 1e-10, f)
    u, _ = run(3, (1, 1, 1), kernel, x, f, xi, rc, M, P, "pkb", "fp64", targets=t)
    ustar, _ = run(3, (1, 1, 1), kernel, x, f, xi, rc, M, P, "pkb", "fp64")
    ref = E.potential(3, [1, 1, 1], kernel, x, f, targets=t)
    assert rel(u, ref) < 1e-10
    assert np.abs(u[50:] - ustar[:10]).max() < 1e-10 * np.abs(ustar).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multi_rhs_equals_single(prec):
    N, R = 600, 5
    x = W.uniform_points(N, (1, 1, 1), seed=61)
    for kernel in KERNELS:
        f = W.strengths(kernel, N, seed=62, n_rhs=R)
        ub, _ = run(3, (1, 1, 1), kernel, x, f, 8.0, 0.35, (32, 32, 32), 10, "pkb", prec)
        for r in range(R):
            us, _ = run(3, (1, 1, 1), kernel, x, f[r], 8.0, 0.35, (32, 32, 32), 10, "pkb", prec)
            bar = 1e-12 if prec == "fp64" else 1e-6
            assert rel(ub[r], us) < bar


def test_edge_cases_small_and_wrapped():
    # one point, points on the boundary and on grid nodes, coordinates outside [0, L)
    box = (1.0, 1.0, 1.0)
    x = np.array([[0.0, 0.0, 0.0], [0.5, 0.25, 0.75], [1.0 - 1e-12, 0.5, 0.1], [0.3, 0.3, 0.3]])
    f = W.strengths("stokeslet", 4, seed=71)
    xi, rc, M, P = _tuned(3, box, "stokeslet", 4, 1e-10, f)
    u1, _ = run(3, box, "stokeslet", x, f, xi, rc, M, P, "pkb", "fp64")
    xs = x + np.array([[1.0, -2.0, 3.0]])          # same points, shifted by lattice vectors
    u2, _ = run(3, box, "stokeslet", xs, f, xi, rc, M, P, "pkb", "fp64")
    ref = E.potential(3, list(box), "stokeslet", x, f)
    assert rel(u1, ref) < 1e-10
    assert np.abs(u1 - u2).max() < 1e-9 * np.abs(u1).max()
    uone, _ = run(3, box, "rotlet", x[:1], W.strengths("rotlet", 1, seed=2), 6.0, 0.45, (24, 24, 24), 10,
                  "pkb", "fp64")
    assert np.all(np.isfinite(uone))
