"""The harmonic potential phi = sum q / |x - y| (SE_HARMONIC: the electrostatic potential of
point charges, kernel H = 1/r) through the C ABI, for D = 3, 2, 1, 0.

One spread component and one output per RHS; Ewald screening, the harmonic modified kernels
(the 2P column, the 1P plane, the 0P precomputed truncated kernel) and the rotlet's parameter
rules. The strengths are N(0,1) charges, so the systems are charged: the 3P zero-mean
constant and the 1P gauge shift are exercised. Checked against
  * the exact Ewald sums of the oracle (pinned by Madelung constants, xi-independence, the
    field and the far-field gauges), FP64 at 1e-10 and FP32 at 1e-5;
  * the oracle's Alg. 1 steps element by element (Fourier part and constants, fixed xi, M, P);
  * the Madelung constants of tests/golden/madelung.txt, computed on the GPU;
  * several RHS with explicit targets, one on a source (the self term -2 xi/sqrt(pi) q).
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

H = "harmonic"


def rel(u, ref):
    u = np.asarray(u, dtype=float).reshape(-1)
    ref = np.asarray(ref, dtype=float).reshape(-1)
    return float(np.sqrt(np.mean((u - ref) ** 2) / np.mean(ref ** 2)))


def plan_for(D, box, N, tol, q, prec, flags=0):
    Q = W.source_quantity(H, q[0] if q.ndim == 3 else q)
    t = se.se_autotune(D, box, se.HARMONIC, Q, N, tol)
    o = t["opts"]
    o.kernel_mask = se.HARMONIC
    o.Q = Q
    o.flags = flags
    return se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def ev(plan, x, f, targets=None, parts=se.PART_ALL):
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.ascontiguousarray(f), dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(np.asarray(targets), dtype=torch.float64, device="cuda")
    u = plan.evaluate(H, xt, ft, tt, parts=parts)
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-12, 1e-10), ("fp32", 1e-7, 1e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_potential_matches_oracle(D, prec, tol, bar):
    box = (1.0, 1.0, 1.0)
    N = 300
    x = W.uniform_points(N, box, seed=3100 + D)
    q = W.strengths(H, N, seed=3200 + D)
    u = ev(plan_for(D, box, N, tol, q, prec), x, q)
    assert u.shape == (N, 1)
    err = rel(u, E.harmonic(D, box, x, q[:, 0]))
    assert 0 < err < bar, err


@pytest.mark.parametrize("box", [(1.0, 1.0, 1.0), (1.0, 1.25, 0.75)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_fourier_part_matches_alg1(D, box):
    """Fixed xi, M, P: the Fourier part plus the constants (3P zero-mean constant, 1P gauge
    shift) against the numpy steps of Alg. 1, FP64 to rounding."""
    N = 150
    x = W.uniform_points(N, box, seed=3300 + D)
    q = W.strengths(H, N, seed=3400 + D)
    xi, P = 7.0, 10
    h = 1.0 / 24
    M = tuple(int(round(b / h)) for b in box)
    o = se.se_opts_default()
    o.kernel_mask = se.HARMONIC
    o.tol_abs = 1e-9
    plan = se.Plan(D, box, xi, 0.3, M, P, "pkb", "fp64", opts=o)
    u = ev(plan, x, q, parts=se.PART_FOURIER | se.PART_CORR)[:, 0]
    info = plan.info()
    if D == 3:
        ref = S.fourier_part_3p(H, x, q, np.array(box), M, xi, "pkb", P)[:, 0] + S.k0_harmonic_3p(box, xi, q)
    else:
        ref = S.fourier_part(D, H, x, q, np.array(box), h, P, xi, "pkb", Mext=list(info.m), s0=info.s0,
                             s_star=info.s_star, kbar_star=info.kbar_star, fM=4)[:, 0]
    assert rel(u, ref) < 1e-12


def _madelung():
    vals = {}
    for line in open(__file__.rsplit("/", 1)[0] + "/golden/madelung.txt"):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


@pytest.mark.parametrize("D", [3, 2, 1])
def test_madelung_constants_on_the_gpu(D):
    """Rock salt (3P), checkerboard (2P), alternating chain (1P), d = 1/2: every ion sees
    -+2 M. A unit cell of one to four copies of the crystal (each still a valid cell)."""
    M = _madelung()
    if D == 3:
        g = np.array([(i, j, k) for i in range(4) for j in range(4) for k in range(4)], dtype=float)
        x, name, box = 0.5 * g, "rock_salt_3d", (2.0, 2.0, 2.0)
    elif D == 2:
        g = np.array([(i, j, 0) for i in range(4) for j in range(4)], dtype=float)
        x, name, box = 0.5 * g + np.array([0, 0, 0.4]), "square_checkerboard_2d", (2.0, 2.0, 1.0)
    else:
        g = np.array([(i, 0, 0) for i in range(4)], dtype=float)
        x, name, box = 0.5 * g + np.array([0, 0.3, 0.6]), "alternating_chain_1d", (2.0, 1.0, 1.0)
    q = np.where(g.sum(axis=1) % 2 == 0, 1.0, -1.0)[:, None]
    u = ev(plan_for(D, box, len(x), 1e-13, q, "fp64"), x, q)[:, 0]
    assert np.abs(u * 0.5 + q[:, 0] * M[name]).max() < 1e-9


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_potential_multi_rhs_explicit_targets(D):
    """4 RHS at explicit targets, one of them on a source (its pair replaced by the self term,
    as in the star form)."""
    box = (1.0, 1.0, 1.0)
    N, R = 300, 4
    x = W.uniform_points(N, box, seed=3500 + D)
    q = W.strengths(H, N, seed=3600 + D, n_rhs=R)
    t = W.uniform_points(90, box, seed=3700 + D)
    t[5] = x[17]
    for prec, tol, bar in (("fp64", 1e-12, 1e-10), ("fp32", 1e-7, 1e-5)):
        u = ev(plan_for(D, box, N, tol, q, prec), x, q, targets=t)
        assert u.shape == (R, 90, 1)
        for r in range(R):
            assert rel(u[r], E.harmonic(D, box, x, q[r, :, 0], targets=t)) < bar, (prec, r)


@pytest.mark.parametrize("D", [3, 0])
def test_potential_block_real_space(D):
    """The dense-block real-space path gives the same potential (FP64, whole sum vs oracle)."""
    box = (1.0, 1.0, 1.0)
    N = 2000
    x = W.clustered_points(N, seed=3800 + D)
    q = W.strengths(H, N, seed=3900 + D)
    u = ev(plan_for(D, box, N, 1e-12, q, "fp64", flags=se.FLAG_REAL_BLOCKS), x, q)
    idx = np.arange(0, N, 7)
    assert rel(u[idx], E.harmonic(D, box, x, q[:, 0], targets=x[idx])) < 1e-10
