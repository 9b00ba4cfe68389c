"""The harmonic field E_j = sum q (x - y)_j / |x - y|^3 (SE_HARMONIC_FIELD: the field of
point charges, -grad of the harmonic kernel H = 1/r) through the C ABI, for D = 3, 2, 1, 0.

It runs the Spectral Ewald chain of Alg. 1 with one spread component per RHS and the rotlet's
screening, modified-kernel tables and parameter rules (both kernels are first derivatives of
H); the operator is the gradient instead of the curl. Checked (1) against the oracle (three
rotlet sums with torques along the axes, pinned against the direct sum), and (2) on one plan
against one rotlet evaluation with torques q e_3, q e_1, q e_2 (E_1 = (Omega q e_3)_2,
E_2 = (Omega q e_1)_3, E_3 = (Omega q e_2)_1), part by part, to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FIELD = "harmonic_field"


def plan_for(D, box, N, tol, q, prec, mask=se.HARMONIC_FIELD):
    Q = W.source_quantity(FIELD, q[0] if q.ndim == 3 else q)
    t = se.se_autotune(D, box, se.HARMONIC_FIELD, Q, N, tol)
    o = t["opts"]
    o.kernel_mask = mask
    o.Q = Q
    return se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def ev(plan, kernel, x, f, targets=None, parts=se.PART_ALL):
    xt = torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    ft = torch.tensor(np.ascontiguousarray(f), dtype=plan.dtype, device="cuda")
    tt = None if targets is None else torch.tensor(np.asarray(targets), dtype=torch.float64, device="cuda")
    u = plan.evaluate(kernel, xt, ft, tt, parts=parts)
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-12, 1e-10), ("fp32", 1e-7, 1e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_field_matches_oracle(D, prec, tol, bar):
    box = (1.0, 1.0, 1.0)
    N = 300
    x = W.uniform_points(N, box, seed=2100 + D)
    q = W.strengths(FIELD, N, seed=2200 + D)
    u = ev(plan_for(D, box, N, tol, q, prec), FIELD, x, q)
    err = E.rms_rel(u, E.potential(D, box, FIELD, x, q))
    assert 0 < err < bar, err


@pytest.mark.parametrize("parts", [se.PART_ALL, se.PART_REAL, se.PART_FOURIER])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_field_equals_rotlet_with_axis_torques(D, parts):
    box = (1.0, 1.0, 1.0)
    N = 400
    x = W.uniform_points(N, box, seed=2300 + D)
    q = W.strengths(FIELD, N, seed=2400 + D)
    plan = plan_for(D, box, N, 1e-10, q, "fp64", mask=se.HARMONIC_FIELD | se.ROTLET)
    e = ev(plan, FIELD, x, q, parts=parts)
    f = np.zeros((3, N, 3))
    f[0, :, 2] = q[:, 0]
    f[1, :, 0] = q[:, 0]
    f[2, :, 1] = q[:, 0]
    u = ev(plan, "rotlet", x, f, parts=parts)
    comb = np.stack([u[0][:, 1], u[1][:, 2], u[2][:, 0]], axis=1)
    assert np.abs(e - comb).max() <= 1e-12 * np.abs(comb).max()


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_field_multi_rhs_explicit_targets(D):
    """4 RHS at explicit targets, one of them on a source (its pair skipped; no self term).
    One input component per RHS: the in-place scaling runs the RHS in reverse order."""
    box = (1.0, 1.0, 1.0)
    N, R = 300, 4
    x = W.uniform_points(N, box, seed=2500 + D)
    q = W.strengths(FIELD, N, seed=2600 + D, n_rhs=R)
    t = W.uniform_points(90, box, seed=2700 + D)
    t[5] = x[17]
    for prec, tol, bar in (("fp64", 1e-12, 1e-10), ("fp32", 1e-7, 1e-5)):
        u = ev(plan_for(D, box, N, tol, q, prec), FIELD, x, q, targets=t)
        for r in range(R):
            assert E.rms_rel(u[r], E.potential(D, box, FIELD, x, q[r], targets=t)) < bar, (prec, r)
