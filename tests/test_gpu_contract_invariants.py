"""Parameter-selection contract and invariants of the GPU path (FP64), through the C ABI.

* Contract (Sec. 4.6: the selected parameters give an RMS error of about the requested
  tolerance, within a factor 10): for a sweep of tolerances the autotuned plan's potential
  is compared with the exact Ewald sums of the oracle at every target.
* Invariants of the sums (Eq. Dp-ewald-decomp and the kernels' definitions): linearity in the
  strengths, permutation of the points, periodic images of the points (coordinates shifted by
  whole periods), and the exact stresslet symmetry under (q, nu) -> (nu, q).
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


def plan_for(D, box, kernel, f, N, tol, prec="fp64"):
    Q = W.source_quantity(kernel, f)
    t = se.se_autotune(D, box, se.KERNELS[kernel], Q, N, tol)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[kernel]
    o.Q = Q
    return se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def evaluate(plan, kernel, x, f):
    u = plan.evaluate(kernel, torch.tensor(np.asarray(x), device="cuda"),
                      torch.tensor(np.asarray(f), dtype=plan.dtype, device="cuda"))
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("D,kernel", [(3, "stokeslet"), (3, "rotlet"), (3, "stresslet"), (2, "stokeslet"),
                                      (0, "stokeslet")])
def test_selected_parameters_meet_the_tolerance(D, kernel, tol):
    """E_rms,rel <= 10 tol at every target (N = 400 uniform points in the unit box)."""
    box = (1.0, 1.0, 1.0)
    N = 400
    x = W.uniform_points(N, box, seed=800 + D)
    f = W.strengths(kernel, N, seed=900 + D)
    u = evaluate(plan_for(D, box, kernel, f, N, tol), kernel, x, f)
    ref = E.potential(D, box, kernel, x, f)
    err = E.rms_rel(u, ref)
    assert 0 < err <= 10 * tol, err


@pytest.mark.parametrize("kernel", ["stokeslet", "rotlet", "stresslet"])
def test_linearity_in_the_strengths(kernel):
    """u(a f1 + b f2) = a u(f1) + b u(f2) (same points, same plan); for the stresslet the
    strength is the pair (q, nu) and the source is q nu^T, so only q is combined."""
    box = (1.0, 1.0, 1.0)
    N = 600
    x = W.uniform_points(N, box, seed=31)
    f1 = W.strengths(kernel, N, seed=32)
    f2 = W.strengths(kernel, N, seed=33)
    if kernel == "stresslet":
        f2[:, 3:] = f1[:, 3:]   # same normals: the source is linear in q
    a, b = 0.7, -1.9
    f = a * f1 + b * f2
    if kernel == "stresslet":
        f[:, 3:] = f1[:, 3:]
    plan = plan_for(3, box, kernel, f1, N, 1e-10)
    lhs = evaluate(plan, kernel, x, f)
    rhs = a * evaluate(plan, kernel, x, f1) + b * evaluate(plan, kernel, x, f2)
    assert E.rms_rel(lhs, rhs) < 1e-13


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_permutation_of_points(D):
    """Permuting the points permutes the potentials."""
    box = (1.0, 1.0, 1.0)
    N = 500
    x = W.uniform_points(N, box, seed=41 + D)
    f = W.strengths("stokeslet", N, seed=51 + D)
    plan = plan_for(D, box, "stokeslet", f, N, 1e-10)
    u = evaluate(plan, "stokeslet", x, f)
    perm = np.random.default_rng(61).permutation(N)
    up = evaluate(plan, "stokeslet", x[perm], f[perm])
    assert E.rms_rel(up, u[perm]) < 1e-13


@pytest.mark.parametrize("D", [3, 2, 1])
def test_periodic_images_of_the_points(D):
    """Shifting coordinates by whole periods in the periodic directions changes nothing."""
    box = (1.0, 1.0, 1.0)
    N = 500
    x = W.uniform_points(N, box, seed=71 + D)
    f = W.strengths("stresslet", N, seed=81 + D)
    plan = plan_for(D, box, "stresslet", f, N, 1e-10)
    u = evaluate(plan, "stresslet", x, f)
    k = np.random.default_rng(91).integers(-2, 3, size=(N, 3)).astype(float)
    k[:, D:] = 0.0   # only the periodic directions
    xs = x + k * np.asarray(box)
    us = evaluate(plan, "stresslet", xs, f)
    assert E.rms_rel(us, u) < 1e-12


def test_stresslet_symmetry_in_q_and_nu():
    """T_jlm is fully symmetric, so (q, nu) and (nu, q) give the same potential."""
    box = (1.0, 1.0, 1.0)
    N = 500
    x = W.uniform_points(N, box, seed=101)
    f = W.strengths("stresslet", N, seed=102)
    g = np.concatenate([f[:, 3:], f[:, :3]], axis=1)
    plan = plan_for(3, box, "stresslet", f, N, 1e-10)
    assert E.rms_rel(evaluate(plan, "stresslet", x, g), evaluate(plan, "stresslet", x, f)) < 1e-13
