"""Boundary-integral workload: the stresslet double layer of a constant density over a
sphere (Eq. stresslet-identity, Sec. 2.5), through the C ABI at explicit targets.

Sources are the nodes of a sphere quadrature (Gauss-Legendre in cos(theta) x trapezoid in
phi) with strengths q = q0 w_n and nu = the outward normal, so that the sum is the
quadrature of the double-layer integral. With T_jlm = -6 r_j r_l r_m / r^5 and the outward
normal it equals 8 pi q0 at every point enclosed by the surface and 0 outside, for every
periodicity (the same identity pins the oracle). This checks the whole GPU path against a
closed form, with no oracle in between, at 18,432 sources and 2,000 targets; the quadrature
is spectrally accurate for targets well away from the surface. One plan then serves
several time steps of a moving surface (plan reuse)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

Q0 = np.array([0.3, -1.1, 0.7])
RADIUS = 0.25


def sphere(center, nth=96, nph=192):
    ct, wt = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C ** 2)
    nrm = np.stack([S * np.cos(P), S * np.sin(P), C], axis=-1).reshape(-1, 3)
    w = (np.outer(wt, np.full(nph, 2 * np.pi / nph)) * RADIUS ** 2).reshape(-1)
    return center + RADIUS * nrm, np.hstack([Q0[None, :] * w[:, None], nrm])


def targets(center, n, seed):
    """n / 2 points within 0.12 of the centre and n / 2 at distances 0.38-0.45 from it (all
    inside the unit box for centres within 0.03 of (0.5, 0.5, 0.5))."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.concatenate([0.12 * rng.random(n // 2) ** (1 / 3), 0.38 + 0.07 * rng.random(n - n // 2)])
    return center + d * r[:, None], np.arange(n) < n // 2


def make_plan(D, x, f, tol, prec):
    Q = float(np.sum((f[:, :3, None] * f[:, None, 3:]) ** 2))
    t = se.se_autotune(D, (1.0, 1.0, 1.0), se.STRESSLET, Q, x.shape[0], tol)
    o = t["opts"]
    o.kernel_mask = se.STRESSLET
    o.Q = Q
    return se.Plan(D, (1.0, 1.0, 1.0), t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def evaluate(plan, x, f, t):
    u = plan.evaluate("stresslet", torch.tensor(x, device="cuda"),
                      torch.tensor(f, dtype=plan.dtype, device="cuda"), torch.tensor(t, device="cuda"))
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


def identity_error(u, inside):
    """max deviation from 8 pi q0 (inside) and 0 (outside), relative to |8 pi q0|."""
    ref = np.where(inside[:, None], 8 * np.pi * Q0[None, :], 0.0)
    return np.abs(u - ref).max() / np.linalg.norm(8 * np.pi * Q0)


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-11, 1e-8), ("fp32", 1e-7, 1e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_double_layer_identity(D, prec, tol, bar):
    c = np.array([0.5, 0.5, 0.5])
    x, f = sphere(c)
    t, inside = targets(c, 2000, seed=40 + D)
    u = evaluate(make_plan(D, x, f, tol, prec), x, f, t)
    assert identity_error(u, inside) < bar


@pytest.mark.parametrize("D", [3, 0])
def test_plan_reuse_over_time_steps(D):
    """One FP32 plan, the surface and its targets moved between evaluations (buffers reused,
    same sizes); every step satisfies the identity."""
    c0 = np.array([0.5, 0.5, 0.5])
    x, f = sphere(c0)
    plan = make_plan(D, x, f, 1e-7, "fp32")
    for k, shift in enumerate([(0, 0, 0), (0.02, -0.01, 0.015), (-0.025, 0.02, -0.01)]):
        c = c0 + np.array(shift)
        x, f = sphere(c)
        t, inside = targets(c, 1000, seed=60 + k)
        assert identity_error(evaluate(plan, x, f, t), inside) < 1e-5, k
