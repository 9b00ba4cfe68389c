"""se_eval_group: several independent configurations of uneven N on one plan, each stage one
launch over all of them. Through the C ABI, against se_eval of each configuration on the same
plan (the same sums: FP64 to rounding, 1e-12; FP32 to 1e-5) and against the oracle, for
D = 3, 2, 1, 0, every kernel, several RHS, an empty configuration and the dense-block
real-space path (whose blocks of 32 sorted targets must not mix configurations).
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

BOX = {3: (1.0, 1.0, 1.0), 2: (1.0, 1.0, 0.5), 1: (2.0, 1.0, 1.0), 0: (1.0, 1.0, 1.0)}


def rel(a, b):
    a = np.asarray(a, dtype=float).reshape(-1)
    b = np.asarray(b, dtype=float).reshape(-1)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def make(D, kernel, sizes, R, seed, clustered=False):
    box = BOX[D]
    xs, fs = [], []
    for c, n in enumerate(sizes):
        if clustered and n > 0:
            x = W.clustered_points(n, seed=seed + c) * np.asarray(box)
        else:
            x = W.uniform_points(n, box, seed=seed + c)
        xs.append(x.reshape(n, 3))
        fs.append(W.strengths(kernel, max(n, 1), seed=seed + 100 + c, n_rhs=R).reshape(R, max(n, 1), -1)[:, :n])
    return box, xs, fs


def plan_for(D, box, kernel, xs, fs, tol, prec, flags=0):
    N = max(len(x) for x in xs)
    Q = min(W.source_quantity(kernel, f[0]) for f in fs if f.shape[1] > 0)
    t = se.se_autotune(D, box, se.KERNELS[kernel], Q, N, tol)
    o = t["opts"]
    o.kernel_mask = se.KERNELS[kernel]
    o.Q = Q
    o.flags = flags
    return se.Plan(D, box, t["xi"], t["rc"], t["M"], t["P"], "pkb", prec, opts=o)


def group_eval(plan, kernel, xs, fs):
    no = se.out_comps(kernel)
    R = fs[0].shape[0]
    src = torch.tensor(np.concatenate(xs), device="cuda")
    f = torch.tensor(np.concatenate([fc.reshape(-1) for fc in fs]), dtype=plan.dtype, device="cuda")
    u = torch.empty(sum(R * len(x) * no for x in xs), dtype=plan.dtype, device="cuda")
    se.se_eval_group(plan.handle, kernel, [len(x) for x in xs], src, f, R, u)
    plan.sync()
    out, b = [], 0
    u = u.cpu().numpy().astype(np.float64)
    for x in xs:
        k = R * len(x) * no
        out.append(u[b:b + k].reshape(R, len(x), no))
        b += k
    return out


def single_evals(plan, kernel, xs, fs):
    out = []
    for x, f in zip(xs, fs):
        if len(x) == 0:
            out.append(np.zeros((f.shape[0], 0, se.out_comps(kernel))))
            continue
        u = plan.evaluate(kernel, torch.tensor(x, device="cuda"), torch.tensor(f, dtype=plan.dtype, device="cuda"))
        plan.sync()
        out.append(u.cpu().numpy().astype(np.float64).reshape(f.shape[0], len(x), -1))
    return out


@pytest.mark.parametrize("D", [3, 2, 1, 0])
@pytest.mark.parametrize("kernel,R", [("stokeslet", 2), ("rotlet", 1), ("stresslet", 1),
                                      ("stokeslet+stresslet", 1), ("harmonic", 3), ("harmonic_field", 1)])
def test_group_equals_single_evaluations_fp64(D, kernel, R):
    box, xs, fs = make(D, kernel, [300, 1100, 0, 650], R, seed=6000 + D)
    plan = plan_for(D, box, kernel, xs, fs, 1e-11, "fp64")
    g = group_eval(plan, kernel, xs, fs)
    s = single_evals(plan, kernel, xs, fs)
    for a, b in zip(g, s):
        if b.size:
            assert rel(a, b) < 1e-12


@pytest.mark.parametrize("D", [3, 1, 0])
def test_group_fp32_and_oracle(D):
    kernel = "stokeslet"
    box, xs, fs = make(D, kernel, [800, 200, 1500], 1, seed=6100 + D)
    p32 = plan_for(D, box, kernel, xs, fs, 1e-7, "fp32")
    g = group_eval(p32, kernel, xs, fs)
    s = single_evals(p32, kernel, xs, fs)
    p64 = plan_for(D, box, kernel, xs, fs, 1e-11, "fp64")
    g64 = group_eval(p64, kernel, xs, fs)
    for c, (a, b, x, f) in enumerate(zip(g, s, xs, fs)):
        assert rel(a, b) < 1e-5
        idx = np.arange(0, len(x), 3)
        ref = E.potential(D, list(box), kernel, x, f[0], targets=x[idx])
        assert E.rms_rel(g64[c][0][idx], ref) < 1e-10
        assert E.rms_rel(a[0][idx], ref) < 1e-5


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("D", [3, 0])
def test_group_dense_block_real_space(D, prec, bar):
    """Clustered configurations with the dense-block real-space path: blocks of 32 sorted
    targets at a configuration boundary go to the per-target kernel."""
    kernel = "stokeslet+stresslet"
    box, xs, fs = make(D, kernel, [3000, 1017, 2500], 1, seed=6200 + D, clustered=True)
    plan = plan_for(D, box, kernel, xs, fs, 1e-11 if prec == "fp64" else 1e-7, prec, flags=se.FLAG_REAL_BLOCKS)
    g = group_eval(plan, kernel, xs, fs)
    s = single_evals(plan, kernel, xs, fs)
    for a, b in zip(g, s):
        assert rel(a, b) < bar
