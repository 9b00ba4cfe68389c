"""The allocation-free real-space entry point (se_real_noalloc) through the C ABI.

Some callers cannot allocate device memory while they run (a framework that owns all device
memory in its own pool, or a time-step loop that must not stall or fail on an allocation);
se_real_noalloc keeps its scratch in a fixed array inside the library instead. This test
checks that it returns what the allocating entry point returns for the real-space part, on
two calls in a row with different inputs (the second call must not see the first one's
scratch contents), in FP64 and FP32, for every periodicity, that a free coordinate outside
the box is reported as it is by the allocating entry point, and that oversized requests are
refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


# (periodicity, box, grid M of the allocating plan, xi, rc): every periodicity, non-cubic
# boxes, and one cut-off small enough that the fixed array's cap of 32 cells per direction
# replaces the allocating path's finer cell list (the sums must still agree)
CASES = [(3, (1.0, 1.0, 1.0), (32, 32, 32), 9.0, 0.37),
         (2, (1.0, 1.0, 0.5), (32, 32, 16), 9.0, 0.3),
         (1, (4.0, 1.0, 1.0), (128, 32, 32), 9.0, 0.3),
         (0, (1.0, 1.0, 1.0), (32, 32, 32), 9.0, 0.3),
         (3, (1.0, 1.0, 1.0), (32, 32, 32), 40.0, 0.05)]


def _reference(D, box, M, kernel, x, f, xi, rc, prec):
    plan = se.Plan(D, box, xi, rc, M, 8, "pkb", prec)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    ft = torch.tensor(f, dtype=plan.dtype, device="cuda")
    u = plan.evaluate(kernel, xt, ft, parts=se.PART_REAL)
    plan.sync()
    return u.cpu().numpy().astype(np.float64)


def _noalloc(D, box, kernel, x, f, xi, rc, prec):
    dt = torch.float32 if prec == "fp32" else torch.float64
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    ft = torch.tensor(f, dtype=dt, device="cuda")
    u = torch.full((x.shape[0], 3), float("nan"), dtype=dt, device="cuda")
    se.se_real_noalloc(D, box, xi, rc, se.KERNELS[kernel], se.FP32 if prec == "fp32" else se.FP64,
                       xt, ft, u, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,bar", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("kernel", ["stokeslet", "rotlet", "stresslet"])
def test_noalloc_matches_allocating_entry_point_twice(kernel, prec, bar, case):
    D, box, M, xi, rc = CASES[case]
    cases = [(1200, 81), (700, 82)]   # two calls in a row, the second one smaller
    for n, seed in cases:
        x = W.uniform_points(n, box, seed=seed + 10 * case)
        f = W.strengths(kernel, n, seed=seed + 1)
        ref = _reference(D, box, M, kernel, x, f, xi, rc, prec)
        got = _noalloc(D, box, kernel, x, f, xi, rc, prec)
        err = np.sqrt(np.mean(np.sum((got - ref) ** 2, axis=1)) / np.mean(np.sum(ref ** 2, axis=1)))
        assert err < bar, (n, err)


@pytest.mark.parametrize("bad", [1.25, -0.1, float("nan")])
def test_noalloc_reports_free_coordinates_out_of_range(bad):
    """A free-direction coordinate outside [0, L) (or a non-finite one) is an error, as for
    se_eval_parts; the next valid call on the same array succeeds again."""
    box = (1.0, 1.0, 1.0)
    x = W.uniform_points(300, box, seed=5)
    x[17, 2] = bad
    f = W.strengths("stokeslet", 300, seed=6)
    xt = torch.tensor(x, device="cuda")
    ft = torch.tensor(f, device="cuda")
    u = torch.zeros((300, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(se.SeError) as e:
        se.se_real_noalloc(0, box, 9.0, 0.3, se.STOKESLET, se.FP64, xt, ft, u, torch.cuda.current_stream())
    assert e.value.code == -2
    x[17, 2] = 0.5
    xt = torch.tensor(x, device="cuda")
    se.se_real_noalloc(0, box, 9.0, 0.3, se.STOKESLET, se.FP64, xt, ft, u, torch.cuda.current_stream())


def test_noalloc_refuses_oversized_requests():
    n = 65537
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    u = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(se.SeError) as e:
        se.se_real_noalloc(3, (1, 1, 1), 9.0, 0.3, se.STOKESLET, se.FP64, x, f, u)
    assert e.value.code == -8
