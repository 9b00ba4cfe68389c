"""Host-side logic of bench.py and the seeded generators (CPU): the evaluation lists of every
workload, the clustered generators, the unit source quantity of the timing experiments and the
real-space pair count against brute force."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402


def test_two_cube_points_lie_in_the_two_cubes():
    x = W.two_cube_points(1001, seed=3)
    lo = np.all(x < 1.0 / 3.0, axis=1)
    hi = np.all(x >= 2.0 / 3.0, axis=1) & np.all(x < 1.0, axis=1)
    assert np.all(lo | hi) and lo.sum() == 500 and hi.sum() == 501


def test_batch_sizes_log_uniform_and_seeded():
    n = W.batch_sizes(64, 2000, 50000, seed=5)
    assert n.shape == (64,) and n.min() >= 2000 and n.max() <= 50000
    assert np.array_equal(n, W.batch_sizes(64, 2000, 50000, seed=5))
    # log-uniform: the median sits near the geometric mean sqrt(2000 * 50000) = 10,000
    assert 5000 < np.median(n) < 20000


@pytest.mark.parametrize("kernel,c", [("stokeslet", 3), ("rotlet", 3), ("stresslet", 6), ("stokeslet+stresslet", 9)])
def test_strengths_layout_and_unit_normals(kernel, c):
    f = W.strengths(kernel, 50, seed=1, n_rhs=2)
    assert f.shape == (2, 50, c)
    if kernel != "stokeslet" and kernel != "rotlet":
        nu = f[..., -3:]
        assert np.allclose(np.linalg.norm(nu, axis=-1), 1.0)


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_unit_q_strengths(kernel):
    f = bench.unit_q_strengths(kernel, 300, seed=2)
    assert abs(W.source_quantity(kernel, f) - 1.0) < 1e-12


def test_source_quantity_of_combined_strengths_adds():
    f = W.strengths("stokeslet+stresslet", 40, seed=4)
    q = W.source_quantity("stokeslet+stresslet", f)
    assert abs(q - W.source_quantity("stokeslet", f[:, :3]) - W.source_quantity("stresslet", f[:, 3:])) < 1e-12


@pytest.mark.parametrize("name", sorted(bench.METRIC_NAMES))
def test_every_workload_builds_its_evaluations(name):
    cfg = W.CONFIGS[name]
    if cfg.get("N", 0) > 300000:
        pytest.skip("large point cloud")
    items = bench.make_items(cfg)
    R = cfg.get("n_rhs", 1)
    n_eval = cfg.get("n_cfg", 1) * len(cfg["kernels"])
    assert len(items) == n_eval
    for it in items:
        assert it["f"].shape == (R, it["N"], bench.COMPS[it["kernel"]])
        assert it["x"].shape == (it["N"], 3)
        assert it["f"].dtype == (np.float32 if cfg["prec"] == "fp32" else np.float64)


def test_real_pairs_clustered_against_brute_force():
    """The k-d tree sample count of pairs within rc against the exact count on a small cloud."""
    cfg = dict(box=(1.0, 1.0, 1.0), points="clustered")
    x = W.clustered_points(6000, seed=9)
    item = dict(N=6000, x=x)
    rc = 0.05
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    exact = float((d2 < rc * rc).sum() - 6000)
    est = bench.real_pairs(cfg, item, rc)
    assert abs(est / exact - 1.0) < 0.1  # a 4096-target sample of 6000


def test_real_pairs_uniform_formula():
    cfg = dict(box=(1.0, 1.0, 0.5))
    item = dict(N=1000)
    assert bench.real_pairs(cfg, item, 0.1) == pytest.approx(1000 * 999 / 0.5 * 4.0 / 3.0 * math.pi * 1e-3)


def test_neighbour_table_matches_the_selection_defaults():
    """The uniform column of the timing experiments' N_rc table is the selection's default
    (Table 5): se_autotune with n_rc = 0 and with the table value give the same xi."""
    import paper_2210_01255_gb300 as se
    for k in ("stokeslet", "stresslet", "rotlet"):
        for D in range(4):
            o1 = se.se_opts_default()
            o1.tol_abs = 1e-8
            o2 = se.se_opts_default()
            o2.tol_abs = 1e-8
            o2.n_rc = bench.NRC_TABLE["uniform"][k][D]
            a = se.se_autotune(D, (1, 1, 1), se.KERNELS[k], 1.0, 100000, 0.0, opts=o1)
            b = se.se_autotune(D, (1, 1, 1), se.KERNELS[k], 1.0, 100000, 0.0, opts=o2)
            assert a["xi"] == pytest.approx(b["xi"], rel=1e-12), (k, D)


def test_traffic_rows_need_matching_parameters_and_sources(tmp_path, monkeypatch):
    """roofline.traffic is read from profiles/traffic_<workload>.txt only for the same
    evaluation, parameters and kernel source; anything else gives None."""
    import hashlib
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2210_01255_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "se_real.cu").write_text("// kernel source\n")
    sha = hashlib.sha256(b"// kernel source\n").hexdigest()[:16]
    p = {"M": [100, 100, 100], "P": 8, "rc": 0.05}
    (tmp_path / "profiles" / "traffic_w.txt").write_text(
        "# header\nreal st %s 1000 %s\nreal st 90:8:0.05000 7 %s\n" % (bench.param_key(p), sha, sha))
    assert bench.kernel_traffic("w", "real", {"st": p}) == 1000.0
    assert bench.kernel_traffic("w", "real", {"st": dict(p, P=10)}) is None
    assert bench.kernel_traffic("w", "spread", {"st": p}) is None
    assert bench.kernel_traffic("other", "real", {"st": p}) is None
    (csrc / "se_real.cu").write_text("// changed\n")
    assert bench.kernel_traffic("w", "real", {"st": p}) is None


def test_both_arms_count_points_alike():
    """config.N: the points of one kernel's evaluations (a workload of two kernels on the same
    points counts them once), the same in the GPU arm and the reference arm."""
    for name in bench.METRIC_NAMES:
        cfg = W.CONFIGS[name]
        items = bench.make_items(cfg)
        n = bench.config_n(items)
        if "n_cfg" in cfg:
            assert n == sum(int(v) for v in W.batch_sizes(cfg["n_cfg"], *cfg["N_range"], seed=cfg["seed"]))
        else:
            assert n == cfg["N"]
