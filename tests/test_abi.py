"""The C-ABI library loads and exports every symbol include/se.h declares; host-only logic
(parameter selection, argument validation) runs without a GPU."""
import math
import os
import re

import pytest

import paper_2210_01255_gb300 as se

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "se.h")).read()
    return sorted(set(re.findall(r"\b(se_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = se.lib()
    names = _declared()
    assert "se_eval" in names and "se_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(se.SIGNATURES), "binding and header disagree"


def test_problem_statement_entry_points_validate_without_gpu():
    """se_plan rejects what se_plan_create rejects; se_eval_batch rejects NULL arrays and a
    non-positive count before any device work."""
    import ctypes
    lib = se.lib()
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(1, 1, 1)
    M = (ctypes.c_int * 3)(32, 32, 32)
    assert lib.se_plan(ctypes.byref(h), 4, box, 10.0, 0.3, M, 8, 2, None) == -1   # periodicity
    assert lib.se_plan(ctypes.byref(h), 3, box, 10.0, 0.3, M, 7, 2, None) == -1   # odd P
    assert lib.se_eval_batch(None, 2, None, None, None, None, None, None) == -1
    plans = (ctypes.c_void_p * 1)(None)
    assert lib.se_eval_batch(plans, 0, None, None, None, None, None, None) == -1


def test_status_strings():
    assert se.se_status_str(0) == "ok"
    assert "unsupported" in se.se_status_str(-7)


def test_plan_argument_validation_without_gpu():
    # invalid arguments are rejected before any device work
    for args in [(4, (1, 1, 1), 10.0, 0.3, (32, 32, 32), 8, 2),     # periodicity
                 (3, (1, 1, 1), -1.0, 0.3, (32, 32, 32), 8, 2),    # xi
                 (3, (1, 1, 1), 10.0, 0.3, (32, 32, 32), 7, 2),    # odd P
                 (3, (1, 1, 1), 10.0, 0.3, (32, 32, 32), 8, 9)]:   # window
        with pytest.raises(se.SeError) as e:
            se.se_plan_create(*args)
        assert e.value.code == -1
    o = se.se_opts_default()
    assert o.tile == 0
    o.tile = 6                                                     # tile depth: 0, 4 or 8
    with pytest.raises(se.SeError) as e:
        se.se_plan_create(3, (1, 1, 1), 10.0, 0.3, (32, 32, 32), 8, 2, o)
    assert e.value.code == -1


# Table 6 of the paper (uniform system): xi from the neighbour count of Table 5 at N = 1e5,
# L = 1, Q = 1 and an absolute real-space tolerance of 1e-8 (Sec. 5.2).
TABLE6 = {("stokeslet", 0): 23.5579, ("stokeslet", 1): 32.3804, ("stokeslet", 2): 41.3955,
          ("stokeslet", 3): 43.0296, ("stresslet", 0): 19.9813, ("stresslet", 1): 31.1944,
          ("stresslet", 2): 39.4021, ("stresslet", 3): 39.4021, ("rotlet", 0): 24.5091,
          ("rotlet", 1): 33.9754, ("rotlet", 2): 43.7207, ("rotlet", 3): 45.4936}


@pytest.mark.parametrize("key", sorted(TABLE6))
def test_autotune_reproduces_table6_xi(key):
    kernel, D = key
    o = se.se_opts_default()
    o.tol_abs = 1e-8
    r = se.se_autotune(D, (1, 1, 1), se.KERNELS[kernel], 1.0, 100000, 0.0, opts=o, xi=0.0)
    assert abs(r["xi"] - TABLE6[key]) < 5e-5


# The clustered-system columns of the same two tables: the neighbour counts N_rc (points only
# in [0,1/3)^3 and [2/3,1)^3; N_rc still counts the mean concentration N / L^3) and the xi
# they give at N = 1e5, tol_abs = 1e-8; passed to the selection through se_opts.n_rc.
NRC_CLUSTERED = {("stokeslet", 0): 800, ("stokeslet", 1): 300, ("stokeslet", 2): 170, ("stokeslet", 3): 120,
                 ("rotlet", 0): 800, ("rotlet", 1): 300, ("rotlet", 2): 170, ("rotlet", 3): 120,
                 ("stresslet", 0): 3000, ("stresslet", 1): 1200, ("stresslet", 2): 370, ("stresslet", 3): 300}
XI_CLUSTERED = {("stokeslet", 0): 34.2623, ("stokeslet", 1): 47.2969, ("stokeslet", 2): 57.0041,
                ("stokeslet", 3): 63.9175, ("stresslet", 0): 25.2392, ("stresslet", 1): 34.3700,
                ("stresslet", 2): 51.0933, ("stresslet", 3): 54.8344, ("rotlet", 0): 36.0043,
                ("rotlet", 1): 50.1320, ("rotlet", 2): 60.7237, ("rotlet", 3): 68.2974}


@pytest.mark.parametrize("key", sorted(XI_CLUSTERED))
def test_autotune_reproduces_clustered_xi_from_n_rc(key):
    kernel, D = key
    o = se.se_opts_default()
    o.tol_abs = 1e-8
    o.n_rc = NRC_CLUSTERED[key]
    r = se.se_autotune(D, (1, 1, 1), se.KERNELS[kernel], 1.0, 100000, 0.0, opts=o, xi=0.0)
    assert abs(r["xi"] - XI_CLUSTERED[key]) < 5e-5


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_harmonic_field_takes_the_rotlet_rules(D):
    """The harmonic field (a first derivative of H like the rotlet) and the harmonic
    potential get the rotlet's parameters and extended-grid options; unknown mask bits are
    rejected."""
    res = []
    for mask in (se.HARMONIC_FIELD, se.ROTLET, se.HARMONIC_FIELD | se.ROTLET, se.HARMONIC,
                 se.HARMONIC | se.HARMONIC_FIELD):
        o = se.se_opts_default()
        o.tol_abs = 1e-8
        r = se.se_autotune(D, (1, 1, 1), mask, 1.0, 20000, 0.0, opts=o)
        res.append((r["xi"], r["rc"], tuple(r["M"]), r["P"], tuple(r["opts"].Mext), r["opts"].s0,
                    r["opts"].s_star, r["opts"].kbar_star))
    assert res[0] == res[1] == res[2] == res[3] == res[4]
    with pytest.raises(se.SeError) as e:
        se.se_autotune(D, (1, 1, 1), 32, 1.0, 20000, 1e-6)
    assert e.value.code == -1


def test_autotune_rules():
    # Sec. 4.6 steps on a case of Sec. 4.6 (N=1000, L=1, Q=1, xi=10)
    o = se.se_opts_default()
    o.tol_abs = 1e-8
    r = se.se_autotune(3, (1, 1, 1), se.STOKESLET, 1.0, 1000, 0.0, opts=o, xi=10.0)
    assert r["P"] % 2 == 0 and r["M"][0] % 4 == 0 and r["M"][0] == r["M"][1] == r["M"][2]
    # free directions: extended grid of Eq. (extended-grid-size) and s0 of Eq. (upsampling-factor-s0)
    r0 = se.se_autotune(0, (1, 1, 1), se.STOKESLET, 1.0, 1000, 0.0, opts=o, xi=10.0)
    M, P = r0["M"][0], r0["P"]
    Mext = r0["opts"].Mext[0]
    assert Mext == 4 * math.ceil((M + P + 1.2 * max(P, 8)) / 4)
    assert abs(r0["opts"].s0 - math.ceil(10 * (1 + math.sqrt(3))) / 10) < 1e-12


def test_window_margin_option():
    """se_opts.P_margin: -1 (default) is the paper's error-pollution rule (+4 points for D >= 1,
    +2 for D = 0); 0 keeps the bare estimate of Eq. (approximation-estimate)."""
    import paper_2210_01255_gb300 as se
    for D, margin in ((3, 4), (2, 4), (0, 2)):
        o = se.se_opts_default()
        assert o.P_margin == -1
        t_paper = se.se_autotune(D, (1.0, 1.0, 1.0), se.STOKESLET, 3000.0, 1000, 1e-8, opts=o)
        o0 = se.se_opts_default()
        o0.P_margin = 0
        t_bare = se.se_autotune(D, (1.0, 1.0, 1.0), se.STOKESLET, 3000.0, 1000, 1e-8, opts=o0)
        assert t_paper["P"] - t_bare["P"] in (margin, margin + 2, margin - 2)  # even rounding
        assert t_paper["P"] > t_bare["P"]
