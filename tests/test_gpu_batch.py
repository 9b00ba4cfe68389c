"""Batches of independent configurations under one CUDA graph (se_batch_*), through the C ABI.

Workload shape: singly periodic stokeslet systems in the box (4,1,1), N log-uniform in
[2e3, 5e4], 16 right-hand sides each, FP32 at 1e-6, each configuration with its own plan.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2210_01255_gb300 as se  # noqa: E402
from paper_2210_01255_gb300 import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BOX = (4.0, 1.0, 1.0)


def _configs(n_cfg, lo, hi, seed, n_rhs):
    rng = np.random.default_rng(seed)
    Ns = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_cfg))).astype(int)
    out = []
    for i, N in enumerate(Ns):
        x = W.uniform_points(int(N), BOX, seed=seed + 1 + i)
        f = W.strengths("stokeslet", int(N), seed=seed + 1000 + i, n_rhs=n_rhs)
        out.append((x, f))
    return out


def _plans(cfgs, stream, tol):
    plans = []
    for x, f in cfgs:
        Q = W.source_quantity("stokeslet", f[0])
        t = se.se_autotune(1, BOX, se.STOKESLET, Q, x.shape[0], tol / 10.0)
        o = t["opts"]
        o.kernel_mask = se.STOKESLET
        o.Q = Q
        plans.append(se.Plan(1, BOX, t["xi"], t["rc"], t["M"], t["P"], "pkb", "fp32", opts=o, stream=stream))
    return plans


def _run_batch(n_cfg, lo, hi, seed, n_rhs, check_oracle):
    stream = torch.cuda.Stream()
    cfgs = _configs(n_cfg, lo, hi, seed, n_rhs)
    with torch.cuda.stream(stream):
        plans = _plans(cfgs, stream, 1e-6)
        xs = [torch.tensor(x, device="cuda") for x, _ in cfgs]
        fs = [torch.tensor(f, dtype=torch.float32, device="cuda") for _, f in cfgs]
        us = [torch.zeros((n_rhs, x.shape[0], 3), dtype=torch.float32, device="cuda") for x, _ in cfgs]
        b = se.se_batch_create([p.handle for p in plans], [se.STOKESLET] * n_cfg, xs, fs, [n_rhs] * n_cfg, us)
        for u in us:
            u.fill_(float("nan"))
        se.se_batch_launch(b)
        stream.synchronize()
        got = [u.cpu().numpy().astype(np.float64) for u in us]
        # same configurations one by one through se_eval
        ref = []
        for p, x, f in zip(plans, xs, fs):
            ref.append(p.evaluate("stokeslet", x, f).cpu().numpy().astype(np.float64))
        stream.synchronize()
        for g_, r_ in zip(got, ref):
            assert E.rms_rel(g_.reshape(-1, 3), r_.reshape(-1, 3)) < 1e-6
        # a second replay on unchanged inputs gives the same potentials (up to the order of the
        # atomic additions of partial grid tiles)
        for u in us:
            u.fill_(float("nan"))
        se.se_batch_launch(b)
        stream.synchronize()
        for u, g_ in zip(us, got):
            assert E.rms_rel(u.cpu().numpy().astype(np.float64).reshape(-1, 3), g_.reshape(-1, 3)) < 1e-6
        # refill one configuration's strengths in place and replay
        fs[0].mul_(-2.0)
        se.se_batch_launch(b)
        stream.synchronize()
        assert E.rms_rel(us[0].cpu().numpy().reshape(-1, 3), -2.0 * got[0].reshape(-1, 3)) < 1e-5
        fs[0].div_(-2.0)
        if check_oracle:
            se.se_batch_launch(b)
            stream.synchronize()
            for i in (0, n_cfg - 1):
                x, f = cfgs[i]
                idx = np.random.default_rng(3).choice(x.shape[0], 8, replace=False)
                for r in (0, n_rhs - 1):
                    e = E.potential(1, BOX, "stokeslet", x, f[r], targets=x[idx])
                    assert E.rms_rel(us[i][r].cpu().numpy()[idx].astype(np.float64), e) < 1e-5
        se.se_batch_destroy(b)
        del plans


def test_batch_graph_matches_individual_evaluations():
    _run_batch(6, 2000, 8000, 50, 4, check_oracle=True)


def test_batch_64_configurations_16_rhs():
    """64 configurations, N log-uniform in [2e3, 5e4], 16 RHS each, one graph launch."""
    _run_batch(64, 2000, 50000, 70, 16, check_oracle=True)


def test_eval_batch_one_call_matches_individual_evaluations():
    """se_eval_batch: 5 configurations (mixed kernels, one on its own stream) in one call
    equal the individual se_eval results; each compared with the oracle at sampled targets."""
    cfgs = _configs(5, 2000, 6000, 90, 2)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    kernels = ["stokeslet", "stokeslet", "stresslet", "rotlet", "stokeslet+stresslet"]
    plans, xs, fs, us, refs = [], [], [], [], []
    for i, ((x, _), k) in enumerate(zip(cfgs, kernels)):
        f = W.strengths(k, x.shape[0], seed=95 + i, n_rhs=2)
        Q = W.source_quantity(k, f[0])
        t = se.se_autotune(1, BOX, se.KERNELS[k], Q, x.shape[0], 1e-7)
        o = t["opts"]
        o.kernel_mask = se.KERNELS[k]
        st = s2 if i == 3 else s1
        p = se.Plan(1, BOX, t["xi"], t["rc"], t["M"], t["P"], "pkb", "fp64", opts=o, stream=st)
        xt = torch.tensor(x, device="cuda")
        ft = torch.tensor(f, device="cuda")
        u_ref = p.evaluate(k, xt, ft)
        p.sync()  # the copy below runs on torch's current stream
        refs.append(u_ref.clone())
        plans.append(p)
        xs.append(xt)
        fs.append(ft)
        us.append(torch.full_like(refs[-1], float("nan")))
    torch.cuda.synchronize()  # inputs and fills complete before the plans' streams write
    se.se_eval_batch([p.handle for p in plans], kernels, xs, fs, [2] * 5, us)
    for p in plans:
        p.sync()
    for i, (u, r) in enumerate(zip(us, refs)):
        assert torch.equal(u, r) or float((u - r).abs().max() / r.abs().max()) < 1e-12, i
        x = cfgs[i][0]
        f = fs[i].cpu().numpy()[1]
        idx = np.random.default_rng(7).choice(x.shape[0], 6, replace=False)
        if kernels[i] == "stokeslet+stresslet":
            e = (E.potential(1, BOX, "stokeslet", x, f[:, :3], targets=x[idx])
                 + E.potential(1, BOX, "stresslet", x, f[:, 3:], targets=x[idx]))
        else:
            e = E.potential(1, BOX, kernels[i], x, f, targets=x[idx])
        assert E.rms_rel(u[1].cpu().numpy()[idx], e) < 1e-6, i
