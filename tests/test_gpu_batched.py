"""Batched contexts: many independent clusters of uneven size in one set of
launches (the pair kernel balances their work), checked cluster by cluster
against the FP64 oracle, plus CUDA-graph stepping and the autotuner."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1801_07986_b300 import pn  # noqa: E402
from paper_1801_07986_b300.inputs import make_cluster  # noqa: E402

DEV = torch.device("cuda:0")
FP64_TOL = 1e-12
MIX_MED, MIX_MAX = 2e-7, 1e-5
SIZES = [300, 1025, 77, 2048, 513, 4100]


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def batch(sizes=SIZES, seed=900):
    xs, vs, ms, Ms, cs, es = [], [], [], [], [], []
    rng = np.random.default_rng(seed)
    for k, n in enumerate(sizes):
        M = float(rng.uniform(0.01, 0.2))
        x, v, m = make_cluster(n, M, seed + k)
        x = x + rng.normal(size=3) * 5.0          # clusters at different places
        xs.append(x); vs.append(v); ms.append(m)
        Ms.append(M)
        cs.append(float(rng.uniform(20.0, 200.0)))
        es.append(float(rng.choice([0.0, 1e-4, 1e-3])))
    off = np.concatenate([[0], np.cumsum(sizes)])
    return (np.concatenate(xs), np.concatenate(vs), np.concatenate(ms), off,
            np.array(cs), np.array(es))


def oracle_accels(orc, x, v, m, off, cs, es):
    return [orc.accel(x[a:b], v[a:b], m[a:b], c=c, eps=e)
            for a, b, c, e in zip(off[:-1], off[1:], cs, es)]


@pytest.mark.parametrize("precision,pair_kernel,spatial",
                         [("fp64", "two_pass", "0"), ("mixed", "fused", "0"),
                          ("mixed", "fused", "1"), ("mixed", "two_pass", "0")])
def test_batched_accel_matches_oracle_per_cluster(orc, monkeypatch, precision, pair_kernel,
                                                  spatial):
    """spatial = 1: the packed kernel on the Hilbert order of every cluster
    (sorted within each cluster's slot range) with cost-balanced workers."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    x, v, m, off, cs, es = batch()
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision=precision, pair_kernel=pair_kernel,
                             device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    for (a, b), want in zip(zip(off[:-1], off[1:]), oracle_accels(orc, x, v, m, off, cs, es)):
        err = rel(got[a:b], want)
        if precision == "fp64":
            assert err.max() <= FP64_TOL, (a, b, err.max())
        else:
            assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (a, b, np.median(err),
                                                                         err.max())
    ctx.close()


def test_batched_energy_per_cluster(orc):
    x, v, m, off, cs, es = batch()
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="mixed", device=0)
    got = pn.pn_energy(ctx, dev(x), dev(v), dev(m))
    assert len(got) == len(SIZES)
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        want = orc.energy(x[a:b], v[a:b], m[a:b], c=cs[k], eps=es[k])
        for key in ("E_N", "E_PN"):
            assert abs(got[k][key] - want[key]) <= 1e-12 * abs(want[key])
    ctx.close()


def test_batched_steps_match_oracle_and_graph_replays_bitwise(orc):
    x, v, m, off, cs, es = batch(sizes=[300, 1025, 513])
    dt = 1.0 / 2048
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="fp64", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    X2, V2, A2 = X.clone(), V.clone(), A.clone()
    n0 = pn.pn_launch_count(ctx)
    pn.pn_step(ctx, X, V, M, A, dt, 6)
    n1 = pn.pn_launch_count(ctx)
    pn.pn_step_graph(ctx, X2, V2, M, A2, dt, 3)     # capture + replay
    pn.pn_step_graph(ctx, X2, V2, M, A2, dt, 3)     # replay of the same graph
    n2 = pn.pn_launch_count(ctx)
    pn.pn_sync(ctx)
    assert torch.equal(X, X2) and torch.equal(V, V2) and torch.equal(A, A2)
    # one step = prologue, global sums, the pair kernel (one FP64 sweep),
    # epilogue with the hole (+ near scatter and near pass when r_near > 0);
    # the kick-drift kernel runs once per call (later steps' ride on the
    # previous epilogue); graph replays count alike
    per = (n1 - n0 - 1) // 6
    assert per in (4, 6) and n1 - n0 == 6 * per + 1
    assert n2 - n1 == 2 * (3 * per + 1)
    xg = X.cpu().numpy()
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        a0 = orc.accel(x[a:b], v[a:b], m[a:b], c=cs[k], eps=es[k])
        xo, vo, ao = orc.step(x[a:b], v[a:b], m[a:b], a0, dt, 6, c=cs[k], eps=es[k])
        assert np.abs(xg[a:b] - xo).max() < 1e-12
    ctx.close()


@pytest.mark.parametrize("spatial", ["0", "1"])
def test_mixed_graph_replays_equal_eager_steps_bitwise(orc, monkeypatch, spatial):
    """Mixed precision with the near-source split and its side stream, on the
    slot order and on the Hilbert order (sorted again every evaluation):
    two replays of a 3-step graph give the same bits as one 6-step pn_step
    call (no step depends on how the steps are grouped into calls), and the
    final state stays within the mixed tolerance of the oracle's 6 KDK
    steps, cluster by cluster (the median relative error of the change of x
    and of v over the steps within 1e-6; the 1PN terms make a median 2e-5
    to 4e-4 of the velocity change in these clusters, so a dropped term
    fails it)."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    x, v, m, off, cs, es = batch(sizes=[300, 1025, 2048, 513])
    dt = 1.0 / 2048
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    X2, V2, A2 = X.clone(), V.clone(), A.clone()
    pn.pn_step(ctx, X, V, M, A, dt, 6)
    pn.pn_step_graph(ctx, X2, V2, M, A2, dt, 3)
    pn.pn_step_graph(ctx, X2, V2, M, A2, dt, 3)
    pn.pn_sync(ctx)
    assert torch.equal(X, X2) and torch.equal(V, V2) and torch.equal(A, A2)
    if spatial == "1":
        _, units = pn.pn_get_pair_stats(ctx)
        assert units > 0            # the spatially ordered kernel ran
    xg, vg = X.cpu().numpy(), V.cpu().numpy()
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        a0 = orc.accel(x[a:b], v[a:b], m[a:b], c=cs[k], eps=es[k])
        xo, vo, _ = orc.step(x[a:b], v[a:b], m[a:b], a0, dt, 6, c=cs[k], eps=es[k])
        # six steps of dt carry the force error as dt^2-sized position error
        # on top of the state: compare the change over the steps
        dx = np.linalg.norm((xg[a:b] - xo), axis=-1)
        scale = np.linalg.norm(xo - x[a:b], axis=-1)
        assert np.median(dx / scale) <= 1e-6, (k, np.median(dx / scale))
        dv = np.linalg.norm((vg[a:b] - vo), axis=-1)
        vscale = np.linalg.norm(vo - v[a:b], axis=-1)
        assert np.median(dv / vscale) <= 1e-6, (k, np.median(dv / vscale))
    ctx.close()


def test_tune_keeps_parity(orc):
    x, v, m, off, cs, es = batch()
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    choice = pn.pn_tune(ctx, X, V, M, A)
    assert choice["targets_per_thread"] in (2, 4) and choice["unroll"] in (1, 2)
    again = pn.pn_tune(ctx, X, V, M, A)
    assert again["cached"] and again["targets_per_thread"] == choice["targets_per_thread"]
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    for (a, b), want in zip(zip(off[:-1], off[1:]), oracle_accels(orc, x, v, m, off, cs, es)):
        err = rel(got[a:b], want)
        assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX
    ctx.close()


TUNE_CHILD = r"""
import sys, torch
from paper_1801_07986_b300 import pn
from paper_1801_07986_b300.inputs import make_cluster
x, v, m = make_cluster(3000, 0.1, 77)
X, V, M = (torch.tensor(a, device="cuda:0") for a in (x, v, m))
A = torch.empty_like(X)
ctx = pn.pn_init(3000, c=30.0, eps=1e-4, precision="mixed", device=0)
t = pn.pn_tune(ctx, X, V, M, A)
print(int(t["cached"]), t["targets_per_thread"], t["unroll"], int(t["packed"]), t["tile"], t["stages"])
"""


def test_tune_reports_tile_and_keeps_its_choice_in_the_cache_file(tmp_path):
    """pn_tune searches the packed kernel's j-tile and buffers too, reports
    them, and with PN_TUNE_CACHE a later process takes the choice from the
    file without timing again (a malformed line before it is skipped)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, PYTHONPATH=root, PN_TUNE_CACHE=str(cache))
    runs = []
    for q in range(2):
        if q == 1:
            cache.write_text("not a tuning line\n" + cache.read_text())
        runs.append(subprocess.run([sys.executable, "-c", TUNE_CHILD], env=env,
                                   capture_output=True, text=True, timeout=600, cwd=root))
    for r in runs:
        assert r.returncode == 0, r.stderr[-2000:]
    first, second = (r.stdout.split() for r in runs)
    assert first[0] == "0" and second[0] == "1"           # timed, then read from the file
    assert first[1:] == second[1:]
    P, unroll, packed, tile, stages = (int(q) for q in first[1:])
    assert (tile, stages) in ((64, 6), (64, 4), (32, 8)) if packed else stages == 0
    lines = cache.read_text().split("\n")
    assert len([q for q in lines if q.strip()]) == 2      # the bad line + the one choice


def test_nonfinite_in_one_cluster_is_reported():
    x, v, m, off, cs, es = batch(sizes=[300, 600])
    x = x.copy()
    x[off[1] + 7] = x[off[1]]          # a star of cluster 1 on its hole
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    with pytest.raises(pn.PNError) as ei:
        pn.pn_sync(ctx)
    assert ei.value.status == pn.PN_ENONFINITE
    ctx.close()


def test_batched64_workload_sampled(orc):
    """The 64-cluster workload (N log-uniform in [512, 32768]) in one batched
    context: sampled stars and the hole of every cluster against the oracle
    (the hole's O(N^2) double sum included, up to N = 31017)."""
    from paper_1801_07986_b300.inputs import batched_workloads
    ws = batched_workloads()
    xs, vs, ms = zip(*(w.state() for w in ws))
    off = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    x, v, m = np.concatenate(xs), np.concatenate(vs), np.concatenate(ms)
    ctx = pn.pn_init_batched(off, c=[w.c for w in ws], eps=[w.eps for w in ws],
                             precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    ctx.close()
    rng = np.random.default_rng(64)
    errs = []
    for k, w in enumerate(ws):
        a, b = off[k], off[k + 1]
        rows = [0] + list(rng.choice(np.arange(1, w.n), 4, replace=False))
        want = orc.accel_rows(x[a:b], v[a:b], m[a:b], rows, c=w.c, eps=w.eps)
        errs.append(rel(got[a:b][rows], want))
    err = np.concatenate(errs)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())
