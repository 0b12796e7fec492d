"""The energy-drift watchdog (pn_set_watchdog) on the 16k workload: the run's
energy (Eq. 7) jumps between steps 100 and 200, where a star passes the
unsoftened hole closer than one step of 1/2048 resolves (the failure mode
Section 4 shows for its own runs).  The watchdog must stay quiet before that
and report PN_EDRIFT with a step in (100, 200], without faulting or hanging."""
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1801_07986_b300 import pn  # noqa: E402
from paper_1801_07986_b300.inputs import WORKLOADS  # noqa: E402

DEV = torch.device("cuda:0")
TOL, EVERY = 1e-2, 10


def _start(precision="mixed"):
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=0)
    X, V, M = (torch.tensor(a, device=DEV) for a in (x, v, m))
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    return w, ctx, X, V, M, A


def test_watchdog_trips_at_the_hole_encounter():
    w, ctx, X, V, M, A = _start()
    E0 = pn.pn_energy(ctx, X, V, M)["E"]
    pn.pn_set_watchdog(ctx, TOL, EVERY)
    tripped = None
    for s in range(EVERY, 301, EVERY):
        pn.pn_step(ctx, X, V, M, A, w.dt, EVERY)
        try:
            pn.pn_sync(ctx)
        except pn.PNError as e:
            assert e.status == pn.PN_EDRIFT, str(e)
            tripped = (s, str(e))
            break
    assert tripped is not None, "no trip in 300 steps"
    s, msg = tripped
    step = int(re.search(r"first at step (\d+)", msg).group(1))
    assert 100 < step <= 200 and step == s, msg
    # the reported change is the energy's own, measured independently (the
    # reference is the first check's, ten steps in, whose energy differs
    # from the start's by far less than the jump)
    E = pn.pn_energy(ctx, X, V, M)["E"]
    change = float(re.search(r"= ([0-9.eE+-]+) above", msg).group(1))
    assert abs(change - abs(E - E0) / abs(E0)) <= 1e-2 * change
    # the device computes on: later steps run and the flag comes back only
    # while the drift stays above the limit
    pn.pn_set_watchdog(ctx, 0.0)
    pn.pn_step(ctx, X, V, M, A, w.dt, 5)
    pn.pn_sync(ctx)
    assert torch.isfinite(X).all()
    ctx.close()


def test_watchdog_in_graph_replays_keeps_its_reference():
    """The reference taken by the first replayed check persists across
    replays of the captured sequence: the second 100-step replay trips."""
    w, ctx, X, V, M, A = _start()
    pn.pn_set_watchdog(ctx, TOL, EVERY)
    pn.pn_step_graph(ctx, X, V, M, A, w.dt, 100)
    pn.pn_sync(ctx)                                # steps 1-100: quiet
    pn.pn_step_graph(ctx, X, V, M, A, w.dt, 100)   # steps 101-200: the encounter
    with pytest.raises(pn.PNError) as ei:
        pn.pn_sync(ctx)
    assert ei.value.status == pn.PN_EDRIFT
    ctx.close()


def test_watchdog_costs_nothing_when_off_and_rejects_bad_arguments():
    w, ctx, X, V, M, A = _start()
    l0 = pn.pn_launch_count(ctx)
    pn.pn_step(ctx, X, V, M, A, w.dt, 20)
    plain = pn.pn_launch_count(ctx) - l0
    pn.pn_set_watchdog(ctx, 1.0, EVERY)
    l0 = pn.pn_launch_count(ctx)
    pn.pn_step(ctx, X, V, M, A, w.dt, 20)
    pn.pn_sync(ctx)
    watched = pn.pn_launch_count(ctx) - l0
    # two checks (steps 30 and 40 of the context's count): 5 energy kernels
    # (prologue, double-single staging, pair sums, per-star and per-cluster
    # sums) + the comparison each, and the kick-drift kernel of step 31, whose
    # kick and drift could not ride on the epilogue of the checked step 30
    assert watched - plain == 2 * 6 + 1
    pn.pn_set_watchdog(ctx, 0.0)
    l0 = pn.pn_launch_count(ctx)
    pn.pn_step(ctx, X, V, M, A, w.dt, 20)
    assert pn.pn_launch_count(ctx) - l0 == plain
    for tol, every in ((-1.0, 10), (float("nan"), 10), (1e-3, 0)):
        with pytest.raises(pn.PNError) as ei:
            pn.pn_set_watchdog(ctx, tol, every)
        assert ei.value.status == pn.PN_EINVAL
    pn.pn_sync(ctx)
    ctx.close()
