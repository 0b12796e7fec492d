"""The measured workloads run as configured, checked against the FP64 oracle
on the GPU's own state along the run (same-state force parity: the oracle
evaluates A where the GPU trajectory is, so chaotic divergence of the two
trajectories does not enter the comparison):

  1k FP64    every step of 100: every body, <= 1e-12; final energy against
             the oracle's on the same state; trajectory against the
             oracle's own 100 steps;
  16k        steps 0, 100, ..., 1000 (mixed) and 0, 100, 200, 300 (FP64):
             sampled stars, the hole at the first and last check;
  128k ecc   steps 0, 50, 100, 150, 200 (mixed): sampled stars of both
             populations.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1801_07986_b300 import pn  # noqa: E402
from paper_1801_07986_b300.inputs import WORKLOADS  # noqa: E402

DEV = torch.device("cuda:0")
FP64_TOL = 1e-12
MIX_MED, MIX_MAX = 2e-7, 1e-5


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


class Run:
    """A context stepping one workload; accel() is A on the current state."""

    def __init__(self, w, precision):
        self.w = w
        x, v, m = w.state()
        self.m = m
        self.ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=0)
        self.X, self.V, self.M = dev(x), dev(v), dev(m)
        self.A = torch.empty_like(self.X)
        pn.pn_accel(self.ctx, self.X, self.V, self.M, self.A)

    def step(self, k):
        pn.pn_step(self.ctx, self.X, self.V, self.M, self.A, self.w.dt, k)

    def state(self):
        pn.pn_sync(self.ctx)
        return self.X.cpu().numpy(), self.V.cpu().numpy()

    def accel(self):
        B = torch.empty_like(self.X)
        pn.pn_accel(self.ctx, self.X, self.V, self.M, B)
        pn.pn_sync(self.ctx)
        return B.cpu().numpy()

    def close(self):
        self.ctx.close()


def test_plummer1k_fp64_every_step_same_state(orc):
    w = WORKLOADS["plummer1k_fp64"]
    r = Run(w, "fp64")
    x0, v0 = r.state()
    worst = 0.0
    for _ in range(w.steps):
        r.step(1)
        x, v = r.state()
        got = r.accel()
        want = orc.accel(x, v, r.m, G=w.G, c=w.c, eps=w.eps)
        worst = max(worst, rel(got, want).max())
    assert worst <= FP64_TOL, worst
    e_gpu = pn.pn_energy(r.ctx, r.X, r.V, r.M)
    e_orc = orc.energy(x, v, r.m, G=w.G, c=w.c, eps=w.eps)
    assert abs(e_gpu["E"] - e_orc["E"]) <= 1e-12 * abs(e_orc["E"])
    e0 = orc.energy(x0, v0, r.m, G=w.G, c=w.c, eps=w.eps)["E"]
    assert abs(e_orc["E"] - e0) <= 1e-4 * abs(e0)          # the run stays physical
    r.close()
    # the oracle's own trajectory from the same start
    a0 = orc.accel(x0, v0, r.m, G=w.G, c=w.c, eps=w.eps)
    xo, vo, _ = orc.step(x0, v0, r.m, a0, w.dt, w.steps, G=w.G, c=w.c, eps=w.eps)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


def _sampled_check(orc, w, x, v, m, got, rng, hole, nrows=120):
    rows = list(rng.choice(np.arange(1, w.n), nrows, replace=False))
    if hole:
        rows = [0] + rows
    want = orc.accel_rows(x, v, m, rows, G=w.G, c=w.c, eps=w.eps)
    return rel(got[rows], want)


@pytest.mark.parametrize("precision,nsteps", [("mixed", 1000), ("fp64", 300)])
def test_plummer16k_same_state_every_100_steps(orc, precision, nsteps):
    w = WORKLOADS["plummer16k"]
    r = Run(w, precision)
    rng = np.random.default_rng(16)
    errs = []
    for s in range(0, nsteps + 1, 100):
        if s:
            r.step(100)
        x, v = r.state()
        err = _sampled_check(orc, w, x, v, r.m, r.accel(), rng, hole=s in (0, nsteps))
        errs.append(err)
        if precision == "fp64":
            assert err.max() <= FP64_TOL, (s, err.max())
        else:
            assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (s, np.median(err),
                                                                         err.max())
    r.close()


def test_plummer128k_eccentric_same_state_every_50_steps(orc):
    w = WORKLOADS["plummer128k_ecc"]
    r = Run(w, "mixed")
    rng = np.random.default_rng(128)
    n_ecc = int(round(w.ecc_frac * (w.n - 1)))
    for s in range(0, w.steps + 1, 50):
        if s:
            r.step(50)
        x, v = r.state()
        got = r.accel()
        assert np.all(np.isfinite(got))
        rows = np.concatenate([rng.choice(np.arange(1, n_ecc + 1), 40, replace=False),
                               rng.choice(np.arange(n_ecc + 1, w.n), 100, replace=False)])
        want = orc.accel_rows(x, v, r.m, rows, G=w.G, c=w.c, eps=w.eps)
        err = rel(got[rows], want)
        assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (s, np.median(err), err.max())
    r.close()
