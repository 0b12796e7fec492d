"""The jerk (Appendix A) and the Hermite integrator on the GPU, against the
FP64 oracle (whose jerk is a complex step of its own Eq. 1-6)."""
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
JERK_TOL = 1e-10          # FP64 jerk vs the oracle, per body (relative)


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def cluster(n, m_bh, seed):
    if n >= 4:
        return make_cluster(n, m_bh, seed)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3))
    x[0] = 0.0
    v = rng.normal(size=(n, 3)) * 0.3
    v[0] = 0.0
    m = np.full(n, 1.0 / (n - 1))
    m[0] = m_bh
    return x, v, m


def gpu_jerk(x, v, m, precision="fp64", **kw):
    n = m.shape[0]
    ctx = pn.pn_init(n, precision=precision, device=0, **kw)
    X, V, M = dev(x), dev(v), dev(m)
    A, J = torch.empty_like(X), torch.empty_like(X)
    pn.pn_jerk(ctx, X, V, M, A, J)
    pn.pn_sync(ctx)
    out = A.cpu().numpy(), J.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("n", [2, 3, 300, 1025])
@pytest.mark.parametrize("c", [12.0, math.inf])
def test_jerk_fp64_matches_oracle(orc, n, c):
    x, v, m = cluster(n, 0.1, 500 + n)
    a_want = orc.accel(x, v, m, c=c, eps=1e-3)
    j_want = orc.jerk(x, v, m, a_want, c=c, eps=1e-3)
    a, j = gpu_jerk(x, v, m, c=c, eps=1e-3)
    assert rel(a, a_want).max() <= 1e-12
    err = rel(j, j_want)
    assert err.max() <= JERK_TOL, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("r_near", [0.05, 0.0])
def test_jerk_strong_field_and_near_hole(orc, r_near):
    """Stars close to the hole at low c, where the 1PN part of the jerk is
    large (and the mixed acceleration path splits near sources off).  In the
    mixed jerk, sources beyond r_near take the hole term in the
    law-of-cosines form and nearer ones (here star 5, 0.01 from the hole)
    the D form; r_near = 0 puts every source on the D form."""
    x, v, m = cluster(600, 0.5, 77)
    x[5] = x[0] + np.array([0.01, 0.0, 0.002])
    v[5] = v[0] + np.array([0.0, 7.0, 0.0])
    c = 6.0
    a_want = orc.accel(x, v, m, c=c, eps=1e-4)
    j_want = orc.jerk(x, v, m, a_want, c=c, eps=1e-4)
    jn = orc.jerk(x, v, m, orc.accel(x, v, m, eps=1e-4), eps=1e-4)
    assert rel(j_want, jn).max() > 1e-2          # the 1PN jerk matters here
    _, j = gpu_jerk(x, v, m, c=c, eps=1e-4)
    assert rel(j, j_want).max() <= JERK_TOL
    # mixed context: a in mixed precision, the jerk's pair sums in FP32 (the
    # jerk enters Hermite's predictor and corrector with dt^2, dt^3 weights)
    a_mix, j_mix = gpu_jerk(x, v, m, precision="mixed", c=c, eps=1e-4, r_near=r_near)
    assert np.median(rel(a_mix, a_want)) <= 2e-7
    err = rel(j_mix, j_want)
    assert np.median(err) <= 2e-5 and err.max() <= 1e-3, (np.median(err), err.max())
    # the hole's jerk against the size of its 1PN part: the mixed pair kernel
    # leaves the stars' Wr sums out and the epilogue restores them from N, U
    # and Z (Wr enters the hole's Eq. 3 terms only); with Wr left out
    # altogether the hole's error here is 3e-4 of its 1PN part, with the
    # restoration 2e-9
    hole_1pn = np.linalg.norm(j_want[0] - jn[0])
    for jj in (j, j_mix):
        assert np.linalg.norm(jj[0] - j_want[0]) <= 1e-6 * hole_1pn, (
            np.linalg.norm(jj[0] - j_want[0]) / hole_1pn)


def test_jerk_plummer16k_against_oracle(orc):
    """The 16k workload's jerk, every body (the hole included), against the
    oracle's complex-step jerk: the FP64 context to JERK_TOL, the mixed
    context (single-precision dual pair sums) to median 1e-6 and max 1e-4."""
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    a_want = orc.accel(x, v, m, G=w.G, c=w.c, eps=w.eps)
    j_want = orc.jerk(x, v, m, a_want, G=w.G, c=w.c, eps=w.eps)
    _, j64 = gpu_jerk(x, v, m, precision="fp64", c=w.c, eps=w.eps)
    err64 = rel(j64, j_want)
    assert err64.max() <= JERK_TOL, err64.max()
    _, jm = gpu_jerk(x, v, m, precision="mixed", c=w.c, eps=w.eps)
    err = rel(jm, j_want)
    assert np.median(err) <= 1e-6 and err.max() <= 1e-4, (np.median(err), err.max())


def test_jerk_batched_per_cluster(orc):
    sizes = [300, 77, 1025]
    xs, vs, ms = zip(*(cluster(s, 0.05 + 0.03 * k, 600 + k) for k, s in enumerate(sizes)))
    off = np.concatenate([[0], np.cumsum(sizes)])
    cs, es = [10.0, 25.0, 60.0], [1e-3, 2e-3, 5e-4]
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="fp64", device=0)
    X, V, M = dev(np.concatenate(xs)), dev(np.concatenate(vs)), dev(np.concatenate(ms))
    A, J = torch.empty_like(X), torch.empty_like(X)
    pn.pn_jerk(ctx, X, V, M, A, J)
    pn.pn_sync(ctx)
    j = J.cpu().numpy()
    for k, (a0, a1) in enumerate(zip(off[:-1], off[1:])):
        want = orc.jerk(xs[k], vs[k], ms[k], c=cs[k], eps=es[k])
        assert rel(j[a0:a1], want).max() <= JERK_TOL
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-6)])
def test_hermite_steps_match_oracle(orc, precision, tol):
    x, v, m = cluster(300, 0.1, 41)
    c, eps, dt, nst = 10.0, 1e-3, 1.0 / 1024, 5
    a0 = orc.accel(x, v, m, c=c, eps=eps)
    xo, vo, ao = orc.hermite_step(x, v, m, a0, dt, nst, c=c, eps=eps)
    ctx = pn.pn_init(300, c=c, eps=eps, precision=precision, integrator="hermite", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_step(ctx, X, V, M, A, dt, nst)
    pn.pn_sync(ctx)
    xg, vg, ag = X.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()
    assert np.abs(xg - xo).max() <= tol * np.abs(xo).max()
    assert rel(vg, vo).max() <= 1e3 * tol
    assert np.median(rel(ag, ao)) <= max(tol, 2e-7)
    ctx.close()


def test_hermite_graph_replay_equals_steps():
    x, v, m = cluster(513, 0.1, 43)
    ctx = pn.pn_init(513, c=20.0, eps=1e-3, precision="mixed", integrator="hermite", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    X2, V2, A2 = X.clone(), V.clone(), A.clone()
    pn.pn_step(ctx, X, V, M, A, 1e-3, 4)
    pn.pn_step_graph(ctx, X2, V2, M, A2, 1e-3, 4)
    pn.pn_sync(ctx)
    assert torch.equal(X, X2) and torch.equal(V, V2) and torch.equal(A, A2)
    ctx.close()


def orbiting(n_stars, m_star, seed, M=1.0):
    """Stars on mildly eccentric orbits at separated radii around the hole."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n_stars + 1, 3))
    v = np.zeros((n_stars + 1, 3))
    for k in range(n_stars):
        r = 1.0 + 4.0 * k / n_stars
        h = rng.normal(size=3)
        h /= np.linalg.norm(h)
        p = np.cross(h, rng.normal(size=3))
        p /= np.linalg.norm(p)
        x[k + 1] = r * p
        v[k + 1] = math.sqrt(M / r) * 1.1 * np.cross(h, p)
    m = np.full(n_stars + 1, m_star)
    m[0] = M
    v[0] = -(m[1:, None] * v[1:]).sum(0) / M
    return x, v, m


def _run(x, v, m, integ, c, dt, nst):
    ctx = pn.pn_init(m.shape[0], c=c, eps=1e-2, precision="fp64", integrator=integ, device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    e0 = pn.pn_energy(ctx, X, V, M)["E"]
    pn.pn_step(ctx, X, V, M, A, dt, nst)
    e1 = pn.pn_energy(ctx, X, V, M)["E"]
    ctx.close()
    return X.cpu().numpy(), abs(e1 / e0 - 1.0)


def test_hermite_is_more_accurate_than_kdk():
    """Section 5's motivation: at the same step the fourth-order scheme
    follows the trajectory (against a fine RK4 run) and, in the Newtonian
    limit where the energy is exactly conserved, keeps it far better than
    the leapfrog.  (The limited-1PN energy of Eq. 7 itself drifts at
    O(1/c^4), so the 1PN comparison is on the trajectory.)"""
    x, v, m = orbiting(63, 1e-4, 45)
    for c in (20.0, math.inf):
        xr, _ = _run(x, v, m, "rk4", c, 1.0 / 512, 1024)
        xk, ek = _run(x, v, m, "kdk", c, 1.0 / 64, 128)
        xh, eh = _run(x, v, m, "hermite", c, 1.0 / 64, 128)
        assert np.abs(xh - xr).max() < 1e-3 * np.abs(xk - xr).max()
        if math.isinf(c):
            assert eh < 1e-2 * ek, (eh, ek)


def test_hermite_batched_per_cluster(orc):
    sizes, cs, es = [200, 77, 513], [10.0, 20.0, 40.0], [1e-3, 2e-3, 5e-4]
    parts = [cluster(s, 0.05 + 0.05 * k, 620 + k) for k, s in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    X = dev(np.concatenate([p[0] for p in parts]))
    V = dev(np.concatenate([p[1] for p in parts]))
    M = dev(np.concatenate([p[2] for p in parts]))
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="fp64", integrator="hermite", device=0)
    A = torch.empty_like(X)
    dt, nst = 1.0 / 1024, 4
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_step(ctx, X, V, M, A, dt, nst)
    pn.pn_sync(ctx)
    xg = X.cpu().numpy()
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        x, v, m = parts[k]
        a0 = orc.accel(x, v, m, c=cs[k], eps=es[k])
        xo, _, _ = orc.hermite_step(x, v, m, a0, dt, nst, c=cs[k], eps=es[k])
        assert np.abs(xg[a:b] - xo).max() <= 1e-11 * np.abs(xo).max()
    ctx.close()
