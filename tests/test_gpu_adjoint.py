"""The adjoint of the accelerations and of KDK steps (pn_accel_vjp,
pn_step_vjp, the torch.autograd trajectory) against the FP64 oracle's exact
directional derivatives (complex step), contracted with the same cotangents,
and against central differences of the GPU's own FP64 path."""
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def state(n, seed, m_bh=0.3):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3))
    x[0] = 0.0
    v = rng.normal(size=(n, 3)) * 0.4
    v[0] = 0.0
    m = np.full(n, 0.02)
    m[0] = m_bh
    return x, v, m


def oracle_vjp_accel(orc, x, v, m, abar, c, eps):
    """abar . J for every input direction (positions, velocities, M, 1/c^2)."""
    n = len(m)
    xb, vb = np.zeros((n, 3)), np.zeros((n, 3))
    z = np.zeros((n, 3))
    for i in range(n):
        for k in range(3):
            e = np.zeros((n, 3))
            e[i, k] = 1.0
            xb[i, k] = np.sum(abar * orc.accel_jvp(x, v, m, e, z, c=c, eps=eps))
            vb[i, k] = np.sum(abar * orc.accel_jvp(x, v, m, z, e, c=c, eps=eps))
    Mb = np.sum(abar * orc.accel_jvp(x, v, m, z, z, dM=1.0, c=c, eps=eps))
    cb = np.sum(abar * orc.accel_jvp(x, v, m, z, z, dinv_c2=1.0, c=c, eps=eps))
    return xb, vb, Mb, cb


@pytest.mark.parametrize("n", [2, 3, 20, 40])
def test_accel_vjp_matches_oracle(orc, n):
    x, v, m = state(n, 700 + n)
    c, eps = 6.0, 1e-2
    abar = np.random.default_rng(n).normal(size=(n, 3))
    want = oracle_vjp_accel(orc, x, v, m, abar, c, eps)
    ctx = pn.pn_init(n, c=c, eps=eps, precision="fp64", device=0)
    X, V, M, AB = dev(x), dev(v), dev(m), dev(abar)
    XB, VB = torch.empty_like(X), torch.empty_like(X)
    scal = pn.pn_accel_vjp(ctx, X, V, M, AB, XB, VB)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    assert np.abs(xb - want[0]).max() <= 1e-10 * np.abs(want[0]).max()
    assert np.abs(vb - want[1]).max() <= 1e-10 * max(np.abs(want[1]).max(), 1e-300)
    assert abs(scal[0, 0] - want[2]) <= 1e-10 * abs(want[2])
    assert abs(scal[0, 1] - want[3]) <= 1e-10 * abs(want[3])


@pytest.mark.parametrize("sweeps", ["merged", "separate"])
@pytest.mark.parametrize("n", [2, 3, 40, 513])
def test_accel_vjp_mixed_small_and_ragged(orc, monkeypatch, n, sweeps):
    """Mixed contexts on the degenerate and ragged sizes (one star; two; a
    cluster one slot past a padded block): every cotangent against the
    oracle's exact one, within the single-precision pair sums' 1e-5 of the
    largest (the mixed adjoint's own tolerance on the adjoint workload)."""
    x, v, m = state(n, 900 + n)
    c, eps = 6.0, 1e-2
    abar = np.random.default_rng(n + 1).normal(size=(n, 3))
    want = oracle_vjp_accel(orc, x, v, m, abar, c, eps)
    if sweeps == "separate":
        monkeypatch.setenv("PN_ADJ_SEPARATE", "1")
    ctx = pn.pn_init(n, c=c, eps=eps, precision="mixed", device=0)
    monkeypatch.delenv("PN_ADJ_SEPARATE", raising=False)
    X, V, M, AB = dev(x), dev(v), dev(m), dev(abar)
    XB, VB = torch.empty_like(X), torch.empty_like(X)
    scal = pn.pn_accel_vjp(ctx, X, V, M, AB, XB, VB)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    assert np.abs(xb - want[0]).max() <= 1e-5 * np.abs(want[0]).max()
    assert np.abs(vb - want[1]).max() <= 1e-5 * max(np.abs(want[1]).max(), 1e-300)
    assert abs(scal[0, 0] - want[2]) <= 1e-5 * abs(want[2])
    assert abs(scal[0, 1] - want[3]) <= 1e-5 * abs(want[3])


def test_accel_vjp_larger_cluster_random_projections(orc):
    """n spanning several tiles and splits: check <xbar, u> + <vbar, w> + M_bar
    dM + c2_bar dc2 against abar . (directional derivative) for random
    directions."""
    x, v, m = make_cluster(1100, 0.1, 71)
    c, eps = 15.0, 1e-3
    rng = np.random.default_rng(9)
    abar = rng.normal(size=x.shape)
    ctx = pn.pn_init(1100, c=c, eps=eps, precision="fp64", device=0)
    XB, VB = torch.empty((1100, 3), dtype=torch.float64, device=DEV), torch.empty(
        (1100, 3), dtype=torch.float64, device=DEV)
    scal = pn.pn_accel_vjp(ctx, dev(x), dev(v), dev(m), dev(abar), XB, VB)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    for trial in range(3):
        u, w = rng.normal(size=x.shape), rng.normal(size=x.shape)
        dM, dc2 = rng.normal(), 1e-3 * rng.normal()
        lhs = np.sum(xb * u) + np.sum(vb * w) + scal[0, 0] * dM + scal[0, 1] * dc2
        rhs = np.sum(abar * orc.accel_jvp(x, v, m, u, w, dM, dc2, c=c, eps=eps))
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("sweeps", ["merged", "separate"])
def test_accel_vjp_mixed_context(orc, sweeps, monkeypatch):
    """Mixed contexts run the reverse pair sweeps in single precision (hi/lo
    positions), both in one pass over the pairs (merged) or, with
    PN_ADJ_SEPARATE, one pass per side: the VJP stays within 1e-5 of the
    oracle's exact one along random directions, and per body within median
    1e-6 / max 1e-4 of the oracle's exact cotangents (20 sampled bodies, the
    hole and a star near it among them, all six components, each from the
    oracle's complex-step derivative along that unit direction)."""
    x, v, m = make_cluster(700, 0.1, 73)
    x[3] = x[0] + np.array([0.004, 0.001, 0.0])        # a star close to the hole
    c, eps = 15.0, 1e-3
    rng = np.random.default_rng(19)
    abar = rng.normal(size=x.shape)
    if sweeps == "separate":
        monkeypatch.setenv("PN_ADJ_SEPARATE", "1")
    ctx = pn.pn_init(700, c=c, eps=eps, precision="mixed", device=0)
    monkeypatch.delenv("PN_ADJ_SEPARATE", raising=False)
    XB, VB = torch.empty((700, 3), dtype=torch.float64, device=DEV), torch.empty(
        (700, 3), dtype=torch.float64, device=DEV)
    scal = pn.pn_accel_vjp(ctx, dev(x), dev(v), dev(m), dev(abar), XB, VB)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    for trial in range(3):
        u, w = rng.normal(size=x.shape), rng.normal(size=x.shape)
        dM, dc2 = rng.normal(), 1e-3 * rng.normal()
        lhs = np.sum(xb * u) + np.sum(vb * w) + scal[0, 0] * dM + scal[0, 1] * dc2
        rhs = np.sum(abar * orc.accel_jvp(x, v, m, u, w, dM, dc2, c=c, eps=eps))
        assert abs(lhs - rhs) <= 1e-5 * abs(rhs), (lhs, rhs)
    # per-body cotangents against the oracle's exact ones
    bodies = [0, 3] + list(rng.choice(np.arange(4, 700), 18, replace=False))
    z = np.zeros_like(x)
    xw, vw = np.zeros((len(bodies), 3)), np.zeros((len(bodies), 3))
    for q, i in enumerate(bodies):
        for k in range(3):
            e = np.zeros_like(x)
            e[i, k] = 1.0
            xw[q, k] = np.sum(abar * orc.accel_jvp(x, v, m, e, z, c=c, eps=eps))
            vw[q, k] = np.sum(abar * orc.accel_jvp(x, v, m, z, e, c=c, eps=eps))
    # the hole's velocity never enters A (it is eliminated through the
    # zero-momentum frame): its cotangent is exactly zero on both sides
    assert not np.any(vw[0]) and not np.any(vb[0])
    for got, want in ((xb[bodies], xw), (vb[bodies][1:], vw[1:])):
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
        assert np.median(err) <= 1e-6 and err.max() <= 1e-4, (np.median(err), err.max())
    Mw = np.sum(abar * orc.accel_jvp(x, v, m, z, z, dM=1.0, c=c, eps=eps))
    cw = np.sum(abar * orc.accel_jvp(x, v, m, z, z, dinv_c2=1.0, c=c, eps=eps))
    assert abs(scal[0, 0] - Mw) <= 1e-6 * abs(Mw), (scal[0, 0], Mw)
    assert abs(scal[0, 1] - cw) <= 1e-6 * abs(cw), (scal[0, 1], cw)


def test_merged_and_separate_sweeps_agree(monkeypatch):
    """The merged reverse sweep and the two separate ones add the same FP32
    pair terms in different orders: on a 3000-body cluster (12 target
    blocks, several source splits, a star near the hole) their VJPs agree
    per body to median 1e-6 and max 5e-5 of the cotangent's norm (FP32 sums
    of thousands of terms, some cancelling), and M, 1/c^2 within 1e-6."""
    n = 3000
    x, v, m = make_cluster(n, 0.1, 5)
    x[7] = x[0] + np.array([0.003, -0.002, 0.001])
    abar = np.random.default_rng(4).normal(size=x.shape)
    out = {}
    for sweeps in ("merged", "separate"):
        if sweeps == "separate":
            monkeypatch.setenv("PN_ADJ_SEPARATE", "1")
        ctx = pn.pn_init(n, c=15.0, eps=1e-3, precision="mixed", device=0)
        monkeypatch.delenv("PN_ADJ_SEPARATE", raising=False)
        XB = torch.empty((n, 3), dtype=torch.float64, device=DEV)
        VB = torch.empty((n, 3), dtype=torch.float64, device=DEV)
        scal = pn.pn_accel_vjp(ctx, dev(x), dev(v), dev(m), dev(abar), XB, VB)
        ctx.close()
        out[sweeps] = (XB.cpu().numpy(), VB.cpu().numpy(), scal)
    (xa, va, sa), (xs, vs, ss) = out["merged"], out["separate"]
    for a, b in ((xa, xs), (va[1:], vs[1:])):
        err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
        assert np.median(err) <= 1e-6 and err.max() <= 5e-5, (np.median(err), err.max())
    assert np.all(np.abs(sa - ss) <= 1e-6 * np.abs(ss)), (sa, ss)


def oracle_step_grad(orc, x, v, m, dt, nst, xbT, vbT, c, eps, vel_mode=0):
    n = len(m)
    gx, gv = np.zeros((n, 3)), np.zeros((n, 3))
    z = np.zeros((n, 3))

    def proj(dx, dv, dM=0.0, dc2=0.0):
        _, _, jx, jv = orc.traj_jvp(x, v, m, dt, nst, dx, dv, dM, dc2, c=c, eps=eps,
                                    vel_mode=vel_mode)
        return np.sum(xbT * jx) + np.sum(vbT * jv)

    for i in range(n):
        for k in range(3):
            e = np.zeros((n, 3))
            e[i, k] = 1.0
            gx[i, k] = proj(e, z)
            gv[i, k] = proj(z, e)
    return gx, gv, proj(z, z, dM=1.0), proj(z, z, dc2=1.0)


@pytest.mark.parametrize("vel_mode,checkpoint", [("vpred_end", 4), ("vpred_end", 0),
                                                 ("vhalf", 3)])
def test_step_vjp_matches_oracle(orc, vel_mode, checkpoint):
    n, nst, dt = 12, 10, 1.0 / 128
    x, v, m = state(n, 800)
    c, eps = 6.0, 1e-2
    rng = np.random.default_rng(11)
    xbT, vbT = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    want = oracle_step_grad(orc, x, v, m, dt, nst, xbT, vbT, c, eps,
                            vel_mode=0 if vel_mode == "vpred_end" else 1)
    ctx = pn.pn_init(n, c=c, eps=eps, precision="fp64", vel_mode=vel_mode, device=0)
    XB, VB = torch.empty((n, 3), dtype=torch.float64, device=DEV), torch.empty(
        (n, 3), dtype=torch.float64, device=DEV)
    scal = pn.pn_step_vjp(ctx, dev(x), dev(v), dev(m), dt, nst, dev(xbT), dev(vbT), XB, VB,
                          checkpoint=checkpoint)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    assert np.abs(xb - want[0]).max() <= 1e-9 * np.abs(want[0]).max()
    assert np.abs(vb - want[1]).max() <= 1e-9 * np.abs(want[1]).max()
    assert abs(scal[0, 0] - want[2]) <= 1e-9 * abs(want[2])
    assert abs(scal[0, 1] - want[3]) <= 1e-9 * abs(want[3])


def test_step_vjp_mixed_trajectory(orc):
    """Mixed-precision forward trajectory, FP64 derivatives: the gradient
    differs from the FP64 one by the trajectory's rounding only."""
    n, nst, dt = 300, 8, 1.0 / 256
    x, v, m = make_cluster(n, 0.1, 81)
    c, eps = 20.0, 1e-3
    rng = np.random.default_rng(13)
    xbT, vbT = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = pn.pn_init(n, c=c, eps=eps, precision=prec, device=0)
        XB, VB = torch.empty((n, 3), dtype=torch.float64, device=DEV), torch.empty(
            (n, 3), dtype=torch.float64, device=DEV)
        scal = pn.pn_step_vjp(ctx, dev(x), dev(v), dev(m), dt, nst, dev(xbT), dev(vbT), XB, VB)
        out[prec] = XB.cpu().numpy(), VB.cpu().numpy(), scal
        ctx.close()
    (x64, v64, s64), (xm, vm, sm) = out["fp64"], out["mixed"]
    assert np.abs(xm - x64).max() <= 1e-5 * np.abs(x64).max()
    assert np.abs(vm - v64).max() <= 1e-5 * np.abs(v64).max()
    assert abs(sm[0, 0] - s64[0, 0]) <= 1e-5 * abs(s64[0, 0])
    # and the FP64 one agrees with the oracle along random directions
    for trial in range(2):
        u, w = rng.normal(size=x.shape), rng.normal(size=x.shape)
        _, _, jx, jv = orc.traj_jvp(x, v, m, dt, nst, u, w, c=c, eps=eps)
        rhs = np.sum(xbT * jx) + np.sum(vbT * jv)
        lhs = np.sum(x64 * u) + np.sum(v64 * w)
        assert abs(lhs - rhs) <= 1e-8 * abs(rhs)
    # the mixed gradient per body against the oracle's exact derivative of
    # the trajectory (complex step) along each unit direction: 12 bodies, the
    # hole among them, all six components
    bodies = [0] + list(rng.choice(np.arange(1, n), 11, replace=False))
    z = np.zeros_like(x)
    xw, vw = np.zeros((len(bodies), 3)), np.zeros((len(bodies), 3))
    for q, i in enumerate(bodies):
        for k in range(3):
            e = np.zeros_like(x)
            e[i, k] = 1.0
            _, _, jx, jv = orc.traj_jvp(x, v, m, dt, nst, e, z, c=c, eps=eps)
            xw[q, k] = np.sum(xbT * jx) + np.sum(vbT * jv)
            _, _, jx, jv = orc.traj_jvp(x, v, m, dt, nst, z, e, c=c, eps=eps)
            vw[q, k] = np.sum(xbT * jx) + np.sum(vbT * jv)
    for got, want in ((xm[bodies], xw), (vm[bodies], vw)):
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
        assert np.median(err) <= 1e-6 and err.max() <= 1e-4, (np.median(err), err.max())


def test_autograd_trajectory_loss_of_the_nearest_stars():
    """The differentiable trajectory (forward pn_step, backward pn_step_vjp)
    on the adjoint workload's loss, sum over the 16 stars nearest the hole of
    |x(T)|^2, against central differences of the FP64 path in M and c."""
    n, nst, dt = 2048, 40, 1.0 / 2048
    x, v, m = make_cluster(n, 0.1, 91)
    near = np.argsort(np.linalg.norm(x[1:] - x[0], axis=1))[:16] + 1
    idx = torch.tensor(near, device=DEV)
    ctx = pn.pn_init(n, c=50.0, eps=1e-4, precision="fp64", device=0)
    X0 = dev(x).requires_grad_(True)
    V0 = dev(v).requires_grad_(True)
    Mt = torch.tensor(0.1, dtype=torch.float64, device=DEV, requires_grad=True)
    ct = torch.tensor(50.0, dtype=torch.float64, device=DEV, requires_grad=True)
    M = dev(m)
    xT, vT = pn.trajectory(ctx, X0, V0, M, Mt, ct, dt, nst)
    loss = (xT[idx] ** 2).sum()
    loss.backward()

    def L(Mv, cv, dx=None):
        mm = m.copy()
        mm[0] = Mv
        xx = x.copy() if dx is None else x + dx
        with torch.no_grad():
            xt, _ = pn.trajectory(ctx, dev(xx), dev(v), dev(mm),
                                  torch.tensor(Mv, dtype=torch.float64),
                                  torch.tensor(cv, dtype=torch.float64), dt, nst)
        return float((xt[idx] ** 2).sum())

    h = 1e-6
    gM = (L(0.1 + h, 50.0) - L(0.1 - h, 50.0)) / (2 * h)
    gc = (L(0.1, 50.0 + h * 50) - L(0.1, 50.0 - h * 50)) / (2 * h * 50)
    assert abs(Mt.grad.item() - gM) <= 1e-5 * abs(gM), (Mt.grad.item(), gM)
    assert abs(ct.grad.item() - gc) <= 1e-4 * abs(gc) + 1e-12, (ct.grad.item(), gc)
    j = int(near[0])
    e = np.zeros_like(x)
    e[j, 0] = h
    gx = (L(0.1, 50.0, e) - L(0.1, 50.0, -e)) / (2 * h)
    assert abs(X0.grad[j, 0].item() - gx) <= 1e-5 * abs(gx), (X0.grad[j, 0].item(), gx)
    ctx.close()


def test_adjoint_workload_gradients_match_central_differences():
    """The adjoint workload (N = 8192 Plummer, M = 0.1, c = 50, dt = 1/2048,
    FP64 states, single-precision pair sums), 200 steps with sqrt(T)
    checkpoints: dL/dM, dL/dc and the largest components of dL/dx0 and
    dL/dv0 (of tagged and of untagged stars) against FP64 central
    differences, and the mixed gradient against the FP64 one over every
    component.  The same check as the bench's adjoint line (1000 steps).

    A difference carries the perturbed runs' FP64 rounding (a few 1e-9
    absolute here), which only the larger components (M, c, the tagged
    stars') dwarf: there both gradients match it within 1e-6.  Everywhere
    the mixed gradient is within 1e-6 of the FP64 one, and no further from
    the difference than the FP64 gradient (which equals the oracle's exact
    derivatives on small systems) plus 1e-6."""
    import bench
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer8k_adjoint"]
    state = w.state()
    x = state[0]
    near = np.argsort(np.linalg.norm(x[1:] - x[0], axis=1))[:16] + 1
    stream = torch.cuda.current_stream(DEV)
    nst = 200
    gm = bench.adjoint_gradient(0, stream, w, state, near, nst, "mixed", from_x0=True)[:4]
    g6 = bench.adjoint_gradient(0, stream, w, state, near, nst, "fp64")[:4]
    assert np.linalg.norm(gm[0] - g6[0]) <= 1e-6 * np.linalg.norm(g6[0])
    assert np.linalg.norm(gm[1] - g6[1]) <= 1e-6 * np.linalg.norm(g6[1])
    out = bench.adjoint_fd_check(0, stream, nst, {"mixed": gm, "fp64": g6}, near)
    assert out["fd_dL_dM_h_vs_2h_rel"] <= 1e-7, out["fd_dL_dM_h_vs_2h_rel"]
    for c in out["checks"]:
        fd = abs(c["central_difference"])
        assert c["rel_mixed_vs_fp64"] <= 1e-6, c
        assert abs(c["mixed"] - c["central_difference"]) <= \
            1e-6 * fd + abs(c["fp64"] - c["central_difference"]), c
        if c["param"] in ("M", "c") or c["tagged"]:
            assert c["rel_err_mixed"] <= 1e-6 and c["rel_err_fp64"] <= 1e-6, c


def test_error_paths():
    x, v, m = state(40, 900)
    X, V, M = dev(x), dev(v), dev(m)
    XB, VB = torch.empty_like(X), torch.empty_like(X)
    ctx = pn.pn_init(40, c=10.0, eps=1e-2, precision="fp64", integrator="rk4", device=0)
    with pytest.raises(pn.PNError) as e:
        pn.pn_step_vjp(ctx, X, V, M, 1e-3, 3, XB, VB, XB.clone(), VB.clone())
    assert "PN_EUNSUPPORTED" in str(e.value)
    with pytest.raises(pn.PNError) as e:
        pn.pn_accel_vjp(ctx, X, V, M, X, X, VB)           # xbar aliases x
    assert "PN_EINVAL" in str(e.value)
    with pytest.raises(pn.PNError) as e:
        pn.pn_jerk(ctx, X, V, M, XB, XB)                  # a aliases jerk
    assert "PN_EINVAL" in str(e.value)
    ctx.close()
    # zero steps: the gradient of the entry state is the cotangent itself
    # plus the entry acceleration's (zero) contribution
    ctx = pn.pn_init(40, c=10.0, eps=1e-2, precision="fp64", device=0)
    xbT, vbT = dev(np.ones((40, 3))), dev(2 * np.ones((40, 3)))
    scal = pn.pn_step_vjp(ctx, X, V, M, 1e-3, 0, xbT, vbT, XB, VB)
    assert torch.equal(XB, xbT) and torch.equal(VB, vbT)
    assert np.all(scal == 0.0)
    ctx.close()


def test_step_vjp_batched_per_cluster(orc):
    """Batched context: one pn_step_vjp over three clusters with their own c
    and eps; each cluster's gradient (positions, velocities, its hole mass and
    1/c^2) equals the oracle's for that cluster alone."""
    sizes, cs, es = [9, 14, 6], [6.0, 9.0, 15.0], [1e-2, 2e-2, 5e-3]
    parts = [state(n, 950 + k, m_bh=0.2 + 0.1 * k) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    x = np.concatenate([p[0] for p in parts])
    v = np.concatenate([p[1] for p in parts])
    m = np.concatenate([p[2] for p in parts])
    n, nst, dt = off[-1], 6, 1.0 / 128
    rng = np.random.default_rng(23)
    xbT, vbT = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    ctx = pn.pn_init_batched(off, c=cs, eps=es, precision="fp64", device=0)
    XB, VB = torch.empty((n, 3), dtype=torch.float64, device=DEV), torch.empty(
        (n, 3), dtype=torch.float64, device=DEV)
    scal = pn.pn_step_vjp(ctx, dev(x), dev(v), dev(m), dt, nst, dev(xbT), dev(vbT), XB, VB,
                          checkpoint=4)
    ctx.close()
    xb, vb = XB.cpu().numpy(), VB.cpu().numpy()
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        want = oracle_step_grad(orc, x[a:b], v[a:b], m[a:b], dt, nst, xbT[a:b], vbT[a:b], cs[k],
                                es[k])
        assert np.abs(xb[a:b] - want[0]).max() <= 1e-9 * np.abs(want[0]).max()
        assert np.abs(vb[a:b] - want[1]).max() <= 1e-9 * np.abs(want[1]).max()
        assert abs(scal[k, 0] - want[2]) <= 1e-9 * abs(want[2])
        assert abs(scal[k, 1] - want[3]) <= 1e-9 * abs(want[3])


@pytest.mark.parametrize("vel_mode,checkpoint", [("vpred_end", 0), ("vhalf", 3)])
def test_saved_checkpoints_give_the_same_trajectory_and_gradient(vel_mode, checkpoint):
    """pn_step_save runs the same trajectory as pn_step, and the backward from
    its checkpoints (pn_step_vjp_saved) equals pn_step_vjp's from the same
    start state, bit for bit, in a batched mixed context."""
    sizes = [700, 300]
    parts = [make_cluster(n, 0.1 + 0.05 * k, 40 + k) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    x = np.concatenate([p[0] for p in parts])
    v = np.concatenate([p[1] for p in parts])
    m = np.concatenate([p[2] for p in parts])
    n, nst, dt = int(off[-1]), 11, 1.0 / 1024
    ctx = pn.pn_init_batched(off, c=[20.0, 35.0], eps=1e-3, precision="mixed",
                             vel_mode=vel_mode, device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    X2, V2, A2 = X.clone(), V.clone(), A.clone()
    ckpt = pn.pn_step_save(ctx, X, V, M, A, dt, nst, checkpoint)
    pn.pn_step(ctx, X2, V2, M, A2, dt, nst)
    pn.pn_sync(ctx)
    assert torch.equal(X, X2) and torch.equal(V, V2) and torch.equal(A, A2)
    rng = np.random.default_rng(3)
    xbT, vbT = dev(rng.normal(size=(n, 3))), dev(rng.normal(size=(n, 3)))
    XB, VB, XB2, VB2 = (torch.empty((n, 3), dtype=torch.float64, device=DEV) for _ in range(4))
    s1 = pn.pn_step_vjp_saved(ctx, ckpt, M, dt, nst, xbT, vbT, XB, VB, checkpoint)
    s2 = pn.pn_step_vjp(ctx, dev(x), dev(v), M, dt, nst, xbT, vbT, XB2, VB2, checkpoint)
    assert torch.equal(XB, XB2) and torch.equal(VB, VB2) and np.array_equal(s1, s2)
    ctx.close()


def test_saved_checkpoints_edge_cases():
    x, v, m = state(40, 901)
    X, V, M = dev(x), dev(v), dev(m)
    XB, VB = torch.empty_like(X), torch.empty_like(X)
    ctx = pn.pn_init(40, c=10.0, eps=1e-2, precision="fp64", device=0)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    # no steps: the cotangents pass through, nothing else contributes
    ckpt = pn.pn_step_save(ctx, X, V, M, A, 1e-3, 0)
    xbT, vbT = dev(np.ones((40, 3))), dev(2 * np.ones((40, 3)))
    scal = pn.pn_step_vjp_saved(ctx, ckpt, M, 1e-3, 0, xbT, vbT, XB, VB)
    assert torch.equal(XB, xbT) and torch.equal(VB, vbT) and np.all(scal == 0.0)
    lib = pn._load()
    assert lib.pn_step_save(ctx.handle, X.data_ptr(), V.data_ptr(), M.data_ptr(), A.data_ptr(),
                            1e-3, 4, 0, None) == pn.PN_EINVAL
    assert lib.pn_step_vjp_saved(ctx.handle, None, M.data_ptr(), 1e-3, 4, 0, xbT.data_ptr(),
                                 vbT.data_ptr(), XB.data_ptr(), VB.data_ptr(),
                                 np.zeros(2).ctypes.data) == pn.PN_EINVAL
    ctx.close()
    ctx = pn.pn_init(40, c=10.0, eps=1e-2, precision="fp64", integrator="rk4", device=0)
    with pytest.raises(pn.PNError) as e:
        pn.pn_step_save(ctx, X, V, M, A, 1e-3, 3)
    assert e.value.status == pn.PN_EUNSUPPORTED
    ctx.close()
