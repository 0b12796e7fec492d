"""GPU (libpn, through the C ABI) vs the FP64 CPU oracle, element by element.

Tolerances (relative force error |a_gpu - a_oracle| / |a_oracle| per body):
  FP64 mode   <= 1e-12 for every body;
  mixed mode  <= 2e-7 median and <= 1e-5 max over all bodies.
Sizes span several 256-star blocks and ragged tails; the 16k and 128k
Plummer workloads are checked on sampled targets in the launch shape the
benchmark uses.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1801_07986_b300 import pn  # noqa: E402
from paper_1801_07986_b300.inputs import WORKLOADS, make_cluster  # noqa: E402

DEV = torch.device("cuda:0")
FP64_TOL = 1e-12
MIX_MED, MIX_MAX = 2e-7, 1e-5


def cluster(n, m_bh, seed):
    """make_cluster, except that tiny systems get random positions (a
    one-star cluster recentred on its own mass would sit on the hole)."""
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


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def gpu_accel(x, v, m, precision, G=1.0, c=math.inf, eps=0.0, vel_mode="vpred_end",
              pair_kernel="fused"):
    n = m.shape[0]
    ctx = pn.pn_init(n, G=G, c=c, eps=eps, precision=precision, vel_mode=vel_mode, device=0,
                     pair_kernel=pair_kernel)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    out = A.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("n", [2, 3, 33, 257, 300, 1024])
def test_fp64_matches_oracle(orc, n):
    x, v, m = cluster(n, 0.1, 100 + n)
    for c in (100.0, 5.0):
        want = orc.accel(x, v, m, c=c, eps=1e-4)
        got = gpu_accel(x, v, m, "fp64", c=c, eps=1e-4)
        err = rel(got, want)
        assert err.max() <= FP64_TOL, (c, err.max(), int(err.argmax()))


PAIR_KERNELS = ["fused", "two_pass"]


@pytest.mark.parametrize("pair_kernel", PAIR_KERNELS + ["fused_spatial"])
@pytest.mark.parametrize("n", [2, 3, 300, 1024, 4097])
def test_mixed_matches_oracle(orc, monkeypatch, n, pair_kernel):
    """fused_spatial: the fused kernel with the spatial order forced on (its
    sort blocks and tile boxes mostly padding at the smallest sizes)."""
    monkeypatch.setenv("PN_SPATIAL", "1" if pair_kernel == "fused_spatial" else "0")
    pair_kernel = pair_kernel.replace("_spatial", "")
    x, v, m = cluster(n, 0.1, 200 + n)
    want = orc.accel(x, v, m, c=20.0, eps=1e-4)
    got = gpu_accel(x, v, m, "mixed", c=20.0, eps=1e-4, pair_kernel=pair_kernel)
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


# fused-kernel variants (PN_FUSED_PACKED, PN_FUSED_TARGETS, PN_FUSED_UNROLL are
# read by pn_init): the packed FP32x2 kernel and every scalar shape
FUSED_VARIANTS = [("1", "4", "1"), ("1", "4", "2"), ("1", "2", "1"), ("1", "2", "2"),
                  ("1s", "4", "1"), ("1s", "4", "2"), ("1s", "2", "1"), ("1s", "2", "2"),
                  ("0", "4", "1"), ("0", "4", "2"),
                  ("0", "4", "3"), ("0", "4", "4"), ("0", "2", "1"), ("0", "2", "2"),
                  ("0", "2", "4"), ("0", "1", "1"), ("0", "1", "2")]


@pytest.mark.parametrize("packed,targets,unroll", FUSED_VARIANTS)
def test_fused_variants_match_oracle(orc, monkeypatch, packed, targets, unroll):
    """Every fused-kernel shape; "1s": the packed kernel on the spatial order."""
    monkeypatch.setenv("PN_SPATIAL", "1" if packed == "1s" else "0")
    packed = packed[0]
    monkeypatch.setenv("PN_FUSED_PACKED", packed)
    monkeypatch.setenv("PN_FUSED_TARGETS", targets)
    monkeypatch.setenv("PN_FUSED_UNROLL", unroll)
    n = 2 * 1024 + 130            # several target blocks and source tiles, ragged tail
    x, v, m = cluster(n, 0.2, 4242)
    x[5] = x[0] + np.array([0.01, 0.0, 0.0])     # a near source of the hole
    want = orc.accel(x, v, m, c=15.0, eps=1e-4)
    ctx = pn.pn_init(n, c=15.0, eps=1e-4, precision="mixed", device=0)
    shape = pn.pn_get_launch(ctx)
    assert shape["packed"] == (packed == "1")
    want_p = (2 if targets == "2" else 4) if packed == "1" else int(targets)
    assert shape["targets_per_thread"] == want_p
    var = pn.pn_get_variant(ctx)
    assert (var["targets_per_thread"], var["unroll"], var["packed"]) == \
        (want_p, int(unroll), int(packed == "1"))
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    ctx.close()
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


# the packed kernel's j-tile and buffer variants (PN_FUSED_TILE,
# PN_FUSED_STAGES): (spatial order, tile, buffers, targets per thread)
TILE_VARIANTS = [("0", 64, 4, "2"), ("0", 64, 4, "4"), ("0", 32, 8, "2"), ("0", 32, 8, "4"),
                 ("1", 64, 4, "2"), ("1", 64, 4, "4")]


@pytest.mark.parametrize("spatial,tile,stages,targets", TILE_VARIANTS)
def test_packed_tile_variants_match_oracle(orc, monkeypatch, spatial, tile, stages, targets):
    monkeypatch.setenv("PN_SPATIAL", spatial)
    monkeypatch.setenv("PN_FUSED_PACKED", "1")
    monkeypatch.setenv("PN_FUSED_TARGETS", targets)
    monkeypatch.setenv("PN_FUSED_TILE", str(tile))
    monkeypatch.setenv("PN_FUSED_STAGES", str(stages))
    n = 2 * 1024 + 130
    x, v, m = cluster(n, 0.2, 4343)
    x[5] = x[0] + np.array([0.01, 0.0, 0.0])
    want = orc.accel(x, v, m, c=15.0, eps=1e-4)
    ctx = pn.pn_init(n, c=15.0, eps=1e-4, precision="mixed", device=0)
    shape = pn.pn_get_launch(ctx)
    assert shape["packed"] and shape["tile"] == tile
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    ctx.close()
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


def test_default_variants():
    """The default fused-kernel instantiation: 2 targets per thread with the
    2-way unroll up to 16384 star slots per cluster, 4 targets without the
    unroll above; the law-of-cosines form, on the spatial order from 2^32
    slot pairs; nothing off the fused kernel (FP64, two-pass)."""
    def variant(n, **kw):
        ctx = pn.pn_init(n, c=15.0, eps=1e-4, device=0, **kw)
        try:
            return pn.pn_get_variant(ctx)
        finally:
            ctx.close()
    small = variant(8192, precision="mixed")
    assert (small["targets_per_thread"], small["unroll"], small["form"], small["tile"],
            small["stages"], small["packed"]) == (2, 2, 1, 64, 6, 1)
    mid = variant(20000, precision="mixed")
    assert (mid["targets_per_thread"], mid["unroll"], mid["form"]) == (4, 1, 1)
    big = variant(70000, precision="mixed")           # 70144^2 > 2^32 slot pairs
    assert (big["targets_per_thread"], big["unroll"], big["form"]) == (4, 1, 2)
    assert not any(variant(3000, precision="fp64").values())
    assert not any(variant(3000, precision="mixed", pair_kernel="two_pass").values())


def test_fp64_fused_equals_two_pass():
    """In FP64 the fused sweep and the two passes form the same sums in the
    same order: bitwise equal accelerations."""
    x, v, m = make_cluster(3000, 0.1, 62)
    a1 = gpu_accel(x, v, m, "fp64", c=30.0, eps=1e-4, pair_kernel="fused")
    a2 = gpu_accel(x, v, m, "fp64", c=30.0, eps=1e-4, pair_kernel="two_pass")
    assert np.array_equal(a1, a2)


def test_plummer1k_workload_fp64_every_body(orc):
    w = WORKLOADS["plummer1k_fp64"]
    x, v, m = w.state()
    want = orc.accel(x, v, m, G=w.G, c=w.c, eps=w.eps)
    got = gpu_accel(x, v, m, "fp64", G=w.G, c=w.c, eps=w.eps)
    assert rel(got, want).max() <= FP64_TOL


def test_newtonian_limit_and_linearity_in_inv_c2(orc):
    x, v, m = make_cluster(700, 0.2, 31)
    eps = 1e-3
    a_inf = gpu_accel(x, v, m, "fp64", c=math.inf, eps=eps)
    assert rel(a_inf, orc.newton_accel(x, m, eps=eps)).max() <= FP64_TOL
    d1 = (gpu_accel(x, v, m, "fp64", c=20.0, eps=eps) - a_inf) * 400.0
    d2 = (gpu_accel(x, v, m, "fp64", c=7.0, eps=eps) - a_inf) * 49.0
    assert rel(d1, d2).max() < 1e-8
    # the 1PN part alone agrees with the oracle's 1PN part
    o1 = (orc.accel(x, v, m, c=20.0, eps=eps) - orc.accel(x, v, m, c=math.inf, eps=eps)) * 400.0
    assert rel(d1, o1).max() < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [2, 3])
def test_energy_smallest_systems(orc, precision, n):
    """The hole and one or two stars (a single tile, padding slots only
    otherwise) with a moving hole: every result within 1e-12 of the oracle."""
    rng = np.random.default_rng(n)
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3)) * 0.3
    m = np.full(n, 0.05)
    m[0] = 0.5
    want = orc.energy(x, v, m, c=8.0, eps=1e-3)
    ctx = pn.pn_init(n, c=8.0, eps=1e-3, precision=precision, device=0)
    got = pn.pn_energy(ctx, dev(x), dev(v), dev(m))
    ctx.close()
    for k in ("E_N", "E_PN"):
        assert abs(got[k] - want[k]) <= 1e-12 * abs(want[k]), k
    pscale = float(np.sum(m[:, None] * np.abs(v)))
    for k in ("P_N", "P_PN"):
        assert np.abs(got[k] - want[k]).max() <= 1e-12 * pscale, k


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-12)])
def test_energy_matches_oracle(orc, precision, tol):
    x, v, m = make_cluster(513, 0.1, 41)
    v = v.copy()
    v[0] = [0.01, -0.02, 0.005]          # a moving hole exercises the v_1 terms
    c, eps = 10.0, 1e-3
    want = orc.energy(x, v, m, c=c, eps=eps)
    ctx = pn.pn_init(513, c=c, eps=eps, precision=precision, device=0)
    got = pn.pn_energy(ctx, dev(x), dev(v), dev(m))
    ctx.close()
    for k in ("E_N", "E_PN"):
        assert abs(got[k] - want[k]) <= tol * abs(want[k]), k
    pscale = float(np.sum(m[:, None] * np.abs(v)))
    for k in ("P_N", "P_PN"):
        assert np.abs(got[k] - want[k]).max() <= tol * pscale, k


def test_energy_double_single_matches_fp64_on_16k(orc):
    """Mixed contexts take the energy's pair sums in double-single arithmetic
    on the FP32 pipe: on the 16k workload (a moving hole, 28 source splits)
    E_N, E_PN and both momenta agree with the FP64 context's to 1e-12, and
    with the oracle's on a 3000-body cluster."""
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    v = v.copy()
    v[0] = [0.01, -0.02, 0.005]
    got = {}
    for precision in ("mixed", "fp64"):
        ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=0)
        got[precision] = pn.pn_energy(ctx, dev(x), dev(v), dev(m))
        ctx.close()
    pscale = float(np.sum(m[:, None] * np.abs(v)))
    for k in ("E_N", "E_PN"):
        assert abs(got["mixed"][k] - got["fp64"][k]) <= 1e-12 * abs(got["fp64"][k]), k
    for k in ("P_N", "P_PN"):
        assert np.abs(got["mixed"][k] - got["fp64"][k]).max() <= 1e-12 * pscale, k
    x, v, m = make_cluster(3000, 0.1, 77)
    v = v.copy()
    v[0] = [-0.01, 0.003, 0.02]
    want = orc.energy(x, v, m, c=20.0, eps=1e-3)
    ctx = pn.pn_init(3000, c=20.0, eps=1e-3, precision="mixed", device=0)
    g = pn.pn_energy(ctx, dev(x), dev(v), dev(m))
    ctx.close()
    for k in ("E_N", "E_PN"):
        assert abs(g[k] - want[k]) <= 1e-12 * abs(want[k]), k
    pscale = float(np.sum(m[:, None] * np.abs(v)))
    for k in ("P_N", "P_PN"):
        assert np.abs(g[k] - want[k]).max() <= 1e-12 * pscale, k


@pytest.mark.parametrize("vel_mode,mode_id", [("vpred_end", 0), ("vhalf", 1)])
def test_steps_fp64_match_oracle(orc, vel_mode, mode_id):
    """20 KDK steps of the 1k workload: same trajectory to round-off, and at
    the final state the force equals the oracle's on the GPU's own state."""
    w = WORKLOADS["plummer1k_fp64"]
    x, v, m = w.state()
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision="fp64", vel_mode=vel_mode, device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    a0 = orc.accel(x, v, m, G=w.G, c=w.c, eps=w.eps)
    pn.pn_step(ctx, X, V, M, A, w.dt, 20)
    pn.pn_sync(ctx)
    xo, vo, ao = orc.step(x, v, m, a0, w.dt, 20, G=w.G, c=w.c, eps=w.eps, vel_mode=mode_id)
    xg, vg, ag = X.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()
    assert np.abs(xg - xo).max() < 1e-12
    assert np.abs(vg - vo).max() < 1e-11 * np.abs(vo).max()
    assert rel(ag, ao).max() < 1e-9
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rk4_steps_match_oracle(orc, precision):
    """The paper's own integrator (RK4, Section 4): 10 steps of the 1k
    workload against the oracle's RK4."""
    w = WORKLOADS["plummer1k_fp64"]
    x, v, m = w.state()
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, integrator="rk4",
                     device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    a0 = orc.accel(x, v, m, G=w.G, c=w.c, eps=w.eps)
    pn.pn_step(ctx, X, V, M, A, w.dt, 10)
    pn.pn_sync(ctx)
    xo, vo, ao = orc.rk4_step(x, v, m, a0, w.dt, 10, G=w.G, c=w.c, eps=w.eps)
    xg, vg, ag = X.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()
    if precision == "fp64":
        assert np.abs(xg - xo).max() < 1e-12
        assert rel(ag, ao).max() < 1e-9
    else:
        # single-precision pair sums: the state drifts by ~dt^2 * 1e-7 |a| per step
        assert np.abs(xg - xo).max() < 1e-10
        err = rel(ag, ao)
        assert np.median(err) < 1e-6 and err.max() < 1e-4
    ctx.close()


def test_step_force_is_accel_at_predicted_velocity():
    """After one step, a equals pn_accel at (x_new, v_half + dt/2 a_old)."""
    x, v, m = make_cluster(1000, 0.1, 51)
    dt = 1.0 / 512
    ctx = pn.pn_init(1000, c=15.0, eps=1e-4, precision="fp64", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    a_old = A.clone()
    v_half = V + 0.5 * dt * a_old
    x_new = X + dt * v_half
    pn.pn_step(ctx, X, V, M, A, dt, 1)
    B = torch.empty_like(X)
    pn.pn_accel(ctx, x_new, v_half + 0.5 * dt * a_old, M, B)
    pn.pn_sync(ctx)
    assert rel(A.cpu().numpy(), B.cpu().numpy()).max() < 1e-13
    ctx.close()


@pytest.mark.parametrize("r_near", [0.05, 0.0])
def test_packed_forms_match_oracle(orc, r_near):
    """The packed kernel's two forms of the hole term of kappa_ij: with near
    sources split off (r_near > 0) the law-of-cosines form a (R_i^2 - r_ij^2)
    runs, without the split (r_near = 0) the dot-product form D_j.d_i.  Stars
    at 0.01 and 0.06 from the hole and a ragged tail."""
    n = 2 * 1024 + 130
    x, v, m = cluster(n, 0.2, 4343)
    x[5] = x[0] + np.array([0.01, 0.0, 0.0])
    x[9] = x[0] + np.array([0.0, -0.06, 0.0])
    want = orc.accel(x, v, m, c=15.0, eps=1e-4)
    ctx = pn.pn_init(n, c=15.0, eps=1e-4, precision="mixed", device=0, r_near=r_near)
    assert pn.pn_get_launch(ctx)["packed"] == 1
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    got = A.cpu().numpy()
    ctx.close()
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


@pytest.mark.parametrize("spatial,balance", [("1", "1"), ("1", "0"), ("0", "1")])
def test_spatial_order_with_tight_pairs(orc, monkeypatch, spatial, balance):
    """The packed kernel on Hilbert-ordered slots (PN_SPATIAL=1, the default
    for large systems; with cost-balanced workers or, PN_BALANCE=0, equal
    unit counts) or in slot order: tight pairs (separations 1e-4 .. 1e-3)
    planted at 1 to 6 from the hole, where the high parts alone would lose the
    separation, and stars near the hole; every body against the oracle."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    monkeypatch.setenv("PN_BALANCE", balance)
    n = 6 * 1024 + 77
    x, v, m = cluster(n, 0.3, 4444)
    rng = np.random.default_rng(44)
    for k in range(40):
        a, b = 10 + 2 * k, 11 + 2 * k
        u = rng.normal(size=3)
        x[a] = x[0] + u / np.linalg.norm(u) * rng.uniform(1.0, 6.0)
        w = rng.normal(size=3)
        x[b] = x[a] + w / np.linalg.norm(w) * 10.0 ** rng.uniform(-4.0, -3.0)
    x[100] = x[0] + np.array([0.003, 0.0, 0.0])
    x[101] = x[0] + np.array([0.0, 0.03, 0.0])
    want = orc.accel(x, v, m, c=25.0, eps=2e-5)
    got = gpu_accel(x, v, m, "mixed", c=25.0, eps=2e-5)
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


@pytest.mark.parametrize("spatial", ["1", "0"])
def test_pair_stats_count_the_units(monkeypatch, spatial):
    """pn_get_pair_stats: every (warp, tile) unit of the spatially ordered
    packed kernel is counted once per evaluation; none without the order."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    n = 6 * 1024 + 77
    x, v, m = cluster(n, 0.3, 4646)
    ctx = pn.pn_init(n, c=25.0, eps=2e-5, precision="mixed", device=0)
    shape = pn.pn_get_launch(ctx)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_set_timing(ctx, True)
    for _ in range(2):
        pn.pn_accel(ctx, X, V, M, A)
    far, allu = pn.pn_get_pair_stats(ctx)
    pn.pn_set_timing(ctx, False)
    ctx.close()
    ns_pad = (n - 1 + 511) // 512 * 512
    ti = shape["threads"] * shape["targets_per_thread"]
    warps = shape["threads"] // 32
    if spatial == "1":
        assert allu == 2 * warps * (ns_pad // ti) * (ns_pad // shape["tile"])
        assert 0 < far < allu
    else:
        assert far == 0 and allu == 0


def test_precision_switch_after_init(orc):
    """A context created in FP64 and switched to mixed by pn_set_params uses
    the mixed records (allocated at pn_init whatever the precision)."""
    n = 1500
    x, v, m = cluster(n, 0.1, 4545)
    want = orc.accel(x, v, m, c=30.0, eps=1e-4)
    ctx = pn.pn_init(n, c=30.0, eps=1e-4, precision="fp64", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    for prec, ok in (("fp64", lambda e: e.max() <= FP64_TOL),
                     ("mixed", lambda e: np.median(e) <= MIX_MED and e.max() <= MIX_MAX)):
        pn.pn_set_params(ctx, precision=prec)
        pn.pn_accel(ctx, X, V, M, A)
        pn.pn_sync(ctx)
        err = rel(A.cpu().numpy(), want)
        assert ok(err), (prec, np.median(err), err.max())
    ctx.close()


@pytest.mark.parametrize("precision,pair_kernel",
                         [("fp64", "two_pass"), ("mixed", "fused"), ("mixed", "two_pass")])
def test_plummer16k_sampled_targets_and_hole(orc, precision, pair_kernel):
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    got = gpu_accel(x, v, m, precision, G=w.G, c=w.c, eps=w.eps, pair_kernel=pair_kernel)
    rng = np.random.default_rng(5)
    targets = np.concatenate([[0, 1, w.n - 1], rng.choice(np.arange(2, w.n - 1), 300, replace=False)])
    want = orc.accel_rows(x, v, m, targets, G=w.G, c=w.c, eps=w.eps)
    err = rel(got[targets], want)
    if precision == "fp64":
        assert err.max() <= FP64_TOL, err.max()
    else:
        assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


@pytest.mark.parametrize("pair_kernel", PAIR_KERNELS)
def test_plummer128k_eccentric_sampled_targets(orc, pair_kernel):
    """The 128k workload with 1% of stars on e = 0.9 orbits about the hole:
    sampled targets (all kinds) against the oracle, mixed precision."""
    w = WORKLOADS["plummer128k_ecc"]
    x, v, m = w.state()
    got = gpu_accel(x, v, m, "mixed", G=w.G, c=w.c, eps=w.eps, pair_kernel=pair_kernel)
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(6)
    n_ecc = int(round(w.ecc_frac * (w.n - 1)))
    targets = np.concatenate([[1, n_ecc, n_ecc + 1, w.n - 1],
                              rng.choice(np.arange(2, n_ecc), 60, replace=False),
                              rng.choice(np.arange(n_ecc + 2, w.n - 1), 140, replace=False)])
    want = orc.accel_rows(x, v, m, targets, G=w.G, c=w.c, eps=w.eps)
    err = rel(got[targets], want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (np.median(err), err.max())


def test_plummer128k_newtonian_momentum_balance():
    """At c = inf the Newtonian pair forces cancel: sum_a m_a a_a = 0 up to
    single-precision pair round-off (a property that holds at any size)."""
    w = WORKLOADS["plummer128k_ecc"]
    x, v, m = w.state()
    a = gpu_accel(x, v, m, "mixed", G=w.G, c=math.inf, eps=w.eps)
    f = (m[:, None] * a).sum(0)
    scale = (m[:, None] * np.abs(a)).sum(0)
    assert np.all(np.abs(f) <= 1e-6 * scale)


@pytest.mark.parametrize("precision,pair_kernel,spatial",
                         [("fp64", "two_pass", "0"), ("mixed", "fused", "0"),
                          ("mixed", "fused", "1"), ("mixed", "two_pass", "0")])
def test_deterministic(monkeypatch, precision, pair_kernel, spatial):
    """Two contexts give bitwise equal accelerations; with the spatial order
    (sort, permutation and balanced worker boundaries decided by the
    positions alone) as without."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    x, v, m = make_cluster(3000, 0.1, 61)
    a1 = gpu_accel(x, v, m, precision, c=30.0, eps=1e-4, pair_kernel=pair_kernel)
    a2 = gpu_accel(x, v, m, precision, c=30.0, eps=1e-4, pair_kernel=pair_kernel)
    assert np.array_equal(a1, a2)


def test_translation_invariance_mixed(orc):
    x, v, m = make_cluster(2000, 0.1, 71)
    shift = np.array([1.0e3, -2.0e3, 5.0e2])
    got = gpu_accel(x + shift, v, m, "mixed", c=20.0, eps=1e-4)
    want = orc.accel(x, v, m, c=20.0, eps=1e-4)
    err = rel(got, want)
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX


@pytest.mark.parametrize("spatial,bad", [("0", "on_hole"), ("1", "on_hole"), ("1", "nan")])
def test_nonfinite_is_reported_and_cleared(monkeypatch, spatial, bad):
    """A star on the hole (r = 0) or at a NaN position gives non-finite
    accelerations, reported as PN_ENONFINITE; with the spatial order the NaN
    also reaches the sort keys and the tile boxes (in slot order otherwise)."""
    monkeypatch.setenv("PN_SPATIAL", spatial)
    x, v, m = make_cluster(300, 0.1, 81)
    x = x.copy()
    if bad == "on_hole":
        x[5] = x[0]                  # a star on top of the hole: r = 0
    else:
        x[5] = np.nan
    ctx = pn.pn_init(300, c=20.0, eps=1e-4, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    with pytest.raises(pn.PNError) as ei:
        pn.pn_sync(ctx)
    assert ei.value.status == pn.PN_ENONFINITE
    x2, _, _ = make_cluster(300, 0.1, 81)
    pn.pn_accel(ctx, dev(x2), V, M, A)
    pn.pn_sync(ctx)                  # flag was cleared
    ctx.close()


def test_tile_copy_timeout_is_reported_and_device_stays_usable(orc, monkeypatch):
    """The packed kernel's tile waits are bounded: with the test hook every
    tile barrier expects 16 bytes that no copy delivers, the waits give up
    after 1 s, and pn_sync reports PN_ETIMEOUT.  The device stays usable."""
    import time
    x, v, m = make_cluster(2048, 0.1, 83)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    monkeypatch.setenv("PN_INJECT_COPY_TIMEOUT", "1")
    ctx = pn.pn_init(2048, c=20.0, eps=1e-4, precision="mixed", device=0)
    monkeypatch.delenv("PN_INJECT_COPY_TIMEOUT")
    t0 = time.time()
    pn.pn_accel(ctx, X, V, M, A)
    with pytest.raises(pn.PNError) as ei:
        pn.pn_sync(ctx)
    assert ei.value.status == pn.PN_ETIMEOUT
    assert time.time() - t0 < 30.0
    ctx.close()
    ctx = pn.pn_init(2048, c=20.0, eps=1e-4, precision="mixed", device=0)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_sync(ctx)
    err = rel(A.cpu().numpy(), orc.accel(x, v, m, c=20.0, eps=1e-4))
    assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX
    ctx.close()


def test_step_host_equals_device_path():
    x, v, m = make_cluster(1500, 0.1, 91)
    dt = 1.0 / 1024
    ctx = pn.pn_init(1500, c=30.0, eps=1e-4, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    a_host = A.cpu().numpy().copy()
    xh, vh = x.copy(), v.copy()
    pn.pn_step(ctx, X, V, M, A, dt, 3)
    pn.pn_step_host(ctx, xh, vh, m.copy(), a_host, dt, 3)
    assert np.array_equal(X.cpu().numpy(), xh)
    assert np.array_equal(V.cpu().numpy(), vh)
    assert np.array_equal(A.cpu().numpy(), a_host)
    ctx.close()


def test_timing_counts_launches():
    x, v, m = make_cluster(2048, 0.1, 95)
    ctx = pn.pn_init(2048, c=30.0, eps=1e-4, precision="mixed", device=0)
    X, V, M = dev(x), dev(v), dev(m)
    A = torch.empty_like(X)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_set_timing(ctx, True)
    pn.pn_step(ctx, X, V, M, A, 1e-3, 70)    # more than the 64-entry event ring
    ms, nl = pn.pn_get_timing(ctx)
    assert list(nl) == [0, 70, 70] and np.all(ms[1:] > 0)     # fused pair kernel + near pass
    shape = pn.pn_get_launch(ctx)
    assert shape["sms"] > 0 and shape["jsplit"] >= 1
    pn.pn_set_timing(ctx, False)
    ctx.close()
