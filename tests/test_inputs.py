"""The seeded input generator: published test vectors and distribution facts."""
import math
import os

import numpy as np

from paper_1801_07986_b300.inputs import (WORKLOADS, SplitMix64, batched_workloads,
                                          make_cluster, splitmix64_scalar)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    s, got = 1234567, []
    for _ in want:
        s, o = splitmix64_scalar(s)
        got.append(o)
    assert got == want
    assert [int(u) for u in SplitMix64(1234567).next_u64(len(want))] == want


def test_stream_blocks_concatenate():
    a = SplitMix64(99)
    b = SplitMix64(99)
    u = np.concatenate([a.uniform(7), a.uniform(13)])
    assert np.array_equal(u, b.uniform(20))
    assert u.min() >= 0.0 and u.max() < 1.0


def _plummer_half_mass_radius(rmax):
    # M(<r) = r^3 (1 + r^2)^(-3/2); the sample is truncated at rmax
    mcut = rmax ** 3 / (1 + rmax * rmax) ** 1.5
    lo, hi = 0.0, rmax
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid ** 3 / (1 + mid * mid) ** 1.5 < 0.5 * mcut:
            lo = mid
        else:
            hi = mid
    return lo


def test_plummer_shape():
    x, v, m = make_cluster(32769, 0.1, 1234)
    assert x.shape == (32769, 3) and v.shape == (32769, 3) and m.shape == (32769,)
    assert np.all(x[0] == 0) and np.all(v[0] == 0) and m[0] == 0.1
    assert math.isclose(m[1:].sum(), 1.0, rel_tol=1e-12)
    r = np.linalg.norm(x[1:], axis=1)
    assert r.max() <= 10.0 + 1e-9
    assert abs(np.median(r) / _plummer_half_mass_radius(10.0) - 1) < 0.03
    # kinetic energy of an isotropic Plummer sphere: 3 pi G M^2 / (64 a)
    ke = 0.5 * (m[1:] * (v[1:] ** 2).sum(1)).sum()
    assert abs(ke / (3 * math.pi / 64) - 1) < 0.05
    np.testing.assert_allclose((m[1:, None] * v[1:]).sum(0), 0.0, atol=1e-15)
    # velocities stay below the local escape speed
    assert np.all((v[1:] ** 2).sum(1) <= 2.0 / np.sqrt(1 + r * r) * (1 + 1e-9) + 1e-3)


def test_eccentric_population():
    w = WORKLOADS["plummer128k_ecc"]
    x, v, m = w.state()
    n_ecc = int(round(w.ecc_frac * (w.n - 1)))
    assert n_ecc == 1311
    mu = w.m_bh + m[1]
    d, u = x[1:1 + n_ecc], v[1:1 + n_ecc]
    r = np.linalg.norm(d, axis=1)
    a = 1.0 / (2.0 / r - (u * u).sum(1) / mu)
    h = np.cross(d, u)
    evec = np.cross(u, h) / mu - d / r[:, None]
    e = np.linalg.norm(evec, axis=1)
    np.testing.assert_allclose(a, 1e-3, rtol=1e-2)
    np.testing.assert_allclose(e, 0.9, atol=2e-3)
    assert r.min() >= 0.9 * 1e-4 and r.max() <= 1.1 * 1.9e-3


def test_workloads_are_deterministic():
    x1, v1, _ = WORKLOADS["plummer1k_fp64"].state()
    x2, v2, _ = WORKLOADS["plummer1k_fp64"].state()
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    ws = batched_workloads()
    assert len(ws) == 64
    ns = np.array([w.n for w in ws])
    assert ns.min() >= 512 and ns.max() <= 32768
    assert all(0.01 <= w.m_bh <= 0.2 and 20 <= w.c <= 200 for w in ws)
