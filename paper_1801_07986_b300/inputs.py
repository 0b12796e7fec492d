"""Seeded synthetic initial conditions: one black hole plus a star cluster.

This module draws positions, velocities and masses and nothing else: it holds
none of the force law, the integrator or the energy.  It is the one module the
CUDA path and the FP64 CPU oracle share, so that both are fed bit-identical
inputs.

Layout of every state returned here (body 0 is the black hole, the paper's
body "#1" of Section 2; bodies 1..N-1 are stars):

* ``x``, ``v``: float64 arrays of shape (N, 3), row-major (x, y, z per body);
* ``m``: float64 array of shape (N,).

Generators used (all restated from their published definitions):

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): a 64-bit counter advanced by the golden-ratio
  increment and passed through a 64-bit finaliser.  Uniforms in [0, 1) take
  the top 53 bits.
* Plummer sphere by the inverse-cumulative-mass method of Aarseth, Henon &
  Wielen (A&A 37, 183, 1974): radius from M(<r)/M = r^3/(r^2+a^2)^(3/2),
  isotropic direction, speed q*v_esc with q drawn by rejection from
  g(q) = q^2 (1-q^2)^(7/2).
* Kepler orbits about the hole from (a, e), an isotropic orbital plane, a
  uniform argument of periapsis and a uniform mean anomaly; Kepler's equation
  E - e sin E = M is solved by Newton iteration.

The paper's own test model (Section 4) is a cold uniform shell 1 < r < 10 drawn
with a linear congruential generator; :func:`cold_shell` provides that shape
(drawn with SplitMix64) as an optional input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_MUL1 = 0xBF58476D1CE4E5B9
_MUL2 = 0x94D049BB133111EB


def splitmix64_scalar(state: int) -> tuple[int, int]:
    """One SplitMix64 step on Python integers: returns (new_state, output)."""
    state = (state + _GAMMA) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * _MUL1) & _MASK64
    z = ((z ^ (z >> 27)) * _MUL2) & _MASK64
    return state, z ^ (z >> 31)


class SplitMix64:
    """Vectorised SplitMix64 stream.

    The k-th output (k = 1, 2, ...) of a stream seeded with ``s`` is
    ``mix(s + k * gamma mod 2^64)``, so a block of outputs is computed at once
    from the counter values; the sequence equals the scalar recurrence.
    """

    def __init__(self, seed: int):
        self._state = int(seed) & _MASK64

    def next_u64(self, n: int) -> np.ndarray:
        n = int(n)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self._state) + k * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_MUL1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_MUL2)
            z = z ^ (z >> np.uint64(31))
        self._state = (self._state + n * _GAMMA) & _MASK64
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1): the top 53 bits of each output times 2^-53."""
        u = self.next_u64(n) >> np.uint64(11)
        return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def _isotropic(rng: SplitMix64, n: int) -> np.ndarray:
    """n unit vectors uniform on the sphere (cos(theta) and phi uniform)."""
    cz = 2.0 * rng.uniform(n) - 1.0
    ph = 2.0 * math.pi * rng.uniform(n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def plummer(rng: SplitMix64, n: int, total_mass: float = 1.0, a: float = 1.0,
            G: float = 1.0, rmax: float = 10.0) -> tuple[np.ndarray, np.ndarray]:
    """Positions and velocities of n Plummer-sphere stars (AHW 1974 sampling).

    Radii beyond ``rmax`` (in units of ``a``) are rejected and redrawn.
    """
    r = np.empty(n)
    filled = 0
    while filled < n:
        k = n - filled
        X = rng.uniform(k)
        with np.errstate(divide="ignore", invalid="ignore"):
            rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        ok = (X > 0.0) & np.isfinite(rr) & (rr <= rmax * a)
        take = rr[ok]
        r[filled:filled + take.size] = take
        filled += take.size
    pos = r[:, None] * _isotropic(rng, n)

    q = np.empty(n)
    filled = 0
    while filled < n:
        k = n - filled
        X4 = rng.uniform(k)
        X5 = rng.uniform(k)
        ok = 0.1 * X5 < X4 * X4 * (1.0 - X4 * X4) ** 3.5
        take = X4[ok]
        q[filled:filled + take.size] = take
        filled += take.size
    vesc = math.sqrt(2.0 * G * total_mass) * (r * r + a * a) ** -0.25
    vel = (q * vesc)[:, None] * _isotropic(rng, n)
    return pos, vel


def kepler_orbits(rng: SplitMix64, n: int, mu: np.ndarray | float, a_orb: float,
                  ecc: float) -> tuple[np.ndarray, np.ndarray]:
    """Relative positions/velocities of n bound Kepler orbits (G(M+m) = mu)."""
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (n,))
    h = _isotropic(rng, n)                       # orbit normal
    om = 2.0 * math.pi * rng.uniform(n)          # argument of periapsis
    Mmean = 2.0 * math.pi * rng.uniform(n)       # mean anomaly
    E = np.where(ecc > 0.8, np.full(n, math.pi), Mmean)
    for _ in range(100):
        f = E - ecc * np.sin(E) - Mmean
        dE = f / (1.0 - ecc * np.cos(E))
        E = E - dE
        if np.max(np.abs(dE)) < 1e-15:
            break
    # orthonormal basis of the orbital plane
    ref = np.where(np.abs(h[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    u1 = np.cross(h, ref)
    u1 /= np.linalg.norm(u1, axis=1, keepdims=True)
    u2 = np.cross(h, u1)
    P = np.cos(om)[:, None] * u1 + np.sin(om)[:, None] * u2
    Q = np.cross(h, P)
    b = a_orb * math.sqrt(1.0 - ecc * ecc)
    nmean = np.sqrt(mu / a_orb ** 3)
    Edot = nmean / (1.0 - ecc * np.cos(E))
    xp = a_orb * (np.cos(E) - ecc)
    yp = b * np.sin(E)
    vxp = -a_orb * np.sin(E) * Edot
    vyp = b * np.cos(E) * Edot
    pos = xp[:, None] * P + yp[:, None] * Q
    vel = vxp[:, None] * P + vyp[:, None] * Q
    return pos, vel


def make_cluster(n_total: int, m_bh: float, seed: int, G: float = 1.0,
                 ecc_frac: float = 0.0, ecc_a: float = 1e-3, ecc_e: float = 0.9,
                 rmax: float = 10.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """A black hole of mass ``m_bh`` at rest at the origin plus n_total-1 stars.

    Stars have equal mass 1/(n_total-1), so the total star mass is 1 (the
    paper's normalisation, Eq. 9).  Star positions and velocities are drawn
    from a Plummer sphere (a = 1) and recentred to zero mass-weighted mean
    position and velocity.  Then ``round(ecc_frac*(n_total-1))`` stars (the
    first ones) are replaced by Kepler orbits of semi-major axis ``ecc_a`` and
    eccentricity ``ecc_e`` about the hole, and star velocities are recentred
    once more so that the stars' total momentum is zero while the hole stays
    at rest (the zero-momentum frame the equations of motion assume).
    """
    if n_total < 2:
        raise ValueError("need the black hole and at least one star")
    ns = n_total - 1
    ms = 1.0 / ns
    rng = SplitMix64(seed)
    pos, vel = plummer(rng, ns, total_mass=1.0, a=1.0, G=G, rmax=rmax)
    pos -= pos.mean(axis=0)
    vel -= vel.mean(axis=0)
    n_ecc = int(round(ecc_frac * ns))
    if n_ecc > 0:
        p2, v2 = kepler_orbits(rng, n_ecc, G * (m_bh + ms), ecc_a, ecc_e)
        pos[:n_ecc] = p2
        vel[:n_ecc] = v2
        vel -= vel.mean(axis=0)
    x = np.zeros((n_total, 3))
    v = np.zeros((n_total, 3))
    m = np.empty(n_total)
    x[1:] = pos
    v[1:] = vel
    m[0] = m_bh
    m[1:] = ms
    return np.ascontiguousarray(x), np.ascontiguousarray(v), m


def cold_shell(n_total: int, m_bh_over_m: float, seed: int, rin: float = 1.0,
               rout: float = 10.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The paper's Section-4 test model: stars uniform in rin < r < rout at rest,
    equal masses summing to 1, a hole of mass ``m_bh_over_m`` star masses at the
    origin, everything cold (v = 0)."""
    ns = n_total - 1
    ms = 1.0 / ns
    rng = SplitMix64(seed)
    u = rng.uniform(ns)
    r = (rin ** 3 + u * (rout ** 3 - rin ** 3)) ** (1.0 / 3.0)
    x = np.zeros((n_total, 3))
    x[1:] = r[:, None] * _isotropic(rng, ns)
    v = np.zeros((n_total, 3))
    m = np.full(n_total, ms)
    m[0] = m_bh_over_m * ms
    return x, v, m


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: cluster shape, physical constants, integrator."""
    name: str
    n: int
    m_bh: float
    c: float
    eps: float
    dt: float
    steps: int
    seed: int
    G: float = 1.0
    ecc_frac: float = 0.0
    ecc_a: float = 1e-3
    ecc_e: float = 0.9
    precisions: tuple = field(default=("mixed",))

    def state(self, n: int | None = None):
        """(x, v, m) of this workload, optionally with a different body count."""
        return make_cluster(self.n if n is None else n, self.m_bh, self.seed, G=self.G,
                            ecc_frac=self.ecc_frac, ecc_a=self.ecc_a, ecc_e=self.ecc_e)


# The five workloads the library is measured and checked on.
WORKLOADS = {
    "plummer1k_fp64": Workload("plummer1k_fp64", n=1024, m_bh=0.1, c=100.0, eps=1e-4,
                               dt=1.0 / 1024, steps=100, seed=1000, precisions=("fp64",)),
    "plummer16k": Workload("plummer16k", n=16384, m_bh=0.05, c=50.0, eps=1e-4,
                           dt=1.0 / 2048, steps=1000, seed=2000, precisions=("fp64", "mixed")),
    "plummer128k_ecc": Workload("plummer128k_ecc", n=131072, m_bh=0.76, c=30.0, eps=5e-5,
                                dt=1.0 / 8192, steps=200, seed=3000, ecc_frac=0.01,
                                ecc_a=1e-3, ecc_e=0.9, precisions=("mixed",)),
    "plummer8k_adjoint": Workload("plummer8k_adjoint", n=8192, m_bh=0.1, c=50.0, eps=1e-4,
                                  dt=1.0 / 2048, steps=1000, seed=5000, precisions=("fp64",)),
}


def batched_workloads(n_clusters: int = 64, seed: int = 4000, nmin: int = 512,
                      nmax: int = 32768) -> list[Workload]:
    """The batched workload: clusters with N log-uniform in [nmin, nmax], hole
    mass uniform in [0.01, 0.2] and c uniform in [20, 200], each with its own
    seed (seed + 1 + k)."""
    rng = SplitMix64(seed)
    u = rng.uniform(3 * n_clusters).reshape(n_clusters, 3)
    out = []
    for k in range(n_clusters):
        n = int(round(math.exp(math.log(nmin) + u[k, 0] * (math.log(nmax) - math.log(nmin)))))
        out.append(Workload(f"batched{k}", n=n, m_bh=0.01 + 0.19 * u[k, 1],
                            c=20.0 + 180.0 * u[k, 2], eps=1e-4, dt=1.0 / 2048, steps=500,
                            seed=seed + 1 + k))
    return out
