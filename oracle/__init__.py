"""FP64 CPU oracle of the limited-1PN N-body equations -- TEST INFRASTRUCTURE.

This package is the checker, not the product.  Only the tests, the package's
``smoke()`` check and the CPU-baseline leg of ``bench.py`` may import it.  It
shares no code with the CUDA path (``paper_1801_07986_b300``); the two meet
only through the seeded input generator ``paper_1801_07986_b300.inputs``,
which holds none of the method's arithmetic.

The arithmetic lives in ``pn_oracle.c`` (plain C, FP64, compensated sums,
OpenMP over targets with a fixed per-target order).  This module compiles it
with gcc on first use (or via :func:`build`) and wraps it with ctypes.

Functions follow the paper (Tatekawa, arXiv:1801.07986):

* :func:`accel`      Section 2, Eq. 1-6 (Eq. 10 softening between stars)
* :func:`accel_rows` the same for selected targets
* :func:`bh_partial` the hole's sums of Eq. 1-3 over a range of outer stars
* :func:`energy`     Section 2, Eq. 7 and Eq. 8
* :func:`step`       kick-drift-kick leapfrog, force at the predicted velocity
* :func:`rk4_step`   the paper's classical fourth-order Runge-Kutta (Section 4)
* :func:`newton_accel`  Newtonian accelerations alone (the c -> infinity limit)
* :func:`eih_accel`, :func:`eih_energy`, :func:`eih_step`  general EIH
  equations (Einstein, Infeld & Hoffmann 1938) used only as a cross-check.

Pins (tests/test_oracle_pins.py): Newtonian brute force, the c -> infinity
limit, the 1PN circular-orbit frequency and periastron advance, exact
polynomial-degree agreement with the general EIH equations, energy and
momentum balance through 1PN order, softening placement, integrator order,
invariances; tests/test_oracle_mutants.py shows each pin catching planted
mistakes.  Parity unpinned: trajectories of the 128k eccentric-orbit workload
(chaotic and outside the 1PN regime), and the choice between the two velocity
modes of the integrator (pinned only by its convergence order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-std=c11", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile pn_oracle.c into liboracle.so (gcc, -ffp-contract=off)."""
    srcs = (_SRC, os.path.join(_HERE, "pn_oracle_accel.inc"))
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                                for f in srcs):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("PN_ORACLE_LIB")   # a prebuilt variant (tests only)
            if not path:
                path = build()
            lib = ctypes.CDLL(path)
            d = ctypes.c_double
            i64 = ctypes.c_int64
            p = ctypes.c_void_p
            lib.orc_accel.argtypes = [i64, p, p, p, d, d, d, p]
            lib.orc_accel_rows.argtypes = [i64, p, p, p, d, d, d, i64, p, p]
            lib.orc_bh_rows.argtypes = [i64, p, p, p, d, d, i64, p, p]
            lib.orc_bh_partial.argtypes = [i64, p, p, p, d, d, i64, i64, p]
            lib.orc_newton_accel.argtypes = [i64, p, p, d, d, p]
            lib.orc_energy.argtypes = [i64, p, p, p, d, d, d, p]
            lib.orc_eih_accel.argtypes = [i64, p, p, p, d, d, p]
            lib.orc_eih_energy.argtypes = [i64, p, p, p, d, d, p]
            lib.orc_step.argtypes = [i64, p, p, p, p, d, d, d, d, i64, ctypes.c_int]
            lib.orc_eih_step.argtypes = [i64, p, p, p, p, d, d, d, i64, ctypes.c_int]
            lib.orc_rk4_step.argtypes = [i64, p, p, p, p, d, d, d, d, i64]
            lib.orc_jerk.argtypes = [i64, p, p, p, d, d, d, p, p]
            lib.orc_accel_jvp.argtypes = [i64, p, p, p, d, d, d, p, p, d, d, p]
            lib.orc_hermite_step.argtypes = [i64, p, p, p, p, d, d, d, d, i64]
            lib.orc_traj_jvp.argtypes = [i64, p, p, p, d, d, d, d, i64, ctypes.c_int, p, p, d, d,
                                         p, p, p, p]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_get_threads.restype = ctypes.c_int
            for f in ("orc_accel", "orc_accel_rows", "orc_bh_rows", "orc_newton_accel",
                      "orc_energy", "orc_eih_accel", "orc_eih_energy", "orc_step",
                      "orc_eih_step", "orc_rk4_step"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _inv_c2(c):
    return 0.0 if np.isinf(c) else 1.0 / (c * c)


def _state(x, v, m):
    m = _f64(m)
    n = m.shape[0]
    return _f64(x, (n, 3)), _f64(v, (n, 3)), m, n


def set_threads(n: int) -> None:
    """Number of OpenMP threads (0 = the OpenMP default)."""
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_get_threads())


def accel(x, v, m, G=1.0, c=np.inf, eps=0.0):
    """Accelerations (N, 3) of all bodies, Eq. 1-6 (body 0 = heavy body)."""
    x, v, m, n = _state(x, v, m)
    a = np.empty((n, 3))
    rc = _load().orc_accel(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), eps, _ptr(a))
    if rc:
        raise ValueError(f"orc_accel failed ({rc})")
    return a


def accel_rows(x, v, m, targets, G=1.0, c=np.inf, eps=0.0):
    """Accelerations of the listed targets only, shape (len(targets), 3)."""
    x, v, m, n = _state(x, v, m)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    a = np.empty((t.shape[0], 3))
    rc = _load().orc_accel_rows(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), eps,
                                t.shape[0], _ptr(t), _ptr(a))
    if rc:
        raise ValueError(f"orc_accel_rows failed ({rc})")
    return a


def bh_rows(x, v, m, js, G=1.0, eps=0.0):
    """Inner double-sum rows of Eq. 3 for the listed outer indices j."""
    x, v, m, n = _state(x, v, m)
    j = np.ascontiguousarray(js, dtype=np.int64)
    out = np.empty((j.shape[0], 3))
    rc = _load().orc_bh_rows(n, _ptr(x), _ptr(v), _ptr(m), G, eps, j.shape[0], _ptr(j), _ptr(out))
    if rc:
        raise ValueError(f"orc_bh_rows failed ({rc})")
    return out


def bh_partial(x, v, m, j0, j1, G=1.0, eps=0.0):
    """The hole's sums of Eq. 1-3 over the outer stars j in [j0, j1): (the
    Newtonian sum, the 1PN sums before 1/c^2), each a 3-vector.  Over
    [1, n) the hole's acceleration is newt + pn / c^2."""
    x, v, m, n = _state(x, v, m)
    out = np.empty(6)
    rc = _load().orc_bh_partial(n, _ptr(x), _ptr(v), _ptr(m), G, eps, int(j0), int(j1),
                                _ptr(out))
    if rc:
        raise ValueError("orc_bh_partial failed")
    return out[:3].copy(), out[3:].copy()


def newton_accel(x, m, G=1.0, eps=0.0):
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    a = np.empty((n, 3))
    rc = _load().orc_newton_accel(n, _ptr(x), _ptr(m), G, eps, _ptr(a))
    if rc:
        raise ValueError("orc_newton_accel failed")
    return a


def energy(x, v, m, G=1.0, c=np.inf, eps=0.0):
    """Eq. 7 and Eq. 8: dict with E_N, E_PN (already times 1/c^2), E, P_N, P_PN, P."""
    x, v, m, n = _state(x, v, m)
    out = np.empty(8)
    rc = _load().orc_energy(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), eps, _ptr(out))
    if rc:
        raise ValueError("orc_energy failed")
    return {"E_N": out[0], "E_PN": out[1], "E": out[0] + out[1],
            "P_N": out[2:5].copy(), "P_PN": out[5:8].copy(), "P": out[2:5] + out[5:8]}


def step(x, v, m, a, dt, nsteps, G=1.0, c=np.inf, eps=0.0, vel_mode=0):
    """Advance copies of (x, v, a) by nsteps KDK steps; returns (x, v, a)."""
    x, v, m, n = _state(x, v, m)
    x, v = x.copy(), v.copy()
    a = _f64(a, (n, 3)).copy()
    rc = _load().orc_step(n, _ptr(x), _ptr(v), _ptr(m), _ptr(a), G, _inv_c2(c), eps,
                          dt, int(nsteps), int(vel_mode))
    if rc:
        raise ValueError(f"orc_step failed ({rc})")
    return x, v, a


def rk4_step(x, v, m, a, dt, nsteps, G=1.0, c=np.inf, eps=0.0):
    """Advance copies of (x, v, a) by nsteps classical RK4 steps (Section 4);
    `a` must hold A at the entry state; returns (x, v, a at the final state)."""
    x, v, m, n = _state(x, v, m)
    x, v = x.copy(), v.copy()
    a = _f64(a, (n, 3)).copy()
    rc = _load().orc_rk4_step(n, _ptr(x), _ptr(v), _ptr(m), _ptr(a), G, _inv_c2(c), eps,
                              dt, int(nsteps))
    if rc:
        raise ValueError(f"orc_rk4_step failed ({rc})")
    return x, v, a


def jerk(x, v, m, a=None, G=1.0, c=np.inf, eps=0.0):
    """Time derivative of the accelerations along the trajectory (Appendix A)
    at (x, v), with `a` = A(x, v) (computed if None), by a complex step of
    the oracle's own Eq. 1-6."""
    x, v, m, n = _state(x, v, m)
    if a is None:
        a = accel(x, v, m, G=G, c=c, eps=eps)
    a = _f64(a, (n, 3))
    out = np.zeros((n, 3))
    rc = _load().orc_jerk(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), eps, _ptr(a), _ptr(out))
    if rc:
        raise ValueError(f"orc_jerk failed ({rc})")
    return out


def accel_jvp(x, v, m, dx, dv, dM=0.0, dinv_c2=0.0, G=1.0, c=np.inf, eps=0.0):
    """Directional derivative of A(x, v; M = m[0], 1/c^2) along
    (dx, dv, dM, dinv_c2), by a complex step of the oracle's Eq. 1-6."""
    x, v, m, n = _state(x, v, m)
    dx, dv = _f64(dx, (n, 3)), _f64(dv, (n, 3))
    out = np.zeros((n, 3))
    rc = _load().orc_accel_jvp(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), eps, _ptr(dx),
                               _ptr(dv), float(dM), float(dinv_c2), _ptr(out))
    if rc:
        raise ValueError(f"orc_accel_jvp failed ({rc})")
    return out


def hermite_step(x, v, m, a, dt, nsteps, G=1.0, c=np.inf, eps=0.0):
    """Advance copies of (x, v, a) by nsteps fourth-order Hermite PEC steps;
    `a` must hold A at the entry state; returns (x, v, a at the final state)."""
    x, v, m, n = _state(x, v, m)
    x, v = x.copy(), v.copy()
    a = _f64(a, (n, 3)).copy()
    rc = _load().orc_hermite_step(n, _ptr(x), _ptr(v), _ptr(m), _ptr(a), G, _inv_c2(c), eps,
                                  dt, int(nsteps))
    if rc:
        raise ValueError(f"orc_hermite_step failed ({rc})")
    return x, v, a


def traj_jvp(x0, v0, m, dt, nsteps, dx0, dv0, dM=0.0, dinv_c2=0.0, G=1.0, c=np.inf, eps=0.0,
             vel_mode=0):
    """Final state of nsteps KDK steps from (x0, v0) (entry acceleration
    A(x0, v0)) and its derivative along the perturbation (dx0, dv0, dM of the
    hole mass m[0], dinv_c2 of 1/c^2), by a complex step; returns
    (x, v, dx, dv)."""
    x0, v0, m, n = _state(x0, v0, m)
    dx0, dv0 = _f64(dx0, (n, 3)), _f64(dv0, (n, 3))
    x, v, dx, dv = (np.zeros((n, 3)) for _ in range(4))
    rc = _load().orc_traj_jvp(n, _ptr(x0), _ptr(v0), _ptr(m), G, _inv_c2(c), eps, dt,
                              int(nsteps), int(vel_mode), _ptr(dx0), _ptr(dv0), float(dM),
                              float(dinv_c2), _ptr(x), _ptr(v), _ptr(dx), _ptr(dv))
    if rc:
        raise ValueError(f"orc_traj_jvp failed ({rc})")
    return x, v, dx, dv


def eih_accel(x, v, m, G=1.0, c=np.inf):
    x, v, m, n = _state(x, v, m)
    a = np.empty((n, 3))
    rc = _load().orc_eih_accel(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), _ptr(a))
    if rc:
        raise ValueError("orc_eih_accel failed")
    return a


def eih_energy(x, v, m, G=1.0, c=np.inf):
    x, v, m, n = _state(x, v, m)
    out = np.empty(8)
    rc = _load().orc_eih_energy(n, _ptr(x), _ptr(v), _ptr(m), G, _inv_c2(c), _ptr(out))
    if rc:
        raise ValueError("orc_eih_energy failed")
    return {"E_N": out[0], "E_PN": out[1], "E": out[0] + out[1],
            "P_N": out[2:5].copy(), "P_PN": out[5:8].copy(), "P": out[2:5] + out[5:8]}


def eih_step(x, v, m, a, dt, nsteps, G=1.0, c=np.inf, vel_mode=0):
    x, v, m, n = _state(x, v, m)
    x, v = x.copy(), v.copy()
    a = _f64(a, (n, 3)).copy()
    rc = _load().orc_eih_step(n, _ptr(x), _ptr(v), _ptr(m), _ptr(a), G, _inv_c2(c), dt,
                              int(nsteps), int(vel_mode))
    if rc:
        raise ValueError("orc_eih_step failed")
    return x, v, a
