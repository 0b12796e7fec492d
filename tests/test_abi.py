"""The C ABI on the host: libpn builds, loads, exports every symbol the
header declares, and rejects bad arguments before touching the GPU."""
import ctypes
import math
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1801_07986_b300 import build, pn
    build.build_library()
    return pn._load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pn_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("pn_init", "pn_accel", "pn_step", "pn_energy", "pn_set_params", "pn_destroy",
                 "pn_last_error", "pn_step_host", "pn_sync"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (pn_[a-z_]+)", out))
    assert set(declared_functions()) <= exported


def test_header_compiles_as_c():
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c", HEADER],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _params(G=1.0, c=50.0, eps=1e-4, precision=1, vel_mode=0, r_near=0.05, pair_kernel=0,
            integrator=0):
    from paper_1801_07986_b300.pn import _Params
    return _Params(G, c, eps, precision, vel_mode, r_near, pair_kernel, integrator)


@pytest.mark.parametrize("n,kw,msg", [
    (1, {}, "n must be"),
    (0, {}, "n must be"),
    (100, {"G": 0.0}, "G must be"),
    (100, {"G": float("nan")}, "G must be"),
    (100, {"c": -1.0}, "c must be"),
    (100, {"c": float("nan")}, "c must be"),
    (100, {"eps": -1e-3}, "eps must be"),
    (100, {"eps": float("inf")}, "eps must be"),
    (100, {"precision": 7}, "precision"),
    (100, {"vel_mode": 3}, "vel_mode"),
    (100, {"r_near": -1.0}, "r_near"),
    (100, {"r_near": float("nan")}, "r_near"),
    (100, {"pair_kernel": 2}, "pair_kernel"),
    (100, {"integrator": 5}, "integrator"),
])
def test_init_rejects_bad_arguments_on_host(lib, n, kw, msg):
    h = ctypes.c_void_p()
    p = _params(**kw)
    st = lib.pn_init(ctypes.byref(h), n, ctypes.byref(p), 0, None)
    assert st == 1  # PN_EINVAL
    assert msg in lib.pn_last_error().decode()
    assert not h.value


def test_null_arguments(lib):
    p = _params()
    assert lib.pn_init(None, 10, ctypes.byref(p), 0, None) == 1
    assert lib.pn_init(ctypes.byref(ctypes.c_void_p()), 10, None, 0, None) == 1
    for name, nargs in (("pn_accel", 5), ("pn_step", 7), ("pn_energy", 5), ("pn_sync", 1),
                        ("pn_step_host", 7), ("pn_set_timing", 2), ("pn_get_launch", 2),
                        ("pn_get_pair_stats", 2), ("pn_get_variant", 2),
                        ("pn_launch_count", 2), ("pn_jerk", 6), ("pn_accel_vjp", 8),
                        ("pn_step_save", 9), ("pn_step_vjp_saved", 11)):
        fn = getattr(lib, name)
        args = [None] * nargs
        if name in ("pn_step", "pn_step_host", "pn_step_save"):
            args[5] = 0.01
            args[6] = 1
        if name == "pn_step_save":
            args[7] = 0
        if name == "pn_step_vjp_saved":
            args[3] = 0.01
            args[4] = 1
            args[5] = 0
        if name == "pn_set_timing":
            args[1] = 1
        assert fn(*args) == 1, name
        assert "NULL" in lib.pn_last_error().decode()
    lib.pn_destroy(None)   # no-op


def test_watchdog_status_plumbing(lib):
    """PN_EDRIFT has one value in the header and the binding, the binding names
    it, and pn_set_watchdog rejects a NULL context on the host."""
    from paper_1801_07986_b300 import pn
    src = open(HEADER).read()
    m = re.search(r"PN_EDRIFT\s*=\s*(\d+)", src)
    assert m and int(m.group(1)) == pn.PN_EDRIFT == 7
    assert pn.STATUS_NAMES[pn.PN_EDRIFT] == "PN_EDRIFT"
    e = pn.PNError(pn.PN_EDRIFT, "energy drift 1e-2 above 1e-3 (cluster 0, first at step 120)")
    assert str(e).startswith("PN_EDRIFT: ") and e.status == 7
    assert lib.pn_set_watchdog(None, 1e-3, 10) == 1
    assert "NULL" in lib.pn_last_error().decode()
    assert lib.pn_set_watchdog(None, 0.0, 0) == 1


def test_injected_allocation_failure():
    code = ("import ctypes; from paper_1801_07986_b300 import pn; lib = pn._load();"
            "p = pn._Params(1.0, 50.0, 1e-4, 1, 0, 0.05, 0, 0); h = ctypes.c_void_p();"
            "print(lib.pn_init(ctypes.byref(h), 100, ctypes.byref(p), 0, None),"
            " lib.pn_last_error().decode())")
    env = dict(os.environ, PN_FAIL_ALLOC="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True).stdout
    assert out.startswith("2 ") and "PN_FAIL_ALLOC" in out


def test_python_binding_fails_loudly_without_library(tmp_path):
    code = ("from paper_1801_07986_b300 import pn\n"
            "try:\n    pn.pn_version()\nexcept RuntimeError as e:\n    print('raised', e)\n")
    env = dict(os.environ, PN_LIBRARY=str(tmp_path / "missing.so"), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True).stdout
    assert out.startswith("raised") and "no CPU fallback" in out


def test_version(lib):
    assert lib.pn_version() >= 100


def test_python_binding_validates_before_calling(lib):
    from paper_1801_07986_b300 import pn
    with pytest.raises(ValueError):
        pn._params(1.0, math.inf, 0.0, "fp32", "vpred_end")
    with pytest.raises(ValueError):
        pn._params(1.0, math.inf, 0.0, "mixed", "rk4")
    with pytest.raises(ValueError):
        pn._params(1.0, math.inf, 0.0, "mixed", "vhalf", 0.05, "three_pass")


def test_batched_init_rejects_bad_offsets_on_host(lib):
    from paper_1801_07986_b300.pn import _Cluster
    p = _params()
    h = ctypes.c_void_p()
    cases = [([0, 1, 10], "cluster 0 has 1 bodies"), ([1, 10, 20], "offsets[0] must be 0"),
             ([0, 10, 10], "cluster 1 has 0 bodies")]
    for off, msg in cases:
        arr = (ctypes.c_int64 * len(off))(*off)
        st = lib.pn_init_batched(ctypes.byref(h), len(off) - 1, arr, None, ctypes.byref(p), 0, None)
        assert st == 1 and msg in lib.pn_last_error().decode(), (off, lib.pn_last_error())
    arr = (ctypes.c_int64 * 3)(0, 10, 20)
    cl = (_Cluster * 2)()
    cl[0].G, cl[0].c, cl[0].eps = 1.0, 10.0, 0.0
    cl[1].G, cl[1].c, cl[1].eps = 1.0, -3.0, 0.0
    st = lib.pn_init_batched(ctypes.byref(h), 2, arr, ctypes.cast(cl, ctypes.c_void_p),
                             ctypes.byref(p), 0, None)
    assert st == 1 and "cluster 1" in lib.pn_last_error().decode()
    assert lib.pn_init_batched(ctypes.byref(h), 0, arr, None, ctypes.byref(p), 0, None) == 1
