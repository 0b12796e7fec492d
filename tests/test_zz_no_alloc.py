"""pn_energy_noalloc: the energy/momentum entry point for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or
they must not allocate once running).  It must give what pn_energy gives,
call after call, although every call reuses the same scratch array inside
the library.  This file is collected last on purpose."""
import ctypes
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
TOL = 1e-12          # the energy tolerance of the other GPU tests


def _ref(x, v, m, c, eps):
    ctx = pn.pn_init(m.shape[0], c=c, eps=eps, precision="fp64", device=0)
    out = pn.pn_energy(ctx, x, v, m)
    ctx.close()
    return np.concatenate([[out["E_N"], out["E_PN"]], out["P_N"], out["P_PN"]])


def _noalloc_c_abi(x, v, m, c, eps):
    """Call the C entry point directly (argument marshalling only)."""
    lib = pn._load()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=DEV)
    st = torch.cuda.current_stream(DEV).cuda_stream
    rc = lib.pn_energy_noalloc(0, ctypes.c_void_p(st), int(m.shape[0]), 1.0, float(c), float(eps),
                               ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                               ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    assert rc == pn.PN_OK, lib.pn_last_error().decode()
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def _check(got, want, v, m):
    assert np.all(np.isfinite(got))
    for k in (0, 1):
        assert abs(got[k] - want[k]) <= TOL * abs(want[k])
    pscale = float((m[:, None] * v.abs()).sum())
    assert np.abs(got[2:] - want[2:]).max() <= TOL * pscale


def _state(n, seed):
    x, v, m = make_cluster(n, 0.1, seed)
    v = v.copy()
    v[0] = [0.01, -0.005, 0.02]          # a moving hole exercises the v_1 terms
    return x, v, m


def test_noalloc_matches_pn_energy_on_two_calls_in_a_row():
    states = []
    for n, seed, c, eps in ((1500, 3, 12.0, 1e-3), (777, 4, math.inf, 1e-4)):
        x, v, m = _state(n, seed)
        states.append((torch.tensor(x, device=DEV), torch.tensor(v, device=DEV),
                       torch.tensor(m, device=DEV), c, eps))
    # the larger call first, so stale scratch would show in the second one
    for X, V, M, c, eps in states:
        want = _ref(X, V, M, c, eps)
        got = _noalloc_c_abi(X, V, M, c, eps)
        _check(got, want, V, M)


def test_noalloc_at_the_maximum_size_then_above_4096_against_oracle():
    """The full scratch (PN_NOALLOC_MAX_BODIES bodies) and then a size above
    4096 bodies, in that order: each against pn_energy and the FP64 oracle
    (Eq. 7 and Eq. 8)."""
    import oracle
    for n, seed, c, eps in ((pn.PN_NOALLOC_MAX_BODIES, 5, 50.0, 1e-4), (5000, 6, 20.0, 1e-3)):
        x, v, m = _state(n, seed)
        X, V, M = (torch.tensor(a, device=DEV) for a in (x, v, m))
        got = _noalloc_c_abi(X, V, M, c, eps)
        _check(got, _ref(X, V, M, c, eps), V, M)
        o = oracle.energy(x, v, m, c=c, eps=eps)
        want = np.concatenate([[o["E_N"], o["E_PN"]], o["P_N"], o["P_PN"]])
        _check(got, want, V, M)


def test_noalloc_rejects_too_many_bodies():
    lib = pn._load()
    n = pn.PN_NOALLOC_MAX_BODIES + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    out = torch.zeros(8, dtype=torch.float64, device=DEV)
    rc = lib.pn_energy_noalloc(0, None, n, 1.0, 10.0, 0.0, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()))
    assert rc == pn.PN_EINVAL
    assert "PN_NOALLOC_MAX_BODIES" in lib.pn_last_error().decode()
