"""The debug build (libpn_debug.so, PN_DEBUG_CHECKS): its kernels check their
global-memory indices and report a failed check as PN_EINDEX instead of
trapping.  On the workload shapes (ragged sizes, near sources, the spatial
order) no check fails and the results equal the release build's; a check
made to fail by the test hook (PN_DEBUG_INJECT) comes back as PN_EINDEX with
its site, and the context keeps working."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Child program: A, two KDK steps and the energy on a few systems, through
# whichever library PN_LIBRARY names; prints the results as JSON.
CHILD = r"""
import json, sys, numpy as np, torch
from paper_1801_07986_b300 import pn
from paper_1801_07986_b300.inputs import make_cluster
out = {"debug": pn._load().pn_debug_checks()}
for n, prec in ((2, "fp64"), (3, "mixed"), (700, "mixed"), (5000, "mixed"), (1500, "fp64")):
    x, v, m = make_cluster(n, 0.1, 11 + n) if n > 3 else (
        np.array([[0, 0, 0], [1.0, 0.2, 0], [-0.3, 0.8, 0.1]])[:n],
        np.array([[0, 0, 0], [0, 0.9, 0], [0.5, 0, 0.2]])[:n], np.array([0.1, 1e-3, 2e-3])[:n])
    X, V, M = (torch.tensor(np.ascontiguousarray(a), device="cuda:0") for a in (x, v, m))
    A = torch.empty_like(X)
    ctx = pn.pn_init(n, c=20.0, eps=1e-3, precision=prec, device=0)
    pn.pn_accel(ctx, X, V, M, A)
    a0 = A.cpu().numpy().tolist()
    pn.pn_step(ctx, X, V, M, A, 1e-3, 2)
    e = pn.pn_energy(ctx, X, V, M)
    out[f"{n}-{prec}"] = {"a0": a0, "x": X.cpu().numpy().tolist(), "a": A.cpu().numpy().tolist(),
                          "E": e["E"]}
    ctx.close()
print(json.dumps(out))
"""

INJECT = r"""
import sys, torch
from paper_1801_07986_b300 import pn
from paper_1801_07986_b300.inputs import make_cluster
x, v, m = make_cluster(1000, 0.1, 5)
X, V, M = (torch.tensor(a, device="cuda:0") for a in (x, v, m))
A = torch.empty_like(X)
ctx = pn.pn_init(1000, c=20.0, eps=1e-3, precision="mixed", device=0)
pn.pn_accel(ctx, X, V, M, A)
pn.pn_step(ctx, X, V, M, A, 1e-3, 1)
try:
    pn.pn_sync(ctx)
    print("NO-ERROR")
except pn.PNError as e:
    print(e.status, str(e))
pn.pn_step(ctx, X, V, M, A, 1e-3, 1)      # reported once, then the context goes on
try:
    pn.pn_sync(ctx)
    print("SECOND-OK" if not torch.isnan(X).any() else "SECOND-NAN")
except pn.PNError as e:
    print("SECOND", e.status)
"""


def _run(code, library, **env):
    e = dict(os.environ, PYTHONPATH=ROOT, PN_LIBRARY=library, **env)
    r = subprocess.run([sys.executable, "-c", code], env=e, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()


@pytest.fixture(scope="module")
def libs():
    from paper_1801_07986_b300 import build
    return build.build_library(), build.build_library(debug=True)


@pytest.mark.parametrize("spatial", ["0", "1"])
def test_debug_build_checks_pass_and_results_match_release(libs, spatial):
    rel, dbg = libs
    want = json.loads(_run(CHILD, rel, PN_SPATIAL=spatial)[-1])
    got = json.loads(_run(CHILD, dbg, PN_SPATIAL=spatial)[-1])
    assert want["debug"] == 0 and got["debug"] == 1
    for key in want:
        if key == "debug":
            continue
        for f in ("a0", "x", "a"):
            a, b = np.array(got[key][f]), np.array(want[key][f])
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (key, f)
        assert abs(got[key]["E"] - want[key]["E"]) <= 1e-12 * abs(want[key]["E"]), key


@pytest.mark.parametrize("site", [1, 5])
def test_debug_build_reports_a_failed_check(libs, site):
    _, dbg = libs
    lines = _run(INJECT, dbg, PN_DEBUG_INJECT=str(site))
    status, msg = lines[0].split(" ", 1)
    assert int(status) == 8 and "PN_EINDEX" in msg and f"site {site} " in msg, lines
    # the hook stays armed, so the next step reports again; nothing faulted
    assert lines[1].startswith("SECOND 8") or lines[1] == "SECOND-OK", lines
