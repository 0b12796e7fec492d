"""Thin ctypes binding of libpn's C ABI (include/pn.h), same names.

Argument marshalling only: every step of the computation runs in libpn's
CUDA kernels.  Device arrays are torch tensors (float64, contiguous, on the
context's device); ``pn_step_host`` takes numpy arrays.  If ``libpn.so`` is
missing the first call raises -- there is no CPU fallback.

    ctx = pn_init(n, G=1.0, c=50.0, eps=1e-4, precision="mixed")
    pn_accel(ctx, x, v, m, a)             # a = A(x, v)
    pn_step(ctx, x, v, m, a, dt, nsteps)  # KDK steps, in place
    e = pn_energy(ctx, x, v, m)           # Eq. 7 / Eq. 8
    pn_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

(PN_OK, PN_EINVAL, PN_ENOMEM, PN_ECUDA, PN_ENONFINITE, PN_ETIMEOUT, PN_EUNSUPPORTED,
 PN_EDRIFT, PN_EINDEX) = range(9)
STATUS_NAMES = {0: "PN_OK", 1: "PN_EINVAL", 2: "PN_ENOMEM", 3: "PN_ECUDA", 4: "PN_ENONFINITE",
                5: "PN_ETIMEOUT", 6: "PN_EUNSUPPORTED", 7: "PN_EDRIFT", 8: "PN_EINDEX"}
PN_FP64, PN_MIXED = 0, 1
PN_VPRED_END, PN_VHALF = 0, 1
PN_PAIR_FUSED, PN_PAIR_TWO_PASS = 0, 1
PN_KDK, PN_RK4, PN_HERMITE = 0, 1, 2
PN_NOALLOC_MAX_BODIES = 16384
_PRECISION = {"fp64": PN_FP64, "mixed": PN_MIXED, PN_FP64: PN_FP64, PN_MIXED: PN_MIXED}
_VEL_MODE = {"vpred_end": PN_VPRED_END, "vhalf": PN_VHALF, PN_VPRED_END: PN_VPRED_END,
             PN_VHALF: PN_VHALF}
_PAIR = {"fused": PN_PAIR_FUSED, "two_pass": PN_PAIR_TWO_PASS, PN_PAIR_FUSED: PN_PAIR_FUSED,
         PN_PAIR_TWO_PASS: PN_PAIR_TWO_PASS}
_INTEGRATOR = {"kdk": PN_KDK, "rk4": PN_RK4, "hermite": PN_HERMITE, PN_KDK: PN_KDK,
               PN_RK4: PN_RK4, PN_HERMITE: PN_HERMITE}


class PNError(RuntimeError):
    """A libpn call returned a status other than PN_OK."""

    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class _Cluster(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("c", ctypes.c_double), ("eps", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("c", ctypes.c_double), ("eps", ctypes.c_double),
                ("precision", ctypes.c_int), ("vel_mode", ctypes.c_int),
                ("r_near", ctypes.c_double), ("pair_kernel", ctypes.c_int),
                ("integrator", ctypes.c_int)]


# Default radius (in the state's length unit) inside which stars are summed
# as near sources of the hole-relative cross terms; see pn_params.r_near.
R_NEAR_DEFAULT = 0.05


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """libpn.so next to this file; PN_LIBRARY=<path> selects another build
    (the debug build libpn_debug.so, whose kernels check their indices)."""
    return os.environ.get("PN_LIBRARY") or os.path.join(HERE, "libpn.so")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is not built: run `python -m paper_1801_07986_b300.build`"
                                   " (or __graft_entry__.build()); there is no CPU fallback")
            lib = ctypes.CDLL(path)
            P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "pn_init": [ctypes.POINTER(P), I64, ctypes.POINTER(_Params), I, P],
                "pn_init_batched": [ctypes.POINTER(P), I, P, P, ctypes.POINTER(_Params), I, P],
                "pn_step_graph": [P, P, P, P, P, D, I64],
                "pn_tune": [P, P, P, P, P, P],
                "pn_set_params": [P, ctypes.POINTER(_Params)],
                "pn_set_stream": [P, P],
                "pn_accel": [P, P, P, P, P],
                "pn_jerk": [P, P, P, P, P, P],
                "pn_accel_vjp": [P, P, P, P, P, P, P, P],
                "pn_step_vjp": [P, P, P, P, D, I64, I64, P, P, P, P, P],
                "pn_step_save": [P, P, P, P, P, D, I64, I64, P],
                "pn_step_vjp_saved": [P, P, P, D, I64, I64, P, P, P, P, P],
                "pn_step": [P, P, P, P, P, D, I64],
                "pn_step_host": [P, P, P, P, P, D, I64],
                "pn_energy": [P, P, P, P, P],
                "pn_sync": [P],
                "pn_set_watchdog": [P, D, I64],
                "pn_set_timing": [P, I],
                "pn_get_timing": [P, P, P],
                "pn_get_launch": [P, P],
                "pn_get_variant": [P, P],
                "pn_get_pair_stats": [P, P],
                "pn_launch_count": [P, P],
                "pn_energy_noalloc": [I, P, I64, D, D, D, P, P, P, P],
                "pn_measure_peaks": [I, P, P],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.pn_last_error.argtypes = []
            lib.pn_last_error.restype = ctypes.c_char_p
            lib.pn_destroy.argtypes = [P]
            lib.pn_destroy.restype = None
            lib.pn_version.argtypes = []
            lib.pn_version.restype = ctypes.c_int
            lib.pn_debug_checks.argtypes = []
            lib.pn_debug_checks.restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(status: int) -> None:
    if status != PN_OK:
        raise PNError(status, pn_last_error())


def pn_last_error() -> str:
    return _load().pn_last_error().decode()


def pn_version() -> int:
    return int(_load().pn_version())


def _params(G, c, eps, precision, vel_mode, r_near=R_NEAR_DEFAULT, pair_kernel="fused",
            integrator="kdk") -> _Params:
    if precision not in _PRECISION:
        raise ValueError(f"precision must be 'fp64' or 'mixed', got {precision!r}")
    if vel_mode not in _VEL_MODE:
        raise ValueError(f"vel_mode must be 'vpred_end' or 'vhalf', got {vel_mode!r}")
    if pair_kernel not in _PAIR:
        raise ValueError(f"pair_kernel must be 'fused' or 'two_pass', got {pair_kernel!r}")
    if integrator not in _INTEGRATOR:
        raise ValueError(f"integrator must be 'kdk', 'rk4' or 'hermite', got {integrator!r}")
    return _Params(float(G), float(c), float(eps), _PRECISION[precision], _VEL_MODE[vel_mode],
                   float(r_near), _PAIR[pair_kernel], _INTEGRATOR[integrator])


class Context:
    """Owns one pn_ctx handle (pn_destroy on close / garbage collection)."""

    def __init__(self, handle: int, n: int, device: int, params: _Params, offsets=None):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self.device = device
        self.params = params
        self.offsets = [0, n] if offsets is None else list(offsets)
        self.n_clusters = len(self.offsets) - 1

    def close(self) -> None:
        if self.handle:
            _load().pn_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch_stream(device, stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    import torch
    return torch.cuda.current_stream(device).cuda_stream


def pn_init(n: int, G: float = 1.0, c: float = math.inf, eps: float = 0.0,
            precision="mixed", vel_mode="vpred_end", device: int | None = None,
            stream=None, r_near: float = R_NEAR_DEFAULT, pair_kernel="fused",
            integrator="kdk") -> Context:
    """Create a context for n bodies (body 0 = the hole)."""
    lib = _load()
    if device is None:
        import torch
        device = torch.cuda.current_device()
    p = _params(G, c, eps, precision, vel_mode, r_near, pair_kernel, integrator)
    h = ctypes.c_void_p()
    _check(lib.pn_init(ctypes.byref(h), int(n), ctypes.byref(p), int(device),
                       ctypes.c_void_p(_torch_stream(device, stream))))
    return Context(h.value, int(n), int(device), p)


def pn_init_batched(offsets, G=1.0, c=math.inf, eps=0.0, precision="mixed",
                    vel_mode="vpred_end", device: int | None = None, stream=None,
                    r_near: float = R_NEAR_DEFAULT, pair_kernel="fused",
                    integrator="kdk") -> Context:
    """Context for independent clusters evaluated together: cluster k holds
    bodies [offsets[k], offsets[k+1]) of the concatenated state, its hole
    first.  G, c, eps may be scalars or per-cluster sequences."""
    lib = _load()
    if device is None:
        import torch
        device = torch.cuda.current_device()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    k = off.shape[0] - 1
    if k < 1:
        raise ValueError("need at least one cluster")
    cl = (_Cluster * k)()
    Gs, cs, es = (np.broadcast_to(np.asarray(q, dtype=np.float64), (k,)) for q in (G, c, eps))
    for i in range(k):
        cl[i].G, cl[i].c, cl[i].eps = float(Gs[i]), float(cs[i]), float(es[i])
    p = _params(float(Gs[0]), float(cs[0]), float(es[0]), precision, vel_mode, r_near,
                pair_kernel, integrator)
    h = ctypes.c_void_p()
    _check(lib.pn_init_batched(ctypes.byref(h), k, off.ctypes.data_as(ctypes.c_void_p),
                               ctypes.cast(cl, ctypes.c_void_p), ctypes.byref(p), int(device),
                               ctypes.c_void_p(_torch_stream(device, stream))))
    ctx = Context(h.value, int(off[-1]), int(device), p, offsets=off.tolist())
    ctx.batched = True
    return ctx


def pn_set_params(ctx: Context, G=None, c=None, eps=None, precision=None, vel_mode=None,
                  r_near=None, pair_kernel=None, integrator=None) -> None:
    q = ctx.params
    p = _params(q.G if G is None else G, q.c if c is None else c, q.eps if eps is None else eps,
                q.precision if precision is None else precision,
                q.vel_mode if vel_mode is None else vel_mode,
                q.r_near if r_near is None else r_near,
                q.pair_kernel if pair_kernel is None else pair_kernel,
                q.integrator if integrator is None else integrator)
    _check(_load().pn_set_params(ctx.handle, ctypes.byref(p)))
    ctx.params = p


def pn_set_stream(ctx: Context, stream) -> None:
    _check(_load().pn_set_stream(ctx.handle, ctypes.c_void_p(getattr(stream, "cuda_stream", stream))))


def _dev(ctx: Context, t, shape, name):
    return _dev_on(ctx.device, t, shape, name)


def _dev_on(device: int, t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor on cuda:{device}")
    if t.dtype != torch.float64 or not t.is_cuda or t.device.index != device:
        raise TypeError(f"{name} must be float64 on cuda:{device} (got {t.dtype}, {t.device})")
    if tuple(t.shape) != shape or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {shape} (got {tuple(t.shape)})")
    return ctypes.c_void_p(t.data_ptr())


def pn_accel(ctx: Context, x, v, m, a) -> None:
    """a = A(x, v) for all bodies (device tensors (n,3), (n,3), (n,), (n,3))."""
    n = ctx.n
    _check(_load().pn_accel(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                            _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a")))


def pn_jerk(ctx: Context, x, v, m, a, jerk) -> None:
    """a = A(x, v) and jerk = dA/dt along the trajectory (Appendix A), for
    all bodies; the jerk is computed in double precision."""
    n = ctx.n
    _check(_load().pn_jerk(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                           _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a"),
                           _dev(ctx, jerk, (n, 3), "jerk")))


def pn_accel_vjp(ctx: Context, x, v, m, abar, xbar, vbar) -> np.ndarray:
    """xbar, vbar = abar . dA/dx, abar . dA/dv (device tensors); returns the
    host array [M_bar, inv_c2_bar] per cluster, shape (n_clusters, 2)."""
    n = ctx.n
    scal = np.zeros(2 * ctx.n_clusters)
    _check(_load().pn_accel_vjp(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                                _dev(ctx, m, (n,), "m"), _dev(ctx, abar, (n, 3), "abar"),
                                _dev(ctx, xbar, (n, 3), "xbar"), _dev(ctx, vbar, (n, 3), "vbar"),
                                scal.ctypes.data_as(ctypes.c_void_p)))
    return scal.reshape(-1, 2)


def pn_step_vjp(ctx: Context, x0, v0, m, dt: float, nsteps: int, xbar_T, vbar_T, xbar0, vbar0,
                checkpoint: int = 0) -> np.ndarray:
    """Gradient of <xbar_T, x_T> + <vbar_T, v_T> through nsteps KDK steps from
    (x0, v0): writes xbar0, vbar0; returns [M_bar, inv_c2_bar] per cluster."""
    n = ctx.n
    scal = np.zeros(2 * ctx.n_clusters)
    _check(_load().pn_step_vjp(ctx.handle, _dev(ctx, x0, (n, 3), "x0"), _dev(ctx, v0, (n, 3), "v0"),
                               _dev(ctx, m, (n,), "m"), float(dt), int(nsteps), int(checkpoint),
                               _dev(ctx, xbar_T, (n, 3), "xbar_T"),
                               _dev(ctx, vbar_T, (n, 3), "vbar_T"),
                               _dev(ctx, xbar0, (n, 3), "xbar0"), _dev(ctx, vbar0, (n, 3), "vbar0"),
                               scal.ctypes.data_as(ctypes.c_void_p)))
    return scal.reshape(-1, 2)


def checkpoint_interval(nsteps: int, checkpoint: int = 0) -> int:
    """Steps between the checkpoints of pn_step_save / pn_step_vjp: checkpoint,
    or for 0 the integer ceiling of sqrt(nsteps)."""
    if checkpoint:
        return int(checkpoint)
    k = 1
    while k * k < nsteps:
        k += 1
    return k


def pn_step_save(ctx: Context, x, v, m, a, dt: float, nsteps: int, checkpoint: int = 0):
    """pn_step that also keeps the adjoint's checkpoints: returns a device
    tensor of ceil(nsteps / K) x 3 x n x 3 doubles (x, v, a before steps 0,
    K, 2K, ...) for pn_step_vjp_saved."""
    import torch
    n = ctx.n
    k = checkpoint_interval(nsteps, checkpoint)
    ncp = (nsteps + k - 1) // k if nsteps > 0 else 0
    ckpt = torch.empty((max(ncp, 1), 3, n, 3), dtype=torch.float64, device=f"cuda:{ctx.device}")
    _check(_load().pn_step_save(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                                _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a"), float(dt),
                                int(nsteps), int(checkpoint), ckpt.data_ptr()))
    return ckpt


def pn_step_vjp_saved(ctx: Context, ckpt, m, dt: float, nsteps: int, xbar_T, vbar_T, xbar0,
                      vbar0, checkpoint: int = 0) -> np.ndarray:
    """pn_step_vjp from the checkpoints pn_step_save returned (same m, dt,
    nsteps, checkpoint): writes xbar0, vbar0; returns [M_bar, inv_c2_bar]
    per cluster."""
    n = ctx.n
    scal = np.zeros(2 * ctx.n_clusters)
    _check(_load().pn_step_vjp_saved(ctx.handle, ckpt.data_ptr(), _dev(ctx, m, (n,), "m"),
                                     float(dt), int(nsteps), int(checkpoint),
                                     _dev(ctx, xbar_T, (n, 3), "xbar_T"),
                                     _dev(ctx, vbar_T, (n, 3), "vbar_T"),
                                     _dev(ctx, xbar0, (n, 3), "xbar0"),
                                     _dev(ctx, vbar0, (n, 3), "vbar0"),
                                     scal.ctypes.data_as(ctypes.c_void_p)))
    return scal.reshape(-1, 2)


def trajectory(ctx: Context, x0, v0, m, M, c, dt: float, nsteps: int, checkpoint: int = 0):
    """Differentiable nsteps of KDK (single-cluster context): returns (x_T,
    v_T) as torch tensors whose backward gives gradients with respect to x0,
    v0, the hole mass M and c (0-d tensors); m[0] is replaced by M and the
    context's c by c.  The forward runs pn_step_save (pn_step keeping the
    adjoint's checkpoints), the backward pn_step_vjp_saved."""
    import torch
    return _Trajectory.apply(x0, v0, M, c, m, ctx, float(dt), int(nsteps), int(checkpoint))


def _trajectory_class():
    import torch

    class Trajectory(torch.autograd.Function):
        @staticmethod
        def forward(fctx, x0, v0, M, c, m, ctx, dt, nsteps, checkpoint):
            mm = m.detach().clone()
            mm[0] = M.detach()
            cc = float(c.detach())
            pn_set_params(ctx, c=cc)
            x, v = x0.detach().clone(), v0.detach().clone()
            a = torch.empty_like(x)
            pn_accel(ctx, x, v, mm, a)
            if ctx.params.integrator == PN_KDK:
                ckpt = pn_step_save(ctx, x, v, mm, a, dt, nsteps, checkpoint)
            else:                   # no adjoint: the backward reports it
                pn_step(ctx, x, v, mm, a, dt, nsteps)
                ckpt = None
            pn_sync(ctx)
            fctx.save_for_backward(x0.detach(), v0.detach(), mm)
            fctx.ckpt = ckpt
            fctx.args = (ctx, dt, nsteps, checkpoint, cc)
            return x, v

        @staticmethod
        def backward(fctx, gx, gv):
            x0, v0, mm = fctx.saved_tensors
            ctx, dt, nsteps, checkpoint, cc = fctx.args
            gx = torch.zeros_like(x0) if gx is None else gx.contiguous()
            gv = torch.zeros_like(v0) if gv is None else gv.contiguous()
            xb, vb = torch.empty_like(x0), torch.empty_like(v0)
            pn_set_params(ctx, c=cc)
            if fctx.ckpt is not None:
                scal = pn_step_vjp_saved(ctx, fctx.ckpt, mm, dt, nsteps, gx, gv, xb, vb,
                                         checkpoint)
            else:
                scal = pn_step_vjp(ctx, x0, v0, mm, dt, nsteps, gx, gv, xb, vb, checkpoint)
            Mb = torch.tensor(scal[0, 0], dtype=x0.dtype, device=x0.device)
            cb = torch.tensor(-2.0 * scal[0, 1] / cc ** 3, dtype=x0.dtype, device=x0.device)
            return xb, vb, Mb, cb, None, None, None, None, None

    return Trajectory


class _LazyTrajectory:
    _cls = None

    def apply(self, *args):
        if _LazyTrajectory._cls is None:
            _LazyTrajectory._cls = _trajectory_class()
        return _LazyTrajectory._cls.apply(*args)


_Trajectory = _LazyTrajectory()


def pn_step(ctx: Context, x, v, m, a, dt: float, nsteps: int = 1) -> None:
    """nsteps KDK steps in place; a must hold A at the entry state."""
    n = ctx.n
    _check(_load().pn_step(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                           _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a"), float(dt),
                           int(nsteps)))


def pn_step_graph(ctx: Context, x, v, m, a, dt: float, nsteps: int) -> None:
    """pn_step recorded once into a CUDA graph per (arrays, dt, nsteps) and
    replayed with one launch."""
    n = ctx.n
    _check(_load().pn_step_graph(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                                 _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a"), float(dt),
                                 int(nsteps)))


def pn_tune(ctx: Context, x, v, m, a) -> dict:
    """Choose the fused kernel's launch shape (targets per thread, unroll,
    packed kernel, j-tile, buffers) by timing candidates on this state (a is
    overwritten with A(x, v)); cached per work bucket, precision and cluster
    class, and in the file PN_TUNE_CACHE names, if any."""
    n = ctx.n
    out = np.zeros(6, dtype=np.int64)
    _check(_load().pn_tune(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                           _dev(ctx, m, (n,), "m"), _dev(ctx, a, (n, 3), "a"),
                           out.ctypes.data_as(ctypes.c_void_p)))
    return {"targets_per_thread": int(out[0]), "unroll": int(out[1]), "cached": bool(out[2]),
            "packed": bool(out[3]), "tile": int(out[4]), "stages": int(out[5])}


def _host(arr, shape, name):
    if not isinstance(arr, np.ndarray) or arr.dtype != np.float64 or arr.shape != shape \
            or not arr.flags.c_contiguous or not arr.flags.writeable:
        raise TypeError(f"{name} must be a writeable C-contiguous float64 numpy array {shape}")
    return arr.ctypes.data_as(ctypes.c_void_p)


def pn_step_host(ctx: Context, x, v, m, a, dt: float, nsteps: int = 1) -> None:
    """pn_step on host (numpy) arrays, copies included; waits for the result."""
    n = ctx.n
    _check(_load().pn_step_host(ctx.handle, _host(x, (n, 3), "x"), _host(v, (n, 3), "v"),
                                _host(m, (n,), "m"), _host(a, (n, 3), "a"), float(dt),
                                int(nsteps)))


def pn_energy(ctx: Context, x, v, m):
    """Eq. 7 energy and Eq. 8 momentum, as a dict like the oracle's (a list
    of dicts, one per cluster, on a batched context).  Pair sums in FP64
    (FP64 context) or double-single (mixed context), the rest in FP64."""
    n = ctx.n
    out = np.zeros(8 * ctx.n_clusters)
    _check(_load().pn_energy(ctx.handle, _dev(ctx, x, (n, 3), "x"), _dev(ctx, v, (n, 3), "v"),
                             _dev(ctx, m, (n,), "m"), out.ctypes.data_as(ctypes.c_void_p)))
    res = []
    for k in range(ctx.n_clusters):
        o = out[8 * k:8 * k + 8]
        res.append({"E_N": o[0], "E_PN": o[1], "E": o[0] + o[1], "P_N": o[2:5].copy(),
                    "P_PN": o[5:8].copy(), "P": o[2:5] + o[5:8]})
    return res if getattr(ctx, "batched", False) else res[0]


def pn_energy_noalloc(x, v, m, out, G: float = 1.0, c: float = math.inf, eps: float = 0.0,
                      device: int | None = None, stream=None) -> None:
    """pn_energy without a context and without any device allocation (for
    callers whose device memory is owned by another allocator): writes the 8
    results of pn_energy into the device tensor `out` (float64, shape (8,)),
    asynchronously on `stream`.  At most PN_NOALLOC_MAX_BODIES (16384)
    bodies; concurrent calls on overlapping streams race on the library's
    shared scratch."""
    import torch
    if device is None:
        device = x.device.index
    n = int(m.shape[0])
    args = (_dev_on(device, x, (n, 3), "x"), _dev_on(device, v, (n, 3), "v"),
            _dev_on(device, m, (n,), "m"), _dev_on(device, out, (8,), "out"))
    st = torch.cuda.current_stream(device).cuda_stream if stream is None \
        else getattr(stream, "cuda_stream", stream)
    _check(_load().pn_energy_noalloc(int(device), ctypes.c_void_p(st), n, float(G), float(c),
                                     float(eps), *args))


def pn_measure_peaks(device: int = 0, stream=None) -> dict:
    """FP32, packed FP32x2 and FP64 FMA TFLOP/s and rsqrt Gop/s measured now on
    `device`."""
    import torch
    out = np.zeros(5)
    st = torch.cuda.current_stream(device).cuda_stream if stream is None \
        else getattr(stream, "cuda_stream", stream)
    _check(_load().pn_measure_peaks(int(device), ctypes.c_void_p(st),
                                    out.ctypes.data_as(ctypes.c_void_p)))
    return {"fp32_fma_tflops": out[0], "fp64_fma_tflops": out[1], "rsqrt_gops": out[2],
            "sms": int(out[3]), "fp32x2_fma_tflops": out[4]}


def pn_set_watchdog(ctx: Context, rel_tol: float, every: int = 100) -> None:
    """Energy-drift watchdog: every `every` steps compare Eq. 7's energy with
    the first check's; a relative change above rel_tol makes the next waiting
    call raise PNError with status PN_EDRIFT.  rel_tol = 0 turns it off."""
    _check(_load().pn_set_watchdog(ctx.handle, float(rel_tol), int(every)))


def pn_sync(ctx: Context) -> None:
    _check(_load().pn_sync(ctx.handle))


def pn_set_timing(ctx: Context, enable: bool) -> None:
    _check(_load().pn_set_timing(ctx.handle, 1 if enable else 0))


def pn_get_timing(ctx: Context):
    """(milliseconds, launches) of pass 1, pass 2 and the near-source pass
    since timing was enabled."""
    ms = np.zeros(3)
    nl = np.zeros(3, dtype=np.int64)
    _check(_load().pn_get_timing(ctx.handle, ms.ctypes.data_as(ctypes.c_void_p),
                                 nl.ctypes.data_as(ctypes.c_void_p)))
    return ms, nl


def pn_get_pair_stats(ctx: Context) -> tuple[int, int]:
    """(far units, all units) of the spatially ordered packed kernel since
    pn_init or the last pn_set_timing(ctx, True)."""
    out = np.zeros(2, dtype=np.int64)
    _check(_load().pn_get_pair_stats(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    return int(out[0]), int(out[1])


def pn_get_launch(ctx: Context) -> dict:
    out = np.zeros(8, dtype=np.int64)
    _check(_load().pn_get_launch(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    keys = ("threads", "targets_per_thread", "tile", "blocks_i", "jsplit", "occupancy", "sms",
            "packed")
    return {k: int(v) for k, v in zip(keys, out)}


def pn_get_variant(ctx: Context) -> dict:
    """The fused pair kernel's instantiation: targets per thread, unroll,
    form (0 dot product, 1 law of cosines, 2 law of cosines on the spatial
    order), tile, stages, packed (all 0 off the fused kernel)."""
    out = np.zeros(6, dtype=np.int64)
    _check(_load().pn_get_variant(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    keys = ("targets_per_thread", "unroll", "form", "tile", "stages", "packed")
    return {k: int(v) for k, v in zip(keys, out)}


def pn_launch_count(ctx: Context) -> int:
    """Kernels the context has launched so far (graph replays included)."""
    out = ctypes.c_int64(0)
    _check(_load().pn_launch_count(ctx.handle, ctypes.byref(out)))
    return int(out.value)


def pn_destroy(ctx: Context) -> None:
    ctx.close()
