// pn_api.cu -- the C ABI of libpn (declared in include/pn.h): argument
// checks, context and scratch management, the integrator loop and the
// device-side error report.  The arithmetic is in pn_kernels.cu.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pn_internal.h"

namespace {

thread_local char g_err[512] = "";

pn_status fail(pn_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

pn_status ok()
{
    g_err[0] = '\0';
    return PN_OK;
}

#define PN_CUDA(call, what)                                                         \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(PN_ECUDA, "%s: %s", what, cudaGetErrorString(e_));          \
    } while (0)

// Makes the context's device current for the duration of a call and
// restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if ((err = cudaGetDevice(&prev)) == cudaSuccess && prev != dev)
            err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

bool params_ok(const pn_params *p)
{
    if (!p)
        return (void)fail(PN_EINVAL, "params is NULL"), false;
    if (!(std::isfinite(p->G) && p->G > 0.0))
        return (void)fail(PN_EINVAL, "G must be finite and > 0 (got %g)", p->G), false;
    if (!(p->c > 0.0))   // INFINITY allowed, NaN and <= 0 rejected
        return (void)fail(PN_EINVAL, "c must be > 0 or INFINITY (got %g)", p->c), false;
    if (!(std::isfinite(p->eps) && p->eps >= 0.0))
        return (void)fail(PN_EINVAL, "eps must be finite and >= 0 (got %g)", p->eps), false;
    if (p->precision != PN_FP64 && p->precision != PN_MIXED)
        return (void)fail(PN_EINVAL, "precision must be PN_FP64 or PN_MIXED (got %d)",
                          p->precision), false;
    if (p->vel_mode != PN_VPRED_END && p->vel_mode != PN_VHALF)
        return (void)fail(PN_EINVAL, "vel_mode must be PN_VPRED_END or PN_VHALF (got %d)",
                          p->vel_mode), false;
    if (!(std::isfinite(p->r_near) && p->r_near >= 0.0))
        return (void)fail(PN_EINVAL, "r_near must be finite and >= 0 (got %g)", p->r_near), false;
    if (p->pair_kernel != PN_PAIR_FUSED && p->pair_kernel != PN_PAIR_TWO_PASS)
        return (void)fail(PN_EINVAL, "pair_kernel must be PN_PAIR_FUSED or PN_PAIR_TWO_PASS (got %d)",
                          p->pair_kernel), false;
    if (p->integrator != PN_KDK && p->integrator != PN_RK4)
        return (void)fail(PN_EINVAL, "integrator must be PN_KDK or PN_RK4 (got %d)", p->integrator),
               false;
    return true;
}

void set_params(pn_ctx *c, const pn_params *p)
{
    c->p = *p;
    c->inv_c2 = std::isinf(p->c) ? 0.0 : 1.0 / (p->c * p->c);
}

void free_all(pn_ctx *c)
{
    void *bufs[] = {c->vp, c->mrec, c->drec, c->part, c->blk, c->glob, c->eout, c->flag,
                    c->flag_step, c->hx, c->hv, c->hm, c->ha, c->nrec, c->ndrec, c->ncount,
                    c->nflag, c->rk_x, c->rk_v, c->rk_a, c->rk_sx, c->rk_sv};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    if (c->timing_on || c->tm.ev0[0][0]) {
        for (int k = 0; k < pn::Timing::kKernels; ++k)
            for (int r = 0; r < pn::Timing::kRing; ++r) {
                if (c->tm.ev0[k][r])
                    cudaEventDestroy(c->tm.ev0[k][r]);
                if (c->tm.ev1[k][r])
                    cudaEventDestroy(c->tm.ev1[k][r]);
            }
    }
}

pn_status check_ctx(pn_ctx *c)
{
    if (!c)
        return fail(PN_EINVAL, "context is NULL");
    return PN_OK;
}

// Reads and clears the device's non-finite flag (stream must be idle).
pn_status report_flag(pn_ctx *c)
{
    int flag = 0;
    unsigned long long step = 0;
    PN_CUDA(cudaMemcpyAsync(&flag, c->flag, sizeof flag, cudaMemcpyDeviceToHost, c->stream),
            "read non-finite flag");
    PN_CUDA(cudaMemcpyAsync(&step, c->flag_step, sizeof step, cudaMemcpyDeviceToHost, c->stream),
            "read non-finite step");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    if (flag) {
        const unsigned long long none = ULLONG_MAX;
        PN_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream), "clear flag");
        PN_CUDA(cudaMemcpyAsync(c->flag_step, &none, sizeof none, cudaMemcpyHostToDevice,
                                c->stream), "clear flag step");
        PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
        return fail(PN_ENONFINITE, "non-finite acceleration produced (first at step %llu)", step);
    }
    return PN_OK;
}

// One evaluation of A(x, vel) into a (kick v by h a if v != NULL).
pn_status evaluate(pn_ctx *c, const double *x, const double *vel, const double *m, double *a,
                   double *v, double h)
{
    PN_CUDA(pn::launch_prologue(c, x, vel, m, false), "prologue launch");
    if (pn::use_fused(c)) {
        PN_CUDA(pn::launch_fused(c), "fused pair launch");
    } else {
        PN_CUDA(pn::launch_pass1(c), "pass-1 launch");
        PN_CUDA(pn::launch_pass2(c), "pass-2 launch");
    }
    PN_CUDA(pn::launch_near(c), "near-pass launch");
    PN_CUDA(pn::launch_epilogue(c, x, vel, m, a, v, h, (unsigned long long)c->step_counter),
            "epilogue launch");
    return PN_OK;
}

pn_status run_rk4(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                  int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) {
        c->step_counter += 1;
        for (int stage = 0; stage < 3; ++stage) {
            PN_CUDA(pn::launch_rk4_stage(c, stage, x, v, a, dt), "rk4 stage launch");
            pn_status st = evaluate(c, c->rk_x, c->rk_v, m, c->rk_a, nullptr, 0.0);
            if (st != PN_OK)
                return st;
        }
        PN_CUDA(pn::launch_rk4_stage(c, 3, x, v, a, dt), "rk4 stage launch");
        pn_status st = evaluate(c, x, v, m, a, nullptr, 0.0);
        if (st != PN_OK)
            return st;
    }
    return PN_OK;
}

pn_status run_steps(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                    int64_t nsteps)
{
    if (c->p.integrator == PN_RK4)
        return run_rk4(c, x, v, m, a, dt, nsteps);
    for (int64_t s = 0; s < nsteps; ++s) {
        c->step_counter += 1;
        PN_CUDA(pn::launch_kick_drift(c, x, v, a, dt), "kick-drift launch");
        pn_status st = evaluate(c, x, c->vp, m, a, v, 0.5 * dt);
        if (st != PN_OK)
            return st;
    }
    return PN_OK;
}

}  // namespace

namespace pn {

// Records an error message for pn_last_error from other translation units.
pn_status set_error(pn_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

}  // namespace pn

extern "C" {

int pn_version(void) { return 100; }

const char *pn_last_error(void) { return g_err; }

pn_status pn_init(pn_ctx **out, int64_t n, const pn_params *params, int device,
                  void *cuda_stream)
{
    if (!out)
        return fail(PN_EINVAL, "ctx output pointer is NULL");
    *out = nullptr;
    if (n < 2)
        return fail(PN_EINVAL, "n must be >= 2 (the hole and at least one star), got %lld",
                    (long long)n);
    if (n > ((int64_t)1 << 31))
        return fail(PN_EINVAL, "n = %lld exceeds the supported 2^31 bodies", (long long)n);
    if (!params_ok(params))
        return PN_EINVAL;
    const char *inj = std::getenv("PN_FAIL_ALLOC");
    if (inj && inj[0] == '1')
        return fail(PN_ENOMEM, "allocation failure injected by PN_FAIL_ALLOC");
    int ndev = 0;
    PN_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev)
        return fail(PN_EINVAL, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard g(device);
    PN_CUDA(g.err, "cudaSetDevice");
    int major = 0, minor = 0, sms = 0;
    PN_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device), "attr");
    PN_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device), "attr");
    PN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "attr");
    if (major != 10 || minor != 3)
        return fail(PN_EUNSUPPORTED, "libpn is built for sm_103a; device %d is sm_%d%d", device,
                    major, minor);

    pn_ctx *c = new (std::nothrow) pn_ctx();
    if (!c)
        return fail(PN_ENOMEM, "host allocation of the context failed");
    c->n = n;
    c->ns = n - 1;
    c->ns_pad = (c->ns + pn::kPad - 1) / pn::kPad * pn::kPad;
    set_params(c, params);
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->sm_count = sms;
    int occ_mix = 0, occ_f64 = 0, occ_fused = 0;
    cudaError_t e = pn::occupancy(&occ_mix, &occ_f64);
    // fused-kernel variant; PN_FUSED_TARGETS / PN_FUSED_UNROLL override (tuning)
    c->fused_P = 4;          // measured fastest on B300 at N = 131072 (4 targets x 2-way unroll)
    c->fused_unroll = 2;
    if (const char *tp = std::getenv("PN_FUSED_TARGETS")) {
        const int v = std::atoi(tp);
        if (v == 1 || v == 2 || v == 4)
            c->fused_P = v;
    }
    if (const char *tu = std::getenv("PN_FUSED_UNROLL")) {
        const int v = std::atoi(tu);
        if (v >= 1 && v <= 4)
            c->fused_unroll = v;
    }
    if (e == cudaSuccess)
        e = pn::fused_occupancy(c->fused_P, c->fused_unroll, &occ_fused);
    if (e != cudaSuccess) {
        delete c;
        return fail(PN_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    }
    pn::shapes(c->ns_pad, sms, occ_mix, occ_f64, &c->mix, &c->f64);
    c->fused_occ = occ_fused > 0 ? occ_fused : 1;
    c->fused_G = (int64_t)c->fused_occ * sms;
    c->fused_segs = (int)pn::fused_segments(c->ns_pad, c->fused_G, c->fused_P);

    const int64_t np = c->ns_pad;
    int64_t part = (int64_t)c->mix.jsplit * (pn::kP1Vals + pn::kP2Vals) * np;
    const int64_t part_f64 = (int64_t)c->f64.jsplit * (pn::kP1Vals + pn::kP2Vals) * np;
    const int64_t part_e = (int64_t)c->f64.jsplit * pn::kEVals * np;
    if (part_f64 > part)
        part = part_f64;
    if (part_e > part)
        part = part_e;
    part += (int64_t)pn::kNearVals * np;   // near-pass partials after both passes
    const int64_t part_fused = (int64_t)(pn::kP1Vals + pn::kP2Vals + pn::kNearVals) * np +
                               c->fused_G * c->fused_segs * pn::kFusedVals *
                                   (pn::kMixThreads * c->fused_P);
    if (part_fused > part)
        part = part_fused;
    c->part_len = part;
    const int64_t nglue = (np + pn::kGlueThreads - 1) / pn::kGlueThreads;
    c->blk_len = nglue * pn::kGlobVals;
    c->nnear_cap = np + pn::kNearTile;

    struct Req { void **p; size_t bytes; } req[] = {
        {(void **)&c->vp, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_x, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_v, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_a, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_sx, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_sv, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->mrec, sizeof(float4) * 5 * (size_t)np},
        {(void **)&c->drec, sizeof(double4_32a) * 4 * (size_t)np},
        {(void **)&c->part, sizeof(double) * (size_t)part},
        {(void **)&c->blk, sizeof(double) * (size_t)c->blk_len},
        {(void **)&c->glob, sizeof(double) * 16},
        {(void **)&c->nrec, sizeof(float4) * 4 * (size_t)c->nnear_cap},
        {(void **)&c->ndrec, sizeof(double4_32a) * 3 * (size_t)c->nnear_cap},
        {(void **)&c->ncount, sizeof(int) * (size_t)(1 + nglue)},
        {(void **)&c->nflag, (size_t)np},
        {(void **)&c->eout, sizeof(double) * 8},
        {(void **)&c->flag, sizeof(int)},
        {(void **)&c->flag_step, sizeof(unsigned long long)},
    };
    for (auto &r : req) {
        e = cudaMalloc(r.p, r.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_all(c);
            delete c;
            return fail(PN_ENOMEM, "cudaMalloc of %zu bytes failed: %s", r.bytes,
                        cudaGetErrorString(e));
        }
    }
    const unsigned long long none = ULLONG_MAX;
    e = cudaMemset(c->flag, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->flag_step, &none, sizeof none, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(PN_ECUDA, "initialising the error flag: %s", cudaGetErrorString(e));
    }
    *out = c;
    return ok();
}

pn_status pn_set_params(pn_ctx *c, const pn_params *params)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!params_ok(params))
        return PN_EINVAL;
    set_params(c, params);
    return ok();
}

pn_status pn_set_stream(pn_ctx *c, void *cuda_stream)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return ok();
}

pn_status pn_accel(pn_ctx *c, const double *x, const double *v, const double *m, double *a)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a)
        return fail(PN_EINVAL, "pn_accel: NULL array");
    if (a == x || a == v || (const void *)a == (const void *)m)
        return fail(PN_EINVAL, "pn_accel: a aliases an input");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    PN_CUDA(cudaMemcpyAsync(c->vp, v, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDeviceToDevice,
                            c->stream), "copy velocities");
    pn_status st = evaluate(c, x, c->vp, m, a, nullptr, 0.0);
    return st == PN_OK ? ok() : st;
}

pn_status pn_step(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                  int64_t nsteps)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a)
        return fail(PN_EINVAL, "pn_step: NULL array");
    if (!(std::isfinite(dt) && dt > 0.0))
        return fail(PN_EINVAL, "pn_step: dt must be finite and > 0 (got %g)", dt);
    if (nsteps < 0)
        return fail(PN_EINVAL, "pn_step: nsteps must be >= 0");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    pn_status st = run_steps(c, x, v, m, a, dt, nsteps);
    return st == PN_OK ? ok() : st;
}

pn_status pn_step_host(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                       int64_t nsteps)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a)
        return fail(PN_EINVAL, "pn_step_host: NULL array");
    if (!(std::isfinite(dt) && dt > 0.0))
        return fail(PN_EINVAL, "pn_step_host: dt must be finite and > 0 (got %g)", dt);
    if (nsteps < 0)
        return fail(PN_EINVAL, "pn_step_host: nsteps must be >= 0");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    const size_t b3 = sizeof(double) * 3 * (size_t)c->n, b1 = sizeof(double) * (size_t)c->n;
    if (!c->hx) {
        void **p[] = {(void **)&c->hx, (void **)&c->hv, (void **)&c->ha};
        for (void **q : p) {
            cudaError_t e = cudaMalloc(q, b3);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(PN_ENOMEM, "cudaMalloc for host-array staging failed");
            }
        }
        if (cudaMalloc((void **)&c->hm, b1) != cudaSuccess) {
            cudaGetLastError();
            return fail(PN_ENOMEM, "cudaMalloc for host-array staging failed");
        }
    }
    PN_CUDA(cudaMemcpyAsync(c->hx, x, b3, cudaMemcpyHostToDevice, c->stream), "copy x in");
    PN_CUDA(cudaMemcpyAsync(c->hv, v, b3, cudaMemcpyHostToDevice, c->stream), "copy v in");
    PN_CUDA(cudaMemcpyAsync(c->hm, m, b1, cudaMemcpyHostToDevice, c->stream), "copy m in");
    PN_CUDA(cudaMemcpyAsync(c->ha, a, b3, cudaMemcpyHostToDevice, c->stream), "copy a in");
    pn_status st = run_steps(c, c->hx, c->hv, c->hm, c->ha, dt, nsteps);
    if (st != PN_OK)
        return st;
    PN_CUDA(cudaMemcpyAsync(x, c->hx, b3, cudaMemcpyDeviceToHost, c->stream), "copy x out");
    PN_CUDA(cudaMemcpyAsync(v, c->hv, b3, cudaMemcpyDeviceToHost, c->stream), "copy v out");
    PN_CUDA(cudaMemcpyAsync(a, c->ha, b3, cudaMemcpyDeviceToHost, c->stream), "copy a out");
    st = report_flag(c);
    return st == PN_OK ? ok() : st;
}

pn_status pn_energy(pn_ctx *c, const double *x, const double *v, const double *m, double out[8])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !out)
        return fail(PN_EINVAL, "pn_energy: NULL array");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    PN_CUDA(pn::launch_energy(c, x, v, m), "energy launch");
    PN_CUDA(cudaMemcpyAsync(out, c->eout, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream),
            "copy energy out");
    pn_status st = report_flag(c);
    return st == PN_OK ? ok() : st;
}

pn_status pn_sync(pn_ctx *c)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    pn_status st = report_flag(c);
    return st == PN_OK ? ok() : st;
}

pn_status pn_set_timing(pn_ctx *c, int enable)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    if (enable && !c->tm.ev0[0][0]) {
        for (int k = 0; k < pn::Timing::kKernels; ++k)
            for (int r = 0; r < pn::Timing::kRing; ++r) {
                PN_CUDA(cudaEventCreate(&c->tm.ev0[k][r]), "cudaEventCreate");
                PN_CUDA(cudaEventCreate(&c->tm.ev1[k][r]), "cudaEventCreate");
            }
    }
    for (int k = 0; k < pn::Timing::kKernels; ++k) {
        c->tm.head[k] = c->tm.count[k] = 0;
        c->tm.ms[k] = 0.0;
        c->tm.launches[k] = 0;
    }
    c->timing_on = enable ? 1 : 0;
    return ok();
}

pn_status pn_get_timing(pn_ctx *c, double ms[3], int64_t launches[3])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!ms || !launches)
        return fail(PN_EINVAL, "pn_get_timing: NULL output");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    for (int k = 0; k < pn::Timing::kKernels; ++k) {
        pn::Timing &t = c->tm;
        while (t.count[k] > 0) {
            const int old = t.head[k];
            float v = 0.0f;
            PN_CUDA(cudaEventElapsedTime(&v, t.ev0[k][old], t.ev1[k][old]), "event time");
            t.ms[k] += v;
            t.launches[k] += 1;
            t.head[k] = (old + 1) % pn::Timing::kRing;
            t.count[k] -= 1;
        }
        ms[k] = t.ms[k];
        launches[k] = t.launches[k];
    }
    return ok();
}

pn_status pn_get_launch(pn_ctx *c, int64_t out[7])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!out)
        return fail(PN_EINVAL, "pn_get_launch: NULL output");
    const pn::Shape &s = c->p.precision == PN_MIXED ? c->mix : c->f64;
    const bool fused = pn::use_fused(c);
    out[0] = s.threads;
    out[1] = fused ? c->fused_P : s.targets;
    out[2] = s.tile;
    out[3] = s.nblk_i;
    out[4] = fused ? c->fused_G : s.jsplit;
    out[5] = fused ? c->fused_occ : s.occupancy;
    out[6] = c->sm_count;
    return ok();
}

void pn_destroy(pn_ctx *c)
{
    if (!c)
        return;
    DeviceGuard g(c->device);
    if (g.err == cudaSuccess)
        cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
