// pn_api.cu -- the C ABI of libpn (declared in include/pn.h): argument
// checks, context and scratch management, the integrator loop and the
// device-side error report.  The arithmetic is in pn_kernels.cu.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
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
    if (p->integrator != PN_KDK && p->integrator != PN_RK4 && p->integrator != PN_HERMITE)
        return (void)fail(PN_EINVAL, "integrator must be PN_KDK, PN_RK4 or PN_HERMITE (got %d)",
                          p->integrator),
               false;
    return true;
}

double inv_c2_of(double c) { return std::isinf(c) ? 0.0 : 1.0 / (c * c); }

// Copies the host cluster table to the device (stream-ordered, then waits:
// table updates are rare and must not race with queued kernels).
pn_status upload_clusters(pn_ctx *c)
{
    PN_CUDA(cudaMemcpyAsync(c->d_clu, c->hclu, sizeof(pn::Clu) * (size_t)c->nclu,
                            cudaMemcpyHostToDevice, c->stream), "upload cluster table");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return PN_OK;
}

// Mode fields for every cluster; G, c, eps and r_near for every cluster too
// when `all_physics` (single-cluster contexts and pn_set_params).
void set_params(pn_ctx *c, const pn_params *p, bool all_physics)
{
    c->p = *p;
    c->any_near = false;
    c->near_all = true;
    for (int k = 0; k < c->nclu; ++k) {
        if (all_physics) {
            c->hclu[k].G = p->G;
            c->hclu[k].inv_c2 = inv_c2_of(p->c);
            c->hclu[k].eps2 = p->eps * p->eps;
            c->hclu[k].r_near = p->r_near > 0.0 ? p->r_near : -1.0;
        }
        if (c->hclu[k].r_near > 0.0)
            c->any_near = true;
        else
            c->near_all = false;
    }
}

void free_all(pn_ctx *c)
{
    void *bufs[] = {c->vp, c->mrec, c->sord, c->bal, c->drec, c->part, c->blk, c->glob, c->eout,
                    c->flag, c->wcount, c->units_cnt,
                    c->flag_step, c->hx, c->hv, c->hm, c->ha, c->nrec, c->ndrec, c->ncount,
                    c->nflag, c->rk_x, c->rk_v, c->rk_a, c->rk_sx, c->rk_sv, c->jbuf, c->hj0, c->hj1, c->abuf,
                    c->wd, c->wd_step, c->epi_done, c->d_clu,
                    c->blk_clu};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    if (c->graph_exec)
        cudaGraphExecDestroy(c->graph_exec);
    if (c->cap_stream)
        cudaStreamDestroy(c->cap_stream);
    if (c->side)
        cudaStreamDestroy(c->side);
    if (c->adj_stream)
        cudaStreamDestroy(c->adj_stream);
    if (c->ev_fork)
        cudaEventDestroy(c->ev_fork);
    if (c->ev_join)
        cudaEventDestroy(c->ev_join);
    delete[] c->hclu;
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
#ifdef PN_DEBUG_CHECKS
    {
        unsigned long long site = 0, s2 = 0;
        long long index = 0, i2 = 0;
        PN_CUDA(pn::debug_take_kernels(c->dbg_inject, &site, &index), "read debug checks");
        PN_CUDA(pn::debug_take_order(c->dbg_inject, &s2, &i2), "read debug checks");
        if (!site && s2) {
            site = s2;
            index = i2;
        }
        if (site)
            return fail(PN_EINDEX, "debug build: an index check failed at site %llu (index %lld)",
                        site, index);
    }
#endif
    if (flag) {
        const unsigned long long none = ULLONG_MAX;
        unsigned long long wstep = 0;
        double wval[2] = {0.0, -1.0};
        if ((flag & 4) && c->wd) {
            PN_CUDA(cudaMemcpyAsync(&wstep, c->wd_step, sizeof wstep, cudaMemcpyDeviceToHost,
                                    c->stream), "read watchdog step");
            PN_CUDA(cudaMemcpyAsync(wval, c->wd + c->nclu, sizeof wval, cudaMemcpyDeviceToHost,
                                    c->stream), "read watchdog change");
            PN_CUDA(cudaMemcpyAsync(c->wd_step, &none, sizeof none, cudaMemcpyHostToDevice,
                                    c->stream), "clear watchdog step");
        }
        PN_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream), "clear flag");
        PN_CUDA(cudaMemcpyAsync(c->flag_step, &none, sizeof none, cudaMemcpyHostToDevice,
                                c->stream), "clear flag step");
        PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
        if (flag & 2)
            return fail(PN_ETIMEOUT, "a bounded wait for a device copy gave up");
        if (flag & 1)
            return fail(PN_ENONFINITE, "non-finite acceleration produced (first at step %llu)",
                        step);
        return fail(PN_EDRIFT,
                    "energy drift |E - E_ref|/|E_ref| = %.6e above %.3e (cluster %d, first at "
                    "step %llu)", wval[0], c->wd_tol, (int)wval[1], wstep);
    }
    return PN_OK;
}

// One evaluation of A(x, vel) into a (kick v by h a if v != NULL).
pn_status evaluate(pn_ctx *c, const double *x, const double *vel, const double *m, double *a,
                   double *v, double h, double dt_next = 0.0)
{
    PN_CUDA(pn::launch_prologue(c, x, vel, m, false), "prologue launch");
    // The pair kernels read only the prologue's records: the cluster sums,
    // the near-source records and the near-source pass fork onto the side
    // stream once the prologue is done and run beside the pair kernel (in
    // the resources that kernel leaves, or in its tail), joining before the
    // epilogue, which reads them all; they are launched after the pair
    // kernel, so that kernel's resident blocks all start at once.  (The
    // spatial order's sort reads the cluster sums: there they come first.)
    const bool sums_first = pn::pairs_need_sums(c);
    if (sums_first || !c->side)
        PN_CUDA(pn::launch_global_sums(c), "global sums launch");
    const bool fork = c->side != nullptr;
    if (!fork)
        PN_CUDA(pn::launch_near_scatter(c, x, m), "near scatter launch");
    if (fork)
        PN_CUDA(cudaEventRecord(c->ev_fork, c->stream), "fork event");
    if (pn::use_fused(c)) {
        PN_CUDA(pn::launch_fused(c), "fused pair launch");
    } else if (pn::use_fused_f64(c)) {
        PN_CUDA(pn::launch_fused_f64(c), "fused FP64 pair launch");
    } else {
        PN_CUDA(pn::launch_pass1(c), "pass-1 launch");
        PN_CUDA(pn::launch_pass2(c), "pass-2 launch");
    }
    if (fork) {
        PN_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork wait");
        cudaStream_t main = c->stream;
        c->stream = c->side;
        cudaError_t e = sums_first ? cudaSuccess : pn::launch_global_sums(c);
        if (e == cudaSuccess)
            e = pn::launch_near_scatter(c, x, m);
        if (e == cudaSuccess)
            e = pn::launch_near(c);
        c->stream = main;
        PN_CUDA(e, "side-stream launch");
        PN_CUDA(cudaEventRecord(c->ev_join, c->side), "join event");
        PN_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join wait");
    } else {
        PN_CUDA(pn::launch_near(c), "near-pass launch");
    }
    PN_CUDA(pn::launch_epilogue(c, x, vel, m, a, v, h, (unsigned long long)c->step_counter,
                                dt_next), "epilogue launch");
    return PN_OK;
}

// The energy-drift watchdog checks the state after this step.
bool watch_due(const pn_ctx *c)
{
    return c->wd_every > 0 && c->step_counter % c->wd_every == 0;
}

// The energy-drift watchdog's check after a step (pn_set_watchdog): Eq. 7
// on the state, compared on the device with the references.
pn_status watch(pn_ctx *c, const double *x, const double *v, const double *m)
{
    if (!watch_due(c))
        return PN_OK;
    PN_CUDA(pn::launch_energy(c, x, v, m), "watchdog energy launch");
    PN_CUDA(pn::launch_watch(c), "watchdog launch");
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
        if (st == PN_OK)
            st = watch(c, x, v, m);
        if (st != PN_OK)
            return st;
    }
    return PN_OK;
}

// Scratch of the jerk and the Hermite steps, allocated on first use (never
// inside a graph capture: pn_step_graph allocates it before capturing).
pn_status ensure_jerk_buffers(pn_ctx *c)
{
    if (c->jbuf)
        return PN_OK;
    const size_t b3 = sizeof(double) * 3 * (size_t)c->n;
    void **p[] = {(void **)&c->jbuf, (void **)&c->hj0, (void **)&c->hj1};
    const size_t bytes[] = {sizeof(double) * pn::jerk_buffer_doubles(c), b3, b3};
    for (int k = 0; k < 3; ++k) {
        if (*p[k])
            continue;
        if (std::getenv("PN_FAIL_ALLOC") || cudaMalloc(p[k], bytes[k]) != cudaSuccess) {
            cudaGetLastError();
            for (int q = 0; q < 3; ++q)
                if (*p[q]) {
                    cudaFree(*p[q]);
                    *p[q] = nullptr;
                }
            return fail(PN_ENOMEM, "cudaMalloc of %zu bytes for the jerk failed", bytes[k]);
        }
    }
    return PN_OK;
}

// Adjoint scratch (and the jerk's, whose records and sums it reuses).
pn_status ensure_adjoint_buffers(pn_ctx *c)
{
    pn_status st = ensure_jerk_buffers(c);
    if (st != PN_OK || c->abuf)
        return st;
    const size_t bytes = sizeof(double) * pn::adjoint_buffer_doubles(c);
    if (std::getenv("PN_FAIL_ALLOC") || cudaMalloc((void **)&c->abuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->abuf = nullptr;
        return fail(PN_ENOMEM, "cudaMalloc of %zu bytes for the adjoint failed", bytes);
    }
    return PN_OK;
}

// Fourth-order Hermite, predict-(evaluate-correct)^2; the stages are stated
// with pn_step in pn.h.  rk_x / rk_v hold (x_e, v_e), rk_a a_1, hj0 / hj1
// the jerks.
pn_status run_hermite(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                      int64_t nsteps)
{
    if (nsteps == 0)
        return PN_OK;
    pn_status st = ensure_jerk_buffers(c);
    if (st != PN_OK)
        return st;
    PN_CUDA(pn::launch_jerk(c, x, v, m, a, c->hj0), "jerk launch");
    for (int64_t s = 0; s < nsteps; ++s) {
        c->step_counter += 1;
        PN_CUDA(pn::launch_hermite(c, 0, x, v, a, c->hj0, nullptr, nullptr, c->rk_x, c->rk_v, dt),
                "hermite predict launch");
        for (int pass = 0; pass < 2; ++pass) {
            st = evaluate(c, c->rk_x, c->rk_v, m, c->rk_a, nullptr, 0.0);
            if (st != PN_OK)
                return st;
            PN_CUDA(pn::launch_jerk(c, c->rk_x, c->rk_v, m, c->rk_a, c->hj1), "jerk launch");
            PN_CUDA(pn::launch_hermite(c, 1, x, v, a, c->hj0, c->rk_a, c->hj1, c->rk_x, c->rk_v,
                                       dt), "hermite correct launch");
        }
        PN_CUDA(pn::launch_hermite(c, 2, x, v, a, c->hj0, c->rk_a, c->hj1, c->rk_x, c->rk_v, dt),
                "hermite commit launch");
        if ((st = watch(c, x, v, m)) != PN_OK)
            return st;
    }
    return evaluate(c, x, v, m, a, nullptr, 0.0);
}

pn_status run_steps(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                    int64_t nsteps)
{
    if (c->p.integrator == PN_RK4)
        return run_rk4(c, x, v, m, a, dt, nsteps);
    if (c->p.integrator == PN_HERMITE)
        return run_hermite(c, x, v, m, a, dt, nsteps);
    bool drifted = false;   // the previous epilogue took this step's kick and drift
    for (int64_t s = 0; s < nsteps; ++s) {
        c->step_counter += 1;
        if (!drifted)
            PN_CUDA(pn::launch_kick_drift(c, x, v, a, dt), "kick-drift launch");
        // the next step's kick and drift ride on this step's epilogue, except
        // after the call's last step and where the watchdog reads the state
        const bool fuse = s + 1 < nsteps && !watch_due(c);
        pn_status st = evaluate(c, x, c->vp, m, a, v, 0.5 * dt, fuse ? dt : 0.0);
        if (st == PN_OK)
            st = watch(c, x, v, m);
        if (st != PN_OK)
            return st;
        drifted = fuse;
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

int pn_debug_checks(void)
{
#ifdef PN_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

const char *pn_last_error(void) { return g_err; }

// Context for one or more clusters: cluster k holds bodies
// [off[k], off[k+1]) of the state arrays, its hole first.  Per-cluster G, c,
// eps come from `cp` (NULL: all from `params`).
static pn_status init_common(pn_ctx **out, int nclu, const int64_t *off, const pn_cluster *cp,
                             const pn_params *params, int device, void *cuda_stream)
{
    if (!params_ok(params))
        return PN_EINVAL;
    const int64_t n = off[nclu];
    if (n > ((int64_t)1 << 31) - (int64_t)nclu * pn::kPad)
        return fail(PN_EINVAL, "n = %lld exceeds the supported 2^31 bodies", (long long)n);
    for (int k = 0; k < nclu; ++k) {
        if (off[k + 1] - off[k] < 2)
            return fail(PN_EINVAL, "cluster %d has %lld bodies (need the hole and a star)", k,
                        (long long)(off[k + 1] - off[k]));
        if (cp) {
            const pn_cluster &q = cp[k];
            if (!(std::isfinite(q.G) && q.G > 0.0) || !(q.c > 0.0) ||
                !(std::isfinite(q.eps) && q.eps >= 0.0))
                return fail(PN_EINVAL, "cluster %d: need G > 0, c > 0 (or INFINITY), eps >= 0", k);
        }
    }
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
    c->hclu = new (std::nothrow) pn::Clu[nclu]();
    if (!c->hclu) {
        delete c;
        return fail(PN_ENOMEM, "host allocation of the cluster table failed");
    }
    c->n = n;
    c->nclu = nclu;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->sm_count = sms;
    int64_t slot = 0, nearc = 0, maxp = 0;
    for (int k = 0; k < nclu; ++k) {
        pn::Clu &C = c->hclu[k];
        C.body0 = off[k];
        C.ns = off[k + 1] - off[k] - 1;
        C.ns_pad = (C.ns + pn::kPad - 1) / pn::kPad * pn::kPad;
        C.slot0 = slot;
        C.near0 = nearc;
        slot += C.ns_pad;
        nearc += C.ns_pad + pn::kNearTile;
        if (C.ns_pad > maxp)
            maxp = C.ns_pad;
        const double G = cp ? cp[k].G : params->G, cc = cp ? cp[k].c : params->c,
                     eps = cp ? cp[k].eps : params->eps;
        C.G = G;
        C.inv_c2 = inv_c2_of(cc);
        C.eps2 = eps * eps;
        C.r_near = params->r_near > 0.0 ? params->r_near : -1.0;
    }
    c->S = slot;
    c->NC = nearc;
    c->max_ns_pad = maxp;
    set_params(c, params, false);

    int occ_mix = 0, occ_f64 = 0;
    cudaError_t e = pn::occupancy(&occ_mix, &occ_f64);
    // fused-kernel variant; PN_FUSED_PACKED / PN_FUSED_TARGETS / PN_FUSED_UNROLL /
    // PN_FUSED_WORKERS override the default (tuning sweeps)
    c->fused_packed = true;  // packed FP32x2 kernel, 4 targets per thread, no unroll:
    c->fused_P = 4;          // measured fastest on B300 at N = 131072 (22.11 ms
    c->fused_unroll = 1;     // against 22.50 with the 2-way unroll)
    // small systems: 2 targets per thread (4 resident blocks per SM, shorter
    // target blocks) with the 2-way unroll, measured 8 % faster per step at
    // N = 8192 and 1 % at 16384 (the unroll: 455 against 461 us at 16384)
    if (c->max_ns_pad <= 16384) {
        c->fused_P = 2;
        c->fused_unroll = 2;
    }
    c->fused_tile = pn::kPackTile;
    c->fused_stages = pn::kPackStages;
    c->workers_max = pn::kPackWorkersMax;
    c->worker_units = 64;
    if (const char *wu = std::getenv("PN_WORKER_UNITS")) {
        const int v = std::atoi(wu);
        if (v >= 1 && v <= 4096)
            c->worker_units = v;
    }
    // test hook: PN_INJECT_COPY_TIMEOUT=1 makes every tile barrier of the
    // packed kernel expect 16 bytes that never arrive, so its bounded waits
    // run out and pn_sync reports PN_ETIMEOUT
    c->inject_tx = 0;
    if (const char *ij = std::getenv("PN_INJECT_COPY_TIMEOUT"))
        c->inject_tx = ij[0] == '1' ? 16u : 0u;
#ifdef PN_DEBUG_CHECKS
    // debug build's test hook: PN_DEBUG_INJECT=<site> makes every index
    // check of that site fail (the access then takes index 0), so the
    // reporting path runs without a bad index
    c->dbg_inject = 0;
    if (const char *di = std::getenv("PN_DEBUG_INJECT"))
        c->dbg_inject = std::atoi(di);
#endif
    // the packed law-of-cosines kernel runs on Hilbert-ordered slots
    // (pn_order.cu) when the pair work is large enough to repay the sort's
    // fixed cost (about ten short launches per evaluation);
    // PN_SPATIAL=0 / 1 overrides
    double pairs = 0.0;
    for (int k = 0; k < nclu; ++k)
        pairs += (double)c->hclu[k].ns_pad * (double)c->hclu[k].ns_pad;
    c->spatial = pairs >= pn::kSpatialMinPairs;
    if (const char *sp = std::getenv("PN_SPATIAL"))
        c->spatial = sp[0] != '0';
    c->far_theta = pn::kFarTheta;
    c->balance = true;          // PN_BALANCE=0: equal unit counts per worker
    if (const char *bl = std::getenv("PN_BALANCE"))
        c->balance = bl[0] != '0';
    if (const char *ft = std::getenv("PN_FAR_THETA")) {
        const double v = std::atof(ft);
        if (v >= 0.02 && v <= 10.0)
            c->far_theta = (float)v;
    }
    if (const char *pw = std::getenv("PN_FUSED_WORKERS")) {
        const int v = std::atoi(pw);
        if (v >= 1 && v <= 64)
            c->workers_max = v;
    }
    if (const char *pk = std::getenv("PN_FUSED_PACKED"))
        c->fused_packed = std::atoi(pk) != 0;
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
    if (c->fused_packed && c->fused_P != 2)
        c->fused_P = 4;             // packed kernel: 2 or 4 targets per thread
    if (c->fused_packed && c->fused_unroll > 2)
        c->fused_unroll = 2;
    if (c->fused_P == 2 && c->fused_unroll == 3)
        c->fused_unroll = 2;
    if (c->fused_P == 1 && c->fused_unroll > 2)
        c->fused_unroll = 2;
    // packed kernel's tile and buffers: PN_FUSED_TILE / PN_FUSED_STAGES
    // (a supported pair; 32-source tiles only on the slot order)
    if (const char *ft = std::getenv("PN_FUSED_TILE"))
        c->fused_tile = std::atoi(ft);
    if (const char *fst = std::getenv("PN_FUSED_STAGES"))
        c->fused_stages = std::atoi(fst);
    if (c->fused_tile == 32 && !std::getenv("PN_FUSED_STAGES"))
        c->fused_stages = 8;
    if (!pn::packed_layout_ok(c->fused_tile, c->fused_stages) ||
        (c->spatial && c->fused_tile != pn::kPackTile)) {
        c->fused_tile = pn::kPackTile;
        c->fused_stages = pn::kPackStages;
    }
    // the adjoint's pair sweeps: one merged pass unless PN_ADJ_SEPARATE is set
    if (const char *as = std::getenv("PN_ADJ_SEPARATE"))
        c->adj_separate = std::atoi(as) != 0;
    pn::FusedShape fs{};
    // segment buffer: the largest over every fused variant (the tuner may switch)
    int64_t seg_max = 0;
    static const pn::FusedVariant variants[] = {
        {1, 1, 0, 0, 0}, {1, 2, 0, 0, 0}, {2, 1, 0, 0, 0}, {2, 2, 0, 0, 0}, {2, 4, 0, 0, 0},
        {4, 1, 0, 0, 0}, {4, 2, 0, 0, 0}, {4, 3, 0, 0, 0}, {4, 4, 0, 0, 0},
        {2, 1, 1, 64, 6}, {2, 2, 1, 64, 6}, {4, 1, 1, 64, 6}, {4, 2, 1, 64, 6},
        {2, 1, 1, 64, 4}, {2, 2, 1, 64, 4}, {4, 1, 1, 64, 4}, {4, 2, 1, 64, 4},
        {2, 1, 1, 32, 8}, {2, 2, 1, 32, 8}, {4, 1, 1, 32, 8}, {4, 2, 1, 32, 8}};
    for (const auto &va : variants) {
        if (e == cudaSuccess)
            e = pn::fused_shape(c, va, &fs);
        const int64_t seg = (c->S / (pn::kMixThreads * va.P) + fs.G) * pn::kMixThreads * va.P;
        if (seg > seg_max)
            seg_max = seg;
        if (va.packed) {        // packed variants: sizes of the worker-balance scratch
            if (fs.units > c->bal_units)
                c->bal_units = fs.units;
            if (fs.G > c->bal_G)
                c->bal_G = fs.G;
        }
    }
    if (e == cudaSuccess)
        e = pn::fused_shape(c, pn::fused_variant(c), &fs);
    if (e != cudaSuccess) {
        delete[] c->hclu;
        delete c;
        return fail(PN_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    }
    pn::shapes(c->S, c->max_ns_pad, sms, occ_mix, occ_f64, &c->mix, &c->f64);
    c->fused_occ = fs.occ;
    c->fused_grid = fs.grid;
    c->fused_G = fs.G;
    c->fused_seg_max = seg_max;
    c->fused_units = pn::fused_units(c->hclu, nclu, pn::fused_variant(c), c->hclu);

    const int64_t S = c->S;
    int64_t part = (int64_t)c->mix.jsplit * (pn::kP1Vals + pn::kP2Vals) * S;
    const int64_t part_f64 = (int64_t)c->f64.jsplit * (pn::kP1Vals + pn::kP2Vals) * S;
    if (part_f64 > part)
        part = part_f64;
    // energy: the split partials, then (mixed contexts) the double-single
    // records, 16 floats per slot
    const int64_t e_js = pn::energy_splits(S, c->sm_count, c->max_ns_pad);
    if (((int64_t)pn::kEVals * e_js + 8) * S > part)
        part = ((int64_t)pn::kEVals * e_js + 8) * S;
    part += (int64_t)pn::kNearVals * S;   // near-pass partials after both passes
    // fused layout: pass sums, near sums, then the largest segment buffer
    const int64_t part_fused = (int64_t)(pn::kP1Vals + pn::kP2Vals + pn::kNearVals) * S +
                               seg_max * pn::kFusedVals;
    if (part_fused > part)
        part = part_fused;
    c->part_len = part;
    const int64_t nglue = S / pn::kGlueThreads;
    c->blk_len = S / pn::kProThreads * pn::kGlobVals;     // the largest per-block partial table

    struct Req { void **p; size_t bytes; } req[] = {
        {(void **)&c->vp, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_x, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_v, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_a, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_sx, sizeof(double) * 3 * (size_t)n},
        {(void **)&c->rk_sv, sizeof(double) * 3 * (size_t)n},
        // mixed: 5 record arrays + the packed kernel's staged sources (9 per slot);
        // allocated whatever the precision, which pn_set_params may change
        {(void **)&c->mrec, sizeof(float4) * 14 * (size_t)S},
        {(void **)&c->drec, sizeof(double4_32a) * 4 * (size_t)S},
        // mixed: the spatial order of the packed kernel (sorted records, boxes, sort scratch)
        {(void **)&c->sord, pn::order_buffer_bytes(S)},
        // and its cost-balanced worker boundaries
        {(void **)&c->bal, pn::balance_buffer_bytes(S, c->bal_units, c->bal_G)},
        {(void **)&c->part, sizeof(double) * (size_t)part},
        {(void **)&c->blk, sizeof(double) * (size_t)c->blk_len},
        {(void **)&c->glob, sizeof(double) * pn::kGlobVals * (size_t)nclu},
        {(void **)&c->nrec, sizeof(float4) * 4 * (size_t)c->NC},
        {(void **)&c->ndrec, sizeof(double4_32a) * 3 * (size_t)c->NC},
        {(void **)&c->ncount, sizeof(int) * (size_t)(nclu + nglue)},
        {(void **)&c->nflag, (size_t)S},
        {(void **)&c->eout, sizeof(double) * 8 * (size_t)nclu},
        {(void **)&c->flag, sizeof(int)},
        {(void **)&c->wcount, sizeof(int)},
        {(void **)&c->units_cnt, 2 * sizeof(unsigned long long)},
        {(void **)&c->flag_step, sizeof(unsigned long long)},
        {(void **)&c->epi_done, sizeof(unsigned) * (size_t)nclu},
        {(void **)&c->d_clu, sizeof(pn::Clu) * (size_t)nclu},
        {(void **)&c->blk_clu, sizeof(int) * (size_t)nglue},
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
    int *hb = new (std::nothrow) int[(size_t)nglue];
    if (!hb) {
        free_all(c);
        delete c;
        return fail(PN_ENOMEM, "host allocation failed");
    }
    for (int k = 0; k < nclu; ++k)
        for (int64_t b = c->hclu[k].slot0 / pn::kGlueThreads;
             b < (c->hclu[k].slot0 + c->hclu[k].ns_pad) / pn::kGlueThreads; ++b)
            hb[b] = k;
    const unsigned long long none = ULLONG_MAX;
    e = cudaMemcpy(c->blk_clu, hb, sizeof(int) * (size_t)nglue, cudaMemcpyHostToDevice);
    delete[] hb;
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_clu, c->hclu, sizeof(pn::Clu) * (size_t)nclu, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(c->flag, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->flag_step, &none, sizeof none, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(c->ncount, 0, sizeof(int) * (size_t)(nclu + nglue));
    if (e == cudaSuccess)
        e = cudaMemset(c->units_cnt, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemset(c->epi_done, 0, sizeof(unsigned) * (size_t)nclu);
    // side stream of the near-source pass (highest priority, so its blocks
    // take the first free slots beside the persistent pair kernel) and its
    // fork / join events
    if (e == cudaSuccess) {
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    }
#ifdef PN_DEBUG_CHECKS
    // arm the test hook's site before the first launch (and clear old records)
    unsigned long long dsite = 0;
    long long dindex = 0;
    if (e == cudaSuccess)
        e = pn::debug_take_kernels(c->dbg_inject, &dsite, &dindex);
    if (e == cudaSuccess)
        e = pn::debug_take_order(c->dbg_inject, &dsite, &dindex);
#endif
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(PN_ECUDA, "initialising the context: %s", cudaGetErrorString(e));
    }
    *out = c;
    return ok();
}

pn_status pn_init(pn_ctx **out, int64_t n, const pn_params *params, int device,
                  void *cuda_stream)
{
    if (!out)
        return fail(PN_EINVAL, "ctx output pointer is NULL");
    *out = nullptr;
    if (n < 2)
        return fail(PN_EINVAL, "n must be >= 2 (the hole and at least one star), got %lld",
                    (long long)n);
    if (!params_ok(params))
        return PN_EINVAL;
    const int64_t off[2] = {0, n};
    return init_common(out, 1, off, nullptr, params, device, cuda_stream);
}

pn_status pn_init_batched(pn_ctx **out, int n_clusters, const int64_t *offsets,
                          const pn_cluster *clusters, const pn_params *params, int device,
                          void *cuda_stream)
{
    if (!out)
        return fail(PN_EINVAL, "ctx output pointer is NULL");
    *out = nullptr;
    if (n_clusters < 1 || !offsets)
        return fail(PN_EINVAL, "need n_clusters >= 1 and an offsets array");
    if (offsets[0] != 0)
        return fail(PN_EINVAL, "offsets[0] must be 0");
    return init_common(out, n_clusters, offsets, clusters, params, device, cuda_stream);
}

pn_status pn_set_params(pn_ctx *c, const pn_params *params)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!params_ok(params))
        return PN_EINVAL;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    set_params(c, params, true);
    pn_status st = upload_clusters(c);
    return st == PN_OK ? ok() : st;
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

pn_status pn_jerk(pn_ctx *c, const double *x, const double *v, const double *m, double *a,
                  double *jerk)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a || !jerk)
        return fail(PN_EINVAL, "pn_jerk: NULL array");
    const void *in[] = {x, v, m};
    for (const void *q : in)
        if (q == a || q == jerk)
            return fail(PN_EINVAL, "pn_jerk: an output aliases an input");
    if (a == jerk)
        return fail(PN_EINVAL, "pn_jerk: a and jerk alias");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    pn_status st = ensure_jerk_buffers(c);
    if (st != PN_OK)
        return st;
    st = evaluate(c, x, v, m, a, nullptr, 0.0);
    if (st != PN_OK)
        return st;
    PN_CUDA(pn::launch_jerk(c, x, v, m, a, jerk), "jerk launch");
    return ok();
}

pn_status pn_accel_vjp(pn_ctx *c, const double *x, const double *v, const double *m,
                       const double *abar, double *xbar, double *vbar, double *scal)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !abar || !xbar || !vbar || !scal)
        return fail(PN_EINVAL, "pn_accel_vjp: NULL array");
    const void *in[] = {x, v, m, abar};
    for (const void *q : in)
        if (q == xbar || q == vbar)
            return fail(PN_EINVAL, "pn_accel_vjp: an output aliases an input");
    if (xbar == vbar)
        return fail(PN_EINVAL, "pn_accel_vjp: xbar and vbar alias");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    pn_status st = ensure_adjoint_buffers(c);
    if (st != PN_OK)
        return st;
    double *dscal = nullptr;
    PN_CUDA(cudaMalloc((void **)&dscal, sizeof(double) * 2 * c->nclu), "cudaMalloc");
    cudaError_t e = pn::launch_accel_vjp(c, x, v, m, abar, xbar, vbar, dscal, false);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scal, dscal, sizeof(double) * 2 * c->nclu, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    cudaFree(dscal);
    PN_CUDA(e, "accel vjp");
    return ok();
}

// Reverse of nsteps KDK steps from (x0, v0), checkpointed: the forward pass
// stores (x, v, a) every K steps; the backward pass re-runs each segment
// from its checkpoint, keeping the K pre-step states, and walks it in
// reverse.  Memory (K + steps/K) 9n doubles.
namespace {
// Workspace of the KDK adjoint: one step's states and cotangents and one
// segment of K pre-step states.
struct AdjWork {
    double *xs, *vs, *as, *xp, *vp, *atot, *xbA, *vpbA, *xb, *vb, *ab, *dscal;
    double *w;
    // one segment's pre-step states (K x 9n doubles); with sums two sets, so
    // that one segment is recomputed while the previous one is reversed
    double *seg[2];
    // mixed contexts with the fused kernel: each recomputed step's 16
    // forward pair sums (16 S doubles) and staged source records (9 S
    // float4), for the reverse of that step (nullptr otherwise)
    double *sums[2];
    float4 *srec[2];
};

// The recomputed segments keep their pair sums for the reverse (see
// AdjWork) where the forward pair kernel is the fused one.
bool adj_saves_sums(const pn_ctx *c) { return pn::use_fused(c); }

constexpr int64_t kAdjSumVals = 16;                       // pair sums per slot
constexpr int64_t kAdjSrecDoubles = 2 * pn::kPackVals;     // 9 float4 per slot

int64_t checkpoint_interval(int64_t nsteps, int64_t checkpoint)
{
    int64_t K = checkpoint;
    if (K == 0) {
        K = 1;
        while (K * K < nsteps)
            ++K;
    }
    return K;
}

// Allocates the workspace, with room for ncp checkpoints after ab when
// own_checkpoints (returned in *cp).
pn_status adj_alloc(pn_ctx *c, int64_t K, int64_t ncp, bool own_checkpoints, AdjWork *W,
                    double **cp)
{
    const size_t n3 = 3 * (size_t)c->n;
    const size_t per_step = adj_saves_sums(c) ? (size_t)(kAdjSumVals + kAdjSrecDoubles) * c->S : 0;
    const int nbuf = per_step ? 2 : 1;
    // (+ 16 doubles: the saved regions start 128-byte aligned)
    const size_t nwork = 11 * n3 + (size_t)(own_checkpoints ? ncp : 0) * 3 * n3 +
                         (size_t)nbuf * K * (3 * n3 + per_step) + (per_step ? 16 : 0);
    W->w = nullptr;
    W->dscal = nullptr;
    for (int b = 0; b < 2; ++b) {
        W->seg[b] = nullptr;
        W->sums[b] = nullptr;
        W->srec[b] = nullptr;
    }
    if (std::getenv("PN_FAIL_ALLOC") ||
        cudaMalloc((void **)&W->w, sizeof(double) * nwork) != cudaSuccess) {
        cudaGetLastError();
        W->w = nullptr;
        return fail(PN_ENOMEM, "cudaMalloc of %zu bytes for the adjoint failed",
                    sizeof(double) * nwork);
    }
    if (cudaMalloc((void **)&W->dscal, sizeof(double) * 2 * c->nclu) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(W->w);
        W->w = nullptr;
        W->dscal = nullptr;
        return fail(PN_ENOMEM, "cudaMalloc for the adjoint failed");
    }
    W->xs = W->w;
    W->vs = W->xs + n3;
    W->as = W->vs + n3;
    W->xp = W->as + n3;
    W->vp = W->xp + n3;
    W->atot = W->vp + n3;
    W->xbA = W->atot + n3;
    W->vpbA = W->xbA + n3;
    W->xb = W->vpbA + n3;
    W->vb = W->xb + n3;
    W->ab = W->vb + n3;
    double *after = W->ab + n3;
    if (own_checkpoints) {
        *cp = after;
        after += (size_t)ncp * 3 * n3;
    }
    for (int b = 0; b < nbuf; ++b) {
        W->seg[b] = after;
        after += (size_t)K * 3 * n3;
    }
    if (per_step) {
        // S is a multiple of 512, so every region after the first stays aligned
        const uintptr_t a = (reinterpret_cast<uintptr_t>(after) + 127) & ~(uintptr_t)127;
        double *p = reinterpret_cast<double *>(a);
        for (int b = 0; b < 2; ++b) {
            W->sums[b] = p;
            p += (size_t)K * kAdjSumVals * c->S;
            W->srec[b] = reinterpret_cast<float4 *>(p);
            p += (size_t)K * kAdjSrecDoubles * c->S;
        }
    }
    return PN_OK;
}

// Switches the near-source split off for the adjoint's recomputed segments
// (every cluster's r_near < 0: the evaluation then uses the form the
// reverse differentiates, and its pair sums serve the reverse directly)
// and back on.
struct FarForm {
    pn_ctx *c = nullptr;
    double *saved = nullptr;
    pn_status enter(pn_ctx *ctx)
    {
        c = ctx;
        if (!c->any_near)
            return PN_OK;
        saved = new (std::nothrow) double[(size_t)c->nclu];
        if (!saved)
            return fail(PN_ENOMEM, "host allocation failed");
        for (int k = 0; k < c->nclu; ++k) {
            saved[k] = c->hclu[k].r_near;
            c->hclu[k].r_near = -1.0;
        }
        set_params(c, &c->p, false);
        return upload_clusters(c);
    }
    pn_status leave()
    {
        if (!saved)
            return PN_OK;
        for (int k = 0; k < c->nclu; ++k)
            c->hclu[k].r_near = saved[k];
        delete[] saved;
        saved = nullptr;
        set_params(c, &c->p, false);
        return upload_clusters(c);
    }
};

void adj_free(pn_ctx *c, AdjWork *W)
{
    cudaStreamSynchronize(c->stream);
    if (W->w)
        cudaFree(W->w);
    if (W->dscal)
        cudaFree(W->dscal);
}

// The forward KDK steps from (x, v, a) in place, writing (x, v, a) before
// steps 0, K, 2K, ... into cp (9 n doubles each); the steps between two
// checkpoints run as one pn_step sequence.
pn_status kdk_forward_checkpoints(pn_ctx *c, double *x, double *v, const double *m, double *a,
                                  double dt, int64_t nsteps, int64_t K, double *cp)
{
    const size_t n3 = 3 * (size_t)c->n, b3 = sizeof(double) * n3;
    for (int64_t s = 0; s < nsteps; s += K) {
        double *q = cp + (size_t)(s / K) * 3 * n3;
        PN_CUDA(cudaMemcpyAsync(q, x, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        PN_CUDA(cudaMemcpyAsync(q + n3, v, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        PN_CUDA(cudaMemcpyAsync(q + 2 * n3, a, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        const pn_status st = run_steps(c, x, v, m, a, dt, s + K < nsteps ? K : nsteps - s);
        if (st != PN_OK)
            return st;
    }
    return PN_OK;
}

// Segment sg (steps [sg K, min((sg + 1) K, nsteps))) forward once more from
// its checkpoint, on c->stream: the pre-step states into W.seg[b] and, where
// kept, each step's pair sums and staged records into W.sums[b] / W.srec[b]
// (the segment's last step is taken too for its sums).
pn_status rerun_segment(pn_ctx *c, const double *cp, int64_t sg, int64_t K, int64_t nsteps,
                        const double *m, double dt, const AdjWork &W, int b)
{
    const size_t n3 = 3 * (size_t)c->n, b3 = sizeof(double) * n3, S = (size_t)c->S;
    const int64_t s0 = sg * K, s1 = s0 + K < nsteps ? s0 + K : nsteps;
    const double *q = cp + (size_t)sg * 3 * n3;
    double *xs = W.xs, *vs = W.vs, *as = W.as;
    PN_CUDA(cudaMemcpyAsync(xs, q, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemcpyAsync(vs, q + n3, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemcpyAsync(as, q + 2 * n3, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    for (int64_t s = s0; s < s1; ++s) {
        double *r = W.seg[b] + (size_t)(s - s0) * 3 * n3;
        PN_CUDA(cudaMemcpyAsync(r, xs, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        PN_CUDA(cudaMemcpyAsync(r + n3, vs, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        PN_CUDA(cudaMemcpyAsync(r + 2 * n3, as, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        if (s + 1 < s1 || W.sums[b]) {
            const pn_status st = run_steps(c, xs, vs, m, as, dt, 1);
            if (st != PN_OK)
                return st;
        }
        if (W.sums[b]) {
            PN_CUDA(cudaMemcpyAsync(W.sums[b] + (size_t)(s - s0) * kAdjSumVals * S, c->part,
                                    sizeof(double) * kAdjSumVals * S, cudaMemcpyDeviceToDevice,
                                    c->stream), "copy sums");
            PN_CUDA(cudaMemcpyAsync(W.srec[b] + (size_t)(s - s0) * pn::kPackVals * S,
                                    c->mrec + 5 * S, sizeof(float4) * pn::kPackVals * S,
                                    cudaMemcpyDeviceToDevice, c->stream), "copy records");
        }
    }
    return PN_OK;
}

// The reverse of segment sg's steps, last to first, on c->stream, from the
// states (and kept sums) in buffers b.
pn_status reverse_segment(pn_ctx *c, int64_t sg, int64_t K, int64_t nsteps, const double *m,
                          double dt, const AdjWork &W, int b)
{
    const size_t n3 = 3 * (size_t)c->n, S = (size_t)c->S;
    const int64_t s0 = sg * K, s1 = s0 + K < nsteps ? s0 + K : nsteps;
    for (int64_t s = s1 - 1; s >= s0; --s) {
        const double *r = W.seg[b] + (size_t)(s - s0) * 3 * n3;
        const double *fs = W.sums[b] ? W.sums[b] + (size_t)(s - s0) * kAdjSumVals * S : nullptr;
        const float4 *fr = W.sums[b] ? W.srec[b] + (size_t)(s - s0) * pn::kPackVals * S : nullptr;
        PN_CUDA(pn::launch_adj_kdk(c, 0, dt, r, r + n3, r + 2 * n3, W.xp, W.vp, W.xb, W.vb, W.ab,
                                   W.atot, nullptr, nullptr), "adjoint step launch");
        PN_CUDA(pn::launch_accel_vjp(c, W.xp, W.vp, m, W.atot, W.xbA, W.vpbA, W.dscal, true, fs,
                                     fr), "accel vjp launch");
        PN_CUDA(pn::launch_adj_kdk(c, 1, dt, nullptr, nullptr, nullptr, nullptr, nullptr, W.xb,
                                   W.vb, W.ab, nullptr, W.xbA, W.vpbA), "adjoint step launch");
    }
    return PN_OK;
}

// The reverse of nsteps KDK steps from their checkpoints cp (the states
// before steps 0, K, 2K, ...): each segment is run forward once more keeping
// its pre-step states, then walked back; last the entry acceleration
// A(x0, v0), x0 and v0 the state before step 0.  Writes xbar0, vbar0 and the
// host array scal.
pn_status kdk_backward(pn_ctx *c, const double *cp, int64_t K, const double *x0,
                       const double *v0, const double *m, double dt, int64_t nsteps,
                       const double *xbar_T, const double *vbar_T, double *xbar0, double *vbar0,
                       double *scal, const AdjWork &W)
{
    const size_t n3 = 3 * (size_t)c->n, b3 = sizeof(double) * n3;
    const int64_t ncp = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    double *xbA = W.xbA, *vpbA = W.vpbA, *xb = W.xb, *vb = W.vb, *ab = W.ab;
    double *dscal = W.dscal;
    pn_status s2 = PN_OK;
    PN_CUDA(cudaMemcpyAsync(xb, xbar_T, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemcpyAsync(vb, vbar_T, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemsetAsync(ab, 0, b3, c->stream), "memset");
    PN_CUDA(cudaMemsetAsync(dscal, 0, sizeof(double) * 2 * c->nclu, c->stream), "memset");
    if (!W.sums[0]) {
        for (int64_t sg = ncp - 1; sg >= 0; --sg) {
            if ((s2 = rerun_segment(c, cp, sg, K, nsteps, m, dt, W, 0)) != PN_OK)
                return s2;
            if ((s2 = reverse_segment(c, sg, K, nsteps, m, dt, W, 0)) != PN_OK)
                return s2;
        }
    } else if (ncp > 0) {
        // segment sg - 1 is recomputed on the adjoint stream while segment sg
        // is reversed on the context's stream (buffers sg % 2 alternate;
        // events order each handoff); the reverse keeps only its own scratch
        // and the kept sums, so the two share no buffer
        if (!c->adj_stream)
            PN_CUDA(cudaStreamCreateWithFlags(&c->adj_stream, cudaStreamNonBlocking),
                    "adjoint stream");
        struct Events {        // the handoff events, destroyed on every return
            cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
            ~Events()
            {
                for (cudaEvent_t x : e)
                    if (x)
                        cudaEventDestroy(x);
            }
        } evs;
        cudaEvent_t *ev = evs.e;
        for (int k = 0; k < 5; ++k)
            PN_CUDA(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming), "event");
        cudaEvent_t start = ev[0], rerun_done[2] = {ev[1], ev[2]}, rev_done[2] = {ev[3], ev[4]};
        cudaStream_t A = c->stream, B = c->adj_stream;
        auto on_b = [&](int64_t sg) -> pn_status {
            c->stream = B;
            const pn_status r = rerun_segment(c, cp, sg, K, nsteps, m, dt, W, (int)(sg % 2));
            c->stream = A;
            if (r != PN_OK)
                return r;
            PN_CUDA(cudaEventRecord(rerun_done[sg % 2], B), "event");
            return PN_OK;
        };
        auto run = [&]() -> pn_status {
            PN_CUDA(cudaEventRecord(start, A), "event");       // checkpoints, cotangents
            PN_CUDA(cudaStreamWaitEvent(B, start, 0), "event wait");
            pn_status r = on_b(ncp - 1);
            for (int64_t sg = ncp - 1; sg >= 0 && r == PN_OK; --sg) {
                PN_CUDA(cudaStreamWaitEvent(A, rerun_done[sg % 2], 0), "event wait");
                if (sg >= 1) {
                    if (sg + 1 <= ncp - 1)       // buffers (sg - 1) % 2 were segment sg + 1's
                        PN_CUDA(cudaStreamWaitEvent(B, rev_done[(sg - 1) % 2], 0), "event wait");
                    if ((r = on_b(sg - 1)) != PN_OK)
                        break;
                }
                if ((r = reverse_segment(c, sg, K, nsteps, m, dt, W, (int)(sg % 2))) != PN_OK)
                    break;
                PN_CUDA(cudaEventRecord(rev_done[sg % 2], A), "event");
            }
            return r;
        };
        s2 = run();
        c->stream = A;
        cudaStreamSynchronize(B);      // (on an error, before the buffers go)
        if (s2 != PN_OK)
            return s2;
    }
    // the entry acceleration A(x0, v0)
    if (x0) {
        PN_CUDA(pn::launch_accel_vjp(c, x0, v0, m, ab, xbA, vpbA, dscal, true),
                "accel vjp launch");
        PN_CUDA(pn::launch_adj_kdk(c, 2, dt, nullptr, nullptr, nullptr, nullptr, nullptr, xb, vb,
                                   ab, nullptr, xbA, vpbA), "adjoint step launch");
    }
    PN_CUDA(cudaMemcpyAsync(xbar0, xb, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemcpyAsync(vbar0, vb, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
    PN_CUDA(cudaMemcpyAsync(scal, dscal, sizeof(double) * 2 * c->nclu, cudaMemcpyDeviceToHost,
                            c->stream), "copy");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return PN_OK;
}

pn_status vjp_args(pn_ctx *c, const char *name, double dt, int64_t nsteps, int64_t checkpoint)
{
    if (!(std::isfinite(dt) && dt > 0.0))
        return fail(PN_EINVAL, "%s: dt must be finite and > 0 (got %g)", name, dt);
    if (nsteps < 0 || checkpoint < 0)
        return fail(PN_EINVAL, "%s: nsteps and checkpoint must be >= 0", name);
    if (c->p.integrator != PN_KDK)
        return fail(PN_EUNSUPPORTED, "%s: only the PN_KDK integrator has an adjoint", name);
    return PN_OK;
}
}  // namespace

pn_status pn_step_vjp(pn_ctx *c, const double *x0, const double *v0, const double *m,
                      double dt, int64_t nsteps, int64_t checkpoint, const double *xbar_T,
                      const double *vbar_T, double *xbar0, double *vbar0, double *scal)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x0 || !v0 || !m || !xbar_T || !vbar_T || !xbar0 || !vbar0 || !scal)
        return fail(PN_EINVAL, "pn_step_vjp: NULL array");
    pn_status st = vjp_args(c, "pn_step_vjp", dt, nsteps, checkpoint);
    if (st != PN_OK)
        return st;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    if ((st = ensure_adjoint_buffers(c)) != PN_OK)
        return st;
    const int64_t K = checkpoint_interval(nsteps, checkpoint);
    const int64_t ncp = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    const size_t n3 = 3 * (size_t)c->n, b3 = sizeof(double) * n3;
    AdjWork W;
    double *cp = nullptr;
    if ((st = adj_alloc(c, K, ncp, true, &W, &cp)) != PN_OK)
        return st;
    // the forward recomputations are not the caller's trajectory: no watchdog checks
    const int64_t wd_every = c->wd_every;
    c->wd_every = 0;
    auto run = [&]() -> pn_status {
        PN_CUDA(cudaMemcpyAsync(W.xs, x0, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        PN_CUDA(cudaMemcpyAsync(W.vs, v0, b3, cudaMemcpyDeviceToDevice, c->stream), "copy");
        pn_status s2 = evaluate(c, W.xs, W.vs, m, W.as, nullptr, 0.0);
        if (s2 == PN_OK)
            s2 = kdk_forward_checkpoints(c, W.xs, W.vs, m, W.as, dt, nsteps, K, cp);
        if (s2 == PN_OK) {
            FarForm far;
            if (W.sums[0])
                s2 = far.enter(c);
            if (s2 == PN_OK)
                s2 = kdk_backward(c, cp, K, x0, v0, m, dt, nsteps, xbar_T, vbar_T, xbar0, vbar0,
                                  scal, W);
            const pn_status s3 = far.leave();
            if (s2 == PN_OK)
                s2 = s3;
        }
        return s2;
    };
    st = run();
    c->wd_every = wd_every;
    adj_free(c, &W);
    return st == PN_OK ? ok() : st;
}

pn_status pn_step_save(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                       int64_t nsteps, int64_t checkpoint, double *ckpt)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a || (nsteps > 0 && !ckpt))
        return fail(PN_EINVAL, "pn_step_save: NULL array");
    pn_status st = vjp_args(c, "pn_step_save", dt, nsteps, checkpoint);
    if (st != PN_OK)
        return st;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    const int64_t K = checkpoint_interval(nsteps, checkpoint);
    st = kdk_forward_checkpoints(c, x, v, m, a, dt, nsteps, K, ckpt);
    return st == PN_OK ? ok() : st;
}

pn_status pn_step_vjp_saved(pn_ctx *c, const double *ckpt, const double *m, double dt,
                            int64_t nsteps, int64_t checkpoint, const double *xbar_T,
                            const double *vbar_T, double *xbar0, double *vbar0, double *scal)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if ((nsteps > 0 && !ckpt) || !m || !xbar_T || !vbar_T || !xbar0 || !vbar0 || !scal)
        return fail(PN_EINVAL, "pn_step_vjp_saved: NULL array");
    pn_status st = vjp_args(c, "pn_step_vjp_saved", dt, nsteps, checkpoint);
    if (st != PN_OK)
        return st;
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    if ((st = ensure_adjoint_buffers(c)) != PN_OK)
        return st;
    const int64_t K = checkpoint_interval(nsteps, checkpoint);
    const size_t n3 = 3 * (size_t)c->n;
    AdjWork W;
    if ((st = adj_alloc(c, K, 0, false, &W, nullptr)) != PN_OK)
        return st;
    const int64_t wd_every = c->wd_every;
    c->wd_every = 0;
    // x0, v0: the state of checkpoint 0 (none without steps: the entry
    // acceleration then has a zero cotangent and is skipped)
    const double *x0 = nsteps > 0 ? ckpt : nullptr;
    const double *v0 = nsteps > 0 ? ckpt + n3 : nullptr;
    FarForm far;
    if (W.sums[0])
        st = far.enter(c);
    if (st == PN_OK)
        st = kdk_backward(c, ckpt, K, x0, v0, m, dt, nsteps, xbar_T, vbar_T, xbar0, vbar0, scal,
                          W);
    const pn_status s3 = far.leave();
    if (st == PN_OK)
        st = s3;
    c->wd_every = wd_every;
    adj_free(c, &W);
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

pn_status pn_step_graph(pn_ctx *c, double *x, double *v, const double *m, double *a, double dt,
                        int64_t nsteps)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a)
        return fail(PN_EINVAL, "pn_step_graph: NULL array");
    if (!(std::isfinite(dt) && dt > 0.0))
        return fail(PN_EINVAL, "pn_step_graph: dt must be finite and > 0 (got %g)", dt);
    if (nsteps < 1)
        return fail(PN_EINVAL, "pn_step_graph: nsteps must be >= 1");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    const void *key[4] = {x, v, m, a};
    const bool same = c->graph_exec && c->graph_dt == dt && c->graph_steps == nsteps &&
                      std::memcmp(key, c->graph_key, sizeof key) == 0;
    if (!same) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        if (c->p.integrator == PN_HERMITE) {
            pn_status st = ensure_jerk_buffers(c);
            if (st != PN_OK)
                return st;
        }
        if (!c->cap_stream)
            PN_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking),
                    "capture stream");
        cudaStream_t user = c->stream;
        c->stream = c->cap_stream;
        c->capturing = true;
        const int64_t before = c->launches;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        pn_status st = e == cudaSuccess ? run_steps(c, x, v, m, a, dt, nsteps) : PN_ECUDA;
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
        c->stream = user;
        c->capturing = false;
        c->graph_launches = c->launches - before;   // captured, not yet run
        c->launches = before;
        if (e != cudaSuccess || e2 != cudaSuccess || st != PN_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            if (st != PN_OK)
                return st;
            return fail(PN_ECUDA, "graph capture: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->graph_exec = nullptr;
            return fail(PN_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        std::memcpy(c->graph_key, key, sizeof key);
        c->graph_dt = dt;
        c->graph_steps = nsteps;
    }
    PN_CUDA(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
    c->launches += c->graph_launches;
    return ok();
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

pn_status pn_energy(pn_ctx *c, const double *x, const double *v, const double *m, double *out)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !out)
        return fail(PN_EINVAL, "pn_energy: NULL array");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    PN_CUDA(pn::launch_energy(c, x, v, m), "energy launch");
    PN_CUDA(cudaMemcpyAsync(out, c->eout, sizeof(double) * 8 * (size_t)c->nclu,
                            cudaMemcpyDeviceToHost, c->stream), "copy energy out");
    pn_status st = report_flag(c);
    return st == PN_OK ? ok() : st;
}

pn_status pn_set_watchdog(pn_ctx *c, double rel_tol, int64_t every)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!(std::isfinite(rel_tol) && rel_tol >= 0.0))
        return fail(PN_EINVAL, "pn_set_watchdog: rel_tol must be finite and >= 0 (got %g)",
                    rel_tol);
    if (rel_tol > 0.0 && every < 1)
        return fail(PN_EINVAL, "pn_set_watchdog: every must be >= 1 (got %lld)",
                    (long long)every);
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    if (rel_tol > 0.0 && !c->wd) {
        if (std::getenv("PN_FAIL_ALLOC") ||
            cudaMalloc((void **)&c->wd, sizeof(double) * (size_t)(c->nclu + 2)) != cudaSuccess ||
            cudaMalloc((void **)&c->wd_step, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            if (c->wd)
                cudaFree(c->wd);
            c->wd = nullptr;
            return fail(PN_ENOMEM, "cudaMalloc for the watchdog failed");
        }
    }
    if (c->wd) {
        // references unset (all-ones bytes are a NaN), no tripped step yet
        const unsigned long long none = ULLONG_MAX;
        PN_CUDA(cudaMemsetAsync(c->wd, 0xff, sizeof(double) * (size_t)c->nclu, c->stream),
                "reset watchdog references");
        PN_CUDA(cudaMemcpyAsync(c->wd_step, &none, sizeof none, cudaMemcpyHostToDevice,
                                c->stream), "reset watchdog step");
        PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    }
    c->wd_tol = rel_tol;
    c->wd_every = rel_tol > 0.0 ? every : 0;
    // a captured step sequence holds the old setting: capture again
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    return ok();
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
    if (enable)
        PN_CUDA(cudaMemsetAsync(c->units_cnt, 0, 2 * sizeof(unsigned long long), c->stream),
                "reset of the pair statistics");
    return ok();
}

pn_status pn_get_pair_stats(pn_ctx *c, int64_t out[2])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!out)
        return fail(PN_EINVAL, "pn_get_pair_stats: NULL output");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    unsigned long long h[2] = {0, 0};
    PN_CUDA(cudaMemcpyAsync(h, c->units_cnt, sizeof h, cudaMemcpyDeviceToHost, c->stream),
            "read of the pair statistics");
    PN_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    out[0] = (int64_t)h[0];
    out[1] = (int64_t)h[1];
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

pn_status pn_get_launch(pn_ctx *c, int64_t out[8])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!out)
        return fail(PN_EINVAL, "pn_get_launch: NULL output");
    const pn::Shape &s = c->p.precision == PN_MIXED ? c->mix : c->f64;
    const bool fused = pn::use_fused(c);
    out[0] = s.threads;
    out[1] = fused ? c->fused_P : s.targets;
    out[2] = fused ? pn::fused_tile_size(pn::fused_variant(c)) : s.tile;
    out[3] = s.nblk_i;
    out[4] = fused ? c->fused_G : s.jsplit;
    out[5] = fused ? c->fused_occ : s.occupancy;
    out[6] = c->sm_count;
    out[7] = fused && c->fused_packed ? 1 : 0;
    return ok();
}

pn_status pn_get_variant(pn_ctx *c, int64_t out[6])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!out)
        return fail(PN_EINVAL, "pn_get_variant: NULL output");
    for (int k = 0; k < 6; ++k)
        out[k] = 0;
    if (pn::use_fused(c)) {
        const pn::FusedVariant v = pn::fused_variant(c);
        out[0] = v.P;
        out[1] = v.unroll;
        out[2] = v.packed ? (pn::packed_loc(c) ? (c->spatial ? 2 : 1) : 0) : 0;
        out[3] = pn::fused_tile_size(v);
        out[4] = v.packed ? v.stages : 0;
        out[5] = v.packed;
    }
    return ok();
}

pn_status pn_launch_count(pn_ctx *c, int64_t *count)
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!count)
        return fail(PN_EINVAL, "pn_launch_count: NULL output");
    *count = c->launches;
    return ok();
}

namespace {
// Autotuner results: the fused-kernel variant found fastest, keyed by the
// pair work (log2 of the tile pairs), the precision and whether the context
// holds one cluster or many.  Kept for the process and, when PN_TUNE_CACHE
// names a file, in that file (one "bucket precision many P unroll packed
// tile stages" line per key, read on the first pn_tune and appended to when
// a new key is tuned).
struct TuneKey {
    int bucket, precision, many;
    bool operator<(const TuneKey &o) const
    {
        if (bucket != o.bucket)
            return bucket < o.bucket;
        if (precision != o.precision)
            return precision < o.precision;
        return many < o.many;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, pn::FusedVariant> g_tune;
bool g_tune_file_read = false;

bool variant_ok(const pn_ctx *c, const pn::FusedVariant &v)
{
    if (!v.packed)
        return (v.P == 1 || v.P == 2 || v.P == 4) && v.unroll >= 1 && v.unroll <= 4;
    return (v.P == 2 || v.P == 4) && (v.unroll == 1 || v.unroll == 2) &&
           pn::packed_layout_ok(v.tile, v.stages) && !(c->spatial && v.tile != pn::kPackTile);
}

// Reads the cache file once (caller holds g_tune_mu); bad lines are skipped.
void read_tune_file()
{
    if (g_tune_file_read)
        return;
    g_tune_file_read = true;
    const char *path = std::getenv("PN_TUNE_CACHE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        TuneKey k;
        pn::FusedVariant v;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d", &k.bucket, &k.precision, &k.many, &v.P,
                        &v.unroll, &v.packed, &v.tile, &v.stages) == 8)
            g_tune[k] = v;
    }
    std::fclose(f);
}

void append_tune_file(const TuneKey &k, const pn::FusedVariant &v)
{
    const char *path = std::getenv("PN_TUNE_CACHE");
    if (!path || !*path)
        return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "%d %d %d %d %d %d %d %d\n", k.bucket, k.precision, k.many, v.P, v.unroll,
                     v.packed, v.tile, v.stages);
        std::fclose(f);
    }
}

pn_status apply_variant(pn_ctx *c, pn::FusedVariant va)
{
    pn::FusedShape fs{};
    PN_CUDA(pn::fused_shape(c, va, &fs), "occupancy");
    const int64_t seg = (c->S / (pn::kMixThreads * va.P) + fs.G) * pn::kMixThreads * va.P;
    if (seg > c->fused_seg_max)
        return fail(PN_EINVAL, "fused variant needs a larger segment buffer");
    c->fused_P = va.P;
    c->fused_unroll = va.unroll;
    c->fused_packed = va.packed != 0;
    if (va.packed) {
        c->fused_tile = va.tile;
        c->fused_stages = va.stages;
    }
    c->fused_occ = fs.occ;
    c->fused_grid = fs.grid;
    c->fused_G = fs.G;
    c->fused_units = pn::fused_units(c->hclu, c->nclu, va, c->hclu);
    if (c->graph_exec) {              // the captured graph holds the old launch shape
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    return upload_clusters(c);
}
}  // namespace

pn_status pn_tune(pn_ctx *c, const double *x, const double *v, const double *m, double *a,
                  int64_t out[6])
{
    if (check_ctx(c) != PN_OK)
        return PN_EINVAL;
    if (!x || !v || !m || !a)
        return fail(PN_EINVAL, "pn_tune: NULL array");
    DeviceGuard g(c->device);
    PN_CUDA(g.err, "cudaSetDevice");
    // scalar: targets per thread x unroll; packed: targets per thread x
    // unroll x (tile, stages)
    static const pn::FusedVariant cand[] = {
        {2, 1, 0, 0, 0}, {2, 2, 0, 0, 0}, {4, 1, 0, 0, 0}, {4, 2, 0, 0, 0},
        {2, 1, 1, 64, 6}, {2, 2, 1, 64, 6}, {4, 1, 1, 64, 6}, {4, 2, 1, 64, 6},
        {2, 1, 1, 64, 4}, {2, 2, 1, 64, 4}, {4, 1, 1, 64, 4}, {4, 2, 1, 64, 4},
        {2, 1, 1, 32, 8}, {2, 2, 1, 32, 8}, {4, 1, 1, 32, 8}, {4, 2, 1, 32, 8}};
    int64_t work = 0;                         // pair work of all clusters, in tiles^2
    for (int k = 0; k < c->nclu; ++k)
        work += (c->hclu[k].ns_pad / pn::kMixTile) * (c->hclu[k].ns_pad / pn::kMixTile);
    int bucket = 0;
    for (int64_t u = work; u > 1; u >>= 1)
        ++bucket;
    const TuneKey key{bucket, c->p.precision, c->nclu > 1 ? 1 : 0};
    pn::FusedVariant best = pn::fused_variant(c);
    double best_ms = -1.0;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        read_tune_file();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && variant_ok(c, it->second)) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached && c->p.precision == PN_MIXED && c->p.pair_kernel == PN_PAIR_FUSED) {
        cudaEvent_t e0, e1;
        PN_CUDA(cudaEventCreate(&e0), "event");
        PN_CUDA(cudaEventCreate(&e1), "event");
        const int was_timing = c->timing_on;
        c->timing_on = 0;
        for (const pn::FusedVariant &cv : cand) {
            if (!variant_ok(c, cv))
                continue;
            pn_status st = apply_variant(c, cv);
            if (st != PN_OK)
                return st;
            PN_CUDA(cudaMemcpyAsync(c->vp, v, sizeof(double) * 3 * (size_t)c->n,
                                    cudaMemcpyDeviceToDevice, c->stream), "copy velocities");
            st = evaluate(c, x, c->vp, m, a, nullptr, 0.0);   // warm-up
            if (st != PN_OK)
                return st;
            PN_CUDA(cudaEventRecord(e0, c->stream), "event");
            for (int r = 0; r < 2 && st == PN_OK; ++r)
                st = evaluate(c, x, c->vp, m, a, nullptr, 0.0);
            PN_CUDA(cudaEventRecord(e1, c->stream), "event");
            PN_CUDA(cudaEventSynchronize(e1), "event sync");
            if (st != PN_OK)
                return st;
            float ms = 0.0f;
            PN_CUDA(cudaEventElapsedTime(&ms, e0, e1), "event time");
            if (best_ms < 0.0 || ms < best_ms) {
                best_ms = ms;
                best = cv;
            }
        }
        c->timing_on = was_timing;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = best;
        append_tune_file(key, best);
    }
    pn_status st = apply_variant(c, best);
    if (st != PN_OK)
        return st;
    if (out) {
        out[0] = best.P;
        out[1] = best.unroll;
        out[2] = cached ? 1 : 0;
        out[3] = best.packed;
        out[4] = pn::fused_tile_size(best);
        out[5] = best.packed ? best.stages : 0;
    }
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
