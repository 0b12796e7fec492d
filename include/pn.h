/*
 * pn.h -- C ABI of libpn: the limited first-order post-Newtonian (1PN)
 * N-body acceleration and integrator of T. Tatekawa, arXiv:1801.07986,
 * on NVIDIA B300 (sm_103a).
 *
 * The system is one heavy body (a black hole, the paper's body "#1") plus
 * n-1 low-mass stars.  The library evaluates
 *   - the hole's acceleration, Section 2, Eq. 1 with Eq. 2 and Eq. 3,
 *   - each star's acceleration, Section 2, Eq. 4 with Eq. 5 and Eq. 6,
 *   - the 1PN energy and momentum, Section 2, Eq. 7 and Eq. 8,
 * with Plummer softening between stars only (Section 4, Eq. 10), and
 * advances the state with a kick-drift-kick leapfrog whose force after the
 * drift is taken at a predicted velocity.
 *
 * Conventions shared by every entry point
 *   - Body 0 is the hole (mass M = m[0]); bodies 1..n-1 are stars.
 *   - x, v, a are n x 3 row-major arrays of double (x, y, z per body);
 *     m is an array of n doubles.
 *   - Pointers passed to pn_accel, pn_step and pn_energy are DEVICE pointers
 *     on the context's device (e.g. torch tensor data_ptr()); pn_step_host
 *     takes HOST pointers.  The caller owns every array it passes; the
 *     library owns its scratch memory, allocated by pn_init and freed by
 *     pn_destroy.
 *   - Work is enqueued on the context's CUDA stream and the calls return
 *     before it finishes, except pn_energy, pn_step_host and pn_sync, which
 *     wait for the stream.
 *   - Every call returns a pn_status and never aborts the process.  On an
 *     error, pn_last_error() gives a message for the calling thread.
 *     Argument errors are caught on the host before anything is launched.
 *     Non-finite accelerations detected on the device are reported by the
 *     next waiting call (pn_sync, pn_energy, pn_step_host) as PN_ENONFINITE,
 *     with the first step index that produced one in the message.
 *   - A context is not thread-safe: one thread at a time per context.
 */
#ifndef PN_H
#define PN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pn_ctx pn_ctx;                  /* opaque, library-owned */

typedef enum {
    PN_OK = 0,
    PN_EINVAL = 1,        /* bad argument (caught on the host)              */
    PN_ENOMEM = 2,        /* device or host allocation failed               */
    PN_ECUDA = 3,         /* a CUDA runtime call failed                     */
    PN_ENONFINITE = 4,    /* a non-finite acceleration was produced         */
    PN_ETIMEOUT = 5,      /* a bounded device-side wait gave up             */
    PN_EUNSUPPORTED = 6,  /* the device is not an sm_103 part               */
    PN_EDRIFT = 7,        /* the energy watchdog saw a drift above its limit */
    PN_EINDEX = 8         /* debug build: a device index check failed       */
} pn_status;

enum { PN_FP64 = 0, PN_MIXED = 1 };            /* pn_params.precision */
enum { PN_VPRED_END = 0, PN_VHALF = 1 };       /* pn_params.vel_mode  */
enum { PN_PAIR_FUSED = 0, PN_PAIR_TWO_PASS = 1 };   /* pn_params.pair_kernel */
enum { PN_KDK = 0, PN_RK4 = 1, PN_HERMITE = 2 };   /* pn_params.integrator  */

/*
 * Physical constants and evaluation mode.
 *   G          gravitational constant (> 0)
 *   c          speed of light (> 0); INFINITY gives the Newtonian equations
 *              (every 1PN term multiplied by exactly 0)
 *   eps        Plummer softening (>= 0) of star-star separations only
 *              (Section 4, Eq. 10); hole-star separations are never softened
 *   precision  PN_FP64: every operation in double precision.
 *              PN_MIXED: pair arithmetic in single precision with the pair
 *              separation formed from a hi/lo split of the hole-relative
 *              positions, per-tile single-precision partial sums carried in
 *              double-single accumulators, and everything O(n) (hole terms,
 *              global sums, assembly, integrator, energy) in double.
 *   vel_mode   velocity at which the force after a drift is evaluated:
 *              PN_VPRED_END  v_half + (dt/2) a_old (second order),
 *              PN_VHALF      v_half.
 *   r_near     (>= 0) stars closer than r_near to the hole are "near"
 *              sources: their hole-relative cross terms (Eq. 6, lines 2-4),
 *              which are large and cancel one another, are summed in a
 *              separate cancellation-free pair form instead of through
 *              global sums.  The result is the same in exact arithmetic;
 *              only rounding changes.  0 disables the split.
 *   pair_kernel PN_PAIR_FUSED: the pass-1 and pass-2 pair sums in a
 *              single sweep over the sources (PN_MIXED: one persistent
 *              kernel; PN_FP64: one double-precision sweep);
 *              PN_PAIR_TWO_PASS: pass 1 (Newtonian sums and the hole's
 *              accumulators) and pass 2 (1PN pair sums) as two kernels.
 *              Same sums, same epilogue (in PN_FP64 bitwise the same).
 *   integrator PN_KDK: kick-drift-kick leapfrog (vel_mode applies), one
 *              force evaluation per step.  PN_RK4: classical fourth-order
 *              Runge-Kutta, the paper's own integrator (Section 4), four
 *              evaluations per step.  PN_HERMITE: fourth-order Hermite with
 *              the jerk (the integrator Section 5 recommends, Appendix A),
 *              two force and jerk evaluations per step.
 */
typedef struct {
    double G;
    double c;
    double eps;
    int precision;
    int vel_mode;
    double r_near;
    int pair_kernel;
    int integrator;
} pn_params;

/*
 * Create a context for n bodies (n >= 2) on CUDA device `device`, enqueuing
 * on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Allocates all scratch memory for n.  Errors: PN_EINVAL (ctx NULL, n < 2,
 * bad params), PN_EUNSUPPORTED (device is not compute capability 10.3),
 * PN_ENOMEM, PN_ECUDA.
 */
pn_status pn_init(pn_ctx **ctx, int64_t n, const pn_params *params, int device,
                  void *cuda_stream);

/* Per-cluster constants of a batched context (see pn_init_batched). */
typedef struct {
    double G;
    double c;      /* INFINITY allowed */
    double eps;
} pn_cluster;

/*
 * A context for many independent clusters evaluated together (one launch of
 * each kernel covers all of them; the pair kernel balances their uneven
 * work over the GPU).  Cluster k holds bodies [offsets[k], offsets[k+1]) of
 * the state arrays, its hole first; offsets[0] = 0 and each cluster has at
 * least 2 bodies.  `clusters[k]` gives its G, c and eps (NULL: every cluster
 * takes params->G, c, eps); the mode fields (precision, vel_mode, r_near,
 * pair_kernel, integrator) come from `params`.  Every entry point then works
 * on the concatenated arrays; pn_energy writes 8 values per cluster.
 * Errors: as pn_init.
 */
pn_status pn_init_batched(pn_ctx **ctx, int n_clusters, const int64_t *offsets,
                          const pn_cluster *clusters, const pn_params *params, int device,
                          void *cuda_stream);

/* Replace the parameters without reallocating; on a batched context every
 * cluster takes the new G, c, eps and r_near.  Waits for the stream.
 * Errors: PN_EINVAL. */
pn_status pn_set_params(pn_ctx *ctx, const pn_params *params);

/* Enqueue subsequent work on another stream of the same device. */
pn_status pn_set_stream(pn_ctx *ctx, void *cuda_stream);

/*
 * a = A(x, v): accelerations of all n bodies (Section 2, Eq. 1-6) at
 * positions x and velocities v, both used as given.  x, v, m, a: device
 * pointers (n x 3, n x 3, n, n x 3 doubles); a must not alias x, v or m.
 * Errors: PN_EINVAL (NULL pointer).
 */
pn_status pn_accel(pn_ctx *ctx, const double *x, const double *v, const double *m,
                   double *a);

/*
 * Advance the state in place by nsteps steps of size dt.
 * PN_KDK (kick-drift-kick):
 *   v_h = v + dt/2 a;  x = x + dt v_h;
 *   v_p = v_h + dt/2 a (PN_VPRED_END) or v_h (PN_VHALF);
 *   a = A(x, v_p);  v = v_h + dt/2 a.
 * PN_RK4: k1 = (v, a), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2),
 *   k4 = f(y + dt k3), y += dt/6 (k1 + 2 k2 + 2 k3 + k4), a = A(y).
 * PN_HERMITE: j = jerk at the entry state, then per step
 *   predict  x_p = x + dt v + dt^2/2 a + dt^3/6 j,  v_p = v + dt a + dt^2/2 j,
 *   twice:   a_1 = A(x_e, v_e), j_1 = jerk(x_e, v_e, a_1),
 *            v_e = v + dt/2 (a + a_1) + dt^2/12 (j - j_1),
 *            x_e = x + dt/2 (v + v_e) + dt^2/12 (a - a_1)
 *   ((x_e, v_e) = (x_p, v_p) in the first pass), and (x, v, a, j) =
 *   (x_e, v_e, a_1, j_1); after the last step a = A(x, v).  The jerk's
 *   precision follows pn_jerk.
 * `a` is carried state: on entry it must hold the acceleration of the entry
 * state (call pn_accel once before the first pn_step); on return it holds
 * the acceleration of the final state.  Device pointers.
 * Errors: PN_EINVAL (NULL pointer, dt not finite or <= 0, nsteps < 0).
 */
pn_status pn_step(pn_ctx *ctx, double *x, double *v, const double *m, double *a,
                  double dt, int64_t nsteps);

/*
 * The jerk (Appendix A): writes a = A(x, v) (the context's precision) and
 * jerk = dA/dt along the trajectory, sum_k [dA/dx_k . v_k + dA/dv_k . a_k],
 * for every body, n x 3 each.  The derivative is taken in forward mode
 * (dual numbers) of the same decomposition the acceleration kernels use,
 * with no near-source split: in double precision in PN_FP64 contexts; in
 * PN_MIXED contexts the dual pair sums run in single precision (hi/lo
 * positions) and everything O(n) in double.  Device pointers; a and jerk must not alias x, v or m.  Allocates
 * its scratch on the first call.  Errors: PN_EINVAL (NULL pointer),
 * PN_ENOMEM, PN_ECUDA; a non-finite jerk is reported by pn_sync as
 * PN_ENONFINITE.
 */
pn_status pn_jerk(pn_ctx *ctx, const double *x, const double *v, const double *m, double *a,
                  double *jerk);

/*
 * Adjoint (vector-Jacobian product) of the accelerations: for the state
 * (x, v), with v the velocities at which A is taken, and a cotangent abar
 * (n x 3) of A(x, v), writes xbar = abar . dA/dx and vbar = abar . dA/dv
 * (n x 3 each, device) and, on the host, scal[2 k] = abar . dA/dM_k and
 * scal[2 k + 1] = abar . dA/d(1/c_k^2) for the hole mass M_k and c_k of
 * cluster k (dA/dc = -2/c^3 dA/d(1/c^2)).  Reverse mode over the same
 * decomposition as the kernels, without the near-source split: in double
 * precision in PN_FP64 contexts; in PN_MIXED contexts the forward pair sums
 * and their reverse run in single precision on hi/lo separations, every
 * per-star and per-cluster term in double.  The paper has no counterpart:
 * it is the gradient of its Eq. 1-6.  Allocates its scratch on the first
 * call; waits.  Errors: PN_EINVAL (NULL pointer, aliasing), PN_ENOMEM,
 * PN_ECUDA.
 */
pn_status pn_accel_vjp(pn_ctx *ctx, const double *x, const double *v, const double *m,
                       const double *abar, double *xbar, double *vbar, double *scal);

/*
 * Adjoint of nsteps PN_KDK steps (pn_step) from (x0, v0), whose entry
 * acceleration is A(x0, v0): given cotangents xbar_T, vbar_T of the final
 * positions and velocities, writes xbar0, vbar0 (the gradient with respect
 * to x0, v0, device, n x 3) and on the host scal[2 k], scal[2 k + 1], the
 * gradient with respect to the hole mass and 1/c^2 of cluster k.  The
 * forward trajectory runs in the context's precision; each step's
 * acceleration is differentiated as pn_accel_vjp does.  Checkpointing: the
 * state is stored every `checkpoint` steps (0: the integer ceiling of
 * sqrt(nsteps)) and each segment is recomputed once on the way back, so
 * memory is (checkpoint + nsteps/checkpoint) x 9n doubles and the forward
 * steps run twice.  In PN_MIXED contexts the recomputation of a segment
 * keeps each step's forward pair sums and staged records for its reverse
 * (34 doubles per star slot per step) and runs on a second, internal
 * stream while the previous segment is reversed, so those buffers and the
 * segment's states are held twice; events order the two streams.
 * Allocates and frees its scratch; waits.
 * Errors: PN_EINVAL, PN_EUNSUPPORTED (integrator other than PN_KDK),
 * PN_ENOMEM, PN_ECUDA, PN_ENONFINITE.
 */
pn_status pn_step_vjp(pn_ctx *ctx, const double *x0, const double *v0, const double *m,
                      double dt, int64_t nsteps, int64_t checkpoint, const double *xbar_T,
                      const double *vbar_T, double *xbar0, double *vbar0, double *scal);

/*
 * The forward half of pn_step_vjp, for callers that run the forward anyway:
 * nsteps PN_KDK steps in place exactly as pn_step (same trajectory, bit for
 * bit), storing the state (x, v, a, n x 3 each) before steps 0, K, 2K, ...
 * into ckpt, K = checkpoint (0: the integer ceiling of sqrt(nsteps)).  ckpt
 * is a caller-owned DEVICE array of ceil(nsteps / K) x 9n doubles; a must
 * hold A(x, v) on entry.  Errors: as pn_step, plus PN_EUNSUPPORTED
 * (integrator other than PN_KDK).
 */
pn_status pn_step_save(pn_ctx *ctx, double *x, double *v, const double *m, double *a, double dt,
                       int64_t nsteps, int64_t checkpoint, double *ckpt);

/*
 * The backward half of pn_step_vjp from the checkpoints pn_step_save wrote
 * for the same (m, dt, nsteps, checkpoint): each segment is recomputed once
 * on the way back (K x 9n doubles of scratch), then differentiated as in
 * pn_step_vjp; the result equals pn_step_vjp's from the same start state.
 * Allocates and frees its scratch; waits.  Errors: as pn_step_vjp.
 */
pn_status pn_step_vjp_saved(pn_ctx *ctx, const double *ckpt, const double *m, double dt,
                            int64_t nsteps, int64_t checkpoint, const double *xbar_T,
                            const double *vbar_T, double *xbar0, double *vbar0, double *scal);

/*
 * pn_step captured into one CUDA graph and launched as a whole: the first
 * call for a given (x, v, m, a, dt, nsteps) records the nsteps steps (every
 * kernel launch of every step) into a graph; later calls with the same
 * arguments replay it with a single launch.  The step index in non-finite
 * reports is the index within the captured sequence.  Kernel timing
 * (pn_set_timing) does not see launches inside the graph.
 * Errors: as pn_step, plus PN_ECUDA if capture or instantiation fails.
 */
pn_status pn_step_graph(pn_ctx *ctx, double *x, double *v, const double *m, double *a,
                        double dt, int64_t nsteps);

/*
 * Autotuner of the fused pair kernel's launch shape: the scalar kernel's
 * targets per thread x source-loop unroll, and the packed FP32x2 kernel's
 * targets per thread x unroll x j-tile (sources per shared-memory tile, 64
 * or 32) x one-tile buffers (6 or 4 at 64 sources, 8 at 32; fewer buffers
 * leave room for more resident blocks; 32-source tiles only without the
 * spatial order).  Times each candidate on the given state (a is
 * overwritten with A(x, v)) and keeps the fastest.  Results are cached per
 * (pair-work bucket, precision, one or many clusters) for the process and,
 * when the environment variable PN_TUNE_CACHE names a file, in that file
 * across processes.  out (may be NULL): [0] targets per thread, [1] unroll,
 * [2] 1 if the result came from the cache, [3] 1 for the packed FP32x2
 * kernel, [4] sources per tile, [5] one-tile buffers (0 for the scalar
 * kernel).  Waits.
 */
pn_status pn_tune(pn_ctx *ctx, const double *x, const double *v, const double *m, double *a,
                  int64_t out[6]);

/*
 * pn_step on HOST arrays: copies x, v, m, a to device buffers owned by the
 * context, runs nsteps steps, copies x, v, a back, and waits.  The arrays
 * may be pageable or pinned host memory.  Errors: as pn_step, plus
 * PN_ENONFINITE.
 */
pn_status pn_step_host(pn_ctx *ctx, double *x, double *v, const double *m, double *a,
                       double dt, int64_t nsteps);

/*
 * 1PN energy (Eq. 7) and momentum (Eq. 8) of the state (x, v).  An FP64
 * context sums the star pairs in double precision; a mixed context sums
 * them as double-single pairs of floats (about 48 bits, on the FP32 pipe;
 * within about 1e-15 relative of the FP64 sums on a 16384-body Plummer
 * cluster); every per-star and per-cluster term is double precision in
 * both.  Device pointers in,
 * host array out[8] (out[8 n_clusters] on a batched context, 8 per cluster):
 *   out[0]  Newtonian energy         out[1]    1/c^2 part of Eq. 7
 *   out[2..4] Newtonian momentum     out[5..7] 1/c^2 part of Eq. 8
 * (E = out[0] + out[1], P = out[2..4] + out[5..7]).  The contract is these
 * eight values per cluster: the Newtonian and 1PN parts are kept apart (a
 * superset of E_N, E_1PN and P) so that a caller can follow each order's
 * conservation.  Waits for the stream.
 * Errors: PN_EINVAL, PN_ENONFINITE (pending from earlier steps), PN_EDRIFT
 * (pending from the watchdog).
 */
pn_status pn_energy(pn_ctx *ctx, const double *x, const double *v, const double *m,
                    double *out);

/* Wait for the context's stream; PN_ENONFINITE if a non-finite acceleration
 * was produced since the last report (the flag is then cleared). */
pn_status pn_sync(pn_ctx *ctx);

/*
 * Kernel timing for measurement.  While enabled, pn_accel/pn_step record a
 * CUDA event pair on the context's stream around each pair-interaction
 * kernel launch.  pn_get_timing waits for the stream and returns, for
 * kernel k (0 = pass 1 of the two-pass kernels, 1 = pass 2 or the fused pair
 * kernel, 2 = near-source pass), the summed milliseconds and launch count
 * since timing was last enabled.
 */
pn_status pn_set_timing(pn_ctx *ctx, int enable);
pn_status pn_get_timing(pn_ctx *ctx, double ms[3], int64_t launches[3]);

/*
 * Work split of the mixed-precision packed pair kernel when it runs on the
 * spatial (Hilbert) order of the stars: out[0] the (warp, source tile) units
 * whose target and source boxes were far enough apart for the pair
 * separation from the high single-precision parts alone, out[1] all units,
 * counted on the device since pn_init or the last pn_set_timing(ctx, 1).
 * Each unit is 64 x (2 x targets per thread x 32) pairs.  Waits for the
 * stream.  Errors: PN_EINVAL (NULL out), PN_ECUDA.
 */
pn_status pn_get_pair_stats(pn_ctx *ctx, int64_t out[2]);

/*
 * Launch shape of the pair kernels for this context: out[0] threads per
 * block, out[1] targets per thread, out[2] sources per shared-memory tile,
 * out[3] blocks along targets, out[4] source splits (two-pass) or
 * stream-K workers (fused), out[5] resident blocks per SM, out[6] SM count,
 * out[7] 1 if the fused kernel is the packed FP32x2 one.
 */
pn_status pn_get_launch(pn_ctx *ctx, int64_t out[8]);

/*
 * The fused pair kernel's instantiation for this context (mixed precision,
 * fused pair kernel): out[0] targets per thread, out[1] source-loop unroll,
 * out[2] form of the hole term (0 dot-product form, 1 law-of-cosines form,
 * 2 law-of-cosines form on the spatial order), out[3] sources per tile,
 * out[4] shared-memory tile buffers (stages; 0 for the scalar kernel),
 * out[5] 1 if it is the packed FP32x2 kernel.  All zero when the context
 * does not run the fused kernel (FP64 or PN_PAIR_TWO_PASS).  No device work.
 * Errors: PN_EINVAL (bad context, NULL out).
 */
pn_status pn_get_variant(pn_ctx *ctx, int64_t out[6]);

/*
 * Number of CUDA kernels this context has launched since pn_init (host-side
 * count, no synchronisation).  A pn_step_graph replay adds the kernels of the
 * captured graph; capturing it adds nothing.  Takes a NULL count as
 * PN_EINVAL.
 */
pn_status pn_launch_count(pn_ctx *ctx, int64_t *count);

/*
 * Energy-drift watchdog.  With rel_tol > 0, every `every` steps of pn_step,
 * pn_step_graph and pn_step_host (counted by the context's step counter)
 * the library evaluates Eq. 7 on the state, as pn_energy does, and compares
 * each cluster's total E = E_N + E_1PN with its reference on the device:
 * the first check after this call takes the reference, later ones trip when
 * |E - E_ref| / |E_ref| > rel_tol (or is not finite).  A trip is reported
 * by the next waiting call (pn_sync, pn_energy, pn_step_host) as PN_EDRIFT,
 * with the first tripping step, the change and the cluster in the message;
 * the reference stays, so later checks compare with it too.  This flags
 * the failure mode Section 4 shows, an energy jump at a close scattering
 * off the hole that the step does not resolve.  Each check costs one
 * energy evaluation (an FP64 O(n^2) pair sum, about 15 steps' time of a
 * mixed-precision context at n = 16384).  The adjoint's forward
 * recomputations are not checked.  Calling again resets the references;
 * rel_tol = 0 turns the watchdog off.  A captured pn_step_graph sequence is
 * captured again after this call.  Allocates a few bytes on first use.
 * Errors: PN_EINVAL (rel_tol < 0 or not finite, every < 1 with rel_tol > 0),
 * PN_ENOMEM, PN_ECUDA.
 */
pn_status pn_set_watchdog(pn_ctx *ctx, double rel_tol, int64_t every);

/*
 * Energy and momentum like pn_energy, for callers that cannot allocate
 * device memory (their GPU memory belongs to another allocator, or they
 * must not allocate after start-up): no context, no cudaMalloc.  The paper
 * has no counterpart; this is a deployment convenience.
 *   n         number of bodies, 2 <= n <= PN_NOALLOC_MAX_BODIES; larger n
 *             is rejected with PN_EINVAL
 *   G, c, eps as in pn_params (c may be INFINITY)
 *   x, v, m   device pointers as for pn_energy
 *   out       DEVICE pointer to 8 doubles, written as pn_energy's out[]
 * Work is enqueued on `cuda_stream` of `device` and the call returns
 * without waiting.  The scratch is a fixed array inside the library (about
 * 5 MiB on every device that loads libpn, held until exit), shared by all
 * calls: calls whose work overlaps on the GPU race on it and must be
 * serialised by the caller; each call writes every scratch byte it reads,
 * so nothing carries over from the previous call.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it for the process; make that first call before any stream
 * capture, and do not call this entry point on a device after
 * cudaDeviceReset (the cached address then no longer exists).  The call
 * reads no host memory after it returns: its one-cluster table is passed
 * by value to a kernel.  Errors: PN_EINVAL (bad arguments, n too large),
 * PN_ECUDA.
 */
#define PN_NOALLOC_MAX_BODIES 16384
pn_status pn_energy_noalloc(int device, void *cuda_stream, int64_t n, double G, double c,
                            double eps, const double *x, const double *v, const double *m,
                            double *out);

/*
 * Roofline denominators measured on `device` now: out[0] FP32 FMA TFLOP/s,
 * out[1] FP64 FMA TFLOP/s, out[2] single-precision rsqrt Gop/s, out[3] SM
 * count, out[4] packed FP32x2 FMA TFLOP/s (independent FMA chains on every
 * SM, CUDA-event timed; allocates and frees a small buffer; waits for the
 * stream).  The paper has no counterpart.  Errors: PN_EINVAL, PN_ENOMEM,
 * PN_ECUDA.
 */
pn_status pn_measure_peaks(int device, void *cuda_stream, double out[5]);

/* Message of the last failed call on this thread ("" if none). */
const char *pn_last_error(void);

/* Free the context and its device memory (NULL is a no-op). */
void pn_destroy(pn_ctx *ctx);

/* Library version, 100 * major + minor. */
int pn_version(void);

/*
 * 1 in the debug build (libpn_debug.so, compiled with PN_DEBUG_CHECKS), 0
 * otherwise.  In the debug build the kernels of the acceleration, step and
 * energy paths check their global-memory indices against the buffers'
 * extents: a failing check records the site and index and substitutes a
 * valid index (no trap, no early exit), and the next waiting call returns
 * PN_EINDEX with the site and index in the message.  The arithmetic is the
 * release build's.
 */
int pn_debug_checks(void);

#ifdef __cplusplus
}
#endif

#endif /* PN_H */
