// pn_internal.h -- context layout and kernel launchers shared by the CUDA
// sources of libpn (not installed; the public ABI is include/pn.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pn.h"

namespace pn {

// Launch shape of the mixed-precision pair kernels (single-precision pairs).
constexpr int kMixThreads = 128;   // threads per block
constexpr int kMixTargets = 2;     // targets held in registers per thread
constexpr int kMixTile = 128;      // sources per shared-memory tile
constexpr int kFlushTiles = 2;     // fused kernel: tiles per single-precision partial
constexpr int kPackTile = 64;      // packed fused kernel: default sources per shared-memory tile
                                   // (the spatial order's box and unit-cost granularity)
constexpr int kPackVals = 9;       // dot-product staged layout (packed kernel form 0, adjoint sweeps): float4 per source
constexpr int kFwdVals = 8;        // law-of-cosines staged layout (packed kernel forms 1, 2): float4 per source
constexpr int kPackFlushSources = 512;  // packed fused kernel: sources per single-precision partial
constexpr int kPackWorkersMax = 4;  // packed fused kernel: stream-K workers per resident block (max)
constexpr int kPackStages = 6;     // packed fused kernel: default one-tile shared buffers
                                   // (tiles between block barriers: half of them)
// Spatial order of the packed kernel by default from this many target-source
// slot pairs per evaluation (sum over clusters of ns_pad^2) on.
constexpr double kSpatialMinPairs = 4294967296.0;
// Far-unit criterion of the spatial order (k_fused_packed): box gap at least
// kFarTheta times the sum of the boxes' largest |d|.
constexpr float kFarTheta = 0.05f;
// Launch shape of the double-precision pair kernels (FP64 mode and energy).
constexpr int kF64Threads = 128;
constexpr int kF64Targets = 1;
constexpr int kF64Tile = 64;
// Star slots are padded to a multiple of this (covers every shape; the fused
// kernel takes up to 4 targets per thread, 512 per block).
constexpr int kPad = 512;
// Threads per block of the O(n) kernels.
constexpr int kGlueThreads = 256;
constexpr int kEpiThreads = 64;    // epilogue blocks: FP64-heavy per star, so spread over every SM
constexpr int kProThreads = 64;    // prologue blocks, likewise (one partial-sum row per block)
constexpr int kGatherThreads = 64; // stream-K gather blocks, likewise

// Values per star written by each pair kernel into its partial-sum buffer.
constexpr int kP1Vals = 6;         // N (3), U, Z, Wr
constexpr int kP2Vals = 10;        // V' (3), Hs (1), Hv (3), E (3)
constexpr int kEVals = 8;          // pot, Smv (3), Snn, Spx (3)
constexpr int kEnergySplitsMax = 32;  // source splits of the energy pair kernel, at most
constexpr int kFusedVals = kP1Vals + kP2Vals;
constexpr int kPackSums = kFusedVals - 1;   // packed fused kernel: the pass-1 sums without Wr
// Near-source pass: sources per tile and values per target.
constexpr int kNearTile = 128;
constexpr int kNearVals = 6;       // P (3), Ee (3)
// Global O(n) sums computed by the prologue (block partials, then totals):
//   Q (3), W over all stars (3), W over far stars (3), SA_far, SB_far, Phi,
//   near-star count (as a double in the block partials), sum of |d_j| (the
//   length scale of the spatial order).
constexpr int kGlobVals = 14;
constexpr int kGlobMeanR = 13;
// Per-block values of the energy epilogue.
constexpr int kEBlockVals = 9;     // eN, ePN, pN (3), pPN (3), sum m/R

// One cluster of the state: a hole (body body0) and ns stars after it.
struct Clu {
    int64_t body0;     // index of the cluster's hole in x, v, m, a
    int64_t ns;        // number of stars
    int64_t slot0;     // first star slot in the record arrays (multiple of kPad)
    int64_t ns_pad;    // star slots, padded to a multiple of kPad
    int64_t unit0;     // first work unit of the fused kernel
    int64_t near0;     // first entry of the cluster's near-record slice
    double G, inv_c2, eps2;
    double r_near;     // near-source radius; <= 0 disables the split
};

struct Shape {
    int threads, targets, tile;     // as above
    int64_t nblk_i;                 // blocks along targets
    int jsplit;                     // source splits (grid.y)
    int tiles_per_split;
    int ntiles;
    int occupancy;                  // resident blocks per SM (pass 2)
};

struct Timing {
    static constexpr int kRing = 64;
    static constexpr int kKernels = 3;   // pass 1, pass 2, near pass
    cudaEvent_t ev0[kKernels][kRing], ev1[kKernels][kRing];
    int head[kKernels], count[kKernels];
    double ms[kKernels];
    int64_t launches[kKernels];
};

}  // namespace pn

struct pn_ctx {
    int64_t n;               // bodies in the state arrays (all clusters)
    int nclu;                // clusters
    int64_t S;               // star slots of all clusters (multiple of kPad)
    int64_t max_ns_pad;      // largest cluster's padded star count
    int64_t NC;              // entries per near-record array (all clusters)
    pn::Clu *hclu;           // host copy of the cluster table
    pn::Clu *d_clu;          // device cluster table
    int *blk_clu;            // device: cluster of each 256-slot block
    bool any_near;           // some cluster has r_near > 0
    bool near_all;           // every cluster has r_near > 0
    bool spatial;            // packed law-of-cosines kernel on Hilbert-ordered slots
    float far_theta;         // spatial order: far-unit criterion (k_fused_packed)
    bool balance;            // spatial order: cost-balanced stream-K workers
    unsigned long long *units_cnt;  // spatial order: [0] far warp-units, [1] all warp-units
    pn_params p;
    int device;
    cudaStream_t stream;
    int sm_count;
    pn::Shape mix, f64;
    int fused_P;             // targets per thread of the fused kernel (1, 2 or 4)
    bool fused_packed;       // packed FP32x2 fused kernel (4 targets per thread)
    int fused_tile;          // packed kernel: sources per shared-memory tile (64 or 32)
    int fused_stages;        // packed kernel: one-tile shared buffers (6, 4 or 8)
    int fused_unroll;        // source-loop unroll of the fused kernel (1 or 2)
    int fused_occ;           // resident fused-kernel blocks per SM
    int64_t fused_grid;      // blocks of the persistent fused kernel (resident)
    int64_t fused_G;         // stream-K workers of the fused kernel
    int64_t fused_seg_max;   // segment buffer length (doubles / kFusedVals), all variants
    int64_t fused_units;     // work units of the fused kernel (all clusters)
    int *wcount;             // next stream-K worker of the packed kernel (zeroed by the prologue)
    int workers_max;         // packed kernel: stream-K workers per resident block, at most
    int worker_units;        // packed kernel: work units per stream-K worker, at least
    unsigned inject_tx;      // test hook: extra bytes each tile's mbarrier expects (0)
    int dbg_inject;          // debug build's test hook: index-check site made to fail (0)

    // scratch, all owned by the context
    double *vp;          // n x 3: velocity at which the force is evaluated
    float4 *mrec;        // mixed records: 5 arrays of S float4
    void *sord;          // mixed: spatial order (pn_order.cu: sorted records, boxes, sort scratch)
    void *bal;           // mixed: cost-balanced stream-K worker boundaries (pn_order.cu)
    int64_t bal_units, bal_G;   // largest unit and worker counts of the packed variants
    double4_32a *drec;   // double records: 4 arrays of S double4_32a
    double *part;        // pair partial sums [jsplit][vals][S] (+ fused segments)
    int64_t part_len;    // doubles in `part`
    double *blk;         // per-block partial sums of the O(n) kernels
    int64_t blk_len;
    double *glob;        // global sums [nclu][kGlobVals]
    float4 *nrec;        // mixed near-source records: 4 arrays of NC
    double4_32a *ndrec;  // double near-source records: 3 arrays of NC
    int *ncount;         // [k] near-star count of cluster k; [nclu + b] prefix offset of block b
    unsigned char *nflag;   // per star slot: 1 if a near source
    double *eout;        // [nclu][8]: energy / momentum results
    int *flag;           // [0] non-finite flag
    unsigned long long *flag_step;   // first step index with a non-finite value
    unsigned *epi_done;  // [nclu] epilogue blocks finished this evaluation (self-resetting)
    int64_t step_counter;
    // energy-drift watchdog (pn_set_watchdog): every wd_every steps (0 = off)
    double wd_tol;
    int64_t wd_every;
    double *wd;          // device: [nclu] reference energies (NaN until taken), then the
                         // first tripping check's relative change and cluster
    unsigned long long *wd_step;   // device: step of the first tripping check

    // RK4 stage buffers (n x 3 each): stage position / velocity, stage
    // acceleration, and the running k-sums of x and v
    double *rk_x, *rk_v, *rk_a, *rk_sx, *rk_sv;
    double *jbuf;            // jerk scratch (allocated by the first pn_jerk / Hermite step)
    double *hj0, *hj1;       // Hermite: jerk at the current state and at the evaluation state
    double *abuf;            // adjoint scratch (allocated by the first VJP call)

    // device copies used by pn_step_host
    double *hx, *hv, *hm, *ha;

    int timing_on;
    bool capturing;          // a CUDA graph is being captured
    pn::Timing tm;

    // the near-source pass's side stream and its fork / join events
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    cudaStream_t adj_stream;   // the adjoint's segment recomputations (created on first use)
    int adj_separate;          // PN_ADJ_SEPARATE: the adjoint's two pair sweeps, not the merged one

    // CUDA graph of pn_step_graph: captured once per (arrays, dt, nsteps)
    cudaStream_t cap_stream;
    cudaGraphExec_t graph_exec;
    const void *graph_key[4];
    double graph_dt;
    int64_t graph_steps;
    int64_t launches;        // kernels launched (a graph replay adds its kernels)
    int64_t graph_launches;  // kernels in the instantiated graph
};

namespace pn {

// O(n) kernels and pair kernels (pn_kernels.cu).  Each returns the first
// launch error (cudaSuccess if none).
cudaError_t launch_kick_drift(pn_ctx *c, double *x, double *v, const double *a, double dt);
cudaError_t launch_rk4_stage(pn_ctx *c, int stage, double *x, double *v, const double *a,
                             double dt);
size_t jerk_buffer_doubles(const pn_ctx *c);
size_t adjoint_buffer_doubles(const pn_ctx *c);
// fwd_saved / srec_saved (mixed contexts with the fused kernel): the 16
// forward pair sums ([value][slot], fused layout) and the staged D-form
// source records of an evaluation at (x, v) without the near-source split;
// nullptr: computed here.
cudaError_t launch_accel_vjp(pn_ctx *c, const double *x, const double *v, const double *m,
                             const double *abar, double *xbar, double *vbar, double *scal,
                             bool accumulate, const double *fwd_saved = nullptr,
                             const float4 *srec_saved = nullptr);
cudaError_t launch_adj_kdk(pn_ctx *c, int stage, double dt, const double *x, const double *v,
                           const double *a, double *xp, double *vp, double *xb, double *vb,
                           double *ab, double *atot, const double *xbA, const double *vpbA);
cudaError_t launch_jerk(pn_ctx *c, const double *x, const double *v, const double *m,
                        const double *a, double *jerk);
cudaError_t launch_hermite(pn_ctx *c, int stage, double *x, double *v, double *a, double *j,
                           const double *a1, const double *j1, double *xe, double *ve,
                           double dt);
// The records of an evaluation (k_prologue; with energy_records the energy's
// double records); then the cluster sums (k_global_sums: totals, near-star
// counts) and the near-source records (k_near_scatter), which the pair
// kernels do not read (except the spatial order's sort: pairs_need_sums).
cudaError_t launch_prologue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            bool energy_records);
cudaError_t launch_global_sums(pn_ctx *c);
cudaError_t launch_near_scatter(pn_ctx *c, const double *x, const double *m);
bool pairs_need_sums(const pn_ctx *c);
cudaError_t launch_pass1(pn_ctx *c);
cudaError_t launch_pass2(pn_ctx *c);
cudaError_t launch_near(pn_ctx *c);
// The epilogue with the hole's reduction (last block of each cluster); with
// v and dt_next > 0 it also takes the next KDK step's kick and drift (x and
// vel are then written).
cudaError_t launch_epilogue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            double *a, double *v, double half_dt, unsigned long long step,
                            double dt_next = 0.0);
cudaError_t launch_energy(pn_ctx *c, const double *x, const double *v, const double *m);
int64_t energy_splits(int64_t S, int sm_count, int64_t max_ns_pad);
cudaError_t launch_watch(pn_ctx *c);   // after launch_energy: compare with the references
cudaError_t launch_energy_on(cudaStream_t st, int64_t S, const Clu *clu, const double *x,
                             const double *v, const double *m, double4_32a *drec, double *part,
                             double *blk, double *out);

pn_status set_error(pn_status s, const char *fmt, ...);

// Debug build: each source file's first failed index check (site 0: none),
// read and cleared; `inject` arms the test hook's site (0: none).  Release
// builds always report none.
cudaError_t debug_take_kernels(int inject, unsigned long long *site, long long *index);
cudaError_t debug_take_order(int inject, unsigned long long *site, long long *index);

void shapes(int64_t S, int64_t max_ns_pad, int sm_count, int occ_mix, int occ_f64, Shape *mix,
            Shape *f64);
cudaError_t occupancy(int *occ_mix, int *occ_f64);
// One launch variant of the fused pair kernel: targets per thread, source
// loop unroll, the packed FP32x2 kernel or the scalar one, and for the packed
// kernel its tile (sources per shared-memory tile) and one-tile buffers.
// Packed (tile, stages): (64, 6) the default, (64, 4) and (32, 8); 32-source
// tiles run on the slot order only (the spatial order works in 64-source
// tiles).
struct FusedVariant {
    int P, unroll, packed, tile, stages;
};
FusedVariant fused_variant(const pn_ctx *c);
bool packed_layout_ok(int tile, int stages);
cudaError_t fused_occupancy(const FusedVariant &v, int *occ);
// The packed pair kernel runs its law-of-cosines form (every cluster splits
// off its near sources); the prologue then stages that form's records.
bool packed_loc(const pn_ctx *c);
cudaError_t launch_fused(pn_ctx *c);
cudaError_t launch_stage_sources(pn_ctx *c, const float4 *rec);
cudaError_t launch_fused_on(pn_ctx *c, const float4 *rec);
bool use_fused(const pn_ctx *c);
bool use_fused_f64(const pn_ctx *c);
cudaError_t launch_fused_f64(pn_ctx *c);
int fused_tile_size(const FusedVariant &v);
struct FusedShape {
    int occ;                 // resident blocks per SM
    int64_t grid, G, units;  // blocks launched, stream-K workers, work units
};
cudaError_t fused_shape(const pn_ctx *c, const FusedVariant &v, FusedShape *out);
int64_t fused_units(const Clu *h, int nclu, const FusedVariant &v, Clu *out);

// Spatial order of the star slots (pn_order.cu).
struct Order {
    float4 *ssrec;     // staged records in sorted order (kFwdVals per slot)
    float4 *box;       // per tile of kPackTile sorted sources: (min d, 0), (max d, max |d|)
    unsigned *keys;    // 2 S sort keys
    int *vals;         // 2 S sort values
    int *perm;         // S: slot of sorted position k (second half of vals)
    int *hist;         // per sort block and digit: counts, then scatter offsets
};
size_t order_buffer_bytes(int64_t S);
Order order_of(pn_ctx *c);
cudaError_t launch_spatial_order(pn_ctx *c);
// Cost-balanced worker boundaries of the packed kernel (NP target pairs per
// thread) on the spatial order: *wb receives the device array wb[0..G].
size_t balance_buffer_bytes(int64_t S, int64_t units, int64_t G);
cudaError_t launch_worker_balance(pn_ctx *c, int NP, const int64_t **wb);

}  // namespace pn
