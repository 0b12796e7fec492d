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
// Launch shape of the double-precision pair kernels (FP64 mode and energy).
constexpr int kF64Threads = 128;
constexpr int kF64Targets = 1;
constexpr int kF64Tile = 64;
// Star slots are padded to a multiple of this (covers both shapes).
constexpr int kPad = 256;
// Threads per block of the O(n) kernels.
constexpr int kGlueThreads = 256;

// Values per star written by each pair kernel into its partial-sum buffer.
constexpr int kP1Vals = 5;         // N (3), U, Y
constexpr int kP2Vals = 9;         // V (3), H (3), E (3)
constexpr int kEVals = 8;          // pot, Smv (3), Snn, Spx (3)
// Global O(n) sums computed by the prologue.
constexpr int kGlobVals = 10;      // Q (3), W (3), SA, SB, Phi, spare
// Per-block values of the energy epilogue.
constexpr int kEBlockVals = 9;     // eN, ePN, pN (3), pPN (3), sum m/R

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
    cudaEvent_t ev0[2][kRing], ev1[2][kRing];
    int head[2], count[2];
    double ms[2];
    int64_t launches[2];
};

}  // namespace pn

struct pn_ctx {
    int64_t n, ns, ns_pad;
    pn_params p;
    double inv_c2;
    int device;
    cudaStream_t stream;
    int sm_count;
    pn::Shape mix, f64;

    // scratch, all owned by the context
    double *vp;          // n x 3: velocity at which the force is evaluated
    float4 *mrec;        // mixed records: 5 arrays of ns_pad float4
    double4_32a *drec;       // double records: 4 arrays of ns_pad double4_32a
    double *part;        // pair partial sums [jsplit][vals][ns_pad]
    int64_t part_len;    // doubles in `part`
    double *blk;         // per-block partial sums of the O(n) kernels
    int64_t blk_len;
    double *glob;        // global sums
    double *eout;        // 8 doubles: energy / momentum result
    int *flag;           // [0] non-finite flag
    unsigned long long *flag_step;   // first step index with a non-finite value
    int64_t step_counter;

    // device copies used by pn_step_host
    double *hx, *hv, *hm, *ha;

    int timing_on;
    pn::Timing tm;
};

namespace pn {

// O(n) kernels and pair kernels (pn_kernels.cu).  Each returns the first
// launch error (cudaSuccess if none).
cudaError_t launch_kick_drift(pn_ctx *c, double *x, double *v, const double *a, double dt);
cudaError_t launch_prologue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            bool energy_records);
cudaError_t launch_pass1(pn_ctx *c);
cudaError_t launch_pass2(pn_ctx *c);
cudaError_t launch_epilogue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            double *a, double *v, double half_dt, unsigned long long step);
cudaError_t launch_energy(pn_ctx *c, const double *x, const double *v, const double *m);

void shapes(int64_t ns_pad, int sm_count, int occ_mix, int occ_f64, Shape *mix, Shape *f64);
cudaError_t occupancy(int *occ_mix, int *occ_f64);

}  // namespace pn
