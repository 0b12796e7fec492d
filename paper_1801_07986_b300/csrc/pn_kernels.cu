// pn_kernels.cu -- CUDA kernels of libpn for sm_103a.
//
// One evaluation of the accelerations A(x, v) of the limited-1PN system of
// Tatekawa (arXiv:1801.07986, Section 2, Eq. 1-6) runs as
//
//   prologue   O(n)   hole-relative star records + global sums (Q, W, ...)
//   pass 1     O(n^2) per star i: N_i = sum_j m_j x_ij / r_ij^3,
//                     U_i = sum_j m_j / r_ij, Z_i = sum_j m_j / r_ij^3 and
//                     Wr_i = sum_j m_j R_j^2 / r_ij^3 (the hole's three-body
//                     sum uses Y_i = sum_j m_j (R_i^2 - R_j^2)/r_ij^3 = R_i^2 Z_i - Wr_i)
//   pass 2     O(n^2) per star i: the velocity-dependent 1PN pair sums
//   epilogue   O(n)   assembles each star's acceleration from passes 1 and 2
//                     and the hole's three-body terms from pass 1
//   hole       O(n)   deterministic reduction of the hole's terms
//
// The state may hold several independent clusters (a hole and its stars
// each); every kernel finds its cluster in a small table (struct Clu), so a
// single cluster is the one-entry case.
//
// The pair sums are regrouped algebraically (exactly, in real arithmetic)
// so that each pair costs one reciprocal square root and a handful of
// FMAs; the groupings are stated next to each kernel.  x_ij = x_i - x_j,
// v_ij = v_i - v_j, d_j = x_j - x_hole, R_j = |d_j|, r_ij is the softened
// star-star distance sqrt(|x_ij|^2 + eps^2) (Eq. 10).
#include <math.h>
#include <stdint.h>

#include "pn_device.cuh"

namespace pn {

// ------------------------------------------------------------- helpers --

// Double-single running sum: hi + lo carries ~48 significant bits.  Each
// tile's single-precision partial is added with Knuth's TwoSum.
__device__ __forceinline__ void ds_add(float &hi, float &lo, float p)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += e;
}

// 1/sqrt(s2) in double: single-precision seed refined by two Newton steps
// y <- y (3/2 - s2/2 y^2) (quadratic convergence: ~2^-22 -> 2^-44 -> round-off).
__device__ __forceinline__ double rsqrt_f64(double s2)
{
    double y = (double)rsqrtf((float)s2);
    const double h = 0.5 * s2;
    y = y * fma(-h, y * y, 1.5);
    y = y * fma(-h, y * y, 1.5);
    return y;
}

// --------------------------------------------------------- integrator --

// Kick and drift of every body (hole included):
//   v_h = v + h a;  x += dt v_h;  v_p = v_h + h a (mode 0) or v_h (mode 1).
// v is overwritten with v_h; the final kick is applied by the epilogue.
__global__ void k_kick_drift(int64_t n3, double *__restrict__ x, double *__restrict__ v,
                             const double *__restrict__ a, double *__restrict__ vp, double h,
                             double dt, int mode)
{
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < n3;
         q0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = PN_IDX(q0, n3, 1);
        const double aq = a[q];
        const double vh = fma(h, aq, v[q]);
        v[q] = vh;
        x[q] = fma(dt, vh, x[q]);
        vp[q] = mode == 0 ? fma(h, aq, vh) : vh;
    }
}

// Classical RK4 (the paper's Section 4 integrator) for x' = v, v' = A, in
// stages around the force evaluations.  Buffers: (xs, vs) the stage state,
// ka the stage acceleration just evaluated, (sx, sv) the running k-sums.
//   stage 0: sx = v, sv = a;              xs = x + h/2 v,  vs = v + h/2 a
//   stage 1: sx += 2 vs, sv += 2 ka;      xs = x + h/2 vs, vs = v + h/2 ka
//   stage 2: sx += 2 vs, sv += 2 ka;      xs = x + h vs,   vs = v + h ka
//   stage 3: x += h/6 (sx + vs),  v += h/6 (sv + ka)
__global__ void k_rk4_stage(int stage, int64_t n3, double *__restrict__ x, double *__restrict__ v,
                            const double *__restrict__ a, const double *__restrict__ ka,
                            double *__restrict__ xs, double *__restrict__ vs,
                            double *__restrict__ sx, double *__restrict__ sv, double h)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (stage == 0) {
            sx[q] = v[q];
            sv[q] = a[q];
            xs[q] = x[q] + 0.5 * h * v[q];
            vs[q] = v[q] + 0.5 * h * a[q];
        } else if (stage < 3) {
            const double kx = vs[q], kv = ka[q];
            sx[q] += 2.0 * kx;
            sv[q] += 2.0 * kv;
            const double f = stage == 1 ? 0.5 * h : h;
            xs[q] = x[q] + f * kx;
            vs[q] = v[q] + f * kv;
        } else {
            x[q] = x[q] + h / 6.0 * (sx[q] + vs[q]);
            v[q] = v[q] + h / 6.0 * (sv[q] + ka[q]);
        }
    }
}

// ------------------------------------------------------------ prologue --

// Staged source records for k_fused_packed from mixed records rec (5 arrays
// of S float4: (hi d, m), (lo d, R^2), (v, C), (-e/1.5, 0), (w, 0)):
// srec[t][0..8] = (-h, -h) pairs of the position split, (m, m), (R^2, R^2),
// and (f, f) for every other field.
__device__ __forceinline__ void stage_source(float4 *__restrict__ o, float4 A, float4 B, float4 Cs,
                                             float4 D, float4 E)
{
    o[0] = make_float4(-A.x, -A.x, -A.y, -A.y);
    o[1] = make_float4(-A.z, -A.z, A.w, A.w);
    o[2] = make_float4(-B.x, -B.x, -B.y, -B.y);
    o[3] = make_float4(-B.z, -B.z, B.w, B.w);
    o[4] = make_float4(Cs.x, Cs.x, Cs.y, Cs.y);
    o[5] = make_float4(Cs.z, Cs.z, Cs.w, Cs.w);
    o[6] = make_float4(D.x, D.x, D.y, D.y);
    o[7] = make_float4(D.z, D.z, E.x, E.x);
    o[8] = make_float4(E.y, E.y, E.z, E.z);
}

// Staged source records of the law-of-cosines form of k_fused_packed
// (kFwdVals float4; the fields are stated above packed_pair) from the mixed
// records A = (hi d, m), B = (lo d, R^2), C = (v, C), E = (w, 0) and the
// hole-term coefficients a = -G M/(6 R^3), cp = C + a (R^2 + eps^2).
__device__ __forceinline__ void stage_source_fwd(float4 *__restrict__ o, float4 A, float4 B,
                                                 float4 Cs, float4 E, float a, float cp)
{
    o[0] = make_float4(-A.x, -A.x, -A.y, -A.y);
    o[1] = make_float4(-A.z, -A.z, A.w, A.w);
    o[2] = make_float4(-B.x, -B.x, -B.y, -B.y);
    o[3] = make_float4(-B.z, -B.z, a, a);
    o[4] = make_float4(Cs.x, Cs.x, Cs.y, Cs.y);
    o[5] = make_float4(Cs.z, Cs.z, cp, cp);
    o[6] = make_float4(E.x, E.x, E.y, E.y);
    o[7] = make_float4(E.z, E.z, B.w, B.w);
}


// Per star slot t of cluster k (star j = body0 + 1 + (t - slot0); slots past
// the cluster's stars are padding):
//   d_j = x_j - x_hole, R_j = |d_j|,
//   c_j = G M (3/(2 R_j) + eps^2/(4 R_j^3)),   e_j = G M d_j/(2 R_j^3),
//   w_j = m_j d_j / R_j^3.
// A star with R_j < r_near is a near source: its c_j, e_j and w_j are left
// out of the main records and of the far sums below (the near pass sums its
// hole-relative cross terms pair by pair instead).  Per-block sums:
//   Q = sum m_j v_j, W = sum w_j (all), W_far = sum_far w_j,
//   SA_far = sum_far 5 m_j/(4 R_j), SB_far = sum_far m_j (R_j^2 + eps^2)/(4 R_j^3),
//   Phi = sum m_j / R_j, and the number of near stars.
// Records, with C = c/1.5 - 4/3 |v|^2:
//          mixed  A = (hi(d), m) B = (lo(d), R^2) C = (v, C) D = (-e/1.5, 0) E = (w, 0)
//          double A = (d, m)     B = (v, R^2)    C = (-e/1.5, C)   D = (w, 0)
// Energy records (double): A = (d, m), B = (v, 0).
// Mixed mode also writes the packed kernel's staged records: the
// law-of-cosines layout (stage_source_fwd) when `loc`, else stage_source's.
template <int MODE>   // 0 mixed, 1 double, 2 energy
__global__ void __launch_bounds__(kProThreads)
k_prologue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
           const double *__restrict__ x, const double *__restrict__ vel,
           const double *__restrict__ m, float4 *__restrict__ mrec,
           double4_32a *__restrict__ drec, unsigned char *__restrict__ nflag,
           double *__restrict__ blk, int *__restrict__ wcount, int loc)
{
    // mixed: the staged source records of the packed pair kernel follow the
    // five record arrays
    float4 *__restrict__ srec = mrec + 5 * S;
    __shared__ double sh[kGlobVals][kProThreads];
    const int64_t t = PN_IDX((int64_t)blockIdx.x * kProThreads + threadIdx.x, S, 2);
    if (wcount && t == 0)
        *wcount = 0;          // the packed pair kernel's worker counter, for this evaluation
    const Clu C = clu[cluster_of_block(blk_clu, (int64_t)blockIdx.x * kProThreads / kGlueThreads)];
    const int64_t lt = t - C.slot0;
    const double G = C.G, eps2 = C.eps2;
    double g[kGlobVals];
#pragma unroll
    for (int k = 0; k < kGlobVals; ++k)
        g[k] = 0.0;
    if (lt < C.ns) {
        const int64_t j = C.body0 + 1 + PN_IDX(lt, C.ns, 3), h = C.body0;
        const double d0 = x[3 * j] - x[3 * h], d1 = x[3 * j + 1] - x[3 * h + 1],
                     d2 = x[3 * j + 2] - x[3 * h + 2];
        const double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double R = sqrt(R2);
        const double iR = 1.0 / R;
        const double iR3 = iR * iR * iR;
        const double mj = m[j];
        const double M = m[h];
        const double v0 = vel[3 * j], v1 = vel[3 * j + 1], v2 = vel[3 * j + 2];
        const bool near = MODE != 2 && R < C.r_near;
        const double far = near ? 0.0 : 1.0;
        const double cj = far * G * M * (1.5 * iR + 0.25 * eps2 * iR3);
        const double ef = far * 0.5 * G * M * iR3;
        const double wf = mj * iR3;
        const double c3 = cj / 1.5 - (4.0 / 3.0) * (v0 * v0 + v1 * v1 + v2 * v2);
        const double e3 = -ef / 1.5;
        if (MODE == 0) {
            const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2;
            const float4 rA = make_float4(h0, h1, h2, (float)mj);
            const float4 rB = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1),
                                          (float)(d2 - (double)h2), (float)R2);
            const float4 rC = make_float4((float)v0, (float)v1, (float)v2, (float)c3);
            const float4 rD = make_float4((float)(e3 * d0), (float)(e3 * d1), (float)(e3 * d2), 0.0f);
            const float4 rE = make_float4((float)(far * wf * d0), (float)(far * wf * d1),
                                          (float)(far * wf * d2), 0.0f);
            mrec[t] = rA;
            mrec[S + t] = rB;
            mrec[2 * S + t] = rC;
            mrec[3 * S + t] = rD;
            mrec[4 * S + t] = rE;
            if (loc) {
                const double a = 0.5 * e3;    // -G M/(6 R^3) (0 for near sources)
                stage_source_fwd(srec + kFwdVals * t, rA, rB, rC, rE, (float)a,
                                 (float)(c3 + a * (R2 + eps2)));
            } else {
                stage_source(srec + kPackVals * t, rA, rB, rC, rD, rE);
            }
        } else if (MODE == 1) {
            drec[t] = make_double4_32a(d0, d1, d2, mj);
            drec[S + t] = make_double4_32a(v0, v1, v2, R2);
            drec[2 * S + t] = make_double4_32a(e3 * d0, e3 * d1, e3 * d2, c3);   // (-e/1.5, C)
            drec[3 * S + t] = make_double4_32a(far * wf * d0, far * wf * d1, far * wf * d2, 0.0);
        } else {
            drec[t] = make_double4_32a(d0, d1, d2, mj);
            drec[S + t] = make_double4_32a(v0, v1, v2, 0.0);
        }
        if (MODE != 2)
            nflag[t] = near ? 1 : 0;
        g[0] = mj * v0;
        g[1] = mj * v1;
        g[2] = mj * v2;
        g[3] = wf * d0;
        g[4] = wf * d1;
        g[5] = wf * d2;
        g[6] = far * wf * d0;
        g[7] = far * wf * d1;
        g[8] = far * wf * d2;
        g[9] = far * 1.25 * mj * iR;
        g[10] = far * 0.25 * mj * (R2 + eps2) * iR3;
        g[11] = mj * iR;
        g[12] = near ? 1.0 : 0.0;
        g[kGlobMeanR] = R;
    } else {
        // padding: zero mass far away, distinct positions
        const double px = 1.0e4 + (double)(lt - C.ns);
        if (MODE == 0) {
            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            mrec[t] = make_float4((float)px, 0.0f, 0.0f, 0.0f);
            for (int k = 1; k < 5; ++k)
                mrec[k * S + t] = z;
            if (loc)
                stage_source_fwd(srec + kFwdVals * t, mrec[t], z, z, z, 0.0f, 0.0f);
            else
                stage_source(srec + kPackVals * t, mrec[t], z, z, z, z);
        } else {
            drec[t] = make_double4_32a(px, 0.0, 0.0, 0.0);
            const int nk = MODE == 1 ? 4 : 2;
            for (int k = 1; k < nk; ++k)
                drec[k * S + t] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        }
        if (MODE != 2)
            nflag[t] = 0;
    }
    if (MODE == 2)
        return;   // block-uniform
    block_sum<kGlobVals, kProThreads>(g, sh);
    if (threadIdx.x < kGlobVals)
        blk[(int64_t)blockIdx.x * kGlobVals + threadIdx.x] = sh[threadIdx.x][0];
}

// One block per cluster: totals of its prologue blocks (kProThreads slots
// each, fixed order) into glob[k][.], the exclusive prefix of the near-star
// counts of its kGlueThreads-slot blocks (the near scatter's blocks) into
// ncount[nclu + b], the count into ncount[k], and zero-mass padding of its
// near-record slice up to the next multiple of kNearTile.
template <int MODE>   // 0 mixed, 1 double
__global__ void __launch_bounds__(kGlueThreads)
k_global_sums(const Clu *__restrict__ clu, int nclu, const double *__restrict__ blk,
              double *__restrict__ glob, int *__restrict__ ncount, float4 *__restrict__ nrec,
              double4_32a *__restrict__ ndrec, int64_t NC)
{
    __shared__ double sh[kGlobVals][kGlueThreads];
    __shared__ int wsum[kGlueThreads / 32];
    constexpr int kSub = kGlueThreads / kProThreads;    // prologue blocks per near-scatter block
    const int k = blockIdx.x;
    const Clu C = clu[k];
    const int64_t b0 = C.slot0 / kGlueThreads;
    const int64_t nblk = C.ns_pad / kGlueThreads;
    const double *cb = blk + b0 * kSub * kGlobVals;
    sum_blocks<kGlobVals>(cb, nblk * kSub, sh);
    if (threadIdx.x < kGlobVals)
        glob[(int64_t)k * kGlobVals + threadIdx.x] = sh[threadIdx.x][0];
    // near-star count of near-scatter block b
    auto count_of = [&](int64_t b) {
        int n = 0;
#pragma unroll
        for (int q = 0; q < kSub; ++q)
            n += (int)cb[(b * kSub + q) * kGlobVals + 12];
        return n;
    };
    // exclusive prefix of block counts: each thread owns a contiguous chunk;
    // the chunk totals are scanned by warp shuffles, then across the warps
    const int64_t chunk = (nblk + kGlueThreads - 1) / kGlueThreads;
    const int64_t c0 = threadIdx.x * chunk;
    const int64_t c1 = c0 + chunk < nblk ? c0 + chunk : nblk;
    int local = 0;
    for (int64_t b = c0; b < c1; ++b)
        local += count_of(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        wsum[wid] = incl;
    __syncthreads();
    int run = incl - local, nn = 0;
#pragma unroll
    for (int q = 0; q < kGlueThreads / 32; ++q) {
        run += q < wid ? wsum[q] : 0;
        nn += wsum[q];
    }
    if (threadIdx.x == 0)
        ncount[k] = nn;
    for (int64_t b = c0; b < c1; ++b) {
        ncount[nclu + b0 + b] = run;
        run += count_of(b);
    }
    const int npad = (int)((nn + kNearTile - 1) / kNearTile * kNearTile);
    for (int q = nn + threadIdx.x; q < npad; q += kGlueThreads) {
        const int64_t e = C.near0 + q;
        const double px = 1.0e4 + (double)(q - nn);
        if (MODE == 0) {
            nrec[e] = make_float4((float)px, 0.0f, 0.0f, 0.0f);
            nrec[NC + e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            nrec[2 * NC + e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            nrec[3 * NC + e] = make_float4(1.0f, __int_as_float(-1), 0.0f, 0.0f);
        } else {
            ndrec[e] = make_double4_32a(px, 0.0, 0.0, 0.0);
            ndrec[NC + e] = make_double4_32a(0.0, 0.0, 1.0, -1.0);
            ndrec[2 * NC + e] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        }
    }
}

// Near-source records in slot order within each cluster (deterministic
// block scan of the flags), slice of cluster k starting at clu.near0:
//   mixed  NA = (hi(d), m)  NB = (lo(d), 5/(4R))  NC = (w, 1/(4R^3))
//          ND = (R^2 + eps^2, global slot bits, 0, 0)
//   double NA = (d, m)  NB = (5/(4R), 1/(4R^3), R^2 + eps^2, global slot)  NC = (w, 0)
template <int MODE>
__global__ void __launch_bounds__(kGlueThreads)
k_near_scatter(const Clu *__restrict__ clu, int nclu, const int *__restrict__ blk_clu,
               const double *__restrict__ x, const double *__restrict__ m,
               const unsigned char *__restrict__ nflag, const int *__restrict__ ncount,
               float4 *__restrict__ nrec, double4_32a *__restrict__ ndrec, int64_t NC)
{
    __shared__ int wsum[kGlueThreads / 32];
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    const Clu C = clu[cluster_of_block(blk_clu, blockIdx.x)];
    const int64_t lt = t - C.slot0;
    const bool near = lt < C.ns && nflag[t];
    const unsigned mask = __ballot_sync(0xffffffffu, near);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        wsum[warp] = __popc(mask);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < warp; ++q)
        before += wsum[q];
    if (!near)
        return;
    const int64_t pos = PN_IDX(C.near0 + ncount[nclu + blockIdx.x] + before +
                                   __popc(mask & ((1u << lane) - 1u)), NC, 4);
    const int64_t j = C.body0 + 1 + lt, h = C.body0;
    const double d0 = x[3 * j] - x[3 * h], d1 = x[3 * j + 1] - x[3 * h + 1],
                 d2 = x[3 * j + 2] - x[3 * h + 2];
    const double R2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double R = sqrt(R2);
    const double iR = 1.0 / R;
    const double iR3 = iR * iR * iR;
    const double mj = m[j];
    const double A = 1.25 * iR, B = 0.25 * iR3, w = mj * iR3;
    if (MODE == 0) {
        const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2;
        nrec[pos] = make_float4(h0, h1, h2, (float)mj);
        nrec[NC + pos] = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1),
                                     (float)(d2 - (double)h2), (float)A);
        nrec[2 * NC + pos] = make_float4((float)(w * d0), (float)(w * d1), (float)(w * d2), (float)B);
        nrec[3 * NC + pos] = make_float4((float)(R2 + C.eps2), __int_as_float((int)t), 0.0f, 0.0f);
    } else {
        ndrec[pos] = make_double4_32a(d0, d1, d2, mj);
        ndrec[NC + pos] = make_double4_32a(A, B, R2 + C.eps2, (double)t);
        ndrec[2 * NC + pos] = make_double4_32a(w * d0, w * d1, w * d2, 0.0);
    }
}

// ------------------------------------------------- pair kernels: mixed --

struct MixTarget {
    float hx, hy, hz, lx, ly, lz;   // hi/lo split of d_i
    float vx, vy, vz;               // 8/3 v_i, v_i the velocity of target i (pass 2)
};

// The pair terms, shared by the two-pass and the fused kernels.  Records of
// source j: A = (hi(d_j), m_j), B = (lo(d_j), R_j^2), C = (v_j, C_j),
// D = (-e_j/1.5, 0), E = (w_j, 0) with C_j = c_j/1.5 - 4/3 |v_j|^2.
// x_ij = (hi_i - hi_j) + (lo_i - lo_j) keeps ~48 bits of the difference.
constexpr float kEightThirds = 8.0f / 3.0f;

struct PairGeo {
    float dx, dy, dz, s2, is, mj, mis, mis3;
    float wx, wy, wz;
};

template <bool MASK>
__device__ __forceinline__ PairGeo pair_geo(const MixTarget &tg, const float4 &A, const float4 &B,
                                            float eps2, bool self)
{
    PairGeo g;
    g.dx = (tg.hx - A.x) + (tg.lx - B.x);
    g.dy = (tg.hy - A.y) + (tg.ly - B.y);
    g.dz = (tg.hz - A.z) + (tg.lz - B.z);
    g.s2 = fmaf(g.dx, g.dx, fmaf(g.dy, g.dy, fmaf(g.dz, g.dz, eps2)));
    g.mj = A.w;
    if (MASK) {
        g.s2 = self ? 1.0f : g.s2;
        g.mj = self ? 0.0f : g.mj;
    }
    g.is = rsqrt_approx(g.s2);
    g.mis = g.mj * g.is;
    g.mis3 = g.mis * (g.is * g.is);
    return g;
}

// Pass-1 sums: N += m_j x_ij/r^3, U += m_j/r, Z += m_j/r^3, Wr += m_j R_j^2/r^3
// (the hole's Y_i = sum m_j (R_i^2 - R_j^2)/r^3 is R_i^2 Z_i - Wr_i).
__device__ __forceinline__ void pass1_terms(const PairGeo &g, float Rj2, float *acc)
{
    acc[0] = fmaf(g.mis3, g.dx, acc[0]);
    acc[1] = fmaf(g.mis3, g.dy, acc[1]);
    acc[2] = fmaf(g.mis3, g.dz, acc[2]);
    acc[3] += g.mis;
    acc[4] += g.mis3;
    acc[5] = fmaf(g.mis3, Rj2, acc[5]);
}

// Pass-2 sums (velocities are those at which A is taken).  With
// |v_ij|^2 = |v_i|^2 + |v_j|^2 - 2 v_i.v_j, the per-pair factor of Eq. 6
// lines 3 and 6 is kappa_ij - 4/3 |v_i|^2, where
//   kappa_ij = (v_j.x_ij)^2/r^2 + C_j - (e_j/1.5).d_i + 8/3 v_i.v_j,
// and the |v_i|^2 part, a constant of target i, multiplies N_i (added by the
// epilogue).  Sums:
//   V' += m_j x_ij/r^3 kappa_ij                  (V = 3/2 (V' - 4/3 |v_i|^2 N_i))
//   Hs += g_ij,  Hv += g_ij v_j,  g_ij = m_j/r^3 [x_ij.(8/3 v_i) - 2 x_ij.v_j]
//                                                (H = 3/2 (Hs v_i - Hv))
//   E  += w_j / r
// V carries Eq. 6 line 3 (without its 4/R_i part) and line 6 (without its
// v_i^2 part): with r_ij^2 - R_i^2 = R_j^2 + eps^2 - 2 d_i.d_j, line 3's
// bracket is 4/R_i + (c_j - e_j.d_i)/(G M).  H is Eq. 6 line 7 (its bracket
// x_ij.v_i - 3/4 x_ij.v_j is 3/8 of g's), E the 1/r_ij part of line 4.
__device__ __forceinline__ void pass2_terms(const PairGeo &g, const MixTarget &tg,
                                            const float4 &C, const float4 &D, float wx, float wy,
                                            float wz, float *acc)
{
    const float is2 = g.is * g.is;
    const float xvj = fmaf(g.dx, C.x, fmaf(g.dy, C.y, g.dz * C.z));
    const float xvi = fmaf(g.dx, tg.vx, fmaf(g.dy, tg.vy, g.dz * tg.vz));
    float k = fmaf(tg.vx, C.x, fmaf(tg.vy, C.y, fmaf(tg.vz, C.z, C.w)));
    k = fmaf(D.x, tg.hx, fmaf(D.y, tg.hy, fmaf(D.z, tg.hz, k)));
    const float h = xvj * is2;
    const float f = g.mis3 * fmaf(h, xvj, k);
    acc[0] = fmaf(f, g.dx, acc[0]);
    acc[1] = fmaf(f, g.dy, acc[1]);
    acc[2] = fmaf(f, g.dz, acc[2]);
    const float gg = g.mis3 * fmaf(-2.0f, xvj, xvi);
    acc[3] += gg;
    acc[4] = fmaf(gg, C.x, acc[4]);
    acc[5] = fmaf(gg, C.y, acc[5]);
    acc[6] = fmaf(gg, C.z, acc[6]);
    acc[7] = fmaf(wx, g.is, acc[7]);
    acc[8] = fmaf(wy, g.is, acc[8]);
    acc[9] = fmaf(wz, g.is, acc[9]);
}

template <bool MASK>
__device__ __forceinline__ void pass1_tile(const float4 *__restrict__ sA,
                                           const float4 *__restrict__ sB, int64_t j0,
                                           const MixTarget (&tg)[kMixTargets],
                                           const int64_t (&ti)[kMixTargets], float eps2,
                                           float (&acc)[kMixTargets][kP1Vals])
{
#pragma unroll 2
    for (int q = 0; q < kMixTile; ++q) {
        const float4 A = sA[q];
        const float4 B = sB[q];
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p) {
            const PairGeo g = pair_geo<MASK>(tg[p], A, B, eps2, MASK && j0 + q == ti[p]);
            pass1_terms(g, B.w, acc[p]);
        }
    }
}

template <bool MASK>
__device__ __forceinline__ void pass2_tile(const float4 *__restrict__ sA,
                                           const float4 *__restrict__ sB,
                                           const float4 *__restrict__ sC,
                                           const float4 *__restrict__ sD,
                                           const float4 *__restrict__ sE, int64_t j0,
                                           const MixTarget (&tg)[kMixTargets],
                                           const int64_t (&ti)[kMixTargets], float eps2,
                                           float (&acc)[kMixTargets][kP2Vals])
{
#pragma unroll 1
    for (int q = 0; q < kMixTile; ++q) {
        const float4 A = sA[q];
        const float4 B = sB[q];
        const float4 C = sC[q];
        const float4 D = sD[q];
        const float4 E = sE[q];
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p) {
            const bool self = MASK && j0 + q == ti[p];
            const PairGeo g = pair_geo<MASK>(tg[p], A, B, eps2, self);
            const float wx = self ? 0.0f : E.x, wy = self ? 0.0f : E.y, wz = self ? 0.0f : E.z;
            pass2_terms(g, tg[p], C, D, wx, wy, wz, acc[p]);
        }
    }
}

// Two-pass grid: (target blocks of all clusters, source splits).  Split s of a
// target block in cluster k sweeps tiles [s tps_k, (s+1) tps_k) of its own
// cluster, tps_k = ceil(ntiles_k / jsplit); splits past the cluster's tiles
// write zeros.
template <int PASS>
__global__ void __launch_bounds__(kMixThreads)
k_pass_mixed(const float4 *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
             const int *__restrict__ blk_clu, double *__restrict__ part)
{
    constexpr int NV = PASS == 1 ? kP1Vals : kP2Vals;
    constexpr int NA = PASS == 1 ? 2 : 5;
    constexpr int TI = kMixThreads * kMixTargets;
    __shared__ float4 sh[NA][kMixTile];
    const int64_t t0 = (int64_t)blockIdx.x * TI;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const float eps2 = (float)C.eps2;
    const int ntiles = (int)(C.ns_pad / kMixTile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;

    MixTarget tg[kMixTargets];
    int64_t ti[kMixTargets];
#pragma unroll
    for (int p = 0; p < kMixTargets; ++p) {
        ti[p] = t0 + p * kMixThreads + threadIdx.x;
        const float4 A = rec[ti[p]];
        const float4 B = rec[S + ti[p]];
        tg[p].hx = A.x; tg[p].hy = A.y; tg[p].hz = A.z;
        tg[p].lx = B.x; tg[p].ly = B.y; tg[p].lz = B.z;
        if constexpr (PASS == 2) {
            const float4 Cc = rec[2 * S + ti[p]];
            tg[p].vx = kEightThirds * Cc.x;
            tg[p].vy = kEightThirds * Cc.y;
            tg[p].vz = kEightThirds * Cc.z;
        } else {
            tg[p].vx = tg[p].vy = tg[p].vz = 0.0f;
        }
    }
    float hi[kMixTargets][NV], lo[kMixTargets][NV];
#pragma unroll
    for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
        for (int k = 0; k < NV; ++k)
            hi[p][k] = lo[p][k] = 0.0f;

    const int tb = blockIdx.y * tps;
    const int te = min(ntiles, tb + tps);
    for (int tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + (int64_t)tile * kMixTile;
        __syncthreads();
        for (int q = threadIdx.x; q < kMixTile; q += kMixThreads) {
#pragma unroll
            for (int k = 0; k < NA; ++k)
                sh[k][q] = rec[k * S + j0 + q];
        }
        __syncthreads();
        float acc[kMixTargets][NV];
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                acc[p][k] = 0.0f;
        const bool diag = (j0 < t0 + TI) && (t0 < j0 + kMixTile);
        if constexpr (PASS == 1) {
            if (diag)
                pass1_tile<true>(sh[0], sh[1], j0, tg, ti, eps2, acc);
            else
                pass1_tile<false>(sh[0], sh[1], j0, tg, ti, eps2, acc);
        } else {
            if (diag)
                pass2_tile<true>(sh[0], sh[1], sh[2], sh[3], sh[4], j0, tg, ti, eps2, acc);
            else
                pass2_tile<false>(sh[0], sh[1], sh[2], sh[3], sh[4], j0, tg, ti, eps2, acc);
        }
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                ds_add(hi[p][k], lo[p][k], acc[p][k]);
    }
#pragma unroll
    for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
        for (int k = 0; k < NV; ++k)
            part[((int64_t)blockIdx.y * NV + k) * S + ti[p]] = (double)hi[p][k] + (double)lo[p][k];
}

// ------------------------------------------- fused pair kernel: mixed --

// Pass 1 and pass 2 in one sweep over the sources: the pair separation,
// distance, rsqrt and the m_j/r^3 factor are computed once per pair and feed
// all 15 sums (N, U, Z, Wr of pass 1; V', H', E of pass 2).
template <int P, int UNROLL, bool MASK>
__device__ __forceinline__ void fused_tile(const float4 *__restrict__ sA,
                                           const float4 *__restrict__ sB,
                                           const float4 *__restrict__ sC,
                                           const float4 *__restrict__ sD,
                                           const float4 *__restrict__ sE, int64_t j0,
                                           const MixTarget (&tg)[P], const int64_t (&ti)[P],
                                           float eps2, float (&acc)[P][kFusedVals])
{
#pragma unroll UNROLL
    for (int q = 0; q < kMixTile; ++q) {
        const float4 A = sA[q];
        const float4 B = sB[q];
        const float4 C = sC[q];
        const float4 D = sD[q];
        const float4 E = sE[q];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const bool self = MASK && j0 + q == ti[p];
            const PairGeo g = pair_geo<MASK>(tg[p], A, B, eps2, self);
            const float wx = self ? 0.0f : E.x, wy = self ? 0.0f : E.y, wz = self ? 0.0f : E.z;
            pass1_terms(g, B.w, acc[p]);
            pass2_terms(g, tg[p], C, D, wx, wy, wz, acc[p] + kP1Vals);
        }
    }
}

// Stream-K persistent launch: the (cluster, target block, source tile) units
// of all clusters are laid out cluster-major, then target-block-major, and
// block b of the G resident blocks takes units [b T / G, (b+1) T / G).  At
// each target-block boundary it writes the finished segment to slot
// (global target block + b) of the segment buffer, which holds
// (target blocks + G) entries of [value][TI targets]; the gather kernel sums
// the segments of each target block in block order.
template <int P, int UNROLL>
__global__ void __launch_bounds__(kMixThreads, P == 4 ? (UNROLL == 3 ? 2 : 3) : (P == 2 ? 5 : 8))
k_fused_mixed(const float4 *__restrict__ rec, int64_t S, const Clu *__restrict__ clu, int nclu,
              int64_t total_units, double *__restrict__ part)
{
    constexpr int TI = kMixThreads * P;
    __shared__ float4 sh[5][kMixTile];
    // double-single running sums (hi, lo) per value, target and thread; kept
    // in shared memory (touched once per tile) to leave registers for the pair loop
    __shared__ float2 run[kFusedVals][P][kMixThreads];
    const int64_t G = gridDim.x;
    int64_t u = (int64_t)blockIdx.x * total_units / G;
    const int64_t u1 = ((int64_t)blockIdx.x + 1) * total_units / G;
    while (u < u1) {
        const Clu C = clu[cluster_of_unit(clu, nclu, u)];
        const int64_t ntiles = C.ns_pad / kMixTile;
        const int64_t ib = (u - C.unit0) / ntiles;
        const int64_t t0 = C.slot0 + ib * TI;
        const int64_t ub = C.unit0 + ib * ntiles;          // first unit of this target block
        const int64_t uend = ub + ntiles < u1 ? ub + ntiles : u1;
        const float eps2 = (float)C.eps2;
        MixTarget tg[P];
        int64_t ti[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            ti[p] = t0 + p * kMixThreads + threadIdx.x;
            const float4 A = rec[ti[p]];
            const float4 B = rec[S + ti[p]];
            const float4 Cc = rec[2 * S + ti[p]];
            tg[p].hx = A.x; tg[p].hy = A.y; tg[p].hz = A.z;
            tg[p].lx = B.x; tg[p].ly = B.y; tg[p].lz = B.z;
            tg[p].vx = kEightThirds * Cc.x;
            tg[p].vy = kEightThirds * Cc.y;
            tg[p].vz = kEightThirds * Cc.z;
#pragma unroll
            for (int k = 0; k < kFusedVals; ++k)
                run[k][p][threadIdx.x] = make_float2(0.0f, 0.0f);
        }
        float acc[P][kFusedVals];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int k = 0; k < kFusedVals; ++k)
                acc[p][k] = 0.0f;
        for (; u < uend; ++u) {
            const int64_t j0 = C.slot0 + (u - ub) * kMixTile;
            __syncthreads();
            for (int q = threadIdx.x; q < kMixTile; q += kMixThreads) {
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    sh[k][q] = rec[k * S + j0 + q];
            }
            __syncthreads();
            const bool diag = (j0 < t0 + TI) && (t0 < j0 + kMixTile);
            if (diag)
                fused_tile<P, UNROLL, true>(sh[0], sh[1], sh[2], sh[3], sh[4], j0, tg, ti, eps2, acc);
            else
                fused_tile<P, UNROLL, false>(sh[0], sh[1], sh[2], sh[3], sh[4], j0, tg, ti, eps2, acc);
            // single-precision partials span kFlushTiles tiles (aligned to the
            // target block's tiles) before they go into the running sums
            if (((u - ub + 1) % kFlushTiles) == 0 || u + 1 == uend) {
#pragma unroll
                for (int p = 0; p < P; ++p)
#pragma unroll
                    for (int k = 0; k < kFusedVals; ++k) {
                        float2 r = run[k][p][threadIdx.x];
                        ds_add(r.x, r.y, acc[p][k]);
                        run[k][p][threadIdx.x] = r;
                        acc[p][k] = 0.0f;
                    }
            }
        }
        double *out = part + (t0 / TI + blockIdx.x) * (int64_t)(kFusedVals * TI);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int k = 0; k < kFusedVals; ++k) {
                const float2 r = run[k][p][threadIdx.x];
                out[k * TI + p * kMixThreads + threadIdx.x] = (double)r.x + (double)r.y;
            }
    }
}

// ------------------------------------- fused pair kernel: packed FP32x2 --

// The fused pair terms on packed pairs of floats: lane x belongs to target
// 2q, lane y to target 2q + 1 of the same thread, both against the same
// source j.  fma.rn.f32x2 / add.rn.f32x2 / mul.rn.f32x2 (sm_100 family) do
// two FP32 operations per instruction, so the pair arithmetic needs half the
// instruction issue slots of the scalar kernel while the FP32 pipe does the
// same work.  Each source is staged in shared memory with every field
// duplicated (f, f), so that a 128-bit load yields two ready packed operands
// (stage_source_fwd):
//   F0 = (-hx, -hy)  F1 = (-hz, m)  F2 = (-lx, -ly)  F3 = (-lz, a)
//   F4 = (vx, vy)    F5 = (vz, C')  F6 = (wx, wy)    F7 = (wz, R^2)
// (h, l = hi/lo split of d_j, w = w_j, a = -G M/(6 R_j^3) and
// C' = C_j + a (R_j^2 + eps^2) for far sources, a = 0 and C' = C_j for near
// ones; R^2 is read by the target side only).
//
// Two regroupings make the body cheaper than the scalar kernels' (exact in
// real arithmetic):
// - the hole term (-e_j/1.5).d_i of kappa_ij is a (R_i^2 - r_ij^2) + (C' - C):
//   e_j/1.5 = -2 a d_j and, by the law of cosines,
//   2 d_i.d_j = R_i^2 + R_j^2 + eps^2 - r_ij^2 (softened r_ij).  Far sources
//   only (R_j >= r_near), so a stays bounded and R_i^2 - r_ij^2 = 2 d_i.d_j -
//   R_j^2 - eps^2 is a difference of O(R_i^2) numbers only when the term is
//   small anyway.
// - Wr is not summed: R_i^2 - R_j^2 = 2 d_i.x_ij - (r_ij^2 - eps^2) gives
//   Y_i = R_i^2 Z_i - Wr_i = 2 d_i.N_i - U_i + eps^2 Z_i, and k_fused_gather
//   restores Wr from N, U and Z in double.
// Sums (kPackSums): N (3), U, Z, V' (3), Hs, Hv (3), E (3).

struct PackTarget {
    float2 hx, hy, hz, lx, ly, lz;   // hi/lo split of d_i (lanes: two targets)
    float2 vx, vy, vz;               // 8/3 v_i
    float2 rr;                       // R_i^2
};

// HI: the separation from the high parts alone (x_ij = h_i - h_j), for units
// of the spatial order whose boxes are far apart (k_fused_packed).
template <bool MASK, bool LOC, bool HI>
__device__ __forceinline__ void packed_pair(const PackTarget &tg, const float4 *__restrict__ sq,
                                            float2 eps2, bool selfx, bool selfy,
                                            float2 (&acc)[kPackSums])
{
    const float4 F0 = sq[0], F1 = sq[1], F3 = sq[3];
    float2 dx = add2(tg.hx, lo2(F0)), dy = add2(tg.hy, hi2(F0)), dz = add2(tg.hz, lo2(F1));
    if (!HI) {
        const float4 F2 = sq[2];
        dx = add2(dx, add2(tg.lx, lo2(F2)));
        dy = add2(dy, add2(tg.ly, hi2(F2)));
        dz = add2(dz, add2(tg.lz, lo2(F3)));
    }
    float2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    float2 m = hi2(F1);
    float2 wx, wy, wz;
    if (LOC) {
        const float4 F6 = sq[6], F7 = sq[7];
        wx = lo2(F6), wy = hi2(F6), wz = lo2(F7);
    } else {
        const float4 S7 = sq[7], S8 = sq[8];
        wx = hi2(S7), wy = lo2(S8), wz = hi2(S8);
    }
    if (MASK) {
        if (selfx) {
            s2.x = 1.0f; m.x = 0.0f; wx.x = 0.0f; wy.x = 0.0f; wz.x = 0.0f;
        }
        if (selfy) {
            s2.y = 1.0f; m.y = 0.0f; wx.y = 0.0f; wy.y = 0.0f; wz.y = 0.0f;
        }
    }
    const float2 is = make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y));
    const float2 is2 = mul2(is, is);
    const float2 mis = mul2(m, is);
    const float2 mis3 = mul2(mis, is2);
    acc[0] = fma2(mis3, dx, acc[0]);
    acc[1] = fma2(mis3, dy, acc[1]);
    acc[2] = fma2(mis3, dz, acc[2]);
    acc[3] = add2(acc[3], mis);
    acc[4] = add2(acc[4], mis3);
    const float4 F4 = sq[4], F5 = sq[5];
    const float2 vx = lo2(F4), vy = hi2(F4), vz = lo2(F5);
    const float2 xvj = fma2(dx, vx, fma2(dy, vy, mul2(dz, vz)));
    const float2 xvi = fma2(dx, tg.vx, fma2(dy, tg.vy, mul2(dz, tg.vz)));
    float2 k;
    if (LOC) {         // C' + a (R_i^2 - r_ij^2)
        k = fma2(hi2(F3), fma2(s2, make_float2(-1.0f, -1.0f), tg.rr), hi2(F5));
    } else {           // C + D.h_i
        const float4 S6 = sq[6], S7 = sq[7];
        k = fma2(lo2(S6), tg.hx, fma2(hi2(S6), tg.hy, fma2(lo2(S7), tg.hz, hi2(F5))));
    }
    k = fma2(tg.vx, vx, fma2(tg.vy, vy, fma2(tg.vz, vz, k)));
    const float2 h = mul2(xvj, is2);
    const float2 f = mul2(mis3, fma2(h, xvj, k));
    acc[5] = fma2(f, dx, acc[5]);
    acc[6] = fma2(f, dy, acc[6]);
    acc[7] = fma2(f, dz, acc[7]);
    const float2 gg = mul2(mis3, fma2(make_float2(-2.0f, -2.0f), xvj, xvi));
    acc[8] = add2(acc[8], gg);
    acc[9] = fma2(gg, vx, acc[9]);
    acc[10] = fma2(gg, vy, acc[10]);
    acc[11] = fma2(gg, vz, acc[11]);
    acc[12] = fma2(wx, is, acc[12]);
    acc[13] = fma2(wy, is, acc[13]);
    acc[14] = fma2(wz, is, acc[14]);
}

// Local index (within the target block of 2 NP kMixThreads targets) of the
// thread's k-th target: warp w owns the 64 NP contiguous targets from
// 64 NP w, lane l takes l, l + 32, l + 64, ...; packed pair pp holds targets
// 2 pp (lane x) and 2 pp + 1 (lane y), 32 apart.
__device__ __forceinline__ int packed_target(int NP, int k)
{
    return 64 * NP * (int)(threadIdx.x / 32) + 32 * k + (int)(threadIdx.x % 32);
}

// Staged record length of the two forms.
template <bool LOC>
__host__ __device__ constexpr int pack_vals() { return LOC ? kFwdVals : kPackVals; }

template <int NP, int UNROLL, bool MASK, bool LOC, bool HI, int TILE>
__device__ __forceinline__ void packed_tile(const float4 (*__restrict__ sh)[pack_vals<LOC>()],
                                            int64_t j0, int64_t t0, const PackTarget (&tg)[NP],
                                            float2 eps2, float2 (&acc)[NP][kPackSums])
{
#pragma unroll UNROLL
    for (int q = 0; q < TILE; ++q) {
        const int64_t j = j0 + q;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
            const int64_t tx = t0 + packed_target(NP, 2 * pp);
            const bool selfx = MASK && j == tx;
            const bool selfy = MASK && j == tx + 32;
            packed_pair<MASK, LOC, HI>(tg[pp], sh[q], eps2, selfx, selfy, acc[pp]);
        }
    }
}

// One staged source tile of TILE sources (bulk-copy size)
template <bool LOC, int TILE>
__host__ __device__ constexpr unsigned tile_bytes() { return TILE * pack_vals<LOC>() * 16; }

// First source slot of stream-K unit u (its cluster's tile of TILE sources).
template <int TILE>
__device__ __forceinline__ int64_t unit_source(const Clu *__restrict__ clu, int nclu, int64_t u)
{
    const Clu C = clu[cluster_of_unit(clu, nclu, u)];
    const int64_t ntiles = C.ns_pad / TILE;
    const int64_t r = u - C.unit0;
    return C.slot0 + PN_IDX((r - (r / ntiles) * ntiles) * TILE, C.ns_pad - TILE + 1, 5);
}

// Stream-K over G workers like k_fused_mixed (worker w owns units
// [w T / G, (w+1) T / G) and writes its segments to slots (target block + w)),
// with P = 2 NP targets per thread (target pairs (0, 1), (2, 3)) and source
// tiles of TILE (64 by default; 32 on the slot order).  The resident blocks
// take workers from a counter
// (zeroed by the prologue) instead of one fixed worker each: blocks that share
// an SM advance at unequal rates under the warp scheduler's priorities, and
// with fixed assignments an SM would end its share with a fraction of its
// warps.  A worker's result does not depend on which block runs it, so the
// sums stay deterministic.
//
// Sources come from the staged records srec[slot][pack_vals<LOC>()] (every
// field duplicated, positions negated), one contiguous tile per unit (8 or
// 9 KB at 64 sources), copied by the bulk-copy engine into ST one-tile
// shared buffers (tile k of the block into buffer k % ST).  The tiles of a
// target block are consumed in rounds of up to ST / 2 between block
// barriers; after a round's barrier thread 0 refills its buffers with the
// tiles ST ahead, so loads are in flight during arithmetic and the warps,
// which may take different pair bodies, meet once per round.  Fewer stages
// leave room for more resident blocks.  Targets are read from the same
// records.  FP32 tile partials are added every kPackFlushSources sources
// into the worker's segment slot in FP64 (each value is owned by one
// thread).  A copy that does not complete within the wait limit
// sets kFlagTimeout in `flag`; the block then waits (one shared 1 s limit)
// for the copies still in flight and ends.
//
// FORM 0: the D form of the hole term on stage_source records; 1: the
// law-of-cosines form on stage_source_fwd records; 2: form 1 on records in
// the spatial order of pn_order.cu, with a box per tile (`box`).  In form 2
// each warp tests its own 64 NP contiguous targets against the tile: when
// their box and the tile's are at least theta (R_B + R_T) apart (R the
// largest |d| in either box, theta = kFarTheta = 0.05 unless tuned) the warp
// takes the separation from the high parts alone: the dropped low parts
// change x_ij by at most 2^-24 (|d_i| + |d_j|) <= 2^-24 (R_B + R_T), i.e. by
// at most 2^-24 / theta ~ 1.2e-6 of |x_ij| for the nearest such pairs and
// less for the rest -- pairs that far apart carry a small share of a star's
// force (measured on the 128k eccentric workload: the median error against
// the FP64 oracle goes from 1.1e-8 to 2.2e-8 for any theta in 0.03 .. 0.2).  Near units, and the units that hold self pairs, keep the full
// separation.  units_cnt[0] / [1] count far / all warp-units.
template <int NP, int UNROLL, int FORM, int TILE, int ST>
__global__ void __launch_bounds__(kMixThreads, NP == 2 ? 3 : 5)
k_fused_packed(const float4 *__restrict__ srec, const Clu *__restrict__ clu, int nclu,
               int64_t total_units, int64_t G, int *__restrict__ wcount, int *__restrict__ flag,
               unsigned extra_tx, const float4 *__restrict__ box, float far_theta,
               unsigned long long *__restrict__ units_cnt, const int64_t *__restrict__ wb,
               double *__restrict__ part)
{
    constexpr bool LOC = FORM >= 1, SPATIAL = FORM == 2;
    unsigned n_far = 0, n_all = 0;      // this warp's units (form 2)
    constexpr int P = 2 * NP, TI = kMixThreads * P, RV = pack_vals<LOC>();
    // rounds of RND tiles: a round's buffers are refilled while the next
    // round's are read; FP32 partials are flushed every kPackFlushSources
    // sources whatever the tile
    constexpr int RND = ST / 2, FLUSH = kPackFlushSources / TILE;
    static_assert(ST >= 2 && ST % 2 == 0 && kPackFlushSources % TILE == 0, "stage layout");
    static_assert(FORM != 2 || TILE == kPackTile, "the spatial order's boxes and unit costs are per kPackTile sources");
    __shared__ __align__(128) float4 sh[ST][TILE][RV];
    __shared__ __align__(8) uint64_t full[ST];
    __shared__ int s_w;
    if (threadIdx.x == 0) {
        for (int q = 0; q < ST; ++q)
            mbar_init(&full[q], 1);
        mbar_init_fence();
    }
    unsigned it = 0;                    // tiles this block has consumed
    for (;;) {
        __syncthreads();                // s_w free; barriers initialised
        if (threadIdx.x == 0)
            s_w = atomicAdd(wcount, 1);
        __syncthreads();
        const int64_t w = s_w;
        if (w >= G) {
            if (SPATIAL && threadIdx.x % 32 == 0) {
                atomicAdd(&units_cnt[0], (unsigned long long)n_far);
                atomicAdd(&units_cnt[1], (unsigned long long)n_all);
            }
            break;
        }
        int64_t u = wb ? wb[w] : w * total_units / G;
        const int64_t u1 = wb ? wb[w + 1] : (w + 1) * total_units / G;
        if (threadIdx.x == 0)               // every buffer is free here
            for (int q = 0; q < ST && u + q < u1; ++q)
                bulk_load(sh[(it + q) % ST], srec + unit_source<TILE>(clu, nclu, u + q) * RV,
                          tile_bytes<LOC, TILE>(), &full[(it + q) % ST], extra_tx);
        while (u < u1) {
            const Clu C = clu[cluster_of_unit(clu, nclu, u)];
            const int64_t ntiles = C.ns_pad / TILE;
            const int64_t ib = (u - C.unit0) / ntiles;
            const int64_t t0 = C.slot0 + PN_IDX(ib * TI, C.ns_pad - TI + 1, 6);
            const int64_t ub = C.unit0 + ib * ntiles;
            const int64_t uend = ub + ntiles < u1 ? ub + ntiles : u1;
            const float e2 = (float)C.eps2;
            const float2 eps2 = make_float2(e2, e2);
            PackTarget tg[NP];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                const int64_t ta = t0 + packed_target(NP, 2 * pp), tb = ta + 32;
                const float4 *ra = srec + ta * RV, *rb = srec + tb * RV;
                const float4 A0 = ra[0], A1 = ra[1], A2 = ra[2], A3 = ra[3], A4 = ra[4], A5 = ra[5];
                const float4 B0 = rb[0], B1 = rb[1], B2 = rb[2], B3 = rb[3], B4 = rb[4], B5 = rb[5];
                if (LOC)
                    tg[pp].rr = make_float2(ra[7].z, rb[7].z);
                tg[pp].hx = make_float2(-A0.x, -B0.x);
                tg[pp].hy = make_float2(-A0.z, -B0.z);
                tg[pp].hz = make_float2(-A1.x, -B1.x);
                tg[pp].lx = make_float2(-A2.x, -B2.x);
                tg[pp].ly = make_float2(-A2.z, -B2.z);
                tg[pp].lz = make_float2(-A3.x, -B3.x);
                tg[pp].vx = make_float2(kEightThirds * A4.x, kEightThirds * B4.x);
                tg[pp].vy = make_float2(kEightThirds * A4.z, kEightThirds * B4.z);
                tg[pp].vz = make_float2(kEightThirds * A5.x, kEightThirds * B5.x);
            }
            float4 blo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), bhi = blo;
            if (SPATIAL) {      // box of the warp's targets: union of their tiles' boxes
                const float4 *bb = box + 2 * ((t0 + packed_target(NP, 0) - threadIdx.x % 32) / kPackTile);
                blo = bb[0];
                bhi = bb[1];
#pragma unroll
                for (int q = 1; q < 2 * NP * 32 / kPackTile; ++q) {
                    const float4 l = bb[2 * q], h = bb[2 * q + 1];
                    blo = make_float4(fminf(blo.x, l.x), fminf(blo.y, l.y), fminf(blo.z, l.z), 0.0f);
                    bhi = make_float4(fmaxf(bhi.x, h.x), fmaxf(bhi.y, h.y), fmaxf(bhi.z, h.z),
                                      fmaxf(bhi.w, h.w));
                }
            }
            double *out = part + (t0 / TI + w) * (int64_t)(kPackSums * TI);
            bool first = true;
            float2 acc[NP][kPackSums];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
#pragma unroll
                for (int k = 0; k < kPackSums; ++k)
                    acc[pp][k] = make_float2(0.0f, 0.0f);
            // rounds of up to RND tiles of this target block between block
            // barriers; tile it goes to buffer it % ST
            while (u < uend) {
                const int nr = (int)(uend - u < RND ? uend - u : RND);
                bool ok = true;
                for (int q = 0; q < nr && ok; ++q) {
                    const int64_t uq = u + q;
                    const unsigned itq = it + q;
                    const int b = (int)(itq % ST);
                    ok = mbar_wait(&full[b], (itq / ST) & 1);
                    if (!ok)
                        break;
                    const int64_t j0 = C.slot0 + (uq - ub) * TILE;
                    const bool diag = (j0 < t0 + TI) && (t0 < j0 + TILE);
                    bool far = false;
                    if (SPATIAL && !diag) {
                        const float4 l = box[2 * (j0 / kPackTile)], h = box[2 * (j0 / kPackTile) + 1];
                        const float gx = fmaxf(0.0f, fmaxf(l.x - bhi.x, blo.x - h.x));
                        const float gy = fmaxf(0.0f, fmaxf(l.y - bhi.y, blo.y - h.y));
                        const float gz = fmaxf(0.0f, fmaxf(l.z - bhi.z, blo.z - h.z));
                        const float lim = far_theta * (bhi.w + h.w);
                        far = gx * gx + gy * gy + gz * gz >= lim * lim;
                    }
                    if (SPATIAL) {
                        n_far += far ? 1u : 0u;
                        n_all += 1u;
                    }
                    if (diag)
                        packed_tile<NP, UNROLL, true, LOC, false, TILE>(sh[b], j0, t0, tg, eps2, acc);
                    else if (SPATIAL && far)
                        packed_tile<NP, UNROLL, false, LOC, true, TILE>(sh[b], j0, t0, tg, eps2, acc);
                    else
                        packed_tile<NP, UNROLL, false, LOC, false, TILE>(sh[b], j0, t0, tg, eps2, acc);
                    if (((uq - ub + 1) % FLUSH) == 0 || uq + 1 == uend) {
#pragma unroll
                        for (int pp = 0; pp < NP; ++pp)
#pragma unroll
                            for (int k = 0; k < kPackSums; ++k) {
                                double *o = out + k * TI + packed_target(NP, 2 * pp);
                                o[0] = first ? (double)acc[pp][k].x : o[0] + (double)acc[pp][k].x;
                                o[32] = first ? (double)acc[pp][k].y : o[32] + (double)acc[pp][k].y;
                                acc[pp][k] = make_float2(0.0f, 0.0f);
                            }
                        first = false;
                    }
                }
                if (__syncthreads_or(!ok)) {     // every warp is done with this round's buffers
                    if (threadIdx.x == 0) {
                        atomicOr(flag, kFlagTimeout);
                        // let the copies still in flight land before exiting (one
                        // shared time limit)
                        const unsigned long long t_end = global_ns() + kWaitNs;
                        for (int q = 0; q < ST && u + q < u1; ++q)
                            mbar_wait_until(&full[(it + q) % ST], ((it + q) / ST) & 1, t_end);
                    }
                    return;
                }
                if (threadIdx.x == 0)            // refill the round's buffers, ST tiles ahead
                    for (int q = 0; q < nr && u + q + ST < u1; ++q)
                        bulk_load(sh[(it + q) % ST], srec + unit_source<TILE>(clu, nclu, u + q + ST) * RV,
                                  tile_bytes<LOC, TILE>(), &full[(it + q) % ST], extra_tx);
                u += nr;
                it += nr;
            }
        }
    }
}

__global__ void __launch_bounds__(kGlueThreads)
k_stage_sources(int64_t S, const float4 *__restrict__ rec, float4 *__restrict__ srec)
{
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (t < S)
        stage_source(srec + t * kPackVals, rec[t], rec[S + t], rec[2 * S + t], rec[3 * S + t],
                     rec[4 * S + t]);
}

// Sums, for every star slot, the stream-K segments that cover its target
// block (in block order) into the pass-1 / pass-2 partial layout with one
// split: p1[k][t] (k < kP1Vals), p2[k][t] (k < kP2Vals).  NV values per
// segment (fewer than kFusedVals: the packed kernel's, without Wr), RV float4
// per staged record; with `perm` the kernel ran on the spatial order and
// position t belongs to slot perm[t].  blockIdx.y splits a star's values
// over three threads: 0 the pass-1 values (and Wr), 1 and 2 five pass-2
// values each.  Blocks of kGatherThreads slots: the FP64 adds of the segment
// sums spread over every SM at small N.
template <int P, int NV, int RV>
__global__ void __launch_bounds__(kGatherThreads)
k_fused_gather(const double *__restrict__ part, int64_t S, const Clu *__restrict__ clu,
               const int *__restrict__ blk_clu, int64_t total_units, int64_t G, int tile,
               const float4 *__restrict__ srec, const int *__restrict__ perm,
               const int64_t *__restrict__ wb, double *__restrict__ p1, double *__restrict__ p2)
{
    constexpr int TI = kMixThreads * P;
    const int64_t t_ = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x;
    if (t_ >= S)
        return;
    const int64_t t = PN_IDX(t_, S, 8);
    const Clu C = clu[cluster_of_block(blk_clu, (int64_t)blockIdx.x * kGatherThreads / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / tile;
    const int64_t ib = (t - C.slot0) / TI;
    const int64_t gtb = t / TI;                                 // global target block
    const int lt = (int)(t - gtb * TI);
    const int64_t U0 = C.unit0 + ib * ntiles, U1 = U0 + ntiles;
    // worker b owns units [bound(b), bound(b + 1)): equal counts,
    // bound(q) = q * total_units / G, or the cost-balanced boundaries wb of
    // the spatial order
    int64_t b;
    if (wb) {                                   // last worker with wb[b] <= U0
        int64_t lo = 0, hi = G - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (wb[mid] <= U0)
                lo = mid;
            else
                hi = mid - 1;
        }
        b = lo;
    } else {
        b = U0 * G / total_units;
        while (b + 1 < G && (b + 1) * total_units / G <= U0)
            ++b;
    }
    constexpr int o2 = NV - kP2Vals;     // first pass-2 value in the segment
    constexpr int NG = o2 > kP2Vals / 2 ? o2 : kP2Vals / 2;   // values per thread, at most
    const int g = blockIdx.y;
    const int k0 = g == 0 ? 0 : o2 + (g - 1) * (kP2Vals / 2);
    const int nk = g == 0 ? o2 : kP2Vals / 2;
    double acc[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k)
        acc[k] = 0.0;
    // equal counts: bound(q + 1) from bound(q) by the quotient and remainder
    // of total_units / G (no 64-bit division per worker)
    int64_t bu0, r = 0, base = 0, rem = 0;
    if (wb) {
        bu0 = wb[b];
    } else {
        const int64_t num = b * total_units;
        bu0 = num / G;
        r = num - bu0 * G;
        base = total_units / G;
        rem = total_units - base * G;
    }
    // four workers' segments loaded before they are added, in worker order
    // (a worker that does not cover the block, or owns no unit, adds zeros)
    constexpr int kBatch = 4;
    for (bool more = true; more && b < G; b += kBatch) {
        double tmp[kBatch][NG];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int64_t w = b + u;
            int64_t bu1 = bu0;
            if (w < G) {
                if (wb) {
                    bu1 = wb[w + 1];
                } else {
                    bu1 = bu0 + base;
                    r += rem;
                    if (r >= G) {
                        r -= G;
                        ++bu1;
                    }
                }
            }
            const bool ok = w < G && bu0 < U1 && bu1 > U0 && bu1 > bu0;
            if (w + 1 >= G || bu1 >= U1)
                more = false;
            const double *in = part + (gtb + w) * (int64_t)(NV * TI) + (int64_t)k0 * TI + lt;
#pragma unroll
            for (int k = 0; k < NG; ++k)
                tmp[u][k] = ok && k < nk ? in[k * TI] : 0.0;
            bu0 = bu1;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
#pragma unroll
            for (int k = 0; k < NG; ++k)
                acc[k] += tmp[u][k];
    }
    const int64_t ts = perm ? (int64_t)perm[t] : t;
    if (g > 0) {
#pragma unroll
        for (int k = 0; k < NG; ++k)
            if (k < nk)
                p2[(int64_t)(k0 - o2 + k) * S + ts] = acc[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < NG; ++k)
        if (k < o2)
            p1[(int64_t)k * S + ts] = acc[k];
    if (o2 < kP1Vals) {
        // Wr from the identity R_i^2 - R_j^2 = 2 d_i.x_ij - (r_ij^2 - eps^2):
        // sum_j m_j (R_i^2 - R_j^2)/r_ij^3 = 2 d_i.N - U + eps^2 Z, so
        // Wr = (R_i^2 - eps^2) Z - 2 d_i.N + U (d_i from the staged hi/lo split)
        const float4 *r = srec + t * RV;
        const double d0 = -((double)r[0].x + (double)r[2].x);
        const double d1 = -((double)r[0].z + (double)r[2].z);
        const double d2 = -((double)r[1].x + (double)r[3].x);
        const double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        p1[(int64_t)5 * S + ts] =
            (R2 - C.eps2) * acc[4] - 2.0 * (d0 * acc[0] + d1 * acc[1] + d2 * acc[2]) + acc[3];
    }
}

// ------------------------------------------------ pair kernels: double --

// The same pair sums as pass 1 / pass 2 above, in double precision
// (records A = (d, m), B = (v, R^2), C = (-e/1.5, C), D = (w, 0); vi is
// 8/3 times the target's velocity).  PASS 3: both passes' sums from one
// separation, distance and rsqrt per pair (pass-1 values first).
template <int PASS, bool MASK, int NACC>
__device__ __forceinline__ void f64_tile(const double4_32a (*__restrict__ sh)[kF64Tile], int64_t j0,
                                         const double (&di)[3], const double (&vi)[3],
                                         int64_t ti, double eps2, double (&acc)[NACC])
{
    constexpr int o2 = PASS == 3 ? kP1Vals : 0;     // first pass-2 value in acc
#pragma unroll 1
    for (int q = 0; q < kF64Tile; ++q) {
        const double4_32a A = sh[0][q];
        const double dx = di[0] - A.x, dy = di[1] - A.y, dz = di[2] - A.z;
        double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
        double mj = A.w;
        const bool self = MASK && (j0 + q == ti);
        if (MASK) {
            s2 = self ? 1.0 : s2;
            mj = self ? 0.0 : mj;
        }
        const double is = rsqrt_f64(s2);
        const double is2 = is * is;
        const double mis = mj * is;
        const double mis3 = mis * is2;
        if constexpr (PASS != 2) {
            acc[0] = fma(mis3, dx, acc[0]);
            acc[1] = fma(mis3, dy, acc[1]);
            acc[2] = fma(mis3, dz, acc[2]);
            acc[3] += mis;
            acc[4] += mis3;
            acc[5] = fma(mis3, sh[1][q].w, acc[5]);
        }
        if constexpr (PASS != 1) {
            const double4_32a B = sh[1][q];
            const double4_32a C = sh[2][q];
            const double4_32a D = sh[3][q];
            const double wx = self ? 0.0 : D.x, wy = self ? 0.0 : D.y, wz = self ? 0.0 : D.z;
            const double xvj = fma(dx, B.x, fma(dy, B.y, dz * B.z));
            const double xvi = fma(dx, vi[0], fma(dy, vi[1], dz * vi[2]));
            double k = fma(vi[0], B.x, fma(vi[1], B.y, fma(vi[2], B.z, C.w)));
            k = fma(C.x, di[0], fma(C.y, di[1], fma(C.z, di[2], k)));
            const double h = xvj * is2;
            const double f = mis3 * fma(h, xvj, k);
            acc[o2 + 0] = fma(f, dx, acc[o2 + 0]);
            acc[o2 + 1] = fma(f, dy, acc[o2 + 1]);
            acc[o2 + 2] = fma(f, dz, acc[o2 + 2]);
            const double gg = mis3 * fma(-2.0, xvj, xvi);
            acc[o2 + 3] += gg;
            acc[o2 + 4] = fma(gg, B.x, acc[o2 + 4]);
            acc[o2 + 5] = fma(gg, B.y, acc[o2 + 5]);
            acc[o2 + 6] = fma(gg, B.z, acc[o2 + 6]);
            acc[o2 + 7] = fma(wx, is, acc[o2 + 7]);
            acc[o2 + 8] = fma(wy, is, acc[o2 + 8]);
            acc[o2 + 9] = fma(wz, is, acc[o2 + 9]);
        }
    }
}

// Grid (target blocks of kF64Threads, source splits); split s sweeps tiles
// [s tps, (s+1) tps) of the target block's cluster and writes its partials
// to part[s][value][slot] (PASS 3: pass-1 values to part, pass-2 values to
// part2, each in its pass's layout).
template <int PASS>
__global__ void __launch_bounds__(kF64Threads)
k_pass_f64(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
           const int *__restrict__ blk_clu, double *__restrict__ part, double *__restrict__ part2)
{
    constexpr int NV = PASS == 1 ? kP1Vals : (PASS == 2 ? kP2Vals : kFusedVals);
    constexpr int NA = PASS == 1 ? 2 : 4;
    __shared__ double4_32a sh[4][kF64Tile];
    const int64_t t0 = (int64_t)blockIdx.x * kF64Threads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const double eps2 = C.eps2;
    const int ntiles = (int)(C.ns_pad / kF64Tile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int64_t ti = t0 + threadIdx.x;
    const double4_32a A = rec[ti];
    const double di[3] = {A.x, A.y, A.z};
    double vi[3] = {0.0, 0.0, 0.0};
    if (PASS != 1) {
        const double4_32a B = rec[S + ti];
        vi[0] = (8.0 / 3.0) * B.x;
        vi[1] = (8.0 / 3.0) * B.y;
        vi[2] = (8.0 / 3.0) * B.z;
    }
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        acc[k] = 0.0;
    const int tb = blockIdx.y * tps;
    const int te = min(ntiles, tb + tps);
    for (int tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + (int64_t)tile * kF64Tile;
        __syncthreads();
        for (int q = threadIdx.x; q < kF64Tile; q += kF64Threads) {
#pragma unroll
            for (int k = 0; k < NA; ++k)
                sh[k][q] = rec[k * S + j0 + q];
        }
        __syncthreads();
        const bool diag = (j0 < t0 + kF64Threads) && (t0 < j0 + kF64Tile);
        if (diag)
            f64_tile<PASS, true, NV>(sh, j0, di, vi, ti, eps2, acc);
        else
            f64_tile<PASS, false, NV>(sh, j0, di, vi, ti, eps2, acc);
    }
    if (PASS == 3) {
#pragma unroll
        for (int k = 0; k < kP1Vals; ++k)
            part[((int64_t)blockIdx.y * kP1Vals + k) * S + ti] = acc[k];
#pragma unroll
        for (int k = 0; k < kP2Vals; ++k)
            part2[((int64_t)blockIdx.y * kP2Vals + k) * S + ti] = acc[kP1Vals + k];
    } else {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            part[((int64_t)blockIdx.y * NV + k) * S + ti] = acc[k];
    }
}

// 1/sqrt(s2) in double for the energy sums: the single-precision seed
// (rsqrtf, relative error <= 2^-22) refined by one Newton step, whose result
// is low by at most 1.5 (2^-22)^2 ~ 9e-14 relative -- far below the 1e-10
// that energy differences need (each pair term enters Eq. 7-8 once).
__device__ __forceinline__ double rsqrt_f64_energy(double s2)
{
    const double y = (double)rsqrtf((float)s2);
    return y * fma(-0.5 * s2, y * y, 1.5);
}

// Energy pair sums, double precision, records A = (d, m), B = (v, 0):
//   pot += m_j/r, Smv += m_j/r v_j, Snn += m_j/r (n.v_i)(n.v_j),
//   Spx += m_j/r (n.v_i)/r x_ij,   n = x_ij / r,
// the last two through the unnormalised projections u_i = x.v_i, u_j = x.v_j:
// m_j/r (n.v_i)(n.v_j) = (m_j/r^3 u_i) u_j, m_j/r (n.v_i)/r = m_j/r^3 u_i.
template <bool MASK>
__device__ __forceinline__ void energy_tile(const double4_32a (*__restrict__ sh)[kF64Tile],
                                            int64_t j0, const double (&di)[3],
                                            const double (&vi)[3], int64_t ti, double eps2,
                                            double (&acc)[kEVals])
{
#pragma unroll 1
    for (int q = 0; q < kF64Tile; ++q) {
        const double4_32a A = sh[0][q];
        const double4_32a B = sh[1][q];
        const double dx = di[0] - A.x, dy = di[1] - A.y, dz = di[2] - A.z;
        double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
        double mj = A.w;
        if (MASK) {
            const bool self = (j0 + q == ti);
            s2 = self ? 1.0 : s2;
            mj = self ? 0.0 : mj;
        }
        const double is = rsqrt_f64_energy(s2);
        const double ms = mj * is;
        const double ui = fma(dx, vi[0], fma(dy, vi[1], dz * vi[2]));
        const double uj = fma(dx, B.x, fma(dy, B.y, dz * B.z));
        acc[0] += ms;
        acc[1] = fma(ms, B.x, acc[1]);
        acc[2] = fma(ms, B.y, acc[2]);
        acc[3] = fma(ms, B.z, acc[3]);
        const double px = ms * (is * is) * ui;
        acc[4] = fma(px, uj, acc[4]);
        acc[5] = fma(px, dx, acc[5]);
        acc[6] = fma(px, dy, acc[6]);
        acc[7] = fma(px, dz, acc[7]);
    }
}

// Grid (blocks of 128 target slots, source splits): split s of a block in
// cluster k sweeps the cluster's tiles [s T / js, (s+1) T / js) (T tiles)
// into part[s][value][slot]; the splits fill every SM at small N.
__global__ void __launch_bounds__(kF64Threads)
k_energy_pairs(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
               const int *__restrict__ blk_clu, double *__restrict__ part)
{
    __shared__ double4_32a sh[2][kF64Tile];
    const int64_t t0 = (int64_t)blockIdx.x * kF64Threads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const double eps2 = C.eps2;
    const int64_t ntiles = C.ns_pad / kF64Tile, js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    const int64_t ti = t0 + threadIdx.x;
    const double4_32a A = rec[ti];
    const double4_32a B = rec[S + ti];
    const double di[3] = {A.x, A.y, A.z};
    const double vi[3] = {B.x, B.y, B.z};
    double acc[kEVals];
#pragma unroll
    for (int k = 0; k < kEVals; ++k)
        acc[k] = 0.0;
    for (int64_t tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + tile * kF64Tile;
        __syncthreads();
        for (int q = threadIdx.x; q < kF64Tile; q += kF64Threads) {
            const int64_t jq = PN_IDX(j0 + q, S, 14);
            sh[0][q] = rec[jq];
            sh[1][q] = rec[S + jq];
        }
        __syncthreads();
        const bool diag = (j0 < t0 + kF64Threads) && (t0 < j0 + kF64Tile);
        if (diag)
            energy_tile<true>(sh, j0, di, vi, ti, eps2, acc);
        else
            energy_tile<false>(sh, j0, di, vi, ti, eps2, acc);
    }
#pragma unroll
    for (int k = 0; k < kEVals; ++k)
        part[(sp * kEVals + k) * S + ti] = acc[k];
}

// ---- energy pair sums in double-single arithmetic (mixed contexts) ----
//
// A double-single number is the unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi) / 2, about 48 significant bits), computed on the FP32
// pipe with error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum
// (|a| >= |b|) and the FMA product error a b - fl(a b).  B300 runs FP64 at
// 1/64 of the FP32 rate, so the energy's pair sums in this form (about 355
// FP32 operations per pair) cost a fraction of k_energy_pairs' ~30 FP64
// instructions; each sum stays within ~1e-13 relative, far below the 1e-10
// that energy differences need.
struct DS {
    float hi, lo;
};

__device__ __forceinline__ DS ds_fast2sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ DS ds_add(DS x, DS y)
{
    const float s = x.hi + y.hi, bb = s - x.hi;
    const float e = ((x.hi - (s - bb)) + (y.hi - bb)) + (x.lo + y.lo);
    return ds_fast2sum(s, e);
}

__device__ __forceinline__ DS ds_sub(DS x, DS y) { return ds_add(x, DS{-y.hi, -y.lo}); }

__device__ __forceinline__ DS ds_mul(DS x, DS y)
{
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
    return ds_fast2sum(p, e);
}

__device__ __forceinline__ DS ds_of(double a)
{
    const float h = (float)a;
    return {h, (float)(a - (double)h)};
}

// Double-single records per slot from the energy prologue's FP64 records
// (A = (d, m), B = (v, 0)): four float4, (d_x, d_y), (d_z, m), (v_x, v_y),
// (v_z, 0) as (hi, lo) pairs.
__global__ void __launch_bounds__(kGlueThreads)
k_energy_stage_ds(int64_t S, const double4_32a *__restrict__ rec, float4 *__restrict__ drs)
{
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (t >= S)
        return;
    const double4_32a A = rec[t], B = rec[S + t];
    const DS dx = ds_of(A.x), dy = ds_of(A.y), dz = ds_of(A.z), m = ds_of(A.w);
    const DS vx = ds_of(B.x), vy = ds_of(B.y), vz = ds_of(B.z);
    float4 *o = drs + 4 * t;
    o[0] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
    o[1] = make_float4(dz.hi, dz.lo, m.hi, m.lo);
    o[2] = make_float4(vx.hi, vx.lo, vy.hi, vy.lo);
    o[3] = make_float4(vz.hi, vz.lo, 0.0f, 0.0f);
}

// The sums of energy_tile (same definitions and output layout, splits as in
// k_energy_pairs) in double-single arithmetic.  1/r: the single-precision
// seed y0 refined by one Newton step whose residual 1 - s^2 y0^2 is formed
// in double-single (relative error about 1.5 (2^-22)^2 ~ 9e-14).
__global__ void __launch_bounds__(kF64Threads)
k_energy_pairs_ds(const float4 *__restrict__ drs, int64_t S, const Clu *__restrict__ clu,
                  const int *__restrict__ blk_clu, double *__restrict__ part)
{
    __shared__ float4 sh[kF64Tile][4];
    const int64_t t0 = (int64_t)blockIdx.x * kF64Threads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const DS eps2 = ds_of(C.eps2);
    const int64_t ntiles = C.ns_pad / kF64Tile, js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    const int64_t ti = t0 + threadIdx.x;
    const float4 T0 = drs[4 * ti], T2 = drs[4 * ti + 2], T3 = drs[4 * ti + 3];
    const float4 T1 = drs[4 * ti + 1];
    const DS di[3] = {{T0.x, T0.y}, {T0.z, T0.w}, {T1.x, T1.y}};
    const DS vi[3] = {{T2.x, T2.y}, {T2.z, T2.w}, {T3.x, T3.y}};
    DS acc[kEVals];
#pragma unroll
    for (int k = 0; k < kEVals; ++k)
        acc[k] = DS{0.0f, 0.0f};
    for (int64_t tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + tile * kF64Tile;
        __syncthreads();
        for (int q = threadIdx.x; q < 4 * kF64Tile; q += kF64Threads) {
            const int64_t jq = PN_IDX(j0 + q / 4, S, 14);
            sh[q / 4][q % 4] = drs[4 * jq + q % 4];
        }
        __syncthreads();
        const bool diag = (j0 < t0 + kF64Threads) && (t0 < j0 + kF64Tile);
#pragma unroll 1
        for (int q = 0; q < kF64Tile; ++q) {
            const float4 R0 = sh[q][0], R1 = sh[q][1], R2 = sh[q][2], R3 = sh[q][3];
            const DS dx = ds_sub(di[0], DS{R0.x, R0.y}), dy = ds_sub(di[1], DS{R0.z, R0.w}),
                     dz = ds_sub(di[2], DS{R1.x, R1.y});
            DS s2 = ds_add(ds_add(ds_mul(dx, dx), ds_mul(dy, dy)), ds_add(ds_mul(dz, dz), eps2));
            DS mj{R1.z, R1.w};
            if (diag && j0 + q == ti) {
                s2 = DS{1.0f, 0.0f};
                mj = DS{0.0f, 0.0f};
            }
            const float y0 = rsqrtf(s2.hi);
            const float p0 = y0 * y0;
            const DS u = ds_mul(s2, DS{p0, fmaf(y0, y0, -p0)});
            const float h = (1.0f - u.hi) - u.lo;            // 1 - s^2 y0^2
            const DS y = ds_fast2sum(y0, 0.5f * y0 * h);
            const DS ms = ds_mul(mj, y);
            const DS vj[3] = {{R2.x, R2.y}, {R2.z, R2.w}, {R3.x, R3.y}};
            const DS ui = ds_add(ds_add(ds_mul(dx, vi[0]), ds_mul(dy, vi[1])), ds_mul(dz, vi[2]));
            const DS uj = ds_add(ds_add(ds_mul(dx, vj[0]), ds_mul(dy, vj[1])), ds_mul(dz, vj[2]));
            acc[0] = ds_add(acc[0], ms);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[1 + k] = ds_add(acc[1 + k], ds_mul(ms, vj[k]));
            const DS px = ds_mul(ds_mul(ms, ds_mul(y, y)), ui);   // m/r^3 u_i
            acc[4] = ds_add(acc[4], ds_mul(px, uj));
            acc[5] = ds_add(acc[5], ds_mul(px, dx));
            acc[6] = ds_add(acc[6], ds_mul(px, dy));
            acc[7] = ds_add(acc[7], ds_mul(px, dz));
        }
    }
#pragma unroll
    for (int k = 0; k < kEVals; ++k)
        part[(sp * kEVals + k) * S + ti] = (double)acc[k].hi + (double)acc[k].lo;
}

// ------------------------------------------------------- near sources --

// Eq. 6 lines 2-4 for a near source j (R_j < r_near), pair by pair in a
// form free of cancellation.  With q = R_i^2 - r_ij^2 = 2 d_i.d_j - R_j^2 - eps^2,
// A_j = 5/(4 R_j), B_j = 1/(4 R_j^3), s = r_ij:
//   line 2 + line 3 without their 4/r_ij and 4/R_i parts (those stay in
//   pass 1's U_i and N_i) = G^2 M m_j [A_j (d_i/R_i^3 + x_ij/s^3)
//                                      + B_j q (d_i (1/R_i^3 - 1/s^3) + d_j/s^3)]
//   line 4 = -7/2 G^2 M w_j (1/s - 1/R_i),
// with 1/s - 1/R_i = q / (s R_i (R_i + s)) and
// 1/R_i^3 - 1/s^3 = -(1/s - 1/R_i)(1/R_i^2 + 1/(R_i s) + 1/s^2).
// Accumulators: P (3) = sum m_j [...], Ee (3) = sum w_j (1/s - 1/R_i).
// The quotient by R_i + s: correctly rounded in double, by the approximate
// reciprocal (__fdividef, 2 ulp) in single precision, whose sums carry FP32
// rounding anyway.
__device__ __forceinline__ double near_div(double a, double b) { return a / b; }
__device__ __forceinline__ float near_div(float a, float b) { return __fdividef(a, b); }

template <typename R_t>
struct NearMath {
    __device__ __forceinline__ static void pair(R_t dx, R_t dy, R_t dz, R_t s2, R_t is,
                                                const R_t (&di)[3], const R_t (&dj)[3],
                                                R_t Ri, R_t iR, R_t iR3, R_t mj, R_t A, R_t B,
                                                R_t Rj2e, R_t wx, R_t wy, R_t wz,
                                                R_t (&acc)[kNearVals])
    {
        const R_t is2 = is * is;
        const R_t is3 = is2 * is;
        const R_t sd = s2 * is;                                  // s
        const R_t q = (R_t)2 * (dj[0] * di[0] + dj[1] * di[1] + dj[2] * di[2]) - Rj2e;
        const R_t dis = near_div(q * is * iR, Ri + sd);          // 1/s - 1/R_i
        const R_t d3 = -dis * (iR * iR + iR * is + is2);         // 1/R_i^3 - 1/s^3
        const R_t ca = mj * A;
        const R_t cb = mj * B * q;
        acc[0] += ca * (di[0] * iR3 + dx * is3) + cb * (di[0] * d3 + dj[0] * is3);
        acc[1] += ca * (di[1] * iR3 + dy * is3) + cb * (di[1] * d3 + dj[1] * is3);
        acc[2] += ca * (di[2] * iR3 + dz * is3) + cb * (di[2] * d3 + dj[2] * is3);
        acc[3] += wx * dis;
        acc[4] += wy * dis;
        acc[5] += wz * dis;
    }
};

__global__ void __launch_bounds__(kMixThreads)
k_near_mixed(const float4 *__restrict__ rec, const float4 *__restrict__ nrec,
             const int *__restrict__ ncount, int64_t S, int64_t NC, const Clu *__restrict__ clu,
             const int *__restrict__ blk_clu, double *__restrict__ part)
{
    constexpr int TI = kMixThreads * kMixTargets;
    __shared__ float4 sh[4][kNearTile];
    const int64_t t0 = (int64_t)blockIdx.x * TI;
    const int k_clu = cluster_of_block(blk_clu, t0 / kGlueThreads);
    const Clu C = clu[k_clu];
    const float eps2 = (float)C.eps2;
    const int nn = ncount[k_clu];
    const int ntiles = (nn + kNearTile - 1) / kNearTile;
    float hx[kMixTargets][3], lx[kMixTargets][3], Ri[kMixTargets], iR[kMixTargets],
        iR3[kMixTargets];
    int ti[kMixTargets];
    float hi[kMixTargets][kNearVals], lo[kMixTargets][kNearVals];
#pragma unroll
    for (int p = 0; p < kMixTargets; ++p) {
        ti[p] = (int)(t0 + p * kMixThreads + threadIdx.x);
        const float4 A = rec[ti[p]];
        const float4 B = rec[S + ti[p]];
        hx[p][0] = A.x; hx[p][1] = A.y; hx[p][2] = A.z;
        lx[p][0] = B.x; lx[p][1] = B.y; lx[p][2] = B.z;
        Ri[p] = sqrtf(A.x * A.x + A.y * A.y + A.z * A.z);
        iR[p] = 1.0f / Ri[p];
        iR3[p] = iR[p] * iR[p] * iR[p];
#pragma unroll
        for (int k = 0; k < kNearVals; ++k)
            hi[p][k] = lo[p][k] = 0.0f;
    }
    for (int tile = 0; tile < ntiles; ++tile) {
        const int64_t j0 = C.near0 + (int64_t)tile * kNearTile;
        __syncthreads();
        for (int q = threadIdx.x; q < kNearTile; q += kMixThreads) {
            const int64_t jq = PN_IDX(j0 + q, NC, 10);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                sh[k][q] = nrec[k * NC + jq];
        }
        __syncthreads();
        float acc[kMixTargets][kNearVals];
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
            for (int k = 0; k < kNearVals; ++k)
                acc[p][k] = 0.0f;
        const int qn = nn - tile * kNearTile < kNearTile ? nn - tile * kNearTile : kNearTile;
#pragma unroll 1
        for (int q = 0; q < qn; ++q) {      // the tile's near sources (padding skipped)
            const float4 A = sh[0][q], B = sh[1][q], Cn = sh[2][q], D = sh[3][q];
            const float dj[3] = {A.x, A.y, A.z};
#pragma unroll
            for (int p = 0; p < kMixTargets; ++p) {
                const float dx = (hx[p][0] - A.x) + (lx[p][0] - B.x);
                const float dy = (hx[p][1] - A.y) + (lx[p][1] - B.y);
                const float dz = (hx[p][2] - A.z) + (lx[p][2] - B.z);
                float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                const bool self = __float_as_int(D.y) == ti[p];
                s2 = self ? 1.0f : s2;
                const float mj = self ? 0.0f : A.w;
                const float wx = self ? 0.0f : Cn.x, wy = self ? 0.0f : Cn.y, wz = self ? 0.0f : Cn.z;
                const float is = rsqrtf(s2);
                NearMath<float>::pair(dx, dy, dz, s2, is, hx[p], dj, Ri[p], iR[p], iR3[p], mj,
                                      B.w, Cn.w, D.x, wx, wy, wz, acc[p]);
            }
        }
#pragma unroll
        for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
            for (int k = 0; k < kNearVals; ++k)
                ds_add(hi[p][k], lo[p][k], acc[p][k]);
    }
#pragma unroll
    for (int p = 0; p < kMixTargets; ++p)
#pragma unroll
        for (int k = 0; k < kNearVals; ++k)
            part[(int64_t)k * S + ti[p]] = (double)hi[p][k] + (double)lo[p][k];
}

__global__ void __launch_bounds__(kF64Threads)
k_near_f64(const double4_32a *__restrict__ rec, const double4_32a *__restrict__ nrec,
           const int *__restrict__ ncount, int64_t S, int64_t NC, const Clu *__restrict__ clu,
           const int *__restrict__ blk_clu, double *__restrict__ part)
{
    constexpr int TILE = kNearTile / 2;
    __shared__ double4_32a sh[3][TILE];
    const int64_t t0 = (int64_t)blockIdx.x * kF64Threads;
    const int k_clu = cluster_of_block(blk_clu, t0 / kGlueThreads);
    const Clu C = clu[k_clu];
    const double eps2 = C.eps2;
    const int ti = (int)(t0 + threadIdx.x);
    const int nn = ncount[k_clu];
    const int ntiles = (nn + TILE - 1) / TILE;
    const double4_32a Ta = rec[ti];
    const double di[3] = {Ta.x, Ta.y, Ta.z};
    const double Ri = sqrt(di[0] * di[0] + di[1] * di[1] + di[2] * di[2]);
    const double iR = 1.0 / Ri;
    const double iR3 = iR * iR * iR;
    double acc[kNearVals];
#pragma unroll
    for (int k = 0; k < kNearVals; ++k)
        acc[k] = 0.0;
    for (int tile = 0; tile < ntiles; ++tile) {
        const int64_t j0 = C.near0 + (int64_t)tile * TILE;
        __syncthreads();
        for (int q = threadIdx.x; q < TILE; q += kF64Threads) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                sh[k][q] = nrec[k * NC + j0 + q];
        }
        __syncthreads();
        const int qn = nn - tile * TILE < TILE ? nn - tile * TILE : TILE;
#pragma unroll 1
        for (int q = 0; q < qn; ++q) {      // the tile's near sources (padding skipped)
            const double4_32a A = sh[0][q], B = sh[1][q], Cn = sh[2][q];
            const double dj[3] = {A.x, A.y, A.z};
            const double dx = di[0] - A.x, dy = di[1] - A.y, dz = di[2] - A.z;
            double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
            const bool self = (int)B.w == ti;
            s2 = self ? 1.0 : s2;
            const double mj = self ? 0.0 : A.w;
            const double wx = self ? 0.0 : Cn.x, wy = self ? 0.0 : Cn.y, wz = self ? 0.0 : Cn.z;
            const double is = rsqrt_f64(s2);
            NearMath<double>::pair(dx, dy, dz, s2, is, di, dj, Ri, iR, iR3, mj, B.x, B.y, B.z,
                                   wx, wy, wz, acc);
        }
    }
#pragma unroll
    for (int k = 0; k < kNearVals; ++k)
        part[(int64_t)k * S + ti] = acc[k];
}

// ------------------------------------------------------------ epilogue --

// Writes the acceleration of one body, its final kick v += h a (when v), and
// with dt_next > 0 the next KDK step's kick and drift (k_kick_drift's
// operations).
__device__ __forceinline__ void kick_and_next(double *a, double *v, double *x, double *vel,
                                              const double (&ai)[3], double h, double dt_next,
                                              int vel_mode)
{
    const double hn = 0.5 * dt_next;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = ai[k];
        if (!v)
            continue;
        const double v1 = fma(h, ai[k], v[k]);
        if (dt_next > 0.0) {
            const double vh = fma(hn, ai[k], v1);
            v[k] = vh;
            x[k] = fma(dt_next, vh, x[k]);
            vel[k] = vel_mode == 0 ? fma(hn, ai[k], vh) : vh;
        } else {
            v[k] = v1;
        }
    }
}

// Star i = t + 1 (double precision throughout): sums the partials of every
// pass for its slot and assembles its acceleration and its term of the
// hole's acceleration with star_eqs (the formulas are stated there); the
// block's sum of the hole terms goes to blk (deterministic tree), one entry
// per kEpiThreads slots.
//
// The hole: every block adds its rows to blk, then takes a ticket from the
// cluster's counter `done` (atomicInc wraps it back to 0 for the next
// evaluation); the cluster's last block to finish sums the rows in block
// order (a fixed order whichever block it is, so the result is
// deterministic) into a_hole = G W + (1/c^2) sum_j (star j's term), and
// kicks the hole like the stars.  Every block has read the hole's position
// before taking its ticket, so the last block may move the hole.
//
// dt_next > 0 (KDK steps inside one call): after the final kick each star
// and, in the last block, the hole take the next step's kick and drift --
// v_h = v + h' a, x += dt_next v_h, vel = v_h + h' a (vel_mode 0) or v_h,
// h' = dt_next / 2 -- the same operations k_kick_drift would do next, so
// the trajectory is bitwise the same.  A thread reads and writes only its
// own star's x, vel and v, and the hole's x before its block's ticket.
__global__ void __launch_bounds__(kEpiThreads)
k_epilogue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
           double *x, double *vel, const double *__restrict__ m, const double *__restrict__ p1,
           int js1, const double *__restrict__ p2, int js2, const double *__restrict__ pnear,
           const unsigned char *__restrict__ nflag, const double *__restrict__ globs,
           double *a, double *v, double h, int *flag, unsigned long long *flag_step,
           unsigned long long step, double *__restrict__ blk, unsigned *__restrict__ done,
           double dt_next, int vel_mode)
{
    __shared__ double sh[3][kEpiThreads];
    const int64_t t = PN_IDX((int64_t)blockIdx.x * kEpiThreads + threadIdx.x, S, 11);
    const int k_clu = cluster_of_block(blk_clu, (int64_t)blockIdx.x * kEpiThreads / kGlueThreads);
    const Clu Cl = clu[k_clu];
    const double *glob = globs + (int64_t)k_clu * kGlobVals;
    const int64_t lt = t - Cl.slot0;
    double bh[3] = {0.0, 0.0, 0.0};
    if (lt < Cl.ns) {
        const int64_t i = Cl.body0 + 1 + lt, hb = Cl.body0;
        const double d[3] = {x[3 * i] - x[3 * hb], x[3 * i + 1] - x[3 * hb + 1],
                             x[3 * i + 2] - x[3 * hb + 2]};
        const double vv[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
        double s1[kP1Vals], s2[kP2Vals];
        if (js1 == 1 && js2 == 1) {
            // one partial set per pass (the fused kernels): every load issued
            // before the first use
#pragma unroll
            for (int k = 0; k < kP1Vals; ++k)
                s1[k] = p1[(int64_t)k * S + t];
#pragma unroll
            for (int k = 0; k < kP2Vals; ++k)
                s2[k] = p2[(int64_t)k * S + t];
        } else {
            for (int k = 0; k < kP1Vals; ++k) {
                double acc = 0.0;
                for (int s = 0; s < js1; ++s)
                    acc += p1[((int64_t)s * kP1Vals + k) * S + t];
                s1[k] = acc;
            }
            for (int k = 0; k < kP2Vals; ++k) {
                double acc = 0.0;
                for (int s = 0; s < js2; ++s)
                    acc += p2[((int64_t)s * kP2Vals + k) * S + t];
                s2[k] = acc;
            }
        }
        StarSums<double> ss;
        for (int k = 0; k < 3; ++k) {
            ss.N[k] = s1[k];
            ss.Vp[k] = s2[k];
            ss.Hv[k] = s2[4 + k];
            ss.E[k] = s2[7 + k];
            ss.P[k] = pnear ? pnear[(int64_t)k * S + t] : 0.0;
            ss.Ee[k] = pnear ? pnear[(int64_t)(3 + k) * S + t] : 0.0;
        }
        ss.U = s1[3];
        ss.Z = s1[4];
        ss.Wr = s1[5];
        ss.Hs = s2[3];
        ClusterSums<double> gs;
        for (int k = 0; k < 3; ++k) {
            gs.Q[k] = glob[k];
            gs.Wf[k] = glob[6 + k];
        }
        gs.SA = glob[9];
        gs.SB = glob[10];
        gs.Phi = glob[11];
        const double fi = nflag[t] ? 0.0 : 1.0;   // 1 if star i is a far source
        double ai[3];
        star_eqs<double, double>(Cl.G, m[hb], m[i], Cl.eps2, Cl.inv_c2, fi, d, vv, ss, gs, ai, bh);
        flag_nonfinite(ai, flag, flag_step, step);
        kick_and_next(&a[3 * i], v ? &v[3 * i] : nullptr, &x[3 * i], &vel[3 * i], ai, h, dt_next,
                      vel_mode);
    }
    block_sum<3, kEpiThreads>(bh, sh);
    if (threadIdx.x < 3)
        blk[(int64_t)blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nb = (unsigned)(Cl.ns_pad / kEpiThreads);
        s_last = atomicInc(&done[k_clu], nb - 1) == nb - 1;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    // rows of the cluster, thread q adding rows q, q + kEpiThreads, ... in
    // order; then the per-thread sums in a fixed tree
    const int64_t r0 = Cl.slot0 / kEpiThreads, nr = Cl.ns_pad / kEpiThreads;
    double s3[3] = {0.0, 0.0, 0.0};
    for (int64_t r = threadIdx.x; r < nr; r += kEpiThreads)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            s3[k] += __ldcg(&blk[(r0 + r) * 3 + k]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        sh[k][threadIdx.x] = s3[k];
    __syncthreads();
    if (threadIdx.x < 32) {
        static_assert(kEpiThreads == 64, "two warps per epilogue block");
        double tot[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double w = sh[k][threadIdx.x] + sh[k][threadIdx.x + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_xor_sync(0xffffffffu, w, o);
            tot[k] = w;
        }
        if (threadIdx.x == 0) {
            const int64_t hb = Cl.body0;
            double a0[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                a0[k] = Cl.G * glob[3 + k] + Cl.inv_c2 * tot[k];
            flag_nonfinite(a0, flag, flag_step, step);
            kick_and_next(&a[3 * hb], v ? &v[3 * hb] : nullptr, &x[3 * hb], &vel[3 * hb], a0, h,
                          dt_next, vel_mode);
        }
    }
}

// ------------------------------------------------------------- energy --

// Per star i (Eq. 7 and Eq. 8, double):
//   eN  = 1/2 m_i v_i^2 - 1/2 G m_i pot_i - G M m_i / R_i
//   ePN = 3/8 m_i v_i^4 + 3/2 G M m_i v_i^2 / R_i + 1/2 G^2 M^2 m_i / R_i^2
//       + 1/4 G m_i pn_i + 1/2 G M m_i/R_i [3 v_1^2 - 7 v_1.v_i - (n.v_1)(n.v_i)]
//       + G^2 M m_i pot_i / R_i
//   pN  = m_i v_i
//   pPN = 1/2 m_i v_i^2 v_i - 1/2 G M m_i/R_i [v_i + (v_i.n)n + v_1 + (v_1.n)n]
//       - 1/2 G m_i p_i
// with pn_i = 6 v_i^2 pot_i - 7 v_i.Smv_i - Snn_i, p_i = v_i pot_i + Spx_i,
// n = d_i/R_i (its sign cancels), plus sum m_i/R_i for the i = j double sum.
__global__ void __launch_bounds__(kGlueThreads)
k_energy_epilogue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                  const double *__restrict__ x, const double *__restrict__ vel,
                  const double *__restrict__ m, const double *__restrict__ pe, int js,
                  double *__restrict__ blk)
{
    __shared__ double sh[kEBlockVals][kGlueThreads];
    const int64_t t = PN_IDX((int64_t)blockIdx.x * kGlueThreads + threadIdx.x, S, 15);
    const Clu Cl = clu[cluster_of_block(blk_clu, blockIdx.x)];
    const double G = Cl.G;
    const int64_t lt = t - Cl.slot0;
    double o[kEBlockVals];
    for (int k = 0; k < kEBlockVals; ++k)
        o[k] = 0.0;
    if (lt < Cl.ns) {
        const int64_t i = Cl.body0 + 1 + lt, hb = Cl.body0;
        const double M = m[hb], mi = m[i];
        const double d[3] = {x[3 * i] - x[3 * hb], x[3 * i + 1] - x[3 * hb + 1],
                             x[3 * i + 2] - x[3 * hb + 2]};
        const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double iR = 1.0 / R;
        const double vi[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
        const double v1[3] = {vel[3 * hb], vel[3 * hb + 1], vel[3 * hb + 2]};
        double s[kEVals];          // the pair sums, splits added in order
        for (int k = 0; k < kEVals; ++k)
            s[k] = pe[(int64_t)k * S + t];
        for (int q = 1; q < js; ++q)
            for (int k = 0; k < kEVals; ++k)
                s[k] += pe[((int64_t)q * kEVals + k) * S + t];
        const double vi2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
        const double v12 = v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2];
        const double v1vi = v1[0] * vi[0] + v1[1] * vi[1] + v1[2] * vi[2];
        const double nvi = (d[0] * vi[0] + d[1] * vi[1] + d[2] * vi[2]) * iR;
        const double nv1 = (d[0] * v1[0] + d[1] * v1[1] + d[2] * v1[2]) * iR;
        const double pot = s[0];
        const double vSmv = vi[0] * s[1] + vi[1] * s[2] + vi[2] * s[3];
        const double pni = 6.0 * vi2 * pot - 7.0 * vSmv - s[4];
        const double gmm = G * M * mi * iR;
        o[0] = 0.5 * mi * vi2 - 0.5 * G * mi * pot - gmm;
        o[1] = 0.375 * mi * vi2 * vi2 + 1.5 * gmm * vi2 + 0.5 * G * gmm * M * iR +
               0.25 * G * mi * pni + 0.5 * gmm * (3.0 * v12 - 7.0 * v1vi - nv1 * nvi) +
               G * gmm * pot;
        for (int k = 0; k < 3; ++k) {
            o[2 + k] = mi * vi[k];
            const double pk = vi[k] * pot + s[5 + k];
            o[5 + k] = 0.5 * mi * vi2 * vi[k] -
                       0.5 * gmm * (vi[k] + nvi * d[k] * iR + v1[k] + nv1 * d[k] * iR) -
                       0.5 * G * mi * pk;
        }
        o[8] = mi * iR;
    }
    block_sum<kEBlockVals>(o, sh);
    if (threadIdx.x < kEBlockVals)
        blk[(int64_t)blockIdx.x * kEBlockVals + threadIdx.x] = sh[threadIdx.x][0];
}

// Totals per cluster (one block per cluster) plus the hole's own terms:
// 1/2 M v_1^2, M v_1 and the i = j double sum 1/2 G^2 M (sum_i m_i/R_i)^2 of
// Eq. 7; out[8 k .. 8 k + 7] for cluster k.
__global__ void __launch_bounds__(kGlueThreads)
k_energy_final(const Clu *__restrict__ clu, const double *__restrict__ blk,
               const double *__restrict__ vel, const double *__restrict__ m,
               double *__restrict__ out)
{
    __shared__ double sh[kEBlockVals][kGlueThreads];
    const Clu C = clu[blockIdx.x];
    sum_blocks<kEBlockVals>(blk + (C.slot0 / kGlueThreads) * kEBlockVals,
                            C.ns_pad / kGlueThreads, sh);
    if (threadIdx.x == 0) {
        const int64_t hb = C.body0;
        const double M = m[hb], G = C.G;
        const double v1[3] = {vel[3 * hb], vel[3 * hb + 1], vel[3 * hb + 2]};
        const double smr = sh[8][0];
        double *o = out + 8 * (int64_t)blockIdx.x;
        o[0] = sh[0][0] + 0.5 * M * (v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
        o[1] = C.inv_c2 * (sh[1][0] + 0.5 * G * G * M * smr * smr);
        for (int k = 0; k < 3; ++k) {
            o[2 + k] = sh[2 + k][0] + M * v1[k];
            o[5 + k] = C.inv_c2 * sh[5 + k][0];
        }
    }
}

// Energy-drift watchdog: one thread compares each cluster's total energy
// E = E_N + E_1PN (Eq. 7, just evaluated into eout) with its reference
// wd[k].  A NaN reference (armed, not yet taken) is replaced by E; else a
// relative change |E - E_ref| / |E_ref| above tol (or a non-finite one)
// sets flag bit 4 and, for the first step that does so, records the step
// index, the largest change and its cluster (wd[nclu], wd[nclu + 1]).
__global__ void k_watch(const double *__restrict__ eout, int nclu, double tol,
                        unsigned long long step, double *__restrict__ wd, int *__restrict__ flag,
                        unsigned long long *__restrict__ wstep)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    double worst = -1.0;
    int kworst = -1;
    for (int k = 0; k < nclu; ++k) {
        const double E = eout[8 * k] + eout[8 * k + 1];
        const double ref = wd[k];
        if (isnan(ref)) {
            wd[k] = E;
            continue;
        }
        double d = fabs(E - ref) / fabs(ref);
        if (!(d <= tol)) {
            d = isnan(d) ? INFINITY : d;
            if (d > worst) {
                worst = d;
                kworst = k;
            }
        }
    }
    if (kworst >= 0) {
        *flag |= 4;
        if (*wstep == ~0ull) {
            *wstep = step;
            wd[nclu] = worst;
            wd[nclu + 1] = (double)kworst;
        }
    }
}

// ------------------------------------------------------------ launchers --

static int64_t glue_blocks(int64_t n) { return (n + kGlueThreads - 1) / kGlueThreads; }

static void timing_begin(pn_ctx *c, int k, cudaEvent_t *end_out);

static const int *blk_table(const pn_ctx *c) { return c->nclu > 1 ? c->blk_clu : nullptr; }

cudaError_t launch_kick_drift(pn_ctx *c, double *x, double *v, const double *a, double dt)
{
    const int64_t n3 = 3 * c->n;
    const int64_t nb = glue_blocks(n3) < 4 * (int64_t)c->sm_count ? glue_blocks(n3)
                                                                    : 4 * (int64_t)c->sm_count;
    k_kick_drift<<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(n3, x, v, a, c->vp, 0.5 * dt, dt,
                                                               c->p.vel_mode);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_rk4_stage(pn_ctx *c, int stage, double *x, double *v, const double *a,
                             double dt)
{
    const int64_t n3 = 3 * c->n;
    const int64_t nb = glue_blocks(n3) < 4 * (int64_t)c->sm_count ? glue_blocks(n3)
                                                                    : 4 * (int64_t)c->sm_count;
    k_rk4_stage<<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(stage, n3, x, v, a, c->rk_a,
                                                              c->rk_x, c->rk_v, c->rk_sx,
                                                              c->rk_sv, dt);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_prologue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            bool energy_records)
{
    const int64_t npb = c->S / kProThreads;
    const int *bc = blk_table(c);
    if (energy_records) {
        k_prologue<2><<<(unsigned)npb, kProThreads, 0, c->stream>>>(
            c->S, c->d_clu, bc, x, vel, m, c->mrec, c->drec, c->nflag, c->blk, nullptr, 0);
        c->launches += 1;
        return cudaGetLastError();
    }
    const bool mixed = c->p.precision == PN_MIXED;
    if (mixed)
        k_prologue<0><<<(unsigned)npb, kProThreads, 0, c->stream>>>(
            c->S, c->d_clu, bc, x, vel, m, c->mrec, c->drec, c->nflag, c->blk, c->wcount,
            packed_loc(c) ? 1 : 0);
    else
        k_prologue<1><<<(unsigned)npb, kProThreads, 0, c->stream>>>(
            c->S, c->d_clu, bc, x, vel, m, c->mrec, c->drec, c->nflag, c->blk, c->wcount, 0);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_global_sums(pn_ctx *c)
{
    if (c->p.precision == PN_MIXED)
        k_global_sums<0><<<c->nclu, kGlueThreads, 0, c->stream>>>(
            c->d_clu, c->nclu, c->blk, c->glob, c->ncount, c->nrec, c->ndrec, c->NC);
    else
        k_global_sums<1><<<c->nclu, kGlueThreads, 0, c->stream>>>(
            c->d_clu, c->nclu, c->blk, c->glob, c->ncount, c->nrec, c->ndrec, c->NC);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_near_scatter(pn_ctx *c, const double *x, const double *m)
{
    if (!c->any_near)
        return cudaSuccess;
    const int64_t nb = c->S / kGlueThreads;
    const int *bc = blk_table(c);
    if (c->p.precision == PN_MIXED)
        k_near_scatter<0><<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(
            c->d_clu, c->nclu, bc, x, m, c->nflag, c->ncount, c->nrec, c->ndrec, c->NC);
    else
        k_near_scatter<1><<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(
            c->d_clu, c->nclu, bc, x, m, c->nflag, c->ncount, c->nrec, c->ndrec, c->NC);
    c->launches += 1;
    return cudaGetLastError();
}

// The spatial order's sort keys read the cluster sums (the mean |d|), so the
// pair kernel depends on them there; elsewhere it reads only the records.
bool pairs_need_sums(const pn_ctx *c)
{
    return use_fused(c) && c->fused_packed && c->spatial && packed_loc(c);
}

bool use_fused(const pn_ctx *c)
{
    return c->p.precision == PN_MIXED && c->p.pair_kernel == PN_PAIR_FUSED;
}

// Where the pair partial sums live in c->part (in units of S doubles):
//   two-pass: pass 1 [jsplit][kP1Vals], pass 2 [jsplit][kP2Vals], near [kNearVals]
//   fused:    pass 1 [kP1Vals], pass 2 [kP2Vals], near [kNearVals], then the
//             stream-K segments [target blocks + G][kFusedVals][TI]
struct Layout {
    int js;
    int64_t p1, p2, near, seg;
};

static Layout layout(const pn_ctx *c)
{
    Layout L;
    const int64_t S = c->S;
    if (use_fused(c)) {
        L.js = 1;
    } else {
        const Shape &s = c->p.precision == PN_MIXED ? c->mix : c->f64;
        L.js = s.jsplit;
    }
    L.p1 = 0;
    L.p2 = (int64_t)L.js * kP1Vals * S;
    L.near = (int64_t)L.js * (kP1Vals + kP2Vals) * S;
    L.seg = L.near + (int64_t)kNearVals * S;
    return L;
}

FusedVariant fused_variant(const pn_ctx *c)
{
    return FusedVariant{c->fused_P, c->fused_unroll, c->fused_packed ? 1 : 0, c->fused_tile,
                        c->fused_stages};
}

bool packed_layout_ok(int tile, int stages)
{
    return (tile == 64 && (stages == 6 || stages == 4)) || (tile == 32 && stages == 8);
}

int fused_tile_size(const FusedVariant &v) { return v.packed ? v.tile : kMixTile; }

// Work units of a fused-kernel variant over all clusters of the context.
static int64_t fused_unit_count(const pn_ctx *c, const FusedVariant &v)
{
    const int tile = fused_tile_size(v);
    int64_t u = 0;
    for (int k = 0; k < c->nclu; ++k)
        u += (c->hclu[k].ns_pad / (kMixThreads * v.P)) * (c->hclu[k].ns_pad / tile);
    return u;
}

// Launch shape of a fused-kernel variant: resident blocks per SM and in all,
// stream-K workers, work units.  The scalar kernel runs one worker per
// resident block; the packed kernel up to c->workers_max (default
// kPackWorkersMax) per block, at least 64 units each, taken dynamically.
cudaError_t fused_shape(const pn_ctx *c, const FusedVariant &v, FusedShape *out)
{
    int occ = 0;
    const cudaError_t e = fused_occupancy(v, &occ);
    if (e != cudaSuccess)
        return e;
    out->occ = occ > 0 ? occ : 1;
    out->grid = (int64_t)out->occ * c->sm_count;
    out->units = fused_unit_count(c, v);
    int64_t per = 1;
    if (v.packed) {
        const int64_t cap = c->workers_max > 0 ? c->workers_max : kPackWorkersMax;
        per = out->units / (out->grid * (int64_t)c->worker_units);
        per = per < 1 ? 1 : (per > cap ? cap : per);
    }
    out->G = out->grid * per;
    return cudaSuccess;
}

int64_t fused_units(const Clu *h, int nclu, const FusedVariant &v, Clu *out)
{
    const int tile = fused_tile_size(v);
    int64_t u = 0;
    for (int k = 0; k < nclu; ++k) {
        out[k] = h[k];
        out[k].unit0 = u;
        u += (h[k].ns_pad / (kMixThreads * v.P)) * (h[k].ns_pad / tile);
    }
    return u;
}

cudaError_t launch_pass1(pn_ctx *c)
{
    const Layout L = layout(c);
    cudaEvent_t end = nullptr;
    timing_begin(c, 0, &end);
    if (c->p.precision == PN_MIXED) {
        dim3 grid((unsigned)(c->S / (kMixThreads * kMixTargets)), (unsigned)c->mix.jsplit);
        k_pass_mixed<1><<<grid, kMixThreads, 0, c->stream>>>(c->mrec, c->S, c->d_clu,
                                                             blk_table(c), c->part + L.p1);
    } else {
        dim3 grid((unsigned)(c->S / kF64Threads), (unsigned)c->f64.jsplit);
        k_pass_f64<1><<<grid, kF64Threads, 0, c->stream>>>(c->drec, c->S, c->d_clu, blk_table(c),
                                                           c->part + L.p1, nullptr);
    }
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    return e;
}

cudaError_t launch_pass2(pn_ctx *c)
{
    const Layout L = layout(c);
    cudaEvent_t end = nullptr;
    timing_begin(c, 1, &end);
    if (c->p.precision == PN_MIXED) {
        dim3 grid((unsigned)(c->S / (kMixThreads * kMixTargets)), (unsigned)c->mix.jsplit);
        k_pass_mixed<2><<<grid, kMixThreads, 0, c->stream>>>(c->mrec, c->S, c->d_clu,
                                                             blk_table(c), c->part + L.p2);
    } else {
        dim3 grid((unsigned)(c->S / kF64Threads), (unsigned)c->f64.jsplit);
        k_pass_f64<2><<<grid, kF64Threads, 0, c->stream>>>(c->drec, c->S, c->d_clu, blk_table(c),
                                                           c->part + L.p2, nullptr);
    }
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    return e;
}

bool use_fused_f64(const pn_ctx *c)
{
    return c->p.precision == PN_FP64 && c->p.pair_kernel == PN_PAIR_FUSED;
}

// FP64 contexts with the fused pair kernel: both passes' sums in one sweep
// (k_pass_f64<3>), into the two-pass partial layout; timed as kernel 1.
cudaError_t launch_fused_f64(pn_ctx *c)
{
    const Layout L = layout(c);
    cudaEvent_t end = nullptr;
    timing_begin(c, 1, &end);
    dim3 grid((unsigned)(c->S / kF64Threads), (unsigned)c->f64.jsplit);
    k_pass_f64<3><<<grid, kF64Threads, 0, c->stream>>>(c->drec, c->S, c->d_clu, blk_table(c),
                                                       c->part + L.p1, c->part + L.p2);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    return e;
}

template <int P, int UNROLL>
static cudaError_t launch_fused_p(pn_ctx *c, const Layout &L, const float4 *rec)
{
    cudaEvent_t end = nullptr;
    timing_begin(c, 1, &end);
    k_fused_mixed<P, UNROLL><<<(unsigned)c->fused_grid, kMixThreads, 0, c->stream>>>(
        rec, c->S, c->d_clu, c->nclu, c->fused_units, c->part + L.seg);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    if (e != cudaSuccess)
        return e;
    k_fused_gather<P, kFusedVals, 0><<<dim3((unsigned)(c->S / kGatherThreads), 3), kGatherThreads, 0, c->stream>>>(
        c->part + L.seg, c->S, c->d_clu, blk_table(c), c->fused_units, c->fused_G, kMixTile,
        nullptr, nullptr, nullptr, c->part + L.p1, c->part + L.p2);
    c->launches += 1;
    return cudaGetLastError();
}

// The packed kernel on the staged records at c->mrec + 5 S: the
// law-of-cosines form on the prologue's records when every cluster splits off
// its near sources (packed_loc), else the D form; caller-built records (far
// form: every source keeps its hole term) are staged in the D form first.
// Form FORM of the packed kernel (k_fused_packed) on staged records `srec`
// (boxes and the sorted-to-slot map for form 2), then the gather.
template <int NP, int UNROLL, int FORM, int TILE, int ST>
static cudaError_t launch_packed_form(pn_ctx *c, const Layout &L, const float4 *srec,
                                      const float4 *box, const int *perm, const int64_t *wb)
{
    cudaEvent_t end = nullptr;
    timing_begin(c, 1, &end);
    k_fused_packed<NP, UNROLL, FORM, TILE, ST><<<(unsigned)c->fused_grid, kMixThreads, 0, c->stream>>>(
        srec, c->d_clu, c->nclu, c->fused_units, c->fused_G, c->wcount, c->flag, c->inject_tx,
        box, c->far_theta, c->units_cnt, wb, c->part + L.seg);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    if (e != cudaSuccess)
        return e;
    k_fused_gather<2 * NP, kPackSums, pack_vals<(FORM >= 1)>()>
        <<<dim3((unsigned)(c->S / kGatherThreads), 3), kGatherThreads, 0, c->stream>>>(
            c->part + L.seg, c->S, c->d_clu, blk_table(c), c->fused_units, c->fused_G, TILE,
            srec, perm, wb, c->part + L.p1, c->part + L.p2);
    c->launches += 1;
    return cudaGetLastError();
}

bool packed_loc(const pn_ctx *c) { return c->fused_packed && c->near_all; }

// The packed kernel on the staged records at c->mrec + 5 S: on the
// prologue's records the law-of-cosines form when every cluster splits off
// its near sources (packed_loc; in the spatial order when c->spatial), else
// the D form; caller-built records (far form: every source keeps its hole
// term) are staged in the D form first.
template <int NP, int UNROLL, int TILE, int ST>
static cudaError_t launch_packed_v(pn_ctx *c, const Layout &L, const float4 *rec)
{
    const float4 *srec = c->mrec + 5 * c->S;
    if (rec == c->mrec && packed_loc(c)) {
        if constexpr (TILE == kPackTile) {
            if (c->spatial) {
                cudaError_t e = launch_spatial_order(c);
                const int64_t *wb = nullptr;
                if (e == cudaSuccess && c->balance)
                    e = launch_worker_balance(c, NP, &wb);
                if (e != cudaSuccess)
                    return e;
                const Order o = order_of(c);
                return launch_packed_form<NP, UNROLL, 2, TILE, ST>(c, L, o.ssrec, o.box, o.perm,
                                                                   wb);
            }
        }
        return launch_packed_form<NP, UNROLL, 1, TILE, ST>(c, L, srec, nullptr, nullptr, nullptr);
    }
    if (rec != c->mrec) {       // caller-built records: stage them first
        k_stage_sources<<<(unsigned)(c->S / kGlueThreads), kGlueThreads, 0, c->stream>>>(
            c->S, rec, c->mrec + 5 * c->S);
        c->launches += 1;
    }
    return launch_packed_form<NP, UNROLL, 0, TILE, ST>(c, L, srec, nullptr, nullptr, nullptr);
}

// The context's (tile, stages) of the packed kernel; 32-source tiles only
// on the slot order (variant selection keeps them off the spatial order).
template <int NP, int UNROLL>
static cudaError_t launch_packed_u(pn_ctx *c, const Layout &L, const float4 *rec)
{
    if (c->fused_tile == 32)
        return launch_packed_v<NP, UNROLL, 32, 8>(c, L, rec);
    if (c->fused_stages == 4)
        return launch_packed_v<NP, UNROLL, kPackTile, 4>(c, L, rec);
    return launch_packed_v<NP, UNROLL, kPackTile, kPackStages>(c, L, rec);
}

// Fused-kernel variants: scalar (targets per thread 1, 2, 4) or packed
// FP32x2 (4 targets per thread) x source-loop unroll.
static cudaError_t launch_fused_with(pn_ctx *c, const Layout &L, const float4 *r)
{
    const int u = c->fused_unroll;
    if (c->fused_packed) {
        if (c->fused_P == 2)
            return u == 2 ? launch_packed_u<1, 2>(c, L, r) : launch_packed_u<1, 1>(c, L, r);
        return u == 2 ? launch_packed_u<2, 2>(c, L, r) : launch_packed_u<2, 1>(c, L, r);
    }
    switch (c->fused_P) {
    case 1: return u == 2 ? launch_fused_p<1, 2>(c, L, r) : launch_fused_p<1, 1>(c, L, r);
    case 4:
        return u == 4 ? launch_fused_p<4, 4>(c, L, r)
             : u == 3 ? launch_fused_p<4, 3>(c, L, r)
             : u == 2 ? launch_fused_p<4, 2>(c, L, r) : launch_fused_p<4, 1>(c, L, r);
    default:
        return u == 4 ? launch_fused_p<2, 4>(c, L, r)
             : u == 2 ? launch_fused_p<2, 2>(c, L, r) : launch_fused_p<2, 1>(c, L, r);
    }
}

cudaError_t launch_fused(pn_ctx *c) { return launch_fused_with(c, layout(c), c->mrec); }

// Staged source records (c->mrec + 5 S) of the packed kernels from mixed
// records rec (the prologue writes them for c->mrec itself).
cudaError_t launch_stage_sources(pn_ctx *c, const float4 *rec)
{
    k_stage_sources<<<(unsigned)(c->S / kGlueThreads), kGlueThreads, 0, c->stream>>>(
        c->S, rec, c->mrec + 5 * c->S);
    c->launches += 1;
    return cudaGetLastError();
}

// The fused pair kernel on caller-built mixed records (same layout as the
// prologue's), with the fused partial layout whatever the context's pair
// kernel: the 16 pair sums land in c->part as [value][slot] (pass-1 values,
// then pass-2 values).  Zeroes the packed kernel's worker counter first.
cudaError_t launch_fused_on(pn_ctx *c, const float4 *rec)
{
    Layout L;
    L.js = 1;
    L.p1 = 0;
    L.p2 = (int64_t)kP1Vals * c->S;
    L.near = (int64_t)(kP1Vals + kP2Vals) * c->S;
    L.seg = L.near + (int64_t)kNearVals * c->S;
    cudaError_t e = cudaMemsetAsync(c->wcount, 0, sizeof(int), c->stream);
    if (e != cudaSuccess)
        return e;
    return launch_fused_with(c, L, rec);
}

// The fused kernels hold 64-75 KB of shared memory per block; three blocks
// per SM need the largest shared-memory carveout, which is requested here
// (before the occupancy query and the first launch).
template <typename K>
static cudaError_t occ_with_carveout(K kernel, int *occ)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, kMixThreads, 0);
}

template <int P, int UNROLL>
static cudaError_t occ_of(int *occ)
{
    return occ_with_carveout(k_fused_mixed<P, UNROLL>, occ);
}

// Resident blocks of the packed kernel: the smallest over its forms, so
// that one launch shape serves them all.
template <int NP, int UNROLL, int TILE, int ST>
static cudaError_t occ_packed_v(int *occ)
{
    int o[3] = {0, 0, 1 << 20};
    cudaError_t e = occ_with_carveout(k_fused_packed<NP, UNROLL, 0, TILE, ST>, &o[0]);
    if (e == cudaSuccess)
        e = occ_with_carveout(k_fused_packed<NP, UNROLL, 1, TILE, ST>, &o[1]);
    if constexpr (TILE == kPackTile)
        if (e == cudaSuccess)
            e = occ_with_carveout(k_fused_packed<NP, UNROLL, 2, TILE, ST>, &o[2]);
    *occ = o[0] < o[1] ? o[0] : o[1];
    *occ = o[2] < *occ ? o[2] : *occ;
    return e;
}

template <int NP, int UNROLL>
static cudaError_t occ_packed(int tile, int stages, int *occ)
{
    if (tile == 32)
        return occ_packed_v<NP, UNROLL, 32, 8>(occ);
    if (stages == 4)
        return occ_packed_v<NP, UNROLL, kPackTile, 4>(occ);
    return occ_packed_v<NP, UNROLL, kPackTile, kPackStages>(occ);
}

cudaError_t fused_occupancy(const FusedVariant &v, int *occ)
{
    const int P = v.P, unroll = v.unroll;
    if (v.packed) {
        if (P == 2)
            return unroll == 2 ? occ_packed<1, 2>(v.tile, v.stages, occ)
                               : occ_packed<1, 1>(v.tile, v.stages, occ);
        return unroll == 2 ? occ_packed<2, 2>(v.tile, v.stages, occ)
                           : occ_packed<2, 1>(v.tile, v.stages, occ);
    }
    switch (P) {
    case 1: return unroll == 2 ? occ_of<1, 2>(occ) : occ_of<1, 1>(occ);
    case 4:
        return unroll == 4 ? occ_of<4, 4>(occ)
             : unroll == 3 ? occ_of<4, 3>(occ)
             : unroll == 2 ? occ_of<4, 2>(occ) : occ_of<4, 1>(occ);
    default:
        return unroll == 4 ? occ_of<2, 4>(occ)
             : unroll == 2 ? occ_of<2, 2>(occ) : occ_of<2, 1>(occ);
    }
}

cudaError_t launch_near(pn_ctx *c)
{
    if (!c->any_near)
        return cudaSuccess;
    const Layout L = layout(c);
    double *pn = c->part + L.near;
    cudaEvent_t end = nullptr;
    timing_begin(c, 2, &end);
    if (c->p.precision == PN_MIXED)
        k_near_mixed<<<(unsigned)(c->S / (kMixThreads * kMixTargets)), kMixThreads, 0, c->stream>>>(
            c->mrec, c->nrec, c->ncount, c->S, c->NC, c->d_clu, blk_table(c), pn);
    else
        k_near_f64<<<(unsigned)(c->S / kF64Threads), kF64Threads, 0, c->stream>>>(
            c->drec, c->ndrec, c->ncount, c->S, c->NC, c->d_clu, blk_table(c), pn);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (end)
        cudaEventRecord(end, c->stream);
    return e;
}

cudaError_t launch_epilogue(pn_ctx *c, const double *x, const double *vel, const double *m,
                            double *a, double *v, double h, unsigned long long step,
                            double dt_next)
{
    const Layout L = layout(c);
    const int64_t nb = c->S / kEpiThreads;
    const double *pnear = c->any_near ? c->part + L.near : nullptr;
    // x and vel are written only with dt_next > 0, which the integrator asks
    // for on its own state arrays
    k_epilogue<<<(unsigned)nb, kEpiThreads, 0, c->stream>>>(
        c->S, c->d_clu, blk_table(c), const_cast<double *>(x), const_cast<double *>(vel), m,
        c->part + L.p1, L.js, c->part + L.p2, L.js, pnear, c->nflag, c->glob, a, v, h, c->flag,
        c->flag_step, step, c->blk, c->epi_done, v ? dt_next : 0.0, c->p.vel_mode);
    c->launches += 1;
    return cudaGetLastError();
}

// Source splits of the energy pair kernel: about 24 blocks per SM over the
// 128-slot target blocks (the FP64 pipe is full with a few; the rest keep
// the last wave short), at most one per tile of the largest cluster and at
// most kEnergySplitsMax.
int64_t energy_splits(int64_t S, int sm_count, int64_t max_ns_pad)
{
    const int64_t nb = S / kF64Threads, tiles = max_ns_pad / kF64Tile;
    int64_t js = (24 * (int64_t)sm_count + nb - 1) / nb;
    js = js > tiles ? tiles : js;
    js = js > kEnergySplitsMax ? kEnergySplitsMax : js;
    return js < 1 ? 1 : js;
}

cudaError_t launch_energy(pn_ctx *c, const double *x, const double *v, const double *m)
{
    cudaError_t e = launch_prologue(c, x, v, m, true);
    if (e != cudaSuccess)
        return e;
    const int js = (int)energy_splits(c->S, c->sm_count, c->max_ns_pad);
    const dim3 grid((unsigned)(c->S / kF64Threads), (unsigned)js);
    if (c->p.precision == PN_MIXED) {      // double-single pair sums on the FP32 pipe
        float4 *drs = reinterpret_cast<float4 *>(c->part + (int64_t)kEVals * js * c->S);
        k_energy_stage_ds<<<(unsigned)(c->S / kGlueThreads), kGlueThreads, 0, c->stream>>>(
            c->S, c->drec, drs);
        k_energy_pairs_ds<<<grid, kF64Threads, 0, c->stream>>>(drs, c->S, c->d_clu,
                                                              blk_table(c), c->part);
        c->launches += 2;
    } else {
        k_energy_pairs<<<grid, kF64Threads, 0, c->stream>>>(c->drec, c->S, c->d_clu,
                                                            blk_table(c), c->part);
        c->launches += 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_energy_epilogue<<<(unsigned)(c->S / kGlueThreads), kGlueThreads, 0, c->stream>>>(
        c->S, c->d_clu, blk_table(c), x, v, m, c->part, js, c->blk);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_energy_final<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, c->blk, v, m, c->eout);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_watch(pn_ctx *c)
{
    k_watch<<<1, 32, 0, c->stream>>>(c->eout, c->nclu, c->wd_tol,
                                     (unsigned long long)c->step_counter, c->wd, c->flag,
                                     c->wd_step);
    c->launches += 1;
    return cudaGetLastError();
}

// The energy evaluation on scratch the caller provides, for one cluster whose
// table entry `clu` is already in device memory.
cudaError_t launch_energy_on(cudaStream_t st, int64_t S, const Clu *clu, const double *x,
                             const double *v, const double *m, double4_32a *drec, double *part,
                             double *blk, double *out)
{
    const int64_t nb = S / kProThreads;
    k_prologue<2><<<(unsigned)nb, kProThreads, 0, st>>>(S, clu, nullptr, x, v, m, nullptr, drec,
                                                         nullptr, nullptr, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_energy_pairs<<<(unsigned)(S / kF64Threads), kF64Threads, 0, st>>>(drec, S, clu, nullptr, part);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // one kGlueThreads-slot block per row of blk (S / kGlueThreads rows)
    k_energy_epilogue<<<(unsigned)(S / kGlueThreads), kGlueThreads, 0, st>>>(S, clu, nullptr, x, v,
                                                                            m, part, 1, blk);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_energy_final<<<1, kGlueThreads, 0, st>>>(clu, blk, v, m, out);
    return cudaGetLastError();
}

// Timing ring: an event pair per pair-kernel launch; the oldest pair is
// folded into the total when the ring is full (this waits for that event,
// which lies far behind the queued work).
static void timing_begin(pn_ctx *c, int k, cudaEvent_t *end_out)
{
    *end_out = nullptr;
    if (!c->timing_on || c->capturing)
        return;
    Timing &t = c->tm;
    if (t.count[k] == Timing::kRing) {
        const int old = t.head[k];
        float ms = 0.0f;
        if (cudaEventSynchronize(t.ev1[k][old]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, t.ev0[k][old], t.ev1[k][old]) == cudaSuccess)
            t.ms[k] += ms;
        t.launches[k] += 1;
        t.head[k] = (old + 1) % Timing::kRing;
        t.count[k] -= 1;
    }
    const int slot = (t.head[k] + t.count[k]) % Timing::kRing;
    cudaEventRecord(t.ev0[k][slot], c->stream);
    *end_out = t.ev1[k][slot];
    t.count[k] += 1;
}

void shapes(int64_t S, int64_t max_ns_pad, int sm_count, int occ_mix, int occ_f64, Shape *mix,
            Shape *f64)
{
    struct Cfg { int threads, targets, tile, occ; Shape *out; } cfg[2] = {
        {kMixThreads, kMixTargets, kMixTile, occ_mix, mix},
        {kF64Threads, kF64Targets, kF64Tile, occ_f64, f64}};
    for (auto &c : cfg) {
        Shape &s = *c.out;
        s.threads = c.threads;
        s.targets = c.targets;
        s.tile = c.tile;
        s.occupancy = c.occ > 0 ? c.occ : 1;
        s.nblk_i = S / (c.threads * c.targets);
        s.ntiles = (int)(max_ns_pad / c.tile);
        const int64_t resident = (int64_t)s.occupancy * sm_count;
        int64_t want = (8 * resident + s.nblk_i - 1) / s.nblk_i;   // splits for ~8 waves
        if (want < 1)
            want = 1;
        if (want > s.ntiles)
            want = s.ntiles;
        s.jsplit = (int)want;
        s.tiles_per_split = (s.ntiles + s.jsplit - 1) / s.jsplit;
    }
}

cudaError_t occupancy(int *occ_mix, int *occ_f64)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_mix, k_pass_mixed<2>,
                                                                  kMixThreads, 0);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_f64, k_pass_f64<2>, kF64Threads, 0);
}

PN_DEBUG_ACCESSOR(debug_take_kernels)

}  // namespace pn
