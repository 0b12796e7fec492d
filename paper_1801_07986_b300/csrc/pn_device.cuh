// pn_device.cuh -- device helpers shared by the kernel files of libpn:
// deterministic block reductions, the cluster lookup, the non-finite flag,
// a forward-mode dual number, and the per-star assembly of Eq. 4-6 (and the
// star's term of Eq. 1-3) written once over the scalar type.
#pragma once

#include <math.h>
#include <stdint.h>

#include "pn_internal.h"

namespace pn {

// Deterministic block sum of K doubles per thread (fixed tree, blockDim =
// BT); thread 0 ends with the totals in sh[k][0].
template <int K, int BT = kGlueThreads>
__device__ __forceinline__ void block_sum(double (&val)[K], double (*sh)[BT])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < K; ++k)
        sh[k][t] = val[k];
    __syncthreads();
    // NPART row segments of RP rows per column, every segment starting
    // inside the block (NPART * K <= BT threads)
    constexpr int NP0 = BT / K;
    constexpr int RP = NP0 >= 1 ? (BT + NP0 - 1) / NP0 : BT;
    constexpr int NPART = (BT + RP - 1) / RP;
    static_assert(NPART * K <= BT || NP0 < 2, "segment threads exceed the block");
    if constexpr (NP0 >= 2) {
        // thread (q, k) sums rows [q RP, (q + 1) RP) of column k in order,
        // then thread k adds the segment sums in order: two barriers, and
        // every thread of the first K * NPART does FP64 work
        if (t < K * NPART) {
            const int k = t % K, q = t / K;
            const int r0 = q * RP, r1 = r0 + RP < BT ? r0 + RP : BT;
            double acc = sh[k][r0];
            for (int r = r0 + 1; r < r1; ++r)
                acc += sh[k][r];
            sh[k][r0] = acc;
        }
        __syncthreads();
        if (t < K) {
            double acc = sh[t][0];
            for (int q = 1; q < NPART; ++q)
                acc += sh[t][q * RP];
            sh[t][0] = acc;
        }
        __syncthreads();
    } else {
        for (int s = BT / 2; s > 0; s >>= 1) {
            if (t < s) {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    sh[k][t] += sh[k][t + s];
            }
            __syncthreads();
        }
    }
}

// Sum per-block partials blk[b*K + k] over b in a fixed order (one block of
// kGlueThreads threads; the totals land in sh[k][0]).  Warp w sums the
// columns k = w, w + 8, ...: lane l adds rows l, l + 32, ... into four
// accumulators (row index mod 128 picks one), which are combined and then
// reduced across the lanes by shuffles -- one block barrier in all, where a
// shared-memory tree over the threads waits at eight.
template <int K>
__device__ __forceinline__ void sum_blocks(const double *__restrict__ blk, int64_t nblk,
                                           double (*sh)[kGlueThreads])
{
    constexpr int NW = kGlueThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < K; k += NW) {
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int64_t b = lane;
        for (; b + 96 < nblk; b += 128) {
            v0 += blk[b * K + k];
            v1 += blk[(b + 32) * K + k];
            v2 += blk[(b + 64) * K + k];
            v3 += blk[(b + 96) * K + k];
        }
        if (b < nblk)
            v0 += blk[b * K + k];
        if (b + 32 < nblk)
            v1 += blk[(b + 32) * K + k];
        if (b + 64 < nblk)
            v2 += blk[(b + 64) * K + k];
        double v = (v0 + v1) + (v2 + v3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            sh[k][0] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ void flag_nonfinite(const double a[3], int *flag,
                                               unsigned long long *flag_step,
                                               unsigned long long step)
{
    if (!(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]))) {
        atomicOr(flag, 1);
        atomicMin(flag_step, step);
    }
}

// Clusters: the state arrays hold one or more independent clusters, each a
// hole (body clu.body0) followed by clu.ns stars.  Star slots of all
// clusters are laid end to end, each cluster padded to a multiple of kPad
// (zero-mass far-away dummies), so every 256-slot block and every target
// block lies inside one cluster; blk_clu[slot / 256] names it (nullptr:
// a single cluster, index 0).
__device__ __forceinline__ int cluster_of_block(const int *__restrict__ blk_clu, int64_t b)
{
    return blk_clu ? blk_clu[b] : 0;
}

// Cluster of work unit u of the fused pair kernels (units are laid out
// cluster-major; clu[k].unit0 is cluster k's first).
__device__ __forceinline__ int cluster_of_unit(const Clu *__restrict__ clu, int nclu, int64_t u)
{
    int lo = 0, hi = nclu - 1;
    while (lo < hi) {                        // last cluster with unit0 <= u
        const int mid = (lo + hi + 1) >> 1;
        if (clu[mid].unit0 <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// 1/sqrt(s2) in single precision: the PTX approximate reciprocal square root
// (one MUFU instruction; max relative error about 2^-23), flushing subnormal
// inputs to zero -- pair distances squared are never subnormal (s2 >= eps^2,
// and unsoftened pairs are far from 1e-38).
__device__ __forceinline__ float rsqrt_approx(float s2)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s2));
    return y;
}

// ------------------------------------------------------- dual numbers --

// Forward-mode dual number v + d eps (eps^2 = 0): evaluating a function on
// Duals gives its value and its derivative along the seeded direction.
struct Dual {
    double v, d;
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {a.v * s, a.d * s}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual operator+(double s, Dual a) { return {s + a.v, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double s) { return {a.v - s, a.d}; }
__device__ __forceinline__ Dual operator-(double s, Dual a) { return {s - a.v, -a.d}; }
__device__ __forceinline__ Dual operator/(double s, Dual a)
{
    const double r = s / a.v;
    return {r, -r * a.d / a.v};
}
__device__ __forceinline__ Dual operator/(Dual a, double s) { return {a.v / s, a.d / s}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double r = a.v / b.v;
    return {r, (a.d - r * b.d) / b.v};
}
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b)
{
    a.v += b.v;
    a.d += b.d;
    return a;
}

__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dual tsqrt(Dual a)
{
    const double s = sqrt(a.v);
    return {s, 0.5 * a.d / s};
}

// ----------------------------------------------- per-star assembly --

// Star i's acceleration (Eq. 4-6) and its term of the hole's 1PN
// acceleration (Eq. 2-3, j = i), from the pair sums of passes 1 and 2, the
// near-source sums and the cluster's global sums, over scalar type T
// (double, or Dual for the jerk and the adjoint).  Velocities vv are those
// at which A is taken; m_i is a constant; the hole mass M and inv_c2 have
// type TM (double, or Dual where they are differentiated).
//   a_i = -G M d_i/R_i^3 - G N_i + (1/c^2) {
//       G M d_i/R_i^3 (4 G M/R_i - v_i^2) + 4 G M (v_i.d_i) v_i/R_i^3   [Eq. 5]
//     + 5 G^2 m_i M d_i/R_i^4                                          [Eq. 6 l.1]
//     + G^2 M d_i/R_i^3 S_i                                            [Eq. 6 l.2]
//     + G [V_i + (4 G M/R_i + v_i^2) N_i]                              [l.3 + l.6]
//     - 7/2 G^2 M [E_i - (W_far - w_i)/R_i]                            [l.4]
//     - G/R_i^3 [4 (v_i.Q) d_i - 3 (Q.d_i) v_i - 4 (v_i.d_i) Q]        [l.1 + l.5]
//     + G H_i                                                          [l.7]
//     + G^2 M (P_i - 7/2 Ee_i) }                                       [near sources]
// with V_i = 3/2 V'_i (pass 2 carries -4/3 of the v_i^2 part, as
// -2 v_i^2 N_i, so the coefficient of N_i applied here is 4 G M/R_i - v_i^2),
// H_i = 3/2 (Hs_i v_i - Hv_i), and over far sources j != i
//   S_i = 4 U_i + sum_far m_j (5/(4R_j) + (R_i^2 - r_ij^2)/(4R_j^3))
//       = 4 U_i + (SA_far - 5 m_i/(4R_i)) + d_i.(W_far - w_i)/2
//         - (SB_far - m_i (R_i^2 + eps^2)/(4 R_i^3))
// (R_i^2 - r_ij^2 = 2 d_i.d_j - R_j^2 - eps^2; the m_i / w_i self terms are
// removed only when star i is itself a far source, fi = 1).  Line 1's self
// term and line 5 together are the k-sum over all stars, hence Q.
// The hole's term (Eq. 2 and Eq. 3 with j = i), Y_i = R_i^2 Z_i - Wr_i:
//   -G w_j (5 G M/R_j - 2 v_j^2 + 3/2 (v_j.d_j)^2/R_j^2) - 3 G m_j/R_j^3 (v_j.d_j) v_j
//   - 4 G^2 m_j w_j / R_j
//   - G^2 w_j [4 (Phi - m_j/R_j) + 5/4 U_j + 1/4 Y_j]
//   - 7/2 G^2 (m_j/R_j) N_j
//   + G/M m_j/R_j^3 [4 (v_j.Q) d_j - 3 (v_j.d_j) Q - 4 (Q.d_j) v_j]
template <class T>
struct StarSums {
    T N[3], U, Z, Wr;        // pass 1
    T Vp[3], Hs, Hv[3], E[3];  // pass 2
    T P[3], Ee[3];           // near-source pass (zero when unused)
};

template <class T>
struct ClusterSums {
    T Q[3], Wf[3], SA, SB, Phi;
};

template <class T, class TM>
__device__ __forceinline__ void star_eqs(double G, const TM &M, double mi, double eps2,
                                         const TM &inv_c2, double fi, const T (&d)[3],
                                         const T (&vv)[3], const StarSums<T> &s,
                                         const ClusterSums<T> &g, T (&ai)[3], T (&bh)[3])
{
    const TM GM = G * M;
    const T R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const T R = tsqrt(R2);
    const T iR = 1.0 / R;
    const T iR3 = iR * iR * iR;
    const T v2 = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
    const T vd = vv[0] * d[0] + vv[1] * d[1] + vv[2] * d[2];
    const T Y = R2 * s.Z - s.Wr;
    T Vv[3], H[3];
    for (int k = 0; k < 3; ++k) {
        Vv[k] = 1.5 * s.Vp[k];
        H[k] = 1.5 * (s.Hs * vv[k] - s.Hv[k]);
    }
    const T wi[3] = {mi * iR3 * d[0], mi * iR3 * d[1], mi * iR3 * d[2]};
    const T Wx[3] = {g.Wf[0] - fi * wi[0], g.Wf[1] - fi * wi[1], g.Wf[2] - fi * wi[2]};
    const T vQ = vv[0] * g.Q[0] + vv[1] * g.Q[1] + vv[2] * g.Q[2];
    const T Qd = g.Q[0] * d[0] + g.Q[1] * d[1] + g.Q[2] * d[2];
    const T S = 4.0 * s.U + (g.SA - fi * 1.25 * mi * iR) +
                0.5 * (d[0] * Wx[0] + d[1] * Wx[1] + d[2] * Wx[2]) -
                (g.SB - fi * 0.25 * mi * (R2 + eps2) * iR3);
    const T cd = GM * iR3 * (4.0 * GM * iR - v2) + 5.0 * G * GM * mi * iR3 * iR +
                 G * GM * iR3 * S - 4.0 * G * iR3 * vQ;
    const T cv = 4.0 * GM * iR3 * vd + 3.0 * G * iR3 * Qd;
    const T cN = G * (4.0 * GM * iR - v2);
    const T cQ = 4.0 * G * iR3 * vd;
    const TM c7 = 3.5 * G * GM;
    for (int k = 0; k < 3; ++k) {
        const T pn = cd * d[k] + cv * vv[k] + G * Vv[k] + cN * s.N[k] -
                     c7 * (s.E[k] - Wx[k] * iR) + cQ * g.Q[k] + G * H[k] +
                     G * GM * (s.P[k] - 3.5 * s.Ee[k]);
        ai[k] = (-GM * iR3 * d[k] - G * s.N[k]) + inv_c2 * pn;
    }
    const T b1 = -G * (5.0 * GM * iR - 2.0 * v2 + 1.5 * vd * vd * iR * iR) -
                 4.0 * G * G * mi * iR - G * G * (4.0 * (g.Phi - mi * iR) + 1.25 * s.U + 0.25 * Y);
    const T gmr3 = G * mi * iR3;
    for (int k = 0; k < 3; ++k)
        bh[k] = b1 * wi[k] - 3.0 * gmr3 * vd * vv[k] - 3.5 * G * G * mi * iR * s.N[k] +
                (gmr3 / M) * (4.0 * vQ * d[k] - 3.0 * vd * g.Q[k] - 4.0 * Qd * vv[k]);
}

// ---- debug build: index checks that report instead of trapping ----
// Compiled with -DPN_DEBUG_CHECKS (libpn_debug.so), PN_IDX(i, n, site)
// checks 0 <= i < n.  A failing check keeps the first (site, index) of its
// source file in dbg_word and yields index 0, so the access stays inside
// the buffer and no thread leaves its kernel, or a barrier, early; the host
// reads and clears the words after each wait (pn::debug_take) and reports
// PN_EINDEX.  dbg_inject (set from PN_DEBUG_INJECT=<site> when a context is
// created) makes every check of that site fail, so the reporting path can
// be tested without a bad index.  Release builds compile PN_IDX to `i`.
// Sites (pn_kernels.cu 1-19, pn_order.cu 20-29):
//   1 kick/drift component       2 prologue slot          3 prologue star
//   4 near-scatter entry         5 packed source tile     6 packed target block
//   8 gather slot               10 near-pass source      11 epilogue slot
//  14 energy-pair source        15 energy-epilogue slot
//  20 sort-scatter destination  21 permuted slot
#ifdef PN_DEBUG_CHECKS
static __device__ unsigned long long dbg_word[2];   // [0] site (0: none), [1] index
static __device__ int dbg_inject;
__device__ __forceinline__ int64_t dbg_idx(int64_t i, int64_t n, int site)
{
    if (i >= 0 && i < n && site != dbg_inject)
        return i;
    if (atomicCAS(&dbg_word[0], 0ull, (unsigned long long)site) == 0ull)
        dbg_word[1] = (unsigned long long)i;
    return 0;
}
#define PN_IDX(i, n, site) ::pn::dbg_idx((int64_t)(i), (int64_t)(n), (site))
// Defines this file's host accessor: arms the injected site, then returns
// and clears the first failed check (site 0: none).
#define PN_DEBUG_ACCESSOR(name)                                                          \
    cudaError_t name(int inject, unsigned long long *site, long long *index)            \
    {                                                                                    \
        unsigned long long w[2] = {0ull, 0ull};                                          \
        cudaError_t e = cudaMemcpyToSymbol(dbg_inject, &inject, sizeof inject);          \
        if (e == cudaSuccess)                                                            \
            e = cudaMemcpyFromSymbol(w, dbg_word, sizeof w);                             \
        if (e == cudaSuccess && w[0]) {                                                  \
            const unsigned long long z[2] = {0ull, 0ull};                                \
            e = cudaMemcpyToSymbol(dbg_word, z, sizeof z);                               \
        }                                                                                \
        *site = w[0];                                                                    \
        *index = (long long)w[1];                                                        \
        return e;                                                                        \
    }
#else
#define PN_IDX(i, n, site) (i)
#define PN_DEBUG_ACCESSOR(name)                                                          \
    cudaError_t name(int, unsigned long long *site, long long *index)                    \
    {                                                                                    \
        *site = 0ull;                                                                    \
        *index = 0;                                                                      \
        return cudaSuccess;                                                              \
    }
#endif

// ---- packed FP32x2 arithmetic (two lanes per register pair) ----
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4 &f) { return make_float2(f.x, f.y); }
__device__ __forceinline__ float2 hi2(const float4 &f) { return make_float2(f.z, f.w); }

// ---- bulk-copy staging (TMA engine, mbarrier completion) ----
constexpr unsigned long long kWaitNs = 1000000000ull;    // a tile wait gives up after 1 s
constexpr int kFlagTimeout = 2;                          // flag bit: a bounded wait gave up

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arms the barrier for `bytes` + `extra` of transaction and starts one bulk
// copy of `bytes` from global `src` to shared `dst` that completes on it.
// Both addresses 16-byte aligned, bytes a multiple of 16.  extra > 0 (a test
// hook) leaves the phase incomplete, so the wait runs out.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                          unsigned extra)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes + extra) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the barrier's phase `parity` until %globaltimer passes t_end
// (checked every 256 polls); false if it did not complete by then.
__device__ __forceinline__ bool mbar_wait_until(uint64_t *bar, unsigned parity,
                                                unsigned long long t_end)
{
    const uint32_t a = smem_addr(bar);
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done)
            return true;
        if ((i & 255) == 0 && global_ns() > t_end)
            return false;
    }
}

// Waits for the barrier's phase `parity` to complete; false once kWaitNs
// have passed (checked every 256 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = smem_addr(bar);
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done)
            return true;
        if ((i & 255) == 0) {
            const unsigned long long t = global_ns();
            if (i == 0)
                t0 = t;
            else if (t - t0 > kWaitNs)
                return false;
        }
    }
}

}  // namespace pn
