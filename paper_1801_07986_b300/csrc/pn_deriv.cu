// pn_deriv.cu -- derivatives of the accelerations of Eq. 1-6 (Tatekawa,
// arXiv:1801.07986): the jerk of Appendix A (forward mode), the
// fourth-order Hermite steps that use it (Section 5), and the adjoint
// (vector-Jacobian product) of A and of kick-drift-kick steps (reverse
// mode), all in double precision.
//
// The jerk is the time derivative along the trajectory,
//   j = sum_k [dA/dx_k . v_k + dA/dv_k . a_k],   a = A(x, v).
// Appendix A prints the expanded derivative (garbled in places).  Here the
// derivative is taken of the same decomposition the acceleration kernels
// evaluate, in forward mode: every quantity is a dual number (value,
// derivative along x' = v, v' = a), in double precision, through the
// records, the cluster sums, the pair sums (one pass with all 16 sums) and
// the per-star assembly (star_eqs).  Stars near the hole are not split off
// (that split only changes single-precision rounding).
#include <math.h>
#include <stdint.h>

#include "pn_device.cuh"

namespace pn {

namespace {

constexpr int kJRec = 8;         // double4 records per star slot
constexpr int kJVals = 12;       // Dual cluster sums: Q (3), W (3), W_far (3), SA, SB, Phi
constexpr int kJTile = 32;       // sources per shared-memory tile
constexpr int kJThreads = 128;

__device__ __forceinline__ Dual dual(double v, double d) { return {v, d}; }

// Records per star slot t (zero-mass far-away padding past the stars):
//   J0 = (d, m)  J1 = (d', 0)  J2 = (v, R^2)  J3 = (v', (R^2)')
//   J4 = (-e/1.5, C)  J5 = (-(e/1.5)', C')  J6 = (w, 0)  J7 = (w', 0)
// (primes: derivatives along the trajectory; C = c/1.5 - 4/3 |v|^2, c, e, w
// as in the acceleration kernels).  Per-block Dual sums of the cluster sums
// (blocks of kProThreads slots, spread over every SM).
__global__ void __launch_bounds__(kProThreads)
k_jerk_prologue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                const double *__restrict__ x, const double *__restrict__ v,
                const double *__restrict__ m, const double *__restrict__ a,
                double4_32a *__restrict__ rec, double *__restrict__ blk)
// a == nullptr: values only (all derivatives zero), for the adjoint
{
    __shared__ double sh[2 * kJVals][kProThreads];
    const int64_t t = (int64_t)blockIdx.x * kProThreads + threadIdx.x;
    const Clu C = clu[cluster_of_block(blk_clu, (int64_t)blockIdx.x * kProThreads / kGlueThreads)];
    const int64_t lt = t - C.slot0;
    double g[2 * kJVals];
#pragma unroll
    for (int k = 0; k < 2 * kJVals; ++k)
        g[k] = 0.0;
    if (lt < C.ns) {
        const int64_t j = C.body0 + 1 + lt, h = C.body0;
        const double GM = C.G * m[h], mj = m[j];
        Dual d[3], vel[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = dual(x[3 * j + k] - x[3 * h + k], a ? v[3 * j + k] - v[3 * h + k] : 0.0);
            vel[k] = dual(v[3 * j + k], a ? a[3 * j + k] : 0.0);
        }
        const Dual R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const Dual iR = 1.0 / tsqrt(R2);
        const Dual iR3 = iR * iR * iR;
        const Dual c = GM * (1.5 * iR + 0.25 * C.eps2 * iR3);
        const Dual Cc = c / 1.5 - (4.0 / 3.0) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
        const Dual ne = -(0.5 * GM / 1.5) * iR3;     // -e/1.5 = ne d
        Dual e3[3], w[3];
        for (int k = 0; k < 3; ++k) {
            e3[k] = ne * d[k];
            w[k] = mj * iR3 * d[k];
        }
        rec[t] = make_double4_32a(d[0].v, d[1].v, d[2].v, mj);
        rec[S + t] = make_double4_32a(d[0].d, d[1].d, d[2].d, 0.0);
        rec[2 * S + t] = make_double4_32a(vel[0].v, vel[1].v, vel[2].v, R2.v);
        rec[3 * S + t] = make_double4_32a(vel[0].d, vel[1].d, vel[2].d, R2.d);
        rec[4 * S + t] = make_double4_32a(e3[0].v, e3[1].v, e3[2].v, Cc.v);
        rec[5 * S + t] = make_double4_32a(e3[0].d, e3[1].d, e3[2].d, Cc.d);
        rec[6 * S + t] = make_double4_32a(w[0].v, w[1].v, w[2].v, 0.0);
        rec[7 * S + t] = make_double4_32a(w[0].d, w[1].d, w[2].d, 0.0);
        Dual q[kJVals];
        for (int k = 0; k < 3; ++k) {
            q[k] = mj * vel[k];
            q[3 + k] = w[k];
            q[6 + k] = w[k];
        }
        q[9] = 1.25 * mj * iR;
        q[10] = 0.25 * mj * (R2 + C.eps2) * iR3;
        q[11] = mj * iR;
        for (int k = 0; k < kJVals; ++k) {
            g[2 * k] = q[k].v;
            g[2 * k + 1] = q[k].d;
        }
    } else {
        const double px = 1.0e4 + (double)(lt - C.ns);
        rec[t] = make_double4_32a(px, 0.0, 0.0, 0.0);
        for (int k = 1; k < kJRec; ++k)
            rec[k * S + t] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    block_sum<2 * kJVals, kProThreads>(g, sh);
    if (threadIdx.x < 2 * kJVals)
        blk[(int64_t)blockIdx.x * 2 * kJVals + threadIdx.x] = sh[threadIdx.x][0];
}

// One block per cluster: its Dual cluster sums, blocks in a fixed order.
__global__ void __launch_bounds__(kGlueThreads)
k_jerk_globals(const Clu *__restrict__ clu, const double *__restrict__ blk,
               double *__restrict__ glob)
{
    __shared__ double sh[2 * kJVals][kGlueThreads];
    const Clu C = clu[blockIdx.x];
    sum_blocks<2 * kJVals>(blk + (C.slot0 / kProThreads) * 2 * kJVals,
                           C.ns_pad / kProThreads, sh);
    if (threadIdx.x < 2 * kJVals)
        glob[(int64_t)blockIdx.x * 2 * kJVals + threadIdx.x] = sh[threadIdx.x][0];
}

template <class T>
__device__ __forceinline__ T mk(double v, double d);
template <>
__device__ __forceinline__ double mk<double>(double v, double) { return v; }
template <>
__device__ __forceinline__ Dual mk<Dual>(double v, double d) { return {v, d}; }

__device__ __forceinline__ double rsq(double s2) { return 1.0 / sqrt(s2); }
__device__ __forceinline__ Dual rsq(Dual s2)
{
    const double y = 1.0 / sqrt(s2.v);
    return {y, -0.5 * y * y * y * s2.d};
}

// Pair sums of passes 1 and 2 (the 16 sums of the fused kernels), in double
// (T = double: the adjoint's forward sums) or on Duals (the jerk), one target
// per thread; grid (target blocks, source splits), split s of a target block
// in cluster k sweeping tiles [s tps, (s+1) tps).  Output
// part[split][value][slot] (double) or part[split][2 value + {0 value,
// 1 derivative}][slot] (Dual).
template <class T>
__global__ void __launch_bounds__(kJThreads)
k_dual_pairs(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
             const int *__restrict__ blk_clu, double *__restrict__ part)
{
    constexpr bool kDual = sizeof(T) == sizeof(Dual);
    __shared__ double4_32a sh[kJRec][kJTile];
    const int64_t t0 = (int64_t)blockIdx.x * kJThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int ntiles = (int)(C.ns_pad / kJTile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int64_t ti = t0 + threadIdx.x;
    const double4_32a T0 = rec[ti], T1 = rec[S + ti], T2 = rec[2 * S + ti], T3 = rec[3 * S + ti];
    const T di[3] = {mk<T>(T0.x, T1.x), mk<T>(T0.y, T1.y), mk<T>(T0.z, T1.z)};
    const T vi[3] = {mk<T>(8.0 / 3.0 * T2.x, 8.0 / 3.0 * T3.x),
                     mk<T>(8.0 / 3.0 * T2.y, 8.0 / 3.0 * T3.y),
                     mk<T>(8.0 / 3.0 * T2.z, 8.0 / 3.0 * T3.z)};
    T acc[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        acc[k] = mk<T>(0.0, 0.0);
    const double eps2 = C.eps2;
    const int tb = blockIdx.y * tps;
    const int te = min(ntiles, tb + tps);
    for (int tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + (int64_t)tile * kJTile;
        __syncthreads();
        for (int q = threadIdx.x; q < kJRec * kJTile; q += kJThreads)
            sh[q / kJTile][q % kJTile] = rec[(q / kJTile) * S + j0 + q % kJTile];
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < kJTile; ++q) {
            if (j0 + q == ti)
                continue;
            const double4_32a A0 = sh[0][q], A1 = sh[1][q], A2 = sh[2][q], A3 = sh[3][q];
            const double4_32a A4 = sh[4][q], A5 = sh[5][q], A6 = sh[6][q], A7 = sh[7][q];
            const T xx[3] = {di[0] - mk<T>(A0.x, A1.x), di[1] - mk<T>(A0.y, A1.y),
                             di[2] - mk<T>(A0.z, A1.z)};
            const T vj[3] = {mk<T>(A2.x, A3.x), mk<T>(A2.y, A3.y), mk<T>(A2.z, A3.z)};
            const T s2 = xx[0] * xx[0] + xx[1] * xx[1] + xx[2] * xx[2] + eps2;
            const T is = rsq(s2);
            const T is2 = is * is;
            const T mis = A0.w * is;
            const T mis3 = mis * is2;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[k] += mis3 * xx[k];
            acc[3] += mis;
            acc[4] += mis3;
            acc[5] += mis3 * mk<T>(A2.w, A3.w);
            const T xvj = xx[0] * vj[0] + xx[1] * vj[1] + xx[2] * vj[2];
            const T xvi = xx[0] * vi[0] + xx[1] * vi[1] + xx[2] * vi[2];
            const T kk = mk<T>(A4.w, A5.w) + (vi[0] * vj[0] + vi[1] * vj[1] + vi[2] * vj[2]) +
                         (mk<T>(A4.x, A5.x) * di[0] + mk<T>(A4.y, A5.y) * di[1] +
                          mk<T>(A4.z, A5.z) * di[2]);
            const T f = mis3 * (xvj * is2 * xvj + kk);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[6 + k] += f * xx[k];
            const T gg = mis3 * (xvi - 2.0 * xvj);
            acc[9] += gg;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[10 + k] += gg * vj[k];
            acc[13] += mk<T>(A6.x, A7.x) * is;
            acc[14] += mk<T>(A6.y, A7.y) * is;
            acc[15] += mk<T>(A6.z, A7.z) * is;
        }
    }
    if constexpr (kDual) {
        double *out = part + (int64_t)blockIdx.y * 2 * kFusedVals * S;
#pragma unroll
        for (int k = 0; k < kFusedVals; ++k) {
            const Dual &r = reinterpret_cast<const Dual &>(acc[k]);
            out[(int64_t)(2 * k) * S + ti] = r.v;
            out[(int64_t)(2 * k + 1) * S + ti] = r.d;
        }
    } else {
        double *out = part + (int64_t)blockIdx.y * kFusedVals * S;
#pragma unroll
        for (int k = 0; k < kFusedVals; ++k)
            out[(int64_t)k * S + ti] = reinterpret_cast<const double &>(acc[k]);
    }
}

// --------------------------------------------- jerk: single precision --
//
// The dual pair sums in FP32 for mixed-precision contexts (the jerk only
// enters Hermite's predictor and corrector with dt^2 and dt^3 weights, so
// single-precision pair terms are enough): value and derivative of every
// pair term, x_ij's value from hi/lo splits of the hole-relative positions,
// partials of kJPackFlush tiles added into FP64 outputs.  Same output layout
// as k_dual_pairs<Dual>.  Every arithmetic step is one f32x2 operation for
// two targets (t, t + 128 of a 256-target block) against one source, on
// duals P2 = (two values, two derivatives).  Staged source records, every
// field duplicated (f, f) and the position terms negated (16 float4 per slot):
//   S0 = (-hx, -hy)  S1 = (-hz, m)    S2 = (-lx, -ly)    S3 = (-lz, al)
//   S4 = (-d'x, -d'y) S5 = (-d'z, al')  S6 = (vx, vy)    S7 = (vz, K)
//   S8 = (ax, ay)    S9 = (az, K')   S10 = (Dx, Dy)     S11 = (Dz, D'x)
//   S12 = (D'y, D'z) S13 = (wx, wy)  S14 = (wz, w'x)    S15 = (w'y, w'z)
// (h, l = hi/lo split of d_j, primes: derivatives along the trajectory,
// a = v', D = -e_j/1.5, C = c_j/1.5 - 4/3 |v_j|^2.  Sources at least r_near
// from the hole take the hole term of kappa in the law-of-cosines form of
// the acceleration kernel: al = D.d_j / (2 R_j^2) = -G M / (6 R_j^3),
// K = C + al (R_j^2 + eps^2); nearer ones keep the D form, with al = 0 and
// K = C.  The Wr sum is left out, the epilogue restoring it.)  Tiles of kJPackTile
// sources move by bulk copies into two shared buffers as in the
// acceleration kernel.

constexpr int kJPackVals = 16;      // float4 per staged source
constexpr int kJPackTile = 64;      // sources per tile
constexpr int kJPackFlush = 8;      // tiles per single-precision partial
constexpr int kJPackTI = 2 * kMixThreads;   // targets per block
constexpr int kJPackBytes = kJPackTile * kJPackVals * 16;

__global__ void __launch_bounds__(kGlueThreads)
k_jerk_stage(int64_t S, const double4_32a *__restrict__ rec, float4 *__restrict__ srec,
             const Clu *__restrict__ clu, const int *__restrict__ blk_clu)
{
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (t >= S)
        return;
    const Clu Cl = clu[cluster_of_block(blk_clu, blockIdx.x)];
    const double4_32a J0 = rec[t], J1 = rec[S + t], J2 = rec[2 * S + t], J3 = rec[3 * S + t];
    const double4_32a J4 = rec[4 * S + t], J5 = rec[5 * S + t], J6 = rec[6 * S + t],
                      J7 = rec[7 * S + t];
    const float h0 = (float)J0.x, h1 = (float)J0.y, h2 = (float)J0.z;
    const float l0 = (float)(J0.x - (double)h0), l1 = (float)(J0.y - (double)h1),
                l2 = (float)(J0.z - (double)h2);
    auto dup = [](double a, double b) {
        return make_float4((float)a, (float)a, (float)b, (float)b);
    };
    float4 *o = srec + t * kJPackVals;
    o[0] = make_float4(-h0, -h0, -h1, -h1);
    o[1] = make_float4(-h2, -h2, (float)J0.w, (float)J0.w);
    // far sources (R_j >= r_near): the law-of-cosines form of the hole term,
    // D_j.d_i = al (R_i^2 - r_ij^2) + al (R_j^2 + eps^2) with al = D_j.d_j /
    // (2 R_j^2), on duals; near sources keep the D form (al = 0 marks them)
    const double R2 = J2.w, R2p = J3.w;
    double al = 0.0, alp = 0.0, K = J4.w, Kp = J5.w;
    if (Cl.r_near > 0.0 && R2 >= Cl.r_near * Cl.r_near) {
        const double Dd = J4.x * J0.x + J4.y * J0.y + J4.z * J0.z;
        const double Dpd = J5.x * J0.x + J5.y * J0.y + J5.z * J0.z;
        const double Ddp = J4.x * J1.x + J4.y * J1.y + J4.z * J1.z;
        al = Dd / (2.0 * R2);
        alp = (Dpd + Ddp) / (2.0 * R2) - al * R2p / R2;
        const double s = R2 + Cl.eps2;
        K = J4.w + al * s;
        Kp = J5.w + alp * s + al * R2p;
    }
    o[2] = make_float4(-l0, -l0, -l1, -l1);
    o[3] = make_float4(-l2, -l2, (float)al, (float)al);
    o[4] = dup(-J1.x, -J1.y);
    o[5] = dup(-J1.z, alp);
    o[6] = dup(J2.x, J2.y);
    o[7] = dup(J2.z, K);
    o[8] = dup(J3.x, J3.y);
    o[9] = dup(J3.z, Kp);
    o[10] = dup(J4.x, J4.y);
    o[11] = dup(J4.z, J5.x);
    o[12] = dup(J5.y, J5.z);
    o[13] = dup(J6.x, J6.y);
    o[14] = dup(J6.z, J7.x);
    o[15] = dup(J7.y, J7.z);
}

struct P2 {
    float2 v, d;     // values and derivatives of two targets' duals
};

// acc += a b on duals (3 packed operations)
__device__ __forceinline__ void p2_acc(P2 &acc, const P2 &a, const P2 &b)
{
    acc.v = fma2(a.v, b.v, acc.v);
    acc.d = fma2(a.d, b.v, fma2(a.v, b.d, acc.d));
}

__device__ __forceinline__ P2 p2_mul(const P2 &a, const P2 &b)
{
    return {mul2(a.v, b.v), fma2(a.d, b.v, mul2(a.v, b.d))};
}

struct JTarget {
    float2 hx, hy, hz, lx, ly, lz;   // hi/lo split of d_i
    float2 dx, dy, dz;               // d_i'
    float2 vx, vy, vz, ax, ay, az;   // 8/3 v_i, 8/3 a_i
    float2 rr, rrp;                  // R_i^2 and its derivative
};

template <bool MASK>
__device__ __forceinline__ void jerk_pair(const JTarget &tg, const float4 *__restrict__ sq,
                                          float2 eps2, bool selfx, bool selfy, P2 (&acc)[kFusedVals])
{
    const float4 S0 = sq[0], S1 = sq[1], S2 = sq[2], S3 = sq[3], S4 = sq[4], S5 = sq[5];
    const P2 x = {add2(add2(tg.hx, lo2(S0)), add2(tg.lx, lo2(S2))), add2(tg.dx, lo2(S4))};
    const P2 y = {add2(add2(tg.hy, hi2(S0)), add2(tg.ly, hi2(S2))), add2(tg.dy, hi2(S4))};
    const P2 z = {add2(add2(tg.hz, lo2(S1)), add2(tg.lz, lo2(S3))), add2(tg.dz, lo2(S5))};
    float2 s2 = fma2(x.v, x.v, fma2(y.v, y.v, fma2(z.v, z.v, eps2)));
    float2 m = hi2(S1);
    const float4 S13 = sq[13], S14 = sq[14], S15 = sq[15];
    P2 wx = {lo2(S13), hi2(S14)}, wy = {hi2(S13), lo2(S15)}, wz = {lo2(S14), hi2(S15)};
    if (MASK) {
        if (selfx) {
            s2.x = 1.0f; m.x = 0.0f;
            wx.v.x = wy.v.x = wz.v.x = wx.d.x = wy.d.x = wz.d.x = 0.0f;
        }
        if (selfy) {
            s2.y = 1.0f; m.y = 0.0f;
            wx.v.y = wy.v.y = wz.v.y = wx.d.y = wy.d.y = wz.d.y = 0.0f;
        }
    }
    // r^-1 = y, (r^-1)' = -y^3 q, (r^-3)' = -3 y^5 q with q = x . x'
    const float2 q = fma2(x.v, x.d, fma2(y.v, y.d, mul2(z.v, z.d)));
    const float2 yy = make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y));
    const float2 y2 = mul2(yy, yy);
    const float2 nq = mul2(q, make_float2(-1.0f, -1.0f));
    const P2 is = {yy, mul2(mul2(y2, yy), nq)};
    const P2 is2 = {y2, mul2(mul2(yy, is.d), make_float2(2.0f, 2.0f))};
    const P2 mis = {mul2(m, yy), mul2(m, is.d)};
    const float2 my3 = mul2(mis.v, y2);
    const P2 mis3 = {my3, mul2(mul2(my3, mul2(y2, nq)), make_float2(3.0f, 3.0f))};
    p2_acc(acc[0], mis3, x);
    p2_acc(acc[1], mis3, y);
    p2_acc(acc[2], mis3, z);
    acc[3].v = add2(acc[3].v, mis.v);
    acc[3].d = add2(acc[3].d, mis.d);
    acc[4].v = add2(acc[4].v, mis3.v);
    acc[4].d = add2(acc[4].d, mis3.d);
    // acc[5] (Wr and its derivative) is not summed: k_jerk_epilogue restores
    // it from N, U and Z by the identity of the acceleration path
    const float4 S6 = sq[6], S7 = sq[7], S8 = sq[8], S9 = sq[9];
    const P2 vjx = {lo2(S6), lo2(S8)}, vjy = {hi2(S6), hi2(S8)}, vjz = {lo2(S7), lo2(S9)};
    // x . v_j, x . (8/3) v_i
    P2 xvj = p2_mul(x, vjx);
    p2_acc(xvj, y, vjy);
    p2_acc(xvj, z, vjz);
    P2 xvi = p2_mul(x, P2{tg.vx, tg.ax});
    p2_acc(xvi, y, P2{tg.vy, tg.ay});
    p2_acc(xvi, z, P2{tg.vz, tg.az});
    // kk = C_j + (8/3) v_i . v_j + D_j . h_i; far sources (al != 0, the same
    // for every lane) take D_j . d_i = al (R_i^2 - r_ij^2) + (K - C)
    const float2 al = hi2(S3);
    P2 kk;
    if (al.x != 0.0f) {
        const float2 alp = hi2(S5);
        const float2 tt = fma2(s2, make_float2(-1.0f, -1.0f), tg.rr);
        kk = P2{fma2(al, tt, hi2(S7)),
                fma2(alp, tt, fma2(al, fma2(q, make_float2(-2.0f, -2.0f), tg.rrp), hi2(S9)))};
    } else {
        const float4 S10 = sq[10], S11 = sq[11], S12 = sq[12];
        kk = P2{hi2(S7), hi2(S9)};
        p2_acc(kk, P2{lo2(S10), hi2(S11)}, P2{tg.hx, tg.dx});
        p2_acc(kk, P2{hi2(S10), lo2(S12)}, P2{tg.hy, tg.dy});
        p2_acc(kk, P2{lo2(S11), hi2(S12)}, P2{tg.hz, tg.dz});
    }
    p2_acc(kk, P2{tg.vx, tg.ax}, vjx);
    p2_acc(kk, P2{tg.vy, tg.ay}, vjy);
    p2_acc(kk, P2{tg.vz, tg.az}, vjz);
    const P2 h = p2_mul(xvj, is2);
    p2_acc(kk, h, xvj);
    const P2 f = p2_mul(mis3, kk);
    p2_acc(acc[6], f, x);
    p2_acc(acc[7], f, y);
    p2_acc(acc[8], f, z);
    const float2 m2 = make_float2(-2.0f, -2.0f);
    const P2 u = {fma2(m2, xvj.v, xvi.v), fma2(m2, xvj.d, xvi.d)};
    const P2 gg = p2_mul(mis3, u);
    acc[9].v = add2(acc[9].v, gg.v);
    acc[9].d = add2(acc[9].d, gg.d);
    p2_acc(acc[10], gg, vjx);
    p2_acc(acc[11], gg, vjy);
    p2_acc(acc[12], gg, vjz);
    p2_acc(acc[13], wx, is);
    p2_acc(acc[14], wy, is);
    p2_acc(acc[15], wz, is);
}

// One output value of a target: first flush writes, later ones add.
__device__ __forceinline__ void jerk_out(double *o, float p, bool first)
{
    *o = first ? (double)p : *o + (double)p;
}

// Grid (target blocks of 256 slots, source splits); split s of a block in a
// cluster with T tiles sweeps tiles [s T / js, (s+1) T / js).  A copy that
// does not complete within the wait limit sets kFlagTimeout in `flag`.
// fpart != nullptr (the caller's splits hold at most kJPackFlush tiles, so a
// split's partial is one FP32 sum): the partials go to fpart as floats, same
// layout, for k_split_sum_f32.
__global__ void __launch_bounds__(kMixThreads, 3)
k_jerk_pairs_packed(const float4 *__restrict__ srec, int64_t S, const Clu *__restrict__ clu,
                    const int *__restrict__ blk_clu, int *__restrict__ flag,
                    double *__restrict__ part, float *__restrict__ fpart)
{
    __shared__ __align__(128) float4 sh[2][kJPackTile][kJPackVals];
    __shared__ __align__(8) uint64_t full[2];
    const int64_t t0 = (int64_t)blockIdx.x * kJPackTI;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / kJPackTile;
    const int64_t js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    double *out = part + sp * 2 * kFusedVals * S;
    float *fout = fpart ? fpart + sp * 2 * kFusedVals * S : nullptr;
    const int64_t ta = t0 + threadIdx.x, tq = ta + kMixThreads;
    if (te <= tb) {               // an empty split still owns its outputs
        for (int k = 0; k < 2 * kFusedVals; ++k) {
            if (fout) {
                fout[k * S + ta] = 0.0f;
                fout[k * S + tq] = 0.0f;
            } else {
                out[k * S + ta] = 0.0;
                out[k * S + tq] = 0.0;
            }
        }
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_load(sh[0], srec + (C.slot0 + tb * kJPackTile) * kJPackVals, kJPackBytes, &full[0], 0);
        if (tb + 1 < te)
            bulk_load(sh[1], srec + (C.slot0 + (tb + 1) * kJPackTile) * kJPackVals, kJPackBytes,
                      &full[1], 0);
    }
    JTarget tg;
    {
        const float4 *ra = srec + ta * kJPackVals, *rb = srec + tq * kJPackVals;
        const float4 A0 = ra[0], A1 = ra[1], A2 = ra[2], A3 = ra[3], A4 = ra[4], A5 = ra[5];
        const float4 A6 = ra[6], A7 = ra[7], A8 = ra[8], A9 = ra[9];
        const float4 B0 = rb[0], B1 = rb[1], B2 = rb[2], B3 = rb[3], B4 = rb[4], B5 = rb[5];
        const float4 B6 = rb[6], B7 = rb[7], B8 = rb[8], B9 = rb[9];
        const float e3 = 8.0f / 3.0f;
        tg.hx = make_float2(-A0.x, -B0.x);
        tg.hy = make_float2(-A0.z, -B0.z);
        tg.hz = make_float2(-A1.x, -B1.x);
        tg.lx = make_float2(-A2.x, -B2.x);
        tg.ly = make_float2(-A2.z, -B2.z);
        tg.lz = make_float2(-A3.x, -B3.x);
        tg.dx = make_float2(-A4.x, -B4.x);
        tg.dy = make_float2(-A4.z, -B4.z);
        tg.dz = make_float2(-A5.x, -B5.x);
        tg.vx = make_float2(e3 * A6.x, e3 * B6.x);
        tg.vy = make_float2(e3 * A6.z, e3 * B6.z);
        tg.vz = make_float2(e3 * A7.x, e3 * B7.x);
        tg.ax = make_float2(e3 * A8.x, e3 * B8.x);
        tg.ay = make_float2(e3 * A8.z, e3 * B8.z);
        tg.az = make_float2(e3 * A9.x, e3 * B9.x);
        tg.rr = fma2(tg.hx, tg.hx, fma2(tg.hy, tg.hy, mul2(tg.hz, tg.hz)));
        tg.rrp = mul2(make_float2(2.0f, 2.0f),
                      fma2(tg.hx, tg.dx, fma2(tg.hy, tg.dy, mul2(tg.hz, tg.dz))));
    }
    const float e2 = (float)C.eps2;
    const float2 eps2 = make_float2(e2, e2);
    P2 acc[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        acc[k] = P2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    bool first = true;
    for (int64_t tile = tb; tile < te; ++tile) {
        const int b = (int)((tile - tb) & 1);
        const bool ok = mbar_wait(&full[b], (unsigned)(((tile - tb) >> 1) & 1));
        const int64_t j0 = C.slot0 + tile * kJPackTile;
        const bool diag = (j0 < t0 + kJPackTI) && (t0 < j0 + kJPackTile);
        if (diag) {
#pragma unroll 1
            for (int q = 0; q < kJPackTile; ++q)
                jerk_pair<true>(tg, sh[b][q], eps2, j0 + q == ta, j0 + q == tq, acc);
        } else {
#pragma unroll 2
            for (int q = 0; q < kJPackTile; ++q)
                jerk_pair<false>(tg, sh[b][q], eps2, false, false, acc);
        }
        if (((tile - tb + 1) % kJPackFlush) == 0 || tile + 1 == te) {
#pragma unroll
            for (int k = 0; k < kFusedVals; ++k) {
                if (fout) {            // the split's only flush
                    fout[(2 * k) * S + ta] = acc[k].v.x;
                    fout[(2 * k) * S + tq] = acc[k].v.y;
                    fout[(2 * k + 1) * S + ta] = acc[k].d.x;
                    fout[(2 * k + 1) * S + tq] = acc[k].d.y;
                } else {
                    jerk_out(out + (2 * k) * S + ta, acc[k].v.x, first);
                    jerk_out(out + (2 * k) * S + tq, acc[k].v.y, first);
                    jerk_out(out + (2 * k + 1) * S + ta, acc[k].d.x, first);
                    jerk_out(out + (2 * k + 1) * S + tq, acc[k].d.y, first);
                }
                acc[k] = P2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
            }
            first = false;
        }
        if (__syncthreads_or(!ok)) {     // every warp is done with buffer b
            if (threadIdx.x == 0) {
                atomicOr(flag, kFlagTimeout);
                if (tile + 1 < te)
                    mbar_wait(&full[b ^ 1], (unsigned)(((tile - tb + 1) >> 1) & 1));
            }
            return;
        }
        if (threadIdx.x == 0 && tile + 2 < te)
            bulk_load(sh[b], srec + (C.slot0 + (tile + 2) * kJPackTile) * kJPackVals, kJPackBytes,
                      &full[b], 0);
    }
}

// Per star: the split partials summed, star_eqs on Duals; the value is the
// acceleration and the derivative the jerk.  Per-block sums of the hole's
// terms (3 values, 3 derivatives) go to blk, one row per kProThreads slots.
__global__ void __launch_bounds__(kProThreads)
k_jerk_epilogue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                const double *__restrict__ x, const double *__restrict__ v,
                const double *__restrict__ m, const double *__restrict__ a,
                const double *__restrict__ part, int js, const double *__restrict__ globs,
                double *__restrict__ jerk, int *flag, unsigned long long *flag_step,
                unsigned long long step, double *__restrict__ blk, int wr_identity)
{
    __shared__ double sh[6][kProThreads];
    const int64_t t = (int64_t)blockIdx.x * kProThreads + threadIdx.x;
    const int k_clu = cluster_of_block(blk_clu, (int64_t)blockIdx.x * kProThreads / kGlueThreads);
    const Clu Cl = clu[k_clu];
    const double *glob = globs + (int64_t)k_clu * 2 * kJVals;
    const int64_t lt = t - Cl.slot0;
    double bh6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (lt < Cl.ns) {
        const int64_t i = Cl.body0 + 1 + lt, hb = Cl.body0;
        Dual d[3], vv[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = dual(x[3 * i + k] - x[3 * hb + k], v[3 * i + k] - v[3 * hb + k]);
            vv[k] = dual(v[3 * i + k], a[3 * i + k]);
        }
        // splits in order for every value; the 32 loads of one split are
        // independent, so they are in flight together
        double sv[2 * kFusedVals];
        for (int k = 0; k < 2 * kFusedVals; ++k)
            sv[k] = 0.0;
        for (int q = 0; q < js; ++q)
#pragma unroll
            for (int k = 0; k < 2 * kFusedVals; ++k)
                sv[k] += part[((int64_t)q * 2 * kFusedVals + k) * S + t];
        Dual s[kFusedVals];
        for (int k = 0; k < kFusedVals; ++k)
            s[k] = dual(sv[2 * k], sv[2 * k + 1]);
        StarSums<Dual> ss;
        for (int k = 0; k < 3; ++k) {
            ss.N[k] = s[k];
            ss.Vp[k] = s[6 + k];
            ss.Hv[k] = s[10 + k];
            ss.E[k] = s[13 + k];
            ss.P[k] = dual(0.0, 0.0);
            ss.Ee[k] = dual(0.0, 0.0);
        }
        ss.U = s[3];
        ss.Z = s[4];
        ss.Wr = s[5];
        if (wr_identity) {
            // the pair kernel left Wr out: R_j^2 = R_i^2 - 2 d_i.x_ij + r_ij^2 - eps^2
            // gives Wr = sum_j m_j R_j^2 / r_ij^3 = (R_i^2 - eps^2) Z - 2 d_i.N + U,
            // here on Duals (the value and its derivative along the trajectory)
            const Dual R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            ss.Wr = (R2 - Cl.eps2) * ss.Z - 2.0 * (d[0] * ss.N[0] + d[1] * ss.N[1] + d[2] * ss.N[2]) +
                    ss.U;
        }
        ss.Hs = s[9];
        ClusterSums<Dual> gs;
        for (int k = 0; k < 3; ++k) {
            gs.Q[k] = dual(glob[2 * k], glob[2 * k + 1]);
            gs.Wf[k] = dual(glob[2 * (6 + k)], glob[2 * (6 + k) + 1]);
        }
        gs.SA = dual(glob[18], glob[19]);
        gs.SB = dual(glob[20], glob[21]);
        gs.Phi = dual(glob[22], glob[23]);
        Dual ai[3], bh[3];
        star_eqs<Dual, double>(Cl.G, m[hb], m[i], Cl.eps2, Cl.inv_c2, 1.0, d, vv, ss, gs, ai, bh);
        const double ji[3] = {ai[0].d, ai[1].d, ai[2].d};
        flag_nonfinite(ji, flag, flag_step, step);
        for (int k = 0; k < 3; ++k) {
            jerk[3 * i + k] = ai[k].d;
            bh6[k] = bh[k].v;
            bh6[3 + k] = bh[k].d;
        }
    }
    block_sum<6, kProThreads>(bh6, sh);
    if (threadIdx.x < 6)
        blk[(int64_t)blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// The hole of each cluster: jerk = d/dt [G W + (1/c^2) sum_j (star j's term)].
__global__ void __launch_bounds__(kGlueThreads)
k_jerk_hole(const Clu *__restrict__ clu, const double *__restrict__ blk,
            const double *__restrict__ globs, double *__restrict__ jerk, int *flag,
            unsigned long long *flag_step, unsigned long long step)
{
    __shared__ double sh[6][kGlueThreads];
    const Clu C = clu[blockIdx.x];
    sum_blocks<6>(blk + (C.slot0 / kProThreads) * 6, C.ns_pad / kProThreads, sh);
    if (threadIdx.x == 0) {
        const double *glob = globs + (int64_t)blockIdx.x * 2 * kJVals;
        double j0[3];
        for (int k = 0; k < 3; ++k)
            j0[k] = C.G * glob[2 * (3 + k) + 1] + C.inv_c2 * sh[3 + k][0];
        flag_nonfinite(j0, flag, flag_step, step);
        for (int k = 0; k < 3; ++k)
            jerk[3 * C.body0 + k] = j0[k];
    }
}

// Hermite stages on all 3n coordinates (body = coordinate / 3):
//   0 predict  xe = x + dt v + dt^2/2 a + dt^3/6 j,  ve = v + dt a + dt^2/2 j
//   1 correct  ve = v + dt/2 (a + a1) + dt^2/12 (j - j1),
//              xe = x + dt/2 (v + ve) + dt^2/12 (a - a1)
//   2 commit   x = xe, v = ve, a = a1, j = j1
__global__ void __launch_bounds__(kGlueThreads)
k_hermite(int stage, int64_t n3, double *__restrict__ x, double *__restrict__ v,
          double *__restrict__ a, double *__restrict__ j, const double *__restrict__ a1,
          const double *__restrict__ j1, double *__restrict__ xe, double *__restrict__ ve,
          double dt)
{
    const double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (stage == 0) {
            xe[q] = x[q] + dt * v[q] + dt2 / 2.0 * a[q] + dt3 / 6.0 * j[q];
            ve[q] = v[q] + dt * a[q] + dt2 / 2.0 * j[q];
        } else if (stage == 1) {
            const double vn = v[q] + dt / 2.0 * (a[q] + a1[q]) + dt2 / 12.0 * (j[q] - j1[q]);
            ve[q] = vn;
            xe[q] = x[q] + dt / 2.0 * (v[q] + vn) + dt2 / 12.0 * (a[q] - a1[q]);
        } else {
            x[q] = xe[q];
            v[q] = ve[q];
            a[q] = a1[q];
            j[q] = j1[q];
        }
    }
}

// ------------------------------------------------------------ adjoint --
//
// Vector-Jacobian product of A: given a cotangent abar (n x 3) of the
// accelerations, the cotangents of the positions, of the velocities at which
// A is taken, of the hole mass M and of inv_c2 = 1/c^2.  Reverse mode over
// the same decomposition, in double precision, without the near-source
// split (far form throughout):
//   star assembly (star_eqs): hand-derived reverse for the inputs that
//     enter nonlinearly (d_i, v_i, M), closed forms for the sums that enter
//     linearly (per star, one thread, O(n));
//   pair sums: hand-derived reverse of the pair terms (below), one sweep
//     over sources per target and one over targets per source (O(n^2));
//   records and cluster sums: their gradient in (d_j, v_j, M) in closed
//     form, contracted with their cotangents (per star, one thread, O(n)).
//
// Pair terms (target i, source j), x = d_i - d_j, s^2 = |x|^2 + eps^2,
// is = 1/s, mis3 = m_j is^3, xvj = x.v_j, xvi = x.v'_i (v' = 8/3 v),
// k = C_j + v'_i.v_j + D_j.d_i (D = -e/1.5), F = xvj^2 is^2 + k,
// Gq = xvi - 2 xvj; with the sums' cotangents (Nb, Ub, Zb, Wrb, Vb, Hsb,
// Hvb, Eb) of target i the pair contributes
//   phi = mis3 (Nb.x + Zb + Wrb R_j^2) + Ub m_j is + mis3 F (Vb.x)
//       + mis3 Gq (Hsb + Hvb.v_j) + is (Eb.w_j).
// With P = Nb.x + Zb + Wrb R_j^2, Vx = Vb.x, Hb = Hsb + Hvb.v_j, Ew = Eb.w_j,
// B = P + F Vx + Gq Hb:
//   dphi/dx    = gx = cx x + mis3 [Nb + F Vb + Hb v'_i + (2 Vx xvj is^2 - 2 Hb) v_j],
//                cx = -3 mis3 is^2 B - 2 mis3 Vx xvj^2 is^4 - Ub mis3 - Ew is^3
//   dphi/dd_i  = gx + mis3 Vx D_j          dphi/dv'_i = mis3 (Hb x + Vx v_j)
//   dphi/dd_j  = -gx (through x)           dphi/dv_j  = mis3 [Vx (2 xvj is^2 x + v'_i)
//                                                       - 2 Hb x] + mis3 Gq Hvb
//   dphi/dR_j^2 = mis3 Wrb   dphi/dC_j = mis3 Vx   dphi/dD_j = mis3 Vx d_i
//   dphi/dw_j  = is Eb

constexpr int kAdjGlob = 11;      // Qb (3), Wfb (3), SAb, SBb, Phib, Mb, ic2b
constexpr int kAdjSrc = 14;       // source cotangents: d (3), v (3), R^2, C, D (3), w (3)

struct PairAdj {
    double x[3], is, is2, mis3, xvj, F, Gq, Vx, Hb, gx[3];
};

// The shared intermediate quantities and dphi/dx of one pair.
__device__ __forceinline__ void pair_adj(const double (&di)[3], const double (&vpi)[3],
                                         const double (&dj)[3], double mj, double R2j,
                                         const double (&vj)[3], double Cj, const double (&Dj)[3],
                                         const double (&wj)[3], double eps2,
                                         const double (&sb)[kFusedVals], PairAdj &p)
{
    for (int k = 0; k < 3; ++k)
        p.x[k] = di[k] - dj[k];
    const double s2 = p.x[0] * p.x[0] + p.x[1] * p.x[1] + p.x[2] * p.x[2] + eps2;
    p.is = 1.0 / sqrt(s2);
    p.is2 = p.is * p.is;
    p.mis3 = mj * p.is * p.is2;
    p.xvj = p.x[0] * vj[0] + p.x[1] * vj[1] + p.x[2] * vj[2];
    const double xvi = p.x[0] * vpi[0] + p.x[1] * vpi[1] + p.x[2] * vpi[2];
    const double kk = Cj + (vpi[0] * vj[0] + vpi[1] * vj[1] + vpi[2] * vj[2]) +
                      (Dj[0] * di[0] + Dj[1] * di[1] + Dj[2] * di[2]);
    p.F = p.xvj * p.xvj * p.is2 + kk;
    p.Gq = xvi - 2.0 * p.xvj;
    const double P = sb[0] * p.x[0] + sb[1] * p.x[1] + sb[2] * p.x[2] + sb[4] + sb[5] * R2j;
    p.Vx = sb[6] * p.x[0] + sb[7] * p.x[1] + sb[8] * p.x[2];
    p.Hb = sb[9] + sb[10] * vj[0] + sb[11] * vj[1] + sb[12] * vj[2];
    const double Ew = sb[13] * wj[0] + sb[14] * wj[1] + sb[15] * wj[2];
    const double B = P + p.F * p.Vx + p.Gq * p.Hb;
    const double cx = -3.0 * p.mis3 * p.is2 * B -
                      2.0 * p.mis3 * p.Vx * p.xvj * p.xvj * p.is2 * p.is2 - sb[3] * p.mis3 -
                      Ew * p.is * p.is2;
    const double cv = 2.0 * p.Vx * p.xvj * p.is2 - 2.0 * p.Hb;
    for (int k = 0; k < 3; ++k)
        p.gx[k] = cx * p.x[k] +
                  p.mis3 * (sb[k] + p.F * sb[6 + k] + p.Hb * vpi[k] + cv * vj[k]);
}

// Cotangents of the inputs that star_eqs uses linearly — the 16 pair sums
// (N, U, Z, Wr, V', Hs, Hv, E) and the cluster sums (Q, W_far, SA, SB, Phi)
// — contracted with ab (of a_i) and bb (of the hole's term, 1/c^2 included),
// in closed form: every coefficient depends on d_i, v_i and M only.  With
// al = ab/c^2 (the cotangent of the 1PN bracket), GM = G M, and the
// bracket's coefficients cN = G (4 GM/R - v^2), cQ = 4 G (v.d)/R^3,
// c7 = 7/2 G GM:
//   Nb = -G ab + cN al - 7/2 G^2 m_i/R bb       Ub = 4 G GM/R^3 (al.d) - 5/4 G^2 (bb.w_i)
//   Zb = -1/4 G^2 R^2 (bb.w_i)   Wrb = 1/4 G^2 (bb.w_i)   V'b = 3/2 G al
//   Hsb = 3/2 G (al.v)   Hvb = -3/2 G al   Eb = -c7 al
//   Qb = -4 G/R^3 (al.d) v + 3 G/R^3 (al.v) d + cQ al
//        + G m_i/(M R^3) [4 (bb.d) v - 3 (v.d) bb - 4 (bb.v) d]
//   Wfb = 1/2 G GM/R^3 (al.d) d + c7/R al    SAb = -SBb = G GM/R^3 (al.d)
//   Phib = -4 G^2 (bb.w_i)
// out: [0..15] the 16 sums' cotangents, [16..24] Q, W_far, SA, SB, Phi.
__device__ __forceinline__ void star_lin_adj(double G, double M, double mi, double inv_c2,
                                             const double (&d)[3], const double (&vv)[3],
                                             const double (&ab)[3], const double (&bb)[3],
                                             double (&out)[25])
{
    const double GM = G * M;
    const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double iR = 1.0 / sqrt(R2);
    const double iR3 = iR * iR * iR;
    const double v2 = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
    const double vd = vv[0] * d[0] + vv[1] * d[1] + vv[2] * d[2];
    double al[3], wi[3];
    for (int k = 0; k < 3; ++k) {
        al[k] = inv_c2 * ab[k];
        wi[k] = mi * iR3 * d[k];
    }
    const double ad = al[0] * d[0] + al[1] * d[1] + al[2] * d[2];
    const double av = al[0] * vv[0] + al[1] * vv[1] + al[2] * vv[2];
    const double bd = bb[0] * d[0] + bb[1] * d[1] + bb[2] * d[2];
    const double bv = bb[0] * vv[0] + bb[1] * vv[1] + bb[2] * vv[2];
    const double bw = bb[0] * wi[0] + bb[1] * wi[1] + bb[2] * wi[2];
    const double cN = G * (4.0 * GM * iR - v2), cQ = 4.0 * G * iR3 * vd, c7 = 3.5 * G * GM;
    const double G2 = G * G, gq = G * mi * iR3 / M, gs = G * GM * iR3 * ad;
    for (int k = 0; k < 3; ++k) {
        out[k] = -G * ab[k] + cN * al[k] - 3.5 * G2 * mi * iR * bb[k];     // N
        out[6 + k] = 1.5 * G * al[k];                                       // V'
        out[10 + k] = -1.5 * G * al[k];                                     // Hv
        out[13 + k] = -c7 * al[k];                                          // E
        out[16 + k] = -4.0 * G * iR3 * ad * vv[k] + 3.0 * G * iR3 * av * d[k] + cQ * al[k] +
                      gq * (4.0 * bd * vv[k] - 3.0 * vd * bb[k] - 4.0 * bv * d[k]);   // Q
        out[19 + k] = 0.5 * gs * d[k] + c7 * iR * al[k];                    // W_far
    }
    out[3] = 4.0 * gs - 1.25 * G2 * bw;          // U
    out[4] = -0.25 * G2 * R2 * bw;               // Z
    out[5] = 0.25 * G2 * bw;                     // Wr
    out[9] = 1.5 * G * av;                       // Hs
    out[22] = gs;                                // SA
    out[23] = -gs;                               // SB
    out[24] = -4.0 * G2 * bw;                    // Phi
}

// Reverse of star_eqs (T = double) for the inputs that enter it
// nonlinearly, d_i, v_i and M, the sums held fixed: with ab the cotangent
// of a_i and bb that of the star's term of the hole's acceleration (1/c^2
// included), the cotangents db, vb and Mb of ab.a_i + bb.bh_i, and the
// values ab.pn_i (pn: the 1PN bracket) and bh_i that the 1/c^2 cotangent
// takes.  Hand-derived, star_eqs' statements walked backwards: every
// intermediate q of the forward (iR, iR3, v2, vd, vQ, Qd, S, cd, cv, cN,
// cQ, c7, b1, gmr3, Wx, w_i, GM) gets its cotangent qb from the statements
// that read it, then passes it on to its own inputs.  With al = ic ab and
// gM = gmr3/M, X = 4 vQ (bb.d) - 3 vd (bb.Q) - 4 Qd (bb.v):
//   cdb = al.d  cvb = al.v  cNb = al.N  cQb = al.Q  c7b = iR (al.Wx) - al.E
//   Sb = G GM iR3 cdb   b1b = bb.w_i   gmr3b = -3 vd (bb.v) + X/M
// (b1's two m_i/R_i terms cancel, so it reads -G(...) - G^2 (4 Phi + ...)).
struct StarAdj {
    double db[3], vb[3], Mb, apn, bh[3];
};

__device__ __forceinline__ void star_vjp(double G, double M, double mi, double eps2, double ic,
                                         double fi, const double (&d)[3], const double (&vv)[3],
                                         const StarSums<double> &s, const ClusterSums<double> &g,
                                         const double (&ab)[3], const double (&bb)[3],
                                         StarAdj &o)
{
    auto dot = [](const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    const double GM = G * M, G2 = G * G;
    const double R2 = dot(d, d);
    const double iR = 1.0 / sqrt(R2), iR2 = iR * iR, iR3 = iR2 * iR;
    const double v2 = dot(vv, vv), vd = dot(vv, d);
    double wi[3], Wx[3], al[3], PE[3];
    for (int k = 0; k < 3; ++k) {
        wi[k] = mi * iR3 * d[k];
        Wx[k] = g.Wf[k] - fi * wi[k];
        al[k] = ic * ab[k];
        PE[k] = s.P[k] - 3.5 * s.Ee[k];
    }
    const double vQ = dot(vv, g.Q), Qd = dot(g.Q, d);
    const double S = 4.0 * s.U + (g.SA - fi * 1.25 * mi * iR) + 0.5 * dot(d, Wx) -
                     (g.SB - fi * 0.25 * mi * (R2 + eps2) * iR3);
    const double A = 4.0 * GM * iR - v2;
    const double cd = GM * iR3 * A + 5.0 * G * GM * mi * iR3 * iR + G * GM * iR3 * S -
                      4.0 * G * iR3 * vQ;
    const double cv = 4.0 * GM * iR3 * vd + 3.0 * G * iR3 * Qd;
    const double cN = G * A, cQ = 4.0 * G * iR3 * vd, c7 = 3.5 * G * GM;
    const double gmr3 = G * mi * iR3, gM = gmr3 / M;
    const double Y = R2 * s.Z - s.Wr;
    const double b1 = -G * (5.0 * GM * iR - 2.0 * v2 + 1.5 * vd * vd * iR2) -
                      4.0 * G2 * mi * iR - G2 * (4.0 * (g.Phi - mi * iR) + 1.25 * s.U + 0.25 * Y);
    // values: ab.pn and bh
    double apn = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double pn = cd * d[k] + cv * vv[k] + G * 1.5 * s.Vp[k] + cN * s.N[k] -
                          c7 * (s.E[k] - Wx[k] * iR) + cQ * g.Q[k] +
                          G * 1.5 * (s.Hs * vv[k] - s.Hv[k]) + G * GM * PE[k];
        apn += ab[k] * pn;
        o.bh[k] = b1 * wi[k] - 3.0 * gmr3 * vd * vv[k] - 3.5 * G2 * mi * iR * s.N[k] +
                  gM * (4.0 * vQ * d[k] - 3.0 * vd * g.Q[k] - 4.0 * Qd * vv[k]);
    }
    o.apn = apn;
    // reverse
    const double abd = dot(ab, d), ad = dot(al, d), av = dot(al, vv), aN = dot(al, s.N);
    const double aQ = dot(al, g.Q), aWx = dot(al, Wx), aE = dot(al, s.E), aPE = dot(al, PE);
    const double bw = dot(bb, wi), bv = dot(bb, vv), bd = dot(bb, d), bQ = dot(bb, g.Q);
    const double bN = dot(bb, s.N);
    const double X = 4.0 * vQ * bd - 3.0 * vd * bQ - 4.0 * Qd * bv;
    const double cdb = ad, cvb = av, cNb = aN, cQb = aQ, c7b = aWx * iR - aE;
    const double Sb = G * GM * iR3 * cdb, b1b = bw, gmr3b = -3.0 * vd * bv + X / M;
    const double GMb = -abd * iR3 + G * aPE + 3.5 * G * c7b + 4.0 * G * iR * cNb +
                       4.0 * iR3 * vd * cvb +
                       cdb * (iR3 * A + 4.0 * GM * iR3 * iR + 5.0 * G * mi * iR3 * iR +
                              G * iR3 * S) -
                       5.0 * G * iR * b1b;
    o.Mb = G * GMb - gM * X / M;
    double iR3b = -GM * abd + 4.0 * G * vd * cQb + (4.0 * GM * vd + 3.0 * G * Qd) * cvb +
                  cdb * (GM * A + 5.0 * G * GM * mi * iR + G * GM * S - 4.0 * G * vQ) +
                  G * mi * gmr3b + fi * 0.25 * mi * (R2 + eps2) * Sb;
    double iRb = c7 * aWx + 4.0 * G * GM * cNb + cdb * (4.0 * GM * GM * iR3 + 5.0 * G * GM * mi * iR3) -
                 3.5 * G2 * mi * bN - b1b * (5.0 * G * GM + 3.0 * G * vd * vd * iR) -
                 fi * 1.25 * mi * Sb;
    const double v2b = -G * cNb - cdb * GM * iR3 + 2.0 * G * b1b;
    const double vdb = 4.0 * G * iR3 * cQb + 4.0 * GM * iR3 * cvb - 3.0 * gmr3 * bv -
                       3.0 * gM * bQ - 3.0 * G * vd * iR2 * b1b;
    const double Qdb = 3.0 * G * iR3 * cvb - 4.0 * gM * bv;
    const double vQb = -4.0 * G * iR3 * cdb + 4.0 * gM * bd;
    double R2b = -0.25 * G2 * s.Z * b1b + fi * 0.25 * mi * iR3 * Sb;
    double wib[3];
    for (int k = 0; k < 3; ++k) {
        const double Wxb = c7 * iR * al[k] + 0.5 * Sb * d[k];
        wib[k] = b1 * bb[k] - fi * Wxb;
    }
    iR3b += mi * dot(wib, d);
    iRb += 3.0 * iR2 * iR3b;
    R2b -= 0.5 * iR3 * iRb;
    for (int k = 0; k < 3; ++k) {
        o.db[k] = -GM * iR3 * ab[k] + cd * al[k] + 0.5 * Sb * Wx[k] + 4.0 * gM * vQ * bb[k] +
                  mi * iR3 * wib[k] + g.Q[k] * Qdb + vv[k] * vdb + 2.0 * d[k] * R2b;
        o.vb[k] = (cv + 1.5 * G * s.Hs) * al[k] - (3.0 * gmr3 * vd + 4.0 * gM * Qd) * bb[k] +
                  g.Q[k] * vQb + d[k] * vdb + 2.0 * vv[k] * v2b;
    }
}

// Per star slot, one thread each: the assembly's reverse.  Inputs: the
// forward sums (part, split-major, double; the js splits added in order),
// the cluster sums (Dual layout, values used) and the cotangent abar.
// Outputs: the sums' cotangents sbar[16][slot], the direct cotangents of d_i
// and of the velocity kbar[6][slot], and per block of kAdjStarSlots slots the
// cotangents of the cluster sums, of M and of inv_c2 (kAdjGlob values, added
// in slot order): star_vjp for d_i, v_i and M, star_lin_adj for the sums
// that enter linearly, and for 1/c^2 ab_i.pn_i + abar_hole.bh_i (A is linear
// in 1/c^2; the hole's term carries 1/c^2 outside).
constexpr int kAdjStarSlots = 32;     // star slots (threads) per block

__global__ void __launch_bounds__(kAdjStarSlots)
k_adj_star(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
           const double *__restrict__ x, const double *__restrict__ v,
           const double *__restrict__ m, const double *__restrict__ part, int js,
           const double *__restrict__ globs, const double *__restrict__ abar,
           double *__restrict__ sbar, double *__restrict__ kbar, double *__restrict__ blk)
{
    __shared__ double sg[kAdjGlob][kAdjStarSlots];
    const int64_t t = (int64_t)blockIdx.x * kAdjStarSlots + threadIdx.x;
    const int k_clu = cluster_of_block(blk_clu, t / kGlueThreads);
    const Clu Cl = clu[k_clu];
    const int64_t lt = t - Cl.slot0;
    const bool star = lt < Cl.ns;
    if (star) {
        const double *glob = globs + (int64_t)k_clu * 2 * kJVals;
        const int64_t i = Cl.body0 + 1 + lt, hb = Cl.body0;
        double f[kFusedVals];
#pragma unroll
        for (int k = 0; k < kFusedVals; ++k) {
            double sv = 0.0;
            for (int q = 0; q < js; ++q)
                sv += part[((int64_t)q * kFusedVals + k) * S + t];
            f[k] = sv;
        }
        double d[3], vv[3], ab[3], bb[3];
        StarSums<double> ss;
        ClusterSums<double> gs;
        for (int k = 0; k < 3; ++k) {
            d[k] = x[3 * i + k] - x[3 * hb + k];
            vv[k] = v[3 * i + k];
            ab[k] = abar[3 * i + k];
            bb[k] = Cl.inv_c2 * abar[3 * hb + k];
            ss.N[k] = f[k];
            ss.Vp[k] = f[6 + k];
            ss.Hv[k] = f[10 + k];
            ss.E[k] = f[13 + k];
            ss.P[k] = 0.0;
            ss.Ee[k] = 0.0;
            gs.Q[k] = glob[2 * k];
            gs.Wf[k] = glob[2 * (6 + k)];     // W_far = W: far form
        }
        ss.U = f[3];
        ss.Z = f[4];
        ss.Wr = f[5];
        ss.Hs = f[9];
        gs.SA = glob[18];
        gs.SB = glob[20];
        gs.Phi = glob[22];
        const double M = m[hb];
        StarAdj o;
        star_vjp(Cl.G, M, m[i], Cl.eps2, Cl.inv_c2, 1.0, d, vv, ss, gs, ab, bb, o);
        double lin[25];
        star_lin_adj(Cl.G, M, m[i], Cl.inv_c2, d, vv, ab, bb, lin);
        for (int k = 0; k < kFusedVals; ++k)
            sbar[(int64_t)k * S + t] = lin[k];
        for (int k = 0; k < 3; ++k) {
            kbar[(int64_t)k * S + t] = o.db[k];
            kbar[(int64_t)(3 + k) * S + t] = o.vb[k];
        }
        for (int k = 0; k < 9; ++k)
            sg[k][threadIdx.x] = lin[16 + k];
        sg[9][threadIdx.x] = o.Mb;
        sg[10][threadIdx.x] = o.apn + (abar[3 * hb] * o.bh[0] + abar[3 * hb + 1] * o.bh[1] +
                                       abar[3 * hb + 2] * o.bh[2]);
    } else {
        for (int k = 0; k < kFusedVals; ++k)
            sbar[(int64_t)k * S + t] = 0.0;
        for (int k = 0; k < 6; ++k)
            kbar[(int64_t)k * S + t] = 0.0;
        for (int k = 0; k < kAdjGlob; ++k)
            sg[k][threadIdx.x] = 0.0;
    }
    __syncwarp();
    // per-block sums over the block's star slots, in slot order
    if (threadIdx.x < kAdjGlob) {
        double g = 0.0;
        for (int w2 = 0; w2 < kAdjStarSlots; ++w2)
            g += sg[threadIdx.x][w2];
        blk[(int64_t)blockIdx.x * kAdjGlob + threadIdx.x] = g;
    }
}

__global__ void __launch_bounds__(kGlueThreads)
k_adj_globals(const Clu *__restrict__ clu, const double *__restrict__ blk,
              double *__restrict__ gbar)
{
    __shared__ double sh[kAdjGlob][kGlueThreads];
    const Clu C = clu[blockIdx.x];
    sum_blocks<kAdjGlob>(blk + (C.slot0 / kAdjStarSlots) * kAdjGlob, C.ns_pad / kAdjStarSlots, sh);
    if (threadIdx.x < kAdjGlob)
        gbar[(int64_t)blockIdx.x * kAdjGlob + threadIdx.x] = sh[threadIdx.x][0];
}

// Reverse pair sweep over sources for each target i (one per thread):
// tpart[split][6][slot] = (dphi/dd_i (3), dphi/dv'_i (3)) summed over j.
__global__ void __launch_bounds__(kJThreads)
k_adj_targets(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
              const int *__restrict__ blk_clu, const double *__restrict__ sbar,
              double *__restrict__ tpart)
{
    __shared__ double4_32a sh[4][kJTile];
    const int64_t t0 = (int64_t)blockIdx.x * kJThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int ntiles = (int)(C.ns_pad / kJTile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int64_t ti = t0 + threadIdx.x;
    const double4_32a T0 = rec[ti], T2 = rec[2 * S + ti];
    const double di[3] = {T0.x, T0.y, T0.z};
    const double vpi[3] = {8.0 / 3.0 * T2.x, 8.0 / 3.0 * T2.y, 8.0 / 3.0 * T2.z};
    double sb[kFusedVals];
    for (int k = 0; k < kFusedVals; ++k)
        sb[k] = sbar[(int64_t)k * S + ti];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int tb = blockIdx.y * tps;
    const int te = min(ntiles, tb + tps);
    for (int tile = tb; tile < te; ++tile) {
        const int64_t j0 = C.slot0 + (int64_t)tile * kJTile;
        __syncthreads();
        for (int q = threadIdx.x; q < 4 * kJTile; q += kJThreads)
            sh[q / kJTile][q % kJTile] = rec[(2 * (q / kJTile)) * S + j0 + q % kJTile];
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < kJTile; ++q) {
            if (j0 + q == ti)
                continue;
            const double4_32a A0 = sh[0][q], A2 = sh[1][q], A4 = sh[2][q], A6 = sh[3][q];
            const double dj[3] = {A0.x, A0.y, A0.z}, vj[3] = {A2.x, A2.y, A2.z};
            const double Dj[3] = {A4.x, A4.y, A4.z}, wj[3] = {A6.x, A6.y, A6.z};
            PairAdj p;
            pair_adj(di, vpi, dj, A0.w, A2.w, vj, A4.w, Dj, wj, C.eps2, sb, p);
            for (int k = 0; k < 3; ++k) {
                acc[k] += p.gx[k] + p.mis3 * p.Vx * Dj[k];
                acc[3 + k] += p.mis3 * (p.Hb * p.x[k] + p.Vx * vj[k]);
            }
        }
    }
    double *out = tpart + (int64_t)blockIdx.y * 6 * S;
    for (int k = 0; k < 6; ++k)
        out[(int64_t)k * S + ti] = acc[k];
}

// Reverse pair sweep over targets for each source j (one per thread):
// spart[split][14][slot] = cotangents of its record (d via x, v, R^2, C, D, w).
__global__ void __launch_bounds__(kJThreads)
k_adj_sources(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
              const int *__restrict__ blk_clu, const double *__restrict__ sbar,
              double *__restrict__ spart)
{
    __shared__ double sd[kJTile][3], sv[kJTile][3], ssb[kJTile][kFusedVals];
    const int64_t t0 = (int64_t)blockIdx.x * kJThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int ntiles = (int)(C.ns_pad / kJTile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int64_t tj = t0 + threadIdx.x;
    const double4_32a A0 = rec[tj], A2 = rec[2 * S + tj], A4 = rec[4 * S + tj],
                      A6 = rec[6 * S + tj];
    const double dj[3] = {A0.x, A0.y, A0.z}, vj[3] = {A2.x, A2.y, A2.z};
    const double Dj[3] = {A4.x, A4.y, A4.z}, wj[3] = {A6.x, A6.y, A6.z};
    double acc[kAdjSrc];
    for (int k = 0; k < kAdjSrc; ++k)
        acc[k] = 0.0;
    const int tb = blockIdx.y * tps;
    const int te = min(ntiles, tb + tps);
    for (int tile = tb; tile < te; ++tile) {
        const int64_t i0 = C.slot0 + (int64_t)tile * kJTile;
        __syncthreads();
        for (int q = threadIdx.x; q < kJTile; q += kJThreads) {
            const double4_32a T0 = rec[i0 + q], T2 = rec[2 * S + i0 + q];
            sd[q][0] = T0.x;
            sd[q][1] = T0.y;
            sd[q][2] = T0.z;
            sv[q][0] = 8.0 / 3.0 * T2.x;
            sv[q][1] = 8.0 / 3.0 * T2.y;
            sv[q][2] = 8.0 / 3.0 * T2.z;
        }
        for (int q = threadIdx.x; q < kJTile * kFusedVals; q += kJThreads)
            ssb[q % kJTile][q / kJTile] = sbar[(int64_t)(q / kJTile) * S + i0 + q % kJTile];
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < kJTile; ++q) {
            if (i0 + q == tj)
                continue;
            const double di[3] = {sd[q][0], sd[q][1], sd[q][2]};
            const double vpi[3] = {sv[q][0], sv[q][1], sv[q][2]};
            double sb[kFusedVals];
            for (int k = 0; k < kFusedVals; ++k)
                sb[k] = ssb[q][k];
            PairAdj p;
            pair_adj(di, vpi, dj, A0.w, A2.w, vj, A4.w, Dj, wj, C.eps2, sb, p);
            const double gg = p.mis3 * p.Gq;
            for (int k = 0; k < 3; ++k) {
                acc[k] -= p.gx[k];
                acc[3 + k] += p.mis3 * (p.Vx * (2.0 * p.xvj * p.is2 * p.x[k] + vpi[k]) -
                                        2.0 * p.Hb * p.x[k]) + gg * sb[10 + k];
                acc[8 + k] += p.mis3 * p.Vx * di[k];
                acc[11 + k] += p.is * sb[13 + k];
            }
            acc[6] += p.mis3 * sb[5];
            acc[7] += p.mis3 * p.Vx;
        }
    }
    double *out = spart + (int64_t)blockIdx.y * kAdjSrc * S;
    for (int k = 0; k < kAdjSrc; ++k)
        out[(int64_t)k * S + tj] = acc[k];
}

// ------------------------------------------- adjoint: single precision --
//
// The two reverse pair sweeps in FP32 for mixed-precision contexts: the
// same pair terms (pair_adj) with x_ij formed from hi/lo splits of the
// hole-relative positions.  Records (float4, per slot, far form): A = (hi d, m),
// B = (lo d, R^2), C = (v, C), D = (-e/1.5, 0), E = (w, 0), made from the
// FP64 records; the forward pair kernel stages them.

// Mixed contexts: the adjoint's forward records straight in their
// single-precision form (rows of 5 float4: hi d and m; lo d and R^2; v and C;
// -e/1.5; w -- k_jerk_prologue's values, without its zero derivatives, hi/lo
// split), and the per-block cluster-sum values in k_jerk_prologue's layout
// (derivative entries zero) for k_jerk_globals.
__global__ void __launch_bounds__(kProThreads)
k_adj_prologue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
               const double *__restrict__ x, const double *__restrict__ v,
               const double *__restrict__ m, float4 *__restrict__ frec, double *__restrict__ blk)
{
    __shared__ double sh[2 * kJVals][kProThreads];
    const int64_t t = (int64_t)blockIdx.x * kProThreads + threadIdx.x;
    const Clu C = clu[cluster_of_block(blk_clu, (int64_t)blockIdx.x * kProThreads / kGlueThreads)];
    const int64_t lt = t - C.slot0;
    double g[2 * kJVals];
#pragma unroll
    for (int k = 0; k < 2 * kJVals; ++k)
        g[k] = 0.0;
    if (lt < C.ns) {
        const int64_t j = C.body0 + 1 + lt, h = C.body0;
        const double GM = C.G * m[h], mj = m[j];
        double d[3], vel[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = x[3 * j + k] - x[3 * h + k];
            vel[k] = v[3 * j + k];
        }
        const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double iR = 1.0 / sqrt(R2);
        const double iR3 = iR * iR * iR;
        const double c = GM * (1.5 * iR + 0.25 * C.eps2 * iR3);
        const double Cc = c / 1.5 - (4.0 / 3.0) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
        const double ne = -(0.5 * GM / 1.5) * iR3;
        double e3[3], w[3];
        for (int k = 0; k < 3; ++k) {
            e3[k] = ne * d[k];
            w[k] = mj * iR3 * d[k];
        }
        const float h0 = (float)d[0], h1 = (float)d[1], h2 = (float)d[2];
        frec[t] = make_float4(h0, h1, h2, (float)mj);
        frec[S + t] = make_float4((float)(d[0] - (double)h0), (float)(d[1] - (double)h1),
                                  (float)(d[2] - (double)h2), (float)R2);
        frec[2 * S + t] = make_float4((float)vel[0], (float)vel[1], (float)vel[2], (float)Cc);
        frec[3 * S + t] = make_float4((float)e3[0], (float)e3[1], (float)e3[2], 0.0f);
        frec[4 * S + t] = make_float4((float)w[0], (float)w[1], (float)w[2], 0.0f);
        for (int k = 0; k < 3; ++k) {
            g[2 * k] = mj * vel[k];
            g[2 * (3 + k)] = w[k];
            g[2 * (6 + k)] = w[k];
        }
        g[18] = 1.25 * mj * iR;
        g[20] = 0.25 * mj * (R2 + C.eps2) * iR3;
        g[22] = mj * iR;
    } else {
        const double px = 1.0e4 + (double)(lt - C.ns);
        const float hp = (float)px;
        const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        frec[t] = make_float4(hp, 0.0f, 0.0f, 0.0f);
        frec[S + t] = make_float4((float)(px - (double)hp), 0.0f, 0.0f, 0.0f);
        frec[2 * S + t] = z;
        frec[3 * S + t] = z;
        frec[4 * S + t] = z;
    }
    block_sum<2 * kJVals, kProThreads>(g, sh);
    if (threadIdx.x < 2 * kJVals)
        blk[(int64_t)blockIdx.x * 2 * kJVals + threadIdx.x] = sh[threadIdx.x][0];
}

// ---- packed sweeps (two targets or two sources per f32x2 lane pair) ----
//
// The same two sweeps with every step of the pair body one f32x2 operation
// for two lanes of the thread, tiles staged by bulk copies into two shared
// buffers, FP32 partials of kAdjPackFlush tiles added into the FP64 outputs.
// Grid (256-slot blocks, splits); split s of a block with T tiles sweeps
// tiles [s T / js, (s+1) T / js).  Sources are the acceleration kernel's
// staged records (9 float4 per slot, fields duplicated, positions negated);
// targets of the source sweep come from k_adj_tstage: 13 float4 per slot,
// (hi d, lo d, 8/3 v, the 16 sum cotangents with the fourth negated), fields
// duplicated.

constexpr int kAdjPackTile = 64;
constexpr int kAdjPackFlush = 8;
constexpr int kAdjTVals = 13;

__global__ void __launch_bounds__(kGlueThreads)
k_adj_tstage(int64_t S, const float4 *__restrict__ frec, const double *__restrict__ sbar,
             float4 *__restrict__ tst)
{
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (t >= S)
        return;
    const float4 A = frec[t], B = frec[S + t], C = frec[2 * S + t];
    float sb[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        sb[k] = (float)sbar[(int64_t)k * S + t];
    sb[3] = -sb[3];
    const float e3 = 8.0f / 3.0f;
    auto dup = [](float a, float b) { return make_float4(a, a, b, b); };
    float4 *o = tst + t * kAdjTVals;
    o[0] = dup(A.x, A.y);
    o[1] = dup(A.z, B.x);
    o[2] = dup(B.y, B.z);
    o[3] = dup(e3 * C.x, e3 * C.y);
    o[4] = dup(e3 * C.z, sb[0]);
#pragma unroll
    for (int k = 0; k < 7; ++k)
        o[5 + k] = dup(sb[1 + 2 * k], sb[2 + 2 * k]);
    o[12] = dup(sb[15], 0.0f);
}

// Intermediates of one packed pair (two lanes), as in pair_adj:
//   x = d_i - d_j (hi/lo), is = 1/s, mis3 = m_j is^3, h = xvj is^2,
//   F = xvj h + k, Gq = xvi - 2 xvj, Vx, Hb, cv = 2 (Vx h - Hb), gx = dphi/dx.
struct AdjP2 {
    float2 x, y, z, is, mis3, F, Gq, Vx, Hb, cv, gx, gy, gz, dx, dy, dz;   // d = d_i (hi + lo)
};

// sb: the target's 16 cotangents with sb[3] negated.
__device__ __forceinline__ void adj_pair2(float2 hx, float2 hy, float2 hz, float2 lx, float2 ly,
                                          float2 lz, float2 vpx, float2 vpy, float2 vpz,
                                          const float2 (&sb)[kFusedVals], float2 nhx, float2 nhy,
                                          float2 nhz, float2 nlx, float2 nly, float2 nlz,
                                          float2 m, float2 R2, float2 vjx, float2 vjy, float2 vjz,
                                          float2 Cj, float2 Dx, float2 Dy, float2 Dz, float2 wx,
                                          float2 wy, float2 wz, float2 eps2, bool selfx,
                                          bool selfy, AdjP2 &p)
{
    p.x = add2(add2(hx, nhx), add2(lx, nlx));
    p.y = add2(add2(hy, nhy), add2(ly, nly));
    p.z = add2(add2(hz, nhz), add2(lz, nlz));
    float2 s2 = fma2(p.x, p.x, fma2(p.y, p.y, fma2(p.z, p.z, eps2)));
    // a lane's own slot contributes nothing (is = 0 zeroes every term, the
    // source sweep's is-weighted w cotangent included)
    if (selfx) {
        s2.x = 1.0f; m.x = 0.0f; wx.x = wy.x = wz.x = 0.0f;
    }
    if (selfy) {
        s2.y = 1.0f; m.y = 0.0f; wx.y = wy.y = wz.y = 0.0f;
    }
    p.is = make_float2(selfx ? 0.0f : rsqrt_approx(s2.x), selfy ? 0.0f : rsqrt_approx(s2.y));
    const float2 is2 = mul2(p.is, p.is);
    p.mis3 = mul2(mul2(m, p.is), is2);
    const float2 xvj = fma2(p.x, vjx, fma2(p.y, vjy, mul2(p.z, vjz)));
    const float2 xvi = fma2(p.x, vpx, fma2(p.y, vpy, mul2(p.z, vpz)));
    float2 kk = fma2(vpx, vjx, fma2(vpy, vjy, fma2(vpz, vjz, Cj)));
    // D_j . d_i with d_i = hi + lo: D_j is large for stars close to the hole
    p.dx = add2(hx, lx);
    p.dy = add2(hy, ly);
    p.dz = add2(hz, lz);
    kk = fma2(Dx, p.dx, fma2(Dy, p.dy, fma2(Dz, p.dz, kk)));
    const float2 h = mul2(xvj, is2);
    p.F = fma2(h, xvj, kk);
    p.Gq = fma2(make_float2(-2.0f, -2.0f), xvj, xvi);
    const float2 P = fma2(sb[0], p.x, fma2(sb[1], p.y, fma2(sb[2], p.z, fma2(sb[5], R2, sb[4]))));
    p.Vx = fma2(sb[6], p.x, fma2(sb[7], p.y, mul2(sb[8], p.z)));
    p.Hb = fma2(sb[10], vjx, fma2(sb[11], vjy, fma2(sb[12], vjz, sb[9])));
    const float2 Ew = fma2(sb[13], wx, fma2(sb[14], wy, mul2(sb[15], wz)));
    const float2 B = fma2(p.F, p.Vx, fma2(p.Gq, p.Hb, P));
    const float2 b = mul2(p.Vx, h);
    // cx = mis3 (-3 is^2 B - 2 Vx h^2 - sb3) - Ew is^3
    float2 a = fma2(mul2(is2, make_float2(-3.0f, -3.0f)), B, sb[3]);
    a = fma2(mul2(b, make_float2(-2.0f, -2.0f)), h, a);
    const float2 cx = fma2(mul2(Ew, make_float2(-1.0f, -1.0f)), mul2(p.is, is2), mul2(p.mis3, a));
    p.cv = fma2(b, make_float2(2.0f, 2.0f), mul2(p.Hb, make_float2(-2.0f, -2.0f)));
    p.gx = fma2(cx, p.x, mul2(p.mis3, fma2(p.cv, vjx, fma2(p.Hb, vpx, fma2(p.F, sb[6], sb[0])))));
    p.gy = fma2(cx, p.y, mul2(p.mis3, fma2(p.cv, vjy, fma2(p.Hb, vpy, fma2(p.F, sb[7], sb[1])))));
    p.gz = fma2(cx, p.z, mul2(p.mis3, fma2(p.cv, vjz, fma2(p.Hb, vpz, fma2(p.F, sb[8], sb[2])))));
}

// Adds (first: stores) one FP32 partial into an FP64 output.
__device__ __forceinline__ void adj_out(double *o, float p, bool first)
{
    *o = first ? (double)p : *o + (double)p;
}

// The bulk-copy tile pipeline shared by the two packed sweeps: tiles
// [tb, te) of VALS float4 per slot starting at slot slot0 of `rec`, into two
// shared buffers; body(tile, first slot) per tile, flush(first) every
// kAdjPackFlush tiles and after the last.  False if a wait gave up (the
// block must then exit: every thread returns false together).
template <int VALS, class Body, class Flush>
__device__ __forceinline__ bool adj_sweep(const float4 *__restrict__ rec, int64_t slot0,
                                          int64_t tb, int64_t te,
                                          float4 (*sh)[kAdjPackTile][VALS], uint64_t *full,
                                          Body body, Flush flush)
{
    constexpr unsigned kBytes = kAdjPackTile * VALS * 16;
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_load(sh[0], rec + (slot0 + tb * kAdjPackTile) * VALS, kBytes, &full[0], 0);
        if (tb + 1 < te)
            bulk_load(sh[1], rec + (slot0 + (tb + 1) * kAdjPackTile) * VALS, kBytes, &full[1], 0);
    }
    bool first = true;
    for (int64_t tile = tb; tile < te; ++tile) {
        const int b = (int)((tile - tb) & 1);
        const bool ok = mbar_wait(&full[b], (unsigned)(((tile - tb) >> 1) & 1));
        body(sh[b], slot0 + tile * kAdjPackTile);
        if (((tile - tb + 1) % kAdjPackFlush) == 0 || tile + 1 == te) {
            flush(first);
            first = false;
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && tile + 1 < te)
                mbar_wait(&full[b ^ 1], (unsigned)(((tile - tb + 1) >> 1) & 1));
            return false;
        }
        if (threadIdx.x == 0 && tile + 2 < te)
            bulk_load(sh[b], rec + (slot0 + (tile + 2) * kAdjPackTile) * VALS, kBytes, &full[b],
                      0);
    }
    return true;
}

// Reverse sweep over sources for two targets per thread: tpart[split][6][slot]
// = (dphi/dd_i, dphi/dv'_i) summed over the split's sources.
__global__ void __launch_bounds__(kMixThreads, 4)
k_adj_targets_packed(const float4 *__restrict__ srec, int64_t S, const Clu *__restrict__ clu,
                     const int *__restrict__ blk_clu, const double *__restrict__ sbar,
                     int *__restrict__ flag, double *__restrict__ tpart)
{
    __shared__ __align__(128) float4 sh[2][kAdjPackTile][kPackVals];
    __shared__ __align__(8) uint64_t full[2];
    const int64_t t0 = (int64_t)blockIdx.x * 2 * kMixThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / kAdjPackTile, js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    double *out = tpart + sp * 6 * S;
    const int64_t ta = t0 + threadIdx.x, tq = ta + kMixThreads;
    if (te <= tb) {
        for (int k = 0; k < 6; ++k) {
            out[k * S + ta] = 0.0;
            out[k * S + tq] = 0.0;
        }
        return;
    }
    const float4 *ra = srec + ta * kPackVals, *rq = srec + tq * kPackVals;
    const float4 A0 = ra[0], A1 = ra[1], A2 = ra[2], A3 = ra[3], A4 = ra[4], A5 = ra[5];
    const float4 B0 = rq[0], B1 = rq[1], B2 = rq[2], B3 = rq[3], B4 = rq[4], B5 = rq[5];
    const float e3 = 8.0f / 3.0f;
    const float2 hx = make_float2(-A0.x, -B0.x), hy = make_float2(-A0.z, -B0.z),
                 hz = make_float2(-A1.x, -B1.x), lx = make_float2(-A2.x, -B2.x),
                 ly = make_float2(-A2.z, -B2.z), lz = make_float2(-A3.x, -B3.x);
    const float2 vpx = make_float2(e3 * A4.x, e3 * B4.x), vpy = make_float2(e3 * A4.z, e3 * B4.z),
                 vpz = make_float2(e3 * A5.x, e3 * B5.x);
    float2 sb[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        sb[k] = make_float2((float)sbar[k * S + ta], (float)sbar[k * S + tq]);
    sb[3] = make_float2(-sb[3].x, -sb[3].y);
    const float e2 = (float)C.eps2;
    const float2 eps2 = make_float2(e2, e2);
    float2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k)
        acc[k] = make_float2(0.0f, 0.0f);
    auto body = [&](const float4 (*tl)[kPackVals], int64_t j0) {
        const bool diag = (j0 < t0 + 2 * kMixThreads) && (t0 < j0 + kAdjPackTile);
#pragma unroll 1
        for (int q = 0; q < kAdjPackTile; ++q) {
            const float4 S0 = tl[q][0], S1 = tl[q][1], S2 = tl[q][2], S3 = tl[q][3],
                         S4 = tl[q][4], S5 = tl[q][5], S6 = tl[q][6], S7 = tl[q][7],
                         S8 = tl[q][8];
            const bool sx = diag && j0 + q == ta, sy = diag && j0 + q == tq;
            AdjP2 p;
            adj_pair2(hx, hy, hz, lx, ly, lz, vpx, vpy, vpz, sb, lo2(S0), hi2(S0), lo2(S1),
                      lo2(S2), hi2(S2), lo2(S3), hi2(S1), hi2(S3), lo2(S4), hi2(S4), lo2(S5),
                      hi2(S5), lo2(S6), hi2(S6), lo2(S7), hi2(S7), lo2(S8), hi2(S8), eps2, sx, sy,
                      p);
            const float2 mVx = mul2(p.mis3, p.Vx), mHb = mul2(p.mis3, p.Hb);
            acc[0] = fma2(mVx, lo2(S6), add2(acc[0], p.gx));
            acc[1] = fma2(mVx, hi2(S6), add2(acc[1], p.gy));
            acc[2] = fma2(mVx, lo2(S7), add2(acc[2], p.gz));
            acc[3] = fma2(mHb, p.x, fma2(mVx, lo2(S4), acc[3]));
            acc[4] = fma2(mHb, p.y, fma2(mVx, hi2(S4), acc[4]));
            acc[5] = fma2(mHb, p.z, fma2(mVx, lo2(S5), acc[5]));
        }
    };
    auto flush = [&](bool first) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            adj_out(out + k * S + ta, acc[k].x, first);
            adj_out(out + k * S + tq, acc[k].y, first);
            acc[k] = make_float2(0.0f, 0.0f);
        }
    };
    if (!adj_sweep<kPackVals>(srec, C.slot0, tb, te, sh, full, body, flush) && threadIdx.x == 0)
        atomicOr(flag, kFlagTimeout);
}

// Reverse sweep over targets for two sources per thread: spart[split][14][slot]
// = cotangents of the source records (d via x, v, R^2, C, D, w).
__global__ void __launch_bounds__(kMixThreads, 3)
k_adj_sources_packed(const float4 *__restrict__ srec, const float4 *__restrict__ tst, int64_t S,
                     const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                     int *__restrict__ flag, double *__restrict__ spart)
{
    __shared__ __align__(128) float4 sh[2][kAdjPackTile][kAdjTVals];
    __shared__ __align__(8) uint64_t full[2];
    const int64_t t0 = (int64_t)blockIdx.x * 2 * kMixThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / kAdjPackTile, js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    double *out = spart + sp * kAdjSrc * S;
    const int64_t ja = t0 + threadIdx.x, jq = ja + kMixThreads;
    if (te <= tb) {
        for (int k = 0; k < kAdjSrc; ++k) {
            out[k * S + ja] = 0.0;
            out[k * S + jq] = 0.0;
        }
        return;
    }
    const float4 *ra = srec + ja * kPackVals, *rq = srec + jq * kPackVals;
    float4 A[kPackVals], B[kPackVals];
#pragma unroll
    for (int k = 0; k < kPackVals; ++k) {
        A[k] = ra[k];
        B[k] = rq[k];
    }
    auto pr = [&](int k, bool high) {
        return high ? make_float2(A[k].z, B[k].z) : make_float2(A[k].x, B[k].x);
    };
    const float2 nhx = pr(0, false), nhy = pr(0, true), nhz = pr(1, false), m = pr(1, true);
    const float2 nlx = pr(2, false), nly = pr(2, true), nlz = pr(3, false), R2 = pr(3, true);
    const float2 vjx = pr(4, false), vjy = pr(4, true), vjz = pr(5, false), Cj = pr(5, true);
    const float2 Dx = pr(6, false), Dy = pr(6, true), Dz = pr(7, false), wx = pr(7, true);
    const float2 wy = pr(8, false), wz = pr(8, true);
    const float e2 = (float)C.eps2;
    const float2 eps2 = make_float2(e2, e2);
    float2 acc[kAdjSrc];
#pragma unroll
    for (int k = 0; k < kAdjSrc; ++k)
        acc[k] = make_float2(0.0f, 0.0f);
    auto body = [&](const float4 (*tl)[kAdjTVals], int64_t i0) {
        const bool diag = (i0 < t0 + 2 * kMixThreads) && (t0 < i0 + kAdjPackTile);
#pragma unroll 1
        for (int q = 0; q < kAdjPackTile; ++q) {
            const float4 *T = tl[q];
            const float4 T0 = T[0], T1 = T[1], T2 = T[2], T3 = T[3], T4 = T[4];
            float2 sb[kFusedVals];
            sb[0] = hi2(T4);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const float4 Tk = T[5 + k];
                sb[1 + 2 * k] = lo2(Tk);
                sb[2 + 2 * k] = hi2(Tk);
            }
            sb[15] = lo2(T[12]);
            const bool sx = diag && i0 + q == ja, sy = diag && i0 + q == jq;
            AdjP2 p;
            adj_pair2(lo2(T0), hi2(T0), lo2(T1), hi2(T1), lo2(T2), hi2(T2), lo2(T3), hi2(T3),
                      lo2(T4), sb, nhx, nhy, nhz, nlx, nly, nlz, m, R2, vjx, vjy, vjz, Cj, Dx, Dy,
                      Dz, wx, wy, wz, eps2, sx, sy, p);
            const float2 mVx = mul2(p.mis3, p.Vx), gg = mul2(p.mis3, p.Gq);
            acc[0] = add2(acc[0], p.gx);         // negated at the flush
            acc[1] = add2(acc[1], p.gy);
            acc[2] = add2(acc[2], p.gz);
            acc[3] = fma2(gg, sb[10], fma2(p.mis3, fma2(p.cv, p.x, mul2(p.Vx, lo2(T3))), acc[3]));
            acc[4] = fma2(gg, sb[11], fma2(p.mis3, fma2(p.cv, p.y, mul2(p.Vx, hi2(T3))), acc[4]));
            acc[5] = fma2(gg, sb[12], fma2(p.mis3, fma2(p.cv, p.z, mul2(p.Vx, lo2(T4))), acc[5]));
            acc[6] = fma2(p.mis3, sb[5], acc[6]);
            acc[7] = add2(acc[7], mVx);
            acc[8] = fma2(mVx, p.dx, acc[8]);
            acc[9] = fma2(mVx, p.dy, acc[9]);
            acc[10] = fma2(mVx, p.dz, acc[10]);
            acc[11] = fma2(p.is, sb[13], acc[11]);
            acc[12] = fma2(p.is, sb[14], acc[12]);
            acc[13] = fma2(p.is, sb[15], acc[13]);
        }
    };
    auto flush = [&](bool first) {
#pragma unroll
        for (int k = 0; k < kAdjSrc; ++k) {
            const float sgn = k < 3 ? -1.0f : 1.0f;
            adj_out(out + k * S + ja, sgn * acc[k].x, first);
            adj_out(out + k * S + jq, sgn * acc[k].y, first);
            acc[k] = make_float2(0.0f, 0.0f);
        }
    };
    if (!adj_sweep<kAdjTVals>(tst, C.slot0, tb, te, sh, full, body, flush) && threadIdx.x == 0)
        atomicOr(flag, kFlagTimeout);
}

// Both reverse sweeps in one pass over the pairs (mixed contexts, replacing
// the two kernels above where the rows fit): two targets per thread as in
// k_adj_targets_packed, their (d, v') cotangents summed in registers over
// the block's sources, and the 14 record cotangents of every source (as in
// k_adj_sources_packed) summed over the block's 256 targets, so that each
// pair's intermediates are computed once for both.  Inside a warp the
// sources rotate: a tile is two chunks of 32 sources; at step q of a chunk
// lane l takes source (l + q) mod 32 together with that source's running
// sums, adds its two targets' terms and hands the sums to lane l - 1, so
// after 32 steps lane l holds source l's sums over the warp's 64 targets
// (each sum visits lanes s, s - 1, ..., a fixed order).  The four warps'
// sums are then added in warp order (shared rows, two sets alternating by
// tile so one barrier per tile suffices) into one FP32 row per target
// block: spf[p][14][slot], p the target block's index within its cluster.
constexpr int kAdjWarps = kMixThreads / 32;

__global__ void __launch_bounds__(kMixThreads, 3)
k_adj_pairs_packed(const float4 *__restrict__ srec, int64_t S, const Clu *__restrict__ clu,
                   const int *__restrict__ blk_clu, const double *__restrict__ sbar,
                   int *__restrict__ flag, double *__restrict__ tpart, float *__restrict__ spf)
{
    __shared__ __align__(128) float4 sh[2][kAdjPackTile][kPackVals];
    __shared__ float red[2][kAdjWarps][kAdjSrc][kAdjPackTile];
    __shared__ __align__(8) uint64_t full[2];
    const int64_t t0 = (int64_t)blockIdx.x * 2 * kMixThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / kAdjPackTile, js = gridDim.y, sp = blockIdx.y;
    const int64_t tb = sp * ntiles / js, te = (sp + 1) * ntiles / js;
    double *out = tpart + sp * 6 * S;
    float *srow = spf + (t0 - C.slot0) / (2 * kMixThreads) * kAdjSrc * S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ta = t0 + threadIdx.x, tq = ta + kMixThreads;
    if (te <= tb) {
        for (int k = 0; k < 6; ++k) {
            out[k * S + ta] = 0.0;
            out[k * S + tq] = 0.0;
        }
        return;
    }
    const float4 *ra = srec + ta * kPackVals, *rq = srec + tq * kPackVals;
    const float4 A0 = ra[0], A1 = ra[1], A2 = ra[2], A3 = ra[3], A4 = ra[4], A5 = ra[5];
    const float4 B0 = rq[0], B1 = rq[1], B2 = rq[2], B3 = rq[3], B4 = rq[4], B5 = rq[5];
    const float e3 = 8.0f / 3.0f;
    const float2 hx = make_float2(-A0.x, -B0.x), hy = make_float2(-A0.z, -B0.z),
                 hz = make_float2(-A1.x, -B1.x), lx = make_float2(-A2.x, -B2.x),
                 ly = make_float2(-A2.z, -B2.z), lz = make_float2(-A3.x, -B3.x);
    const float2 vpx = make_float2(e3 * A4.x, e3 * B4.x), vpy = make_float2(e3 * A4.z, e3 * B4.z),
                 vpz = make_float2(e3 * A5.x, e3 * B5.x);
    float2 sb[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        sb[k] = make_float2((float)sbar[k * S + ta], (float)sbar[k * S + tq]);
    sb[3] = make_float2(-sb[3].x, -sb[3].y);
    const float e2 = (float)C.eps2;
    const float2 eps2 = make_float2(e2, e2);
    float2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k)
        acc[k] = make_float2(0.0f, 0.0f);
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    constexpr unsigned kBytes = kAdjPackTile * kPackVals * 16;
    if (threadIdx.x == 0) {
        bulk_load(sh[0], srec + (C.slot0 + tb * kAdjPackTile) * kPackVals, kBytes, &full[0], 0);
        if (tb + 1 < te)
            bulk_load(sh[1], srec + (C.slot0 + (tb + 1) * kAdjPackTile) * kPackVals, kBytes,
                      &full[1], 0);
    }
    bool first = true;
    for (int64_t tile = tb; tile < te; ++tile) {
        const int b = (int)((tile - tb) & 1);
        const bool ok = mbar_wait(&full[b], (unsigned)(((tile - tb) >> 1) & 1));
        const int64_t j0 = C.slot0 + tile * kAdjPackTile;
        const bool diag = (j0 < t0 + 2 * kMixThreads) && (t0 < j0 + kAdjPackTile);
        const float4 (*tl)[kPackVals] = sh[b];
#pragma unroll 1
        for (int ch = 0; ch < kAdjPackTile; ch += 32) {
            float s[kAdjSrc];
#pragma unroll
            for (int k = 0; k < kAdjSrc; ++k)
                s[k] = 0.0f;
#pragma unroll 1
            for (int q = 0; q < 32; ++q) {
                const int u = ch + ((lane + q) & 31);
                const float4 S0 = tl[u][0], S1 = tl[u][1], S2 = tl[u][2], S3 = tl[u][3],
                             S4 = tl[u][4], S5 = tl[u][5], S6 = tl[u][6], S7 = tl[u][7],
                             S8 = tl[u][8];
                const bool sx = diag && j0 + u == ta, sy = diag && j0 + u == tq;
                AdjP2 p;
                adj_pair2(hx, hy, hz, lx, ly, lz, vpx, vpy, vpz, sb, lo2(S0), hi2(S0), lo2(S1),
                          lo2(S2), hi2(S2), lo2(S3), hi2(S1), hi2(S3), lo2(S4), hi2(S4),
                          lo2(S5), hi2(S5), lo2(S6), hi2(S6), lo2(S7), hi2(S7), lo2(S8),
                          hi2(S8), eps2, sx, sy, p);
                const float2 mVx = mul2(p.mis3, p.Vx), mHb = mul2(p.mis3, p.Hb);
                // the targets' sums
                acc[0] = fma2(mVx, lo2(S6), add2(acc[0], p.gx));
                acc[1] = fma2(mVx, hi2(S6), add2(acc[1], p.gy));
                acc[2] = fma2(mVx, lo2(S7), add2(acc[2], p.gz));
                acc[3] = fma2(mHb, p.x, fma2(mVx, lo2(S4), acc[3]));
                acc[4] = fma2(mHb, p.y, fma2(mVx, hi2(S4), acc[4]));
                acc[5] = fma2(mHb, p.z, fma2(mVx, lo2(S5), acc[5]));
                // the source's terms from both targets (d via x negated at the store)
                const float2 gg = mul2(p.mis3, p.Gq);
                float2 c[kAdjSrc];
                c[0] = p.gx;
                c[1] = p.gy;
                c[2] = p.gz;
                c[3] = fma2(gg, sb[10], mul2(p.mis3, fma2(p.cv, p.x, mul2(p.Vx, vpx))));
                c[4] = fma2(gg, sb[11], mul2(p.mis3, fma2(p.cv, p.y, mul2(p.Vx, vpy))));
                c[5] = fma2(gg, sb[12], mul2(p.mis3, fma2(p.cv, p.z, mul2(p.Vx, vpz))));
                c[6] = mul2(p.mis3, sb[5]);
                c[7] = mVx;
                c[8] = mul2(mVx, p.dx);
                c[9] = mul2(mVx, p.dy);
                c[10] = mul2(mVx, p.dz);
                c[11] = mul2(p.is, sb[13]);
                c[12] = mul2(p.is, sb[14]);
                c[13] = mul2(p.is, sb[15]);
#pragma unroll
                for (int k = 0; k < kAdjSrc; ++k)
                    s[k] = __shfl_sync(0xffffffffu, s[k] + c[k].x + c[k].y, (lane + 1) & 31);
            }
#pragma unroll
            for (int k = 0; k < kAdjSrc; ++k)
                red[b][wid][k][ch + lane] = s[k];
        }
        if (((tile - tb + 1) % kAdjPackFlush) == 0 || tile + 1 == te) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                adj_out(out + k * S + ta, acc[k].x, first);
                adj_out(out + k * S + tq, acc[k].y, first);
                acc[k] = make_float2(0.0f, 0.0f);
            }
            first = false;
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && tile + 1 < te)
                mbar_wait(&full[b ^ 1], (unsigned)(((tile - tb + 1) >> 1) & 1));
            if (threadIdx.x == 0)
                atomicOr(flag, kFlagTimeout);
            return;
        }
        if (threadIdx.x == 0 && tile + 2 < te)
            bulk_load(sh[b], srec + (C.slot0 + (tile + 2) * kAdjPackTile) * kPackVals, kBytes,
                      &full[b], 0);
        // this tile's source rows: the warps' sums in warp order (set b is
        // written again two tiles on, after the next barrier)
        for (int e = threadIdx.x; e < kAdjSrc * kAdjPackTile; e += kMixThreads) {
            const int k = e / kAdjPackTile, u = e % kAdjPackTile;
            float r = red[b][0][k][u];
#pragma unroll
            for (int w = 1; w < kAdjWarps; ++w)
                r += red[b][w][k][u];
            srow[(int64_t)k * S + j0 + u] = k < 3 ? -r : r;
        }
    }
}

// The merged sweep's partials summed, one thread per value and slot, eight
// loads in flight: e < 14 S, value k = e / S of slot t = e % S, adds its
// cluster's FP32 source rows in target-block order into spart[e] -- a
// compensated FP32 sum (Knuth's TwoSum carrying each addition's rounding
// error), so no FP64 additions, whose pipe runs at 1/64 of FP32's; the
// remaining 6 S threads add the jst FP64 target splits in split order into
// split 0 (as k_split_sum).
__global__ void __launch_bounds__(kGlueThreads)
k_adj_row_sums(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
               const float *__restrict__ spf, double *__restrict__ spart,
               double *__restrict__ tpart, int jst)
{
    const int64_t e = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    const int64_t stride = (int64_t)kAdjSrc * S;
    if (e >= stride) {
        const int64_t f = e - stride, ts = 6 * S;
        if (f >= ts)
            return;
        double acc = tpart[f];
        for (int q = 1; q < jst; ++q)
            acc += tpart[(int64_t)q * ts + f];
        tpart[f] = acc;
        return;
    }
    const int64_t t = e % S;
    const Clu C = clu[cluster_of_block(blk_clu, t / kGlueThreads)];
    const int64_t np = C.ns_pad / (2 * kMixThreads);
    float hi = 0.0f, lo = 0.0f;
    auto add = [&](float x) {        // hi + lo += x, the rounding error of hi + x kept in lo
        const float sum = hi + x, z = sum - hi;
        lo += (hi - (sum - z)) + (x - z);
        hi = sum;
    };
    int64_t p = 0;
    for (; p + 8 <= np; p += 8) {
        float r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            r[i] = spf[(p + i) * stride + e];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            add(r[i]);
    }
    for (; p < np; ++p)
        add(spf[p * stride + e]);
    spart[e] = (double)hi + (double)lo;
}

// Split partials of the jerk's and the reverse sweeps' pair kernels summed in
// place: part holds js splits of nv values of S slots ([split][value][slot]);
// thread (k, t) adds the js partials of value k of slot t, in split order,
// into split 0.  One thread per value and slot with eight loads in flight,
// so the sum runs at L2 bandwidth (the per-star kernels that read the totals
// stalled on these loads).
__global__ void __launch_bounds__(kGlueThreads)
k_split_sum(int64_t S, int nv, int js, double *__restrict__ part)
{
    const int64_t e = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (e >= nv * S)
        return;
    const int64_t stride = (int64_t)nv * S;
    double acc = part[e];
    int q = 1;
    for (; q + 8 <= js; q += 8) {
        double p[8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            p[r] = part[(int64_t)(q + r) * stride + e];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            acc += p[r];
    }
    for (; q < js; ++q)
        acc += part[(int64_t)q * stride + e];
    part[e] = acc;
}

// FP32 split partials (fpart, [split][value][slot], each one FP32 sum)
// added in split order by a compensated FP32 sum (Knuth's TwoSum carrying
// every addition's rounding error: no FP64 additions, whose pipe runs at
// 1/64 of FP32's) into split 0 of the FP64 layout, out[value][slot].
__global__ void __launch_bounds__(kGlueThreads)
k_split_sum_f32(int64_t S, int nv, int js, const float *__restrict__ fpart,
                double *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (e >= nv * S)
        return;
    const int64_t stride = (int64_t)nv * S;
    float hi = 0.0f, lo = 0.0f;
    auto add = [&](float x) {
        const float sum = hi + x, z = sum - hi;
        lo += (hi - (sum - z)) + (x - z);
        hi = sum;
    };
    int q = 0;
    for (; q + 8 <= js; q += 8) {
        float r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            r[i] = fpart[(int64_t)(q + i) * stride + e];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            add(r[i]);
    }
    for (; q < js; ++q)
        add(fpart[(int64_t)q * stride + e]);
    out[e] = (double)hi + (double)lo;
}

// Per star slot, one thread each: the records' and cluster sums' reverse for
// star j (d_j, v_j and M), plus every cotangent gathered so far; writes the
// star's xbar and vbar and, per block of kAdjStarSlots slots, -sum dbar (the
// hole's xbar) and the M cotangent (4 values, added in slot order).  The
// record and cluster-sum terms that depend on d_j, v_j and M, contracted
// with their cotangents (sp: the source sweep's 14, gb: the cluster sums'),
// with GM = G M, Wb = W cotangent + G abar_hole, D8 = sp_D.d_j,
// Wd = (sp_w + Wb).d_j:
//   a = sp_R2 R^2 + sp_C [GM (iR + eps^2 iR3/6) - 4/3 v^2] - GM/3 iR3 D8
//       + m_j iR3 Wd + m_j (gb_Q.v) + m_j (5/4 gb_SA iR + 1/4 gb_SB (R^2 + eps^2) iR3
//       + gb_Phi iR)
// (C_j = c/1.5 - 4/3 v^2 with c = GM (1.5 iR + 1/4 eps^2 iR3), D_j = -e/1.5
// = -GM/3 iR3 d_j, w_j = m_j iR3 d_j); its gradient in closed form:
//   da/dM   = G [sp_C (iR + eps^2 iR3/6) - iR3 D8/3]
//   da/dv   = -8/3 sp_C v + m_j gb_Q
//   da/dd   = iR3 (m_j (sp_w + Wb) - GM/3 sp_D) + 2 d R2b, where
//   R2b = sp_R2 + 1/4 gb_SB m_j iR3 - iR3/2 [da/diR + 3 iR^2 da/diR3],
//   da/diR  = sp_C GM + m_j (5/4 gb_SA + gb_Phi),
//   da/diR3 = sp_C GM eps^2/6 - GM/3 D8 + m_j Wd + 1/4 gb_SB m_j (R^2 + eps^2).
__global__ void __launch_bounds__(kAdjStarSlots)
k_adj_records(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
              const double *__restrict__ x, const double *__restrict__ v,
              const double *__restrict__ m, const double *__restrict__ abar,
              const double *__restrict__ kbar, const double *__restrict__ tpart, int jst,
              const double *__restrict__ spart, int jss, const double *__restrict__ gbar,
              double *__restrict__ xbar, double *__restrict__ vbar, double *__restrict__ blk)
{
    constexpr int kNT = 6;
    __shared__ double h4_[4][kAdjStarSlots];
    const int64_t t = (int64_t)blockIdx.x * kAdjStarSlots + threadIdx.x;
    const int k_clu = cluster_of_block(blk_clu, t / kGlueThreads);
    const Clu Cl = clu[k_clu];
    const double *gb = gbar + (int64_t)k_clu * kAdjGlob;
    const int64_t lt = t - Cl.slot0;
    const bool star = lt < Cl.ns;
    for (int k = 0; k < 4; ++k)
        h4_[k][threadIdx.x] = 0.0;
    if (star) {
        const int64_t j = Cl.body0 + 1 + lt, hb = Cl.body0;
        // split sums of the target (6) and source (14) partials, splits in order
        double tp[kNT], sp[kAdjSrc];
#pragma unroll
        for (int k = 0; k < kNT; ++k) {
            double a = 0.0;
            for (int q = 0; q < jst; ++q)
                a += tpart[((int64_t)q * kNT + k) * S + t];
            tp[k] = a;
        }
#pragma unroll
        for (int k = 0; k < kAdjSrc; ++k) {
            double a = 0.0;
            for (int q = 0; q < jss; ++q)
                a += spart[((int64_t)q * kAdjSrc + k) * S + t];
            sp[k] = a;
        }
        const double mj = m[j], G = Cl.G, eps2 = Cl.eps2, GM = G * m[hb];
        double d[3], vv[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = x[3 * j + k] - x[3 * hb + k];
            vv[k] = v[3 * j + k];
        }
        const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double iR = 1.0 / sqrt(R2), iR3 = iR * iR * iR;
        double Ws[3], D8 = 0.0, Wd = 0.0;
        for (int k = 0; k < 3; ++k) {
            Ws[k] = sp[11 + k] + gb[3 + k] + G * abar[3 * hb + k];
            D8 += sp[8 + k] * d[k];
            Wd += Ws[k] * d[k];
        }
        const double daiR = sp[7] * GM + mj * (1.25 * gb[6] + gb[8]);
        const double daiR3 = sp[7] * GM * eps2 / 6.0 - GM / 3.0 * D8 + mj * Wd +
                             0.25 * gb[7] * mj * (R2 + eps2);
        const double R2b = sp[6] + 0.25 * gb[7] * mj * iR3 -
                           0.5 * iR3 * (daiR + 3.0 * iR * iR * daiR3);
        for (int k = 0; k < 3; ++k) {
            const double ud = iR3 * (mj * Ws[k] - GM / 3.0 * sp[8 + k]) + 2.0 * d[k] * R2b;
            const double uv = -8.0 / 3.0 * sp[7] * vv[k] + mj * gb[k];
            const double dbar = kbar[(int64_t)k * S + t] + tp[k] + sp[k] + ud;
            xbar[3 * j + k] = dbar;
            vbar[3 * j + k] = kbar[(int64_t)(3 + k) * S + t] + 8.0 / 3.0 * tp[3 + k] + sp[3 + k] + uv;
            h4_[k][threadIdx.x] = -dbar;
        }
        h4_[3][threadIdx.x] = G * (sp[7] * (iR + eps2 * iR3 / 6.0) - iR3 * D8 / 3.0);
    }
    __syncwarp();
    // per-block sums over the block's star slots, in slot order
    if (threadIdx.x < 4) {
        double g = 0.0;
        for (int w2 = 0; w2 < kAdjStarSlots; ++w2)
            g += h4_[threadIdx.x][w2];
        blk[(int64_t)blockIdx.x * 4 + threadIdx.x] = g;
    }
}

// The hole of each cluster: its xbar (its velocity does not enter Eq. 1-6),
// and the cluster's M and inv_c2 cotangents, scal[2 k] and scal[2 k + 1]
// (added to scal's contents when `accumulate`).
__global__ void __launch_bounds__(kGlueThreads)
k_adj_hole(const Clu *__restrict__ clu, const double *__restrict__ blk,
           const double *__restrict__ gbar, double *__restrict__ xbar, double *__restrict__ vbar,
           double *__restrict__ scal, int accumulate)
{
    __shared__ double sh[4][kGlueThreads];
    const Clu C = clu[blockIdx.x];
    sum_blocks<4>(blk + (C.slot0 / kAdjStarSlots) * 4, C.ns_pad / kAdjStarSlots, sh);
    if (threadIdx.x == 0) {
        const double *gb = gbar + (int64_t)blockIdx.x * kAdjGlob;
        for (int k = 0; k < 3; ++k) {
            xbar[3 * C.body0 + k] = sh[k][0];
            vbar[3 * C.body0 + k] = 0.0;
        }
        const double mb = sh[3][0] + gb[9], cb = gb[10];
        scal[2 * blockIdx.x] = accumulate ? scal[2 * blockIdx.x] + mb : mb;
        scal[2 * blockIdx.x + 1] = accumulate ? scal[2 * blockIdx.x + 1] + cb : cb;
    }
}

// Reverse of one kick-drift-kick step (pn_step), coordinate-wise, h = dt/2:
//   stage 0 (forward quantities): vh = v + h a, xp = x + dt vh,
//            vp = vh + h a (vel_mode 0) or vh;
//   stage 1 (given xb_A, vpb_A = VJP of A at (xp, vp) with cotangent
//            ab + h vb): vhb = vb + vpb_A + dt (xb + xb_A);
//            xb = xb + xb_A;  ab = h vhb + (vel_mode 0 ? h vpb_A : 0);  vb = vhb;
//   stage 2: xb += xb_A, vb += vpb_A (the entry acceleration's VJP).
__global__ void __launch_bounds__(kGlueThreads)
k_adj_kdk(int stage, int64_t n3, int vel_mode, double dt, const double *__restrict__ x,
          const double *__restrict__ v, const double *__restrict__ a, double *__restrict__ xp,
          double *__restrict__ vp, double *__restrict__ xb, double *__restrict__ vb,
          double *__restrict__ ab, double *__restrict__ atot, const double *__restrict__ xbA,
          const double *__restrict__ vpbA)
{
    const double h = 0.5 * dt;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (stage == 0) {
            const double vh = v[q] + h * a[q];   // forward quantities of the step
            xp[q] = x[q] + dt * vh;
            vp[q] = vel_mode == 0 ? vh + h * a[q] : vh;
            atot[q] = ab[q] + h * vb[q];
        } else if (stage == 2) {
            xb[q] += xbA[q];
            vb[q] += vpbA[q];
        } else {
            const double xnew = xb[q] + xbA[q];
            const double vhb = vb[q] + vpbA[q] + dt * xnew;
            xb[q] = xnew;
            ab[q] = h * vhb + (vel_mode == 0 ? h * vpbA[q] : 0.0);
            vb[q] = vhb;
        }
    }
}

}  // namespace

// Buffers: rec 8 x S double4, part js x 32 x S, blk (S/256) x 24, glob
// nclu x 24, hole terms (S/256) x 6, float records 9 x S float4.
int64_t jerk_part_splits(const pn_ctx *c)
{
    const int64_t nb = c->S / kJThreads;
    int64_t js = (8 * (int64_t)c->sm_count * 4 + nb - 1) / nb;   // ~8 waves of 4 blocks/SM
    const int64_t tiles = c->max_ns_pad / kJTile;
    js = js < 1 ? 1 : (js > tiles ? tiles : js);
    return js > 64 ? 64 : js;
}

// Source splits of the packed FP32 jerk kernel: about eight waves of 3
// blocks per SM over the 256-target blocks, at least one tile per split and
// never more than the FP64 kernel's splits (the partial buffer holds those).
static int64_t jerk_pack_splits(const pn_ctx *c)
{
    const int64_t nb = c->S / kJPackTI;
    int64_t js = (8 * 3 * (int64_t)c->sm_count) / nb;
    const int64_t tiles = c->max_ns_pad / kJPackTile;
    const int64_t cap = jerk_part_splits(c);
    js = js < 1 ? 1 : js;
    js = js > tiles ? tiles : js;
    return js > cap ? cap : js;
}

size_t jerk_buffer_doubles(const pn_ctx *c)
{
    const int64_t S = c->S, npb = S / kProThreads;
    return (size_t)(kJRec * 4 * S + jerk_part_splits(c) * 2 * kFusedVals * S +
                    npb * 2 * kJVals + (int64_t)c->nclu * 2 * kJVals + npb * 6 +
                    32 * S);   // + staged float records of the packed pass (16 float4)
}

cudaError_t launch_jerk(pn_ctx *c, const double *x, const double *v, const double *m,
                        const double *a, double *jerk)
{
    const int64_t S = c->S, nglue = S / kGlueThreads;
    const int js = (int)jerk_part_splits(c);
    double *base = c->jbuf;
    double4_32a *rec = reinterpret_cast<double4_32a *>(base);
    double *part = base + kJRec * 4 * S;
    const int64_t npb = S / kProThreads;      // prologue / epilogue blocks
    double *blk = part + (int64_t)js * 2 * kFusedVals * S;
    double *glob = blk + npb * 2 * kJVals;
    double *bhb = glob + (int64_t)c->nclu * 2 * kJVals;
    const int *bc = c->nclu > 1 ? c->blk_clu : nullptr;
    const unsigned long long step = (unsigned long long)c->step_counter;
    k_jerk_prologue<<<(unsigned)npb, kProThreads, 0, c->stream>>>(S, c->d_clu, bc, x, v, m, a,
                                                                  rec, blk);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_jerk_globals<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, blk, glob);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    dim3 grid((unsigned)(S / kJThreads), (unsigned)js);
    int jsum = js;
    if (c->p.precision == PN_MIXED) {
        // single-precision dual pair sums on staged float records (after the
        // hole terms)
        float4 *srec = reinterpret_cast<float4 *>(bhb + npb * 6);
        const int jp = (int)jerk_pack_splits(c);
        static bool carveout = false;     // 3 blocks of 32 KB per SM
        if (!carveout) {
            cudaFuncSetAttribute(k_jerk_pairs_packed,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            carveout = true;
        }
        // splits of at most kJPackFlush tiles: FP32 partials (one flush each)
        // in the upper half of the partial region, summed by k_split_sum_f32
        const int64_t tps = (c->max_ns_pad / kJPackTile + jp - 1) / jp;
        float *fpart = (jp > 1 && tps <= kJPackFlush)
                           ? reinterpret_cast<float *>(part + (int64_t)js * kFusedVals * S)
                           : nullptr;
        k_jerk_stage<<<(unsigned)nglue, kGlueThreads, 0, c->stream>>>(S, rec, srec, c->d_clu, bc);
        k_jerk_pairs_packed<<<dim3((unsigned)(S / kJPackTI), (unsigned)jp), kMixThreads, 0,
                              c->stream>>>(srec, S, c->d_clu, bc, c->flag, part, fpart);
        c->launches += 2;
        jsum = jp;
        if (fpart) {
            if ((e = cudaGetLastError()) != cudaSuccess)
                return e;
            k_split_sum_f32<<<(unsigned)((2 * kFusedVals * S + kGlueThreads - 1) / kGlueThreads),
                              kGlueThreads, 0, c->stream>>>(S, 2 * kFusedVals, jp, fpart, part);
            c->launches += 1;
            jsum = 1;
        }
    } else {
        k_dual_pairs<Dual><<<grid, kJThreads, 0, c->stream>>>(rec, S, c->d_clu, bc, part);
        c->launches += 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if (jsum > 1) {
        k_split_sum<<<(unsigned)((2 * kFusedVals * S + kGlueThreads - 1) / kGlueThreads),
                      kGlueThreads, 0, c->stream>>>(S, 2 * kFusedVals, jsum, part);
        c->launches += 1;
    }
    k_jerk_epilogue<<<(unsigned)npb, kProThreads, 0, c->stream>>>(
        S, c->d_clu, bc, x, v, m, a, part, 1, glob, jerk, c->flag, c->flag_step, step, bhb,
        c->p.precision == PN_MIXED ? 1 : 0);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_jerk_hole<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, bhb, glob, jerk, c->flag,
                                                        c->flag_step, step);
    c->launches += 1;
    return cudaGetLastError();
}

// Splits of the packed adjoint sweeps: about eight waves of 3 blocks per SM
// over the 256-slot blocks, at least one tile per split, at most the FP64
// sweeps' splits (the partial buffers hold those).
static int64_t adj_pack_splits(const pn_ctx *c)
{
    const int64_t nb = c->S / (2 * kMixThreads);
    int64_t js = (8 * 3 * (int64_t)c->sm_count) / nb;
    const int64_t tiles = c->max_ns_pad / kAdjPackTile;
    const int64_t cap = jerk_part_splits(c);
    js = js < 1 ? 1 : js;
    js = js > tiles ? tiles : js;
    return js > cap ? cap : js;
}

// Target-block rows of the merged sweep's source sums (FP32, rows x 14 x S):
// one per target block of the largest cluster, or 0 where the two separate
// sweeps run instead (PN_ADJ_SEPARATE set when the context was created, or
// rows above kAdjRowBytes).  Independent of the precision, which
// pn_set_params may change after the scratch exists.
constexpr size_t kAdjRowBytes = size_t(4) << 30;

static int64_t adj_rows(const pn_ctx *c)
{
    const int64_t rows = c->max_ns_pad / (2 * kMixThreads);
    if (c->adj_separate || (size_t)rows * kAdjSrc * c->S * sizeof(float) > kAdjRowBytes)
        return 0;
    return rows;
}

// Adjoint scratch (doubles): sbar 16 S, kbar 6 S, target partials js 6 S,
// source partials js 14 S, staged targets of the packed sweep 26 S (13
// float4 per slot), block cotangents (S/32) 11, cluster cotangents nclu 11,
// hole blocks (S/32) 4, then the merged sweep's FP32 source rows.
size_t adjoint_buffer_doubles(const pn_ctx *c)
{
    const int64_t S = c->S, js = jerk_part_splits(c);
    return (size_t)((16 + 6) * S + js * (6 + kAdjSrc) * S + kAdjTVals * 2 * S +
                    (S / kAdjStarSlots) * (kAdjGlob + 4) + (int64_t)c->nclu * kAdjGlob +
                    (adj_rows(c) * kAdjSrc * S + 1) / 2);
}

cudaError_t launch_accel_vjp(pn_ctx *c, const double *x, const double *v, const double *m,
                             const double *abar, double *xbar, double *vbar, double *scal,
                             bool accumulate, const double *fwd_saved, const float4 *srec_saved)
{
    const int64_t S = c->S, nglue = S / kGlueThreads;
    const int js = (int)jerk_part_splits(c);
    double4_32a *rec = reinterpret_cast<double4_32a *>(c->jbuf);
    double *part = c->jbuf + kJRec * 4 * S;
    double *jblk = part + (int64_t)js * 2 * kFusedVals * S;
    double *jglob = jblk + S / kProThreads * 2 * kJVals;
    double *sbar = c->abuf, *kbar = sbar + 16 * S, *tpart = kbar + 6 * S;
    double *spart = tpart + (int64_t)js * 6 * S;
    // staged targets of the packed source sweep (13 float4 per slot, 16-byte aligned)
    float4 *tst = reinterpret_cast<float4 *>(spart + (int64_t)js * kAdjSrc * S);
    double *kblk = spart + (int64_t)js * kAdjSrc * S + kAdjTVals * 2 * S;
    double *gbar = kblk + (S / kAdjStarSlots) * kAdjGlob, *hblk = gbar + (int64_t)c->nclu * kAdjGlob;
    const int *bc = c->nclu > 1 ? c->blk_clu : nullptr;
    dim3 grid((unsigned)(S / kJThreads), (unsigned)js);
    const bool mixed = c->p.precision == PN_MIXED;
    // mixed contexts: single-precision records (hi/lo positions, far form)
    // in the upper half of the pair-sum region
    float4 *frec = reinterpret_cast<float4 *>(part + (int64_t)js * kFusedVals * S);
    cudaError_t e;
    // forward: records and cluster sums (values); the 16 pair sums in double,
    // or (mixed) by the fused pair kernel on the single-precision records
    if (mixed)     // the single-precision records directly
        k_adj_prologue<<<(unsigned)(S / kProThreads), kProThreads, 0, c->stream>>>(
            S, c->d_clu, bc, x, v, m, frec, jblk);
    else
        k_jerk_prologue<<<(unsigned)(S / kProThreads), kProThreads, 0, c->stream>>>(
            S, c->d_clu, bc, x, v, m, nullptr, rec, jblk);
    k_jerk_globals<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, jblk, jglob);
    c->launches += 2;
    const double *fwd = part;
    int jsf = js;
    if (mixed) {
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        // the forward pair sums: given by the caller (an evaluation at this
        // state without the near-source split, fused layout), or computed here
        if (fwd_saved) {
            fwd = fwd_saved;
        } else {
            if ((e = launch_fused_on(c, frec)) != cudaSuccess)
                return e;
            fwd = c->part;
        }
        jsf = 1;
    } else {
        k_dual_pairs<double><<<grid, kJThreads, 0, c->stream>>>(rec, S, c->d_clu, bc, part);
        c->launches += 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // reverse
    k_adj_star<<<(unsigned)(S / kAdjStarSlots), kAdjStarSlots, 0, c->stream>>>(S, c->d_clu, bc, x, v, m, fwd, jsf,
                                                               jglob, abar, sbar, kbar, kblk);
    k_adj_globals<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, kblk, gbar);
    int jsr = js, jss = js;
    if (mixed) {
        // packed sweeps: sources from the staged records of the forward pass
        const float4 *srec = srec_saved ? srec_saved : c->mrec + 5 * S;
        if (!srec_saved && !c->fused_packed)   // the scalar forward kernel stages nothing
            if ((e = launch_stage_sources(c, frec)) != cudaSuccess)
                return e;
        jsr = (int)adj_pack_splits(c);
        static bool carveout = false;     // 4 and 3 blocks per SM need the large carveout
        if (!carveout) {
            cudaFuncSetAttribute(k_adj_targets_packed,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            cudaFuncSetAttribute(k_adj_sources_packed,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            cudaFuncSetAttribute(k_adj_pairs_packed,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            carveout = true;
        }
        const dim3 pgrid((unsigned)(S / (2 * kMixThreads)), (unsigned)jsr);
        if (adj_rows(c) > 0) {
            // one pass for both sweeps; the source rows summed into split 0
            float *spf = reinterpret_cast<float *>(hblk + (S / kAdjStarSlots) * 4);
            k_adj_pairs_packed<<<pgrid, kMixThreads, 0, c->stream>>>(srec, S, c->d_clu, bc, sbar,
                                                                    c->flag, tpart, spf);
            k_adj_row_sums<<<(unsigned)(((kAdjSrc + 6) * S + kGlueThreads - 1) / kGlueThreads),
                             kGlueThreads, 0, c->stream>>>(S, c->d_clu, bc, spf, spart, tpart,
                                                           jsr);
            jss = 1;
            jsr = 1;
        } else {
            k_adj_tstage<<<(unsigned)nglue, kGlueThreads, 0, c->stream>>>(S, frec, sbar, tst);
            k_adj_targets_packed<<<pgrid, kMixThreads, 0, c->stream>>>(srec, S, c->d_clu, bc,
                                                                      sbar, c->flag, tpart);
            k_adj_sources_packed<<<pgrid, kMixThreads, 0, c->stream>>>(srec, tst, S, c->d_clu, bc,
                                                                      c->flag, spart);
            jss = jsr;
        }
        c->launches += 1;
    } else {
        k_adj_targets<<<grid, kJThreads, 0, c->stream>>>(rec, S, c->d_clu, bc, sbar, tpart);
        k_adj_sources<<<grid, kJThreads, 0, c->stream>>>(rec, S, c->d_clu, bc, sbar, spart);
    }
    if (jsr > 1) {              // the sweeps' split partials, summed into split 0
        k_split_sum<<<(unsigned)((6 * S + kGlueThreads - 1) / kGlueThreads), kGlueThreads, 0,
                      c->stream>>>(S, 6, jsr, tpart);
        c->launches += 1;
    }
    if (jss > 1) {
        k_split_sum<<<(unsigned)((kAdjSrc * S + kGlueThreads - 1) / kGlueThreads), kGlueThreads,
                      0, c->stream>>>(S, kAdjSrc, jss, spart);
        c->launches += 1;
    }
    k_adj_records<<<(unsigned)(S / kAdjStarSlots), kAdjStarSlots, 0, c->stream>>>(
        S, c->d_clu, bc, x, v, m, abar, kbar, tpart, 1, spart, 1, gbar, xbar, vbar, hblk);
    k_adj_hole<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, hblk, gbar, xbar, vbar, scal,
                                                       accumulate ? 1 : 0);
    c->launches += 6;
    return cudaGetLastError();
}

cudaError_t launch_adj_kdk(pn_ctx *c, int stage, double dt, const double *x, const double *v,
                           const double *a, double *xp, double *vp, double *xb, double *vb,
                           double *ab, double *atot, const double *xbA, const double *vpbA)
{
    const int64_t n3 = 3 * c->n;
    int64_t nb = (n3 + kGlueThreads - 1) / kGlueThreads;
    if (nb > 4 * (int64_t)c->sm_count)
        nb = 4 * (int64_t)c->sm_count;
    k_adj_kdk<<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(stage, n3, c->p.vel_mode, dt, x, v, a,
                                                            xp, vp, xb, vb, ab, atot, xbA, vpbA);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_hermite(pn_ctx *c, int stage, double *x, double *v, double *a, double *j,
                           const double *a1, const double *j1, double *xe, double *ve,
                           double dt)
{
    const int64_t n3 = 3 * c->n;
    int64_t nb = (n3 + kGlueThreads - 1) / kGlueThreads;
    if (nb > 4 * (int64_t)c->sm_count)
        nb = 4 * (int64_t)c->sm_count;
    k_hermite<<<(unsigned)nb, kGlueThreads, 0, c->stream>>>(stage, n3, x, v, a, j, a1, j1, xe,
                                                            ve, dt);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace pn
