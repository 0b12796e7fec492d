// pn_jerk.cu -- the jerk (Appendix A of Tatekawa, arXiv:1801.07986): the
// time derivative of the accelerations of Eq. 1-6 along the trajectory,
//   j = sum_k [dA/dx_k . v_k + dA/dv_k . a_k],   a = A(x, v),
// and the fourth-order Hermite steps that use it (Section 5).
//
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
// as in the acceleration kernels).  Per-block Dual sums of the cluster sums.
__global__ void __launch_bounds__(kGlueThreads)
k_jerk_prologue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                const double *__restrict__ x, const double *__restrict__ v,
                const double *__restrict__ m, const double *__restrict__ a,
                double4_32a *__restrict__ rec, double *__restrict__ blk)
{
    __shared__ double sh[2 * kJVals][kGlueThreads];
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    const Clu C = clu[cluster_of_block(blk_clu, blockIdx.x)];
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
            d[k] = dual(x[3 * j + k] - x[3 * h + k], v[3 * j + k] - v[3 * h + k]);
            vel[k] = dual(v[3 * j + k], a[3 * j + k]);
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
    block_sum<2 * kJVals>(g, sh);
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
    sum_blocks<2 * kJVals>(blk + (C.slot0 / kGlueThreads) * 2 * kJVals,
                           C.ns_pad / kGlueThreads, sh);
    if (threadIdx.x < 2 * kJVals)
        glob[(int64_t)blockIdx.x * 2 * kJVals + threadIdx.x] = sh[threadIdx.x][0];
}

// Pair sums of passes 1 and 2 (the 16 sums of the fused kernels) on Duals,
// one target per thread; grid (target blocks, source splits), split s of a
// target block in cluster k sweeping tiles [s tps, (s+1) tps).  Output
// part[split][2 value + {0 value, 1 derivative}][slot].
__global__ void __launch_bounds__(kJThreads)
k_jerk_pairs(const double4_32a *__restrict__ rec, int64_t S, const Clu *__restrict__ clu,
             const int *__restrict__ blk_clu, double *__restrict__ part)
{
    __shared__ double4_32a sh[kJRec][kJTile];
    const int64_t t0 = (int64_t)blockIdx.x * kJThreads;
    const Clu C = clu[cluster_of_block(blk_clu, t0 / kGlueThreads)];
    const int ntiles = (int)(C.ns_pad / kJTile);
    const int tps = (ntiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int64_t ti = t0 + threadIdx.x;
    const double4_32a T0 = rec[ti], T1 = rec[S + ti], T2 = rec[2 * S + ti], T3 = rec[3 * S + ti];
    const Dual di[3] = {dual(T0.x, T1.x), dual(T0.y, T1.y), dual(T0.z, T1.z)};
    const Dual vi[3] = {dual(8.0 / 3.0 * T2.x, 8.0 / 3.0 * T3.x),
                        dual(8.0 / 3.0 * T2.y, 8.0 / 3.0 * T3.y),
                        dual(8.0 / 3.0 * T2.z, 8.0 / 3.0 * T3.z)};
    Dual acc[kFusedVals];
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k)
        acc[k] = dual(0.0, 0.0);
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
            const Dual xx[3] = {di[0] - dual(A0.x, A1.x), di[1] - dual(A0.y, A1.y),
                                di[2] - dual(A0.z, A1.z)};
            const Dual vj[3] = {dual(A2.x, A3.x), dual(A2.y, A3.y), dual(A2.z, A3.z)};
            const Dual s2 = xx[0] * xx[0] + xx[1] * xx[1] + xx[2] * xx[2] + eps2;
            const double y = 1.0 / sqrt(s2.v);
            const Dual is = dual(y, -0.5 * y * y * y * s2.d);
            const Dual is2 = is * is;
            const Dual mis = A0.w * is;
            const Dual mis3 = mis * is2;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[k] += mis3 * xx[k];
            acc[3] += mis;
            acc[4] += mis3;
            acc[5] += mis3 * dual(A2.w, A3.w);
            const Dual xvj = xx[0] * vj[0] + xx[1] * vj[1] + xx[2] * vj[2];
            const Dual xvi = xx[0] * vi[0] + xx[1] * vi[1] + xx[2] * vi[2];
            const Dual kk = dual(A4.w, A5.w) + (vi[0] * vj[0] + vi[1] * vj[1] + vi[2] * vj[2]) +
                            (dual(A4.x, A5.x) * di[0] + dual(A4.y, A5.y) * di[1] +
                             dual(A4.z, A5.z) * di[2]);
            const Dual f = mis3 * (xvj * is2 * xvj + kk);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[6 + k] += f * xx[k];
            const Dual gg = mis3 * (xvi - 2.0 * xvj);
            acc[9] += gg;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                acc[10 + k] += gg * vj[k];
            acc[13] += dual(A6.x, A7.x) * is;
            acc[14] += dual(A6.y, A7.y) * is;
            acc[15] += dual(A6.z, A7.z) * is;
        }
    }
    double *out = part + (int64_t)blockIdx.y * 2 * kFusedVals * S;
#pragma unroll
    for (int k = 0; k < kFusedVals; ++k) {
        out[(int64_t)(2 * k) * S + ti] = acc[k].v;
        out[(int64_t)(2 * k + 1) * S + ti] = acc[k].d;
    }
}

// Per star: the split partials summed, star_eqs on Duals; the value is the
// acceleration and the derivative the jerk.  Per-block sums of the hole's
// terms (3 values, 3 derivatives) go to blk.
__global__ void __launch_bounds__(kGlueThreads)
k_jerk_epilogue(int64_t S, const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
                const double *__restrict__ x, const double *__restrict__ v,
                const double *__restrict__ m, const double *__restrict__ a,
                const double *__restrict__ part, int js, const double *__restrict__ globs,
                double *__restrict__ jerk, int *flag, unsigned long long *flag_step,
                unsigned long long step, double *__restrict__ blk)
{
    __shared__ double sh[6][kGlueThreads];
    const int64_t t = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    const int k_clu = cluster_of_block(blk_clu, blockIdx.x);
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
        Dual s[kFusedVals];
        for (int k = 0; k < kFusedVals; ++k) {
            double sv = 0.0, sd = 0.0;
            for (int q = 0; q < js; ++q) {
                sv += part[((int64_t)q * 2 * kFusedVals + 2 * k) * S + t];
                sd += part[((int64_t)q * 2 * kFusedVals + 2 * k + 1) * S + t];
            }
            s[k] = dual(sv, sd);
        }
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
        star_eqs<Dual>(Cl.G, m[hb], m[i], Cl.eps2, Cl.inv_c2, 1.0, d, vv, ss, gs, ai, bh);
        const double ji[3] = {ai[0].d, ai[1].d, ai[2].d};
        flag_nonfinite(ji, flag, flag_step, step);
        for (int k = 0; k < 3; ++k) {
            jerk[3 * i + k] = ai[k].d;
            bh6[k] = bh[k].v;
            bh6[3 + k] = bh[k].d;
        }
    }
    block_sum<6>(bh6, sh);
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
    sum_blocks<6>(blk + (C.slot0 / kGlueThreads) * 6, C.ns_pad / kGlueThreads, sh);
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

}  // namespace

// Buffers: rec 8 x S double4, part js x 32 x S, blk (S/256) x 24, glob
// nclu x 24, hole terms (S/256) x 6.
int64_t jerk_part_splits(const pn_ctx *c)
{
    const int64_t nb = c->S / kJThreads;
    int64_t js = (8 * (int64_t)c->sm_count * 4 + nb - 1) / nb;   // ~8 waves of 4 blocks/SM
    const int64_t tiles = c->max_ns_pad / kJTile;
    js = js < 1 ? 1 : (js > tiles ? tiles : js);
    return js > 64 ? 64 : js;
}

size_t jerk_buffer_doubles(const pn_ctx *c)
{
    const int64_t S = c->S, nglue = S / kGlueThreads;
    return (size_t)(kJRec * 4 * S + jerk_part_splits(c) * 2 * kFusedVals * S +
                    nglue * 2 * kJVals + (int64_t)c->nclu * 2 * kJVals + nglue * 6);
}

cudaError_t launch_jerk(pn_ctx *c, const double *x, const double *v, const double *m,
                        const double *a, double *jerk)
{
    const int64_t S = c->S, nglue = S / kGlueThreads;
    const int js = (int)jerk_part_splits(c);
    double *base = c->jbuf;
    double4_32a *rec = reinterpret_cast<double4_32a *>(base);
    double *part = base + kJRec * 4 * S;
    double *blk = part + (int64_t)js * 2 * kFusedVals * S;
    double *glob = blk + nglue * 2 * kJVals;
    double *bhb = glob + (int64_t)c->nclu * 2 * kJVals;
    const int *bc = c->nclu > 1 ? c->blk_clu : nullptr;
    const unsigned long long step = (unsigned long long)c->step_counter;
    k_jerk_prologue<<<(unsigned)nglue, kGlueThreads, 0, c->stream>>>(S, c->d_clu, bc, x, v, m, a,
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
    k_jerk_pairs<<<grid, kJThreads, 0, c->stream>>>(rec, S, c->d_clu, bc, part);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_jerk_epilogue<<<(unsigned)nglue, kGlueThreads, 0, c->stream>>>(
        S, c->d_clu, bc, x, v, m, a, part, js, glob, jerk, c->flag, c->flag_step, step, bhb);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_jerk_hole<<<c->nclu, kGlueThreads, 0, c->stream>>>(c->d_clu, bhb, glob, jerk, c->flag,
                                                        c->flag_step, step);
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
