/*
 * pn_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, FP64 CPU evaluation of the limited first-order
 * post-Newtonian (1PN) N-body equations of T. Tatekawa, "Accelerating
 * N-body simulation of self-gravitating systems with limited first-order
 * post-Newtonian approximation" (arXiv:1801.07986):
 *
 *   Section 2, Eq. 1-3  acceleration of the massive body ("#1", index 0 here)
 *   Section 2, Eq. 4-6  acceleration of a low-mass star i
 *   Section 2, Eq. 7-8  1PN energy and momentum
 *   Section 4, Eq. 10   Plummer softening between stars
 *
 * plus, for cross-checks only, the general EIH equations and EIH energy
 * (Einstein, Infeld & Hoffmann 1938; Lorentz & Droste 1917), of which the
 * paper's equations are the one-heavy-body limit (Section 2).
 *
 * Every sum is written the way the paper prints it: one loop per printed
 * sum, the heavy body's double sums over (j, k) as explicit double loops,
 * no algebraic regrouping.  Accumulation is compensated (Knuth TwoSum), and
 * each target's sum runs in a fixed order, so results do not depend on the
 * number of OpenMP threads.  Build with -ffp-contract=off.
 *
 * Only the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path.
 *
 * Readings of the printed equations (the paper is garbled in places):
 *  R1  x_ab = x_a - x_b and v_ab = v_a - v_b for every pair, although the
 *      text below Eq. 1 and below Eq. 6 prints the opposite order; only this
 *      order makes the Newtonian terms attractive and reproduces EIH.
 *  R2  Eq. 4's star-star Newtonian term divides by r_ij^3 (the cube is
 *      missing in print).
 *  R3  Eq. 2's (3/2)(v_j . n_1j) term is squared, as in Eq. 6 and EIH.
 *  R4  Eq. 5's v_a is v_i.
 *  R5  Sums over j, k run over stars; a star sum for target i skips j = i.
 *      In Eq. 3 the first two double sums skip k = j; the last one (the
 *      terms that replace the heavy body's velocity) keeps k = j, like the
 *      explicit self term printed in Eq. 6.
 *  R6  The heavy body's velocity never enters Eqs. 1-6 (they assume the
 *      zero-momentum frame); it is evolved as state and used in Eqs. 7-8.
 *  R7  Softening (Eq. 10) applies to star-star separations only, to every
 *      occurrence of r_ij (1/r, 1/r^3, r^2, and n_ij = x_ij / r_ij); body-star
 *      separations are never softened.
 *  R8  In Eq. 7 the last double sum keeps i = j; the other double sums of
 *      Eqs. 7-8 run over ordered pairs i != j.
 *  R9  Integrator: kick-drift-kick leapfrog whose force after the drift is
 *      evaluated at the predicted velocity v_half + (dt/2) a_old (vel_mode 0)
 *      or at v_half (vel_mode 1); the paper's own classical RK4
 *      (Section 4), orc_rk4_step; and the fourth-order Hermite scheme the
 *      paper recommends (Section 5), orc_hermite_step, iterated once (two
 *      evaluate-correct passes) because the force depends on velocity.
 *  R10 The jerk (Appendix A) is the time derivative of the same Eq. 1-6
 *      along the trajectory, with every a_j in it the full (1PN)
 *      acceleration; the hole's own velocity enters through d/dt x_1j.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* The accelerations, Section 2 (pn_oracle_accel.inc), in double ... */
#define REAL double
#define SQRT sqrt
#include "pn_oracle_accel.inc"
#undef REAL
#undef SQRT

/* ... and in double complex for the complex-step jerk (orc_jerk). */
#define REAL double complex
#define SQRT csqrt
#define ksum ksum_cs
#define ksum3 ksum3_cs
#define kadd kadd_cs
#define kval kval_cs
#define kadd3 kadd3_cs
#define kval3 kval3_cs
#define dot dot_cs
#define sub sub_cs
#define row row_cs
#define star_accel star_accel_cs
#define bh_double_sum_row bh_double_sum_row_cs
#define bh_accel bh_accel_cs
#define bh_partial bh_partial_cs
#include "pn_oracle_accel.inc"
#undef REAL
#undef SQRT
#undef ksum
#undef ksum3
#undef kadd
#undef kval
#undef kadd3
#undef kval3
#undef dot
#undef sub
#undef row
#undef star_accel
#undef bh_double_sum_row
#undef bh_accel
#undef bh_partial

static int check_args(int64_t n, const void *x, const void *v, const void *m)
{
    if (n < 2 || !x || !v || !m)
        return 1;
    return 0;
}

/* Accelerations of all n bodies (body 0 = heavy body).  Returns 0 on success. */
int orc_accel(int64_t n, const double *x, const double *v, const double *m,
              double G, double inv_c2, double eps, double *a)
{
    if (check_args(n, x, v, m) || !a)
        return 1;
    double *rows = (double *)calloc((size_t)(3 * n), sizeof(double));
    if (!rows)
        return 2;
    bh_accel(n, x, v, m, G, inv_c2, eps, rows, a);
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t i = 1; i < n; ++i)
        star_accel(n, x, v, m, G, inv_c2, eps, i, a + 3 * i);
    free(rows);
    return 0;
}

/*
 * Directional derivative of the accelerations of Eq. 1-6 along
 * (dx, dv, dM of the hole mass m[0], dinv_c2 of 1/c^2), by a complex step:
 * Im A(x + i h dx, v + i h dv; M + i h dM, inv_c2 + i h dinv_c2) / h with
 * h = 1e-20 (relative error O(h^2), no cancellation).
 */
int orc_accel_jvp(int64_t n, const double *x, const double *v, const double *m,
                  double G, double inv_c2, double eps, const double *dx, const double *dv,
                  double dM, double dinv_c2, double *out)
{
    if (check_args(n, x, v, m) || !dx || !dv || !out)
        return 1;
    const double h = 1e-20;
    const size_t n3 = 3 * (size_t)n;
    double complex *xc = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *vc = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *mc = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    double complex *ac = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *rows = (double complex *)calloc(n3, sizeof(double complex));
    int rc = 0;
    if (!xc || !vc || !mc || !ac || !rows) {
        rc = 2;
    } else {
        for (size_t q = 0; q < n3; ++q) {
            xc[q] = x[q] + I * (h * dx[q]);
            vc[q] = v[q] + I * (h * dv[q]);
        }
        for (int64_t q = 0; q < n; ++q)
            mc[q] = m[q];
        mc[0] = m[0] + I * (h * dM);
        const double complex ic2 = inv_c2 + I * (h * dinv_c2);
        bh_accel_cs(n, xc, vc, mc, G, ic2, eps, rows, ac);
        int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
        for (int64_t i = 1; i < n; ++i)
            star_accel_cs(n, xc, vc, mc, G, ic2, eps, i, ac + 3 * i);
        for (size_t q = 0; q < n3; ++q)
            out[q] = cimag(ac[q]) / h;
    }
    free(xc);
    free(vc);
    free(mc);
    free(ac);
    free(rows);
    return rc;
}

/*
 * Jerk: the time derivative of the accelerations of Eq. 1-6 along the
 * trajectory (Appendix A), j = sum_k [dA/dx_k . v_k + dA/dv_k . a_k] with
 * a = A(x, v) given: the directional derivative along (v, a).  Appendix A
 * prints the expanded derivative, garbled in places; here the derivative is
 * taken of the same equations the oracle evaluates.
 */
int orc_jerk(int64_t n, const double *x, const double *v, const double *m,
             double G, double inv_c2, double eps, const double *a, double *jerk)
{
    if (check_args(n, x, v, m) || !a || !jerk)
        return 1;
    return orc_accel_jvp(n, x, v, m, G, inv_c2, eps, v, a, 0.0, 0.0, jerk);
}

/* Accelerations of the listed targets only (index 0 = heavy body). */
int orc_accel_rows(int64_t n, const double *x, const double *v, const double *m,
                   double G, double inv_c2, double eps, int64_t nrows,
                   const int64_t *targets, double *a_rows)
{
    if (check_args(n, x, v, m) || !targets || !a_rows || nrows < 0)
        return 1;
    for (int64_t r = 0; r < nrows; ++r)
        if (targets[r] < 0 || targets[r] >= n)
            return 1;
    int nt = orc_get_threads();
    for (int64_t r = 0; r < nrows; ++r) {
        if (targets[r] != 0)
            continue;
        double *rows = (double *)calloc((size_t)(3 * n), sizeof(double));
        if (!rows)
            return 2;
        bh_accel(n, x, v, m, G, inv_c2, eps, rows, a_rows + 3 * r);
        free(rows);
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t r = 0; r < nrows; ++r)
        if (targets[r] != 0)
            star_accel(n, x, v, m, G, inv_c2, eps, targets[r], a_rows + 3 * r);
    return 0;
}

/* The heavy body's sums of Eq. 1-3 over the outer stars j in [j0, j1):
 * out[0..2] the Newtonian sum, out[3..5] the 1PN sums before the 1/c^2
 * factor (the hole's acceleration over [1, n) is out[0..2] + inv_c2
 * out[3..5]).  Ranges that partition [1, n) add up to the whole. */
int orc_bh_partial(int64_t n, const double *x, const double *v, const double *m,
                   double G, double eps, int64_t j0, int64_t j1, double *out)
{
    if (check_args(n, x, v, m) || !out || j0 < 1 || j1 > n || j0 > j1)
        return 1;
    double *rows = (double *)calloc((size_t)(3 * n), sizeof(double));
    if (!rows)
        return 2;
    bh_partial(n, x, v, m, G, eps, j0, j1, rows, out, out + 3);
    free(rows);
    return 0;
}

/* The heavy body's inner double-sum rows of Eq. 3 for the listed outer
 * indices j (each 1 <= j < n); used to time a bounded sample of that work. */
int orc_bh_rows(int64_t n, const double *x, const double *v, const double *m,
                double G, double eps, int64_t nrows, const int64_t *js,
                double *out)
{
    if (check_args(n, x, v, m) || !js || !out)
        return 1;
    for (int64_t r = 0; r < nrows; ++r)
        if (js[r] < 1 || js[r] >= n)
            return 1;
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t r = 0; r < nrows; ++r)
        bh_double_sum_row(n, x, v, m, G, eps, js[r], out + 3 * r);
    return 0;
}

/* Newtonian accelerations alone, written out directly: the body-star terms
 * unsoftened, the star-star terms softened (Eq. 1 and Eq. 4 with c -> inf). */
int orc_newton_accel(int64_t n, const double *x, const double *m, double G,
                     double eps, double *a)
{
    if (n < 2 || !x || !m || !a)
        return 1;
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        ksum3 acc;
        memset(&acc, 0, sizeof acc);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double d[3];
            sub(row(x, j), row(x, i), d);             /* points from i to j */
            double r2 = dot(d, d);
            if (i != 0 && j != 0)
                r2 += eps * eps;
            const double r = sqrt(r2);
            kadd3(&acc, G * m[j] / (r2 * r), d);
        }
        kval3(&acc, a + 3 * i);
    }
    return 0;
}

/*
 * 1PN energy (Eq. 7) and momentum (Eq. 8).
 * out[0] = Newtonian energy, out[1] = inv_c2 * (the 1/c^2 bracket of Eq. 7),
 * out[2..4] = Newtonian momentum, out[5..7] = 1/c^2 part of Eq. 8.
 */
int orc_energy(int64_t n, const double *x, const double *v, const double *m,
               double G, double inv_c2, double eps, double *out)
{
    if (check_args(n, x, v, m) || !out)
        return 1;
    const double M = m[0];
    const double *x1 = row(x, 0), *v1 = row(v, 0);
    const double e2 = eps * eps;
    const double v1_2 = dot(v1, v1);
    /* per-star pair sums, each in fixed j order, added in i order below */
    double *pe = (double *)calloc((size_t)(9 * n), sizeof(double));
    if (!pe)
        return 2;
    int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t i = 1; i < n; ++i) {
        const double *xi = row(x, i), *vi = row(v, i);
        const double mi = m[i];
        double xi1[3];
        sub(xi, x1, xi1);
        const double r1i = sqrt(dot(xi1, xi1));
        const double vi2 = dot(vi, vi);
        ksum s_pot, s_pn, s_3b, s_bb;
        ksum3 s_p;
        memset(&s_pot, 0, sizeof s_pot);
        memset(&s_pn, 0, sizeof s_pn);
        memset(&s_3b, 0, sizeof s_3b);
        memset(&s_bb, 0, sizeof s_bb);
        memset(&s_p, 0, sizeof s_p);
        for (int64_t j = 1; j < n; ++j) {
            const double *xj = row(x, j), *vj = row(v, j);
            const double mj = m[j];
            double xj1[3];
            sub(xj, x1, xj1);
            const double r1j = sqrt(dot(xj1, xj1));
            /* (1/2) sum_{i,j} G^2 M m_i m_j/(r_1i r_1j), i = j included (R8) */
            kadd(&s_bb, G * G * M * mi * mj / (r1i * r1j));
            if (j == i)
                continue;
            double xij[3];
            sub(xi, xj, xij);
            const double rij = sqrt(dot(xij, xij) + e2);
            const double nvi = dot(xij, vi) / rij, nvj = dot(xij, vj) / rij;
            const double gmm = G * mi * mj / rij;
            /* -(1/2) sum_{i,j} G m_i m_j / r_ij */
            kadd(&s_pot, -0.5 * gmm);
            /* (1/4) sum_{i,j} G m_i m_j/r_ij [6 v_i^2 - 7 v_i.v_j - (n.v_i)(n.v_j)] */
            kadd(&s_pn, 0.25 * gmm * (6.0 * vi2 - 7.0 * dot(vi, vj) - nvi * nvj));
            /* sum_{i,j} G^2 M m_i m_j / (r_ij r_1i) */
            kadd(&s_3b, G * gmm * M / r1i);
            /* Eq. 8: -1/2 sum_{i,j} G m_i m_j/r_ij [v_i + (v_i . n_ij) n_ij] */
            double w[3];
            w[0] = vi[0] + nvi * xij[0] / rij;
            w[1] = vi[1] + nvi * xij[1] / rij;
            w[2] = vi[2] + nvi * xij[2] / rij;
            kadd3(&s_p, -0.5 * gmm, w);
        }
        double *o = pe + 9 * i;
        o[0] = kval(&s_pot);
        o[1] = kval(&s_pn);
        o[2] = kval(&s_3b);
        o[3] = kval(&s_bb);
        kval3(&s_p, o + 4);
    }

    ksum eN, ePN;
    ksum3 pN, pPN;
    memset(&eN, 0, sizeof eN);
    memset(&ePN, 0, sizeof ePN);
    memset(&pN, 0, sizeof pN);
    memset(&pPN, 0, sizeof pPN);
    /* (1/2) M v_1^2 and M v_1 */
    kadd(&eN, 0.5 * M * v1_2);
    kadd3(&pN, M, v1);
    for (int64_t i = 1; i < n; ++i) {
        const double *xi = row(x, i), *vi = row(v, i);
        const double mi = m[i];
        double xi1[3];
        sub(xi, x1, xi1);
        const double r1i = sqrt(dot(xi1, xi1));
        const double vi2 = dot(vi, vi);
        const double n1i_vi = dot(xi1, vi) / r1i, n1i_v1 = dot(xi1, v1) / r1i;
        const double gmm = G * M * mi / r1i;
        const double *o = pe + 9 * i;
        /* Eq. 7, Newtonian part */
        kadd(&eN, 0.5 * mi * vi2);
        kadd(&eN, o[0]);
        kadd(&eN, -gmm);
        /* Eq. 7, 1/c^2 bracket */
        kadd(&ePN, 0.375 * mi * vi2 * vi2);
        kadd(&ePN, 1.5 * gmm * vi2);
        kadd(&ePN, 0.5 * G * G * M * M * mi / (r1i * r1i));
        kadd(&ePN, o[1]);
        kadd(&ePN, 0.5 * gmm * (3.0 * v1_2 - 7.0 * dot(v1, vi) - n1i_v1 * n1i_vi));
        kadd(&ePN, o[2]);
        kadd(&ePN, 0.5 * o[3]);
        /* Eq. 8 */
        kadd3(&pN, mi, vi);
        kadd3(&pPN, 0.5 * mi * vi2, vi);
        double w[3];
        w[0] = vi[0] + n1i_vi * xi1[0] / r1i;
        w[1] = vi[1] + n1i_vi * xi1[1] / r1i;
        w[2] = vi[2] + n1i_vi * xi1[2] / r1i;
        kadd3(&pPN, -0.5 * gmm, w);
        w[0] = v1[0] + n1i_v1 * xi1[0] / r1i;
        w[1] = v1[1] + n1i_v1 * xi1[1] / r1i;
        w[2] = v1[2] + n1i_v1 * xi1[2] / r1i;
        kadd3(&pPN, -0.5 * gmm, w);
        static const double one = 1.0;
        kadd3(&pPN, one, o + 4);
    }
    free(pe);
    double p0[3], p1[3];
    kval3(&pN, p0);
    kval3(&pPN, p1);
    out[0] = kval(&eN);
    out[1] = inv_c2 * kval(&ePN);
    for (int d = 0; d < 3; ++d) {
        out[2 + d] = p0[d];
        out[5 + d] = inv_c2 * p1[d];
    }
    return 0;
}

/* ============================================== general EIH (checks) == */

/*
 * EIH accelerations of n bodies of equal status (no softening):
 *   a_a = sum_{b!=a} G m_b n_ba/r_ab^2 [1 + (1/c^2)(v_a^2 + 2 v_b^2
 *           - 4 v_a.v_b - 3/2 (n_ab.v_b)^2 - 4 sum_{c!=a} G m_c/r_ac
 *           - sum_{c!=b} G m_c/r_bc + 1/2 (x_b - x_a).a_b)]
 *       + (1/c^2) sum_{b!=a} G m_b/r_ab^2 [n_ab.(4 v_a - 3 v_b)] (v_a - v_b)
 *       + (7/(2 c^2)) sum_{b!=a} G m_b a_b / r_ab
 * with n_ab = (x_a - x_b)/r_ab and a_b the Newtonian acceleration of b.
 */
int orc_eih_accel(int64_t n, const double *x, const double *v, const double *m,
                  double G, double inv_c2, double *a)
{
    if (check_args(n, x, v, m) || !a)
        return 1;
    double *aN = (double *)calloc((size_t)(3 * n), sizeof(double));
    double *phi = (double *)calloc((size_t)n, sizeof(double));
    if (!aN || !phi) {
        free(aN);
        free(phi);
        return 2;
    }
    for (int64_t b = 0; b < n; ++b) {
        ksum3 acc;
        ksum p;
        memset(&acc, 0, sizeof acc);
        memset(&p, 0, sizeof p);
        for (int64_t c = 0; c < n; ++c) {
            if (c == b)
                continue;
            double d[3];
            sub(row(x, c), row(x, b), d);
            const double r = sqrt(dot(d, d));
            kadd3(&acc, G * m[c] / (r * r * r), d);
            kadd(&p, G * m[c] / r);
        }
        kval3(&acc, aN + 3 * b);
        phi[b] = kval(&p);
    }
    for (int64_t ia = 0; ia < n; ++ia) {
        const double *xa = row(x, ia), *va = row(v, ia);
        ksum3 newt, pn;
        memset(&newt, 0, sizeof newt);
        memset(&pn, 0, sizeof pn);
        for (int64_t ib = 0; ib < n; ++ib) {
            if (ib == ia)
                continue;
            const double *xb = row(x, ib), *vb = row(v, ib);
            double dba[3], nab[3], w[3], vab[3];
            sub(xb, xa, dba);                         /* x_b - x_a */
            const double r = sqrt(dot(dba, dba));
            nab[0] = -dba[0] / r;
            nab[1] = -dba[1] / r;
            nab[2] = -dba[2] / r;
            const double nab_vb = dot(nab, vb);
            const double br = dot(va, va) + 2.0 * dot(vb, vb) - 4.0 * dot(va, vb)
                              - 1.5 * nab_vb * nab_vb - 4.0 * phi[ia] - phi[ib]
                              + 0.5 * dot(dba, aN + 3 * ib);
            const double f = G * m[ib] / (r * r * r);
            kadd3(&newt, f, dba);
            kadd3(&pn, f * br, dba);
            w[0] = 4.0 * va[0] - 3.0 * vb[0];
            w[1] = 4.0 * va[1] - 3.0 * vb[1];
            w[2] = 4.0 * va[2] - 3.0 * vb[2];
            sub(va, vb, vab);
            kadd3(&pn, G * m[ib] / (r * r) * dot(nab, w), vab);
            kadd3(&pn, 3.5 * G * m[ib] / r, aN + 3 * ib);
        }
        double an[3], ap[3];
        kval3(&newt, an);
        kval3(&pn, ap);
        for (int d = 0; d < 3; ++d)
            a[3 * ia + d] = an[d] + inv_c2 * ap[d];
    }
    free(aN);
    free(phi);
    return 0;
}

/* EIH (Lagrangian) energy and momentum.
 * out[0] Newtonian energy, out[1] inv_c2 * 1PN energy bracket:
 *   3/8 sum m v^4 + 1/4 sum_{a!=b} G m_a m_b/r_ab (6 v_a^2 - 7 v_a.v_b
 *   - (n_ab.v_a)(n_ab.v_b)) + 1/2 sum_a sum_{b!=a} sum_{c!=a}
 *   G^2 m_a m_b m_c / (r_ab r_ac);
 * out[2..4] sum m_a v_a, out[5..7] inv_c2 * 1PN momentum bracket:
 *   sum 1/2 m_a v_a^2 v_a - 1/2 sum_{a!=b} G m_a m_b/r_ab
 *   [v_a + (v_a.n_ab) n_ab].                                              */
int orc_eih_energy(int64_t n, const double *x, const double *v, const double *m,
                   double G, double inv_c2, double *out)
{
    if (check_args(n, x, v, m) || !out)
        return 1;
    ksum e0, e1;
    ksum3 p0, p1;
    memset(&e0, 0, sizeof e0);
    memset(&e1, 0, sizeof e1);
    memset(&p0, 0, sizeof p0);
    memset(&p1, 0, sizeof p1);
    for (int64_t a = 0; a < n; ++a) {
        const double *xa = row(x, a), *va = row(v, a);
        const double va2 = dot(va, va);
        kadd(&e0, 0.5 * m[a] * va2);
        kadd(&e1, 0.375 * m[a] * va2 * va2);
        kadd3(&p0, m[a], va);
        kadd3(&p1, 0.5 * m[a] * va2, va);
        for (int64_t b = 0; b < n; ++b) {
            if (b == a)
                continue;
            const double *xb = row(x, b), *vb = row(v, b);
            double d[3];
            sub(xa, xb, d);
            const double r = sqrt(dot(d, d));
            const double na = dot(d, va) / r, nb = dot(d, vb) / r;
            const double gmm = G * m[a] * m[b] / r;
            kadd(&e0, -0.5 * gmm);
            kadd(&e1, 0.25 * gmm * (6.0 * va2 - 7.0 * dot(va, vb) - na * nb));
            double w[3];
            w[0] = va[0] + na * d[0] / r;
            w[1] = va[1] + na * d[1] / r;
            w[2] = va[2] + na * d[2] / r;
            kadd3(&p1, -0.5 * gmm, w);
            for (int64_t c = 0; c < n; ++c) {
                if (c == a)
                    continue;
                double dc[3];
                sub(xa, row(x, c), dc);
                const double rc = sqrt(dot(dc, dc));
                kadd(&e1, 0.5 * G * G * m[a] * m[b] * m[c] / (r * rc));
            }
        }
    }
    double q0[3], q1[3];
    kval3(&p0, q0);
    kval3(&p1, q1);
    out[0] = kval(&e0);
    out[1] = inv_c2 * kval(&e1);
    for (int d = 0; d < 3; ++d) {
        out[2 + d] = q0[d];
        out[5 + d] = inv_c2 * q1[d];
    }
    return 0;
}

/* ========================================================= integrator == */

typedef int (*accel_fn)(int64_t, const double *, const double *, const double *,
                        double, double, double, double *);

static int eih_as_accel(int64_t n, const double *x, const double *v,
                        const double *m, double G, double inv_c2, double eps,
                        double *a)
{
    (void)eps;
    return orc_eih_accel(n, x, v, m, G, inv_c2, a);
}

/*
 * nsteps of kick-drift-kick leapfrog (reading R9).  `a` holds the
 * acceleration at the entry state and is updated; x and v are updated.
 *   v_h = v + dt/2 a;  x = x + dt v_h;
 *   v_p = v_h + dt/2 a (vel_mode 0)  or  v_h (vel_mode 1);
 *   a = A(x, v_p);  v = v_h + dt/2 a.
 */
static int kdk_steps(accel_fn f, int64_t n, double *x, double *v,
                     const double *m, double *a, double G, double inv_c2,
                     double eps, double dt, int64_t nsteps, int vel_mode)
{
    if (check_args(n, x, v, m) || !a || nsteps < 0 || !(dt > 0.0) ||
        (vel_mode != 0 && vel_mode != 1))
        return 1;
    double *vh = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!vh || !vp) {
        free(vh);
        free(vp);
        return 2;
    }
    const double h = 0.5 * dt;
    int rc = 0;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        for (int64_t q = 0; q < 3 * n; ++q) {
            vh[q] = v[q] + h * a[q];
            x[q] = x[q] + dt * vh[q];
            vp[q] = vel_mode == 0 ? vh[q] + h * a[q] : vh[q];
        }
        rc = f(n, x, vp, m, G, inv_c2, eps, a);
        for (int64_t q = 0; q < 3 * n; ++q)
            v[q] = vh[q] + h * a[q];
    }
    free(vh);
    free(vp);
    return rc;
}

int orc_step(int64_t n, double *x, double *v, const double *m, double *a,
             double G, double inv_c2, double eps, double dt, int64_t nsteps,
             int vel_mode)
{
    return kdk_steps(orc_accel, n, x, v, m, a, G, inv_c2, eps, dt, nsteps, vel_mode);
}

/*
 * nsteps of the classical fourth-order Runge-Kutta method (the paper's own
 * integrator, Section 4) for x' = v, v' = A(x, v):
 *   k1 = (v, A(x, v)),  k2 = f(y + dt/2 k1),  k3 = f(y + dt/2 k2),
 *   k4 = f(y + dt k3),  y += dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * `a` holds A at the entry state (k1's acceleration) and on return holds A
 * at the final state, so each step costs four evaluations.
 */
int orc_rk4_step(int64_t n, double *x, double *v, const double *m, double *a,
                 double G, double inv_c2, double eps, double dt, int64_t nsteps)
{
    if (check_args(n, x, v, m) || !a || nsteps < 0 || !(dt > 0.0))
        return 1;
    const size_t b = sizeof(double) * 3 * (size_t)n;
    double *xs = (double *)malloc(b), *vs = (double *)malloc(b);
    double *k2v = (double *)malloc(b), *k3v = (double *)malloc(b), *k4v = (double *)malloc(b);
    double *k2x = (double *)malloc(b), *k3x = (double *)malloc(b), *k4x = (double *)malloc(b);
    double *bufs[] = {xs, vs, k2v, k3v, k4v, k2x, k3x, k4x};
    int rc = 0;
    for (int q = 0; q < 8; ++q)
        if (!bufs[q])
            rc = 2;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        /* k2 at y + dt/2 k1 */
        for (int64_t q = 0; q < 3 * n; ++q) {
            xs[q] = x[q] + 0.5 * dt * v[q];
            vs[q] = v[q] + 0.5 * dt * a[q];
            k2x[q] = vs[q];
        }
        rc = orc_accel(n, xs, vs, m, G, inv_c2, eps, k2v);
        /* k3 at y + dt/2 k2 */
        for (int64_t q = 0; q < 3 * n && rc == 0; ++q) {
            xs[q] = x[q] + 0.5 * dt * k2x[q];
            vs[q] = v[q] + 0.5 * dt * k2v[q];
            k3x[q] = vs[q];
        }
        if (rc == 0)
            rc = orc_accel(n, xs, vs, m, G, inv_c2, eps, k3v);
        /* k4 at y + dt k3 */
        for (int64_t q = 0; q < 3 * n && rc == 0; ++q) {
            xs[q] = x[q] + dt * k3x[q];
            vs[q] = v[q] + dt * k3v[q];
            k4x[q] = vs[q];
        }
        if (rc == 0)
            rc = orc_accel(n, xs, vs, m, G, inv_c2, eps, k4v);
        for (int64_t q = 0; q < 3 * n && rc == 0; ++q) {
            x[q] = x[q] + dt / 6.0 * (v[q] + 2.0 * k2x[q] + 2.0 * k3x[q] + k4x[q]);
            v[q] = v[q] + dt / 6.0 * (a[q] + 2.0 * k2v[q] + 2.0 * k3v[q] + k4v[q]);
        }
        if (rc == 0)
            rc = orc_accel(n, x, v, m, G, inv_c2, eps, a);
    }
    for (int q = 0; q < 8; ++q)
        free(bufs[q]);
    return rc;
}

/*
 * Forward-mode derivative of a kick-drift-kick trajectory (reading R9,
 * vel_mode 0 or 1) by a complex step: the state, the hole mass m[0] and
 * inv_c2 are perturbed by i h (dx0, dv0, dM, dinv_c2) with h = 1e-20, the
 * entry acceleration is A(x0, v0) of the perturbed state, and the nsteps
 * steps run in complex arithmetic.  x, v receive the final state, dx, dv its
 * derivative along the perturbation.  The adjoint's checks contract this
 * with a cotangent, one direction at a time.
 */
int orc_traj_jvp(int64_t n, const double *x0, const double *v0, const double *m,
                 double G, double inv_c2, double eps, double dt, int64_t nsteps,
                 int vel_mode, const double *dx0, const double *dv0, double dM,
                 double dinv_c2, double *x, double *v, double *dx, double *dv)
{
    if (check_args(n, x0, v0, m) || !dx0 || !dv0 || !x || !v || !dx || !dv || nsteps < 0 ||
        !(dt > 0.0) || (vel_mode != 0 && vel_mode != 1))
        return 1;
    const double h = 1e-20;
    const size_t n3 = 3 * (size_t)n;
    double complex *xc = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *vc = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *vh = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *vp = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *ac = (double complex *)malloc(sizeof(double complex) * n3);
    double complex *mc = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    double complex *rows = (double complex *)calloc(n3, sizeof(double complex));
    int rc = 0;
    if (!xc || !vc || !vh || !vp || !ac || !mc || !rows)
        rc = 2;
    const double complex ic2 = inv_c2 + I * (h * dinv_c2);
    if (rc == 0) {
        for (size_t q = 0; q < n3; ++q) {
            xc[q] = x0[q] + I * (h * dx0[q]);
            vc[q] = v0[q] + I * (h * dv0[q]);
        }
        for (int64_t q = 0; q < n; ++q)
            mc[q] = m[q];
        mc[0] = m[0] + I * (h * dM);
    }
    const int nt = orc_get_threads();
    /* entry acceleration, then the steps */
    for (int64_t s = -1; s < nsteps && rc == 0; ++s) {
        const double complex *xe = xc, *ve = vc;
        if (s >= 0) {
            for (size_t q = 0; q < n3; ++q) {
                vh[q] = vc[q] + 0.5 * dt * ac[q];
                xc[q] = xc[q] + dt * vh[q];
                vp[q] = vel_mode == 0 ? vh[q] + 0.5 * dt * ac[q] : vh[q];
            }
            ve = vp;
        }
        bh_accel_cs(n, xe, ve, mc, G, ic2, eps, rows, ac);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
        for (int64_t i = 1; i < n; ++i)
            star_accel_cs(n, xe, ve, mc, G, ic2, eps, i, ac + 3 * i);
        if (s >= 0)
            for (size_t q = 0; q < n3; ++q)
                vc[q] = vh[q] + 0.5 * dt * ac[q];
    }
    if (rc == 0)
        for (size_t q = 0; q < n3; ++q) {
            x[q] = creal(xc[q]);
            v[q] = creal(vc[q]);
            dx[q] = cimag(xc[q]) / h;
            dv[q] = cimag(vc[q]) / h;
        }
    free(xc);
    free(vc);
    free(vh);
    free(vp);
    free(ac);
    free(mc);
    free(rows);
    return rc;
}

/*
 * nsteps of the fourth-order Hermite scheme (the integrator the paper
 * recommends for collisional runs, Section 5, with the jerk of Appendix A),
 * for x' = v, v' = A(x, v), in the predict-(evaluate-correct)^2 form:
 *   predict   x_p = x + dt v + dt^2/2 a + dt^3/6 j,   v_p = v + dt a + dt^2/2 j
 *   evaluate  a_1 = A(x_e, v_e),  j_1 = jerk at (x_e, v_e, a_1)
 *   correct   v' = v + dt/2 (a + a_1) + dt^2/12 (j - j_1)
 *             x' = x + dt/2 (v + v') + dt^2/12 (a - a_1)
 * with (x_e, v_e) the predicted state in the first pass and the corrected
 * one in the second.  A depends on v, so one pass would leave an O(dt^3)
 * velocity error inside a_1 (third order); the second pass restores fourth
 * order.  The second pass's a_1, j_1 (taken one correction before the final
 * state, an O(dt^5) difference) start the next step.  `a` holds A at the
 * entry state, where the jerk is computed; on return it holds A evaluated at
 * the final state.
 */
int orc_hermite_step(int64_t n, double *x, double *v, const double *m, double *a,
                     double G, double inv_c2, double eps, double dt, int64_t nsteps)
{
    if (check_args(n, x, v, m) || !a || nsteps < 0 || !(dt > 0.0))
        return 1;
    const size_t b = sizeof(double) * 3 * (size_t)n;
    double *j0 = (double *)malloc(b), *xe = (double *)malloc(b), *ve = (double *)malloc(b);
    double *a1 = (double *)malloc(b), *j1 = (double *)malloc(b);
    double *bufs[] = {j0, xe, ve, a1, j1};
    int rc = 0;
    for (int q = 0; q < 5; ++q)
        if (!bufs[q])
            rc = 2;
    if (rc == 0 && nsteps > 0)
        rc = orc_jerk(n, x, v, m, G, inv_c2, eps, a, j0);
    const double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        for (int64_t q = 0; q < 3 * n; ++q) {
            xe[q] = x[q] + dt * v[q] + dt2 / 2.0 * a[q] + dt3 / 6.0 * j0[q];
            ve[q] = v[q] + dt * a[q] + dt2 / 2.0 * j0[q];
        }
        for (int pass = 0; pass < 2 && rc == 0; ++pass) {
            rc = orc_accel(n, xe, ve, m, G, inv_c2, eps, a1);
            if (rc == 0)
                rc = orc_jerk(n, xe, ve, m, G, inv_c2, eps, a1, j1);
            for (int64_t q = 0; q < 3 * n && rc == 0; ++q) {
                ve[q] = v[q] + dt / 2.0 * (a[q] + a1[q]) + dt2 / 12.0 * (j0[q] - j1[q]);
                xe[q] = x[q] + dt / 2.0 * (v[q] + ve[q]) + dt2 / 12.0 * (a[q] - a1[q]);
            }
        }
        for (int64_t q = 0; q < 3 * n && rc == 0; ++q) {
            x[q] = xe[q];
            v[q] = ve[q];
            a[q] = a1[q];
            j0[q] = j1[q];
        }
    }
    if (rc == 0 && nsteps > 0)
        rc = orc_accel(n, x, v, m, G, inv_c2, eps, a);
    for (int q = 0; q < 5; ++q)
        free(bufs[q]);
    return rc;
}

int orc_eih_step(int64_t n, double *x, double *v, const double *m, double *a,
                 double G, double inv_c2, double dt, int64_t nsteps, int vel_mode)
{
    return kdk_steps(eih_as_accel, n, x, v, m, a, G, inv_c2, 0.0, dt, nsteps, vel_mode);
}
