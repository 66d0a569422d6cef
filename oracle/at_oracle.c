/*
 * FP64 CPU oracle for the Axilrod-Teller three-body sum.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library. The GPU
 * library shares no code, header or constant with it.
 *
 * What it computes (Lee, Ozakin, Gray, "Multibody Multipole Methods"):
 *   phi(x_i,x_j,x_k) = (1 + 3 cos t_i cos t_j cos t_k)
 *                      / (|x_i-x_j|^3 |x_i-x_k|^3 |x_j-x_k|^3)     (Sec. 1, Axilrod-Teller)
 *   Phi(x)           = sum_{j<k; j,k != x} phi(x, x_j, x_k)       (Sec. 1, Eq. 1, n = 3)
 * The cosines are formed from vector dot products of the edge vectors
 * (definition of the angle at a vertex), not from squared distances.
 * Every sum is a Neumaier-compensated FP64 sum. The energy
 *   E = sum_{a<b<c} phi(x_a, x_b, x_c)
 * is a separate enumeration, so that sum_i Phi_i = 3E is a real check.
 *
 * Gradients (no counterpart in the paper; the derivative of the definition):
 *   dE/dx_i = sum_{j<k; j,k != i} d phi(x_i, x_j, x_k) / d x_i
 * written out through the chain rule on r_ij, r_ik and the three cosines.
 *
 * Parity status: phi, Phi, E, grad and VJP are pinned by closed forms,
 * a 50-digit brute force, invariances and identities in the tests.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------- Neumaier compensated summation ---------------- */
typedef struct { double s, c; } nsum_t;

static inline void nsum_add(nsum_t* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum_t* a) { return a->s + a->c; }

static inline double dot3(const double* u, const double* v) {
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}
static inline void sub3(const double* a, const double* b, double* out) {
    out[0] = a[0] - b[0]; out[1] = a[1] - b[1]; out[2] = a[2] - b[2];
}

/* Axilrod-Teller phi (Sec. 1). The angle t_i at vertex x_i is the angle
 * between the edge vectors x_j - x_i and x_k - x_i. */
double oracle_at_phi(const double* xi, const double* xj, const double* xk) {
    double eij[3], eik[3], eji[3], ejk[3], eki[3], ekj[3];
    sub3(xj, xi, eij); sub3(xk, xi, eik);
    sub3(xi, xj, eji); sub3(xk, xj, ejk);
    sub3(xi, xk, eki); sub3(xj, xk, ekj);
    double rij = sqrt(dot3(eij, eij));
    double rik = sqrt(dot3(eik, eik));
    double rjk = sqrt(dot3(ejk, ejk));
    double ci = dot3(eij, eik) / (rij * rik);
    double cj = dot3(eji, ejk) / (rij * rjk);
    double ck = dot3(eki, ekj) / (rik * rjk);
    double den = rij * rij * rij * rik * rik * rik * rjk * rjk * rjk;
    return (1.0 + 3.0 * ci * cj * ck) / den;
}

static int nthreads_or_default(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return nthreads_or_default(0); }

/* Phi(x_i) for each requested particle i (Eq. 1 with n = 3): all pairs
 * j < k of the other particles. Also returns sum |phi| if absout != NULL
 * (used to judge cancellation in FP32 comparisons). */
int oracle_phi(const double* X, int64_t N, const int64_t* idx, int64_t n_idx,
               double* out, double* absout, int nthreads) {
    if (N < 0 || n_idx < 0) return -1;
    int nt = nthreads_or_default(nthreads);
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (q = 0; q < n_idx; ++q) {
        int64_t i = idx[q];
        nsum_t acc = {0.0, 0.0}, aacc = {0.0, 0.0};
        const double* xi = X + 3 * i;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int64_t k = j + 1; k < N; ++k) {
                if (k == i) continue;
                double p = oracle_at_phi(xi, X + 3 * j, X + 3 * k);
                nsum_add(&acc, p);
                if (absout) nsum_add(&aacc, fabs(p));
            }
        }
        out[q] = nsum_get(&acc);
        if (absout) absout[q] = nsum_get(&aacc);
    }
    return 0;
}

/* Sum over the terms of Phi(x_i) of the magnitudes of their two parts,
 * (1 + 3 |cos_i cos_j cos_k|) / (r_ij^3 r_ik^3 r_jk^3): the scale of the
 * rounding error of evaluating each term, which |phi| understates where
 * 1 + 3 cos cos cos cancels inside a term. */
int oracle_phi_parts(const double* X, int64_t N, const int64_t* idx, int64_t n_idx, double* out,
                     int nthreads) {
    if (N < 0 || n_idx < 0) return -1;
    int nt = nthreads_or_default(nthreads);
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (q = 0; q < n_idx; ++q) {
        int64_t i = idx[q];
        nsum_t acc = {0.0, 0.0};
        const double* xi = X + 3 * i;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int64_t k = j + 1; k < N; ++k) {
                if (k == i) continue;
                double u[3], v[3], w[3];
                sub3(X + 3 * j, xi, u); sub3(X + 3 * k, xi, v); sub3(X + 3 * k, X + 3 * j, w);
                double ru = sqrt(dot3(u, u)), rv = sqrt(dot3(v, v)), rw = sqrt(dot3(w, w));
                double ci = dot3(u, v) / (ru * rv);
                double cj = -dot3(u, w) / (ru * rw);
                double ck = dot3(v, w) / (rv * rw);
                double D = ru * ru * ru * rv * rv * rv * rw * rw * rw;
                nsum_add(&acc, (1.0 + 3.0 * fabs(ci * cj * ck)) / D);
            }
        }
        out[q] = nsum_get(&acc);
    }
    return 0;
}

/* Total three-body energy E = sum over unordered triples a < b < c. */
int oracle_energy(const double* X, int64_t N, double* out, int nthreads) {
    if (N < 0) return -1;
    int nt = nthreads_or_default(nthreads);
    double* part = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    if (!part) return -2;
    int64_t a;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (a = 0; a < N; ++a) {
        nsum_t acc = {0.0, 0.0};
        for (int64_t b = a + 1; b < N; ++b)
            for (int64_t c = b + 1; c < N; ++c)
                nsum_add(&acc, oracle_at_phi(X + 3 * a, X + 3 * b, X + 3 * c));
        part[a] = nsum_get(&acc);
    }
    nsum_t tot = {0.0, 0.0};
    for (int64_t t = 0; t < N; ++t) nsum_add(&tot, part[t]);
    *out = nsum_get(&tot);
    free(part);
    return 0;
}

/* d phi(x_i, x_j, x_k) / d x_i, written out from the definition.
 * With u = x_j - x_i, v = x_k - x_i, w = x_k - x_j:
 *   cos_i = u.v/(r_ij r_ik), cos_j = (-u).w/(r_ij r_jk), cos_k = v.w/(r_ik r_jk)
 *   D = r_ij^3 r_ik^3 r_jk^3, Nn = 1 + 3 cos_i cos_j cos_k, phi = Nn / D
 *   d r_ij/dx_i = -u/r_ij,  d r_ik/dx_i = -v/r_ik,  r_jk independent of x_i
 *   d(u.v)/dx_i = -(u+v), d((-u).w)/dx_i = w, d(v.w)/dx_i = -w
 *   d phi/dx_i = 3(cj ck dci + ci ck dcj + ci cj dck)/D + 3 phi (u/r_ij^2 + v/r_ik^2) */
static void at_grad_first(const double* xi, const double* xj, const double* xk,
                          double* g /* out[3] */, double* phi_out) {
    double u[3], v[3], w[3];
    sub3(xj, xi, u); sub3(xk, xi, v); sub3(xk, xj, w);
    double rij2 = dot3(u, u), rik2 = dot3(v, v), rjk2 = dot3(w, w);
    double rij = sqrt(rij2), rik = sqrt(rik2), rjk = sqrt(rjk2);
    double uv = dot3(u, v), uw = dot3(u, w), vw = dot3(v, w);
    double ci = uv / (rij * rik);
    double cj = -uw / (rij * rjk);
    double ck = vw / (rik * rjk);
    double D = rij2 * rij * rik2 * rik * rjk2 * rjk;
    double phi = (1.0 + 3.0 * ci * cj * ck) / D;
    for (int d = 0; d < 3; ++d) {
        double dci = -(u[d] + v[d]) / (rij * rik) + ci * (u[d] / rij2 + v[d] / rik2);
        double dcj = w[d] / (rij * rjk) + cj * (u[d] / rij2);
        double dck = -w[d] / (rik * rjk) + ck * (v[d] / rik2);
        double dN = 3.0 * (cj * ck * dci + ci * ck * dcj + ci * cj * dck);
        g[d] = dN / D + 3.0 * phi * (u[d] / rij2 + v[d] / rik2);
    }
    if (phi_out) *phi_out = phi;
}

/* d phi(x_i, x_j, x_k) / d x_i at one triple (the tree-forces oracle's step). */
void oracle_at_grad(const double* xi, const double* xj, const double* xk, double* g) {
    at_grad_first(xi, xj, xk, g, NULL);
}

/* Gradient of E with respect to x_i for each requested i (forces are -grad). */
int oracle_grad(const double* X, int64_t N, const int64_t* idx, int64_t n_idx,
                double* out3, double* normout, int nthreads) {
    if (N < 0 || n_idx < 0) return -1;
    int nt = nthreads_or_default(nthreads);
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (q = 0; q < n_idx; ++q) {
        int64_t i = idx[q];
        nsum_t acc[3] = {{0, 0}, {0, 0}, {0, 0}}, nrm = {0, 0};
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int64_t k = j + 1; k < N; ++k) {
                if (k == i) continue;
                double g[3];
                at_grad_first(X + 3 * i, X + 3 * j, X + 3 * k, g, NULL);
                for (int d = 0; d < 3; ++d) nsum_add(&acc[d], g[d]);
                if (normout) nsum_add(&nrm, sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
            }
        }
        for (int d = 0; d < 3; ++d) out3[3 * q + d] = nsum_get(&acc[d]);
        if (normout) normout[q] = nsum_get(&nrm);
    }
    return 0;
}

/* Vector-Jacobian product of Phi: out_m = d/dx_m sum_l g_l Phi_l.
 * sum_l g_l Phi_l = sum_{a<b<c} (g_a + g_b + g_c) phi_abc, so
 * out_m = sum_{j<k; j,k != m} (g_m + g_j + g_k) d phi(x_m,x_j,x_k)/d x_m. */
int oracle_vjp(const double* X, int64_t N, const double* gw, const int64_t* idx,
               int64_t n_idx, double* out3, double* normout, int nthreads) {
    if (N < 0 || n_idx < 0) return -1;
    int nt = nthreads_or_default(nthreads);
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (q = 0; q < n_idx; ++q) {
        int64_t m = idx[q];
        nsum_t acc[3] = {{0, 0}, {0, 0}, {0, 0}}, nrm = {0, 0};
        for (int64_t j = 0; j < N; ++j) {
            if (j == m) continue;
            for (int64_t k = j + 1; k < N; ++k) {
                if (k == m) continue;
                double g[3];
                at_grad_first(X + 3 * m, X + 3 * j, X + 3 * k, g, NULL);
                double wgt = gw[m] + gw[j] + gw[k];
                for (int d = 0; d < 3; ++d) nsum_add(&acc[d], wgt * g[d]);
                if (normout) nsum_add(&nrm, fabs(wgt) * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
            }
        }
        for (int d = 0; d < 3; ++d) out3[3 * q + d] = nsum_get(&acc[d]);
        if (normout) normout[q] = nsum_get(&nrm);
    }
    return 0;
}
