/* Truncated three-body far-field expansion, FP64 (§3.2).
 *
 * TEST INFRASTRUCTURE ONLY: the oracle the GPU far-field operator is checked
 * against. Nothing in the GPU library links or calls it.
 *
 * What it computes. For a potential that is a product of pairwise functions,
 *   phi(x, y2, y3) = g12(x - y2) * g13(x - y3) * g23(y2 - y3),
 * and two source sets P2, P3 with centres c2, c3, the contribution of P2 x P3
 * to a point x, Phi(x; P2 x P3) = sum_{y2 in P2} sum_{y3 in P3} phi(x, y2, y3),
 * is approximated by the p-th order far-field expansion of §3.2
 * (Eq. truncated_three_body_farfield_expansion):
 *
 *   sum_{|a| <= p} sum_{a12 <= a} sum_{a13 <= a - a12} sum_{b <= a - a12 - a13}
 *       C(a12 + b, a12) C(a - a12 - b, a13)
 *       M_{a12 + b}(P2, c2) M_{a - a12 - b}(P3, c3) (-1)^{|b|}
 *       D^{a12} g12(x - c2) D^{a13} g13(x - c3) D^{a - a12 - a13} g23(c2 - c3)
 *
 * with multi-index binomials C(g, a) = prod_d C(g_d, a_d) and the far-field
 * moments of §3.1 (Eq. two_body_farfield_expansion),
 *   M_a(P, c) = sum_{y in P} (-1)^{|a|} (y - c)^a / a!.
 * (Expanding each factor in a Taylor series about the centres and collecting
 * the powers of y2 - c2 and y3 - c3 gives exactly these coefficients and
 * signs when M carries the (-1)^{|a|} of its two-body definition.)
 *
 * Pairwise functions are powers of squared lengths, g(v) = (v.v)^s. The
 * Axilrod-Teller potential is a sum of such products: with a = |x - y2|^2,
 * b = |x - y3|^2, c = |y2 - y3|^2 the law of cosines gives
 *   cos t1 cos t2 cos t3 = (b + c - a)(a + c - b)(a + b - c) / (8abc),
 * so phi = (abc)^(-3/2) + (3/8) (b + c - a)(a + c - b)(a + b - c) (abc)^(-5/2),
 * and the cubic expands into ten monomials a^i b^j c^k, each giving the
 * product term with exponents (i - 5/2, j - 5/2, k - 5/2). The expansion of
 * the sum is the sum of the expansions (it is linear in phi).
 *
 * Derivatives: the Taylor coefficients of g at v0 are those of the binomial
 * series |v0|^(2s) sum_k C(s, k) q(t)^k with q(t) = (2 v0.t + t.t)/|v0|^2,
 * truncated at total degree p (q has no constant term, so k <= p suffices);
 * D^a g(v0) = a! times the coefficient of t^a.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FF_PMAX 8
#define FF_NMAX 165 /* C(FF_PMAX + 3, 3) */

typedef struct {
    int n;                                         /* number of multi-indices with |a| <= p */
    int a[FF_NMAX][3];                             /* the multi-indices, by degree then lexicographic */
    int idx[FF_PMAX + 1][FF_PMAX + 1][FF_PMAX + 1]; /* inverse map, -1 beyond degree p */
} ff_index;

static void ff_make_index(int p, ff_index* I) {
    I->n = 0;
    for (int i = 0; i <= FF_PMAX; ++i)
        for (int j = 0; j <= FF_PMAX; ++j)
            for (int k = 0; k <= FF_PMAX; ++k) I->idx[i][j][k] = -1;
    for (int deg = 0; deg <= p; ++deg)
        for (int i = deg; i >= 0; --i)
            for (int j = deg - i; j >= 0; --j) {
                const int k = deg - i - j;
                I->a[I->n][0] = i;
                I->a[I->n][1] = j;
                I->a[I->n][2] = k;
                I->idx[i][j][k] = I->n;
                I->n++;
            }
}

static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

static double binom_int(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

/* generalised binomial C(s, k) = s (s - 1) ... (s - k + 1) / k! */
static double binom_real(double s, int k) {
    double c = 1.0;
    for (int i = 0; i < k; ++i) c *= (s - i) / (i + 1);
    return c;
}

/* c = a * b truncated at degree p (coefficient arrays in ff_index order) */
static void poly_mul(const ff_index* I, const double* a, const double* b, double* c) {
    double tmp[FF_NMAX];
    for (int q = 0; q < I->n; ++q) tmp[q] = 0.0;
    for (int u = 0; u < I->n; ++u) {
        if (a[u] == 0.0) continue;
        for (int v = 0; v < I->n; ++v) {
            const int i = I->a[u][0] + I->a[v][0], j = I->a[u][1] + I->a[v][1],
                      k = I->a[u][2] + I->a[v][2];
            if (i + j + k > FF_PMAX) continue;
            const int w = I->idx[i][j][k];
            if (w >= 0) tmp[w] += a[u] * b[v];
        }
    }
    memcpy(c, tmp, sizeof(double) * I->n);
}

/* out[q] = D^{a_q} g_s(v0), g_s(v) = (v.v)^s, for every |a_q| <= p */
static void ff_derivs(const ff_index* I, int p, const double v0[3], double s, double* out) {
    const double r2 = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
    double q[FF_NMAX], qk[FF_NMAX], ser[FF_NMAX];
    for (int t = 0; t < I->n; ++t) q[t] = qk[t] = ser[t] = 0.0;
    for (int d = 0; d < 3; ++d) {
        int e[3] = {0, 0, 0};
        e[d] = 1;
        if (p >= 1) q[I->idx[e[0]][e[1]][e[2]]] = 2.0 * v0[d] / r2;
        e[d] = 2;
        if (p >= 2) q[I->idx[e[0]][e[1]][e[2]]] = 1.0 / r2;
    }
    qk[0] = 1.0; /* q^0 */
    for (int k = 0; k <= p; ++k) {
        const double ck = binom_real(s, k);
        for (int t = 0; t < I->n; ++t) ser[t] += ck * qk[t];
        poly_mul(I, qk, q, qk);
    }
    const double scale = pow(r2, s);
    for (int t = 0; t < I->n; ++t)
        out[t] = scale * ser[t] * fact(I->a[t][0]) * fact(I->a[t][1]) * fact(I->a[t][2]);
}

/* Neumaier-compensated accumulator */
typedef struct {
    double s, c;
} ksum;

static void kadd(ksum* k, double v) {
    const double t = k->s + v;
    if (fabs(k->s) >= fabs(v))
        k->c += (k->s - t) + v;
    else
        k->c += (v - t) + k->s;
    k->s = t;
}

static void centre_of_mass(const double* Y, int64_t n, double c[3]) {
    for (int d = 0; d < 3; ++d) {
        ksum k = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) kadd(&k, Y[3 * i + d]);
        c[d] = (k.s + k.c) / (double)n;
    }
}

/* M_a(P, c) = sum_{y in P} (-1)^{|a|} (y - c)^a / a! */
static void ff_moments(const ff_index* I, const double* Y, int64_t n, const double c[3], double* M) {
    for (int t = 0; t < I->n; ++t) {
        const int* a = I->a[t];
        const double sign = ((a[0] + a[1] + a[2]) % 2) ? -1.0 : 1.0;
        const double inv = 1.0 / (fact(a[0]) * fact(a[1]) * fact(a[2]));
        ksum k = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            double m = 1.0;
            for (int d = 0; d < 3; ++d) m *= pow(Y[3 * i + d] - c[d], a[d]);
            kadd(&k, m);
        }
        M[t] = sign * inv * (k.s + k.c);
    }
}

static double mbinom(const int g[3], const int a[3]) {
    return binom_int(g[0], a[0]) * binom_int(g[1], a[1]) * binom_int(g[2], a[2]);
}

/* The Axilrod-Teller product terms: expands (b + c - a)(a + c - b)(a + b - c)
 * as a product of three linear forms in (a, b, c) and lists every monomial
 * a^i b^j c^k with its coefficient times 3/8, then the (abc)^(-3/2) term. */
int oracle_at_product_terms(double* s12, double* s13, double* s23, double* w) {
    const double L[3][3] = {{-1.0, 1.0, 1.0}, {1.0, -1.0, 1.0}, {1.0, 1.0, -1.0}};
    double cub[4][4][4];
    memset(cub, 0, sizeof(cub));
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v)
            for (int x = 0; x < 3; ++x) {
                int e[3] = {0, 0, 0};
                e[u]++;
                e[v]++;
                e[x]++;
                cub[e[0]][e[1]][e[2]] += L[0][u] * L[1][v] * L[2][x];
            }
    int n = 0;
    for (int i = 3; i >= 0; --i)
        for (int j = 3 - i; j >= 0; --j) {
            const int k = 3 - i - j;
            if (cub[i][j][k] == 0.0) continue;
            s12[n] = i - 2.5;
            s13[n] = j - 2.5;
            s23[n] = k - 2.5;
            w[n] = 0.375 * cub[i][j][k];
            ++n;
        }
    s12[n] = s13[n] = s23[n] = -1.5;
    w[n] = 1.0;
    return n + 1;
}

/* multi-index list for order p: writes n(p) triples into a (may be NULL), returns n(p) */
int oracle_ff_index(int p, int* a) {
    if (p < 0 || p > FF_PMAX) return -1;
    ff_index I;
    ff_make_index(p, &I);
    if (a)
        for (int t = 0; t < I.n; ++t)
            for (int d = 0; d < 3; ++d) a[3 * t + d] = I.a[t][d];
    return I.n;
}

int oracle_ff_derivs(const double* v0, double s, int p, double* out) {
    if (p < 0 || p > FF_PMAX) return -1;
    ff_index I;
    ff_make_index(p, &I);
    ff_derivs(&I, p, v0, s, out);
    return I.n;
}

int oracle_ff_moments(const double* Y, int64_t n, const double* c, int p, double* out) {
    if (p < 0 || p > FF_PMAX) return -1;
    ff_index I;
    ff_make_index(p, &I);
    double cc[3];
    if (c)
        memcpy(cc, c, sizeof(cc));
    else
        centre_of_mass(Y, n, cc);
    ff_moments(&I, Y, n, cc, out);
    return I.n;
}

/* The p-th order expansion at every query point. nterms = 0 selects the
 * Axilrod-Teller terms; c2, c3 = NULL selects the centres of mass. */
int oracle_farfield3(const double* Xq, int64_t nq, const double* Y2, int64_t n2, const double* Y3,
                     int64_t n3, const double* c2_in, const double* c3_in, int p, int nterms,
                     const double* s12_in, const double* s13_in, const double* s23_in,
                     const double* w_in, double* out, int nthreads) {
    if (p < 0 || p > FF_PMAX || n2 <= 0 || n3 <= 0) return -1;
    double s12[16], s13[16], s23[16], w[16];
    if (nterms <= 0) {
        nterms = oracle_at_product_terms(s12, s13, s23, w);
    } else {
        if (nterms > 16) return -1;
        memcpy(s12, s12_in, sizeof(double) * nterms);
        memcpy(s13, s13_in, sizeof(double) * nterms);
        memcpy(s23, s23_in, sizeof(double) * nterms);
        memcpy(w, w_in, sizeof(double) * nterms);
    }
    ff_index I;
    ff_make_index(p, &I);
    double c2[3], c3[3], wv[3];
    if (c2_in)
        memcpy(c2, c2_in, sizeof(c2));
    else
        centre_of_mass(Y2, n2, c2);
    if (c3_in)
        memcpy(c3, c3_in, sizeof(c3));
    else
        centre_of_mass(Y3, n3, c3);
    double M2[FF_NMAX], M3[FF_NMAX];
    ff_moments(&I, Y2, n2, c2, M2);
    ff_moments(&I, Y3, n3, c3, M3);
    for (int d = 0; d < 3; ++d) wv[d] = c2[d] - c3[d];
    double Dw[16][FF_NMAX];
    for (int m = 0; m < nterms; ++m) ff_derivs(&I, p, wv, s23[m], Dw[m]);
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t q = 0; q < nq; ++q) {
        const double* x = Xq + 3 * q;
        double u[3], v[3];
        for (int d = 0; d < 3; ++d) {
            u[d] = x[d] - c2[d];
            v[d] = x[d] - c3[d];
        }
        ksum acc = {0.0, 0.0};
        for (int m = 0; m < nterms; ++m) {
            double Du[FF_NMAX], Dv[FF_NMAX];
            ff_derivs(&I, p, u, s12[m], Du);
            ff_derivs(&I, p, v, s13[m], Dv);
            for (int ta = 0; ta < I.n; ++ta) {
                const int* a = I.a[ta];
                for (int i12 = 0; i12 <= a[0]; ++i12)
                for (int j12 = 0; j12 <= a[1]; ++j12)
                for (int k12 = 0; k12 <= a[2]; ++k12) {
                    const int a12[3] = {i12, j12, k12};
                    for (int i13 = 0; i13 <= a[0] - i12; ++i13)
                    for (int j13 = 0; j13 <= a[1] - j12; ++j13)
                    for (int k13 = 0; k13 <= a[2] - k12; ++k13) {
                        const int a13[3] = {i13, j13, k13};
                        const int a23[3] = {a[0] - i12 - i13, a[1] - j12 - j13, a[2] - k12 - k13};
                        const double dg = Du[I.idx[i12][j12][k12]] * Dv[I.idx[i13][j13][k13]] *
                                          Dw[m][I.idx[a23[0]][a23[1]][a23[2]]];
                        for (int ib = 0; ib <= a23[0]; ++ib)
                        for (int jb = 0; jb <= a23[1]; ++jb)
                        for (int kb = 0; kb <= a23[2]; ++kb) {
                            const int b[3] = {ib, jb, kb};
                            const int g2[3] = {i12 + ib, j12 + jb, k12 + kb};    /* a12 + b */
                            const int g3[3] = {a[0] - g2[0], a[1] - g2[1], a[2] - g2[2]}; /* a - a12 - b */
                            const double sign = ((ib + jb + kb) % 2) ? -1.0 : 1.0;
                            const double t = mbinom(g2, a12) * mbinom(g3, a13) *
                                             M2[I.idx[g2[0]][g2[1]][g2[2]]] *
                                             M3[I.idx[g3[0]][g3[1]][g3[2]]] * sign * dg;
                            kadd(&acc, w[m] * t);
                        }
                    }
                }
            }
        }
        out[q] = acc.s + acc.c;
    }
    return 0;
}

/* The exact sum the expansion approximates: for every query point,
 * sum_{y2 in P2} sum_{y3 in P3} of the product terms (nterms > 0), or of the
 * Axilrod-Teller phi by its cosine definition (nterms = 0). */
extern double oracle_at_phi(const double* xi, const double* xj, const double* xk);

int oracle_pairset_sum(const double* Xq, int64_t nq, const double* Y2, int64_t n2, const double* Y3,
                       int64_t n3, int nterms, const double* s12, const double* s13,
                       const double* s23, const double* w, double* out, int nthreads) {
    if (nterms > 16) return -1;
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t q = 0; q < nq; ++q) {
        const double* x = Xq + 3 * q;
        ksum acc = {0.0, 0.0};
        for (int64_t i = 0; i < n2; ++i)
            for (int64_t j = 0; j < n3; ++j) {
                const double* y2 = Y2 + 3 * i;
                const double* y3 = Y3 + 3 * j;
                if (nterms <= 0) {
                    kadd(&acc, oracle_at_phi(x, y2, y3));
                    continue;
                }
                double a = 0.0, b = 0.0, c = 0.0;
                for (int d = 0; d < 3; ++d) {
                    a += (x[d] - y2[d]) * (x[d] - y2[d]);
                    b += (x[d] - y3[d]) * (x[d] - y3[d]);
                    c += (y2[d] - y3[d]) * (y2[d] - y3[d]);
                }
                for (int m = 0; m < nterms; ++m)
                    kadd(&acc, w[m] * pow(a, s12[m]) * pow(b, s13[m]) * pow(c, s23[m]));
            }
        out[q] = acc.s + acc.c;
    }
    return 0;
}
