/*
 * Serial FP64 restatement of the multi-tree approximation.
 *
 * TEST INFRASTRUCTURE ONLY (see at_oracle.c). Plain recursion in the order
 * of the paper's algorithms; no blocking, no batching, no reordering.
 *
 *   tree   : Algorithm 1's role (bottom-up phase, Sec. 3) with the readings
 *            below: points sorted by Morton key of a 2^21 grid over the
 *            bounding cube (ties by index), ranges halved until <= leaf_size;
 *            each node has [begin, end) in depth-first rank (Fig. 2), an
 *            exact FP64 bounding box, count and centre of mass.
 *   Phi^l  : summary statistic of Sec. 4 ("lower bound on the accumulated
 *            potentials"), read for a potential of either sign as a lower
 *            bound on |Phi|: seeded before the traversal with |S(x)|, S the
 *            exact sum over triples inside x's seed node (the ancestor
 *            seed_up levels above its leaf); Phi^l(P) = min over P's points
 *            (Sec. 5, Phi^l(P) = min over children). The Monte Carlo stop
 *            test runs per particle and uses the particle's own Phi^l(x)
 *            (Algorithm 5 keeps Phi^l per particle). The paper's Phi^l +
 *            delta^l (Eq. deterministic_prune) becomes Phi^l - T_i max|phi|,
 *            and Phi^l + T_i (mu - z sigma) (Eq. prob_rel_error_termination)
 *            becomes Phi^l - T_i (|mu| + z sigma): the magnitude left after
 *            the current tuple's contribution in the worst case.
 *   recurse: Algorithm 2 (MTPotentialCanonical) from (root, root, root):
 *            CanSummarize -> Summarize; all leaves -> base case (exact);
 *            else split the internal node of largest diameter (all of its
 *            copies at once; only non-decreasing child combinations).
 *   rules  : p = 0 interval bound with the absolute rule (Sec. 4, tau/T^root)
 *            and the hybrid rule Eq. (deterministic_prune); Monte Carlo
 *            Algorithms 3-5 with the relative stop test Eq.
 *            (prob_rel_error_termination) in the reading chosen by mc_rule.
 *   top-down: node accumulators pushed to points (Sec. 3, step 3).
 *
 * Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * counter = (sorted point index, node ids, sample number), key = seed.
 *
 * Parity status: pinned by the exact-result special case eps = tau = 0, the
 * per-point tuple-count partition invariant, brute force of the interval
 * bound, the guarantees of Sec. 5 and Philox known-answer vectors; the
 * credited values (Summarize, Algorithm 5), the Monte Carlo partner draws
 * and the top-down push by an exact rebuild of the result from the record
 * of prunes (oracle_tree_potential_trace) and by uniformity of the draws
 * over the valid tuples (oracle_mc_draw).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double oracle_at_phi(const double* xi, const double* xj, const double* xk);

/* ---------------- Philox-4x32-10 ---------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform integer in [0, n) from a 32-bit draw (multiply-shift) */
static inline int64_t draw_below(uint32_t r, int64_t n) {
    return (int64_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* ---------------- tree ---------------- */
typedef struct {
    int64_t N, n_nodes, n_leaves;
    int depth;
    int64_t* perm;     /* sorted position -> original index */
    double* Xs;        /* sorted coordinates, 3 per point */
    int64_t* begin;    /* per node */
    int64_t* end;
    double* lo;        /* 3 per node */
    double* hi;
    double* cen;       /* centre of mass, 3 per node */
    double* diam2;     /* squared bbox diagonal */
    double* phil;      /* Phi^l per node */
    double* pphil;     /* Phi^l per sorted point, |S(x)| */
    double* nscale;    /* forces: A^l per node (min over its points) */
    double* pscale;    /* forces: A^l per sorted point */
} otree;

static uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu, r = 0;
    for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1u) << (3 * b);
    return r;
}

typedef struct { uint64_t key; int64_t idx; } keyidx;
static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* p = (const keyidx*)a;
    const keyidx* q = (const keyidx*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

int oracle_tree_depth(int64_t N, int leaf_size) {
    int d = 0;
    while (((N + ((int64_t)1 << d) - 1) >> d) > leaf_size) ++d;
    return d;
}

static void tree_build(const double* X, int64_t N, int leaf_size, otree* t) {
    memset(t, 0, sizeof(*t));
    t->N = N;
    double lo[3] = {X[0], X[1], X[2]}, hi[3] = {X[0], X[1], X[2]};
    for (int64_t i = 1; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            if (X[3 * i + d] < lo[d]) lo[d] = X[3 * i + d];
            if (X[3 * i + d] > hi[d]) hi[d] = X[3 * i + d];
        }
    double ext = hi[0] - lo[0];
    if (hi[1] - lo[1] > ext) ext = hi[1] - lo[1];
    if (hi[2] - lo[2] > ext) ext = hi[2] - lo[2];
    double scale = ext > 0.0 ? 2097152.0 / ext : 0.0;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        uint64_t key = 0;
        for (int d = 0; d < 3; ++d) {
            double q = floor((X[3 * i + d] - lo[d]) * scale);
            uint32_t qi = q < 0.0 ? 0u : (q > 2097151.0 ? 2097151u : (uint32_t)q);
            key |= spread3(qi) << d;
        }
        ki[i].key = key;
        ki[i].idx = i;
    }
    qsort(ki, (size_t)N, sizeof(keyidx), cmp_keyidx);
    t->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    t->Xs = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    for (int64_t s = 0; s < N; ++s) {
        t->perm[s] = ki[s].idx;
        for (int d = 0; d < 3; ++d) t->Xs[3 * s + d] = X[3 * ki[s].idx + d];
    }
    free(ki);
    t->depth = oracle_tree_depth(N, leaf_size);
    t->n_nodes = ((int64_t)2 << t->depth) - 1;
    t->n_leaves = (int64_t)1 << t->depth;
    int64_t M = t->n_nodes;
    t->begin = (int64_t*)malloc(sizeof(int64_t) * M);
    t->end = (int64_t*)malloc(sizeof(int64_t) * M);
    t->lo = (double*)malloc(sizeof(double) * 3 * M);
    t->hi = (double*)malloc(sizeof(double) * 3 * M);
    t->cen = (double*)malloc(sizeof(double) * 3 * M);
    t->diam2 = (double*)malloc(sizeof(double) * M);
    t->phil = (double*)calloc((size_t)M, sizeof(double));
    for (int d = 0; d <= t->depth; ++d) {
        int64_t first = ((int64_t)1 << d) - 1;
        for (int64_t q = 0; q < ((int64_t)1 << d); ++q) {
            int64_t v = first + q;
            t->begin[v] = (q * N) >> d;
            t->end[v] = ((q + 1) * N) >> d;
            double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
            double s[3] = {0, 0, 0};
            for (int64_t p = t->begin[v]; p < t->end[v]; ++p)
                for (int k = 0; k < 3; ++k) {
                    double x = t->Xs[3 * p + k];
                    if (x < l[k]) l[k] = x;
                    if (x > h[k]) h[k] = x;
                    s[k] += x;
                }
            int64_t cnt = t->end[v] - t->begin[v];
            for (int k = 0; k < 3; ++k) {
                t->lo[3 * v + k] = l[k];
                t->hi[3 * v + k] = h[k];
                t->cen[3 * v + k] = cnt > 0 ? s[k] / (double)cnt : 0.0;
            }
            double dx = h[0] - l[0], dy = h[1] - l[1], dz = h[2] - l[2];
            t->diam2[v] = cnt > 0 ? dx * dx + dy * dy + dz * dz : 0.0;
        }
    }
}

static void tree_free(otree* t) {
    free(t->perm); free(t->Xs); free(t->begin); free(t->end); free(t->lo);
    free(t->hi); free(t->cen); free(t->diam2); free(t->phil); free(t->pphil);
    free(t->nscale); free(t->pscale);
}

static inline int64_t node_n(const otree* t, int64_t v) { return t->end[v] - t->begin[v]; }
static inline int is_leaf(const otree* t, int64_t v) { return v >= t->n_nodes - t->n_leaves; }

/* ---------------- decision trace (for the tests' credit pins) ----------------
 * Caller-provided buffers; a full buffer keeps counting but stops writing.
 *   tri   : 4 int64 per prune: kind (0 = deterministic, 1 = Monte Carlo), P1, P2, P3
 *   mc_*  : one entry per point of a Monte Carlo prune: prune number (index
 *           into tri), sorted point index, sample mean mu, sigma_mu, samples
 */
typedef struct {
    int64_t cap_tri, n_tri;
    int64_t* tri;
    int64_t cap_mc, n_mc;
    int64_t* mc_tri;
    int64_t* mc_pt;
    double* mc_mean;   /* dim per entry: 1 (potential) or 3 (forces) */
    double* mc_sig;
    int64_t* mc_m;
} otrace;

/* ---------------- state of one solve ---------------- */
typedef struct {
    const otree* t;
    double eps, tau, alpha, z, troot, zeta;
    int m_limit, mc_rule;
    uint32_t key[2];
    double* node_acc;   /* per node */
    double* pt_acc;     /* per sorted point: base cases + Monte Carlo */
    double* pt_cmp;     /* Neumaier compensation of pt_acc */
    int64_t* node_cnt;  /* tuple counts (invariant check) */
    int64_t* pt_cnt;
    int64_t det_prunes, mc_prunes, mc_attempts, base_cases, visited, mc_samples;
    otrace* trace;      /* optional */
    int forces;         /* 1: tree forces (node_acc3, pt_acc3, force rules) */
    double* node_acc3;  /* 3 per node */
    double* pt_acc3;    /* 3 per sorted point, Neumaier-compensated by pt_cmp3 */
    double* pt_cmp3;
} osolve;

static int64_t trace_prune(osolve* S, int kind, const int64_t P[3]) {
    otrace* tr = S->trace;
    if (!tr) return -1;
    int64_t k = tr->n_tri++;
    if (k < tr->cap_tri) {
        tr->tri[4 * k] = kind;
        for (int s = 0; s < 3; ++s) tr->tri[4 * k + 1 + s] = P[s];
    }
    return k;
}

static double choose2(double n) { return n * (n - 1.0) * 0.5; }

/* T_i of Fig. 4 for the slot holding x (slot in {0,1,2}) */
static double tuples_for_slot(const int64_t P[3], const double n[3], int slot) {
    int e01 = P[0] == P[1], e12 = P[1] == P[2];
    if (e01 && e12) return choose2(n[0] - 1.0);                          /* (a) */
    if (e01) return slot == 2 ? choose2(n[0]) : (n[0] - 1.0) * n[2];     /* (b) */
    if (e12) return slot == 0 ? choose2(n[1]) : n[0] * (n[1] - 1.0);     /* (c) */
    if (slot == 0) return n[1] * n[2];                                   /* (d) */
    if (slot == 1) return n[0] * n[2];
    return n[0] * n[1];
}

/* squared minimum and maximum distance between two boxes (Fig. 3) */
static void box_d2(const otree* t, int64_t p, int64_t q, double* dl, double* du) {
    double l = 0.0, u = 0.0;
    for (int k = 0; k < 3; ++k) {
        double a = t->lo[3 * q + k] - t->hi[3 * p + k];
        double b = t->lo[3 * p + k] - t->hi[3 * q + k];
        double g = a > b ? a : b;
        if (g < 0.0) g = 0.0;
        l += g * g;
        double c = t->hi[3 * q + k] - t->lo[3 * p + k];
        double e = t->hi[3 * p + k] - t->lo[3 * q + k];
        double m = c > e ? c : e;
        u += m * m;
    }
    *dl = l;
    *du = u;
}

static void imul(double a0, double a1, double b0, double b1, double* r0, double* r1) {
    double p[4] = {a0 * b0, a0 * b1, a1 * b0, a1 * b1};
    double lo = p[0], hi = p[0];
    for (int i = 1; i < 4; ++i) {
        if (p[i] < lo) lo = p[i];
        if (p[i] > hi) hi = p[i];
    }
    *r0 = lo;
    *r1 = hi;
}

/* Interval [phi_lo, phi_hi] of the Axilrod-Teller phi over all point
 * triples of (P1, P2, P3), from the box distance bounds (Sec. 4: bounds from
 * d^l and d^u; the angular factor, which is not monotone, is bounded by
 * interval arithmetic on the law-of-cosines form, read as the split of
 * phi into parts that Sec. 4 suggests for non-monotone potentials). */
void oracle_phi_interval(const double sq_lo[3], const double sq_hi[3], double* plo, double* phi) {
    /* sq[0] = c (slots 1-2), sq[1] = b (slots 1-3), sq[2] = a (slots 2-3) */
    double cl = sq_lo[0], cu = sq_hi[0], bl = sq_lo[1], bu = sq_hi[1], al = sq_lo[2], au = sq_hi[2];
    double Cl = -1.0, Ch = 0.125;
    double Dl = 8.0 * al * bl * cl, Dh = 8.0 * au * bu * cu;
    if (Dl > 0.0) {
        double U0 = bl + cl - au, U1 = bu + cu - al;
        double V0 = al + cl - bu, V1 = au + cu - bl;
        double W0 = al + bl - cu, W1 = au + bu - cl;
        double p0, p1, q0, q1;
        imul(U0, U1, V0, V1, &p0, &p1);
        imul(p0, p1, W0, W1, &q0, &q1);
        double lo = q0 / Dl < q0 / Dh ? q0 / Dl : q0 / Dh;
        double hi = q1 / Dl > q1 / Dh ? q1 / Dl : q1 / Dh;
        if (lo > Cl) Cl = lo;
        if (hi < Ch) Ch = hi;
        if (Cl > Ch) Cl = Ch; /* empty after rounding: keep a point */
    }
    double nl = 1.0 + 3.0 * Cl, nh = 1.0 + 3.0 * Ch;
    double Sl = al * bl * cl, Sh = au * bu * cu;
    double R3l = Sl * sqrt(Sl), R3h = Sh * sqrt(Sh);
    double hiv = nh >= 0.0 ? (R3l > 0.0 ? nh / R3l : INFINITY) : nh / R3h;
    double lov = nl >= 0.0 ? nl / R3h : (R3l > 0.0 ? nl / R3l : -INFINITY);
    *phi = hiv + fabs(hiv) * 1e-13;
    *plo = lov - fabs(lov) * 1e-13;
}

/* two-sided normal quantile z with P(|Z| > z) = alpha, by bisection on erfc */
double oracle_z_two_sided(double alpha) {
    if (!(alpha > 0.0)) return INFINITY;
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (erfc(mid / sqrt(2.0)) > alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* --- MC: draw one tuple containing sorted point x from the other slots --- */
static void draw_partners(const osolve* S, const int64_t P[3], int slot, int64_t x,
                          uint32_t r0, uint32_t r1, int64_t* y, int64_t* z) {
    const otree* t = S->t;
    int e01 = P[0] == P[1], e12 = P[1] == P[2];
    int64_t b0 = t->begin[P[0]], b1 = t->begin[P[1]], b2 = t->begin[P[2]];
    int64_t n0 = node_n(t, P[0]), n1 = node_n(t, P[1]), n2 = node_n(t, P[2]);
    /* pair of distinct points from [b, b+n) excluding x if inside */
#define PAIR_FROM(b, n, excl)                                          \
    do {                                                               \
        int64_t m_ = (n) - ((excl) ? 1 : 0);                           \
        int64_t u_ = draw_below(r0, m_), w_ = draw_below(r1, m_ - 1);  \
        if (w_ >= u_) ++w_;                                            \
        if (excl) {                                                    \
            if ((b) + u_ >= x) ++u_;                                   \
            if ((b) + w_ >= x) ++w_;                                   \
        }                                                              \
        *y = (b) + u_;                                                 \
        *z = (b) + w_;                                                 \
    } while (0)
    if (e01 && e12) {                          /* (a): pair from P \ {x} */
        PAIR_FROM(b0, n0, 1);
    } else if (e01) {                          /* (b) P,P,Q */
        if (slot == 2) {
            PAIR_FROM(b0, n0, 0);
        } else {
            int64_t u = draw_below(r0, n0 - 1);
            if (b0 + u >= x) ++u;
            *y = b0 + u;
            *z = b2 + draw_below(r1, n2);
        }
    } else if (e12) {                          /* (c) P,Q,Q */
        if (slot == 0) {
            PAIR_FROM(b1, n1, 0);
        } else {
            *y = b0 + draw_below(r0, n0);
            int64_t u = draw_below(r1, n1 - 1);
            if (b1 + u >= x) ++u;
            *z = b1 + u;
        }
    } else {                                   /* (d) distinct */
        int64_t bb[3] = {b0, b1, b2}, nn[3] = {n0, n1, n2};
        int o1 = slot == 0 ? 1 : 0, o2 = slot == 2 ? 1 : 2;
        *y = bb[o1] + draw_below(r0, nn[o1]);
        *z = bb[o2] + draw_below(r1, nn[o2]);
    }
#undef PAIR_FROM
}

/* Algorithm 4 for point x (sorted index) of slot `slot`; returns 1 if the
 * point passes, and its estimate T_i * mu in *est (mu, sigma_mu and the
 * number of samples in mus[0..2]). */
static int mc_point(osolve* S, const int64_t P[3], int slot, int64_t x, double Ti, double phil,
                    double* est, double mus[3]) {
    const otree* t = S->t;
    double mean = 0.0, m2 = 0.0;
    int m = 0, pass = 0;
    double sig = 0.0;
    uint32_t r[4] = {0, 0, 0, 0};
    for (;;) {
        /* one Philox call per two samples: sample m uses words 2(m%2), 2(m%2)+1
           of the call with counter index m/2 */
        if ((m & 1) == 0) {
            int c = m >> 1;
            uint32_t ctr[4] = {(uint32_t)x, (uint32_t)P[0] | ((uint32_t)(c & 0xFF) << 24),
                               (uint32_t)P[1] | ((uint32_t)((c >> 8) & 0xFF) << 24), (uint32_t)P[2]};
            oracle_philox4x32_10(ctr, S->key, r);
        }
        int64_t y, z;
        draw_partners(S, P, slot, x, (m & 1) ? r[2] : r[0], (m & 1) ? r[3] : r[1], &y, &z);
        double f = oracle_at_phi(t->Xs + 3 * x, t->Xs + 3 * y, t->Xs + 3 * z);
        ++m;
        double dlt = f - mean;
        mean += dlt * (1.0 / (double)m);                 /* running mean */
        m2 += dlt * (f - mean);                          /* running sum of squares */
        if (m >= 2 && (m >= 30 || m >= S->m_limit)) { /* the loop can only end here */
            /* sigma_mu = s / sqrt(m), s^2 = m2 / (m - 1) (sample variance with m-1) */
            sig = sqrt(m2 * (1.0 / (double)(m - 1)) * (1.0 / (double)m));
            double lhs = S->z * sig, rhs;
            double lb = phil - Ti * (fabs(mean) + S->z * sig);
            if (lb < 0.0) lb = 0.0;
            if (S->mc_rule == 1) /* as printed: T_i z sigma <= (eps lb + tau T_i) / T^root */
                rhs = (S->eps * lb / Ti + S->tau) * (1.0 / S->troot);
            else                 /* T_i on both terms */
                rhs = (S->eps * lb + S->tau) * (1.0 / S->troot);
            pass = lhs <= rhs;
            if ((pass && m >= 30) || m >= S->m_limit) break;
        } else if (m >= S->m_limit) {
            pass = 0;
            break;
        }
    }
    S->mc_samples += m;
    *est = Ti * mean;
    mus[0] = mean;
    mus[1] = sig;
    mus[2] = (double)m;
    return pass;
}

/* Neumaier-compensated per-point accumulation */
static void pt_add(osolve* S, int64_t p, double x) {
    double a = S->pt_acc[p], t = a + x;
    if (fabs(a) >= fabs(x)) S->pt_cmp[p] += (a - t) + x;
    else S->pt_cmp[p] += (x - t) + a;
    S->pt_acc[p] = t;
}

static void base_case_forces(osolve* S, const int64_t P[3]);

static void base_case(osolve* S, const int64_t P[3]) {
    if (S->forces) {
        base_case_forces(S, P);
        return;
    }
    const otree* t = S->t;
    int e01 = P[0] == P[1], e12 = P[1] == P[2];
    for (int64_t i = t->begin[P[0]]; i < t->end[P[0]]; ++i)
        for (int64_t j = t->begin[P[1]]; j < t->end[P[1]]; ++j) {
            if (e01 && j <= i) continue;
            for (int64_t k = t->begin[P[2]]; k < t->end[P[2]]; ++k) {
                if (e12 && k <= j) continue;
                double f = oracle_at_phi(t->Xs + 3 * i, t->Xs + 3 * j, t->Xs + 3 * k);
                pt_add(S, i, f); pt_add(S, j, f); pt_add(S, k, f);
                if (S->pt_cnt) { S->pt_cnt[i]++; S->pt_cnt[j]++; S->pt_cnt[k]++; }
            }
        }
    S->base_cases++;
}

static void recurse(osolve* S, int64_t P1, int64_t P2, int64_t P3);

static int try_summarize_forces(osolve* S, const int64_t P[3]);

static int try_summarize(osolve* S, const int64_t P[3]) {
    if (S->forces) return try_summarize_forces(S, P);
    const otree* t = S->t;
    double n[3] = {(double)node_n(t, P[0]), (double)node_n(t, P[1]), (double)node_n(t, P[2])};
    double T[3];
    for (int s = 0; s < 3; ++s) T[s] = tuples_for_slot(P, n, s);
    /* distinct slots: slot s is "first of its node" if s == 0 or P[s] != P[s-1] */
    int first[3] = {1, P[1] != P[0], P[2] != P[1]};
    /* ---- deterministic p = 0 rule ---- */
    double sl[3], sh[3];
    box_d2(t, P[0], P[1], &sl[0], &sh[0]);
    box_d2(t, P[0], P[2], &sl[1], &sh[1]);
    box_d2(t, P[1], P[2], &sl[2], &sh[2]);
    double plo, phi_hi;
    oracle_phi_interval(sl, sh, &plo, &phi_hi);
    double width = phi_hi - plo;
    double lb = INFINITY, amax = fabs(plo) > fabs(phi_hi) ? fabs(plo) : fabs(phi_hi);
    for (int s = 0; s < 3; ++s) {
        if (!first[s]) continue;
        double v = t->phil[P[s]] - T[s] * amax;
        if (v < lb) lb = v;
    }
    double budget = (S->eps * (lb > 0.0 ? lb : 0.0) + S->tau) / S->troot;
    if (width <= budget) {
        double f = oracle_at_phi(t->cen + 3 * P[0], t->cen + 3 * P[1], t->cen + 3 * P[2]);
        for (int s = 0; s < 3; ++s) {
            if (!first[s]) continue;
            S->node_acc[P[s]] += T[s] * f;
            if (S->node_cnt) S->node_cnt[P[s]] += (int64_t)T[s];
        }
        S->det_prunes++;
        trace_prune(S, 0, P);
        return 1;
    }
    /* ---- Monte Carlo rule (Algorithm 3) ---- */
    if (S->alpha > 0.0) {
        double tmin = T[0];
        for (int s = 1; s < 3; ++s) if (T[s] < tmin) tmin = T[s];
        if (tmin >= 1.0 && S->zeta * S->m_limit <= tmin) { /* every slot has tuples to draw */
            S->mc_attempts++;
            int64_t total = 0;
            for (int s = 0; s < 3; ++s) if (first[s]) total += node_n(t, P[s]);
            double* est = (double*)malloc(sizeof(double) * (size_t)total);
            double* mus = (double*)malloc(sizeof(double) * 3 * (size_t)total);
            int64_t q = 0;
            int ok = 1;
            for (int s = 0; s < 3 && ok; ++s) {
                if (!first[s]) continue;
                for (int64_t x = t->begin[P[s]]; x < t->end[P[s]]; ++x) {
                    if (!mc_point(S, P, s, x, T[s], t->pphil[x], &est[q], mus + 3 * q)) {
                        ok = 0;
                        break;
                    }
                    ++q;
                }
            }
            if (ok) { /* Algorithm 5 */
                int64_t k = trace_prune(S, 1, P);
                q = 0;
                for (int s = 0; s < 3; ++s) {
                    if (!first[s]) continue;
                    for (int64_t x = t->begin[P[s]]; x < t->end[P[s]]; ++x) {
                        if (S->trace) {
                            otrace* tr = S->trace;
                            int64_t e = tr->n_mc++;
                            if (e < tr->cap_mc) {
                                tr->mc_tri[e] = k;
                                tr->mc_pt[e] = x;
                                tr->mc_mean[e] = mus[3 * q];
                                tr->mc_sig[e] = mus[3 * q + 1];
                                tr->mc_m[e] = (int64_t)mus[3 * q + 2];
                            }
                        }
                        pt_add(S, x, est[q++]);
                        if (S->pt_cnt) S->pt_cnt[x] += (int64_t)T[s];
                    }
                }
                S->mc_prunes++;
            }
            free(est);
            free(mus);
            if (ok) return 1;
        }
    }
    return 0;
}

static void recurse(osolve* S, int64_t P1, int64_t P2, int64_t P3) {
    const otree* t = S->t;
    int64_t P[3] = {P1, P2, P3};
    S->visited++;
    if (try_summarize(S, P)) return;
    if (is_leaf(t, P1) && is_leaf(t, P2) && is_leaf(t, P3)) {
        base_case(S, P);
        return;
    }
    /* split the internal node of largest diameter (first slot on ties) */
    int ks = -1;
    double best = -1.0;
    for (int s = 0; s < 3; ++s) {
        if (is_leaf(t, P[s])) continue;
        if (t->diam2[P[s]] > best) { best = t->diam2[P[s]]; ks = s; }
    }
    int64_t v = P[ks], L = 2 * v + 1, R = 2 * v + 2;
    int e01 = P1 == P2, e12 = P2 == P3;
    if (e01 && e12) {                     /* (v, v, v) */
        recurse(S, L, L, L); recurse(S, L, L, R); recurse(S, L, R, R); recurse(S, R, R, R);
    } else if (e01 && ks <= 1) {          /* (v, v, Q) */
        recurse(S, L, L, P3); recurse(S, L, R, P3); recurse(S, R, R, P3);
    } else if (e12 && ks >= 1) {          /* (Q, v, v) */
        recurse(S, P1, L, L); recurse(S, P1, L, R); recurse(S, P1, R, R);
    } else {                              /* v occupies one slot */
        int64_t A[3] = {P1, P2, P3}, B[3] = {P1, P2, P3};
        A[ks] = L; B[ks] = R;
        recurse(S, A[0], A[1], A[2]); recurse(S, B[0], B[1], B[2]);
    }
}


/* ======================= tree forces (no counterpart in the paper) =======================
 * F(x) = -sum over the tuples {y, z} containing x of grad_x phi(x, y, z), the
 * negative gradient of the total energy. The recursion is Algorithm 2 with
 * the same splits; the value a prune credits and the rules that allow it are
 * those of the force error criterion (one component d at a time)
 *     |F~_d(x) - F_d(x)| <= eps S(x) + tau,
 *     S(x) = sum over the tuples containing x of |grad_x phi|_2,
 * a sum of magnitudes, which cancelling terms cannot shrink.
 *   seed  : A^l(x) = the same sum over the tuples inside x's seed node, a
 *           lower bound of S(x) (non-negative terms over a subset of the
 *           tuples); A^l(P) = min over P's points.
 *   p = 0 : with u, v the edges at slot s and the pair-vector form of the
 *           gradient, |grad_x phi|_2 <= 3R/r_u (|5t-1| + 2) + 3R/r_v (|5t-1| + 2)
 *           <= 18 R_max (1/d^l_u + 1/d^l_v) = M_s over all point triples of
 *           the boxes (|5t - 1| <= 4 because the cosine product lies in
 *           [-1, 1/8]); crediting T_s grad phi(c1, c2, c3) to slot s errs by at
 *           most 2 M_s per tuple and component, so a triple is summarized iff
 *           2 M_s <= (eps A^l(P_s) + tau) / T^root for every distinct slot.
 *   MC    : Algorithm 4 with the three components of grad_x phi as the
 *           sample; a point passes iff z sigma_d <= (eps A^l(x) + tau)/T^root
 *           for d = 1, 2, 3 (sigma_d from the (m - 1) sample variance).
 * Every credit is -T times a gradient (a force), pushed top-down like the
 * potential's node accumulators.
 */
void oracle_at_grad(const double* xi, const double* xj, const double* xk, double* g);

static double grad_norm(const double* xi, const double* xj, const double* xk) {
    double g[3];
    oracle_at_grad(xi, xj, xk, g);
    return sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

/* A^l: exact sum of |grad_x phi|_2 over the tuples inside each point's seed node */
static void seed_scale(otree* t, int seed_up) {
    int64_t N = t->N;
    t->pscale = (double*)calloc((size_t)N, sizeof(double));
    int sd = t->depth - seed_up;
    if (sd < 0) sd = 0;
    int64_t first = ((int64_t)1 << sd) - 1;
    for (int64_t q = 0; q < ((int64_t)1 << sd); ++q) {
        int64_t v = first + q, b = t->begin[v], e = t->end[v];
        int64_t p;
#pragma omp parallel for schedule(dynamic, 8)
        for (p = b; p < e; ++p) {
            double acc = 0.0, cmp = 0.0;
            for (int64_t y = b; y < e; ++y) {
                if (y == p) continue;
                for (int64_t z = y + 1; z < e; ++z) {
                    if (z == p) continue;
                    double f = grad_norm(t->Xs + 3 * p, t->Xs + 3 * y, t->Xs + 3 * z);
                    double s2 = acc + f;
                    cmp += fabs(acc) >= f ? (acc - s2) + f : (f - s2) + acc;
                    acc = s2;
                }
            }
            t->pscale[p] = acc + cmp;
        }
    }
    t->nscale = (double*)malloc(sizeof(double) * (size_t)t->n_nodes);
    for (int64_t v = 0; v < t->n_nodes; ++v) {
        double m = INFINITY;
        for (int64_t p = t->begin[v]; p < t->end[v]; ++p) if (t->pscale[p] < m) m = t->pscale[p];
        t->nscale[v] = t->begin[v] < t->end[v] ? m : 0.0;
    }
}

static void pt_add3(osolve* S, int64_t p, const double g[3], double sgn) {
    for (int d = 0; d < 3; ++d) {
        double a = S->pt_acc3[3 * p + d], x = sgn * g[d], t2 = a + x;
        if (fabs(a) >= fabs(x)) S->pt_cmp3[3 * p + d] += (a - t2) + x;
        else S->pt_cmp3[3 * p + d] += (x - t2) + a;
        S->pt_acc3[3 * p + d] = t2;
    }
}

/* gradient of phi with respect to the point of slot s of (a0, a1, a2) */
static void grad_slot(const double* a0, const double* a1, const double* a2, int s, double g[3]) {
    if (s == 0) oracle_at_grad(a0, a1, a2, g);
    else if (s == 1) oracle_at_grad(a1, a0, a2, g);
    else oracle_at_grad(a2, a0, a1, g);
}

static void base_case_forces(osolve* S, const int64_t P[3]) {
    const otree* t = S->t;
    int e01 = P[0] == P[1], e12 = P[1] == P[2];
    for (int64_t i = t->begin[P[0]]; i < t->end[P[0]]; ++i)
        for (int64_t j = t->begin[P[1]]; j < t->end[P[1]]; ++j) {
            if (e01 && j <= i) continue;
            for (int64_t k = t->begin[P[2]]; k < t->end[P[2]]; ++k) {
                if (e12 && k <= j) continue;
                const double *a = t->Xs + 3 * i, *b = t->Xs + 3 * j, *c = t->Xs + 3 * k;
                double g[3];
                grad_slot(a, b, c, 0, g); pt_add3(S, i, g, -1.0);
                grad_slot(a, b, c, 1, g); pt_add3(S, j, g, -1.0);
                grad_slot(a, b, c, 2, g); pt_add3(S, k, g, -1.0);
                if (S->pt_cnt) { S->pt_cnt[i]++; S->pt_cnt[j]++; S->pt_cnt[k]++; }
            }
        }
    S->base_cases++;
}

/* Algorithm 4 for point x with the gradient as a 3-component sample; returns 1
 * if the point passes, its force estimate -T_i mu in est[3] and mu, sigma_mu
 * (3 each) and the sample count in mus[0..6]. */
static int mc_point_forces(osolve* S, const int64_t P[3], int slot, int64_t x, double Ti,
                           double ascale, double est[3], double mus[7]) {
    const otree* t = S->t;
    double mean[3] = {0, 0, 0}, m2[3] = {0, 0, 0}, sig[3] = {0, 0, 0};
    int m = 0, pass = 0;
    uint32_t r[4] = {0, 0, 0, 0};
    const double rhs = (S->eps * ascale + S->tau) * (1.0 / S->troot);
    for (;;) {
        if ((m & 1) == 0) {
            int c = m >> 1;
            uint32_t ctr[4] = {(uint32_t)x, (uint32_t)P[0] | ((uint32_t)(c & 0xFF) << 24),
                               (uint32_t)P[1] | ((uint32_t)((c >> 8) & 0xFF) << 24), (uint32_t)P[2]};
            oracle_philox4x32_10(ctr, S->key, r);
        }
        int64_t y, z;
        draw_partners(S, P, slot, x, (m & 1) ? r[2] : r[0], (m & 1) ? r[3] : r[1], &y, &z);
        double g[3];
        oracle_at_grad(t->Xs + 3 * x, t->Xs + 3 * y, t->Xs + 3 * z, g);
        ++m;
        for (int d = 0; d < 3; ++d) {
            double dlt = g[d] - mean[d];
            mean[d] += dlt * (1.0 / (double)m);
            m2[d] += dlt * (g[d] - mean[d]);
        }
        if (m >= 2 && (m >= 30 || m >= S->m_limit)) {
            pass = 1;
            for (int d = 0; d < 3; ++d) {
                sig[d] = sqrt(m2[d] * (1.0 / (double)(m - 1)) * (1.0 / (double)m));
                if (!(S->z * sig[d] <= rhs)) pass = 0;
            }
            if ((pass && m >= 30) || m >= S->m_limit) break;
        } else if (m >= S->m_limit) {
            pass = 0;
            break;
        }
    }
    S->mc_samples += m;
    for (int d = 0; d < 3; ++d) {
        est[d] = -Ti * mean[d];
        mus[d] = mean[d];
        mus[3 + d] = sig[d];
    }
    mus[6] = (double)m;
    return pass;
}

static int try_summarize_forces(osolve* S, const int64_t P[3]) {
    const otree* t = S->t;
    double n[3] = {(double)node_n(t, P[0]), (double)node_n(t, P[1]), (double)node_n(t, P[2])};
    double T[3];
    for (int s = 0; s < 3; ++s) T[s] = tuples_for_slot(P, n, s);
    int first[3] = {1, P[1] != P[0], P[2] != P[1]};
    /* ---- deterministic p = 0 rule for the gradient ---- */
    double sl[3], sh[3];
    box_d2(t, P[0], P[1], &sl[0], &sh[0]);
    box_d2(t, P[0], P[2], &sl[1], &sh[1]);
    box_d2(t, P[1], P[2], &sl[2], &sh[2]);
    if (sl[0] > 0.0 && sl[1] > 0.0 && sl[2] > 0.0) {
        double prod = sl[0] * sl[1] * sl[2];
        double rmax = 1.0 / (prod * sqrt(prod));
        double inv[3] = {1.0 / sqrt(sl[0]), 1.0 / sqrt(sl[1]), 1.0 / sqrt(sl[2])};
        /* edges at each slot: slot 0 -> (0-1, 0-2), slot 1 -> (0-1, 1-2), slot 2 -> (0-2, 1-2) */
        double M[3] = {18.0 * rmax * (inv[0] + inv[1]), 18.0 * rmax * (inv[0] + inv[2]),
                       18.0 * rmax * (inv[1] + inv[2])};
        int ok = 1;
        for (int s = 0; s < 3; ++s) {
            if (!first[s]) continue;
            double budget = (S->eps * t->nscale[P[s]] + S->tau) / S->troot;
            if (!(2.0 * M[s] <= budget)) ok = 0;
        }
        if (ok) {
            const double *c0 = t->cen + 3 * P[0], *c1 = t->cen + 3 * P[1], *c2 = t->cen + 3 * P[2];
            for (int s = 0; s < 3; ++s) {
                if (!first[s]) continue;
                double g[3];
                grad_slot(c0, c1, c2, s, g);
                for (int d = 0; d < 3; ++d) S->node_acc3[3 * P[s] + d] += -T[s] * g[d];
                if (S->node_cnt) S->node_cnt[P[s]] += (int64_t)T[s];
            }
            S->det_prunes++;
            trace_prune(S, 0, P);
            return 1;
        }
    }
    /* ---- Monte Carlo rule (Algorithm 3) ---- */
    if (S->alpha > 0.0) {
        double tmin = T[0];
        for (int s = 1; s < 3; ++s) if (T[s] < tmin) tmin = T[s];
        if (tmin >= 1.0 && S->zeta * S->m_limit <= tmin) {
            S->mc_attempts++;
            int64_t total = 0;
            for (int s = 0; s < 3; ++s) if (first[s]) total += node_n(t, P[s]);
            double* est = (double*)malloc(sizeof(double) * 3 * (size_t)total);
            double* mus = (double*)malloc(sizeof(double) * 7 * (size_t)total);
            int64_t q = 0;
            int ok = 1;
            for (int s = 0; s < 3 && ok; ++s) {
                if (!first[s]) continue;
                for (int64_t x = t->begin[P[s]]; x < t->end[P[s]]; ++x) {
                    if (!mc_point_forces(S, P, s, x, T[s], t->pscale[x], est + 3 * q,
                                         mus + 7 * q)) {
                        ok = 0;
                        break;
                    }
                    ++q;
                }
            }
            if (ok) { /* Algorithm 5 */
                int64_t k = trace_prune(S, 1, P);
                q = 0;
                for (int s = 0; s < 3; ++s) {
                    if (!first[s]) continue;
                    for (int64_t x = t->begin[P[s]]; x < t->end[P[s]]; ++x) {
                        if (S->trace) {
                            otrace* tr = S->trace;
                            int64_t e = tr->n_mc++;
                            if (e < tr->cap_mc) {
                                tr->mc_tri[e] = k;
                                tr->mc_pt[e] = x;
                                for (int d = 0; d < 3; ++d) {
                                    tr->mc_mean[3 * e + d] = mus[7 * q + d];
                                    tr->mc_sig[3 * e + d] = mus[7 * q + 3 + d];
                                }
                                tr->mc_m[e] = (int64_t)mus[7 * q + 6];
                            }
                        }
                        pt_add3(S, x, est + 3 * q, 1.0);
                        ++q;
                        if (S->pt_cnt) S->pt_cnt[x] += (int64_t)T[s];
                    }
                }
                S->mc_prunes++;
            }
            free(est);
            free(mus);
            if (ok) return 1;
        }
    }
    return 0;
}

int oracle_phi(const double* X, int64_t N, const int64_t* idx, int64_t n_idx, double* out,
               double* absout, int nthreads);

/* exact seed: for each point, the exact sum (Eq. 1) over the triples inside
 * its seed node, i.e. Phi of the point within the seed node's point set */
static void seed_phil(otree* t, int seed_up) {
    int64_t N = t->N;
    double* seed = (double*)calloc((size_t)N, sizeof(double));
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t p = 0; p < N; ++p) idx[p] = p;
    int sd = t->depth - seed_up;
    if (sd < 0) sd = 0;
    int64_t first = ((int64_t)1 << sd) - 1;
    for (int64_t q = 0; q < ((int64_t)1 << sd); ++q) {
        int64_t v = first + q, b = t->begin[v], n = t->end[v] - t->begin[v];
        oracle_phi(t->Xs + 3 * b, n, idx, n, seed + b, NULL, 0);
    }
    free(idx);
    t->pphil = (double*)malloc(sizeof(double) * (size_t)N);
    for (int64_t p = 0; p < N; ++p) t->pphil[p] = fabs(seed[p]);
    for (int64_t v = 0; v < t->n_nodes; ++v) {
        double m = INFINITY;
        for (int64_t p = t->begin[v]; p < t->end[v]; ++p) if (fabs(seed[p]) < m) m = fabs(seed[p]);
        t->phil[v] = t->begin[v] < t->end[v] ? m : 0.0;
    }
    free(seed);
}

/*
 * Tree approximation of Phi for all particles (original order).
 *   absolute != 0: eps is ignored and tau is the bound (Def. 2.1);
 *   otherwise Def. 2.3 with (eps, tau), alpha = 0 deterministic.
 *   counts (optional, int64 per particle): tuples credited to each particle.
 *   stats (optional, int64[6]): visited, det prunes, MC prunes, MC attempts,
 *   base cases, MC samples.
 */
static int tree_solve(const double* X, int64_t N, double eps, double tau, double alpha,
                      int leaf_size, int m_limit, double zeta, uint64_t seed, int mc_rule,
                      int seed_up, int forces, double* out, int64_t* counts, int64_t* stats,
                      otrace* trace) {
    const int dim = forces ? 3 : 1;
    if (N < 3) {
        for (int64_t i = 0; i < N * dim; ++i) out[i] = 0.0;
        for (int64_t i = 0; i < N; ++i) if (counts) counts[i] = 0;
        return 0;
    }
    otree t;
    tree_build(X, N, leaf_size, &t);
    if (forces) seed_scale(&t, seed_up);
    else seed_phil(&t, seed_up);
    osolve S;
    memset(&S, 0, sizeof(S));
    S.t = &t;
    S.eps = eps; S.tau = tau; S.alpha = alpha; S.zeta = zeta;
    S.m_limit = m_limit; S.mc_rule = mc_rule;
    S.trace = trace;
    S.forces = forces;
    S.troot = choose2((double)(N - 1));
    S.z = oracle_z_two_sided(alpha);
    S.key[0] = (uint32_t)seed; S.key[1] = (uint32_t)(seed >> 32);
    S.node_acc = (double*)calloc((size_t)t.n_nodes, sizeof(double));
    S.pt_acc = (double*)calloc((size_t)N, sizeof(double));
    S.pt_cmp = (double*)calloc((size_t)N, sizeof(double));
    if (forces) {
        S.node_acc3 = (double*)calloc(3 * (size_t)t.n_nodes, sizeof(double));
        S.pt_acc3 = (double*)calloc(3 * (size_t)N, sizeof(double));
        S.pt_cmp3 = (double*)calloc(3 * (size_t)N, sizeof(double));
    }
    if (counts) {
        S.node_cnt = (int64_t*)calloc((size_t)t.n_nodes, sizeof(int64_t));
        S.pt_cnt = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    }
    recurse(&S, 0, 0, 0);
    /* top-down: push node accumulators to points */
    for (int64_t v = 0; v < t.n_nodes; ++v) {
        if (v > 0) {
            int64_t par = (v - 1) / 2;
            S.node_acc[v] += S.node_acc[par];
            if (forces)
                for (int d = 0; d < 3; ++d) S.node_acc3[3 * v + d] += S.node_acc3[3 * par + d];
            if (counts) S.node_cnt[v] += S.node_cnt[par];
        }
    }
    int64_t lf = t.n_nodes - t.n_leaves;
    for (int64_t v = lf; v < t.n_nodes; ++v)
        for (int64_t p = t.begin[v]; p < t.end[v]; ++p) {
            if (forces)
                for (int d = 0; d < 3; ++d)
                    out[3 * t.perm[p] + d] = (S.pt_acc3[3 * p + d] + S.pt_cmp3[3 * p + d]) +
                                             S.node_acc3[3 * v + d];
            else
                out[t.perm[p]] = (S.pt_acc[p] + S.pt_cmp[p]) + S.node_acc[v];
            if (counts) counts[t.perm[p]] = S.pt_cnt[p] + S.node_cnt[v];
        }
    if (stats) {
        stats[0] = S.visited; stats[1] = S.det_prunes; stats[2] = S.mc_prunes;
        stats[3] = S.mc_attempts; stats[4] = S.base_cases; stats[5] = S.mc_samples;
    }
    free(S.node_acc); free(S.pt_acc); free(S.pt_cmp);
    free(S.node_acc3); free(S.pt_acc3); free(S.pt_cmp3);
    if (counts) { free(S.node_cnt); free(S.pt_cnt); }
    tree_free(&t);
    return 0;
}

int oracle_tree_potential(const double* X, int64_t N, double eps, double tau, double alpha,
                          int leaf_size, int m_limit, double zeta, uint64_t seed, int mc_rule,
                          int seed_up, double* out, int64_t* counts, int64_t* stats) {
    return tree_solve(X, N, eps, tau, alpha, leaf_size, m_limit, zeta, seed, mc_rule, seed_up, 0,
                      out, counts, stats, NULL);
}

/*
 * Tree approximation of the forces F = -grad E (3 per particle, original
 * order) under the force criterion above; arguments as oracle_tree_potential
 * (no mc_rule: the force stop test has one form).
 */
int oracle_tree_forces(const double* X, int64_t N, double eps, double tau, double alpha,
                       int leaf_size, int m_limit, double zeta, uint64_t seed, int seed_up,
                       double* out3, int64_t* counts, int64_t* stats) {
    return tree_solve(X, N, eps, tau, alpha, leaf_size, m_limit, zeta, seed, 0, seed_up, 1, out3,
                      counts, stats, NULL);
}

/* The same solve (forces = 0) or the tree forces (forces = 1, out has 3 per
 * particle), recording every prune (see otrace) into caller buffers: tri
 * (4 x cap_tri int64), and per Monte Carlo point mc_tri, mc_pt, mc_m (int64)
 * and mc_mean, mc_sig (1 or 3 doubles each), cap_mc entries. n_out[0..1]
 * receive the number of prunes and of Monte Carlo point entries (which may
 * exceed the capacities; entries past them are not written). */
int oracle_tree_potential_trace(const double* X, int64_t N, double eps, double tau, double alpha,
                                int leaf_size, int m_limit, double zeta, uint64_t seed,
                                int mc_rule, int seed_up, int forces, double* out, int64_t* stats,
                                int64_t* tri, int64_t cap_tri, int64_t* mc_tri, int64_t* mc_pt,
                                double* mc_mean, double* mc_sig, int64_t* mc_m, int64_t cap_mc,
                                int64_t* n_out) {
    otrace tr;
    memset(&tr, 0, sizeof(tr));
    tr.cap_tri = cap_tri; tr.tri = tri;
    tr.cap_mc = cap_mc; tr.mc_tri = mc_tri; tr.mc_pt = mc_pt;
    tr.mc_mean = mc_mean; tr.mc_sig = mc_sig; tr.mc_m = mc_m;
    int rc = tree_solve(X, N, eps, tau, alpha, leaf_size, m_limit, zeta, seed, mc_rule, seed_up,
                        forces, out, NULL, stats, &tr);
    n_out[0] = tr.n_tri;
    n_out[1] = tr.n_mc;
    return rc;
}

/* The Monte Carlo partner draw alone (for tests): node triple P (node ids,
 * equal ids = the same node) with point ranges [begin[s], end[s]) per slot,
 * point x of slot `slot`; draw n partner pairs from the 32-bit words
 * r[2m], r[2m+1] into yz[2m], yz[2m+1]. */
int oracle_mc_draw(const int64_t P[3], const int64_t begin[3], const int64_t end[3], int slot,
                   int64_t x, const uint32_t* r, int64_t n, int64_t* yz) {
    int64_t b[3], e[3], Q[3];
    Q[0] = 0;
    Q[1] = P[1] == P[0] ? 0 : 1;
    Q[2] = P[2] == P[1] ? Q[1] : 2;
    for (int s = 0; s < 3; ++s) {
        b[Q[s]] = begin[s];
        e[Q[s]] = end[s];
    }
    otree t;
    memset(&t, 0, sizeof(t));
    t.begin = b;
    t.end = e;
    osolve S;
    memset(&S, 0, sizeof(S));
    S.t = &t;
    for (int64_t m = 0; m < n; ++m)
        draw_partners(&S, Q, slot, x, r[2 * m], r[2 * m + 1], yz + 2 * m, yz + 2 * m + 1);
    return 0;
}

/* The tree alone: sorted permutation and node table (for tests). */
int oracle_tree_layout(const double* X, int64_t N, int leaf_size, int64_t* perm,
                       int64_t* begin, int64_t* end, double* lo, double* hi, double* cen) {
    otree t;
    tree_build(X, N, leaf_size, &t);
    memcpy(perm, t.perm, sizeof(int64_t) * (size_t)N);
    memcpy(begin, t.begin, sizeof(int64_t) * (size_t)t.n_nodes);
    memcpy(end, t.end, sizeof(int64_t) * (size_t)t.n_nodes);
    memcpy(lo, t.lo, sizeof(double) * 3 * (size_t)t.n_nodes);
    memcpy(hi, t.hi, sizeof(double) * 3 * (size_t)t.n_nodes);
    memcpy(cen, t.cen, sizeof(double) * 3 * (size_t)t.n_nodes);
    tree_free(&t);
    return 0;
}
