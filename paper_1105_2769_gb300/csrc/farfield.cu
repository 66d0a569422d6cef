// Three-body far-field expansion of Axilrod-Teller sums (§3.2, Eq.
// truncated_three_body_farfield_expansion), orders p = 0..6.
//
// For query points x and two source sets P2, P3 with centres of mass c2, c3
// the p-th order expansion of
//   Phi(x; P2 x P3) = sum_{y2 in P2} sum_{y3 in P3} phi(x, y2, y3).
//
// Axilrod-Teller as products of pairwise powers. With a = |x - y2|^2,
// b = |x - y3|^2, c = |y2 - y3|^2 the law of cosines turns the cosine product
// into (b + c - a)(a + c - b)(a + b - c) / (8abc), so
//   phi = (abc)^(-3/2) + (3/8) (b + c - a)(a + c - b)(a + b - c) (abc)^(-5/2).
// The cubic has ten monomials a^i b^j c^k: -a^3 - b^3 - c^3 - 2abc and the six
// a^2 b-type terms with coefficient 1. The abc monomial and the (abc)^(-3/2)
// term share exponents, so phi is a sum of ten products
//   w_m (a)^(s12_m) (b)^(s13_m) (c)^(s23_m),  s = i - 5/2 etc.,
// each a product of pairwise functions g(v) = (v.v)^s, which is the form the
// paper's expansion is written for. The expansion of the sum is the sum of
// the ten expansions.
//
// Factorisation used here. With t^s_a(v) = D^a (v.v)^s / a! (Taylor
// coefficients) the expansion of one product term is
//   sum_{a12, a13} t^{s12}_{a12}(x - c2) t^{s13}_{a13}(x - c3) K[a12, a13],
//   K[a12, a13] = w a12! a13! sum_{a23} sum_{b <= a23} C(a12 + b, a12) C(a13 + a23 - b, a13)
//                 (-1)^|b| M_{a12 + b}(P2) M_{a13 + a23 - b}(P3) D^{a23} (w23.w23)^{s23}
// over |a12| + |a13| + |a23| <= p, w23 = c2 - c3, with the far-field moments
// of §3.1, M_a(P, c) = sum_y (-1)^|a| (y - c)^a / a!. This is the paper's
// quadruple sum with a = a12 + a13 + a23 regrouped: K holds everything that
// does not depend on x, so it is formed once per call (FP64), and a query
// point costs the Taylor coefficients of four powers at x - c2 and at x - c3
// and one contraction with K per product term (FP32 arithmetic after the
// FP64 differences x - c, K in shared memory) instead of the O(p^6) sum per
// point.
//
// Taylor coefficients come from a recurrence: f = (v.v)^s satisfies
// (v.v) grad f = 2 s v f; the coefficient of t^a on both sides at v0 + t gives
//   |a| |v0|^2 t_a = (2s - 2|a| + 2) sum_d v0_d t_{a - e_d} + (2s - |a| + 2) sum_d t_{a - 2 e_d}.
//
// Kernels, in stream order: coordinate sums per block of each source set;
// moments per block about the centre; one block finishing the moments, the
// centres and the Taylor coefficients of the four powers at c2 - c3; K, one
// warp per coefficient (a12, a13); the query sweep. Every reduction runs in a
// fixed order, so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "mbm_internal.h"

namespace {

constexpr int kPMax = 6;
constexpr int kTerms = 10;
constexpr int kSumThreads = 256;
constexpr int kMomThreads = 128;
constexpr int kEvalThreads = 128;

// number of multi-indices with |a| <= k
__host__ __device__ constexpr int ff_n(int k) { return k < 0 ? 0 : (k + 1) * (k + 2) * (k + 3) / 6; }
// position of (i, j, l): by degree, then i descending, then j descending
__host__ __device__ constexpr int ff_idx(int i, int j, int l) {
    return ff_n(i + j + l - 1) + (j + l) * (j + l + 1) / 2 + l;
}
__host__ __device__ constexpr int pad4(int x) { return (x + 3) / 4 * 4; }
// floats of K per product term at order P: rows a12 of degree d hold the
// columns a13 with |a13| <= P - d, padded to a multiple of four
__host__ __device__ constexpr int k_stride(int P) {
    int s = 0;
    for (int d = 0; d <= P; ++d) s += (d + 1) * (d + 2) / 2 * pad4(ff_n(P - d));
    return s;
}

struct MultiIndexTable {
    unsigned char a[ff_n(kPMax)][3];
};
constexpr MultiIndexTable make_table() {
    MultiIndexTable t{};
    int n = 0;
    for (int k = 0; k <= kPMax; ++k)
        for (int i = k; i >= 0; --i)
            for (int j = k - i; j >= 0; --j) {
                t.a[n][0] = (unsigned char)i;
                t.a[n][1] = (unsigned char)j;
                t.a[n][2] = (unsigned char)(k - i - j);
                ++n;
            }
    return t;
}
__constant__ MultiIndexTable kAl = make_table();

// The ten product terms, grouped by s12 in the order the query sweep visits
// them: (2 s12, 2 s13) = (1, -5), (-1, -3), (-1, -5), (-3, -1), (-3, -3),
// (-3, -5), (-5, 1), (-5, -1), (-5, -3), (-5, -5); 2 s23 = -3 - 2 s12 - 2 s13
// (the exponents of a term sum to -9/2). Weights 3/8 times the cubic's
// coefficient (-1 on a^3, b^3, c^3; 1 on the a^2 b types), and 1/4 on
// (-3, -3, -3) = 1 - (3/8) 2.
__host__ __device__ constexpr int term_s23x2(int m) {
    return m == 0 ? -5 : m == 1 ? -5 : m == 2 ? -3 : m == 3 ? -5 : m == 4 ? -3
         : m == 5 ? -1 : m == 6 ? -5 : m == 7 ? -3 : m == 8 ? -1 : 1;
}
__host__ __device__ constexpr double term_w(int m) {
    return m == 4 ? 0.25 : (m == 0 || m == 6 || m == 9) ? -0.375 : 0.375;
}

// factorials and binomial coefficients up to 6 (every index of the sums is <= p)
struct SmallTables {
    double fact[kPMax + 1];
    double inv[kPMax + 1];  // 1 / k (inv[0] unused)
    double binom[kPMax + 1][kPMax + 1];
};
constexpr SmallTables make_small() {
    SmallTables t{};
    double f = 1.0;
    for (int n = 0; n <= kPMax; ++n) {
        if (n > 0) f *= n;
        t.fact[n] = f;
        t.inv[n] = n > 0 ? 1.0 / n : 0.0;
        for (int k = 0; k <= kPMax; ++k) t.binom[n][k] = 0.0;
        t.binom[n][0] = 1.0;
        for (int k = 1; k <= n; ++k)
            t.binom[n][k] = (n > 0 ? t.binom[n - 1][k - 1] : 0.0) + (k <= n - 1 ? t.binom[n - 1][k] : 0.0);
    }
    return t;
}
__constant__ SmallTables kSmall = make_small();

__device__ __forceinline__ double fact_d(int n) { return kSmall.fact[n]; }

// ---------------------------------------------------------------- sums
// part[set][b][3]: coordinate sums of block b's chunk of each source set.
__global__ void __launch_bounds__(kSumThreads)
ff_sums_kernel(const double* __restrict__ Y2, int64_t n2, const double* __restrict__ Y3, int64_t n3,
               int nb, double* __restrict__ part, int* __restrict__ flags) {
    __shared__ double red[3][kSumThreads];
    const int set = blockIdx.y;
    const double* Y = set ? Y3 : Y2;
    const int64_t n = set ? n3 : n2;
    const int64_t chunk = (n + nb - 1) / nb;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    double s[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kSumThreads)
        for (int d = 0; d < 3; ++d) {
            const double v = Y[3 * i + d];
            bad |= !isfinite(v);
            s[d] += v;
        }
    if (bad) atomicOr(flags, MBM_FLAG_NONFINITE);
    for (int d = 0; d < 3; ++d) red[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[((int64_t)set * nb + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------- moments
// mpart[set][b][a] = sum over block b's chunk of (y - c)^a / a! (no sign yet).
__global__ void __launch_bounds__(kMomThreads)
ff_moments_kernel(const double* __restrict__ Y2, int64_t n2, const double* __restrict__ Y3, int64_t n3,
                  int nb, int p, const double* __restrict__ part, double* __restrict__ mpart) {
    __shared__ double pw[kMomThreads][3][kPMax + 1];  // (y_d - c_d)^k / k! of staged points
    __shared__ double cen[3];
    const int set = blockIdx.y;
    const double* Y = set ? Y3 : Y2;
    const int64_t n = set ? n3 : n2;
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[((int64_t)set * nb + b) * 3 + threadIdx.x];
        cen[threadIdx.x] = s / (double)n;
    }
    __syncthreads();
    const int na = ff_n(p);
    const int t = threadIdx.x;
    const int ai = t < na ? kAl.a[t][0] : 0, aj = t < na ? kAl.a[t][1] : 0,
              al = t < na ? kAl.a[t][2] : 0;
    const int64_t chunk = (n + nb - 1) / nb;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    double acc = 0.0;
    for (int64_t s0 = b0; s0 < b1; s0 += kMomThreads) {
        const int64_t i = s0 + t;
        if (i < b1) {
            for (int d = 0; d < 3; ++d) {
                const double v = Y[3 * i + d] - cen[d];
                double m = 1.0;
                pw[t][d][0] = 1.0;
                for (int k = 1; k <= p; ++k) {
                    m = m * v * kSmall.inv[k];
                    pw[t][d][k] = m;
                }
            }
        }
        __syncthreads();
        const int cnt = (int)(b1 - s0 < kMomThreads ? b1 - s0 : kMomThreads);
        if (t < na)
            for (int q = 0; q < cnt; ++q) acc += pw[q][0][ai] * pw[q][1][aj] * pw[q][2][al];
        __syncthreads();
    }
    if (t < na) mpart[((int64_t)set * nb + blockIdx.x) * ff_n(kPMax) + t] = acc;
}

// ---------------------------------------------------------------- finish
// fin layout (doubles): M2[84], M3[84], D23[4][84] (D^a (w.w)^s for 2s = 1, -1,
// -3, -5), c2[3], c3[3].
constexpr int kFinM2 = 0, kFinM3 = ff_n(kPMax), kFinD = 2 * ff_n(kPMax),
              kFinC = 6 * ff_n(kPMax), kFinDoubles = 6 * ff_n(kPMax) + 8;

__global__ void __launch_bounds__(kMomThreads)
ff_finish_kernel(int64_t n2, int64_t n3, int nb, int p, const double* __restrict__ part,
                 const double* __restrict__ mpart, double* __restrict__ fin, int* __restrict__ flags) {
    __shared__ double w[3];
    __shared__ double D[4][ff_n(kPMax)];
    const int na = ff_n(p);
    const int t = threadIdx.x;
    if (t < 6) {
        const int set = t / 3, d = t % 3;
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[((int64_t)set * nb + b) * 3 + d];
        fin[kFinC + t] = s / (double)(set ? n3 : n2);
    }
    for (int q = t; q < 2 * na; q += kMomThreads) {
        const int set = q / na, a = q % na;
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += mpart[((int64_t)set * nb + b) * ff_n(kPMax) + a];
        const int deg = kAl.a[a][0] + kAl.a[a][1] + kAl.a[a][2];
        fin[(set ? kFinM3 : kFinM2) + a] = (deg & 1) ? -s : s;
    }
    __syncthreads();
    if (t < 3) w[t] = fin[kFinC + t] - fin[kFinC + 3 + t];
    __syncthreads();
    const double r2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    if (t == 0 && !(r2 > 0.0)) atomicOr(flags, MBM_FLAG_COINCIDENT);
    // Taylor coefficients of (w.w)^s at w by the recurrence, one degree level
    // at a time (every coefficient of a level depends only on lower levels)
    const double ir2 = 1.0 / r2;
    if (t < 4) D[t][0] = pow(sqrt(r2), (double)(1 - 2 * t));  // 2s = 1, -1, -3, -5
    __syncthreads();
    for (int k = 1; k <= p; ++k) {
        const int lo = ff_n(k - 1), cnt = ff_n(k) - lo;
        for (int q = t; q < 4 * cnt; q += kMomThreads) {
            const int sidx = q / cnt, a = lo + q % cnt, s2 = 1 - 2 * sidx;
            const int i = kAl.a[a][0], j = kAl.a[a][1], l = kAl.a[a][2];
            double A = 0.0, B = 0.0;
            if (i > 0) A += w[0] * D[sidx][ff_idx(i - 1, j, l)];
            if (j > 0) A += w[1] * D[sidx][ff_idx(i, j - 1, l)];
            if (l > 0) A += w[2] * D[sidx][ff_idx(i, j, l - 1)];
            if (i > 1) B += D[sidx][ff_idx(i - 2, j, l)];
            if (j > 1) B += D[sidx][ff_idx(i, j - 2, l)];
            if (l > 1) B += D[sidx][ff_idx(i, j, l - 2)];
            D[sidx][a] = ((s2 - 2 * k + 2) * A + (s2 - k + 2) * B) * (kSmall.inv[k] * ir2);
        }
        __syncthreads();
    }
    for (int q = t; q < 4 * na; q += kMomThreads) {  // D = a! t
        const int sidx = q / na, a = q % na;
        fin[kFinD + sidx * ff_n(kPMax) + a] =
            D[sidx][a] * fact_d(kAl.a[a][0]) * fact_d(kAl.a[a][1]) * fact_d(kAl.a[a][2]);
    }
}

// ---------------------------------------------------------------- K
// Grid (row a12, column group): warp w of a block owns column a13 =
// 4 blockIdx.y + w of row a12; its lanes take the a23 terms of the sum and
// a fixed butterfly adds them, so results do not depend on scheduling.
// K[m][row offset + col] in FP32. The moments, the g23 derivatives and the
// small tables are staged in shared memory first: the lanes of a warp index
// them at different places.
constexpr int kKWarps = 4;

__global__ void __launch_bounds__(kKWarps * 32)
ff_k_kernel(int p, const double* __restrict__ fin, float* __restrict__ K) {
    __shared__ double M2[ff_n(kPMax)], M3[ff_n(kPMax)], D23[4][ff_n(kPMax)];
    __shared__ int binom[kPMax + 1][kPMax + 1];  // C(n, k) <= 20: products of six fit in int
    __shared__ double fact[kPMax + 1];
    __shared__ unsigned char al[ff_n(kPMax)][3];
    const int na = ff_n(p);
    for (int q = threadIdx.x; q < na; q += kKWarps * 32) {
        M2[q] = fin[kFinM2 + q];
        M3[q] = fin[kFinM3 + q];
        for (int d = 0; d < 3; ++d) al[q][d] = kAl.a[q][d];
        for (int sidx = 0; sidx < 4; ++sidx) D23[sidx][q] = fin[kFinD + sidx * ff_n(kPMax) + q];
    }
    for (int q = threadIdx.x; q < (kPMax + 1) * (kPMax + 1); q += kKWarps * 32)
        binom[q / (kPMax + 1)][q % (kPMax + 1)] = (int)kSmall.binom[q / (kPMax + 1)][q % (kPMax + 1)];
    if (threadIdx.x <= kPMax) fact[threadIdx.x] = kSmall.fact[threadIdx.x];
    __syncthreads();
    const int r = blockIdx.x;  // a12 index
    const int i12 = al[r][0], j12 = al[r][1], l12 = al[r][2], d12 = i12 + j12 + l12;
    const int L = ff_n(p - d12);
    const int c = blockIdx.y * kKWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= pad4(L)) return;
    int off = 0;
    for (int d = 0; d < d12; ++d) off += (d + 1) * (d + 2) / 2 * pad4(ff_n(p - d));
    off += (r - ff_n(d12 - 1)) * pad4(L);
    const int stride = k_stride(p);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // by the power of g23: 2s = 1, -1, -3, -5
    double f = 0.0;
    if (c < L) {
        const int i13 = al[c][0], j13 = al[c][1], l13 = al[c][2];
        const int d13 = i13 + j13 + l13;
        for (int q = lane; q < ff_n(p - d12 - d13); q += 32) {  // a23
            const int i23 = al[q][0], j23 = al[q][1], l23 = al[q][2];
            double S = 0.0;
            for (int ib = 0; ib <= i23; ++ib)
                for (int jb = 0; jb <= j23; ++jb)
                    for (int lb = 0; lb <= l23; ++lb) {
                        const int gi = i12 + ib, gj = j12 + jb, gl = l12 + lb;  // a12 + b
                        const int hi = i13 + i23 - ib, hj = j13 + j23 - jb,
                                  hl = l13 + l23 - lb;  // a13 + a23 - b
                        int cb = binom[gi][i12] * binom[gj][j12] * binom[gl][l12] *
                                 binom[hi][i13] * binom[hj][j13] * binom[hl][l13];
                        if ((ib + jb + lb) & 1) cb = -cb;
                        S = fma((double)cb * M2[ff_idx(gi, gj, gl)], M3[ff_idx(hi, hj, hl)], S);
                    }
#pragma unroll
            for (int sidx = 0; sidx < 4; ++sidx) acc[sidx] += S * D23[sidx][q];
        }
        f = fact[i12] * fact[j12] * fact[l12] * fact[i13] * fact[j13] * fact[l13];
    }
#pragma unroll
    for (int sidx = 0; sidx < 4; ++sidx)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[sidx] += __shfl_xor_sync(0xffffffffu, acc[sidx], o);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < kTerms; ++m)
            K[m * stride + off + c] = (float)(acc[(1 - term_s23x2(m)) / 2] * term_w(m) * f);
    }
}

// ---------------------------------------------------------------- query sweep
// Taylor coefficients of (v.v)^(S2/2) at v, |a| <= P, in FP32 registers.
template <int P, int S2>
__device__ __forceinline__ void taylor(float vx, float vy, float vz, float r2inv, float r0,
                                       float (&t)[ff_n(P)]) {
    t[0] = r0;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
        const float ca = (float)(S2 - 2 * k + 2) / (float)k * r2inv;
        const float cb = (float)(S2 - k + 2) / (float)k * r2inv;
#pragma unroll
        for (int i = k; i >= 0; --i)
#pragma unroll
            for (int j = k - i; j >= 0; --j) {
                const int l = k - i - j;
                float A = 0.f, B = 0.f;
                if (i > 0) A = fmaf(vx, t[ff_idx(i - 1, j, l)], A);
                if (j > 0) A = fmaf(vy, t[ff_idx(i, j - 1, l)], A);
                if (l > 0) A = fmaf(vz, t[ff_idx(i, j, l - 1)], A);
                if (i > 1) B += t[ff_idx(i - 2, j, l)];
                if (j > 1) B += t[ff_idx(i, j - 2, l)];
                if (l > 1) B += t[ff_idx(i, j, l - 2)];
                t[ff_idx(i, j, l)] = (S2 - k + 2 == 0) ? ca * A : fmaf(cb, B, ca * A);
            }
    }
}

// sum_{a12, a13} tu[a12] tv[a13] K[a12, a13] over the padded row layout
template <int P>
__device__ __forceinline__ float contract(const float (&tu)[ff_n(P)], const float (&tv)[ff_n(P)],
                                          const float* __restrict__ Km) {
    float acc = 0.f;
    int off = 0;
#pragma unroll
    for (int d = 0; d <= P; ++d) {
        const int L = ff_n(P - d);
#pragma unroll
        for (int r = ff_n(d - 1); r < ff_n(d); ++r) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int q = 0; q < pad4(L) / 4; ++q) {
                const float4 k4 = *reinterpret_cast<const float4*>(Km + off + 4 * q);
                s0 = fmaf(tv[4 * q], k4.x, s0);
                if (4 * q + 1 < L) s1 = fmaf(tv[4 * q + 1], k4.y, s1);
                if (4 * q + 2 < L) s0 = fmaf(tv[4 * q + 2], k4.z, s0);
                if (4 * q + 3 < L) s1 = fmaf(tv[4 * q + 3], k4.w, s1);
            }
            acc = fmaf(tu[r], s0 + s1, acc);
            off += pad4(L);
        }
    }
    return acc;
}

template <int P>
__global__ void __launch_bounds__(kEvalThreads)
ff_eval_kernel(const double* __restrict__ Xq, int64_t nq, const float* __restrict__ Kg,
               const double* __restrict__ fin, double* __restrict__ out, int* __restrict__ flags) {
    extern __shared__ float4 smem4[];
    float* Ks = reinterpret_cast<float*>(smem4);
    constexpr int kStride = k_stride(P);
    for (int q = threadIdx.x; q < kTerms * kStride / 4; q += kEvalThreads)
        smem4[q] = reinterpret_cast<const float4*>(Kg)[q];
    __syncthreads();
    const double c2x = fin[kFinC], c2y = fin[kFinC + 1], c2z = fin[kFinC + 2];
    const double c3x = fin[kFinC + 3], c3y = fin[kFinC + 4], c3z = fin[kFinC + 5];
    for (int64_t i = (int64_t)blockIdx.x * kEvalThreads + threadIdx.x; i < nq;
         i += (int64_t)gridDim.x * kEvalThreads) {
        // x - c in FP64 (the difference of two far-apart points), rounded once
        const double x = Xq[3 * i], y = Xq[3 * i + 1], z = Xq[3 * i + 2];
        const float fux = (float)(x - c2x), fuy = (float)(y - c2y), fuz = (float)(z - c2z);
        const float fvx = (float)(x - c3x), fvy = (float)(y - c3y), fvz = (float)(z - c3z);
        const float ru2 = fmaf(fux, fux, fmaf(fuy, fuy, fuz * fuz));
        const float rv2 = fmaf(fvx, fvx, fmaf(fvy, fvy, fvz * fvz));
        if (!(ru2 > 0.f) || !(rv2 > 0.f) || !isfinite(ru2 + rv2)) {
            atomicOr(flags, isfinite(ru2 + rv2) ? MBM_FLAG_COINCIDENT : MBM_FLAG_NONFINITE);
            out[i] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const float iu = rsqrtf(ru2), iv = rsqrtf(rv2);
        const float u2i = iu * iu, v2i = iv * iv;
        const float ru = ru2 * iu, rv = rv2 * iv;  // |u|, |v|
        const float iu3 = iu * u2i, iv3 = iv * v2i;
        const float iu5 = iu3 * u2i, iv5 = iv3 * v2i;
        float tu[ff_n(P)], tv[ff_n(P)];
        float acc = 0.f;  // the terms' own FP32 roundings set the error scale
        // terms in the order of term_s23x2 / term_w: (2 s12, 2 s13)
        taylor<P, 1>(fux, fuy, fuz, u2i, ru, tu);
        taylor<P, -5>(fvx, fvy, fvz, v2i, iv5, tv);
        acc += contract<P>(tu, tv, Ks + 0 * kStride);
        taylor<P, -1>(fux, fuy, fuz, u2i, iu, tu);
        taylor<P, -3>(fvx, fvy, fvz, v2i, iv3, tv);
        acc += contract<P>(tu, tv, Ks + 1 * kStride);
        taylor<P, -5>(fvx, fvy, fvz, v2i, iv5, tv);
        acc += contract<P>(tu, tv, Ks + 2 * kStride);
        taylor<P, -3>(fux, fuy, fuz, u2i, iu3, tu);
        taylor<P, -1>(fvx, fvy, fvz, v2i, iv, tv);
        acc += contract<P>(tu, tv, Ks + 3 * kStride);
        taylor<P, -3>(fvx, fvy, fvz, v2i, iv3, tv);
        acc += contract<P>(tu, tv, Ks + 4 * kStride);
        taylor<P, -5>(fvx, fvy, fvz, v2i, iv5, tv);
        acc += contract<P>(tu, tv, Ks + 5 * kStride);
        taylor<P, -5>(fux, fuy, fuz, u2i, iu5, tu);
        taylor<P, 1>(fvx, fvy, fvz, v2i, rv, tv);
        acc += contract<P>(tu, tv, Ks + 6 * kStride);
        taylor<P, -1>(fvx, fvy, fvz, v2i, iv, tv);
        acc += contract<P>(tu, tv, Ks + 7 * kStride);
        taylor<P, -3>(fvx, fvy, fvz, v2i, iv3, tv);
        acc += contract<P>(tu, tv, Ks + 8 * kStride);
        taylor<P, -5>(fvx, fvy, fvz, v2i, iv5, tv);
        acc += contract<P>(tu, tv, Ks + 9 * kStride);
        out[i] = (double)acc;
    }
}

template <int P>
cudaError_t launch_eval(const double* Xq, int64_t nq, const float* K, const double* fin, double* out,
                        int* flags, int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)kTerms * k_stride(P) * sizeof(float);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(ff_eval_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
    });
    if (attr_err != cudaSuccess) return attr_err;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ff_eval_kernel<P>,
                                                                  kEvalThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t want = (nq + kEvalThreads - 1) / kEvalThreads;
    const int64_t cap = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(want < cap ? want : cap);
    ff_eval_kernel<P><<<grid, kEvalThreads, smem, s>>>(Xq, nq, K, fin, out, flags);
    return cudaGetLastError();
}

cudaError_t launch_eval_p(int p, const double* Xq, int64_t nq, const float* K, const double* fin,
                          double* out, int* flags, int num_sms, cudaStream_t s) {
    switch (p) {
        case 0: return launch_eval<0>(Xq, nq, K, fin, out, flags, num_sms, s);
        case 1: return launch_eval<1>(Xq, nq, K, fin, out, flags, num_sms, s);
        case 2: return launch_eval<2>(Xq, nq, K, fin, out, flags, num_sms, s);
        case 3: return launch_eval<3>(Xq, nq, K, fin, out, flags, num_sms, s);
        case 4: return launch_eval<4>(Xq, nq, K, fin, out, flags, num_sms, s);
        case 5: return launch_eval<5>(Xq, nq, K, fin, out, flags, num_sms, s);
        default: return launch_eval<6>(Xq, nq, K, fin, out, flags, num_sms, s);
    }
}

// blocks per source set for the sums and moments: chunks of at least 128
// points, at most four blocks per SM
int source_blocks(int64_t n2, int64_t n3, int num_sms) {
    const int64_t n = n2 > n3 ? n2 : n3;
    int64_t nb = (n + kMomThreads - 1) / kMomThreads;
    if (nb > 4 * (int64_t)num_sms) nb = 4 * (int64_t)num_sms;
    return nb < 1 ? 1 : (int)nb;
}

}  // namespace

size_t mbm_farfield3_scratch_bytes(int64_t n2, int64_t n3, int num_sms) {
    const int nb = source_blocks(n2, n3, num_sms);
    return mbm_align_up((size_t)2 * nb * 3 * sizeof(double), 256) +
           mbm_align_up((size_t)2 * nb * ff_n(kPMax) * sizeof(double), 256) +
           mbm_align_up((size_t)kFinDoubles * sizeof(double), 256) +
           mbm_align_up((size_t)kTerms * k_stride(kPMax) * sizeof(float), 256);
}

// Enqueue the whole expansion; scratch must hold mbm_farfield3_scratch_bytes.
// With ctx, its timing events bracket the query sweep.
cudaError_t launch_farfield3(mbm_ctx* ctx, const double* Xq, int64_t nq, const double* Y2,
                             int64_t n2, const double* Y3, int64_t n3, int p, double* out,
                             void* scratch, int* flags, int num_sms, cudaStream_t s) {
    const int nb = source_blocks(n2, n3, num_sms);
    char* b = static_cast<char*>(scratch);
    auto* part = reinterpret_cast<double*>(b);
    b += mbm_align_up((size_t)2 * nb * 3 * sizeof(double), 256);
    auto* mpart = reinterpret_cast<double*>(b);
    b += mbm_align_up((size_t)2 * nb * ff_n(kPMax) * sizeof(double), 256);
    auto* fin = reinterpret_cast<double*>(b);
    b += mbm_align_up((size_t)kFinDoubles * sizeof(double), 256);
    auto* K = reinterpret_cast<float*>(b);
    ff_sums_kernel<<<dim3(nb, 2), kSumThreads, 0, s>>>(Y2, n2, Y3, n3, nb, part, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ff_moments_kernel<<<dim3(nb, 2), kMomThreads, 0, s>>>(Y2, n2, Y3, n3, nb, p, part, mpart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ff_finish_kernel<<<1, kMomThreads, 0, s>>>(n2, n3, nb, p, part, mpart, fin, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ff_k_kernel<<<dim3(ff_n(p), pad4(ff_n(p)) / kKWarps), kKWarps * 32, 0, s>>>(p, fin, K);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ctx) mbm_time_begin(ctx, s);
    e = launch_eval_p(p, Xq, nq, K, fin, out, flags, num_sms, s);
    if (ctx) mbm_time_end(ctx, s);
    return e;
}

extern "C" mbm_status mbm_farfield3(mbm_ctx* ctx, const double* Xq_dev, int64_t nq,
                                    const double* Y2_dev, int64_t n2, const double* Y3_dev,
                                    int64_t n3, int p, int validate, double* out_dev,
                                    mbm_stream_t stream) {
    if (!ctx) return mbm_fail(MBM_EINVAL, "ctx is NULL");
    if (p < 0 || p > kPMax) return mbm_fail(MBM_EINVAL, "order p must be in [0, 6]");
    if (nq < 0 || n2 < 0 || n3 < 0) return mbm_fail(MBM_EINVAL, "negative size");
    if (nq > ((int64_t)1 << 40) || n2 > ((int64_t)1 << 40) || n3 > ((int64_t)1 << 40))
        return mbm_fail(MBM_EINVAL, "size too large (max 2^40)");
    if (nq > 0 && (!Xq_dev || !out_dev)) return mbm_fail(MBM_EINVAL, "NULL query points or output");
    if ((n2 > 0 && !Y2_dev) || (n3 > 0 && !Y3_dev)) return mbm_fail(MBM_EINVAL, "NULL source set");
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nq == 0) return MBM_OK;
    if (n2 == 0 || n3 == 0) {  // empty double sum
        MBM_CUDA_TRY(cudaMemsetAsync(out_dev, 0, (size_t)nq * sizeof(double), s));
        return MBM_OK;
    }
    MBM_TRY(mbm_scratch_reserve(ctx, mbm_farfield3_scratch_bytes(n2, n3, ctx->num_sms)));
    MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    MBM_CUDA_TRY(launch_farfield3(ctx, Xq_dev, nq, Y2_dev, n2, Y3_dev, n3, p, out_dev,
                                  ctx->scratch, ctx->d_flags, ctx->num_sms, s));
    if (validate) return mbm_check_flags(ctx, s);
    return MBM_OK;
}
