// Multi-tree approximation of Phi on the GPU (Algorithm 2 with the p = 0 and
// Monte Carlo rules of Sec. 4).
//
//   a4 tree build   : bounding cube -> 63-bit Morton keys (2^21 grid) -> radix
//                     sort (ties by index) -> balanced ranges halved to <= leaf
//                     size; FP64 boxes, centres of mass, squared diameters.
//   seed            : Phi^l (Sec. 4 summary statistic, read as a lower bound on
//                     |Phi|): |exact sum over each particle's seed node|, min
//                     over every node (Sec. 5: Phi^l(P) = min over children).
//   a5/a6 traversal : node triples from (root, root, root), one thread each,
//                     in chunks of B triples taken from a stack of level
//                     buffers (the deepest level first, so memory stays
//                     bounded); per triple the p = 0 interval bound, T_i of
//                     Fig. 4 and the budget of Eq. (deterministic_prune)
//                     decide: prune (accumulate T_i phi(c1,c2,c3) per node),
//                     Monte Carlo candidate, base case, or split the
//                     largest-diameter node (all of its copies;
//                     non-decreasing child triples).
//   a7 Monte Carlo  : Algorithms 3-5; a lane per particle draws tuples with
//                     Philox-4x32-10, FP32 phi, FP64 Welford statistics and
//                     stop test; a triple passes only if all its particles do,
//                     so each candidate first tests its weakest particles
//                     (smallest Phi^l; 32, 16 or 10 per node for 1, 2 or 3
//                     distinct nodes) and stops at the first failure.
//   a8 base cases   : exhaustive leaf triples with the Fig. 4 masks, FP32 bulk
//                     (tile_fp32.cuh), FP64 accumulation; each flush of the
//                     base list is sorted by (y, z) leaf pair so a CTA shares
//                     one (j,k) table across the x leaves of a pair.
//   a9 top-down     : node accumulators summed along each leaf's root path.
//
// Every bound decision is computed in FP64 in the same operation order as the
// serial restatement (explicit round-to-nearest intrinsics, no contraction),
// and Phi^l is fixed before the traversal, so this order makes the same
// decisions as a depth-first recursion. Monte Carlo samples are FP32 phi
// values, so a stop test on the edge may rarely differ from an FP64 sample.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mbm_tree_api.h"
#include "sort_scan.h"
#include "tile_fp32.cuh"

struct mbm_tree {
    mbm_ctx* ctx = nullptr;
    int device = 0;
    int64_t N = 0;
    int leaf_size = 32;
    int depth = 0;
    int64_t n_nodes = 0, n_leaves = 0;
    int seed_levels = 2;
    void* mem = nullptr;
    size_t bytes = 0;
    int64_t* perm = nullptr;  // sorted position -> original index
    double* xs = nullptr;     // sorted coordinates, 3 per particle
    float4* xh = nullptr;     // sorted hi/lo FP32 coordinates
    float4* xl = nullptr;
    double* nlo = nullptr;    // per node, 3 each
    double* nhi = nullptr;
    double* ncen = nullptr;
    double* ndiam2 = nullptr; // per node
    double* nphil = nullptr;  // per node
    double* pphil = nullptr;  // per sorted particle: |S(x)|
    int* weak = nullptr;      // per node: up to 32 sorted positions of smallest Phi^l(x)
};

namespace {

using mbm_tile::kTile;
using ull = unsigned long long;

// ---------------------------------------------------------------------------
// Node geometry helpers (implicit complete binary tree in heap order).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void node_range(int64_t v, int64_t N, int64_t& b, int64_t& e) {
#ifdef __CUDA_ARCH__
    const int d = 63 - __clzll((long long)(v + 1));
#else
    int d = 0;
    while ((v + 1) >> (d + 1)) ++d;
#endif
    const int64_t q = v + 1 - ((int64_t)1 << d);
    b = (q * N) >> d;
    e = ((q + 1) * N) >> d;
}

int tree_depth(int64_t N, int leaf) {
    int d = 0;
    while (((N + ((int64_t)1 << d) - 1) >> d) > leaf) ++d;
    return d;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t r = 0;
#pragma unroll
    for (int b = 0; b < 21; ++b) r |= (uint64_t)((v >> b) & 1u) << (3 * b);
    return r;
}

// ---------------------------------------------------------------------------
// a4: build.
// ---------------------------------------------------------------------------
__global__ void bbox_partial_kernel(const double* __restrict__ X, int64_t N, double* part) {
    __shared__ double s[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const double x = X[3 * i + k];
            lo[k] = fmin(lo[k], x);
            hi[k] = fmax(hi[k], x);
        }
    for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = lo[k];
        s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + o]);
                s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void bbox_final_kernel(const double* part, int nb, double* box) {
    if (threadIdx.x >= 6) return;
    const int k = threadIdx.x;
    double v = part[k];
    for (int b = 1; b < nb; ++b) v = k < 3 ? fmin(v, part[6 * b + k]) : fmax(v, part[6 * b + k]);
    box[k] = v;
}

__global__ void morton_kernel(const double* __restrict__ X, int64_t N, const double* box,
                              unsigned long long* keys, int* idx, int* flags) {
    const double l0 = box[0], l1 = box[1], l2 = box[2];
    double ext = __dsub_rn(box[3], l0);
    if (__dsub_rn(box[4], l1) > ext) ext = __dsub_rn(box[4], l1);
    if (__dsub_rn(box[5], l2) > ext) ext = __dsub_rn(box[5], l2);
    const double scale = ext > 0.0 ? __ddiv_rn(2097152.0, ext) : 0.0;
    const double lo[3] = {l0, l1, l2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
        for (int d = 0; d < 3; ++d) {
            if (!isfinite(X[3 * i + d])) atomicOr(flags, MBM_FLAG_NONFINITE);
            const double q = floor(__dmul_rn(__dsub_rn(X[3 * i + d], lo[d]), scale));
            const uint32_t qi = q < 0.0 ? 0u : (q > 2097151.0 ? 2097151u : (uint32_t)q);
            key |= spread3(qi) << d;
        }
        keys[i] = key;
        idx[i] = (int)i;
    }
}

__global__ void gather_kernel(const double* __restrict__ X, int64_t N, const int* __restrict__ sidx,
                              int64_t* perm, double* xs, float4* xh, float4* xl) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = sidx[s];
        perm[s] = o;
        const double x = X[3 * o], y = X[3 * o + 1], z = X[3 * o + 2];
        xs[3 * s] = x;
        xs[3 * s + 1] = y;
        xs[3 * s + 2] = z;
        const float hx = (float)x, hy = (float)y, hz = (float)z;
        xh[s] = make_float4(hx, hy, hz, 0.f);
        xl[s] = make_float4((float)(x - (double)hx), (float)(y - (double)hy),
                            (float)(z - (double)hz), 0.f);
    }
}

// One warp per leaf: box, coordinate sums.
__global__ void leaf_stats_kernel(const double* __restrict__ xs, int64_t N, int64_t first_leaf,
                                  int64_t n_leaves, double* nlo, double* nhi, double* nsum) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_leaves) return;
    const int64_t v = first_leaf + w;
    int64_t b, e;
    node_range(v, N, b, e);
    double lo[3], hi[3], sm[3];
    for (int k = 0; k < 3; ++k) {
        const bool in = b + lane < e;
        const double x = in ? xs[3 * (b + lane) + k] : 0.0;
        lo[k] = in ? x : INFINITY;
        hi[k] = in ? x : -INFINITY;
        sm[k] = x;
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            sm[k] += __shfl_xor_sync(0xffffffffu, sm[k], o);
        }
    if (lane < 3) {
        nlo[3 * v + lane] = lane == 0 ? lo[0] : (lane == 1 ? lo[1] : lo[2]);
        nhi[3 * v + lane] = lane == 0 ? hi[0] : (lane == 1 ? hi[1] : hi[2]);
        nsum[3 * v + lane] = lane == 0 ? sm[0] : (lane == 1 ? sm[1] : sm[2]);
    }
}

__global__ void internal_stats_kernel(int64_t first, int64_t count, double* nlo, double* nhi,
                                      double* nsum) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t v = first + t, L = 2 * v + 1, R = 2 * v + 2;
    for (int k = 0; k < 3; ++k) {
        nlo[3 * v + k] = fmin(nlo[3 * L + k], nlo[3 * R + k]);
        nhi[3 * v + k] = fmax(nhi[3 * L + k], nhi[3 * R + k]);
        nsum[3 * v + k] = nsum[3 * L + k] + nsum[3 * R + k];
    }
}

__global__ void node_finish_kernel(int64_t N, int64_t n_nodes, const double* nlo, const double* nhi,
                                   double* ncen /* holds sums on entry */, double* ndiam2) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n_nodes) return;
    int64_t b, e;
    node_range(v, N, b, e);
    const double cnt = (double)(e - b);
    for (int k = 0; k < 3; ++k) ncen[3 * v + k] = cnt > 0 ? ncen[3 * v + k] / cnt : 0.0;
    const double dx = __dsub_rn(nhi[3 * v], nlo[3 * v]);
    const double dy = __dsub_rn(nhi[3 * v + 1], nlo[3 * v + 1]);
    const double dz = __dsub_rn(nhi[3 * v + 2], nlo[3 * v + 2]);
    ndiam2[v] = cnt > 0 ? __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))
                        : 0.0;
}

// ---------------------------------------------------------------------------
// Range triples (base cases and the Phi^l seed), one warp each, FP32 bulk.
// ---------------------------------------------------------------------------
struct WarpSmem {
    mbm_tile::TabPair tab[kTile][kTile / 2];
    float4 sJh[kTile], sJl[kTile], sKh[kTile], sKl[kTile];
    float redJ[kTile][kTile + 1];
    float redK[kTile][kTile + 1];
};
constexpr int kRangeWarps = 4;

// All triples (i in R1, j in R2, k in R3) with i<j if R1 == R2, j<k if
// R2 == R3 and i<k if R1 == R3; each credited to its three members in out[].
__device__ void range_triple(WarpSmem& w, const float4* __restrict__ xh,
                             const float4* __restrict__ xl, int64_t b1, int n1, int64_t b2, int n2,
                             int64_t b3, int n3, bool e12, bool e23, bool e13, double* out,
                             int* flags) {
    const int lane = threadIdx.x & 31;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    w.sJh[lane] = lane < n2 ? xh[b2 + lane] : z4;
    w.sJl[lane] = lane < n2 ? xl[b2 + lane] : z4;
    w.sKh[lane] = lane < n3 ? xh[b3 + lane] : z4;
    w.sKl[lane] = lane < n3 ? xl[b3 + lane] : z4;
    __syncwarp();
    bool bad = false;
    for (int e = lane; e < kTile * kTile; e += 32) {
        const int jj = e >> 5, kk = e & 31;
        const bool v = jj < n2 && kk < n3 && (!e23 || jj < kk);
        bad |= mbm_tile::build_table_entry(w.tab, jj, kk, w.sJh[jj], w.sJl[jj], w.sKh[kk],
                                           w.sKl[kk], v);
    }
    if (bad) atomicOr(flags, MBM_FLAG_COINCIDENT);
    __syncwarp();
    const bool iv = lane < n1;
    const float4 ih = iv ? xh[b1 + lane] : z4;
    const float4 il = iv ? xl[b1 + lane] : z4;
    const float acc_i = mbm_tile::tile_triples(w.tab, w.sJh, w.sJl, w.sKh, w.sKl, ih, il, iv, lane,
                                               n2, n3, e12, e13, w.redJ, w.redK);
    const float rj = mbm_tile::row_sum(w.redJ, lane);
    const float rk = mbm_tile::row_sum(w.redK, lane);
    if (lane < n2) atomicAdd(&out[b2 + lane], (double)rj);
    if (lane < n3) atomicAdd(&out[b3 + lane], (double)rk);
    if (iv) atomicAdd(&out[b1 + lane], (double)acc_i);
    __syncwarp();
}

// Seed items: for each seed node A (level sd), chunk triples I <= J <= K of
// its 32-point chunks. `combos` lists (I,J,K) for the maximum chunk count.
__global__ void __launch_bounds__(kRangeWarps * 32)
seed_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int64_t N, int sd,
            int64_t n_seed_nodes, const int4* __restrict__ combos, int n_combos, double* seed,
            int* flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem& w = reinterpret_cast<WarpSmem*>(smem_raw)[threadIdx.x >> 5];
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (item >= n_seed_nodes * n_combos) return;
    const int64_t a = item / n_combos;
    const int4 c = combos[item % n_combos];
    int64_t b, e;
    node_range(((int64_t)1 << sd) - 1 + a, N, b, e);
    const int64_t n = e - b;
    const int chunks = (int)((n + kTile - 1) / kTile);
    if (c.z >= chunks) return;  // warp-uniform
    auto len = [&](int q) { const int64_t r = n - (int64_t)q * kTile; return (int)(r < kTile ? r : kTile); };
    range_triple(w, xh, xl, b + (int64_t)c.x * kTile, len(c.x), b + (int64_t)c.y * kTile, len(c.y),
                 b + (int64_t)c.z * kTile, len(c.z), c.x == c.y, c.y == c.z, c.x == c.z, seed,
                 flags);
}

// Grouped base cases. One flush of the base list is sorted by its (y, z)
// leaf pair (items are canonical, x <= y <= z), and every run of equal pair
// is cut into pieces of at most kPiece items. A CTA takes a piece, builds the
// (j,k) table of the pair once and its warps sweep the x leaves of the piece,
// so the table and the (y, z) row sums are shared by up to kPiece leaf
// triples. Every leaf triple runs the exhaustive tile routine with the Fig. 4
// masks (x == y: i < j; y == z: j < k).
constexpr int kBaseWarps = 4;
constexpr int kPiece = 64;

// First particle of node v (recomputed where keeping it live costs registers).
__device__ __noinline__ int64_t leaf_first(int64_t v, int64_t N) {
    int64_t b, e;
    node_range(v, N, b, e);
    return b;
}

__device__ __forceinline__ unsigned leaf_triple_count(int x, int y, int z, unsigned n1,
                                                      unsigned n2, unsigned n3) {
    if (x == y && y == z) return n1 * (n1 - 1) * (n1 - 2) / 6;
    if (x == y) return n1 * (n1 - 1) / 2 * n3;
    if (y == z) return n1 * (n2 * (n2 - 1) / 2);
    return n1 * n2 * n3;
}

// Sort keys of one flush, and the number of point triples it holds (Fig. 4
// cases; at most 32^3 per leaf triple, summed per warp in 32 bits).
__global__ void base_key_kernel(const int4* __restrict__ items, int64_t n, int64_t N,
                                int64_t first_leaf, int d, ull* __restrict__ key,
                                int* __restrict__ val, ull* __restrict__ n_triples) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t base = q0 - (threadIdx.x & 31); base < n; base += stride) {
        const int64_t q = base + (threadIdx.x & 31);
        unsigned c = 0;
        if (q < n) {
            const int4 t = items[q];
            key[q] = ((ull)(t.y - first_leaf) << d) | (ull)(t.z - first_leaf);
            val[q] = t.x;
            int64_t b1, e1, b2, e2, b3, e3;
            node_range(t.x, N, b1, e1);
            node_range(t.y, N, b2, e2);
            node_range(t.z, N, b3, e3);
            c = leaf_triple_count(t.x, t.y, t.z, (unsigned)(e1 - b1), (unsigned)(e2 - b2),
                                  (unsigned)(e3 - b3));
        }
        const unsigned w = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(n_triples, (ull)w);
    }
}

// flag[q] = 1 where a piece starts: the first item of a run, and every
// kPiece-th item after it (keys are sorted; the run start is found by
// binary search).
__global__ void base_piece_flag_kernel(const ull* __restrict__ key, int64_t n,
                                       int* __restrict__ flag) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const ull k = key[q];
        int64_t lo = 0, hi = q;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < k) lo = mid + 1;
            else hi = mid;
        }
        flag[q] = ((q - lo) % kPiece) == 0 ? 1 : 0;
    }
}

// heads[pos[q]] = q for every piece start; heads[n_pieces] = n.
__global__ void base_piece_heads_kernel(const int* __restrict__ flag, const int* __restrict__ pos,
                                        int64_t n, int* __restrict__ heads,
                                        int* __restrict__ n_pieces) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (flag[q]) heads[pos[q]] = (int)q;
        if (q == n - 1) {
            const int np = pos[q] + flag[q];
            heads[np] = (int)n;
            *n_pieces = np;
        }
    }
}

struct BaseSmem {
    mbm_tile::TabPair tab[kTile][kTile / 2];
    float4 sJh[kTile], sJl[kTile], sKh[kTile], sKl[kTile];
    float redJ[kBaseWarps][kTile][kTile + 1];
    float redK[kBaseWarps][kTile][kTile + 1];
    double wsum[2][kBaseWarps][kTile];
    long long b2, b3;  // first particle of the y and z leaves
    int Y, Z, n2, n3, st, en;
};

__global__ void __launch_bounds__(kBaseWarps * 32, 4)
base_group_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int64_t N,
                  int64_t first_leaf, int d, const ull* __restrict__ key,
                  const int* __restrict__ val, const int* __restrict__ heads,
                  const int* __restrict__ n_pieces_p, unsigned* __restrict__ piece_ctr,
                  double* __restrict__ acc, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BaseSmem& sm = *reinterpret_cast<BaseSmem*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int n_pieces = *n_pieces_p;
    for (;;) {
        if (threadIdx.x == 0) {
            const int pc = (int)atomicAdd(piece_ctr, 1u);
            sm.st = pc < n_pieces ? heads[pc] : -1;
            if (pc < n_pieces) {
                sm.en = heads[pc + 1];
                const ull k = key[sm.st];
                const int64_t Y = first_leaf + (int64_t)(k >> d);
                const int64_t Z = first_leaf + (int64_t)(k & ((1ull << d) - 1));
                int64_t b2, e2, b3, e3;
                node_range(Y, N, b2, e2);
                node_range(Z, N, b3, e3);
                sm.Y = (int)Y;
                sm.Z = (int)Z;
                sm.b2 = b2;
                sm.b3 = b3;
                sm.n2 = (int)(e2 - b2);
                sm.n3 = (int)(e3 - b3);
            }
        }
        __syncthreads();
        if (sm.st < 0) break;
        if (threadIdx.x < kTile) {
            const int n2 = sm.n2;
            sm.sJh[threadIdx.x] = threadIdx.x < n2 ? xh[sm.b2 + threadIdx.x] : z4;
            sm.sJl[threadIdx.x] = threadIdx.x < n2 ? xl[sm.b2 + threadIdx.x] : z4;
        } else if (threadIdx.x < 2 * kTile) {
            const int kk = threadIdx.x - kTile, n3 = sm.n3;
            sm.sKh[kk] = kk < n3 ? xh[sm.b3 + kk] : z4;
            sm.sKl[kk] = kk < n3 ? xl[sm.b3 + kk] : z4;
        }
        __syncthreads();
        bool bad = false;
        {
            const int n2 = sm.n2, n3 = sm.n3;
            const bool e23 = sm.Y == sm.Z;
            for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
                const int jj = e >> 5, kk = e & 31;
                const bool v = jj < n2 && kk < n3 && (!e23 || jj < kk);
                bad |= mbm_tile::build_table_entry(sm.tab, jj, kk, sm.sJh[jj], sm.sJl[jj],
                                                   sm.sKh[kk], sm.sKl[kk], v);
            }
        }
        if (bad) atomicOr(flags, MBM_FLAG_COINCIDENT);
        __syncthreads();
        sm.wsum[0][warp][lane] = 0.0;
        sm.wsum[1][warp][lane] = 0.0;
        const int en = sm.en;
        for (int q = sm.st + warp; q < en; q += kBaseWarps) {
            const int X = val[q];
            int64_t b1, e1;
            node_range(X, N, b1, e1);
            const int n1 = (int)(e1 - b1);
            const bool iv = lane < n1;
            const float4 ih = iv ? xh[b1 + lane] : z4;
            const float4 il = iv ? xl[b1 + lane] : z4;
            const float acc_i = mbm_tile::tile_triples(sm.tab, sm.sJh, sm.sJl, sm.sKh, sm.sKl, ih,
                                                       il, iv, lane, sm.n2, sm.n3, X == sm.Y,
                                                       X == sm.Z, sm.redJ[warp], sm.redK[warp]);
            sm.wsum[0][warp][lane] += (double)mbm_tile::row_sum(sm.redJ[warp], lane);
            sm.wsum[1][warp][lane] += (double)mbm_tile::row_sum(sm.redK[warp], lane);
            __syncwarp();
            if (iv) atomicAdd(&acc[leaf_first(X, N) + lane], (double)acc_i);
        }
        __syncthreads();
        if (warp < 2) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < kBaseWarps; ++w) tot += sm.wsum[warp][w][lane];
            const int nn = warp == 0 ? sm.n2 : sm.n3;
            const long long b = warp == 0 ? sm.b2 : sm.b3;
            if (lane < nn) atomicAdd(&acc[b + lane], tot);
        }
        __syncthreads();
    }
}

// Tuple counts of base cases by enumeration (validation only).
__global__ void base_count_kernel(int64_t N, const int4* __restrict__ items, int64_t n_items,
                                  unsigned long long* cnt) {
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item >= n_items) return;
    const int4 t = items[item];
    int64_t b1, e1, b2, e2, b3, e3;
    node_range(t.x, N, b1, e1);
    node_range(t.y, N, b2, e2);
    node_range(t.z, N, b3, e3);
    for (int64_t i = b1 + lane; i < e1; i += 32)
        for (int64_t j = b2; j < e2; ++j) {
            if (t.x == t.y && j <= i) continue;
            for (int64_t k = b3; k < e3; ++k) {
                if (t.y == t.z && k <= j) continue;
                atomicAdd(&cnt[i], 1ULL);
                atomicAdd(&cnt[j], 1ULL);
                atomicAdd(&cnt[k], 1ULL);
            }
        }
}

// Phi^l per node: |seed| per particle, min over leaves, then up the tree.
__global__ void phil_leaf_kernel(const double* __restrict__ seed, int64_t N, int64_t first_leaf,
                                 int64_t n_leaves, double* nphil, double* pphil) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_leaves) return;
    const int64_t v = first_leaf + w;
    int64_t b, e;
    node_range(v, N, b, e);
    double m = b + lane < e ? fabs(seed[b + lane]) : INFINITY;
    if (b + lane < e) pphil[b + lane] = m;
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) nphil[v] = b < e ? m : 0.0;
}

// Per leaf: its particles in ascending Phi^l(x) (ties by position), padded with -1.
__global__ void weak_leaf_kernel(const double* __restrict__ pphil, int64_t N, int64_t first_leaf,
                                 int64_t n_leaves, int* weak) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_leaves) return;
    const int64_t v = first_leaf + w;
    int64_t b, e;
    node_range(v, N, b, e);
    const bool in = b + lane < e;
    const double key = in ? pphil[b + lane] : INFINITY;
    int rank = 0;  // rank of this lane's particle by (key, position)
    for (int o = 0; o < 32; ++o) {
        const double k2 = __shfl_sync(0xffffffffu, key, o);
        const bool in2 = __shfl_sync(0xffffffffu, (int)in, o) != 0;
        if (in2 && (k2 < key || (k2 == key && o < lane))) ++rank;
    }
    weak[v * 32 + lane] = -1;
    __syncwarp();
    if (in) weak[v * 32 + rank] = (int)(b + lane);
}

// Per internal node: the 32 smallest of its children's lists (merge).
__global__ void weak_internal_kernel(int64_t first, int64_t count, const double* __restrict__ pphil,
                                     int* weak) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t v = first + t;
    const int* A = weak + (2 * v + 1) * 32;
    const int* Bl = weak + (2 * v + 2) * 32;
    int ia = 0, ib = 0;
    for (int o = 0; o < 32; ++o) {
        const int a = ia < 32 ? A[ia] : -1, b = ib < 32 ? Bl[ib] : -1;
        int pick;
        if (a < 0 && b < 0) pick = -1;
        else if (b < 0) pick = a;
        else if (a < 0) pick = b;
        else pick = (pphil[a] < pphil[b] || (pphil[a] == pphil[b] && a < b)) ? a : b;
        if (pick >= 0 && pick == a) ++ia;
        else if (pick >= 0) ++ib;
        weak[v * 32 + o] = pick;
    }
}

__global__ void phil_internal_kernel(int64_t first, int64_t count, double* nphil) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t v = first + t;
    nphil[v] = fmin(nphil[2 * v + 1], nphil[2 * v + 2]);
}

// ---------------------------------------------------------------------------
// a5/a6: bound evaluator and traversal.
// ---------------------------------------------------------------------------
struct Trav {
    int64_t N, n_nodes, n_leaves;
    const double *nlo, *nhi, *ncen, *ndiam2, *nphil, *pphil;
    const int* weak;
    const double* xs;
    const float4 *xh, *xl;
    double eps, tau, troot, zeta, z, alpha;
    double inv_troot;          // 1 / T^root
    const double* rcp;         // rcp[m] = 1/m (correctly rounded), m = 1..m_limit
    int m_limit, mc_rule;
    uint32_t key0, key1;
    double* node_acc;
    double* pt_acc;
    ull* node_cnt;  // optional
    ull* pt_cnt;    // optional
    int4* next;
    ull* n_next;
    int64_t cap_next;
    int4* mc;
    ull* n_mc;
    int64_t cap_mc;
    int4* base;
    ull* n_base;
    int64_t cap_base;
    int* flags;
    ull* stat;  // visited, det, mc prunes, mc attempts, base, samples
    // tree forces only
    const double *nscale, *pscale;  // A^l per node (min) and per sorted particle
    double* node_acc3;              // 3 per node
    double* pt_acc3;                // 3 per sorted particle
};

__device__ __forceinline__ bool is_leaf(const Trav& p, int64_t v) {
    return v >= p.n_nodes - p.n_leaves;
}

__device__ __forceinline__ double choose2(double n) {
    return __dmul_rn(__dmul_rn(n, __dsub_rn(n, 1.0)), 0.5);
}

// T_i of Fig. 4 for the particle's slot.
__device__ double tuples_for_slot(const int64_t P[3], const double n[3], int slot) {
    const bool e01 = P[0] == P[1], e12 = P[1] == P[2];
    if (e01 && e12) return choose2(__dsub_rn(n[0], 1.0));
    if (e01) return slot == 2 ? choose2(n[0]) : __dmul_rn(__dsub_rn(n[0], 1.0), n[2]);
    if (e12) return slot == 0 ? choose2(n[1]) : __dmul_rn(n[0], __dsub_rn(n[1], 1.0));
    if (slot == 0) return __dmul_rn(n[1], n[2]);
    if (slot == 1) return __dmul_rn(n[0], n[2]);
    return __dmul_rn(n[0], n[1]);
}

// Squared minimum and maximum point distances between two boxes (Fig. 3).
__device__ void box_d2(const Trav& p, int64_t a, int64_t b, double& dl, double& du) {
    double l = 0.0, u = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double x = __dsub_rn(p.nlo[3 * b + k], p.nhi[3 * a + k]);
        const double y = __dsub_rn(p.nlo[3 * a + k], p.nhi[3 * b + k]);
        double g = x > y ? x : y;
        if (g < 0.0) g = 0.0;
        l = __dadd_rn(l, __dmul_rn(g, g));
        const double c = __dsub_rn(p.nhi[3 * b + k], p.nlo[3 * a + k]);
        const double e = __dsub_rn(p.nhi[3 * a + k], p.nlo[3 * b + k]);
        const double m = c > e ? c : e;
        u = __dadd_rn(u, __dmul_rn(m, m));
    }
    dl = l;
    du = u;
}

__device__ void interval_mul(double a0, double a1, double b0, double b1, double& r0, double& r1) {
    const double q[4] = {__dmul_rn(a0, b0), __dmul_rn(a0, b1), __dmul_rn(a1, b0), __dmul_rn(a1, b1)};
    double lo = q[0], hi = q[0];
    for (int i = 1; i < 4; ++i) {
        if (q[i] < lo) lo = q[i];
        if (q[i] > hi) hi = q[i];
    }
    r0 = lo;
    r1 = hi;
}

// [phi_lo, phi_hi] over all point triples, from squared-distance intervals
// c (slots 1-2), b (slots 1-3), a (slots 2-3): the cosine product by interval
// arithmetic on (b+c-a)(a+c-b)(a+b-c)/(8abc) within [-1, 1/8], the distance
// factor by its monotone bounds.
__device__ void phi_interval(double cl, double cu, double bl, double bu, double al, double au,
                             double& plo, double& phi) {
    double Cl = -1.0, Ch = 0.125;
    const double Dl = __dmul_rn(__dmul_rn(__dmul_rn(8.0, al), bl), cl);
    const double Dh = __dmul_rn(__dmul_rn(__dmul_rn(8.0, au), bu), cu);
    if (Dl > 0.0) {
        const double U0 = __dsub_rn(__dadd_rn(bl, cl), au), U1 = __dsub_rn(__dadd_rn(bu, cu), al);
        const double V0 = __dsub_rn(__dadd_rn(al, cl), bu), V1 = __dsub_rn(__dadd_rn(au, cu), bl);
        const double W0 = __dsub_rn(__dadd_rn(al, bl), cu), W1 = __dsub_rn(__dadd_rn(au, bu), cl);
        double p0, p1, q0, q1;
        interval_mul(U0, U1, V0, V1, p0, p1);
        interval_mul(p0, p1, W0, W1, q0, q1);
        const double a0 = __ddiv_rn(q0, Dl), a1 = __ddiv_rn(q0, Dh);
        const double c0 = __ddiv_rn(q1, Dl), c1 = __ddiv_rn(q1, Dh);
        const double lo = a0 < a1 ? a0 : a1;
        const double hi = c0 > c1 ? c0 : c1;
        if (lo > Cl) Cl = lo;
        if (hi < Ch) Ch = hi;
        if (Cl > Ch) Cl = Ch;
    }
    const double nl = __dadd_rn(1.0, __dmul_rn(3.0, Cl));
    const double nh = __dadd_rn(1.0, __dmul_rn(3.0, Ch));
    const double Sl = __dmul_rn(__dmul_rn(al, bl), cl), Sh = __dmul_rn(__dmul_rn(au, bu), cu);
    const double R3l = __dmul_rn(Sl, __dsqrt_rn(Sl)), R3h = __dmul_rn(Sh, __dsqrt_rn(Sh));
    const double hiv = nh >= 0.0 ? (R3l > 0.0 ? __ddiv_rn(nh, R3l) : INFINITY) : __ddiv_rn(nh, R3h);
    const double lov = nl >= 0.0 ? __ddiv_rn(nl, R3h) : (R3l > 0.0 ? __ddiv_rn(nl, R3l) : -INFINITY);
    phi = __dadd_rn(hiv, __dmul_rn(fabs(hiv), 1e-13));
    plo = __dsub_rn(lov, __dmul_rn(fabs(lov), 1e-13));
}

// phi at three points (FP64, law of cosines on squared sides).
__device__ double phi_f64(const double* x, const double* y, const double* z) {
    double c = 0, b = 0, a = 0;
    for (int k = 0; k < 3; ++k) {
        const double u = y[k] - x[k], v = z[k] - x[k], w = z[k] - y[k];
        c += u * u;
        b += v * v;
        a += w * w;
    }
    const double P = (b + c - a) * (a + c - b) * (a + b - c);
    const double S = a * b * c;
    return (S + 0.375 * P) / (S * S * sqrt(S));
}

// d phi(a, b, c) / d a in FP64 (pair-vector form): with u = b - a, v = c - a,
// w = c - b, unit vectors e, p1 = e_u.e_v, p2 = e_u.e_w, p3 = e_v.e_w,
// t = p1 p2 p3 and R = (r_u r_v r_w)^-3,
//   grad = -g_u - g_v,  g_u = 3R/r_u (q e_u - p2 p3 e_v - p1 p3 e_w),
//   g_v = 3R/r_v (q e_v - p2 p3 e_u - p1 p2 e_w),  q = 5t - 1.
__device__ void grad_first_f64(const double* a, const double* b, const double* c, double g[3]) {
    double u[3], v[3], w[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = b[k] - a[k];
        v[k] = c[k] - a[k];
        w[k] = c[k] - b[k];
    }
    const double ru = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double rv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double rw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double p1 = 0.0, p2 = 0.0, p3 = 0.0;
    for (int k = 0; k < 3; ++k) {
        u[k] /= ru;
        v[k] /= rv;
        w[k] /= rw;
    }
    for (int k = 0; k < 3; ++k) {
        p1 += u[k] * v[k];
        p2 += u[k] * w[k];
        p3 += v[k] * w[k];
    }
    const double rr = ru * rv * rw;
    const double R3 = 3.0 / (rr * rr * rr);
    const double q = 5.0 * p1 * p2 * p3 - 1.0;
    const double su = R3 / ru, sv = R3 / rv;
    for (int k = 0; k < 3; ++k) {
        const double gu = su * (q * u[k] - p2 * p3 * v[k] - p1 * p3 * w[k]);
        const double gv = sv * (q * v[k] - p2 * p3 * u[k] - p1 * p2 * w[k]);
        g[k] = -gu - gv;
    }
}

// The gradient with respect to the point of slot s of (a0, a1, a2).
__device__ void grad_slot_f64(const double* a0, const double* a1, const double* a2, int s,
                              double g[3]) {
    if (s == 0) grad_first_f64(a0, a1, a2, g);
    else if (s == 1) grad_first_f64(a1, a0, a2, g);
    else grad_first_f64(a2, a0, a1, g);
}

// Warp-aggregated append: returns this lane's first slot.
__device__ __forceinline__ ull warp_append(ull* counter, int count) {
    const int lane = threadIdx.x & 31;
    int incl = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    ull base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(counter, (ull)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (ull)(incl - count);
}

// Children of a split (Algorithm 2 with all copies of the node split at once).
__device__ int split_children(const Trav& p, const int64_t P[3], int4 out[4]) {
    int ks = -1;
    double best = -1.0;
    for (int s = 0; s < 3; ++s) {
        if (is_leaf(p, P[s])) continue;
        const double d = p.ndiam2[P[s]];
        if (d > best) {
            best = d;
            ks = s;
        }
    }
    const int64_t v = P[ks], L = 2 * v + 1, R = 2 * v + 2;
    const bool e01 = P[0] == P[1], e12 = P[1] == P[2];
    if (e01 && e12) {
        out[0] = make_int4((int)L, (int)L, (int)L, 0);
        out[1] = make_int4((int)L, (int)L, (int)R, 0);
        out[2] = make_int4((int)L, (int)R, (int)R, 0);
        out[3] = make_int4((int)R, (int)R, (int)R, 0);
        return 4;
    }
    if (e01 && ks <= 1) {
        out[0] = make_int4((int)L, (int)L, (int)P[2], 0);
        out[1] = make_int4((int)L, (int)R, (int)P[2], 0);
        out[2] = make_int4((int)R, (int)R, (int)P[2], 0);
        return 3;
    }
    if (e12 && ks >= 1) {
        out[0] = make_int4((int)P[0], (int)L, (int)L, 0);
        out[1] = make_int4((int)P[0], (int)L, (int)R, 0);
        out[2] = make_int4((int)P[0], (int)R, (int)R, 0);
        return 3;
    }
    int64_t A[3] = {P[0], P[1], P[2]}, B[3] = {P[0], P[1], P[2]};
    A[ks] = L;
    B[ks] = R;
    out[0] = make_int4((int)A[0], (int)A[1], (int)A[2], 0);
    out[1] = make_int4((int)B[0], (int)B[1], (int)B[2], 0);
    return 2;
}

// Node sizes, T_i and distinct-slot flags of a triple.
__device__ void triple_counts(const Trav& p, const int64_t P[3], double n[3], double T[3],
                              bool first[3]) {
    for (int s = 0; s < 3; ++s) {
        int64_t b, e;
        node_range(P[s], p.N, b, e);
        n[s] = (double)(e - b);
    }
    for (int s = 0; s < 3; ++s) T[s] = tuples_for_slot(P, n, s);
    first[0] = true;
    first[1] = P[1] != P[0];
    first[2] = P[2] != P[1];
}

enum : int { kActNone = 0, kActDet = 1, kActMC = 2, kActBase = 3, kActSplit = 4 };

// F = false: the potential (p = 0 interval of phi, credit T_i phi(c1, c2, c3)).
// F = true : the forces (bound M_s on |grad phi|_2 over the boxes, prune iff
//            2 M_s <= (eps A^l(P_s) + tau) / T^root for every distinct slot;
//            credit -T_s grad_s phi(c1, c2, c3)).
template <bool F>
__global__ void classify_kernel(const int4* __restrict__ front, int64_t n_front, Trav p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int act = kActNone;
    int4 kids[4];
    int n_kids = 0;
    int4 me = make_int4(0, 0, 0, 0);
    if (i < n_front) {
        me = front[i];
        const int64_t P[3] = {me.x, me.y, me.z};
        double n[3], T[3];
        bool first[3];
        triple_counts(p, P, n, T, first);
        double sl[3], sh[3];
        box_d2(p, P[0], P[1], sl[0], sh[0]);
        box_d2(p, P[0], P[2], sl[1], sh[1]);
        box_d2(p, P[1], P[2], sl[2], sh[2]);
        // Touching boxes (d^l = 0, e.g. a repeated node) leave phi_hi = +inf:
        // the width is infinite and the rule cannot prune; skip its arithmetic.
        bool prune = false;
        if (F) {
            if (sl[0] > 0.0 && sl[1] > 0.0 && sl[2] > 0.0) {
                const double prod = __dmul_rn(__dmul_rn(sl[0], sl[1]), sl[2]);
                const double rmax = __ddiv_rn(1.0, __dmul_rn(prod, __dsqrt_rn(prod)));
                const double i0 = __ddiv_rn(1.0, __dsqrt_rn(sl[0]));
                const double i1 = __ddiv_rn(1.0, __dsqrt_rn(sl[1]));
                const double i2 = __ddiv_rn(1.0, __dsqrt_rn(sl[2]));
                const double r18 = __dmul_rn(18.0, rmax);
                // edges at slot 0: (0-1, 0-2); slot 1: (0-1, 1-2); slot 2: (0-2, 1-2)
                const double M[3] = {__dmul_rn(r18, __dadd_rn(i0, i1)),
                                     __dmul_rn(r18, __dadd_rn(i0, i2)),
                                     __dmul_rn(r18, __dadd_rn(i1, i2))};
                prune = true;
                for (int s2 = 0; s2 < 3; ++s2) {
                    if (!first[s2]) continue;
                    const double budget = __ddiv_rn(
                        __dadd_rn(__dmul_rn(p.eps, p.nscale[P[s2]]), p.tau), p.troot);
                    if (!(__dmul_rn(2.0, M[s2]) <= budget)) prune = false;
                }
            }
        } else if (sl[0] > 0.0 && sl[1] > 0.0 && sl[2] > 0.0) {
            double plo, phi_hi;
            phi_interval(sl[0], sh[0], sl[1], sh[1], sl[2], sh[2], plo, phi_hi);
            const double width = __dsub_rn(phi_hi, plo);
            const double amax = fabs(plo) > fabs(phi_hi) ? fabs(plo) : fabs(phi_hi);
            double lb = INFINITY;
            for (int s = 0; s < 3; ++s) {
                if (!first[s]) continue;
                const double v = __dsub_rn(p.nphil[P[s]], __dmul_rn(T[s], amax));
                if (v < lb) lb = v;
            }
            const double budget =
                __ddiv_rn(__dadd_rn(__dmul_rn(p.eps, lb > 0.0 ? lb : 0.0), p.tau), p.troot);
            prune = width <= budget;
        }
        if (prune) {
            act = kActDet;
            if (F) {
                for (int s = 0; s < 3; ++s) {
                    if (!first[s]) continue;
                    double g[3];
                    grad_slot_f64(p.ncen + 3 * P[0], p.ncen + 3 * P[1], p.ncen + 3 * P[2], s, g);
                    for (int d = 0; d < 3; ++d) atomicAdd(&p.node_acc3[3 * P[s] + d], -T[s] * g[d]);
                    if (p.node_cnt) atomicAdd(&p.node_cnt[P[s]], (ull)T[s]);
                }
            } else {
                const double f = phi_f64(p.ncen + 3 * P[0], p.ncen + 3 * P[1], p.ncen + 3 * P[2]);
                for (int s = 0; s < 3; ++s) {
                    if (!first[s]) continue;
                    atomicAdd(&p.node_acc[P[s]], T[s] * f);
                    if (p.node_cnt) atomicAdd(&p.node_cnt[P[s]], (ull)T[s]);
                }
            }
        } else {
            double tmin = T[0];
            for (int s = 1; s < 3; ++s)
                if (T[s] < tmin) tmin = T[s];
            if (p.alpha > 0.0 && tmin >= 1.0 && __dmul_rn(p.zeta, (double)p.m_limit) <= tmin) {
                act = kActMC;
            } else if (is_leaf(p, P[0]) && is_leaf(p, P[1]) && is_leaf(p, P[2])) {
                act = kActBase;
            } else {
                act = kActSplit;
                n_kids = split_children(p, P, kids);
            }
        }
    }
    // statistics
    const unsigned act_mask = __ballot_sync(0xffffffffu, act != kActNone);
    const unsigned det_mask = __ballot_sync(0xffffffffu, act == kActDet);
    const unsigned mc_mask = __ballot_sync(0xffffffffu, act == kActMC);
    if ((threadIdx.x & 31) == 0) {
        if (act_mask) atomicAdd(&p.stat[0], (ull)__popc(act_mask));
        if (det_mask) atomicAdd(&p.stat[1], (ull)__popc(det_mask));
        if (mc_mask) atomicAdd(&p.stat[3], (ull)__popc(mc_mask));
    }
    // appends
    const ull mo = warp_append(p.n_mc, act == kActMC ? 1 : 0);
    if (act == kActMC) {
        if ((int64_t)mo < p.cap_mc) p.mc[mo] = me;
        else atomicOr(p.flags, MBM_FLAG_OVERFLOW);
    }
    const ull bo = warp_append(p.n_base, act == kActBase ? 1 : 0);
    if (act == kActBase) {
        if ((int64_t)bo < p.cap_base) p.base[bo] = me;
        else atomicOr(p.flags, MBM_FLAG_OVERFLOW);
    }
    const ull no = warp_append(p.n_next, n_kids);
    for (int c = 0; c < n_kids; ++c) {
        if ((int64_t)(no + c) < p.cap_next) p.next[no + c] = kids[c];
        else atomicOr(p.flags, MBM_FLAG_OVERFLOW);
    }
}

// ---------------------------------------------------------------------------
// a7: Monte Carlo (Algorithms 3-5).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t r[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    r[0] = c0;
    r[1] = c1;
    r[2] = c2;
    r[3] = c3;
}

__device__ __forceinline__ int64_t draw_below(uint32_t r, int64_t n) {
    return (int64_t)(((ull)r * (ull)n) >> 32);
}

// Distinct (u, w) from [b, b+n) minus x if excl; a uniform unordered pair.
__device__ __forceinline__ void pair_from(int64_t b, int64_t n, bool excl, int64_t x, uint32_t r0,
                                          uint32_t r1, int64_t& y, int64_t& z) {
    const int64_t m = n - (excl ? 1 : 0);
    int64_t u = draw_below(r0, m), w = draw_below(r1, m - 1);
    if (w >= u) ++w;
    if (excl) {
        if (b + u >= x) ++u;
        if (b + w >= x) ++w;
    }
    y = b + u;
    z = b + w;
}

// One tuple containing sorted particle x (slot `slot`) of triple P.
__device__ void draw_partners(const int64_t P[3], const int64_t bb[3], const int64_t nn[3], int slot,
                              int64_t x, uint32_t r0, uint32_t r1, int64_t& y, int64_t& z) {
    const bool e01 = P[0] == P[1], e12 = P[1] == P[2];
    if (e01 && e12) {
        pair_from(bb[0], nn[0], true, x, r0, r1, y, z);
    } else if (e01) {
        if (slot == 2) {
            pair_from(bb[0], nn[0], false, x, r0, r1, y, z);
        } else {
            int64_t u = draw_below(r0, nn[0] - 1);
            if (bb[0] + u >= x) ++u;
            y = bb[0] + u;
            z = bb[2] + draw_below(r1, nn[2]);
        }
    } else if (e12) {
        if (slot == 0) {
            pair_from(bb[1], nn[1], false, x, r0, r1, y, z);
        } else {
            y = bb[0] + draw_below(r0, nn[0]);
            int64_t u = draw_below(r1, nn[1] - 1);
            if (bb[1] + u >= x) ++u;
            z = bb[1] + u;
        }
    } else {
        const int o1 = slot == 0 ? 1 : 0, o2 = slot == 2 ? 1 : 2;
        y = bb[o1] + draw_below(r0, nn[o1]);
        z = bb[o2] + draw_below(r1, nn[o2]);
    }
}

// Unit vector and r^-3 of one pair for Monte Carlo samples: one Newton step
// on rsqrt, rho = y^3 (a few ulp; a sample's rounding is far below the
// sampling error it feeds).
__device__ __forceinline__ mbm_tile::PairF pair_sample(float4 ph, float4 pl, float4 qh, float4 ql) {
    const float dx = (qh.x - ph.x) + (ql.x - pl.x);
    const float dy = (qh.y - ph.y) + (ql.y - pl.y);
    const float dz = (qh.z - ph.z) + (ql.z - pl.z);
    const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float y = rsqrtf(s);
    y = fmaf(0.5f * y, fmaf(-s * y, y, 1.0f), y);
    mbm_tile::PairF r;
    r.ex = dx * y;
    r.ey = dy * y;
    r.ez = dz * y;
    r.rho = y * y * y;
    return r;
}

// phi of one point triple in FP32 bulk (direction-cosine form); the first
// point is given (hi/lo), the other two are loaded.
__device__ __forceinline__ float phi_fp32(float4 ah, float4 al, const float4* xh, const float4* xl,
                                          int64_t b, int64_t c) {
    const float4 bh = xh[b], bl = xl[b], ch = xh[c], cl = xl[c];
    const mbm_tile::PairF ab = pair_sample(ah, al, bh, bl);
    const mbm_tile::PairF ac = pair_sample(ah, al, ch, cl);
    const mbm_tile::PairF bc = pair_sample(bh, bl, ch, cl);
    const float p1 = ab.ex * ac.ex + ab.ey * ac.ey + ab.ez * ac.ez;
    const float p2 = ab.ex * bc.ex + ab.ey * bc.ey + ab.ez * bc.ez;
    const float p3 = ac.ex * bc.ex + ac.ey * bc.ey + ac.ez * bc.ez;
    const float n = fmaf(p1 * p2 * p3, -3.0f, 1.0f);
    return n * (ab.rho * ac.rho * bc.rho);
}

// Particles of a candidate in order: slot 0's node, then each later distinct node.
__device__ __forceinline__ void candidate_point(const Trav& p, const int64_t P[3], int64_t u,
                                                int& slot, int64_t& x) {
    int64_t off = 0;
    for (int s = 0; s < 3; ++s) {
        if (s > 0 && P[s] == P[s - 1]) continue;
        int64_t b, e;
        node_range(P[s], p.N, b, e);
        if (u < off + (e - b)) {
            slot = s;
            x = b + (u - off);
            return;
        }
        off += e - b;
    }
    slot = 2;
    x = 0;
}


// Algorithm 4 for up to 32 particles of candidate P, one per lane. A
// particle that fails sets *fail; all lanes stop once *fail is set (Algorithm 3
// returns false at the first failing particle). Returns T_i * mean.
__device__ double mc_warp(const Trav& p, const int64_t P[3], const int64_t bb[3],
                          const int64_t nn[3], bool active, int slot, int64_t x, double Ti,
                          volatile int* fail) {
    const int lane = threadIdx.x & 31;
    const double phil = active ? p.pphil[x] : 0.0;  // the particle's own Phi^l
    // The bound never exceeds rhs_max = (eps Phi^l(x) + tau)/T^root (rule 0;
    // rule 1 divides the eps term by T_i), so z^2 sigma^2 > rhs_max^2 (with
    // slack for rounding) fails the stop test without evaluating it.
    const double rhs_max = __dmul_rn(
        __dadd_rn(p.mc_rule == 1 ? __ddiv_rn(__dmul_rn(p.eps, phil), Ti) : __dmul_rn(p.eps, phil),
                  p.tau),
        p.inv_troot);
    const double reject_v = __dmul_rn(__dmul_rn(rhs_max, rhs_max) / (p.z * p.z), 1.0 + 1e-9);
    // m2 never decreases with m, so at every later m' <= m_limit the variance
    // of the mean is at least m2 / ((m_limit - 1) m_limit). Once that exceeds
    // reject_v the stop test cannot pass any more and the particle would fail
    // at m_limit: it fails now (same decision, fewer samples). An update of
    // m2 can round below zero only when a sample lies within a few ulps of
    // the mean, by at most ~ulp(mean)^2 per sample; the relative and the
    // mean^2 slack cover m_limit such updates.
    const double hopeless_m2 =
        __dmul_rn(__dmul_rn(reject_v, (double)(p.m_limit - 1) * (double)p.m_limit), 1.0 + 1e-9);
    double mean = 0.0, m2 = 0.0;
    int m = 0, next_test = 30;
    bool pass = false, done = !active;
    int samples = 0, iter = 0;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xh0 = active ? p.xh[x] : z4, xl0 = active ? p.xl[x] : z4;
    // One sample: Welford update and the stop test of Algorithm 4 at count m.
    auto step = [&](double f) {
        ++m;
        ++samples;
        // Welford updates of the running mean and sum of squares (fused)
        const double dlt = __dsub_rn(f, mean);
        mean = __fma_rn(dlt, p.rcp[m], mean);
        m2 = __fma_rn(dlt, __dsub_rn(f, mean), m2);
        // Tests before next_test are skipped: each would fail the
        // variance comparison below (m2 never decreases).
        const bool testing = m >= 2 && ((m >= 30 && m >= next_test) || m >= p.m_limit);
        const double var_mu = testing ? __dmul_rn(__dmul_rn(m2, p.rcp[m - 1]), p.rcp[m]) : 0.0;
        if (m >= 2 && m2 > hopeless_m2 &&
            m2 > hopeless_m2 + 1e-20 * mean * mean) {  // no later m can pass
            pass = false;
            done = true;
        } else if (testing && var_mu > reject_v) {  // cannot pass at this m
            pass = false;
            if (m >= p.m_limit) {
                done = true;
            } else if (reject_v > 0.0) {
                // The first m' that can pass has (m'-1) m' >= m2 / reject_v; the
                // root is taken in FP32 from a bound shrunk by 1e-4 (and by the
                // rounding slack of m2), so every skipped m' would fail here.
                const float K =
                    (float)((m2 - 1e-20 * mean * mean) / reject_v) * 0.9999f;
                if (K > 0.0f) {
                    const float root = 0.5f * (1.0f + sqrtf(fmaf(4.0f, K, 1.0f)));
                    const int nt = root < (float)p.m_limit ? (int)root : p.m_limit;
                    if (nt > next_test) next_test = nt;
                }
            }
        } else if (testing) {  // the test can end the loop only here
            // sigma_mu = sqrt(m2 / (m-1) / m), with exact reciprocals
            const double sig = __dsqrt_rn(var_mu);
            const double lhs = __dmul_rn(p.z, sig);
            double lb = __dsub_rn(phil, __dmul_rn(Ti, __dadd_rn(fabs(mean), __dmul_rn(p.z, sig))));
            if (lb < 0.0) lb = 0.0;
            const double rhs =
                p.mc_rule == 1
                    ? __dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(p.eps, lb), Ti), p.tau), p.inv_troot)
                    : __dmul_rn(__dadd_rn(__dmul_rn(p.eps, lb), p.tau), p.inv_troot);
            pass = lhs <= rhs;
            if ((pass && m >= 30) || m >= p.m_limit) done = true;
        } else if (m >= p.m_limit) {  // m_limit < 2
            pass = false;
            done = true;
        }
        if (done && !pass) *fail = 1;
    };
    while (__any_sync(0xffffffffu, !done)) {
        if (!done) {
            // One Philox call serves samples m and m+1 (m even; words 0,1 and
            // 2,3). Both are drawn and evaluated before either is used, so
            // their point loads overlap; they are then taken in order, and the
            // second is dropped if the first ends the loop.
            const int c = m >> 1;
            const uint32_t ctr1 = (uint32_t)P[0] | ((uint32_t)(c & 0xFF) << 24);
            const uint32_t ctr2 = (uint32_t)P[1] | ((uint32_t)((c >> 8) & 0xFF) << 24);
            uint32_t rr[4];
            philox4x32_10((uint32_t)x, ctr1, ctr2, (uint32_t)P[2], p.key0, p.key1, rr);
            int64_t y0, z0, y1, z1;
            draw_partners(P, bb, nn, slot, x, rr[0], rr[1], y0, z0);
            draw_partners(P, bb, nn, slot, x, rr[2], rr[3], y1, z1);
            const float f0 = phi_fp32(xh0, xl0, p.xh, p.xl, y0, z0);
            const float f1 = phi_fp32(xh0, xl0, p.xh, p.xl, y1, z1);
            step((double)f0);
            if (!done) step((double)f1);
        }
        if ((++iter & 15) == 0) {  // another particle already failed: stop the warp
            int f = lane == 0 ? *fail : 0;
            if (__shfl_sync(0xffffffffu, f, 0)) break;
        }
    }
    int tot = samples;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) atomicAdd(&p.stat[5], (ull)tot);
    return __dmul_rn(Ti, mean);
}


// Unit vector, r^-3 and r^-1 of one pair (as pair_sample).
struct PairFY {
    float ex, ey, ez, rho, y;
};
__device__ __forceinline__ PairFY pair_sample_y(float4 ph, float4 pl, float4 qh, float4 ql) {
    const float dx = (qh.x - ph.x) + (ql.x - pl.x);
    const float dy = (qh.y - ph.y) + (ql.y - pl.y);
    const float dz = (qh.z - ph.z) + (ql.z - pl.z);
    const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float y = rsqrtf(s);
    y = fmaf(0.5f * y, fmaf(-s * y, y, 1.0f), y);
    PairFY r;
    r.ex = dx * y;
    r.ey = dy * y;
    r.ez = dz * y;
    r.y = y;
    r.rho = y * y * y;
    return r;
}

// grad_a phi(a, b, c) in FP32 bulk (pair-vector form, as grad_first_f64),
// from hi/lo coordinates of a, b and c.
__device__ __forceinline__ float3 grad_first_fp32(float4 ah, float4 al, float4 bh, float4 bl,
                                                  float4 ch, float4 cl) {
    const PairFY ab = pair_sample_y(ah, al, bh, bl);
    const PairFY ac = pair_sample_y(ah, al, ch, cl);
    const PairFY bc = pair_sample_y(bh, bl, ch, cl);
    const float p1 = ab.ex * ac.ex + ab.ey * ac.ey + ab.ez * ac.ez;
    const float p2 = ab.ex * bc.ex + ab.ey * bc.ey + ab.ez * bc.ez;
    const float p3 = ac.ex * bc.ex + ac.ey * bc.ey + ac.ez * bc.ez;
    const float q = fmaf(5.0f, p1 * p2 * p3, -1.0f);
    const float R3 = 3.0f * (ab.rho * ac.rho * bc.rho);
    const float su = R3 * ab.y, sv = R3 * ac.y;  // 3R / r_ab, 3R / r_ac
    const float p23 = p2 * p3, p13 = p1 * p3, p12 = p1 * p2;
    float3 g;
    g.x = -su * (q * ab.ex - p23 * ac.ex - p13 * bc.ex) - sv * (q * ac.ex - p23 * ab.ex - p12 * bc.ex);
    g.y = -su * (q * ab.ey - p23 * ac.ey - p13 * bc.ey) - sv * (q * ac.ey - p23 * ab.ey - p12 * bc.ey);
    g.z = -su * (q * ab.ez - p23 * ac.ez - p13 * bc.ez) - sv * (q * ac.ez - p23 * ab.ez - p12 * bc.ez);
    return g;
}

// Algorithm 4 for the forces: the sample is the three components of
// grad_x phi(x, y, z); a particle passes iff z sigma_d <= rhs for d = 1..3 with
// rhs = (eps A^l(x) + tau) / T^root (the force criterion). Same draws, counts
// and early stops as mc_warp. Writes the estimate -T_i mu to est[3].
__device__ void mc_warp_forces(const Trav& p, const int64_t P[3], const int64_t bb[3],
                               const int64_t nn[3], bool active, int slot, int64_t x, double Ti,
                               volatile int* fail, double est[3]) {
    const int lane = threadIdx.x & 31;
    const double scale = active ? p.pscale[x] : 0.0;
    const double rhs = __dmul_rn(__dadd_rn(__dmul_rn(p.eps, scale), p.tau), p.inv_troot);
    const double reject_v = __dmul_rn(__dmul_rn(rhs, rhs) / (p.z * p.z), 1.0 + 1e-9);
    const double hopeless_m2 =
        __dmul_rn(__dmul_rn(reject_v, (double)(p.m_limit - 1) * (double)p.m_limit), 1.0 + 1e-9);
    double mean[3] = {0.0, 0.0, 0.0}, m2[3] = {0.0, 0.0, 0.0};
    int m = 0;
    bool pass = false, done = !active;
    int samples = 0, iter = 0;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xh0 = active ? p.xh[x] : z4, xl0 = active ? p.xl[x] : z4;
    auto step = [&](float3 g) {
        ++m;
        ++samples;
        const double gv[3] = {(double)g.x, (double)g.y, (double)g.z};
        double m2max = 0.0, mmax = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double dlt = __dsub_rn(gv[d], mean[d]);
            mean[d] = __fma_rn(dlt, p.rcp[m], mean[d]);
            m2[d] = __fma_rn(dlt, __dsub_rn(gv[d], mean[d]), m2[d]);
            m2max = fmax(m2max, m2[d]);
            mmax = fmax(mmax, fabs(mean[d]));
        }
        const bool testing = m >= 2 && (m >= 30 || m >= p.m_limit);
        if (m >= 2 && m2max > hopeless_m2 && m2max > hopeless_m2 + 1e-20 * mmax * mmax) {
            pass = false;  // no later m can pass (m2 never decreases)
            done = true;
        } else if (testing) {
            pass = true;
            for (int d = 0; d < 3; ++d) {
                const double sig = __dsqrt_rn(__dmul_rn(__dmul_rn(m2[d], p.rcp[m - 1]), p.rcp[m]));
                if (!(__dmul_rn(p.z, sig) <= rhs)) pass = false;
            }
            if ((pass && m >= 30) || m >= p.m_limit) done = true;
        } else if (m >= p.m_limit) {
            pass = false;
            done = true;
        }
        if (done && !pass) *fail = 1;
    };
    while (__any_sync(0xffffffffu, !done)) {
        if (!done) {
            const int c = m >> 1;
            const uint32_t ctr1 = (uint32_t)P[0] | ((uint32_t)(c & 0xFF) << 24);
            const uint32_t ctr2 = (uint32_t)P[1] | ((uint32_t)((c >> 8) & 0xFF) << 24);
            uint32_t rr[4];
            philox4x32_10((uint32_t)x, ctr1, ctr2, (uint32_t)P[2], p.key0, p.key1, rr);
            int64_t y0, z0, y1, z1;
            draw_partners(P, bb, nn, slot, x, rr[0], rr[1], y0, z0);
            draw_partners(P, bb, nn, slot, x, rr[2], rr[3], y1, z1);
            const float3 g0 = grad_first_fp32(xh0, xl0, p.xh[y0], p.xl[y0], p.xh[z0], p.xl[z0]);
            const float3 g1 = grad_first_fp32(xh0, xl0, p.xh[y1], p.xl[y1], p.xh[z1], p.xl[z1]);
            step(g0);
            if (!done) step(g1);
        }
        if ((++iter & 15) == 0) {
            int f = lane == 0 ? *fail : 0;
            if (__shfl_sync(0xffffffffu, f, 0)) break;
        }
    }
    int tot = samples;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) atomicAdd(&p.stat[5], (ull)tot);
    for (int d = 0; d < 3; ++d) est[d] = -__dmul_rn(Ti, mean[d]);
}

__device__ __forceinline__ void candidate_geometry(const Trav& p, const int64_t P[3], double T[3],
                                                   bool first[3], int64_t bb[3], int64_t nn[3],
                                                   int64_t& U) {
    double n[3];
    triple_counts(p, P, n, T, first);
    U = 0;
    for (int s = 0; s < 3; ++s) {
        int64_t e;
        node_range(P[s], p.N, bb[s], e);
        nn[s] = e - bb[s];
        if (first[s]) U += nn[s];
    }
}

// Probe: each distinct node's particles with the smallest Phi^l(x) (the
// likeliest to fail) run first, a warp per candidate: 32, 16 or 10 of them
// per node for 1, 2 or 3 distinct nodes, so the lanes are filled. A particle's
// draws depend only on its own ids, so decisions do not depend on this order.
template <bool F>
__global__ void mc_probe_kernel(const int4* __restrict__ mc, int64_t n_c, int* cand_fail, Trav p) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= n_c) return;
    const int4 t = mc[c];
    const int64_t P[3] = {t.x, t.y, t.z};
    volatile int* fail = cand_fail + c;
    double T[3];
    bool first[3];
    int64_t bb[3], nn[3], U;
    candidate_geometry(p, P, T, first, bb, nn, U);
    int ds[3], d = 0;  // distinct slots in order
    for (int s = 0; s < 3; ++s)
        if (first[s]) ds[d++] = s;
    const int per = d == 1 ? 32 : (d == 2 ? 16 : 10);
    const int q = lane / per;
    const int slot = q < d ? ds[q] : 0;
    const int x = q < d ? p.weak[P[slot] * 32 + (lane % per)] : -1;
    if (F) {
        double e3[3];
        mc_warp_forces(p, P, bb, nn, x >= 0, slot, x >= 0 ? x : 0, T[slot], fail, e3);
    } else {
        mc_warp(p, P, bb, nn, x >= 0, slot, x >= 0 ? x : 0, T[slot], fail);
    }
}

__global__ void mc_sizes_kernel(const int4* __restrict__ mc, int64_t n_mc, int64_t N,
                                const int* __restrict__ cand_fail, int64_t* chunks) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_mc) return;
    if (cand_fail[c]) {
        chunks[c] = 0;
        return;
    }
    const int4 t = mc[c];
    const int64_t P[3] = {t.x, t.y, t.z};
    int64_t U = 0;
    for (int s = 0; s < 3; ++s) {
        if (s > 0 && P[s] == P[s - 1]) continue;
        int64_t b, e;
        node_range(P[s], N, b, e);
        U += e - b;
    }
    chunks[c] = (U + 31) / 32;
}

// One warp per 32-particle chunk of a candidate that passed the probe
// (forces: 3 estimates per particle).
template <bool F>
__global__ void mc_kernel(const int4* __restrict__ mc, int64_t c0, int64_t n_c,
                          const int64_t* __restrict__ chunk_off /* exclusive, n_c + 1 */,
                          int* cand_fail, double* est, Trav p) {
    const int lane = threadIdx.x & 31;
    const int64_t rel = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (rel >= chunk_off[n_c] - chunk_off[0]) return;
    const int64_t chunk = chunk_off[0] + rel;
    int64_t lo = 0, hi = n_c;  // largest c with chunk_off[c] <= chunk
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        if (chunk_off[mid] <= chunk) lo = mid;
        else hi = mid;
    }
    const int64_t c = lo;
    volatile int* fail = cand_fail + c;
    if (*fail) return;  // warp-uniform
    const int4 t = mc[c0 + c];
    const int64_t P[3] = {t.x, t.y, t.z};
    double T[3];
    bool first[3];
    int64_t bb[3], nn[3], U;
    candidate_geometry(p, P, T, first, bb, nn, U);
    const int64_t u = (chunk - chunk_off[c]) * 32 + lane;
    const bool active = u < U;
    int slot = 0;
    int64_t x = 0;
    if (active) candidate_point(p, P, u, slot, x);
    if (F) {
        double e3[3];
        mc_warp_forces(p, P, bb, nn, active, slot, x, T[slot], fail, e3);
        if (active)
            for (int d = 0; d < 3; ++d) est[3 * (rel * 32 + lane) + d] = e3[d];
    } else {
        const double e = mc_warp(p, P, bb, nn, active, slot, x, T[slot], fail);
        if (active) est[rel * 32 + lane] = e;
    }
}

// Algorithm 5 for passing candidates; failing ones go on to base/split.
template <bool F>
__global__ void mc_commit_kernel(const int4* __restrict__ mc, int64_t c0, int64_t n_c,
                                 const int64_t* __restrict__ chunk_off, const int* cand_fail,
                                 const double* est, Trav p) {
    const int64_t c = blockIdx.x;
    if (c >= n_c) return;
    const int4 t = mc[c0 + c];
    const int64_t P[3] = {t.x, t.y, t.z};
    if (!cand_fail[c]) {
        double n[3], T[3];
        bool first[3];
        triple_counts(p, P, n, T, first);
        int64_t U = 0;
        for (int s = 0; s < 3; ++s)
            if (first[s]) U += (int64_t)n[s];
        for (int64_t u = threadIdx.x; u < U; u += blockDim.x) {
            int slot;
            int64_t x;
            candidate_point(p, P, u, slot, x);
            const int64_t eo = chunk_off[c] * 32 + u - chunk_off[0] * 32;
            if (F) {
                for (int d = 0; d < 3; ++d) atomicAdd(&p.pt_acc3[3 * x + d], est[3 * eo + d]);
            } else {
                atomicAdd(&p.pt_acc[x], est[eo]);
            }
            if (p.pt_cnt) atomicAdd(&p.pt_cnt[x], (ull)T[slot]);
        }
        if (threadIdx.x == 0) atomicAdd(&p.stat[2], 1ULL);
        return;
    }
    if (threadIdx.x != 0) return;
    if (is_leaf(p, P[0]) && is_leaf(p, P[1]) && is_leaf(p, P[2])) {
        const ull o = atomicAdd(p.n_base, 1ULL);
        if ((int64_t)o < p.cap_base) p.base[o] = t;
        else atomicOr(p.flags, MBM_FLAG_OVERFLOW);
        return;
    }
    int4 kids[4];
    const int k = split_children(p, P, kids);
    const ull o = atomicAdd(p.n_next, (ull)k);
    for (int q = 0; q < k; ++q) {
        if ((int64_t)(o + q) < p.cap_next) p.next[o + q] = kids[q];
        else atomicOr(p.flags, MBM_FLAG_OVERFLOW);
    }
}

// ---------------------------------------------------------------------------
// a9: top-down push and output in the caller's order.
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(int64_t N, int depth, int64_t n_nodes, int64_t n_leaves,
                                const int64_t* __restrict__ perm, const double* __restrict__ pt_acc,
                                const double* __restrict__ node_acc, const ull* pt_cnt,
                                const ull* node_cnt, double* out, int64_t* counts_out) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int64_t q = (s << depth) / N;
    const int64_t first_leaf = n_nodes - n_leaves;
    int64_t b, e;
    node_range(first_leaf + q, N, b, e);
    while (b > s) {
        --q;
        node_range(first_leaf + q, N, b, e);
    }
    while (e <= s) {
        ++q;
        node_range(first_leaf + q, N, b, e);
    }
    int64_t v = first_leaf + q;
    double acc = 0.0;
    ull cnt = 0;
    for (;;) {
        acc += node_acc[v];
        if (node_cnt) cnt += node_cnt[v];
        if (v == 0) break;
        v = (v - 1) / 2;
    }
    out[perm[s]] = pt_acc[s] + acc;
    if (counts_out) counts_out[perm[s]] = (int64_t)(cnt + pt_cnt[s]);
}

// ---------------------------------------------------------------------------
// Tree forces: seed of the force scale, base cases, top-down push.
// ---------------------------------------------------------------------------
// A^l(x) = sum over the tuples inside x's seed node of |grad_x phi|_2, a warp
// per 32-particle chunk of a seed node (all lanes read the same partners).
__global__ void __launch_bounds__(128)
seed_scale_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int64_t N, int sd,
                  int chunks_per_node, double* __restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_nodes = (int64_t)1 << sd;
    if (item >= n_nodes * chunks_per_node) return;
    int64_t b, e;
    node_range(n_nodes - 1 + item / chunks_per_node, N, b, e);
    const int64_t x = b + (item % chunks_per_node) * 32 + lane;
    if (b + (item % chunks_per_node) * 32 >= e) return;  // warp-uniform
    const bool act = x < e;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ah = act ? xh[x] : z4, al = act ? xl[x] : z4;
    double acc = 0.0;
    for (int64_t y = b; y < e; ++y) {
        const float4 bh = xh[y], bl = xl[y];
        float row = 0.f;
        for (int64_t z = y + 1; z < e; ++z) {
            const float3 g = grad_first_fp32(ah, al, bh, bl, xh[z], xl[z]);
            const float n2 = fmaf(g.z, g.z, fmaf(g.y, g.y, g.x * g.x));
            row += (y != x && z != x) ? sqrtf(n2) : 0.f;
        }
        acc += (double)row;
    }
    if (act) scale[x] = acc;
}

// Exact forces of base cases (Fig. 4 leaf triples), a warp per item: for each
// distinct slot, a lane per particle a of that leaf sums grad_a phi over the
// partner pairs (b, c) the canonical case allows, and credits -grad. The
// partner pairs' terms (unit vector, r^-3) are built once per slot in the
// warp's shared table; a's terms to 8 columns c are held in registers and
// its term to row b is formed once per row, so the inner loop is the
// gradient alone. Masked pairs have zero terms and contribute exactly 0.
constexpr int kForceWarps = 4;
constexpr int kForceCols = 8;
// Largest seed level of the force criterion's A^l: the seed pass costs the
// seed node's size squared per particle and, for gradients, outweighs the
// base cases it saves beyond 2 048-point seed nodes (N = 65 536, eps = 1e-2:
// 11.3 s at 6 levels, 12.7 s at 7, 21.2 s at 8).
constexpr int kForceSeedMax = 6;

// The partner table holds half of the c columns at a time (8 KB per warp), so
// that five 4-warp CTAs (96 registers a thread) fit an SM: 20 warps.
constexpr int kForceHalf = kTile / 2;
struct ForceWarpSmem {
    float4 ph[3][kTile], pl[3][kTile];  // the three leaves (hi/lo)
    float4 tab[kTile][kForceHalf];      // partner pair (b, c): (e_bc, rho_bc), c in this half
};

__device__ __forceinline__ float3 grad_from_terms(const PairFY& ab, const PairFY& ac, float4 bc) {
    const float p1 = ab.ex * ac.ex + ab.ey * ac.ey + ab.ez * ac.ez;
    const float p2 = ab.ex * bc.x + ab.ey * bc.y + ab.ez * bc.z;
    const float p3 = ac.ex * bc.x + ac.ey * bc.y + ac.ez * bc.z;
    const float q = fmaf(5.0f, p1 * p2 * p3, -1.0f);
    const float R3 = 3.0f * (ab.rho * ac.rho * bc.w);
    const float su = R3 * ab.y, sv = R3 * ac.y;
    const float p23 = p2 * p3, p13 = p1 * p3, p12 = p1 * p2;
    float3 g;
    g.x = -su * (q * ab.ex - p23 * ac.ex - p13 * bc.x) - sv * (q * ac.ex - p23 * ab.ex - p12 * bc.x);
    g.y = -su * (q * ab.ey - p23 * ac.ey - p13 * bc.y) - sv * (q * ac.ey - p23 * ab.ey - p12 * bc.y);
    g.z = -su * (q * ab.ez - p23 * ac.ez - p13 * bc.z) - sv * (q * ac.ez - p23 * ab.ez - p12 * bc.z);
    return g;
}

__global__ void __launch_bounds__(kForceWarps * 32, 5)
base_forces_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int64_t N,
                   const int4* __restrict__ items, int64_t n_items, double* __restrict__ acc3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    ForceWarpSmem& sm = reinterpret_cast<ForceWarpSmem*>(smem_raw)[w];
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (item >= n_items) return;
    const int4 t = items[item];
    const int L[3] = {t.x, t.y, t.z};
    int64_t b[3];
    int n[3];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < 3; ++s) {
        int64_t e;
        node_range(L[s], N, b[s], e);
        n[s] = (int)(e - b[s]);
        sm.ph[s][lane] = lane < n[s] ? xh[b[s] + lane] : z4;
        sm.pl[s][lane] = lane < n[s] ? xl[b[s] + lane] : z4;
    }
    __syncwarp();
    for (int s = 0; s < 3; ++s) {
        if (s > 0 && L[s] == L[s - 1]) continue;
        const int o1 = s == 0 ? 1 : 0, o2 = s == 2 ? 1 : 2;
        const bool same = L[o1] == L[o2];
        const bool ex1 = L[o1] == L[s], ex2 = L[o2] == L[s];
        const float4 ah = sm.ph[s][lane], al = sm.pl[s][lane];
        const bool act = lane < n[s];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int h0 = 0; h0 < n[o2]; h0 += kForceHalf) {
            __syncwarp();  // the previous pass is done with the table
            for (int e = lane; e < kTile * kForceHalf; e += 32) {
                const int bi = e / kForceHalf, cr = e % kForceHalf, ci = h0 + cr;
                const bool v = bi < n[o1] && ci < n[o2] && (!same || bi < ci);
                float4 ent = z4;
                if (v) {
                    const PairFY bc = pair_sample_y(sm.ph[o1][bi], sm.pl[o1][bi], sm.ph[o2][ci],
                                                    sm.pl[o2][ci]);
                    ent = make_float4(bc.ex, bc.ey, bc.ez, bc.rho);
                }
                sm.tab[bi][cr] = ent;
            }
            __syncwarp();
            const int h1 = h0 + kForceHalf < n[o2] ? h0 + kForceHalf : n[o2];
            for (int cb = h0; cb < h1; cb += kForceCols) {
                PairFY ac[kForceCols];
#pragma unroll
                for (int q = 0; q < kForceCols; ++q) {
                    const int ci = cb + q;
                    const bool v = act && ci < n[o2] && !(ex2 && ci == lane);
                    ac[q] = pair_sample_y(ah, al, sm.ph[o2][ci & 31], sm.pl[o2][ci & 31]);
                    if (!v) ac[q] = PairFY{0.f, 0.f, 0.f, 0.f, 0.f};
                }
                for (int bi = 0; bi < n[o1]; ++bi) {
                    PairFY ab = pair_sample_y(ah, al, sm.ph[o1][bi], sm.pl[o1][bi]);
                    if (!act || (ex1 && bi == lane)) ab = PairFY{0.f, 0.f, 0.f, 0.f, 0.f};
                    float rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll
                    for (int q = 0; q < kForceCols; ++q) {
                        const float3 g = grad_from_terms(ab, ac[q], sm.tab[bi][cb - h0 + q]);
                        rx += g.x;
                        ry += g.y;
                        rz += g.z;
                    }
                    gx += (double)rx;
                    gy += (double)ry;
                    gz += (double)rz;
                }
            }
        }
        if (act) {
            const int64_t a = b[s] + lane;
            atomicAdd(&acc3[3 * a], -gx);
            atomicAdd(&acc3[3 * a + 1], -gy);
            atomicAdd(&acc3[3 * a + 2], -gz);
        }
    }
}

// Top-down push of the force accumulators and output in the caller's order.
__global__ void finalize3_kernel(int64_t N, int depth, int64_t n_nodes, int64_t n_leaves,
                                 const int64_t* __restrict__ perm, const double* __restrict__ pt3,
                                 const double* __restrict__ node3, const ull* pt_cnt,
                                 const ull* node_cnt, double* out3, int64_t* counts_out) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int64_t q = (s << depth) / N;
    const int64_t first_leaf = n_nodes - n_leaves;
    int64_t b, e;
    node_range(first_leaf + q, N, b, e);
    while (b > s) {
        --q;
        node_range(first_leaf + q, N, b, e);
    }
    while (e <= s) {
        ++q;
        node_range(first_leaf + q, N, b, e);
    }
    int64_t v = first_leaf + q;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    ull cnt = 0;
    for (;;) {
        a0 += node3[3 * v];
        a1 += node3[3 * v + 1];
        a2 += node3[3 * v + 2];
        if (node_cnt) cnt += node_cnt[v];
        if (v == 0) break;
        v = (v - 1) / 2;
    }
    const int64_t o = perm[s];
    out3[3 * o] = pt3[3 * s] + a0;
    out3[3 * o + 1] = pt3[3 * s + 1] + a1;
    out3[3 * o + 2] = pt3[3 * s + 2] + a2;
    if (counts_out) counts_out[o] = (int64_t)(cnt + pt_cnt[s]);
}

// Two-sided normal quantile: z with P(|Z| > z) = alpha, bisection on erfc.
double z_two_sided(double alpha) {
    if (!(alpha > 0.0)) return INFINITY;
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (std::erfc(mid / std::sqrt(2.0)) > alpha) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

unsigned grid_of(int64_t threads, int block) {
    int64_t g = (threads + block - 1) / block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 2147483647));
}

// (I,J,K) chunk triples, I <= J <= K < c.
std::vector<int4> chunk_combos(int c) {
    std::vector<int4> v;
    for (int i = 0; i < c; ++i)
        for (int j = i; j < c; ++j)
            for (int k = j; k < c; ++k) v.push_back(make_int4(i, j, k, 0));
    return v;
}

struct Carve {
    char* p;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = mbm_align_up(off, 256);
        T* r = reinterpret_cast<T*>(p + off);
        off += n * sizeof(T);
        return r;
    }
};

size_t carve_size(const std::vector<size_t>& parts) {
    size_t s = 0;
    for (size_t b : parts) s = mbm_align_up(s, 256) + b;
    return mbm_align_up(s, 256);
}

std::vector<size_t> tree_parts(int64_t N, int64_t n_nodes) {
    return {(size_t)N * 8, (size_t)N * 24, (size_t)N * 16, (size_t)N * 16,   // perm xs xh xl
            (size_t)n_nodes * 24, (size_t)n_nodes * 24, (size_t)n_nodes * 24,  // lo hi cen
            (size_t)n_nodes * 8, (size_t)n_nodes * 8, (size_t)N * 8,           // diam2 phil pphil
            (size_t)n_nodes * 32 * 4};                                          // weak
}

// Buffer capacities of one traversal and its scratch layout.
struct TravPlan {
    int64_t B = 0, cap_lvl = 0, cap_mc = 0, cap_base = 0, cap_est = 0;
    int max_levels = 0;
    size_t scan_tmp_bytes = 0, sort_bytes = 0;
    std::vector<size_t> parts;
};

TravPlan trav_plan(int64_t N, int depth, const mbm_config& cfg, bool forces) {
    const int m_limit = cfg.m_limit;
    const bool counting = cfg.tuple_counts != nullptr;
    TravPlan q;
    const int64_t n_nodes = ((int64_t)2 << depth) - 1, n_leaves = (int64_t)1 << depth;
    // Frontier chunk B: a chunk of B node triples yields at most 4B children,
    // B Monte Carlo candidates and B base cases, so no list can overflow.
    q.B = std::max<int64_t>(1 << 14, std::min<int64_t>(1 << 20, 16 * N));
    if (cfg.trav_chunk > 0) q.B = cfg.trav_chunk;
    q.max_levels = 3 * depth + 8;
    q.cap_lvl = 4 * q.B;
    q.cap_mc = q.B;
    // Base list: large flushes give long runs of equal (y, z) leaf pairs to the
    // grouped base kernel; never more than the number of canonical leaf
    // triples, which bounds the whole traversal's base cases.
    const double L = (double)n_leaves;
    const double all = L * (L + 1.0) * (L + 2.0) / 6.0;
    int64_t want = std::min<int64_t>(1 << 27, std::max<int64_t>(1 << 22, 512 * N));
    if ((double)want > all) want = (int64_t)all;
    if (cfg.base_cap > 0) want = cfg.base_cap;
    q.cap_base = std::max<int64_t>(q.B, want);
    // one candidate's estimates (its distinct nodes are disjoint, rounded up
    // to 32-point chunks) never exceed N + 96, so every batch holds at least one
    q.cap_est = 3 * N + 64 * 1024;
    if (cfg.est_cap > 0) q.cap_est = std::max<int64_t>(N + 128, cfg.est_cap);
    q.scan_tmp_bytes = mbm_scan_temp_bytes_i64(q.cap_mc + 1);
    // Base-case grouping: radix sort of (y, z) keys over 2 * depth bits and a
    // scan of piece flags share one temporary buffer.
    q.sort_bytes = mbm_sort_temp_bytes(q.cap_base);
    const size_t scan_bytes = mbm_scan_temp_bytes_i32(q.cap_base);
    q.sort_bytes = std::max(q.sort_bytes, scan_bytes);
    const size_t cb = (size_t)q.cap_base;
    q.parts = {
        (size_t)N * 8, (size_t)n_nodes * 8,                                // pt_acc node_acc
        counting ? (size_t)N * 8 : 0, counting ? (size_t)n_nodes * 8 : 0,  // counts
        (size_t)q.max_levels * q.cap_lvl * 16,                             // level buffers
        (size_t)q.cap_mc * 16, cb * 16,                                    // mc, base
        (size_t)(q.cap_mc + 2) * 8, (size_t)q.cap_mc * 4,                  // chunk_off, fail
        (size_t)q.cap_est * (forces ? 24 : 8), 256, q.scan_tmp_bytes,      // est, counters
        (size_t)(m_limit + 1) * 8,                                         // 1/m table
        cb * 8, cb * 8, cb * 4, cb * 4,                                    // base keys, x
        (cb + 1) * 4, (cb + 1) * 4, (cb + 1) * 4, 64, q.sort_bytes,        // flag pos heads
        forces ? (size_t)N * 24 : 0, forces ? (size_t)n_nodes * 24 : 0,    // pt_acc3 node_acc3
        forces ? (size_t)N * 8 : 0, forces ? (size_t)n_nodes * 8 : 0};     // pscale nscale
    return q;
}

}  // namespace

// ---------------------------------------------------------------------------
// Tree build (ABI).
// ---------------------------------------------------------------------------
static mbm_status build_tree(mbm_ctx* ctx, const double* X, int64_t N, const mbm_config& cfg,
                             cudaStream_t s, mbm_tree** out) {
    if (N < 3) return mbm_fail(MBM_EINVAL, "tree needs N >= 3");
    if (cfg.leaf_size < 2 || cfg.leaf_size > kTile) return mbm_fail(MBM_EINVAL, "leaf_size must be in [2, 32]");
    if (cfg.seed_levels < 0 || cfg.seed_levels > 8) return mbm_fail(MBM_EINVAL, "seed_levels must be in [0, 8]");
    const int depth = tree_depth(N, cfg.leaf_size);
    const int64_t n_nodes = ((int64_t)2 << depth) - 1, n_leaves = (int64_t)1 << depth;
    if (n_nodes >= (1 << 24)) return mbm_fail(MBM_EINVAL, "tree too large (node ids are 24-bit)");
    mbm_tree* t = new (std::nothrow) mbm_tree();
    if (!t) return mbm_fail(MBM_ENOMEM, "host allocation failed");
    t->ctx = ctx;
    t->device = ctx->device;
    t->N = N;
    t->leaf_size = cfg.leaf_size;
    t->depth = depth;
    t->n_nodes = n_nodes;
    t->n_leaves = n_leaves;
    t->seed_levels = cfg.seed_levels;
    const std::vector<size_t> parts = tree_parts(N, n_nodes);
    t->bytes = carve_size(parts);
    mbm_status st = mbm_budget_charge(ctx, t->bytes);
    if (st != MBM_OK) {
        delete t;
        return st;
    }
    cudaError_t e = cudaMalloc(&t->mem, t->bytes);
    if (e != cudaSuccess) {
        mbm_budget_release(ctx, t->bytes);
        delete t;
        return mbm_cuda_fail(e, "cudaMalloc(tree)");
    }
    Carve cv{static_cast<char*>(t->mem)};
    t->perm = cv.take<int64_t>(N);
    t->xs = cv.take<double>(3 * N);
    t->xh = cv.take<float4>(N);
    t->xl = cv.take<float4>(N);
    t->nlo = cv.take<double>(3 * n_nodes);
    t->nhi = cv.take<double>(3 * n_nodes);
    t->ncen = cv.take<double>(3 * n_nodes);
    t->ndiam2 = cv.take<double>(n_nodes);
    t->nphil = cv.take<double>(n_nodes);
    t->pphil = cv.take<double>(N);
    t->weak = cv.take<int>((size_t)n_nodes * 32);

    // Temporary scratch: box partials, keys/indices (double-buffered), sort temp, seed sums.
    const int nb = 256;
    const size_t sort_tmp_bytes = mbm_sort_temp_bytes(N);
    const int sd = std::max(0, depth - cfg.seed_levels);
    const int64_t max_seed = (N + ((int64_t)1 << sd) - 1) >> sd;  // ceil(N / 2^sd)
    const int chunks = (int)((max_seed + kTile - 1) / kTile);
    const std::vector<int4> cmb = chunk_combos(chunks);
    const std::vector<size_t> sparts = {(size_t)nb * 48, 64, (size_t)N * 8, (size_t)N * 8,
                                        (size_t)N * 4, (size_t)N * 4, sort_tmp_bytes, (size_t)N * 8,
                                        cmb.size() * 16};
    st = mbm_scratch_reserve(ctx, carve_size(sparts));
    if (st != MBM_OK) {
        mbm_tree_free(t);
        return st;
    }
    Carve sc{static_cast<char*>(ctx->scratch)};
    double* part = sc.take<double>(nb * 6);
    double* box = sc.take<double>(8);
    ull* k0 = sc.take<ull>(N);
    ull* k1 = sc.take<ull>(N);
    int* i0 = sc.take<int>(N);
    int* i1 = sc.take<int>(N);
    void* sort_tmp = sc.take<char>(sort_tmp_bytes);
    double* seed = sc.take<double>(N);
    int4* combos = sc.take<int4>(cmb.size());

#define TRY_LAUNCH()                                                           \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess) {                                               \
            mbm_tree_free(t);                                                  \
            return mbm_cuda_fail(e_, "tree build launch");                     \
        }                                                                      \
    } while (0)

    bbox_partial_kernel<<<nb, 256, 0, s>>>(X, N, part);
    bbox_final_kernel<<<1, 32, 0, s>>>(part, nb, box);
    morton_kernel<<<grid_of(N, 256), 256, 0, s>>>(X, N, box, k0, i0, ctx->d_flags);
    TRY_LAUNCH();
    e = mbm_sort_pairs_u64(k0, k1, i0, i1, N, 0, 63, sort_tmp, s);
    if (e != cudaSuccess) {
        mbm_tree_free(t);
        return mbm_cuda_fail(e, "radix sort");
    }
    gather_kernel<<<grid_of(N, 256), 256, 0, s>>>(X, N, i1, t->perm, t->xs, t->xh, t->xl);
    const int64_t first_leaf = n_nodes - n_leaves;
    leaf_stats_kernel<<<grid_of(n_leaves * 32, 256), 256, 0, s>>>(t->xs, N, first_leaf, n_leaves,
                                                                  t->nlo, t->nhi, t->ncen);
    for (int d = depth - 1; d >= 0; --d) {
        const int64_t first = ((int64_t)1 << d) - 1, cnt = (int64_t)1 << d;
        internal_stats_kernel<<<grid_of(cnt, 256), 256, 0, s>>>(first, cnt, t->nlo, t->nhi,
                                                                t->ncen);
    }
    node_finish_kernel<<<grid_of(n_nodes, 256), 256, 0, s>>>(N, n_nodes, t->nlo, t->nhi, t->ncen,
                                                             t->ndiam2);
    TRY_LAUNCH();

    // Phi^l seed: exact sums over triples inside each seed node.
    e = cudaMemcpyAsync(combos, cmb.data(), cmb.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(seed, 0, (size_t)N * 8, s);
    if (e != cudaSuccess) {
        mbm_tree_free(t);
        return mbm_cuda_fail(e, "seed set-up");
    }
    const int64_t n_seed_nodes = (int64_t)1 << sd;
    const size_t wsm = sizeof(WarpSmem) * kRangeWarps;
    cudaFuncSetAttribute((const void*)seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)wsm);
    seed_kernel<<<grid_of(n_seed_nodes * (int64_t)cmb.size() * 32, kRangeWarps * 32),
                  kRangeWarps * 32, wsm, s>>>(t->xh, t->xl, N, sd, n_seed_nodes, combos,
                                              (int)cmb.size(), seed, ctx->d_flags);
    phil_leaf_kernel<<<grid_of(n_leaves * 32, 256), 256, 0, s>>>(seed, N, first_leaf, n_leaves,
                                                                 t->nphil, t->pphil);
    for (int d = depth - 1; d >= 0; --d) {
        const int64_t first = ((int64_t)1 << d) - 1, cnt = (int64_t)1 << d;
        phil_internal_kernel<<<grid_of(cnt, 256), 256, 0, s>>>(first, cnt, t->nphil);
    }
    weak_leaf_kernel<<<grid_of(n_leaves * 32, 256), 256, 0, s>>>(t->pphil, N, first_leaf, n_leaves,
                                                                 t->weak);
    for (int d = depth - 1; d >= 0; --d) {
        const int64_t first = ((int64_t)1 << d) - 1, cnt = (int64_t)1 << d;
        weak_internal_kernel<<<grid_of(cnt, 256), 256, 0, s>>>(first, cnt, t->pphil, t->weak);
    }
    TRY_LAUNCH();
#undef TRY_LAUNCH
    *out = t;
    return MBM_OK;
}

extern "C" mbm_status mbm_tree_build(mbm_ctx* ctx, const double* X_dev, int64_t N,
                                     const mbm_config* cfg, mbm_stream_t stream, mbm_tree** out) {
    if (!ctx || !out) return mbm_fail(MBM_EINVAL, "NULL ctx or out");
    if (!X_dev) return mbm_fail(MBM_EINVAL, "NULL X");
    *out = nullptr;
    mbm_config c;
    if (cfg) c = *cfg;
    else mbm_config_default(&c);
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    return build_tree(ctx, X_dev, N, c, reinterpret_cast<cudaStream_t>(stream), out);
}

extern "C" mbm_status mbm_tree_free(mbm_tree* t) {
    if (!t) return MBM_OK;
    cudaSetDevice(t->device);
    cudaDeviceSynchronize();
    if (t->mem) cudaFree(t->mem);
    if (t->ctx) mbm_budget_release(t->ctx, t->bytes);
    delete t;
    return MBM_OK;
}

extern "C" mbm_status mbm_tree_info(const mbm_tree* t, int64_t* n_nodes, int64_t* n_leaves,
                                    int32_t* depth) {
    if (!t) return mbm_fail(MBM_EINVAL, "NULL tree");
    if (n_nodes) *n_nodes = t->n_nodes;
    if (n_leaves) *n_leaves = t->n_leaves;
    if (depth) *depth = t->depth;
    return MBM_OK;
}

extern "C" mbm_status mbm_tree_export(const mbm_tree* t, int64_t* perm, double* lo, double* hi,
                                      double* cen, double* phil, mbm_stream_t stream) {
    if (!t) return mbm_fail(MBM_EINVAL, "NULL tree");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const auto d2d = cudaMemcpyDeviceToDevice;
    if (perm) MBM_CUDA_TRY(cudaMemcpyAsync(perm, t->perm, (size_t)t->N * 8, d2d, s));
    if (lo) MBM_CUDA_TRY(cudaMemcpyAsync(lo, t->nlo, (size_t)t->n_nodes * 24, d2d, s));
    if (hi) MBM_CUDA_TRY(cudaMemcpyAsync(hi, t->nhi, (size_t)t->n_nodes * 24, d2d, s));
    if (cen) MBM_CUDA_TRY(cudaMemcpyAsync(cen, t->ncen, (size_t)t->n_nodes * 24, d2d, s));
    if (phil) MBM_CUDA_TRY(cudaMemcpyAsync(phil, t->nphil, (size_t)t->n_nodes * 8, d2d, s));
    return MBM_OK;
}

// ---------------------------------------------------------------------------
// Tree potential.
// ---------------------------------------------------------------------------
namespace {

struct Timer {
    bool on;
    cudaEvent_t e[6];
    cudaStream_t s;
    Timer(bool on_, cudaStream_t s_) : on(on_), s(s_) {
        if (on)
            for (auto& x : e) cudaEventCreate(&x);
    }
    ~Timer() {
        if (on)
            for (auto& x : e) cudaEventDestroy(x);
    }
    void mark(int i) {
        if (on) cudaEventRecord(e[i], s);
    }
    double ms(int a, int b) {
        float v = 0.f;
        if (on) cudaEventElapsedTime(&v, e[a], e[b]);
        return v;
    }
};

}  // namespace

// One traversal of Algorithm 2 for the potential (F = false, out: N) or the
// forces (F = true, out: 3 N; the force criterion of classify_kernel<true>).
template <bool F>
static mbm_status tree_solve(mbm_ctx* ctx, const double* X, int64_t N, double eps, double alpha,
                             bool absolute, const mbm_config& cfg, mbm_tree* tree_in, double* phi,
                             mbm_stats* stats, cudaStream_t s) {
    if (cfg.m_limit < 2 || cfg.m_limit > 65535) return mbm_fail(MBM_EINVAL, "m_limit must be in [2, 65535]");
    if (!(cfg.zeta >= 0.0)) return mbm_fail(MBM_EINVAL, "zeta must be >= 0");
    if (!(cfg.tau >= 0.0)) return mbm_fail(MBM_EINVAL, "tau must be >= 0");
    Timer tm(stats != nullptr || ctx->timing, s);
    tm.mark(0);
    mbm_tree* tree = tree_in;
    bool own = false;
    if (tree) {
        if (tree->N != N || tree->device != ctx->device)
            return mbm_fail(MBM_EINVAL, "tree does not match X");
    } else {
        MBM_TRY(build_tree(ctx, X, N, cfg, s, &tree));
        own = true;
    }
    tm.mark(1);
    struct Owner {
        mbm_tree* t;
        bool own;
        ~Owner() {
            if (own) mbm_tree_free(t);
        }
    } owner{tree, own};

    const int64_t n_nodes = tree->n_nodes, n_leaves = tree->n_leaves;
    const bool counting = cfg.tuple_counts != nullptr;
    const TravPlan plan = trav_plan(N, tree->depth, cfg, F);
    const int64_t B = plan.B, cap_lvl = plan.cap_lvl, cap_mc = plan.cap_mc;
    const int64_t cap_base = plan.cap_base, cap_est = plan.cap_est;
    const int max_levels = plan.max_levels;
    size_t scan_tmp_bytes = plan.scan_tmp_bytes, sort_bytes = plan.sort_bytes;
    const int d = tree->depth;
    const int64_t first_leaf = n_nodes - n_leaves;
    const double z = z_two_sided(alpha);
    const std::vector<size_t>& parts = plan.parts;
    MBM_TRY(mbm_scratch_reserve(ctx, carve_size(parts)));
    Carve sc{static_cast<char*>(ctx->scratch)};
    double* pt_acc = sc.take<double>(N);
    double* node_acc = sc.take<double>(n_nodes);
    ull* pt_cnt = counting ? sc.take<ull>(N) : nullptr;
    ull* node_cnt = counting ? sc.take<ull>(n_nodes) : nullptr;
    int4* lvl = sc.take<int4>((size_t)max_levels * cap_lvl);
    int4* mcl = sc.take<int4>(cap_mc);
    int4* basel = sc.take<int4>(cap_base);
    int64_t* chunk_off = sc.take<int64_t>(cap_mc + 2);
    int* cand_fail = sc.take<int>(cap_mc);
    double* est = sc.take<double>(cap_est * (F ? 3 : 1));
    ull* ctr = sc.take<ull>(32);  // 0 n_next, 1 n_mc, 2 n_base, 3.. statistics
    void* scan_tmp = sc.take<char>(scan_tmp_bytes);
    double* rcp = sc.take<double>(cfg.m_limit + 1);
    ull* bkey = sc.take<ull>(cap_base);
    ull* bkey2 = sc.take<ull>(cap_base);
    int* bval = sc.take<int>(cap_base);
    int* bval2 = sc.take<int>(cap_base);
    int* bflag = sc.take<int>(cap_base + 1);
    int* bpos = sc.take<int>(cap_base + 1);
    int* bheads = sc.take<int>(cap_base + 1);
    int* bmeta = sc.take<int>(16);  // 0 n_pieces, 1 piece counter
    void* sort_tmp = sc.take<char>(sort_bytes);
    double* pt_acc3 = F ? sc.take<double>(3 * N) : nullptr;
    double* node_acc3 = F ? sc.take<double>(3 * n_nodes) : nullptr;
    double* pscale = F ? sc.take<double>(N) : nullptr;
    double* nscale = F ? sc.take<double>(n_nodes) : nullptr;
    ull* h = reinterpret_cast<ull*>(ctx->h_flags) + 8;  // pinned, after the status word
    {
        std::vector<double> r(cfg.m_limit + 1, 0.0);
        for (int m = 1; m <= cfg.m_limit; ++m) r[m] = 1.0 / (double)m;
        MBM_CUDA_TRY(cudaMemcpyAsync(rcp, r.data(), r.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        MBM_CUDA_TRY(cudaStreamSynchronize(s));
    }

    MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    MBM_CUDA_TRY(cudaMemsetAsync(pt_acc, 0, (size_t)N * 8, s));
    MBM_CUDA_TRY(cudaMemsetAsync(node_acc, 0, (size_t)n_nodes * 8, s));
    if (counting) {
        MBM_CUDA_TRY(cudaMemsetAsync(pt_cnt, 0, (size_t)N * 8, s));
        MBM_CUDA_TRY(cudaMemsetAsync(node_cnt, 0, (size_t)n_nodes * 8, s));
    }
    MBM_CUDA_TRY(cudaMemsetAsync(ctr, 0, 32 * sizeof(ull), s));
    if (F) {
        MBM_CUDA_TRY(cudaMemsetAsync(pt_acc3, 0, (size_t)N * 24, s));
        MBM_CUDA_TRY(cudaMemsetAsync(node_acc3, 0, (size_t)n_nodes * 24, s));
        // A^l: exact sum of |grad_x phi|_2 over each particle's seed node
        // (the tree's seed level, at most kForceSeedMax), min per node bottom-up.
        const int sd = std::max(0, tree->depth - std::min(tree->seed_levels, kForceSeedMax));
        const int64_t max_seed = (N + ((int64_t)1 << sd) - 1) >> sd;
        const int cpn = (int)((max_seed + 31) / 32);
        seed_scale_kernel<<<grid_of(((int64_t)1 << sd) * cpn * 32, 128), 128, 0, s>>>(
            tree->xh, tree->xl, N, sd, cpn, pscale);
        phil_leaf_kernel<<<grid_of(n_leaves * 32, 256), 256, 0, s>>>(pscale, N, n_nodes - n_leaves,
                                                                     n_leaves, nscale, pscale);
        for (int dd = tree->depth - 1; dd >= 0; --dd) {
            const int64_t first = ((int64_t)1 << dd) - 1, cnt = (int64_t)1 << dd;
            phil_internal_kernel<<<grid_of(cnt, 256), 256, 0, s>>>(first, cnt, nscale);
        }
        MBM_CUDA_TRY(cudaGetLastError());
    }
    const int4 root = make_int4(0, 0, 0, 0);
    MBM_CUDA_TRY(cudaMemcpyAsync(lvl, &root, sizeof(int4), cudaMemcpyHostToDevice, s));

    Trav p;
    p.N = N;
    p.n_nodes = n_nodes;
    p.n_leaves = n_leaves;
    p.nlo = tree->nlo;
    p.nhi = tree->nhi;
    p.ncen = tree->ncen;
    p.ndiam2 = tree->ndiam2;
    p.nphil = tree->nphil;
    p.pphil = tree->pphil;
    p.weak = tree->weak;
    p.xs = tree->xs;
    p.xh = tree->xh;
    p.xl = tree->xl;
    p.eps = absolute ? 0.0 : eps;
    p.tau = absolute ? eps : cfg.tau;
    p.troot = (double)(N - 1) * (double)(N - 2) * 0.5;
    p.inv_troot = 1.0 / p.troot;
    p.rcp = rcp;
    p.zeta = cfg.zeta;
    p.z = z;
    p.alpha = alpha;
    p.m_limit = cfg.m_limit;
    p.mc_rule = cfg.mc_rule;
    p.key0 = (uint32_t)cfg.seed;
    p.key1 = (uint32_t)(cfg.seed >> 32);
    p.node_acc = node_acc;
    p.pt_acc = pt_acc;
    p.node_cnt = node_cnt;
    p.pt_cnt = pt_cnt;
    p.n_next = ctr + 0;
    p.n_mc = ctr + 1;
    p.n_base = ctr + 2;
    p.stat = ctr + 3;
    p.cap_next = cap_lvl;
    p.cap_mc = cap_mc;
    p.cap_base = cap_base;
    p.mc = mcl;
    p.base = basel;
    p.flags = ctx->d_flags;
    p.nscale = nscale;
    p.pscale = pscale;
    p.node_acc3 = node_acc3;
    p.pt_acc3 = pt_acc3;

    const size_t bsm = sizeof(BaseSmem);
    MBM_CUDA_TRY(cudaFuncSetAttribute((const void*)base_group_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
    if (F)
        MBM_CUDA_TRY(cudaFuncSetAttribute((const void*)base_forces_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(ForceWarpSmem) * kForceWarps)));
    int base_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&base_per_sm, base_group_kernel,
                                                      kBaseWarps * 32, bsm) != cudaSuccess ||
        base_per_sm < 1)
        base_per_sm = 1;
    const unsigned base_grid = (unsigned)(base_per_sm * std::max(1, ctx->num_sms));
    // Base cases run whenever the list could not take another chunk (Phi^l is
    // fixed, so base cases may run in any order); their time is accumulated.
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> base_ev;
    int64_t total_base = 0;
    auto flush_base = [&](int64_t n) -> mbm_status {
        if (n <= 0) return MBM_OK;
        cudaEvent_t a = nullptr, b = nullptr;
        if (tm.on) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
        }
        base_key_kernel<<<grid_of(n, 256), 256, 0, s>>>(basel, n, N, first_leaf, d, bkey, bval,
                                                        ctr + 12);
        if (F) {  // exact forces of each leaf triple, a warp each
            base_forces_kernel<<<grid_of(n * 32, kForceWarps * 32), kForceWarps * 32,
                                 sizeof(ForceWarpSmem) * kForceWarps, s>>>(tree->xh, tree->xl, N,
                                                                          basel, n, pt_acc3);
            MBM_CUDA_TRY(cudaGetLastError());
            if (tm.on) {
                cudaEventRecord(b, s);
                base_ev.emplace_back(a, b);
            }
            if (counting)
                base_count_kernel<<<grid_of(n * 32, 256), 256, 0, s>>>(N, basel, n, pt_cnt);
            total_base += n;
            return MBM_OK;
        }
        MBM_CUDA_TRY(mbm_sort_pairs_u64(bkey, bkey2, bval, bval2, n, 0, std::max(1, 2 * d),
                                        sort_tmp, s));
        base_piece_flag_kernel<<<grid_of(n, 256), 256, 0, s>>>(bkey2, n, bflag);
        MBM_CUDA_TRY(mbm_exclusive_scan_i32(bflag, bpos, n, sort_tmp, s));
        base_piece_heads_kernel<<<grid_of(n, 256), 256, 0, s>>>(bflag, bpos, n, bheads, bmeta);
        MBM_CUDA_TRY(cudaMemsetAsync(bmeta + 1, 0, sizeof(int), s));
        base_group_kernel<<<base_grid, kBaseWarps * 32, bsm, s>>>(
            tree->xh, tree->xl, N, first_leaf, d, bkey2, bval2, bheads, bmeta,
            reinterpret_cast<unsigned*>(bmeta + 1), pt_acc, ctx->d_flags);
        MBM_CUDA_TRY(cudaGetLastError());
        if (tm.on) {
            cudaEventRecord(b, s);
            base_ev.emplace_back(a, b);
        }
        if (counting) base_count_kernel<<<grid_of(n * 32, 256), 256, 0, s>>>(N, basel, n, pt_cnt);
        total_base += n;
        return MBM_OK;
    };

    tm.mark(2);
    struct Level {
        int64_t count, done;
    };
    std::vector<Level> stack{{1, 0}};
    int64_t n_base = 0, levels_seen = 1, n_chunks = 0, n_flushes = 0, n_batches = 0;
    std::vector<int64_t> off;
    while (!stack.empty()) {
        const int li = (int)stack.size() - 1;
        if (stack[li].done >= stack[li].count) {
            stack.pop_back();
            continue;
        }
        if (li + 1 >= max_levels) return mbm_fail(MBM_EOVERFLOW, "traversal deeper than expected");
        const int64_t take = std::min<int64_t>(B, stack[li].count - stack[li].done);
        if (n_base + take > cap_base) {
            MBM_TRY(flush_base(n_base));
            n_flushes += n_base > 0;
            n_base = 0;
            MBM_CUDA_TRY(cudaMemsetAsync(ctr + 2, 0, sizeof(ull), s));
        }
        int4* cur = lvl + (size_t)li * cap_lvl + stack[li].done;
        p.next = lvl + (size_t)(li + 1) * cap_lvl;
        MBM_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(ull), s));  // n_next, n_mc
        classify_kernel<F><<<grid_of(take, 256), 256, 0, s>>>(cur, take, p);
        MBM_CUDA_TRY(cudaGetLastError());
        ++n_chunks;
        stack[li].done += take;
        MBM_CUDA_TRY(cudaMemcpyAsync(h, ctr, 3 * sizeof(ull), cudaMemcpyDeviceToHost, s));
        MBM_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t n_mc = (int64_t)h[1];
        if (n_mc > 0) {
            MBM_CUDA_TRY(cudaMemsetAsync(cand_fail, 0, (size_t)n_mc * sizeof(int), s));
            mc_probe_kernel<F><<<grid_of(n_mc * 32, 256), 256, 0, s>>>(mcl, n_mc, cand_fail, p);
            mc_sizes_kernel<<<grid_of(n_mc, 256), 256, 0, s>>>(mcl, n_mc, N, cand_fail, chunk_off);
            MBM_CUDA_TRY(cudaMemsetAsync(chunk_off + n_mc, 0, sizeof(int64_t), s));
            MBM_CUDA_TRY(mbm_exclusive_scan_i64(chunk_off, chunk_off, n_mc + 1, scan_tmp, s));
            off.resize(n_mc + 1);
            MBM_CUDA_TRY(cudaMemcpyAsync(off.data(), chunk_off, (n_mc + 1) * sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, s));
            MBM_CUDA_TRY(cudaStreamSynchronize(s));
            int64_t c0 = 0;
            while (c0 < n_mc) {  // batches whose estimates fit the buffer
                int64_t c1 = c0 + 1;
                while (c1 < n_mc && (off[c1 + 1] - off[c0]) * 32 <= cap_est) ++c1;
                const int64_t chunks = off[c1] - off[c0];
                mc_kernel<F><<<grid_of(chunks * 32, 128), 128, 0, s>>>(mcl + c0, 0, c1 - c0,
                                                                    chunk_off + c0, cand_fail + c0,
                                                                    est, p);
                mc_commit_kernel<F><<<(unsigned)(c1 - c0), 256, 0, s>>>(
                    mcl + c0, 0, c1 - c0, chunk_off + c0, cand_fail + c0, est, p);
                MBM_CUDA_TRY(cudaGetLastError());
                ++n_batches;
                c0 = c1;
            }
            MBM_CUDA_TRY(cudaMemcpyAsync(h, ctr, 3 * sizeof(ull), cudaMemcpyDeviceToHost, s));
            MBM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        n_base = (int64_t)h[2];
        if (h[0] > 0) {
            stack.push_back({(int64_t)h[0], 0});
            levels_seen = std::max<int64_t>(levels_seen, (int64_t)stack.size());
        }
    }
    MBM_TRY(flush_base(n_base));
    n_flushes += n_base > 0;
    tm.mark(3);
    tm.mark(4);
    if (F)
        finalize3_kernel<<<grid_of(N, 256), 256, 0, s>>>(N, tree->depth, n_nodes, n_leaves,
                                                         tree->perm, pt_acc3, node_acc3, pt_cnt,
                                                         node_cnt, phi, cfg.tuple_counts);
    else
        finalize_kernel<<<grid_of(N, 256), 256, 0, s>>>(N, tree->depth, n_nodes, n_leaves,
                                                        tree->perm, pt_acc, node_acc, pt_cnt,
                                                        node_cnt, phi, cfg.tuple_counts);
    MBM_CUDA_TRY(cudaGetLastError());
    tm.mark(5);
    double base_ms = 0.0;
    if (tm.on) {
        MBM_CUDA_TRY(cudaStreamSynchronize(s));
        for (auto& ev : base_ev) {
            float v = 0.f;
            cudaEventElapsedTime(&v, ev.first, ev.second);
            base_ms += v;
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        if (ctx->timing) mbm_time_set_ms(ctx, base_ms);
    }
    MBM_CUDA_TRY(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (stats) {
        MBM_CUDA_TRY(cudaMemcpyAsync(h, ctr, 13 * sizeof(ull), cudaMemcpyDeviceToHost, s));
        MBM_CUDA_TRY(cudaStreamSynchronize(s));
        stats->node_triples_visited = (int64_t)h[3];
        stats->det_prunes = (int64_t)h[4];
        stats->mc_prunes = (int64_t)h[5];
        stats->mc_attempts = (int64_t)h[6];
        stats->base_cases = total_base;
        stats->mc_samples = (int64_t)h[8];
        stats->levels = levels_seen;
        stats->ms_build = tm.ms(0, 1);
        stats->ms_traverse = tm.ms(2, 3) - base_ms;
        stats->ms_base = base_ms;
        stats->ms_finalize = tm.ms(4, 5);
        stats->base_triples = (int64_t)h[12];
        stats->chunks = n_chunks;
        stats->base_flushes = n_flushes;
        stats->mc_batches = n_batches;
    }
    if (cfg.validate) return mbm_check_flags(ctx, s);
    return MBM_OK;
}

mbm_status mbm_tree_potential(mbm_ctx* ctx, const double* X, int64_t N, double eps, double alpha,
                              bool absolute, const mbm_config& cfg, mbm_tree* tree, double* phi,
                              mbm_stats* stats, cudaStream_t s) {
    return tree_solve<false>(ctx, X, N, eps, alpha, absolute, cfg, tree, phi, stats, s);
}

mbm_status mbm_tree_forces(mbm_ctx* ctx, const double* X, int64_t N, double eps, double alpha,
                           bool absolute, const mbm_config& cfg, mbm_tree* tree, double* F3,
                           mbm_stats* stats, cudaStream_t s) {
    return tree_solve<true>(ctx, X, N, eps, alpha, absolute, cfg, tree, F3, stats, s);
}

size_t mbm_tree_solve_bytes(int64_t N, const mbm_config& cfg, bool forces) {
    if (N < 3 || cfg.leaf_size < 2) return 0;
    const int depth = tree_depth(N, cfg.leaf_size);
    const int64_t n_nodes = ((int64_t)2 << depth) - 1;
    const TravPlan plan = trav_plan(N, depth, cfg, forces);
    return carve_size(tree_parts(N, n_nodes)) + carve_size(plan.parts);
}
