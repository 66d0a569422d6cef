// Exhaustive Axilrod-Teller sums on the GPU (every unordered triple once).
//
// Phi(x_i) = sum_{j<k; j,k != i} phi(x_i, x_j, x_k)   (Eq. 1, n = 3; Sec. 1)
//
// Each unordered triple a < b < c is evaluated once and credited to all
// three members, which is the same sum (each triple appears in exactly the
// three slices Phi(x_a), Phi(x_b), Phi(x_c)).
//
// FP32 bulk evaluates each triple in the direction-cosine form (see
// tile_fp32.cuh: unit edge vectors and r^-3 per pair, 14 FP32 operations and
// 23 FLOPs per triple). FP64 evaluates the law-of-cosines form on squared
// side lengths c = r_ij^2, b = r_ik^2, a = r_jk^2:
//   cos t_i cos t_j cos t_k = P / (8abc),  P = (b+c-a)(a+c-b)(a+b-c),
//   phi = (abc + 0.375 P) A B C,  A = a^(-5/2), B = b^(-5/2), C = c^(-5/2).
//
// Work decomposition (both precisions): particles are cut into tiles of 32.
// A CTA owns one tile pair (J, K), J <= K, and its warps sweep every tile
// I <= J; a lane owns one particle i of I. Pair quantities are hoisted to
// the loop level where they are constant: (j,k) in a shared-memory table
// built once per CTA item, (i,k) once per I tile, (i,j) once per j.
// Diagonal tiles (I = J, J = K) are handled by zeroing the pair factor of
// out-of-order pairs, so masked triples contribute exactly 0. Items come
// from a global counter, largest (most I tiles) first.
#include <algorithm>

#include "bulk_copy.cuh"
#include "device_math.cuh"
#include "mbm_internal.h"
#include "tile_fp32.cuh"

namespace {

constexpr int kTile = 32;
constexpr int kWarps32 = 8;   // FP32 kernel: 8 warps per CTA
constexpr int kWarps64 = 4;   // FP64 kernel: 4 warps per CTA

// ---------------------------------------------------------------------------
// Step a1: input pack.
// ---------------------------------------------------------------------------
__global__ void pack_hilo_kernel(const double* __restrict__ X, int64_t N, float4* __restrict__ xh,
                                 float4* __restrict__ xl, int* __restrict__ flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(flags, MBM_FLAG_NONFINITE);
        const float hx = (float)x, hy = (float)y, hz = (float)z;
        xh[i] = make_float4(hx, hy, hz, 0.f);
        xl[i] = make_float4((float)(x - (double)hx), (float)(y - (double)hy),
                            (float)(z - (double)hz), 0.f);
    }
}

__global__ void pack_f64_kernel(const double* __restrict__ X, int64_t N, double4_32a* __restrict__ x4,
                                int* __restrict__ flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(flags, MBM_FLAG_NONFINITE);
        x4[i] = make_double4_32a(x, y, z, 0.0);
    }
}

// ---------------------------------------------------------------------------
// Step a3, FP32 bulk: FP32 triple arithmetic (direction-cosine form, see
// tile_fp32.cuh), per-tile FP32 partial sums, FP64 accumulation across tiles.
// ---------------------------------------------------------------------------
struct Fp32Smem {
    mbm_tile::TabPair tab[kTile][kTile / 2];
    float4 sJh[kTile], sJl[kTile], sKh[kTile], sKl[kTile];
    float redJ[kWarps32][kTile][kTile + 1];
    float redK[kWarps32][kTile][kTile + 1];
    double wsum[2][kWarps32][kTile];
    long long item;
};

__global__ void __launch_bounds__(kWarps32 * 32, 2)
exh_fp32_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int N, int NT,
                long long n_items, unsigned long long* __restrict__ counter,
                double* __restrict__ phi, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Fp32Smem& sm = *reinterpret_cast<Fp32Smem*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    for (;;) {
        if (threadIdx.x == 0) sm.item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long t = sm.item;
        if (t >= n_items) break;
        int J, K;
        decode_pair_item(t, NT, J, K);
        const int nJ = min(kTile, N - J * kTile), nK = min(kTile, N - K * kTile);
        if (threadIdx.x < kTile) {
            const int j = J * kTile + threadIdx.x;
            sm.sJh[threadIdx.x] = j < N ? xh[j] : zero4;
            sm.sJl[threadIdx.x] = j < N ? xl[j] : zero4;
        } else if (threadIdx.x < 2 * kTile) {
            const int kk = threadIdx.x - kTile, k = K * kTile + kk;
            sm.sKh[kk] = k < N ? xh[k] : zero4;
            sm.sKl[kk] = k < N ? xl[k] : zero4;
        }
        __syncthreads();
        // (j,k) table; every unordered pair of the set is a valid entry of
        // exactly one table, which is where coincident points are caught.
        bool bad = false;
        for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
            const int jj = e >> 5, kk = e & 31;
            const bool v = jj < nJ && kk < nK && (J != K || jj < kk);
            bad |= mbm_tile::build_table_entry(sm.tab, jj, kk, sm.sJh[jj], sm.sJl[jj], sm.sKh[kk],
                                               sm.sKl[kk], v);
        }
        if (bad) atomicOr(flags, MBM_FLAG_COINCIDENT);
        __syncthreads();

        double run_j = 0.0, run_k = 0.0;
        for (int I = warp; I <= J; I += kWarps32) {
            const int i = I * kTile + lane;
            const bool iv = i < N;
            const float4 ih = iv ? xh[i] : zero4;
            const float4 il = iv ? xl[i] : zero4;
            const float acc_i = mbm_tile::tile_triples(sm.tab, sm.sJh, sm.sJl, sm.sKh, sm.sKl, ih,
                                                       il, iv, lane, nJ, nK, I == J, I == K,
                                                       sm.redJ[warp], sm.redK[warp]);
            run_j += (double)mbm_tile::row_sum(sm.redJ[warp], lane);
            run_k += (double)mbm_tile::row_sum(sm.redK[warp], lane);
            __syncwarp();
            if (iv) atomicAdd(&phi[i], (double)acc_i);
        }
        sm.wsum[0][warp][lane] = run_j;
        sm.wsum[1][warp][lane] = run_k;
        __syncthreads();
        if (warp < 2) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps32; ++w) tot += sm.wsum[warp][w][lane];
            const int idx = (warp == 0 ? J : K) * kTile + lane;
            if (idx < N) atomicAdd(&phi[idx], tot);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Step a3 with a pair table. Every pair term the FP32 sweep uses -- the unit
// vector e_ab = (x_b - x_a)/r_ab and rho_ab = r_ab^-3 of each pair a < b -- is
// computed once per solve in FP64 from the FP64 input and rounded once to
// FP32, so each is correctly rounded (the in-kernel FP32 set-up carries a few
// ulp), and the sweep no longer spends FP32 pipe time or MUFU work on pair
// set-up. Layout: one 16 KB mbm_tile::PairBlock per tile pair (A, B),
// A <= B, blocks of row A contiguous; a block holds the pair terms from
// particle A*32 + r to B*32 + c in two planes indexed [c / 2][r]. Entries of
// pairs that are absent (beyond N) or not ordered (A == B, r >= c) are zero.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ long long pt_block(int A, int B, int NT) {
    return (long long)A * NT - (long long)A * (A - 1) / 2 + (B - A);
}

__global__ void __launch_bounds__(256)
pair_table_kernel(const double* __restrict__ X, int N, int NT,
                  mbm_tile::PairBlock* __restrict__ pt, int* __restrict__ flags) {
    const int A = blockIdx.y;
    const long long per_row = (long long)(NT - A) * (kTile * kTile / 2);
    mbm_tile::PairBlock* rowbase = pt + pt_block(A, A, NT);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < per_row;
         q += (long long)gridDim.x * blockDim.x) {
        const int B = A + (int)(q >> 9);
        const int p = (int)(q >> 5) & 15, r = (int)q & 31;
        const int a = A * kTile + r;
        float v[2][4];
        int bad = 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int col = 2 * p + c, b = B * kTile + col;
            v[c][0] = v[c][1] = v[c][2] = v[c][3] = 0.f;
            if (a < N && b < N && (A < B || r < col)) {
                const double dx = X[3 * (int64_t)b] - X[3 * (int64_t)a];
                const double dy = X[3 * (int64_t)b + 1] - X[3 * (int64_t)a + 1];
                const double dz = X[3 * (int64_t)b + 2] - X[3 * (int64_t)a + 2];
                const double s2 = dx * dx + dy * dy + dz * dz;
                if (!isfinite(s2)) {
                    bad |= MBM_FLAG_NONFINITE;
                } else if (!(s2 > 0.0)) {
                    bad |= MBM_FLAG_COINCIDENT;
                } else {
                    const double y = 1.0 / sqrt(s2);
                    v[c][0] = (float)(dx * y);
                    v[c][1] = (float)(dy * y);
                    v[c][2] = (float)(dz * y);
                    v[c][3] = (float)(y * y * y);
                }
            }
        }
        if (bad) atomicOr(flags, bad);
        mbm_tile::PairBlock& blk = rowbase[B - A];
        blk.xy[p][r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
        blk.zr[p][r] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
    }
}

struct PtSmem {
    mbm_tile::PairBlock tab;            // (j, k) table of the current item
    mbm_tile::IjRing ring[kWarps32];    // per-warp staging of (i, j) pair terms
    float redJ[kWarps32][kTile][kTile + 1];
    float redK[kWarps32][kTile][kTile + 1];
    double wsum[2][kWarps32][kTile];
    unsigned long long bar;
    long long item;
};

// An item's (j, k) table is block (J, K) of the pair table: one 16 KB bulk
// copy, issued by thread 0 as soon as the previous item's warps are done
// with the buffer.
__device__ __forceinline__ void issue_item_table(PtSmem& sm, long long t, int NT,
                                                 const mbm_tile::PairBlock* pt) {
    int J, K;
    decode_pair_item(t, NT, J, K);
    const unsigned bytes = (unsigned)sizeof(mbm_tile::PairBlock);
    mbar_arrive_expect_tx(&sm.bar, bytes);
    bulk_copy_g2s(&sm.tab, pt + pt_block(J, K, NT), bytes, &sm.bar);
}

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: a copy that never lands

__global__ void __launch_bounds__(kWarps32 * 32, 2)
exh_fp32_pt_kernel(const mbm_tile::PairBlock* __restrict__ pt, int N, int NT, long long n_items,
                   unsigned long long* __restrict__ counter, double* __restrict__ phi,
                   int* __restrict__ flags) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PtSmem& sm = *reinterpret_cast<PtSmem*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    bool pending = false;  // thread 0: a table copy issued and not yet waited for
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        mbar_fence_init();
        const long long t = (long long)atomicAdd(counter, 1ULL);
        sm.item = t;
        if (t < n_items) {
            issue_item_table(sm, t, NT, pt);
            pending = true;
        }
    }
    __syncthreads();
    unsigned parity = 0u;
    for (;;) {
        const long long t = sm.item;
        if (t >= n_items) break;
        const bool ok = mbar_wait_bounded(&sm.bar, parity, kWaitCycles);
        if (ok) {
            parity ^= 1u;
            pending = false;
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(flags, MBM_FLAG_TIMEOUT);
            break;
        }
        int J, K;
        decode_pair_item(t, NT, J, K);
        double run_j = 0.0, run_k = 0.0;
        for (int I = warp; I <= J; I += kWarps32) {
            const int i = I * kTile + lane;
            // the warp's next (I, K) block is streamed from memory: ask L2 for it now
            if (I + kWarps32 <= J) {
                const char* nb = reinterpret_cast<const char*>(pt + pt_block(I + kWarps32, K, NT));
                for (int o = lane * 128; o < (int)sizeof(mbm_tile::PairBlock); o += 32 * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + o));
            }
            const float acc_i = mbm_tile::tile_triples_table(
                sm.tab, pt + pt_block(I, K, NT), pt + pt_block(I, J, NT), lane, sm.ring[warp],
                sm.redJ[warp], sm.redK[warp]);
            run_j += (double)mbm_tile::row_sum(sm.redJ[warp], lane);
            run_k += (double)mbm_tile::row_sum(sm.redK[warp], lane);
            __syncwarp();
            if (i < N) atomicAdd(&phi[i], (double)acc_i);
        }
        sm.wsum[0][warp][lane] = run_j;
        sm.wsum[1][warp][lane] = run_k;
        __syncthreads();  // every warp is done with the table buffer
        if (threadIdx.x == 0) {
            const long long tn = (long long)atomicAdd(counter, 1ULL);
            sm.item = tn;
            if (tn < n_items) {
                issue_item_table(sm, tn, NT, pt);
                pending = true;
            }
        }
        if (warp < 2) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps32; ++w) tot += sm.wsum[warp][w][lane];
            const int idx = (warp == 0 ? J : K) * kTile + lane;
            if (idx < N) atomicAdd(&phi[idx], tot);
        }
        __syncthreads();
    }
    // A copy is still in flight here only after a timed-out wait: give it a
    // bounded chance to land before the CTA's shared memory is released.
    if (threadIdx.x == 0 && pending) mbar_wait_bounded(&sm.bar, parity, kWaitCycles);
}

// ---------------------------------------------------------------------------
// Step a2 in FP64: the same decomposition with FP64 everywhere. Per-lane
// (i,k) quantities live in per-warp shared memory (FP64 registers would not
// fit), the (j,k) table in shared memory, accumulators in registers.
// ---------------------------------------------------------------------------
struct Fp64Smem {
    double2 tab[kTile][kTile];             // (a, A) for (j, k)
    double2 bw[kWarps64][kTile][kTile];    // (b, B) for (k, lane)
    double red[kWarps64][kTile][kTile + 1];
    double wsum[2][kWarps64][kTile];
    double4_32a sJ[kTile], sK[kTile];
    long long item;
};

__global__ void __launch_bounds__(kWarps64 * 32, 1)
exh_fp64_kernel(const double4_32a* __restrict__ x4, int N, int NT, long long n_items,
                unsigned long long* __restrict__ counter, double* __restrict__ phi,
                int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Fp64Smem& sm = *reinterpret_cast<Fp64Smem*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const double4_32a zero4 = make_double4_32a(0.0, 0.0, 0.0, 0.0);

    for (;;) {
        if (threadIdx.x == 0) sm.item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long t = sm.item;
        if (t >= n_items) break;
        int J, K;
        decode_pair_item(t, NT, J, K);
        if (threadIdx.x < kTile) {
            const int j = J * kTile + threadIdx.x;
            sm.sJ[threadIdx.x] = j < N ? x4[j] : zero4;
        } else if (threadIdx.x < 2 * kTile) {
            const int kk = threadIdx.x - kTile, k = K * kTile + kk;
            sm.sK[kk] = k < N ? x4[k] : zero4;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
            const int jj = e >> 5, kk = e & 31;
            const int j = J * kTile + jj, k = K * kTile + kk;
            double a = 1.0, A = 0.0;
            if (j < N && k < N && (J != K || jj < kk)) {
                const double dx = sm.sJ[jj].x - sm.sK[kk].x;
                const double dy = sm.sJ[jj].y - sm.sK[kk].y;
                const double dz = sm.sJ[jj].z - sm.sK[kk].z;
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 > 0.0) {
                    a = d2;
                    A = inv_pow52d(d2);
                } else {
                    atomicOr(flags, MBM_FLAG_COINCIDENT);
                }
            }
            sm.tab[jj][kk] = make_double2(a, A);
        }
        __syncthreads();

        double run_j = 0.0, run_k = 0.0;
        for (int I = warp; I <= J; I += kWarps64) {
            const int i = I * kTile + lane;
            const bool iv = i < N;
            const double4_32a xi = iv ? x4[i] : zero4;
#pragma unroll 4
            for (int kk = 0; kk < kTile; ++kk) {
                const bool v = iv && (K * kTile + kk < N) && (I != K || lane < kk);
                const double dx = xi.x - sm.sK[kk].x;
                const double dy = xi.y - sm.sK[kk].y;
                const double dz = xi.z - sm.sK[kk].z;
                const double b = dx * dx + dy * dy + dz * dz;
                sm.bw[warp][kk][lane] = make_double2(v ? b : 1.0, v ? inv_pow52d(b) : 0.0);
            }
            __syncwarp();
            double acc[kTile];
#pragma unroll
            for (int kk = 0; kk < kTile; ++kk) acc[kk] = 0.0;
            double acc_i = 0.0;
#pragma unroll 1
            for (int jj = 0; jj < kTile; ++jj) {
                const int j = J * kTile + jj;
                const bool v = iv && (j < N) && (I != J || lane < jj);
                const double dx = xi.x - sm.sJ[jj].x;
                const double dy = xi.y - sm.sJ[jj].y;
                const double dz = xi.z - sm.sJ[jj].z;
                double c = dx * dx + dy * dy + dz * dz;
                const double C = v ? inv_pow52d(c) : 0.0;
                c = v ? c : 1.0;
                const double ncc = -c * c, c375 = 0.375 * c;
                double s = 0.0;
#pragma unroll
                for (int kk = 0; kk < kTile; ++kk) {
                    const double2 aA = sm.tab[jj][kk];
                    const double2 bB = sm.bw[warp][kk][lane];
                    const double d = aA.x - bB.x;
                    const double e = aA.x + bB.x;
                    const double uv = fma(d, d, ncc);
                    const double w = fma(e, -0.375, c375);
                    const double P = uv * w;
                    const double n = fma(aA.x, bB.x * c, P);
                    const double ABC = aA.y * (bB.y * C);
                    s = fma(n, ABC, s);
                    acc[kk] = fma(n, ABC, acc[kk]);
                }
                acc_i += s;
                sm.red[warp][jj][lane] = s;
            }
            __syncwarp();
            double sj = 0.0;
            for (int m = 0; m < kTile; ++m) sj += sm.red[warp][lane][m];
            run_j += sj;
            __syncwarp();
#pragma unroll
            for (int kk = 0; kk < kTile; ++kk) sm.red[warp][kk][lane] = acc[kk];
            __syncwarp();
            double sk = 0.0;
            for (int m = 0; m < kTile; ++m) sk += sm.red[warp][lane][m];
            run_k += sk;
            __syncwarp();
            if (iv) atomicAdd(&phi[i], acc_i);
        }
        sm.wsum[0][warp][lane] = run_j;
        sm.wsum[1][warp][lane] = run_k;
        __syncthreads();
        if (warp < 2) {
            double tot = 0.0;
            for (int w = 0; w < kWarps64; ++w) tot += sm.wsum[warp][w][lane];
            const int idx = (warp == 0 ? J : K) * kTile + lane;
            if (idx < N) atomicAdd(&phi[idx], tot);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Exact Phi (FP32 bulk) for a sample of particles: every pair j < k of the
// set against each sampled particle i (pairs containing i drop out because
// their distance is exactly zero). A warp owns one tile pair (J, K) with its
// own table; lanes are the sampled particles.
// ---------------------------------------------------------------------------
struct SampleWarpSmem {
    mbm_tile::TabPair tab[kTile][kTile / 2];
    float4 sJh[kTile], sJl[kTile], sKh[kTile], sKl[kTile];
    float redJ[kTile][kTile + 1];
    float redK[kTile][kTile + 1];
};
constexpr int kSampleWarps = 4;

__global__ void __launch_bounds__(kSampleWarps * 32, 1)
sampled_fp32_kernel(const float4* __restrict__ xh, const float4* __restrict__ xl, int N, int NT,
                    const int64_t* __restrict__ idx, int n_idx, double* __restrict__ out,
                    long long n_items, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SampleWarpSmem& w = reinterpret_cast<SampleWarpSmem*>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < n_items;
         t += warps) {
        int J, K;
        decode_pair_item(t, NT, J, K);
        const int nJ = min(kTile, N - J * kTile), nK = min(kTile, N - K * kTile);
        w.sJh[lane] = lane < nJ ? xh[J * kTile + lane] : z4;
        w.sJl[lane] = lane < nJ ? xl[J * kTile + lane] : z4;
        w.sKh[lane] = lane < nK ? xh[K * kTile + lane] : z4;
        w.sKl[lane] = lane < nK ? xl[K * kTile + lane] : z4;
        __syncwarp();
        for (int e = lane; e < kTile * kTile; e += 32) {
            const int jj = e >> 5, kk = e & 31;
            mbm_tile::build_table_entry(w.tab, jj, kk, w.sJh[jj], w.sJl[jj], w.sKh[kk], w.sKl[kk],
                                        jj < nJ && kk < nK && (J != K || jj < kk));
        }
        __syncwarp();
        for (int q0 = 0; q0 < n_idx; q0 += kTile) {
            const int q = q0 + lane;
            const int64_t i0 = q < n_idx ? idx[q] : 0;
            const bool bad = q < n_idx && (i0 < 0 || i0 >= N);  // skipped and reported
            if (bad && t == 0) atomicOr(flags, MBM_FLAG_INDEX);
            const bool iv = q < n_idx && !bad;
            const int64_t i = iv ? i0 : 0;
            const float4 ih = iv ? xh[i] : z4, il = iv ? xl[i] : z4;
            const float acc = mbm_tile::tile_triples(w.tab, w.sJh, w.sJl, w.sKh, w.sKl, ih, il, iv,
                                                     lane, nJ, nK, false, false, w.redJ, w.redK);
            if (iv) atomicAdd(&out[q], (double)acc);
        }
        __syncwarp();
    }
}

int grid_for(const void* kernel, int threads, size_t smem, int num_sms, long long items) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * (num_sms > 0 ? num_sms : 1);
    if (g > items) g = items;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_pack_hilo(const double* X, int64_t N, float4* xhi, float4* xlo, int* flags,
                             cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (N + threads - 1) / threads;
    pack_hilo_kernel<<<(unsigned)(blocks < 65535 ? blocks : 65535), threads, 0, s>>>(X, N, xhi, xlo,
                                                                                    flags);
    return cudaGetLastError();
}

cudaError_t launch_pack_f64(const double* X, int64_t N, double4_32a* x4, int* flags, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (N + threads - 1) / threads;
    pack_f64_kernel<<<(unsigned)(blocks < 65535 ? blocks : 65535), threads, 0, s>>>(X, N, x4, flags);
    return cudaGetLastError();
}

cudaError_t launch_exh_fp32(const float4* xhi, const float4* xlo, int64_t N, double* phi,
                            unsigned long long* counter, int* flags, int num_sms,
                            cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long items = (long long)NT * (NT + 1) / 2;
    const int threads = kWarps32 * 32;
    const size_t smem = sizeof(Fp32Smem);
    cudaError_t e = cudaFuncSetAttribute((const void*)exh_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void*)exh_fp32_kernel, threads, smem, num_sms, items);
    exh_fp32_kernel<<<grid, threads, smem, s>>>(xhi, xlo, (int)N, NT, items, counter, phi, flags);
    return cudaGetLastError();
}

size_t pair_table_bytes(int64_t N) {
    const long long NT = (N + kTile - 1) / kTile;
    return (size_t)(NT * (NT + 1) / 2) * sizeof(mbm_tile::PairBlock);
}

cudaError_t launch_pair_table(const double* X, int64_t N, void* table, int* flags, cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long per_row0 = (long long)NT * (kTile * kTile / 2);
    const int gx = (int)std::min<long long>((per_row0 + 255) / 256, 1024);
    pair_table_kernel<<<dim3(gx, NT), 256, 0, s>>>(X, (int)N, NT,
                                                   static_cast<mbm_tile::PairBlock*>(table), flags);
    return cudaGetLastError();
}

cudaError_t launch_exh_fp32_table(const void* table, int64_t N, double* phi,
                                  unsigned long long* counter, int* flags, int num_sms,
                                  cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long items = (long long)NT * (NT + 1) / 2;
    const int threads = kWarps32 * 32;
    const size_t smem = sizeof(PtSmem);
    cudaError_t e = cudaFuncSetAttribute((const void*)exh_fp32_pt_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void*)exh_fp32_pt_kernel, threads, smem, num_sms, items);
    exh_fp32_pt_kernel<<<grid, threads, smem, s>>>(
        static_cast<const mbm_tile::PairBlock*>(table), (int)N, NT, items, counter, phi, flags);
    return cudaGetLastError();
}

cudaError_t launch_exh_fp64(const double4_32a* x4, int64_t N, double* phi, unsigned long long* counter,
                            int* flags, int num_sms, cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long items = (long long)NT * (NT + 1) / 2;
    const int threads = kWarps64 * 32;
    const size_t smem = sizeof(Fp64Smem);
    cudaError_t e = cudaFuncSetAttribute((const void*)exh_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void*)exh_fp64_kernel, threads, smem, num_sms, items);
    exh_fp64_kernel<<<grid, threads, smem, s>>>(x4, (int)N, NT, items, counter, phi, flags);
    return cudaGetLastError();
}

cudaError_t launch_sampled_fp32(const float4* xhi, const float4* xlo, int64_t N,
                                const int64_t* idx, int64_t n_idx, double* out, int* flags,
                                int num_sms, cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long items = (long long)NT * (NT + 1) / 2;
    const int threads = kSampleWarps * 32;
    const size_t smem = sizeof(SampleWarpSmem) * kSampleWarps;
    cudaError_t e = cudaFuncSetAttribute((const void*)sampled_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void*)sampled_fp32_kernel, threads, smem, num_sms,
                              (items + kSampleWarps - 1) / kSampleWarps);
    sampled_fp32_kernel<<<grid, threads, smem, s>>>(xhi, xlo, (int)N, NT, idx, (int)n_idx, out,
                                                    items, flags);
    return cudaGetLastError();
}
