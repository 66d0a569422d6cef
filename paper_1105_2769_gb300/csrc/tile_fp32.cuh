// FP32-bulk evaluation of all point triples of a tile triple (I, J, K).
//
// phi(x_i, x_j, x_k) = (1 + 3 cos t_i cos t_j cos t_k) / (r_ij r_ik r_jk)^3   (Sec. 1)
//
// With unit edge vectors e_ij = (x_j - x_i)/r_ij, e_ik, e_jk:
//   cos t_i = e_ij . e_ik,  cos t_j = -e_ij . e_jk,  cos t_k = e_ik . e_jk,
// so phi = (1 - 3 p1 p2 p3) rho_ij rho_ik rho_jk, p1 = e_ij.e_ik, p2 = e_ij.e_jk,
// p3 = e_ik.e_jk, rho = r^-3. No squared lengths are subtracted, so a triangle
// with one short side keeps full FP32 relative accuracy in every term.
//
// Loop structure: a lane owns particle i of tile I. (j,k) quantities come from
// a shared-memory table built once per (J, K); (i,k) quantities are held in
// registers for one half (16 columns) of K; (i,j) quantities are formed per j.
// With p1' = (-3 e_ij).e_ik (the -3 folded into a per-row copy of e_ij),
// q = n rho_jk = rho_jk + p1' p2 p3 rho_jk, and
//   row sum    sum_k phi = rho_ij sum_k q rho_ik,
//   column sum sum_j phi = rho_ik sum_j q rho_ij,
// the loop per pair of triples (packed f32x2) is 9 for the dot products, 2 for
// p1' p2 p3, 1 for q, 1 for the row sum, 1 for the column sum: 14 operations
// per triple, 9 of them FMA -> 23 FLOPs per triple (FMA = 2).
#pragma once

#include "device_math.cuh"

namespace mbm_tile {

constexpr int kTile = 32;
constexpr int kHalf = 16;   // K columns held in registers at once
constexpr int kPairs = 8;   // f32x2 column pairs per half

// Table entry for two adjacent columns k, k+1 of row j.
struct __align__(16) TabPair {
    float4 xy;  // (ex_k, ex_k+1, ey_k, ey_k+1)
    float4 zr;  // (ez_k, ez_k+1, rho_k, rho_k+1)
};

struct PairF {
    float ex, ey, ez, rho;
};

// Unit vector from p to q and rho = |q - p|^-3, from hi/lo coordinates.
// rsqrt is refined by one Newton step (y <- y + y (1 - s y^2)/2, residual by
// FMA); rho = y^3 is refined by one Newton step for rho^-2 = s^3
// (rho <- rho + rho (1 - s^3 rho^2)/2). Returns s in *s_out (0 = coincident).
__device__ __forceinline__ PairF pair_unit(float4 ph, float4 pl, float4 qh, float4 ql,
                                           float* s_out) {
    const float dx = (qh.x - ph.x) + (ql.x - pl.x);
    const float dy = (qh.y - ph.y) + (ql.y - pl.y);
    const float dz = (qh.z - ph.z) + (ql.z - pl.z);
    const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float y = rsqrtf(s);
    const float h = s * y;
    y = fmaf(0.5f * y, fmaf(-h, y, 1.0f), y);
    float rho = y * y * y;
    const float q = s * rho;
    rho = fmaf(0.5f * rho, fmaf(-q * q, s, 1.0f), rho);
    *s_out = s;
    PairF r;
    r.ex = dx * y;
    r.ey = dy * y;
    r.ez = dz * y;
    r.rho = rho;
    return r;
}

// Build row j's entries of the (j,k) table (all k of the K tile). valid(j,k)
// masked entries get rho = 0 so every triple through them contributes 0.
// Returns true if some valid pair is coincident.
__device__ __forceinline__ bool build_table_entry(TabPair (*tab)[kTile / 2], int jj, int kk,
                                                  float4 jh, float4 jl, float4 kh, float4 kl,
                                                  bool valid) {
    float s = 1.f;
    PairF p = pair_unit(jh, jl, kh, kl, &s);
    bool bad = false;
    if (!valid) {
        p.ex = p.ey = p.ez = 0.f;
        p.rho = 0.f;
    } else if (!(s > 0.f)) {
        bad = true;
        p.ex = p.ey = p.ez = 0.f;
        p.rho = 0.f;
    }
    float* xy = reinterpret_cast<float*>(&tab[jj][kk >> 1].xy);
    float* zr = reinterpret_cast<float*>(&tab[jj][kk >> 1].zr);
    const int o = kk & 1;
    xy[o] = p.ex;
    xy[2 + o] = p.ey;
    zr[o] = p.ez;
    zr[2 + o] = p.rho;
    return bad;
}

// One row j against the 8 column pairs (16 columns k) held in registers:
// the 14-operation loop of the header comment. Column pair p of the row is
// xy[p * stride], zr[p * stride] (float4: (ex_k, ex_k+1, ey_k, ey_k+1) and
// (ez_k, ez_k+1, rho_k, rho_k+1)). Adds q rho_ij to the column accumulators
// acc[p] and returns the packed row sum sum_k q rho_ik (the caller multiplies
// by rho_ij).
__device__ __forceinline__ float2 row_half(const float4* xy, const float4* zr, int stride,
                                           const float2* vx, const float2* vy, const float2* vz,
                                           const float2* rk, float2* acc, float2 ux, float2 uy,
                                           float2 uz, float2 u3x, float2 u3y, float2 u3z,
                                           float2 rij2) {
    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
        const float4 t0 = xy[p * stride];
        const float4 t1 = zr[p * stride];
        const float2 wx = make_float2(t0.x, t0.y);
        const float2 wy = make_float2(t0.z, t0.w);
        const float2 wz = make_float2(t1.x, t1.y);
        const float2 rjk = make_float2(t1.z, t1.w);
        float2 p1 = f2_mul(u3x, vx[p]);                // -3 cos t_i
        p1 = f2_fma(u3y, vy[p], p1);
        p1 = f2_fma(u3z, vz[p], p1);
        float2 p2 = f2_mul(ux, wx);                    // -cos t_j
        p2 = f2_fma(uy, wy, p2);
        p2 = f2_fma(uz, wz, p2);
        float2 p3 = f2_mul(vx[p], wx);                 // cos t_k
        p3 = f2_fma(vy[p], wy, p3);
        p3 = f2_fma(vz[p], wz, p3);
        const float2 t = f2_mul(f2_mul(p1, p2), p3);   // 3 cos cos cos
        const float2 q = f2_fma(t, rjk, rjk);          // (1 + 3 cos cos cos) rho_jk
        s2 = f2_fma(q, rk[p], s2);                     // row sum (x rho_ij later)
        acc[p] = f2_fma(q, rij2, acc[p]);              // column sums (x rho_ik later)
    }
    return s2;
}

// All triples of one I tile against the table (J rows x K columns).
//   ih, il         : lane's particle (hi/lo); iv: lane holds a particle
//   sJh/sJl, sKh/sKl: tile coordinates in shared memory
//   nJ             : valid rows; the K validity is already in the table
//   maskIJ         : require lane < jj  (I == J);  maskIK: lane < kk (I == K)
//   redJ[jj][lane] : receives the lane's row sums (sum over k) for each j
//   redK[kk][lane] : receives the lane's column sums (sum over j) for each k
// Returns the lane's total (its particle's share).
__device__ __forceinline__ float tile_triples(const TabPair (*tab)[kTile / 2], const float4* sJh,
                                              const float4* sJl, const float4* sKh,
                                              const float4* sKl, float4 ih, float4 il, bool iv,
                                              int lane, int nJ, int nK, bool maskIJ, bool maskIK,
                                              float (*redJ)[kTile + 1], float (*redK)[kTile + 1]) {
    float acc_i = 0.f;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int kb = half * kHalf;
        float2 vx[kPairs], vy[kPairs], vz[kPairs], rk[kPairs], acc[kPairs];
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
            float e[2][4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int kk = kb + 2 * p + q;
                float s;
                const PairF pr = pair_unit(ih, il, sKh[kk], sKl[kk], &s);
                const bool v = iv && kk < nK && (!maskIK || lane < kk) && s > 0.f;
                e[q][0] = v ? pr.ex : 0.f;
                e[q][1] = v ? pr.ey : 0.f;
                e[q][2] = v ? pr.ez : 0.f;
                e[q][3] = v ? pr.rho : 0.f;
            }
            vx[p] = make_float2(e[0][0], e[1][0]);
            vy[p] = make_float2(e[0][1], e[1][1]);
            vz[p] = make_float2(e[0][2], e[1][2]);
            rk[p] = make_float2(e[0][3], e[1][3]);
            acc[p] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int jj = 0; jj < kTile; ++jj) {
            float s;
            const PairF pu = pair_unit(ih, il, sJh[jj], sJl[jj], &s);
            const bool v = iv && jj < nJ && (!maskIJ || lane < jj) && s > 0.f;
            const float ex = v ? pu.ex : 0.f, ey = v ? pu.ey : 0.f, ez = v ? pu.ez : 0.f;
            const float2 ux = f2_splat(ex), uy = f2_splat(ey), uz = f2_splat(ez);
            const float2 u3x = f2_splat(-3.0f * ex), u3y = f2_splat(-3.0f * ey),
                         u3z = f2_splat(-3.0f * ez);
            const float rij = v ? pu.rho : 0.f;
            const float2 rij2 = f2_splat(rij);
            const TabPair* row = tab[jj] + (kb >> 1);
            const float2 s2 = row_half(&row->xy, &row->zr, 2, vx, vy, vz, rk, acc, ux, uy, uz,
                                       u3x, u3y, u3z, rij2);
            const float srow = (s2.x + s2.y) * rij;
            acc_i += srow;
            if (half == 0) redJ[jj][lane] = srow;
            else redJ[jj][lane] += srow;
        }
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
            const float2 c = f2_mul(acc[p], rk[p]);
            redK[kb + 2 * p][lane] = c.x;
            redK[kb + 2 * p + 1][lane] = c.y;
        }
    }
    __syncwarp();
    return acc_i;
}

// Pair-table block of one tile pair (A, B): 32 x 32 pair terms from particle
// A*32 + r to B*32 + c, stored as two planes indexed [column pair p][row r],
// so that a warp whose lanes are rows reads 512 contiguous bytes per plane.
struct PairBlock {
    float4 xy[kTile / 2][kTile];  // (ex_c, ex_c+1, ey_c, ey_c+1), c = 2p
    float4 zr[kTile / 2][kTile];  // (ez_c, ez_c+1, rho_c, rho_c+1)
};

// Per-warp staging ring of the lane's (i, j) pair terms: slot s holds one
// column pair of the (I, J) block (both planes, 32 lanes).
struct IjRing {
    float4 xy[2][kTile];
    float4 zr[2][kTile];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_1() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// The same sweep with every pair term read from a precomputed pair table
// (unit vector and r^-3 of each pair, computed in FP64 and rounded once to
// FP32) instead of formed from coordinates:
//   tab : block (J, K) in shared memory (rows j, columns k)
//   bIK : block (I, K) in global memory (the lane's row: its (i, k) terms)
//   bIJ : block (I, J) in global memory (the lane's row: its (i, j) terms),
//         staged one column pair ahead through the warp's ring by cp.async
//         (each lane copies and reads only its own entries)
// Masked and absent pairs are zero in the table, so no masks are needed here.
__device__ __forceinline__ float tile_triples_table(const PairBlock& tab,
                                                    const PairBlock* __restrict__ bIK,
                                                    const PairBlock* __restrict__ bIJ, int lane,
                                                    IjRing& ring, float (*redJ)[kTile + 1],
                                                    float (*redK)[kTile + 1]) {
    float acc_i = 0.f;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int kb = half * kHalf;
        float2 vx[kPairs], vy[kPairs], vz[kPairs], rk[kPairs], acc[kPairs];
        cp_async16(&ring.xy[0][lane], &bIJ->xy[0][lane]);
        cp_async16(&ring.zr[0][lane], &bIJ->zr[0][lane]);
        cp_async_commit();
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
            const float4 a = __ldg(&bIK->xy[(kb >> 1) + p][lane]);
            const float4 b = __ldg(&bIK->zr[(kb >> 1) + p][lane]);
            vx[p] = make_float2(a.x, a.y);
            vy[p] = make_float2(a.z, a.w);
            vz[p] = make_float2(b.x, b.y);
            rk[p] = make_float2(b.z, b.w);
            acc[p] = make_float2(0.f, 0.f);
        }
#pragma unroll 1
        for (int jp = 0; jp < kTile / 2; ++jp) {
            if (jp + 1 < kTile / 2) {
                cp_async16(&ring.xy[(jp + 1) & 1][lane], &bIJ->xy[jp + 1][lane]);
                cp_async16(&ring.zr[(jp + 1) & 1][lane], &bIJ->zr[jp + 1][lane]);
            }
            cp_async_commit();
            cp_async_wait_1();  // this column pair's copies have landed
            const float4 cxy = ring.xy[jp & 1][lane], czr = ring.zr[jp & 1][lane];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int jj = 2 * jp + o;
                const float ex = o ? cxy.y : cxy.x, ey = o ? cxy.w : cxy.z;
                const float ez = o ? czr.y : czr.x, rij = o ? czr.w : czr.z;
                const float2 s2 = row_half(&tab.xy[kb >> 1][jj], &tab.zr[kb >> 1][jj], kTile, vx,
                                           vy, vz, rk, acc, f2_splat(ex), f2_splat(ey),
                                           f2_splat(ez), f2_splat(-3.0f * ex),
                                           f2_splat(-3.0f * ey), f2_splat(-3.0f * ez),
                                           f2_splat(rij));
                const float srow = (s2.x + s2.y) * rij;
                acc_i += srow;
                if (half == 0) redJ[jj][lane] = srow;
                else redJ[jj][lane] += srow;
            }
        }
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
            const float2 c = f2_mul(acc[p], rk[p]);
            redK[kb + 2 * p][lane] = c.x;
            redK[kb + 2 * p + 1][lane] = c.y;
        }
    }
    __syncwarp();
    return acc_i;
}

// Sum of row `r` of a 32 x 33 reduction buffer (one lane per row).
__device__ __forceinline__ float row_sum(const float (*red)[kTile + 1], int r) {
    float s = 0.f;
#pragma unroll 8
    for (int m = 0; m < kTile; ++m) s += red[r][m];
    return s;
}

}  // namespace mbm_tile
