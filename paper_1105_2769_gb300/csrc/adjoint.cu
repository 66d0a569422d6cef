// Forces and vector-Jacobian products of Phi (no counterpart in the paper;
// the derivative of the Axilrod-Teller summand of Eq. 1).
//
// For a triple (i, j, k) with unit edge vectors e_u = e_ij, e_v = e_ik,
// e_w = e_jk, p1 = e_u.e_v, p2 = e_u.e_w, p3 = e_v.e_w, t = p1 p2 p3 and
// R = (r_ij r_ik r_jk)^-3, phi = R (1 - 3t), and
//   grad_i phi = -c1 e_u - c2 e_v + c3 e_w,
//   c1 = s_u q - s_v p2 p3,  c2 = s_v q - s_u p2 p3,  c3 = s_u p1 p3 + s_v p1 p2,
//   q = 5t - 1,  s_u = 3R / r_ij,  s_v = 3R / r_ik.
// (From phi = L^-3/2 - 3 G L^-5/2 with L = |u|^2 |v|^2 |w|^2 and
// G = (u.v)(u.w)(v.w), u = x_j - x_i, v = x_k - x_i, w = x_k - x_j.)
//
// Gather form: a lane owns particle i and sums grad_i over every pair j < k
// of the set (pairs through i drop out: their distance is exactly zero), so
// each triple is evaluated once per member and no cross-lane reduction is
// needed. A CTA owns 8 consecutive I tiles (one per warp) and a chunk of (J,K)
// tile pairs; the (j,k) table is shared by its warps. The e_u terms are
// summed per j and the e_v terms per column before the vector products, so
// the inner loop carries one 3-vector FMA per triple.
//   VJP:    grad_m sum_l g_l Phi_l = sum_{j<k} (g_m + g_j + g_k) grad_m phi(m,j,k)
//   forces: F_i = -sum_{j<k} grad_i phi(i,j,k)      (weights 1)
// Inner loop (per lane-triple, FP32): 9 (dots) + 4 (A1, t, A2, A3) + 1 (q)
// + 2 (R) + 1 (W) + 2 (s_u, s_v) + 6 (c1, c2, c3) + 5 (sums) = 30 operations.
#include <cstring>

#include "device_math.cuh"
#include "mbm_internal.h"
#include "mbm_tree_api.h"

namespace {

constexpr int kTile = 32;
constexpr int kWarps = 8;

template <typename Real>
struct Vec4 {
    Real x, y, z, w;
};

template <typename Real>
struct AdjSmem {
    Vec4<Real> tab[kTile][kTile];  // (e_w, rho_w) for (j, k)
    Vec4<Real> sJ[kTile], sJl[kTile], sK[kTile], sKl[kTile];
    Real gJ[kTile], gK[kTile];
};

struct PairU32 {
    float ex, ey, ez, rho, i3;
};

// Unit vector p->q, rho = r^-3 and 3/r, FP32 from hi/lo coordinates (rsqrt
// refined by one Newton step).
__device__ __forceinline__ PairU32 pair32(float4 ph, float4 pl, float4 qh, float4 ql, bool& ok) {
    const float dx = (qh.x - ph.x) + (ql.x - pl.x);
    const float dy = (qh.y - ph.y) + (ql.y - pl.y);
    const float dz = (qh.z - ph.z) + (ql.z - pl.z);
    const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float y = rsqrtf(s);
    const float h = s * y;
    y = fmaf(0.5f * y, fmaf(-h, y, 1.0f), y);
    ok = s > 0.f;
    PairU32 r;
    r.ex = dx * y;
    r.ey = dy * y;
    r.ez = dz * y;
    r.rho = y * y * y;
    r.i3 = 3.0f * y;
    return r;
}

struct PairU64 {
    double ex, ey, ez, rho, i3;
};

__device__ __forceinline__ PairU64 pair64(double4_32a p, double4_32a q, bool& ok) {
    const double dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    const double s = dx * dx + dy * dy + dz * dz;
    ok = s > 0.0;
    const double y = ok ? rsqrt(s) : 0.0;
    PairU64 r;
    r.ex = dx * y;
    r.ey = dy * y;
    r.ez = dz * y;
    r.rho = y * y * y;
    r.i3 = 3.0 * y;
    return r;
}

// Loader of a particle in either precision.
struct Pts32 {
    const float4* xh;
    const float4* xl;
};
struct Pts64 {
    const double4_32a* x;
};

template <typename Real, int KSUB, typename Pts>
__global__ void __launch_bounds__(kWarps * 32, 1)
adjoint_kernel(Pts pts, int N, int NT, const double* __restrict__ g, long long pairs_per_chunk,
               long long n_chunks, long long n_pairs, double* __restrict__ grad, double sign) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmem<Real>& sm = *reinterpret_cast<AdjSmem<Real>*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int groups = (NT + kWarps - 1) / kWarps;
    for (long long item = blockIdx.x; item < (long long)groups * n_chunks; item += gridDim.x) {
        const int grp = (int)(item / n_chunks);
        const long long chunk = item % n_chunks;
        const int I = grp * kWarps + warp;
        const int i = I * kTile + lane;
        const bool iv = I < NT && i < N;
        Vec4<Real> xi{0, 0, 0, 0}, xil{0, 0, 0, 0};
        if constexpr (sizeof(Real) == 4) {
            if (iv) {
                const float4 a = pts.xh[i], b = pts.xl[i];
                xi = {a.x, a.y, a.z, 0.f};
                xil = {b.x, b.y, b.z, 0.f};
            }
        } else {
            if (iv) {
                const double4_32a a = pts.x[i];
                xi = {a.x, a.y, a.z, 0.0};
            }
        }
        const Real gi = (g && iv) ? (Real)g[i] : (Real)0;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        const long long p0 = chunk * pairs_per_chunk;
        const long long p1 = p0 + pairs_per_chunk < n_pairs ? p0 + pairs_per_chunk : n_pairs;
        for (long long t = p0; t < p1; ++t) {
            int J, K;
            decode_pair_item(t, NT, J, K);
            const int nJ = min(kTile, N - J * kTile), nK = min(kTile, N - K * kTile);
            __syncthreads();  // previous table no longer in use
            if (threadIdx.x < kTile) {
                const int jj = threadIdx.x, j = J * kTile + jj;
                if constexpr (sizeof(Real) == 4) {
                    const float4 a = jj < nJ ? pts.xh[j] : make_float4(0, 0, 0, 0);
                    const float4 b = jj < nJ ? pts.xl[j] : make_float4(0, 0, 0, 0);
                    sm.sJ[jj] = {a.x, a.y, a.z, 0.f};
                    sm.sJl[jj] = {b.x, b.y, b.z, 0.f};
                } else {
                    const double4_32a a = jj < nJ ? pts.x[j] : make_double4_32a(0, 0, 0, 0);
                    sm.sJ[jj] = {a.x, a.y, a.z, 0.0};
                }
                sm.gJ[jj] = (g && jj < nJ) ? (Real)g[j] : (Real)0;
            } else if (threadIdx.x < 2 * kTile) {
                const int kk = threadIdx.x - kTile, k = K * kTile + kk;
                if constexpr (sizeof(Real) == 4) {
                    const float4 a = kk < nK ? pts.xh[k] : make_float4(0, 0, 0, 0);
                    const float4 b = kk < nK ? pts.xl[k] : make_float4(0, 0, 0, 0);
                    sm.sK[kk] = {a.x, a.y, a.z, 0.f};
                    sm.sKl[kk] = {b.x, b.y, b.z, 0.f};
                } else {
                    const double4_32a a = kk < nK ? pts.x[k] : make_double4_32a(0, 0, 0, 0);
                    sm.sK[kk] = {a.x, a.y, a.z, 0.0};
                }
                sm.gK[kk] = (g && kk < nK) ? (Real)g[k] : (Real)0;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
                const int jj = e >> 5, kk = e & 31;
                const bool v = jj < nJ && kk < nK && (J != K || jj < kk);
                bool ok;
                Vec4<Real> ent{0, 0, 0, 0};
                if constexpr (sizeof(Real) == 4) {
                    const PairU32 pr = pair32(make_float4(sm.sJ[jj].x, sm.sJ[jj].y, sm.sJ[jj].z, 0),
                                              make_float4(sm.sJl[jj].x, sm.sJl[jj].y, sm.sJl[jj].z, 0),
                                              make_float4(sm.sK[kk].x, sm.sK[kk].y, sm.sK[kk].z, 0),
                                              make_float4(sm.sKl[kk].x, sm.sKl[kk].y, sm.sKl[kk].z, 0),
                                              ok);
                    if (v && ok) ent = {pr.ex, pr.ey, pr.ez, pr.rho};
                } else {
                    const PairU64 pr = pair64(make_double4_32a(sm.sJ[jj].x, sm.sJ[jj].y, sm.sJ[jj].z, 0),
                                              make_double4_32a(sm.sK[kk].x, sm.sK[kk].y, sm.sK[kk].z, 0),
                                              ok);
                    if (v && ok) ent = {pr.ex, pr.ey, pr.ez, pr.rho};
                }
                sm.tab[jj][kk] = ent;
            }
            __syncthreads();
            if (!iv) continue;
            // ---- lane's particle i against the table ----
            Real G1x = 0, G1y = 0, G1z = 0, G3x = 0, G3y = 0, G3z = 0;
            Real G2x = 0, G2y = 0, G2z = 0;
            for (int kb = 0; kb < kTile; kb += KSUB) {
                Real vx[KSUB], vy[KSUB], vz[KSUB], rv[KSUB], sv[KSUB], a2[KSUB];
#pragma unroll
                for (int q = 0; q < KSUB; ++q) {
                    const int kk = kb + q;
                    bool ok;
                    Real ex, ey, ez, rho, i3;
                    if constexpr (sizeof(Real) == 4) {
                        const PairU32 pr = pair32(make_float4(xi.x, xi.y, xi.z, 0),
                                                  make_float4(xil.x, xil.y, xil.z, 0),
                                                  make_float4(sm.sK[kk].x, sm.sK[kk].y, sm.sK[kk].z, 0),
                                                  make_float4(sm.sKl[kk].x, sm.sKl[kk].y, sm.sKl[kk].z, 0),
                                                  ok);
                        ex = pr.ex; ey = pr.ey; ez = pr.ez; rho = pr.rho; i3 = pr.i3;
                    } else {
                        const PairU64 pr = pair64(make_double4_32a(xi.x, xi.y, xi.z, 0),
                                                  make_double4_32a(sm.sK[kk].x, sm.sK[kk].y, sm.sK[kk].z, 0),
                                                  ok);
                        ex = pr.ex; ey = pr.ey; ez = pr.ez; rho = pr.rho; i3 = pr.i3;
                    }
                    const bool v = kk < nK && ok;  // k == i gives zero distance
                    vx[q] = v ? ex : (Real)0;
                    vy[q] = v ? ey : (Real)0;
                    vz[q] = v ? ez : (Real)0;
                    rv[q] = v ? rho : (Real)0;
                    sv[q] = v ? i3 : (Real)0;
                    a2[q] = 0;
                }
#pragma unroll 1
                for (int jj = 0; jj < nJ; ++jj) {
                    bool ok;
                    Real ux, uy, uz, ru, su;
                    if constexpr (sizeof(Real) == 4) {
                        const PairU32 pr = pair32(make_float4(xi.x, xi.y, xi.z, 0),
                                                  make_float4(xil.x, xil.y, xil.z, 0),
                                                  make_float4(sm.sJ[jj].x, sm.sJ[jj].y, sm.sJ[jj].z, 0),
                                                  make_float4(sm.sJl[jj].x, sm.sJl[jj].y, sm.sJl[jj].z, 0),
                                                  ok);
                        ux = pr.ex; uy = pr.ey; uz = pr.ez; ru = pr.rho; su = pr.i3;
                    } else {
                        const PairU64 pr = pair64(make_double4_32a(xi.x, xi.y, xi.z, 0),
                                                  make_double4_32a(sm.sJ[jj].x, sm.sJ[jj].y, sm.sJ[jj].z, 0),
                                                  ok);
                        ux = pr.ex; uy = pr.ey; uz = pr.ez; ru = pr.rho; su = pr.i3;
                    }
                    if (!ok) continue;  // j == i (lane-divergent, rare)
                    const Real wij = g ? gi + sm.gJ[jj] : (Real)1;
                    Real a1 = 0;
                    const Vec4<Real>* row = sm.tab[jj] + kb;
#pragma unroll
                    for (int q = 0; q < KSUB; ++q) {
                        const Vec4<Real> w = row[q];
                        const Real p1 = ux * vx[q] + uy * vy[q] + uz * vz[q];
                        const Real p2 = ux * w.x + uy * w.y + uz * w.z;
                        const Real p3 = vx[q] * w.x + vy[q] * w.y + vz[q] * w.z;
                        const Real A1 = p2 * p3;
                        const Real tt = p1 * A1;
                        const Real A2 = p1 * p3, A3 = p1 * p2;
                        const Real qf = (Real)5 * tt - (Real)1;
                        const Real W = g ? wij + sm.gK[kb + q] : (Real)1;
                        const Real RW = ru * rv[q] * w.w * W;
                        const Real s_u = RW * su, s_v = RW * sv[q];
                        const Real c1 = s_u * qf - s_v * A1;
                        const Real c2 = s_v * qf - s_u * A1;
                        const Real c3 = s_u * A2 + s_v * A3;
                        a1 += c1;
                        a2[q] += c2;
                        G3x += c3 * w.x;
                        G3y += c3 * w.y;
                        G3z += c3 * w.z;
                    }
                    G1x += a1 * ux;
                    G1y += a1 * uy;
                    G1z += a1 * uz;
                }
#pragma unroll
                for (int q = 0; q < KSUB; ++q) {
                    G2x += a2[q] * vx[q];
                    G2y += a2[q] * vy[q];
                    G2z += a2[q] * vz[q];
                }
            }
            gx += (double)(G3x - G1x - G2x);
            gy += (double)(G3y - G1y - G2y);
            gz += (double)(G3z - G1z - G2z);
        }
        if (iv) {
            atomicAdd(&grad[3 * (int64_t)i], sign * gx);
            atomicAdd(&grad[3 * (int64_t)i + 1], sign * gy);
            atomicAdd(&grad[3 * (int64_t)i + 2], sign * gz);
        }
    }
}

__global__ void pack64_kernel(const double* __restrict__ X, int64_t N, double4_32a* x4, int* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(flags, MBM_FLAG_NONFINITE);
        x4[i] = make_double4_32a(x, y, z, 0.0);
    }
}

template <typename Real, int KSUB, typename Pts>
cudaError_t launch_adjoint(Pts pts, int64_t N, const double* g, double* grad, double sign,
                           int num_sms, cudaStream_t s) {
    const int NT = (int)((N + kTile - 1) / kTile);
    const long long n_pairs = (long long)NT * (NT + 1) / 2;
    const int groups = (NT + kWarps - 1) / kWarps;
    // enough items for ~4 waves; at least 64 pairs per chunk to amortise the table
    const long long want_items = (long long)(num_sms > 0 ? num_sms : 1) * 4;
    long long n_chunks = (want_items + groups - 1) / groups;
    if (n_chunks < 1) n_chunks = 1;
    long long ppc = (n_pairs + n_chunks - 1) / n_chunks;
    if (ppc < 64) ppc = 64;
    n_chunks = (n_pairs + ppc - 1) / ppc;
    const size_t smem = sizeof(AdjSmem<Real>);
    auto kern = adjoint_kernel<Real, KSUB, Pts>;
    cudaError_t e = cudaFuncSetAttribute((const void*)kern,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long long items = (long long)groups * n_chunks;
    int grid = (int)(items < 65535 ? items : 65535);
    kern<<<grid, kWarps * 32, smem, s>>>(pts, (int)N, NT, g, ppc, n_chunks, n_pairs, grad, sign);
    return cudaGetLastError();
}

mbm_status run_adjoint(mbm_ctx* ctx, const double* X, int64_t N, const double* g, int mode,
                       double* out, double sign, cudaStream_t s) {
    if (mode != MBM_EXH_FP32 && mode != MBM_EXH_FP64)
        return mbm_fail(MBM_ENOTSUP, "forces and VJP support MBM_EXH_FP32 and MBM_EXH_FP64");
    MBM_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)N * 3 * sizeof(double), s));
    if (N < 3) return MBM_OK;
    const size_t pack = mode == MBM_EXH_FP32 ? (size_t)N * 2 * sizeof(float4)
                                             : (size_t)N * sizeof(double4_32a);
    MBM_TRY(mbm_scratch_reserve(ctx, 256 + pack));
    char* base = static_cast<char*>(ctx->scratch) + 256;
    MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    mbm_time_begin(ctx, s);
    if (mode == MBM_EXH_FP32) {
        auto* xh = reinterpret_cast<float4*>(base);
        auto* xl = xh + N;
        MBM_CUDA_TRY(launch_pack_hilo(X, N, xh, xl, ctx->d_flags, s));
        MBM_CUDA_TRY((launch_adjoint<float, 16>(Pts32{xh, xl}, N, g, out, sign, ctx->num_sms, s)));
    } else {
        auto* x4 = reinterpret_cast<double4_32a*>(base);
        const int64_t blocks = (N + 255) / 256;
        pack64_kernel<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(X, N, x4,
                                                                                 ctx->d_flags);
        MBM_CUDA_TRY(cudaGetLastError());
        MBM_CUDA_TRY((launch_adjoint<double, 8>(Pts64{x4}, N, g, out, sign, ctx->num_sms, s)));
    }
    mbm_time_end(ctx, s);
    return MBM_OK;
}

}  // namespace

extern "C" mbm_status mbm_forces_ex(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                                    double alpha, int mode, const mbm_config* cfg, mbm_tree* tree,
                                    double* F_dev, mbm_stats* stats, mbm_stream_t stream) {
    if (!ctx) return mbm_fail(MBM_EINVAL, "ctx is NULL");
    if (N < 0) return mbm_fail(MBM_EINVAL, "N < 0");
    if (N > 0 && (!X_dev || !F_dev)) return mbm_fail(MBM_EINVAL, "NULL X or output");
    if (!(eps >= 0.0)) return mbm_fail(MBM_EINVAL, "eps must be >= 0");
    if (!(alpha >= 0.0 && alpha < 1.0)) return mbm_fail(MBM_EINVAL, "alpha must be in [0, 1)");
    const int base_mode = mode & 0xff;
    if (base_mode != MBM_EXH_FP64 && base_mode != MBM_EXH_FP32 && base_mode != MBM_TREE)
        return mbm_fail(MBM_EINVAL, "unknown mode");
    if ((mode & ~0x1ff) != 0 || ((mode & MBM_ABS) && base_mode != MBM_TREE))
        return mbm_fail(MBM_EINVAL, "unknown mode flags");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    mbm_config c;
    if (cfg) c = *cfg;
    else mbm_config_default(&c);
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    if (N == 0) return MBM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (base_mode == MBM_TREE) {
        if (N < 3) {
            MBM_CUDA_TRY(cudaMemsetAsync(F_dev, 0, (size_t)N * 3 * sizeof(double), s));
            return MBM_OK;
        }
        return mbm_tree_forces(ctx, X_dev, N, eps, alpha, (mode & MBM_ABS) != 0, c, tree, F_dev,
                               stats, s);
    }
    return run_adjoint(ctx, X_dev, N, nullptr, mode, F_dev, -1.0, s);
}

extern "C" mbm_status mbm_forces(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                                 double alpha, int mode, double* F_dev, mbm_stream_t stream) {
    return mbm_forces_ex(ctx, X_dev, N, eps, alpha, mode, nullptr, nullptr, F_dev, nullptr,
                         stream);
}

extern "C" mbm_status mbm_potential_vjp(mbm_ctx* ctx, const double* X_dev, int64_t N,
                                        const double* g_dev, int mode, double* gradX_dev,
                                        mbm_stream_t stream) {
    if (!ctx) return mbm_fail(MBM_EINVAL, "ctx is NULL");
    if (N < 0) return mbm_fail(MBM_EINVAL, "N < 0");
    if (N > 0 && (!X_dev || !gradX_dev || !g_dev)) return mbm_fail(MBM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    if (N == 0) return MBM_OK;
    return run_adjoint(ctx, X_dev, N, g_dev, mode, gradX_dev, 1.0,
                       reinterpret_cast<cudaStream_t>(stream));
}
