// C ABI entry points: contexts, scratch, validation and the exhaustive
// solves. The tree path, the adjoint and the serving loop have their own
// translation units; this file dispatches to them.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "mbm_internal.h"
#include "mbm_tree_api.h"

namespace {
thread_local std::string g_last_error;
}

void mbm_set_error(const std::string& msg) { g_last_error = msg; }

mbm_status mbm_fail(mbm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

mbm_status mbm_cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MBM_ENOMEM : MBM_ECUDA;
}

extern "C" const char* mbm_version(void) { return "mbm 0.1 (sm_103a)"; }

extern "C" const char* mbm_last_error(void) { return g_last_error.c_str(); }

extern "C" void mbm_config_default(mbm_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->tau = 0.0;
    cfg->leaf_size = 32;
    cfg->m_limit = 256;
    cfg->zeta = 32.0;
    cfg->seed = 0x5eed5eedULL;
    cfg->mc_rule = 0;
    cfg->validate = 1;
    cfg->seed_levels = 8;
    cfg->tuple_counts = nullptr;
}

mbm_status mbm_budget_charge(mbm_ctx* ctx, size_t bytes) {
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return mbm_fail(MBM_EBUDGET, "request exceeds the context's HBM budget (" +
                                         std::to_string(ctx->in_use + bytes) + " > " +
                                         std::to_string(ctx->budget) + " bytes)");
    ctx->in_use += bytes;
    return MBM_OK;
}

void mbm_budget_release(mbm_ctx* ctx, size_t bytes) {
    ctx->in_use = bytes > ctx->in_use ? 0 : ctx->in_use - bytes;
}

mbm_status mbm_scratch_reserve(mbm_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->scratch_bytes) return MBM_OK;
    size_t want = mbm_align_up(bytes + bytes / 4, 1 << 20);  // grow with headroom
    if (ctx->budget && ctx->in_use - ctx->scratch_bytes + want > ctx->budget) want = bytes;
    const size_t old = ctx->scratch_bytes;
    mbm_budget_release(ctx, old);
    mbm_status st = mbm_budget_charge(ctx, want);
    if (st != MBM_OK) {
        mbm_budget_charge(ctx, old);
        return st;
    }
    if (ctx->scratch) {
        // The old arena may still be read by work in flight on any stream.
        cudaDeviceSynchronize();
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        mbm_budget_release(ctx, want);
        ctx->scratch = nullptr;
        return mbm_cuda_fail(e, "cudaMalloc(scratch)");
    }
    ctx->scratch_bytes = want;
    return MBM_OK;
}

mbm_status mbm_check_flags(mbm_ctx* ctx, cudaStream_t stream) {
    MBM_CUDA_TRY(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost,
                                 stream));
    MBM_CUDA_TRY(cudaStreamSynchronize(stream));
    const int f = ctx->h_flags[0];
    if (f) MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), stream));
    if (f & MBM_FLAG_NONFINITE) return mbm_fail(MBM_EINVAL, "non-finite coordinate in X");
    if (f & MBM_FLAG_COINCIDENT)
        return mbm_fail(MBM_EINVAL, "two particles coincide (phi is undefined at r = 0)");
    if (f & MBM_FLAG_OVERFLOW) return mbm_fail(MBM_EOVERFLOW, "device work list overflow");
    if (f & MBM_FLAG_TIMEOUT) return mbm_fail(MBM_ETIMEDOUT, "device wait timed out");
    if (f & MBM_FLAG_INDEX) return mbm_fail(MBM_EINVAL, "particle index outside [0, N)");
    return MBM_OK;
}

extern "C" mbm_status mbm_ctx_create(int device, size_t hbm_budget_bytes, mbm_ctx** out) {
    if (!out) return mbm_fail(MBM_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    MBM_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return mbm_fail(MBM_EINVAL, "no such CUDA device");
    MBM_CUDA_TRY(cudaSetDevice(device));
    mbm_ctx* ctx = new (std::nothrow) mbm_ctx();
    if (!ctx) return mbm_fail(MBM_ENOMEM, "host allocation failed");
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&ctx->d_flags, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_flags, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_flags, 256);
    if (e != cudaSuccess) {
        if (ctx->d_flags) cudaFree(ctx->d_flags);
        delete ctx;
        return mbm_cuda_fail(e, "context set-up");
    }
    *out = ctx;
    return MBM_OK;
}

extern "C" mbm_status mbm_ctx_destroy(mbm_ctx* ctx) {
    if (!ctx) return MBM_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return MBM_OK;
}

extern "C" size_t mbm_ctx_bytes_in_use(const mbm_ctx* ctx) { return ctx ? ctx->in_use : 0; }

extern "C" mbm_status mbm_ctx_set_timing(mbm_ctx* ctx, int enable) {
    if (!ctx) return mbm_fail(MBM_EINVAL, "ctx is NULL");
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    if (enable && !ctx->ev0) {
        MBM_CUDA_TRY(cudaEventCreate(&ctx->ev0));
        MBM_CUDA_TRY(cudaEventCreate(&ctx->ev1));
    }
    ctx->timing = enable != 0;
    ctx->timed = false;
    return MBM_OK;
}

extern "C" double mbm_ctx_last_kernel_ms(mbm_ctx* ctx) {
    if (!ctx) return -1.0;
    if (ctx->timed_ms >= 0.0) return ctx->timed_ms;
    if (!ctx->timed) return -1.0;
    if (cudaEventSynchronize(ctx->ev1) != cudaSuccess) return -1.0;
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) != cudaSuccess) return -1.0;
    return (double)ms;
}

void mbm_time_begin(mbm_ctx* ctx, cudaStream_t s) {
    if (ctx->timing) {
        cudaEventRecord(ctx->ev0, s);
        ctx->timed = false;
        ctx->timed_ms = -1.0;
    }
}

void mbm_time_set_ms(mbm_ctx* ctx, double ms) {
    ctx->timed = false;
    ctx->timed_ms = ms;
}

void mbm_time_end(mbm_ctx* ctx, cudaStream_t s) {
    if (ctx->timing) {
        cudaEventRecord(ctx->ev1, s);
        ctx->timed = true;
    }
}

// ---------------------------------------------------------------------------
// Exhaustive solves (steps a1 + a2/a3).
// ---------------------------------------------------------------------------
// Largest N whose FP32-bulk solve reads a pair table (NT(NT+1)/2 blocks of
// 16 KB: 8.6 GB at N = 32 768, 34 GB at 65 536). Larger sets, or a table that
// does not fit the context's budget or the device, form pair terms in the
// kernel instead (FP32 set-up, a few ulp per pair term).
constexpr int64_t kPairTableMaxN = 65536;

static mbm_status run_exhaustive(mbm_ctx* ctx, const double* X, int64_t N, int mode, double* phi,
                                 int validate, cudaStream_t s) {
    const size_t hdr = 256;  // work counter
    if (mode == MBM_EXH_FP32 && N <= kPairTableMaxN) {
        const size_t tb = pair_table_bytes(N);
        const mbm_status rs = mbm_scratch_reserve(ctx, hdr + tb);
        if (rs == MBM_OK) {
            char* base = static_cast<char*>(ctx->scratch);
            auto* counter = reinterpret_cast<unsigned long long*>(base);
            MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
            MBM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
            MBM_CUDA_TRY(cudaMemsetAsync(phi, 0, (size_t)N * sizeof(double), s));
            MBM_CUDA_TRY(launch_pair_table(X, N, base + hdr, ctx->d_flags, s));
            mbm_time_begin(ctx, s);
            MBM_CUDA_TRY(launch_exh_fp32_table(base + hdr, N, phi, counter, ctx->d_flags,
                                               ctx->num_sms, s));
            mbm_time_end(ctx, s);
            if (validate) return mbm_check_flags(ctx, s);
            return MBM_OK;
        }
        if (rs != MBM_EBUDGET && rs != MBM_ENOMEM) return rs;
        cudaGetLastError();  // clear a failed allocation; take the path without a table
    }
    const size_t pack = mode == MBM_EXH_FP32 ? (size_t)N * 2 * sizeof(float4)
                                             : (size_t)N * sizeof(double4_32a);
    MBM_TRY(mbm_scratch_reserve(ctx, hdr + pack));
    char* base = static_cast<char*>(ctx->scratch);
    auto* counter = reinterpret_cast<unsigned long long*>(base);
    MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    MBM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    MBM_CUDA_TRY(cudaMemsetAsync(phi, 0, (size_t)N * sizeof(double), s));
    if (mode == MBM_EXH_FP32) {
        auto* xh = reinterpret_cast<float4*>(base + hdr);
        auto* xl = xh + N;
        MBM_CUDA_TRY(launch_pack_hilo(X, N, xh, xl, ctx->d_flags, s));
        mbm_time_begin(ctx, s);
        MBM_CUDA_TRY(launch_exh_fp32(xh, xl, N, phi, counter, ctx->d_flags, ctx->num_sms, s));
        mbm_time_end(ctx, s);
    } else {
        auto* x4 = reinterpret_cast<double4_32a*>(base + hdr);
        MBM_CUDA_TRY(launch_pack_f64(X, N, x4, ctx->d_flags, s));
        mbm_time_begin(ctx, s);
        MBM_CUDA_TRY(launch_exh_fp64(x4, N, phi, counter, ctx->d_flags, ctx->num_sms, s));
        mbm_time_end(ctx, s);
    }
    if (validate) return mbm_check_flags(ctx, s);
    return MBM_OK;
}

static mbm_status check_common(mbm_ctx* ctx, const double* X, int64_t N, const void* out) {
    if (!ctx) return mbm_fail(MBM_EINVAL, "ctx is NULL");
    if (N < 0) return mbm_fail(MBM_EINVAL, "N < 0");
    if (N > ((int64_t)1 << 31) - 64) return mbm_fail(MBM_EINVAL, "N too large (max 2^31 - 64)");
    if (N > 0 && (!X || !out)) return mbm_fail(MBM_EINVAL, "NULL X or output");
    return MBM_OK;
}

extern "C" mbm_status mbm_potential_ex(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                                       double alpha, int mode, const mbm_config* cfg,
                                       mbm_tree* tree, double* phi_dev, mbm_stats* stats,
                                       mbm_stream_t stream) {
    MBM_TRY(check_common(ctx, X_dev, N, phi_dev));
    mbm_config c;
    if (cfg) c = *cfg;
    else mbm_config_default(&c);
    if (!(eps >= 0.0)) return mbm_fail(MBM_EINVAL, "eps must be >= 0");
    if (!(alpha >= 0.0 && alpha < 1.0)) return mbm_fail(MBM_EINVAL, "alpha must be in [0, 1)");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const int base_mode = mode & 0xff;
    if (base_mode != MBM_EXH_FP64 && base_mode != MBM_EXH_FP32 && base_mode != MBM_TREE)
        return mbm_fail(MBM_EINVAL, "unknown mode");
    if ((mode & ~0x1ff) != 0 || ((mode & MBM_ABS) && base_mode != MBM_TREE))
        return mbm_fail(MBM_EINVAL, "unknown mode flags");
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (N < 3) {
        if (N > 0) MBM_CUDA_TRY(cudaMemsetAsync(phi_dev, 0, (size_t)N * sizeof(double), s));
        return MBM_OK;
    }
    if (base_mode == MBM_TREE)
        return mbm_tree_potential(ctx, X_dev, N, eps, alpha, (mode & MBM_ABS) != 0, c, tree,
                                  phi_dev, stats, s);
    return run_exhaustive(ctx, X_dev, N, base_mode, phi_dev, c.validate, s);
}

extern "C" mbm_status mbm_potential(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                                    double alpha, int mode, double* phi_dev, mbm_stream_t stream) {
    return mbm_potential_ex(ctx, X_dev, N, eps, alpha, mode, nullptr, nullptr, phi_dev, nullptr,
                            stream);
}

extern "C" mbm_status mbm_potential_host(mbm_ctx* ctx, const double* X_host, int64_t N, double eps,
                                         double alpha, int mode, const mbm_config* cfg,
                                         double* phi_host, mbm_stream_t stream) {
    MBM_TRY(check_common(ctx, X_host, N, phi_host));
    if (N == 0) return MBM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    // Host-side staging buffers are separate from the solve's scratch arena.
    const size_t xb = (size_t)N * 3 * sizeof(double), pb = (size_t)N * sizeof(double);
    MBM_TRY(mbm_budget_charge(ctx, xb + pb));
    void* dX = nullptr;
    void* dP = nullptr;
    cudaError_t e = cudaMallocAsync(&dX, xb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&dP, pb, s);
    mbm_status st = MBM_OK;
    if (e != cudaSuccess) {
        st = mbm_cuda_fail(e, "cudaMallocAsync(host staging)");
    } else {
        e = cudaMemcpyAsync(dX, X_host, xb, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = mbm_cuda_fail(e, "cudaMemcpyAsync(X)");
        if (st == MBM_OK)
            st = mbm_potential_ex(ctx, static_cast<double*>(dX), N, eps, alpha, mode, cfg, nullptr,
                                  static_cast<double*>(dP), nullptr, stream);
        if (st == MBM_OK) {
            e = cudaMemcpyAsync(phi_host, dP, pb, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) st = mbm_cuda_fail(e, "cudaMemcpyAsync(phi)");
        }
    }
    if (dX) cudaFreeAsync(dX, s);
    if (dP) cudaFreeAsync(dP, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == MBM_OK) st = mbm_cuda_fail(e, "cudaStreamSynchronize");
    mbm_budget_release(ctx, xb + pb);
    return st;
}

extern "C" mbm_status mbm_potential_sampled(mbm_ctx* ctx, const double* X_dev, int64_t N,
                                            const int64_t* idx_dev, int64_t n_idx,
                                            double* out_dev, mbm_stream_t stream) {
    MBM_TRY(check_common(ctx, X_dev, N, out_dev));
    if (n_idx < 0 || n_idx > (1 << 20)) return mbm_fail(MBM_EINVAL, "n_idx must be in [0, 2^20]");
    if (n_idx > 0 && !idx_dev) return mbm_fail(MBM_EINVAL, "NULL idx");
    std::lock_guard<std::mutex> lock(ctx->mu);
    MBM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n_idx == 0) return MBM_OK;
    MBM_CUDA_TRY(cudaMemsetAsync(out_dev, 0, (size_t)n_idx * sizeof(double), s));
    if (N < 3) return MBM_OK;
    MBM_TRY(mbm_scratch_reserve(ctx, 256 + (size_t)N * 2 * sizeof(float4)));
    char* base = static_cast<char*>(ctx->scratch);
    auto* xh = reinterpret_cast<float4*>(base + 256);
    auto* xl = xh + N;
    MBM_CUDA_TRY(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    MBM_CUDA_TRY(launch_pack_hilo(X_dev, N, xh, xl, ctx->d_flags, s));
    mbm_time_begin(ctx, s);
    MBM_CUDA_TRY(launch_sampled_fp32(xh, xl, N, idx_dev, n_idx, out_dev, ctx->d_flags,
                                     ctx->num_sms, s));
    mbm_time_end(ctx, s);
    return mbm_check_flags(ctx, s);
}
