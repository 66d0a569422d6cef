// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/mbm.h"

// ---------------------------------------------------------------------------
// Error reporting (thread-local message behind mbm_last_error()).
// ---------------------------------------------------------------------------
void mbm_set_error(const std::string& msg);
mbm_status mbm_fail(mbm_status st, const std::string& msg);
mbm_status mbm_cuda_fail(cudaError_t e, const char* what);

#define MBM_CUDA_TRY(call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return mbm_cuda_fail(e_, #call);    \
    } while (0)

#define MBM_TRY(call)                          \
    do {                                       \
        mbm_status s_ = (call);                \
        if (s_ != MBM_OK) return s_;           \
    } while (0)

// Device-side status word bits (written with atomicOr, read after a sync).
enum : int {
    MBM_FLAG_NONFINITE = 1,   // a coordinate is NaN or Inf
    MBM_FLAG_COINCIDENT = 2,  // two particles at zero distance
    MBM_FLAG_OVERFLOW = 4,    // a bounded work list overflowed
    MBM_FLAG_TIMEOUT = 8,     // a bounded device wait gave up
    MBM_FLAG_INDEX = 16       // a particle index outside [0, N)
};

// ---------------------------------------------------------------------------
// Context: one GPU, a growable scratch arena, a device status word.
// ---------------------------------------------------------------------------
struct mbm_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;       // 0 = unlimited
    size_t in_use = 0;       // bytes held by scratch + trees
    void* scratch = nullptr; // device arena
    size_t scratch_bytes = 0;
    int* d_flags = nullptr;  // device status word (+ padding)
    int* h_flags = nullptr;  // pinned host mirror
    std::mutex mu;           // one solve at a time per context
    bool timing = false;     // record events around the dominant kernel
    bool timed = false;      // the last solve recorded events
    double timed_ms = -1.0;  // >= 0: the last solve's dominant-kernel time, summed
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Event helpers: no-ops unless ctx->timing.
void mbm_time_begin(mbm_ctx* ctx, cudaStream_t s);
void mbm_time_end(mbm_ctx* ctx, cudaStream_t s);
// Report an already summed dominant-kernel time for the last solve.
void mbm_time_set_ms(mbm_ctx* ctx, double ms);

// Make sure the arena holds at least `bytes`; may reallocate (synchronous).
mbm_status mbm_scratch_reserve(mbm_ctx* ctx, size_t bytes);
// Charge/uncharge library-owned bytes against the budget.
mbm_status mbm_budget_charge(mbm_ctx* ctx, size_t bytes);
void mbm_budget_release(mbm_ctx* ctx, size_t bytes);
// Synchronise `stream`, read and clear the status word, map it to a status.
mbm_status mbm_check_flags(mbm_ctx* ctx, cudaStream_t stream);

static inline size_t mbm_align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Launchers (each .cu file owns its kernels).
// ---------------------------------------------------------------------------
// Input pack (step a1): FP64 AoS -> FP32 hi/lo float4 pairs, finite check.
cudaError_t launch_pack_hilo(const double* X, int64_t N, float4* xhi, float4* xlo, int* flags,
                             cudaStream_t s);
// Input pack to FP64 float4-like (x, y, z, 0) double quads.
cudaError_t launch_pack_f64(const double* X, int64_t N, double4_32a* x4, int* flags, cudaStream_t s);

// Exhaustive sums (steps a2/a3). phi must be zeroed by the caller.
// counter: one zeroed unsigned long long of scratch for dynamic scheduling.
cudaError_t launch_exh_fp32(const float4* xhi, const float4* xlo, int64_t N, double* phi,
                            unsigned long long* counter, int* flags, int num_sms,
                            cudaStream_t s);
// Pair table of the FP32-bulk sum (unit vector and r^-3 of every pair, FP64
// rounded once to FP32): its size, its build from X, and the sum that reads it.
size_t pair_table_bytes(int64_t N);
cudaError_t launch_pair_table(const double* X, int64_t N, void* table, int* flags, cudaStream_t s);
cudaError_t launch_exh_fp32_table(const void* table, int64_t N, double* phi,
                                  unsigned long long* counter, int* flags, int num_sms,
                                  cudaStream_t s);
cudaError_t launch_exh_fp64(const double4_32a* x4, int64_t N, double* phi, unsigned long long* counter,
                            int* flags, int num_sms, cudaStream_t s);
// Exact FP32-bulk Phi of sampled particles idx[0..n_idx) (out zeroed by the caller).
cudaError_t launch_sampled_fp32(const float4* xhi, const float4* xlo, int64_t N,
                                const int64_t* idx, int64_t n_idx, double* out, int* flags,
                                int num_sms, cudaStream_t s);
