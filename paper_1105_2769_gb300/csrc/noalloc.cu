// Exhaustive FP32-bulk Phi without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// owns all device memory through its own pool and budget, a latency-bound
// loop where an allocation (and the synchronisation cudaFree implies) would
// stall other streams, or a plugin running inside a process that forbids
// foreign allocations. This entry point serves them: its scratch (work
// counter, status word and the packed hi/lo coordinates) lives in a
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the first call on each device resolves the
// address with cudaGetSymbolAddress, with that device current, and caches it
// for the process. The cache assumes the device's primary context lives as
// long as the process: a caller that resets the device must not call this
// entry point again (include/mbm.h says so).
#include <mutex>

#include "mbm_internal.h"

namespace {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr size_t kHeader = 256;  // counter at 0, status word at 64
constexpr size_t kScratchBytes = kHeader + (size_t)kNoAllocMaxN * 2 * sizeof(float4);
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set-up on first use).
mbm_status scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mbm_cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return MBM_OK;
}

}  // namespace

extern "C" mbm_status mbm_potential_fp32_noalloc(const double* X_dev, int64_t N, double* phi_dev,
                                                 mbm_stream_t stream) {
    if (N < 0) return mbm_fail(MBM_EINVAL, "N < 0");
    if (N > kNoAllocMaxN)
        return mbm_fail(MBM_EINVAL, "N exceeds the no-allocation entry point's maximum of 65536 "
                                    "particles; use mbm_potential");
    if (N > 0 && (!X_dev || !phi_dev)) return mbm_fail(MBM_EINVAL, "NULL X or output");
    int device = 0;
    MBM_CUDA_TRY(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) return mbm_fail(MBM_EINVAL, "device index too large");
    void* base = nullptr;
    MBM_TRY(scratch_address(device, &base));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) return MBM_OK;
    MBM_CUDA_TRY(cudaMemsetAsync(phi_dev, 0, (size_t)N * sizeof(double), s));
    if (N < 3) return MBM_OK;
    int num_sms = 0;
    MBM_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    char* b = static_cast<char*>(base);
    auto* counter = reinterpret_cast<unsigned long long*>(b);
    auto* flags = reinterpret_cast<int*>(b + 64);
    auto* xh = reinterpret_cast<float4*>(b + kHeader);
    auto* xl = xh + N;
    // The array keeps the previous call's contents: reset what starts at zero.
    MBM_CUDA_TRY(cudaMemsetAsync(b, 0, kHeader, s));
    MBM_CUDA_TRY(launch_pack_hilo(X_dev, N, xh, xl, flags, s));
    MBM_CUDA_TRY(launch_exh_fp32(xh, xl, N, phi_dev, counter, flags, num_sms, s));
    return MBM_OK;
}
