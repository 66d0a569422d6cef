// Device radix sort of (64-bit key, 32-bit value) pairs and exclusive prefix
// sums, written for the tree path (Morton keys of the build, leaf-pair keys of
// the base-case flushes, Monte Carlo chunk offsets, base-case piece heads).
//
// Sort: least-significant-digit radix sort, 8-bit digits over [bit0, bit1),
// stable, so equal keys keep their input order (the Morton order breaks ties
// by particle index this way). Each pass over a tile of kTileItems items per
// block: (1) per-block digit histograms, stored digit-major; (2) an exclusive
// scan of those counts gives every (digit, block) its first output slot;
// (3) the block scatters its tile, each warp a contiguous part of it, ranking
// equal digits within 32 items by a match mask and carrying running per-warp
// digit counters, so the output keeps the input order within every digit.
//
// Scan: blocks of 1024 items scanned in shared memory, the block totals
// scanned the same way (recursively), then added back.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sort_scan.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kPerThread = 16;
constexpr int kTileItems = kThreads * kPerThread;  // 4096 items per block and pass
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kThreads)
digit_hist_kernel(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                  unsigned* __restrict__ hist, int n_blocks) {
    __shared__ unsigned h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileItems;
    for (int q = threadIdx.x; q < kTileItems; q += kThreads) {
        const int64_t i = base + q;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kThreads)
        hist[(int64_t)d * n_blocks + blockIdx.x] = h[d];
}

// Stable scatter of one tile: warp w owns items [w * 512, (w + 1) * 512) of the tile.
__global__ void __launch_bounds__(kThreads)
digit_scatter_kernel(const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
                     unsigned long long* __restrict__ kout, int* __restrict__ vout, int64_t n,
                     int shift, const unsigned* __restrict__ offs, int n_blocks) {
    __shared__ unsigned wcount[kWarpsPerBlock][kRadix];  // per warp: its digit counts, then cursors
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kPerWarp = kTileItems / kWarpsPerBlock;
    const int64_t base = (int64_t)blockIdx.x * kTileItems + (int64_t)warp * kPerWarp;
    for (int d = lane; d < kRadix; d += 32) wcount[warp][d] = 0;
    __syncwarp();
    for (int q = lane; q < kPerWarp; q += 32) {
        const int64_t i = base + q;
        if (i < n) atomicAdd(&wcount[warp][(unsigned)(kin[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    // cursor of (warp, digit) = global start of (digit, block) + counts of earlier warps
    for (int d = threadIdx.x; d < kRadix; d += kThreads) {
        unsigned run = offs[(int64_t)d * n_blocks + blockIdx.x];
        for (int w = 0; w < kWarpsPerBlock; ++w) {
            const unsigned c = wcount[w][d];
            wcount[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int q0 = 0; q0 < kPerWarp; q0 += 32) {
        const int64_t i = base + q0 + lane;
        const bool ok = i < n;
        const unsigned long long k = ok ? kin[i] : 0ull;
        const unsigned d = ok ? ((unsigned)(k >> shift) & (kRadix - 1)) : kRadix;  // kRadix: none
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        const int leader = __ffs(peers) - 1;
        unsigned start = 0;
        if (ok && lane == leader) start = wcount[warp][d];
        start = __shfl_sync(0xffffffffu, start, leader);
        if (ok) {
            kout[start + rank] = k;
            vout[start + rank] = vin[i];
        }
        __syncwarp();
        if (ok && lane == leader) wcount[warp][d] = start + __popc(peers);
        __syncwarp();
    }
}

constexpr int kScanThreads = 512;
constexpr int kScanItems = 2 * kScanThreads;  // items per block

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
block_scan_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n, T* __restrict__ sums) {
    __shared__ T s[kScanItems];
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    for (int q = threadIdx.x; q < kScanItems; q += kScanThreads)
        s[q] = base + q < n ? in[base + q] : T(0);
    __syncthreads();
    // up-sweep
    for (int off = 1; off < kScanItems; off <<= 1) {
        const int idx = (threadIdx.x + 1) * off * 2 - 1;
        if (idx < kScanItems) s[idx] += s[idx - off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (sums) sums[blockIdx.x] = s[kScanItems - 1];
        s[kScanItems - 1] = T(0);
    }
    __syncthreads();
    // down-sweep
    for (int off = kScanItems / 2; off >= 1; off >>= 1) {
        const int idx = (threadIdx.x + 1) * off * 2 - 1;
        if (idx < kScanItems) {
            const T t = s[idx - off];
            s[idx - off] = s[idx];
            s[idx] += t;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < kScanItems; q += kScanThreads)
        if (base + q < n) out[base + q] = s[q];
}

template <typename T>
__global__ void add_block_offsets_kernel(T* __restrict__ out, int64_t n, const T* __restrict__ offs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanItems];
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename T>
size_t scan_temp_bytes_t(int64_t n) {
    size_t bytes = 0;
    while (n > kScanItems) {
        n = ceil_div(n, kScanItems);
        bytes += ((size_t)n * sizeof(T) + 255) / 256 * 256;
    }
    return bytes;
}

template <typename T>
cudaError_t exclusive_scan_t(const T* in, T* out, int64_t n, void* temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = ceil_div(n, kScanItems);
    if (nb == 1) {
        block_scan_kernel<T><<<1, kScanThreads, 0, s>>>(in, out, n, (T*)nullptr);
        return cudaGetLastError();
    }
    T* sums = static_cast<T*>(temp);
    char* rest = static_cast<char*>(temp) + ((size_t)nb * sizeof(T) + 255) / 256 * 256;
    block_scan_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_t<T>(sums, sums, nb, rest, s);
    if (e != cudaSuccess) return e;
    add_block_offsets_kernel<T><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

}  // namespace

size_t mbm_scan_temp_bytes_i32(int64_t n) { return scan_temp_bytes_t<int>(n); }
size_t mbm_scan_temp_bytes_i64(int64_t n) { return scan_temp_bytes_t<long long>(n); }

cudaError_t mbm_exclusive_scan_i32(const int* in, int* out, int64_t n, void* temp, cudaStream_t s) {
    return exclusive_scan_t<int>(in, out, n, temp, s);
}

cudaError_t mbm_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp,
                                   cudaStream_t s) {
    return exclusive_scan_t<long long>(reinterpret_cast<const long long*>(in),
                                       reinterpret_cast<long long*>(out), n, temp, s);
}

size_t mbm_sort_temp_bytes(int64_t n) {
    const int64_t nb = ceil_div(n > 0 ? n : 1, kTileItems);
    const size_t hist = (size_t)kRadix * nb;
    size_t b = ((size_t)n * 8 + 255) / 256 * 256 + ((size_t)n * 4 + 255) / 256 * 256;  // ping-pong
    b += 2 * ((hist * sizeof(unsigned) + 255) / 256 * 256);                            // counts, offsets
    b += scan_temp_bytes_t<int>((int64_t)hist);
    return b;
}

cudaError_t mbm_sort_pairs_u64(const unsigned long long* keys_in, unsigned long long* keys_out,
                               const int* vals_in, int* vals_out, int64_t n, int bit0, int bit1,
                               void* temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = ceil_div(n, kTileItems);
    const size_t hist = (size_t)kRadix * nb;
    char* t = static_cast<char*>(temp);
    auto* k_alt = reinterpret_cast<unsigned long long*>(t);
    t += ((size_t)n * 8 + 255) / 256 * 256;
    auto* v_alt = reinterpret_cast<int*>(t);
    t += ((size_t)n * 4 + 255) / 256 * 256;
    auto* counts = reinterpret_cast<unsigned*>(t);
    t += (hist * sizeof(unsigned) + 255) / 256 * 256;
    auto* offs = reinterpret_cast<unsigned*>(t);
    t += (hist * sizeof(unsigned) + 255) / 256 * 256;
    void* scan_tmp = t;
    const int passes = bit1 > bit0 ? (bit1 - bit0 + 7) / 8 : 0;
    if (passes == 0) {
        cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals_out, vals_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        return e;
    }
    // The last pass must write keys_out: start from the buffer that makes it so.
    const unsigned long long* src_k = keys_in;
    const int* src_v = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        unsigned long long* dk = to_out ? keys_out : k_alt;
        int* dv = to_out ? vals_out : v_alt;
        const int shift = bit0 + 8 * p;
        digit_hist_kernel<<<(unsigned)nb, kThreads, 0, s>>>(src_k, n, shift, counts, (int)nb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = exclusive_scan_t<int>(reinterpret_cast<const int*>(counts), reinterpret_cast<int*>(offs),
                                  (int64_t)hist, scan_tmp, s);
        if (e != cudaSuccess) return e;
        digit_scatter_kernel<<<(unsigned)nb, kThreads, 0, s>>>(src_k, src_v, dk, dv, n, shift, offs,
                                                               (int)nb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        src_k = dk;
        src_v = dv;
    }
    return cudaSuccess;
}
