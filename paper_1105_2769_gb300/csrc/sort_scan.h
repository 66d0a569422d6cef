// Radix sort of (64-bit key, 32-bit value) pairs and exclusive prefix sums
// (sort_scan.cu): the device sorting and scanning of the tree path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Temporary bytes of mbm_sort_pairs_u64 for n items.
size_t mbm_sort_temp_bytes(int64_t n);
// Stable sort of (keys_in, vals_in) by key bits [bit0, bit1) into
// (keys_out, vals_out); the inputs are not modified.
cudaError_t mbm_sort_pairs_u64(const unsigned long long* keys_in, unsigned long long* keys_out,
                               const int* vals_in, int* vals_out, int64_t n, int bit0, int bit1,
                               void* temp, cudaStream_t s);

// Exclusive prefix sums (out may equal in) and their temporary bytes.
size_t mbm_scan_temp_bytes_i32(int64_t n);
size_t mbm_scan_temp_bytes_i64(int64_t n);
cudaError_t mbm_exclusive_scan_i32(const int* in, int* out, int64_t n, void* temp, cudaStream_t s);
cudaError_t mbm_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp,
                                   cudaStream_t s);
