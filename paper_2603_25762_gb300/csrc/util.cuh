// Small device utilities: scans, bitonic sort, warp helpers; the SplitMix64 draws
// come from draw.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "draw.cuh"

namespace qh {

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---- host-callable launch helpers (util.cu)
struct Ctx;
// Exclusive scan of int64 counts (n elements) -> out (n+1 elements, out[n] = total).
// Scratch for the tile totals comes from the context; false when it cannot be had.
bool scan_i64(Ctx* ctx, cudaStream_t s, const int64_t* in, int64_t* out, int64_t n);
bool scan_i32_to_i64(Ctx* ctx, cudaStream_t s, const int32_t* in, int64_t* out, int64_t n);
// Inclusive running maximum of int32.
bool scan_max_i32(Ctx* ctx, cudaStream_t s, const int32_t* in, int32_t* out, int64_t n);
// Sort n uint64 keys ascending in place; buffer must hold next_pow2(n) keys.
void sort_u64(cudaStream_t s, uint64_t* keys, int64_t n, int64_t cap);
int64_t next_pow2(int64_t n);

}  // namespace qh
