// Small device utilities: scans, bitonic sort, warp helpers, SplitMix64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qh {

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output n of the stream with
// initial state `key` is mix(key + (n + 1) * 0x9E3779B97F4A7C15).
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_out(uint64_t key, uint64_t n) {
  return sm64_mix(key + (n + 1) * 0x9E3779B97F4A7C15ULL);
}
// Initial bSB draw on [-0.1, 0.1]: 24-bit uniform from the top bits, scaled in
// FP64 and rounded once to FP32.
__device__ __forceinline__ float init_draw(uint64_t key, int32_t replica, int32_t node,
                                           int which) {
  uint64_t v = sm64_out(key, ((((uint64_t)(uint32_t)replica) << 24) | (uint64_t)(uint32_t)node) *
                                     2ull + (uint64_t)which);
  double u = (double)(v >> 40) * (1.0 / 16777216.0);
  return (float)(u * 0.2 - 0.1);
}
__host__ __device__ __forceinline__ uint64_t init_key(uint64_t seed, int32_t block, int32_t iter) {
  return sm64_out(seed, (((uint64_t)(uint32_t)block) << 16) | (uint64_t)(uint32_t)iter);
}

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
