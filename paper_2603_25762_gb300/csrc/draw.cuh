// Seeded draws of the bSB initial state, shared by host and device code.
//
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) gives a 64-bit word per (key, n); the
// top 24 bits m make a uniform u = m / 2^24 on [0, 1), and the initial value is the
// FP64 expression u * 0.2 - 0.1 rounded once to FP32. That result is obtained here
// with two FP32 operations, bit for bit: GB300 runs FP64 at a small fraction of its
// FP32 rate, and the initial-state kernel writes two draws per vertex and replica.
// Plain C++ (no CUDA types), so a host compiler checks it against the FP64 expression
// over all 2^24 values of m.
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define QH_DRAW_FN __host__ __device__ __forceinline__
#else
#define QH_DRAW_FN static inline
#endif

namespace qh {

// Output n of the SplitMix64 stream with initial state `key`:
// mix(key + (n + 1) * 0x9E3779B97F4A7C15).
QH_DRAW_FN uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
QH_DRAW_FN uint64_t sm64_out(uint64_t key, uint64_t n) {
  return sm64_mix(key + (n + 1) * 0x9E3779B97F4A7C15ULL);
}

// (float)((double)m / 2^24 * 0.2 - 0.1) for 0 <= m < 2^24, without FP64.
//
// The doubles 0.1 and 0.2 share their significand, so the exact value of the FP64
// expression before its roundings is k * 0.2 * 2^-24 with k = m - 2^23 (|k| <= 2^23,
// exact in FP32). With 0.2 = H + L, H the FP32 nearest to the double 0.2 and L the FP32
// nearest to the rest, the fused k * H + fl(k * L), rounded once, then scaled by 2^-24
// (exact: every nonzero result is a normal FP32 above 2^-27), gives the FP64
// expression's FP32 result for every one of the 2^24 values of m. That is an exhaustive
// check of this function against the expression, not a bound: a host test repeats it.
QH_DRAW_FN float init_scale_u24(uint32_t m) {
  const float k = (float)((int32_t)m - (1 << 23));
  const float H = 0x1.99999ap-3f, L = -0x1.99999ap-29f;
  return fmaf(k, H, k * L) * 0x1p-24f;
}

// Initial bSB draw on [-0.1, 0.1): the 24-bit uniform from the top bits of SplitMix64
// output 2 * ((replica << 24) | node) + which of the block's key.
QH_DRAW_FN float init_draw(uint64_t key, int32_t replica, int32_t node, int which) {
  const uint64_t v = sm64_out(key, ((((uint64_t)(uint32_t)replica) << 24) |
                                    (uint64_t)(uint32_t)node) * 2ull + (uint64_t)which);
  return init_scale_u24((uint32_t)(v >> 40));
}
QH_DRAW_FN uint64_t init_key(uint64_t seed, int32_t block, int32_t iter) {
  return sm64_out(seed, (((uint64_t)(uint32_t)block) << 16) | (uint64_t)(uint32_t)iter);
}

}  // namespace qh
