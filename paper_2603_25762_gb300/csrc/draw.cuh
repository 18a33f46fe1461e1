// Seeded draws of the bSB initial state, shared by host and device code.
//
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) gives a 64-bit word per (key, n); the
// top 24 bits m make a uniform u = m / 2^24 on [0, 1), and the initial value is the
// FP64 expression u * 0.2 - 0.1 rounded once to FP32. That FP64 expression is
// evaluated here in integer arithmetic, bit for bit: GB300 runs FP64 at a small
// fraction of its integer rate, and the initial-state kernel writes two draws per
// vertex and replica. Plain C++ (no CUDA types), so a host compiler checks it against
// the FP64 expression over all 2^24 values of m.
#pragma once

#include <stdint.h>
#include <string.h>

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

QH_DRAW_FN int draw_bitlen64(uint64_t v) {  // position of the highest set bit + 1; 0 for 0
  int n = 0;
  if (v >> 32) { v >>= 32; n += 32; }
  if (v >> 16) { v >>= 16; n += 16; }
  if (v >> 8) { v >>= 8; n += 8; }
  if (v >> 4) { v >>= 4; n += 4; }
  if (v >> 2) { v >>= 2; n += 2; }
  if (v >> 1) { v >>= 1; n += 1; }
  return n + (int)v;
}

// (float)((double)m / 2^24 * 0.2 - 0.1) for 0 <= m < 2^24, without FP64.
//
// The doubles 0.1 and 0.2 share their significand M = 0x1999999999999A (0.2 = M * 2^-55,
// 0.1 = M * 2^-56), so the exact value of u * 0.2 - 0.1 is k * M * 2^-79 with
// k = m - 2^23, and the FP64 evaluation rounds that product to 53 significant bits
// (once with a fused multiply-add, or twice without: the two give the same FP32 result
// for every m). The FP32 result is that double rounded to 24 bits, both roundings to
// nearest, ties to even. |k| * M < 2^76, and every nonzero result lies between 2^-27
// and 0.1, inside FP32's normal range.
QH_DRAW_FN float init_scale_u24(uint32_t m) {
  const int32_t k = (int32_t)m - (1 << 23);
  if (k == 0) return 0.f;
  const uint64_t a = (uint64_t)(k < 0 ? -k : k);
  const uint64_t M = 0x1999999999999AULL;
  // P = a * M as hi:lo (a < 2^24, M < 2^53).
  const uint64_t t1 = a * (M >> 32), t0 = a * (M & 0xFFFFFFFFULL);
  const uint64_t lo = t0 + (t1 << 32);
  const uint64_t hi = (t1 >> 32) + (lo < t0 ? 1u : 0u);
  const int len = hi != 0 ? 64 + draw_bitlen64(hi) : draw_bitlen64(lo);
  // Round P to 53 bits: q * 2^s. The dropped bits (s <= 23) all lie in lo.
  int s = len > 53 ? len - 53 : 0;
  uint64_t q = lo, rem = 0, half = 0;
  if (s > 0) {
    q = (lo >> s) | (hi << (64 - s));
    rem = lo & ((1ULL << s) - 1);
    half = 1ULL << (s - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q >> 53) { q >>= 1; ++s; }
  }
  // Round q to 24 bits: q2 * 2^(s + s2).
  const int qlen = draw_bitlen64(q);
  int s2 = qlen > 24 ? qlen - 24 : 0;
  uint64_t q2 = q;
  if (s2 > 0) {
    q2 = q >> s2;
    rem = q & ((1ULL << s2) - 1);
    half = 1ULL << (s2 - 1);
    if (rem > half || (rem == half && (q2 & 1))) ++q2;
    if (q2 >> 24) { q2 >>= 1; ++s2; }
  }
  // q2 * 2^(s + s2 - 79) as FP32 bits; q2 has its top bit at 2^(len2 - 1).
  const int len2 = draw_bitlen64(q2);
  const int e = s + s2 - 79 + len2 - 1;  // unbiased exponent of the result
  const uint32_t mant = (uint32_t)((q2 << (24 - len2)) & 0x7FFFFFu);
  const uint32_t bits = (k < 0 ? 0x80000000u : 0u) | ((uint32_t)(e + 127) << 23) | mant;
  float f;
  memcpy(&f, &bits, sizeof f);
  return f;
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
