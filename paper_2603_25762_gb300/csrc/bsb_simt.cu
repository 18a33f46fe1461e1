// SIMT kernels of the bSB solve and the phasing step:
//  - initial state (SplitMix64 draws), FP32 tiled J x X step (the plain FP32
//    GPU bSB), exact cut evaluation, replica selection, early stop,
//  - SNP refinement (flip counter, sign inversion), read voting, parity swap.
#include <algorithm>
#include <type_traits>

#include "qh_internal.cuh"
#include "util.cuh"

namespace qh {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ init
__global__ void k_init_state(const RowTile* __restrict__ rt, const int32_t* __restrict__ pad_node,
                             const int32_t* __restrict__ local, int32_t n_pad, int32_t R,
                             int32_t replica_base, uint64_t seed, int32_t iter, float* x, float* y,
                             __nv_bfloat16* xh, const int32_t* __restrict__ active, int32_t sb) {
  int32_t col = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t r = blockIdx.y;
  if (col >= n_pad || r >= R) return;
  int32_t b = rt[col / TILE].block;
  if (active != nullptr && !active[b]) return;
  int32_t v = pad_node[col];
  float xv = 0.f, yv = 0.f;
  if (v >= 0) {
    uint64_t key = init_key(seed, b, iter);
    xv = init_draw(key, replica_base + r, local[v], 0);
    yv = init_draw(key, replica_base + r, local[v], 1);
  }
  size_t idx = (size_t)r * n_pad + col;
  x[idx] = xv;
  y[idx] = yv;
  if (xh != nullptr) xh[idx] = __float2bfloat16_rn(v >= 0 ? sb_operand(sb, xv) : 0.f);
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, __nv_bfloat16* xh, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) xh[i] = __float2bfloat16_rn(x[i]);
}

// Product operand of a discrete-SB state: sgn(x) at real vertices, 0 at padding.
// State layout [R][n_pad] (r_vm = 0) or vertex-major [n_pad][r_vm].
__global__ void k_x_to_sign_bf16(const float* __restrict__ x, __nv_bfloat16* xh, int64_t n,
                                 int32_t n_pad, int32_t r_vm, const int32_t* __restrict__ pad_node) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t col = r_vm > 0 ? i / r_vm : i % n_pad;
  xh[i] = __float2bfloat16_rn(pad_node[col] >= 0 ? sb_operand(QH_SB_DISCRETE, x[i]) : 0.f);
}

// ------------------------------------------------------------------ FP32 step
constexpr int F_RT = 64;   // replicas per CTA
constexpr int F_KC = 32;   // K chunk staged in shared memory

__global__ void __launch_bounds__(256) k_step_f32(StepArgs a) {
  const int32_t t = a.t;
  const double a0d = a.a0;
  __shared__ __align__(16) float Js[F_KC][TILE + 4];
  __shared__ __align__(16) float Xs[F_KC][F_RT + 4];
  const RowTile rt = a.rt[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, wg = tid >> 5;
  const int32_t r0 = blockIdx.y * F_RT;
  const int32_t sb = a.steps_b[rt.block];
  const bool live = (a.active == nullptr || a.active[rt.block]) && t < sb;
  if (!live) {
    if (a.z_out == nullptr && a.xout != a.xin) {  // carry a frozen block to the next buffer
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) {
          int32_t row = lane + 32 * i, r = r0 + wg * 8 + j;
          if (row < rt.valid && r < a.R) {
            size_t idx = (size_t)r * a.n_pad + rt.row0 + row;
            a.xout[idx] = a.xin[idx];
          }
        }
    }
    return;
  }
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int32_t e = 0; e < rt.n_hi; ++e) {
    const float* Jt = a.tile_f32 + (size_t)(rt.f32_begin + e) * (TILE * TILE);
    const int32_t cbase = a.tile_col[rt.tile_begin + e] * TILE;
    for (int kc = 0; kc < TILE; kc += F_KC) {
      for (int idx = tid; idx < TILE * (F_KC / 4); idx += 256) {
        int row = idx / (F_KC / 4), k4 = idx % (F_KC / 4);
        float4 v = *reinterpret_cast<const float4*>(Jt + (size_t)row * TILE + kc + k4 * 4);
        Js[k4 * 4 + 0][row] = v.x;
        Js[k4 * 4 + 1][row] = v.y;
        Js[k4 * 4 + 2][row] = v.z;
        Js[k4 * 4 + 3][row] = v.w;
      }
      for (int idx = tid; idx < F_RT * (F_KC / 4); idx += 256) {
        int rep = idx / (F_KC / 4), k4 = idx % (F_KC / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + rep < a.R)
          v = *reinterpret_cast<const float4*>(a.xin + (size_t)(r0 + rep) * a.n_pad + cbase + kc +
                                               k4 * 4);
        if (a.sb == QH_SB_DISCRETE)  // J sgn(x); padding columns meet zero columns of J
          v = make_float4(sb_operand(a.sb, v.x), sb_operand(a.sb, v.y), sb_operand(a.sb, v.z),
                          sb_operand(a.sb, v.w));
        Xs[k4 * 4 + 0][rep] = v.x;
        Xs[k4 * 4 + 1][rep] = v.y;
        Xs[k4 * 4 + 2][rep] = v.z;
        Xs[k4 * 4 + 3][rep] = v.w;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < F_KC; ++k) {
        float av[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = Js[k][lane + 32 * i];
        float4 b0 = *reinterpret_cast<const float4*>(&Xs[k][wg * 8]);
        float4 b1 = *reinterpret_cast<const float4*>(&Xs[k][wg * 8 + 4]);
        float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  const double at = a0d * (double)t / (double)sb;
  const float coef_x = (float)(-(a0d - at));
  const float c0 = a.c0[rt.block];
  const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int32_t row = lane + 32 * i, r = r0 + wg * 8 + j;
      if (row >= rt.valid || r >= a.R) continue;
      size_t idx = (size_t)r * a.n_pad + rt.row0 + row;
      if (a.z_out != nullptr) {
        a.z_out[idx] = acc[i][j];
        continue;
      }
      float x = a.xin[idx], y = a.y[idx];
      sb_update(a.sb, acc[i][j], x, y, a.dt, coef_x, a.dta0, c0, fe);
      a.xout[idx] = x;
      a.y[idx] = y;
    }
}

// ------------------------------------------------------------------ CSR storage
// CSR step CTAs: 2 vertices (warps) each, 32 warps per SM at 64 registers.  Vertices
// of one CTA differ in degree and the CTA's slot frees with its slowest warp, so small
// CTAs keep more warps resident (measured faster than 4- and 8-warp CTAs).
#ifndef CSR_CTA
#define CSR_CTA 64
#endif
// The discrete-SB operand of four gathered values.
__device__ __forceinline__ float4 sgn4(float4 v) {
  return make_float4(sb_operand(QH_SB_DISCRETE, v.x), sb_operand(QH_SB_DISCRETE, v.y),
                     sb_operand(QH_SB_DISCRETE, v.z), sb_operand(QH_SB_DISCRETE, v.w));
}

// Vertex-major state ([n_pad][R]): initial draws, thread per (vertex, replica).
__global__ void k_init_state_vm(const RowTile* __restrict__ rt, const int32_t* __restrict__ pad_node,
                                const int32_t* __restrict__ local, int32_t n_pad, int32_t R,
                                int32_t replica_base, uint64_t seed, int32_t iter, float* x,
                                float* y, __nv_bfloat16* xh, const int32_t* __restrict__ active,
                                int32_t sb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_pad * R) return;
  const int32_t col = (int32_t)(i / R), r = (int32_t)(i % R);
  const int32_t b = rt[col / TILE].block;
  if (active != nullptr && !active[b]) return;
  const int32_t v = pad_node[col];
  float xv = 0.f, yv = 0.f;
  if (v >= 0) {
    uint64_t key = init_key(seed, b, iter);
    xv = init_draw(key, replica_base + r, local[v], 0);
    yv = init_draw(key, replica_base + r, local[v], 1);
  }
  x[i] = xv;
  y[i] = yv;
  if (xh != nullptr) xh[i] = __float2bfloat16_rn(v >= 0 ? sb_operand(sb, xv) : 0.f);
}

__global__ void k_signs_vm(const float* __restrict__ x, int64_t n, int8_t* st) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) st[i] = x[i] >= 0.f ? 1 : -1;
}

// One bSB step on CSR storage: warp per padded vertex; lane l owns replicas
// 4l .. 4l+3 of every 128-replica chunk.  The row's (column, J) pairs are read 32 at
// a time and broadcast by shuffle; each neighbour costs one 8-byte (BF16) or 16-byte
// (FP32) load per lane, i.e. a contiguous replica slice per warp.
// DISC (FP32 operands only): discrete SB, the product takes sgn of each gathered x.
// BF16 operands already hold the variant's operand (sgn(x) for discrete SB).
template <bool BF16, bool DISC>
__global__ void __launch_bounds__(CSR_CTA, 1024 / CSR_CTA) k_step_csr(StepArgs a, const int64_t* __restrict__ prow,
                                                  const int32_t* __restrict__ pcol,
                                                  const float* __restrict__ pval,
                                                  const __nv_bfloat16* __restrict__ xh_in) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= a.n_pad) return;
  const RowTile rt = a.rt[row / TILE];
  const int32_t sb = a.steps_b[rt.block];
  const bool live = (a.active == nullptr || a.active[rt.block]) && a.t < sb;
  if (row - rt.row0 >= rt.valid) return;  // padding vertex: state stays zero
  const size_t rbase = (size_t)row * a.R;
  if (!live) {
    if (!BF16 && a.z_out == nullptr && a.xout != a.xin)  // carry a frozen block forward
      for (int32_t r = 4 * lane; r < a.R; r += 128)
        *reinterpret_cast<float4*>(a.xout + rbase + r) =
            *reinterpret_cast<const float4*>(a.xin + rbase + r);
    return;
  }
  const int64_t e0 = prow[row], e1 = prow[row + 1];
  const double at = a.a0 * (double)a.t / (double)sb;
  const float coef_x = (float)(-(a.a0 - at));
  const float c0 = a.c0[rt.block];
  const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
  for (int32_t r0 = 0; r0 < a.R; r0 += 128) {
    const int32_t r = r0 + 4 * lane;
    const bool on = r < a.R;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (a.zb != nullptr && on) {  // the band product, from the tensor cores
      const float4 z0 = *reinterpret_cast<const float4*>(a.zb + rbase + r);
      acc[0] = z0.x;
      acc[1] = z0.y;
      acc[2] = z0.z;
      acc[3] = z0.w;
    }
    // the next 32-edge group's columns and weights load while this group's gathers
    // are in flight (they stream from DRAM); lanes past the row's end hold column 0 and
    // J = 0: a valid address contributing nothing
    int32_t cl_n = e0 + lane < e1 ? pcol[e0 + lane] : 0;
    float vl_n = e0 + lane < e1 ? pval[e0 + lane] : 0.f;
    for (int64_t e = e0; e < e1; e += 32) {
      const int ne = (e1 - e) < 32 ? (int)(e1 - e) : 32;
      const int32_t cl = cl_n;
      const float vl = vl_n;
      cl_n = e + 32 + lane < e1 ? pcol[e + 32 + lane] : 0;
      vl_n = e + 32 + lane < e1 ? pval[e + 32 + lane] : 0.f;
      // NB neighbours per batch, all loads issued before the first FMA: the step is
      // bound by the latency of these gathers (16 per batch measured slower than 8)
      constexpr int NB = 8;
#pragma unroll
      for (int k = 0; k < 32; k += NB) {
        if (k >= ne) break;
        int32_t cc[NB];
        float jv[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          cc[q] = __shfl_sync(0xffffffffu, cl, k + q);
          jv[q] = __shfl_sync(0xffffffffu, vl, k + q);
        }
        if (!on) continue;
        if (BF16) {
          uint2 u[NB];
#pragma unroll
          for (int q = 0; q < NB; ++q)
            u[q] = *reinterpret_cast<const uint2*>(xh_in + (size_t)cc[q] * a.R + r);
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&u[q].x);
            const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&u[q].y);
            acc[0] = fmaf(jv[q], __low2float(lo), acc[0]);
            acc[1] = fmaf(jv[q], __high2float(lo), acc[1]);
            acc[2] = fmaf(jv[q], __low2float(hi), acc[2]);
            acc[3] = fmaf(jv[q], __high2float(hi), acc[3]);
          }
        } else {
          float4 xv[NB];
#pragma unroll
          for (int q = 0; q < NB; ++q)
            xv[q] = *reinterpret_cast<const float4*>(a.xin + (size_t)cc[q] * a.R + r);
          if (DISC)
#pragma unroll
            for (int q = 0; q < NB; ++q) xv[q] = sgn4(xv[q]);
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            acc[0] = fmaf(jv[q], xv[q].x, acc[0]);
            acc[1] = fmaf(jv[q], xv[q].y, acc[1]);
            acc[2] = fmaf(jv[q], xv[q].z, acc[2]);
            acc[3] = fmaf(jv[q], xv[q].w, acc[3]);
          }
        }
      }
    }
    if (!on) continue;
    const size_t idx = rbase + r;
    if (a.z_out != nullptr) {
      *reinterpret_cast<float4*>(a.z_out + idx) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      continue;
    }
    const float* xsrc = BF16 ? a.x : a.xin;
    float4 xv = *reinterpret_cast<const float4*>(xsrc + idx);
    float4 yv = *reinterpret_cast<const float4*>(a.y + idx);
    float xs[4] = {xv.x, xv.y, xv.z, xv.w}, ys[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) sb_update(a.sb, acc[j], xs[j], ys[j], a.dt, coef_x, a.dta0, c0, fe);
    float* xdst = BF16 ? a.x : a.xout;
    *reinterpret_cast<float4*>(xdst + idx) = make_float4(xs[0], xs[1], xs[2], xs[3]);
    *reinterpret_cast<float4*>(a.y + idx) = make_float4(ys[0], ys[1], ys[2], ys[3]);
    if (BF16) {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(sb_operand(a.sb, xs[0]), sb_operand(a.sb, xs[1]));
      __nv_bfloat162 p1 = __floats2bfloat162_rn(sb_operand(a.sb, xs[2]), sb_operand(a.sb, xs[3]));
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&p0);
      u.y = *reinterpret_cast<uint32_t*>(&p1);
      *reinterpret_cast<uint2*>(a.xh_out + idx) = u;
    }
  }
}

// The CSR step for R a multiple of 8: each lane owns 8 consecutive replicas (one
// 16-byte X_hat load per neighbour for BF16 operands, two for FP32), L = 32 / P lanes
// cover one neighbour's replica row, and the warp walks P neighbours of its vertex at
// once (P = 2 at R = 128).  The P partial sums meet in a shuffle butterfly; the lanes
// of the first neighbour stream then apply the update.  Per neighbour this costs about
// half the instructions of k_step_csr: two shuffles, one address, the loads and four
// packed FP32x2 FMAs per lane.  Both CSR kernels are bound by the latency of the
// gathers: they run at 64 registers, 32 warps per SM, a few bytes spilled in some
// instantiations, which measured faster than 24 warps without spills.
template <bool BF16, int P, bool ZB, bool DISC>
__global__ void __launch_bounds__(CSR_CTA, 1024 / CSR_CTA) k_step_csr8(StepArgs a, const int64_t* __restrict__ prow,
                                                   const int32_t* __restrict__ pcol,
                                                   const float* __restrict__ pval,
                                                   const __nv_bfloat16* __restrict__ xh_in) {
  constexpr int L = 32 / P;                 // lanes per neighbour row
  constexpr int NB0 = BF16 ? 8 : 4;
  constexpr int NB = NB0 < 32 / P ? NB0 : 32 / P;  // neighbours per lane per batch
  constexpr int STEP = P * NB;                       // edges per batch, at most 32
  static_assert(STEP <= 32 && 32 % STEP == 0, "batches tile the 32-edge group");
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int sub = lane / L, li = lane % L;
  if (row >= a.n_pad) return;
  const RowTile rt = a.rt[row / TILE];
  const int32_t sb = a.steps_b[rt.block];
  const bool live = (a.active == nullptr || a.active[rt.block]) && a.t < sb;
  if (row - rt.row0 >= rt.valid) return;  // padding vertex: state stays zero
  const size_t rbase = (size_t)row * a.R;
  if (!live) {
    if (!BF16 && a.z_out == nullptr && a.xout != a.xin)  // carry a frozen block forward
      for (int32_t r = 4 * lane; r < a.R; r += 128)
        *reinterpret_cast<float4*>(a.xout + rbase + r) =
            *reinterpret_cast<const float4*>(a.xin + rbase + r);
    return;
  }
  const int64_t e0 = prow[row], e1 = prow[row + 1];
  for (int32_t r0 = 0; r0 < a.R; r0 += 8 * L) {
    const int32_t r = r0 + 8 * li;
    const bool on = r < a.R;
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    if (ZB && on && sub == 0) {  // the band product, from the tensor cores
      const float4 z0 = *reinterpret_cast<const float4*>(a.zb + rbase + r);
      const float4 z1 = *reinterpret_cast<const float4*>(a.zb + rbase + r + 4);
      acc[0] = make_float2(z0.x, z0.y);
      acc[1] = make_float2(z0.z, z0.w);
      acc[2] = make_float2(z1.x, z1.y);
      acc[3] = make_float2(z1.z, z1.w);
    }
    // next group's columns and weights prefetched as in k_step_csr
    int32_t cl_n = e0 + lane < e1 ? pcol[e0 + lane] : 0;
    float vl_n = e0 + lane < e1 ? pval[e0 + lane] : 0.f;
    for (int64_t e = e0; e < e1; e += 32) {
      const int ne = (e1 - e) < 32 ? (int)(e1 - e) : 32;
      const int32_t cl = cl_n;
      const float vl = vl_n;
      cl_n = e + 32 + lane < e1 ? pcol[e + 32 + lane] : 0;
      vl_n = e + 32 + lane < e1 ? pval[e + 32 + lane] : 0.f;
#pragma unroll
      for (int k = 0; k < 32; k += STEP) {
        if (k >= ne) break;
        int32_t cc[NB];
        float jv[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int src = k + q * P + sub;  // < 32: STEP divides 32
          cc[q] = __shfl_sync(0xffffffffu, cl, src);
          jv[q] = __shfl_sync(0xffffffffu, vl, src);
        }
        if (!on) continue;
        if (BF16) {
          uint4 u[NB];
#pragma unroll
          for (int q = 0; q < NB; ++q)
            u[q] = *reinterpret_cast<const uint4*>(xh_in + (size_t)cc[q] * a.R + r);
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            const float2 j2 = make_float2(jv[q], jv[q]);
            const uint32_t w[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
#pragma unroll
            for (int j = 0; j < 4; ++j)  // BF16 pair -> two FP32 values, exactly
              acc[j] = __ffma2_rn(j2, make_float2(__uint_as_float(w[j] << 16),
                                                  __uint_as_float(w[j] & 0xffff0000u)), acc[j]);
          }
        } else {
          float4 xv[NB][2];
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            const float4* src4 = reinterpret_cast<const float4*>(a.xin + (size_t)cc[q] * a.R + r);
            xv[q][0] = DISC ? sgn4(src4[0]) : src4[0];
            xv[q][1] = DISC ? sgn4(src4[1]) : src4[1];
          }
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            const float2 j2 = make_float2(jv[q], jv[q]);
            acc[0] = __ffma2_rn(j2, make_float2(xv[q][0].x, xv[q][0].y), acc[0]);
            acc[1] = __ffma2_rn(j2, make_float2(xv[q][0].z, xv[q][0].w), acc[1]);
            acc[2] = __ffma2_rn(j2, make_float2(xv[q][1].x, xv[q][1].y), acc[2]);
            acc[3] = __ffma2_rn(j2, make_float2(xv[q][1].z, xv[q][1].w), acc[3]);
          }
        }
      }
    }
    // the P neighbour streams of the same replicas meet
#pragma unroll
    for (int off = 16; off >= L; off >>= 1)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, off);
        acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, off);
      }
    if (!on || sub != 0) continue;
    const size_t idx = rbase + r;
    float zs[8] = {acc[0].x, acc[0].y, acc[1].x, acc[1].y, acc[2].x, acc[2].y, acc[3].x, acc[3].y};
    if (a.z_out != nullptr) {
      *reinterpret_cast<float4*>(a.z_out + idx) = make_float4(zs[0], zs[1], zs[2], zs[3]);
      *reinterpret_cast<float4*>(a.z_out + idx + 4) = make_float4(zs[4], zs[5], zs[6], zs[7]);
      continue;
    }
    // the update's constants, taken after the gathers (fewer live registers there)
    const double at = a.a0 * (double)a.t / (double)sb;
    const float coef_x = (float)(-(a.a0 - at));
    const float c0 = a.c0[rt.block];
    const float fe = deform_force(a.deform, rt.block, a.t, sb);
    const float* xsrc = BF16 ? a.x : a.xin;
    float xs[8], ys[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4 xv = *reinterpret_cast<const float4*>(xsrc + idx + 4 * h);
      const float4 yv = *reinterpret_cast<const float4*>(a.y + idx + 4 * h);
      xs[4 * h] = xv.x; xs[4 * h + 1] = xv.y; xs[4 * h + 2] = xv.z; xs[4 * h + 3] = xv.w;
      ys[4 * h] = yv.x; ys[4 * h + 1] = yv.y; ys[4 * h + 2] = yv.z; ys[4 * h + 3] = yv.w;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sb_update(a.sb, zs[j], xs[j], ys[j], a.dt, coef_x, a.dta0, c0, fe);
    float* xdst = BF16 ? a.x : a.xout;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      *reinterpret_cast<float4*>(xdst + idx + 4 * h) =
          make_float4(xs[4 * h], xs[4 * h + 1], xs[4 * h + 2], xs[4 * h + 3]);
      *reinterpret_cast<float4*>(a.y + idx + 4 * h) =
          make_float4(ys[4 * h], ys[4 * h + 1], ys[4 * h + 2], ys[4 * h + 3]);
    }
    if (BF16) {
      uint4 u;
      uint32_t* uw = &u.x;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 p2 =
            __floats2bfloat162_rn(sb_operand(a.sb, xs[2 * j]), sb_operand(a.sb, xs[2 * j + 1]));
        uw[j] = *reinterpret_cast<uint32_t*>(&p2);
      }
      *reinterpret_cast<uint4*>(a.xh_out + idx) = u;
    }
  }
}

__global__ void k_transpose(const float* __restrict__ in, float* out, int64_t rows, int64_t cols) {
  __shared__ float t[32][33];
  const int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    int64_t r = r0 + k, c = c0 + tx;
    if (r < rows && c < cols) t[k][tx] = in[r * cols + c];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int64_t c = c0 + k, r = r0 + tx;
    if (r < rows && c < cols) out[c * rows + r] = t[tx][k];
  }
}

// ------------------------------------------------------------------ signs / cut
// signs_t[col][r] = sgn(x[r][col]) with sgn(0) = +1, via a 32 x 32 transpose tile.
__global__ void k_signs_t(const float* __restrict__ x, int32_t n_pad, int32_t R, int8_t* st) {
  __shared__ int8_t tile[32][33];
  int32_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    int32_t r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < R && c < n_pad) ? (x[(size_t)r * n_pad + c] >= 0.f ? 1 : -1) : 1;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int32_t c = c0 + k, r = r0 + tx;
    if (c < n_pad && r < R) st[(size_t)c * R + r] = tile[tx][k];
  }
}

// Warp per vertex a: node_val[pad(a)][r] = s_a * sum_b w_ab s_b, integer weights in
// int32 (row sums stay far below 2^31).  Lane l owns `per` consecutive replicas (a
// multiple of 4, at most 32, sized so the warp spans R), so one pass over the vertex's
// edges covers up to 1,024 replicas with 4-byte sign loads.
__global__ void k_cut_nodes(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ block_of,
                            const int32_t* __restrict__ pad_index, const int8_t* __restrict__ st,
                            int32_t R, int32_t per, double* node_val,
                            const int32_t* __restrict__ active) {
  int32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0 || (active != nullptr && !active[b])) return;
  const int32_t pa = pad_index[a];
  const int64_t e0 = rp[a], e1 = rp[a + 1];
  const bool vec = (R & 3) == 0;
  for (int32_t r0 = 0; r0 < R; r0 += 32 * per) {
    const int32_t r = r0 + per * lane;
    const int nr = max(0, min(per, R - r));
    int32_t acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0;
    // edges in groups of 32: each lane loads one edge's weight and padded column (the
    // next group's while this group is summed), the warp takes them in order by shuffle
    int32_t wv_n = e0 + lane < e1 ? (int32_t)w[e0 + lane] : 0;
    int32_t pv_n = wv_n != 0 ? pad_index[col[e0 + lane]] : 0;
    for (int64_t eg = e0; eg < e1; eg += 32) {
      const int ne = e1 - eg < 32 ? (int)(e1 - eg) : 32;
      const int32_t wv = wv_n, pv = pv_n;
      const int64_t en = eg + 32 + lane;
      wv_n = en < e1 ? (int32_t)w[en] : 0;
      pv_n = wv_n != 0 ? pad_index[col[en]] : 0;
#pragma unroll 4
      for (int k = 0; k < ne; ++k) {
        const int32_t wi = __shfl_sync(0xffffffffu, wv, k);
        const int32_t p = __shfl_sync(0xffffffffu, pv, k);
        // zero edges may reach vertices outside every block: skipped before any load
        if (wi == 0 || nr <= 0) continue;
        const int8_t* sb = st + (size_t)p * R + r;
        if (vec && nr == per) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (4 * q >= per) break;
            char4 c = *reinterpret_cast<const char4*>(sb + 4 * q);
            acc[4 * q + 0] += wi * c.x;
            acc[4 * q + 1] += wi * c.y;
            acc[4 * q + 2] += wi * c.z;
            acc[4 * q + 3] += wi * c.w;
          }
        } else {
#pragma unroll
          for (int k2 = 0; k2 < 32; ++k2)
            if (k2 < nr) acc[k2] += wi * sb[k2];
        }
      }
    }
    const int8_t* sa = st + (size_t)pa * R + r;
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < nr) node_val[(size_t)pa * R + r + k] = (double)sa[k] * (double)acc[k];
  }
}

// Real weights, at most 4 replicas (the final parity cut): FP64, the lanes of the
// vertex's warp stride over its edges and the partial sums are combined in a fixed
// shuffle order, so the result does not depend on scheduling.
__global__ void k_cut_nodes_few(int32_t n, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const double* __restrict__ w,
                                const int32_t* __restrict__ block_of,
                                const int32_t* __restrict__ pad_index,
                                const int8_t* __restrict__ st, int32_t R, double* node_val,
                                const int32_t* __restrict__ active) {
  int32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0 || (active != nullptr && !active[b])) return;
  const int32_t pa = pad_index[a];
  const int64_t e0 = rp[a], e1 = rp[a + 1];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    const double we = w[e];
    if (we == 0.0) continue;  // zero edges may reach vertices outside every block
    const int8_t* sb = st + (size_t)pad_index[col[e]] * R;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < R) acc[k] += sb[k] > 0 ? we : -we;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  if (lane < R) {
    double v = acc[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
      if (lane == k) v = acc[k];
    node_val[(size_t)pa * R + lane] = (double)st[(size_t)pa * R + lane] * v;
  }
}

// Real weights over many replicas: the same per-vertex sums, accumulated in FP32 with
// compensation.  Each weight is split into FP32 hi + lo parts, and each running sum
// is kept as an unevaluated pair (hi, lo) updated with the exact rounding error of the
// hi addition (Knuth's TwoSum), which carries about 48 bits: within ~1e-11 of the FP64
// sum even over thousands of edges, at FP32 speed (this part's FP64 rate is a small
// fraction of its FP32 rate).  Signs are +-1, so the terms are exact negations.
template <int PER>
__global__ void k_cut_nodes_df(int32_t n, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ col, const double* __restrict__ w,
                               const int32_t* __restrict__ block_of,
                               const int32_t* __restrict__ pad_index, const int8_t* __restrict__ st,
                               int32_t R, int32_t per, double* node_val,
                               const int32_t* __restrict__ active) {
  int32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0 || (active != nullptr && !active[b])) return;
  const int32_t pa = pad_index[a];
  const int64_t e0 = rp[a], e1 = rp[a + 1];
  const bool vec = (R & 3) == 0;
  for (int32_t r0 = 0; r0 < R; r0 += 32 * per) {
    const int32_t r = r0 + per * lane;
    const int nr = max(0, min(per, R - r));
    float hi[PER], lo[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) hi[k] = lo[k] = 0.f;
    auto add = [&](int k, int sg, float wh, float wl) {
      const float th = sg > 0 ? wh : -wh, tl = sg > 0 ? wl : -wl;
      const float s = __fadd_rn(hi[k], th);
      const float bp = __fsub_rn(s, hi[k]);
      const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bp)), __fsub_rn(th, bp));
      hi[k] = s;
      lo[k] = __fadd_rn(lo[k], __fadd_rn(err, tl));
    };
    // edges in groups of 32, as in k_cut_nodes; the terms still go in edge order
    double wv_n = e0 + lane < e1 ? w[e0 + lane] : 0.0;
    int32_t pv_n = wv_n != 0.0 ? pad_index[col[e0 + lane]] : 0;
    for (int64_t eg = e0; eg < e1; eg += 32) {
      const int ne = e1 - eg < 32 ? (int)(e1 - eg) : 32;
      const float whv = (float)wv_n, wlv = (float)(wv_n - (double)(float)wv_n);
      const bool nzv = wv_n != 0.0;
      const int32_t pv = pv_n;
      const int64_t en = eg + 32 + lane;
      wv_n = en < e1 ? w[en] : 0.0;
      pv_n = wv_n != 0.0 ? pad_index[col[en]] : 0;
#pragma unroll 4
      for (int k = 0; k < ne; ++k) {
        const float wh = __shfl_sync(0xffffffffu, whv, k);
        const float wl = __shfl_sync(0xffffffffu, wlv, k);
        const int32_t p = __shfl_sync(0xffffffffu, pv, k);
        const bool nz = __shfl_sync(0xffffffffu, (int)nzv, k) != 0;
        // zero edges may reach vertices outside every block: skipped before any load
        if (!nz || nr <= 0) continue;
        const int8_t* sb = st + (size_t)p * R + r;
        if (vec && nr == per) {
#pragma unroll
          for (int q = 0; q < PER / 4; ++q) {
            if (4 * q >= per) break;
            const char4 c = *reinterpret_cast<const char4*>(sb + 4 * q);
            add(4 * q + 0, c.x, wh, wl);
            add(4 * q + 1, c.y, wh, wl);
            add(4 * q + 2, c.z, wh, wl);
            add(4 * q + 3, c.w, wh, wl);
          }
        } else {
#pragma unroll
          for (int k2 = 0; k2 < PER; ++k2)
            if (k2 < nr) add(k2, sb[k2], wh, wl);
        }
      }
    }
    const int8_t* sa = st + (size_t)pa * R + r;
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (k < nr) node_val[(size_t)pa * R + r + k] = (double)sa[k] * ((double)hi[k] + (double)lo[k]);
  }
}

// CTA per (block, 32 replicas): 32 vertex slices per replica summed in a fixed
// order, then the 32 slice sums in order: cut = (sum_w - s^T W s) / 4.
__global__ void __launch_bounds__(1024) k_cut_reduce(int32_t nb, const int32_t* __restrict__ pad_off,
                                                     const int64_t* __restrict__ block_ptr, int32_t R,
                                                     const double* __restrict__ node_val,
                                                     const double* __restrict__ sum_w, double* cuts,
                                                     const int32_t* __restrict__ active) {
  __shared__ double part[32][33];
  const int32_t b = blockIdx.y;
  if (active != nullptr && !active[b]) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int32_t r = blockIdx.x * 32 + tx;
  const int32_t p0 = pad_off[b];
  const int32_t sz = (int32_t)(block_ptr[b + 1] - block_ptr[b]);
  double s = 0.0;
  if (r < R)
    for (int32_t p = ty; p < sz; p += 32) s += node_val[(size_t)(p0 + p) * R + r];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && r < R) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += part[k][tx];
    cuts[(size_t)b * R + r] = 0.25 * (sum_w[b] - t);
  }
}

// Cuts from the product z = J S of the replicas' signs (tensor cores, exact for integer
// weights whose row sums of |J| stay below 2^24): cut_r = (sum W + sum_a s_a z_a) / 4
// (J = -W).  z, S in the state layout [R][n_pad].  CTA (replica group, chunk, block): a
// warp per replica, the lanes striding over the chunk's CUT_CHUNK padded columns; each
// warp's integer partial sum goes into acc[b][r] by an FP64 atomic add, exact and so
// independent of the order.  k_cut_finish then forms the cuts.
constexpr int CUT_CHUNK = 512;

__global__ void __launch_bounds__(1024) k_cut_from_product(
    const int32_t* __restrict__ pad_off, const int64_t* __restrict__ block_ptr, int32_t R,
    int32_t n_pad, const float* __restrict__ z, const __nv_bfloat16* __restrict__ s,
    double* acc, const int32_t* __restrict__ active) {
  const int32_t b = blockIdx.z;
  if (active != nullptr && !active[b]) return;
  const int32_t sz = (int32_t)(block_ptr[b + 1] - block_ptr[b]);
  const int32_t c0 = blockIdx.y * CUT_CHUNK;
  if (c0 >= sz) return;
  const int lane = threadIdx.x & 31;
  const int32_t r = blockIdx.x * 32 + (threadIdx.x >> 5);
  if (r >= R) return;
  const int32_t c1 = min(sz, c0 + CUT_CHUNK);
  const size_t row = (size_t)r * n_pad + pad_off[b];
  double t = 0.0;
  for (int32_t p = c0 + lane; p < c1; p += 32) t += (double)(__bfloat162float(s[row + p]) * z[row + p]);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) atomicAdd(acc + (size_t)b * R + r, t);
}

__global__ void k_cut_finish(int32_t nb, int32_t R, const double* __restrict__ acc,
                             const double* __restrict__ sum_w, double* cuts,
                             const int32_t* __restrict__ active) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nb * R) return;
  const int32_t b = (int32_t)(i / R);
  if (active != nullptr && !active[b]) return;
  cuts[i] = 0.25 * (sum_w[b] + acc[i]);
}

__global__ void k_pick_best(int32_t nb, int32_t R, const double* __restrict__ cuts, int32_t* best_r,
                            double* best_cut, const int32_t* __restrict__ active) {
  __shared__ double sv[256];
  __shared__ int32_t si[256];
  const int32_t b = blockIdx.x;
  if (b >= nb || (active != nullptr && !active[b])) return;
  double best = -INFINITY;
  int32_t bi = INT32_MAX;
  for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
    double c = cuts[(size_t)b * R + r];
    if (c > best) {  // r ascends per thread: ties keep the lower replica
      best = c;
      bi = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      double v2 = sv[threadIdx.x + off];
      int32_t i2 = si[threadIdx.x + off];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    best_r[b] = si[0];
    best_cut[b] = sv[0];
  }
}

// Early stop on a stalled best energy: a check after t_done steps compares the block's
// best cut over replicas with the best of its earlier checks.  Checks happen only while
// the block's own schedule has steps left (t_done < steps_b): a block whose schedule is
// shorter than the longest one is not checked after it has finished.
__global__ void k_early_stop(int32_t nb, const double* __restrict__ best_cut, double* best_seen,
                             int32_t* stall, int32_t* active, int32_t* steps_run, int32_t patience,
                             int32_t t_done, const int32_t* __restrict__ steps_b) {
  int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !active[b] || t_done >= steps_b[b]) return;
  if (best_cut[b] > best_seen[b]) {
    best_seen[b] = best_cut[b];
    stall[b] = 0;
  } else if (++stall[b] >= patience) {
    active[b] = 0;
    steps_run[b] = t_done;
  }
}

// Best during the run (track_best): after a check's pick, a running block whose best cut
// beats the kept one keeps it (cut, replica; flag = 1 to copy its spins); at the end the
// kept result replaces the final one unless the final is strictly better.
__global__ void k_track_check(int32_t nb, const double* __restrict__ best_cut,
                              const int32_t* __restrict__ best_r,
                              const int32_t* __restrict__ active, int32_t t_done,
                              const int32_t* __restrict__ steps_b, double* kept_cut,
                              int32_t* kept_r, int32_t* flag) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  flag[b] = 0;
  if (!active[b] || t_done >= steps_b[b]) return;
  if (best_cut[b] > kept_cut[b]) {  // strictly better: ties keep the earlier check
    kept_cut[b] = best_cut[b];
    kept_r[b] = best_r[b];
    flag[b] = 1;
  }
}

__global__ void k_track_final(int32_t nb, double* best_cut, int32_t* best_r,
                              const int32_t* __restrict__ active,
                              const double* __restrict__ kept_cut,
                              const int32_t* __restrict__ kept_r, int32_t* flag) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  flag[b] = 0;
  if (!active[b] || kept_r[b] < 0 || kept_cut[b] < best_cut[b]) return;
  best_cut[b] = kept_cut[b];
  best_r[b] = kept_r[b];
  flag[b] = 1;
}

__global__ void k_copy_spins(int32_t n, const int32_t* __restrict__ block_of,
                             const int32_t* __restrict__ flag, const int8_t* __restrict__ src,
                             int8_t* dst) {
  const int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int32_t b = block_of[a];
  if (b >= 0 && flag[b]) dst[a] = src[a];
}

__global__ void k_extract_spins(int32_t n, const int32_t* __restrict__ block_of,
                                const int32_t* __restrict__ pad_index, const int8_t* __restrict__ st,
                                int32_t R, const int32_t* __restrict__ best_r, int8_t* spins,
                                const int32_t* __restrict__ active) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0) {
    spins[a] = 0;
    return;
  }
  if (active != nullptr && !active[b]) return;
  spins[a] = st[(size_t)pad_index[a] * R + best_r[b]];
}

// ------------------------------------------------------------------ block sums
__global__ void k_node_sums(int32_t n, const int64_t* __restrict__ rp, const double* __restrict__ w,
                            double* sw, double* sj2) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  double s = 0.0, q = 0.0;
  for (int64_t e = rp[a]; e < rp[a + 1]; ++e) {
    s += w[e];
    q += w[e] * w[e];
  }
  sw[a] = s;
  sj2[a] = q;
}

__global__ void k_block_sums(int32_t nb, const int64_t* __restrict__ block_ptr,
                             const int32_t* __restrict__ perm, const double* __restrict__ sw,
                             const double* __restrict__ sj2, double* sum_w, double* sum_j2) {
  __shared__ double ps[256], pq[256];
  const int32_t b = blockIdx.x;
  if (b >= nb) return;
  double s = 0.0, q = 0.0;
  for (int64_t k = block_ptr[b] + threadIdx.x; k < block_ptr[b + 1]; k += blockDim.x) {
    s += sw[perm[k]];
    q += sj2[perm[k]];
  }
  ps[threadIdx.x] = s;
  pq[threadIdx.x] = q;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      ps[threadIdx.x] += ps[threadIdx.x + off];
      pq[threadIdx.x] += pq[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sum_w[b] = ps[0];
    sum_j2[b] = pq[0];
  }
}

// ------------------------------------------------------------------ SNP refinement
// Per active block: stop if the best cut is <= 0 or all spins agree; otherwise
// add 1 to C on the smaller subset (tie: the subset without the block's lowest
// vertex).  Thread per block, vertices in ascending order.
// With deformation (deform != nullptr): a failed solve (cut <= 0, or one subset empty)
// of a block with tries left keeps the block active for a re-solve with field strength
// deform_h 2^(k-1) on its k-th try, and accepts nothing (k_gauge skips blocks whose
// deform entry is nonzero); an accepted partition clears the field and the try count.
__global__ void __launch_bounds__(256) k_refine_prepare(int32_t nb, const int64_t* __restrict__ block_ptr,
                                 const int32_t* __restrict__ perm, const int8_t* __restrict__ spins,
                                 const double* __restrict__ best_cut, int32_t* active, int32_t* C,
                                 float* deform, int32_t* tries, float deform_h,
                                 int32_t deform_tries) {
  // CTA per block: count the +1 side, then flag the smaller side in parallel
  __shared__ int64_t part[256];
  __shared__ int32_t go;
  const int32_t b = blockIdx.x;
  if (b >= nb || !active[b]) return;  // CTA-uniform
  const int64_t k0 = block_ptr[b], k1 = block_ptr[b + 1];
  int64_t npos = 0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) npos += spins[perm[k]] > 0;
  part[threadIdx.x] = npos;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
    __syncthreads();
  }
  npos = part[0];
  const int64_t sz = k1 - k0;
  if (threadIdx.x == 0) {
    go = !(best_cut[b] <= 0.0 || npos == 0 || npos == sz);
    if (deform != nullptr) {
      if (go) {
        deform[b] = 0.f;
        tries[b] = 0;
      } else if (tries[b] < deform_tries) {
        tries[b] += 1;
        deform[b] = ldexpf(deform_h, tries[b] - 1);
      } else {
        deform[b] = 0.f;
        active[b] = 0;
      }
    } else if (!go) {
      active[b] = 0;
    }
  }
  __syncthreads();
  if (!go) return;
  // the smaller subset; on a tie, the subset that does not hold the lowest vertex
  const int8_t small = (2 * npos < sz) ? 1 : (2 * npos > sz) ? -1 : (int8_t)(-spins[perm[k0]]);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
    if (spins[perm[k]] == small) C[perm[k]] += 1;
}

// w'_ab = -w_ab for edges crossing the partition (s_a != s_b) of active blocks.
// Blocks waiting for a deformed re-solve (deform[b] != 0) keep their weights.
// Warp per vertex, the lanes striding over its row.  gauge (or nullptr): the product of
// the partitions that inverted each vertex's weights so far, updated with this one.
__global__ void k_gauge(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ block_of, const int8_t* __restrict__ spins,
                        double* w, const int32_t* __restrict__ active,
                        const float* __restrict__ deform, int8_t* gauge) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0 || !active[b] || (deform != nullptr && deform[b] != 0.f)) return;
  int8_t sa = spins[a];
  for (int64_t e = rp[a] + lane; e < rp[a + 1]; e += 32)
    if (spins[col[e]] != sa) w[e] = -w[e];
  if (gauge != nullptr && lane == 0) gauge[a] = (int8_t)(gauge[a] * sa);
}

// The weights under a gauge: w[e] = w0[e] g_a g_b (a resumed refinement's starting graph).
__global__ void k_apply_gauge(int32_t n, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ col, const double* __restrict__ w0,
                              const int8_t* __restrict__ gauge, double* w) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n) return;
  const int8_t ga = gauge[a];
  for (int64_t e = rp[a] + lane; e < rp[a + 1]; e += 32)
    w[e] = ga * gauge[col[e]] < 0 ? -w0[e] : w0[e];
}

// ------------------------------------------------------------------ phase
// Read voting (consistency processing), thread per SNP.
__global__ void k_vote(int32_t n, const int64_t* __restrict__ cov_ptr, const int32_t* __restrict__ cov_frag,
                       const int8_t* __restrict__ cov_allele, const int32_t* __restrict__ block_of,
                       const int8_t* __restrict__ spins, int8_t* hap1, int8_t* hap2,
                       int32_t* block_id) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t b0 = cov_ptr[j], b1 = cov_ptr[j + 1];
  // the block most of the SNP's fragments belong to (ties: the lower block); usually
  // they all belong to one, which one pass finds
  int32_t best = -1, bestc = 0;
  bool one = true;
  for (int64_t k = b0; k < b1 && one; ++k) {
    const int32_t bk = block_of[cov_frag[k]];
    if (bk < 0) continue;
    if (best < 0) best = bk;
    one = bk == best;
  }
  if (!one) {
    best = -1;
    for (int64_t k = b0; k < b1; ++k) {
      int32_t bk = block_of[cov_frag[k]];
      if (bk < 0) continue;
      int32_t c = 0;
      for (int64_t q = b0; q < b1; ++q) c += block_of[cov_frag[q]] == bk;
      if (c > bestc || (c == bestc && bk < best)) {
        bestc = c;
        best = bk;
      }
    }
  }
  int8_t h = 0;
  if (best >= 0) {
    int32_t c1p = 0, c1m = 0, c2p = 0, c2m = 0;
    for (int64_t k = b0; k < b1; ++k) {
      int32_t i = cov_frag[k];
      if (block_of[i] != best) continue;
      int8_t s = spins[i], al = cov_allele[k];
      if (s > 0) {
        if (al > 0) ++c1p; else ++c1m;
      } else if (s < 0) {
        if (al > 0) ++c2p; else ++c2m;
      }
    }
    int32_t d1 = c1p - c1m, d2 = c2p - c2m;
    if (!(c1p + c1m + c2p + c2m == 0 || (d1 == 0 && d2 == 0))) {
      if ((d1 > 0 && d2 < 0) || (d1 < 0 && d2 > 0)) {
        h = d1 > 0 ? 1 : -1;
      } else {
        int32_t a1 = d1 < 0 ? -d1 : d1, a2 = d2 < 0 ? -d2 : d2;
        if (a1 >= a2)
          h = d1 > 0 ? 1 : -1;
        else
          h = d2 > 0 ? -1 : 1;
      }
    }
  }
  hap1[j] = h;
  hap2[j] = (int8_t)(-h);
  block_id[j] = h != 0 ? best : -1;
}

__global__ void k_parity(int32_t n, const int32_t* __restrict__ block_of, const int32_t* __restrict__ C,
                         int8_t* hap1, int8_t* hap2, int32_t* block_id) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int32_t b = block_of[u];
  if (b >= 0 && C[u] < 0) b = -1;  // block not solved (partial solution): unphased
  int8_t h = b >= 0 ? ((C[u] % 2 == 0) ? 1 : -1) : 0;
  hap1[u] = h;
  hap2[u] = (int8_t)(-h);
  block_id[u] = b;
}

}  // namespace

void launch_init_state(cudaStream_t s, const Graph& g, int32_t R, int32_t replica_base,
                       uint64_t seed, int32_t iter, float* x, float* y, __nv_bfloat16* xh,
                       const int32_t* active, int32_t sb) {
  if (g.n_pad == 0 || R == 0) return;
  if (g.csr_mode) {
    const int64_t n = (int64_t)g.n_pad * R;
    k_init_state_vm<<<::qh::counted(nblk(n)), 256, 0, s>>>(g.rt, g.pad_node, g.local, g.n_pad, R,
                                                          replica_base, seed, iter, x, y, xh,
                                                          active, sb);
    return;
  }
  dim3 grid(nblk(g.n_pad), R);
  k_init_state<<<::qh::counted(grid), 256, 0, s>>>(g.rt, g.pad_node, g.local, g.n_pad, R, replica_base, seed, iter,
                                    x, y, xh, active, sb);
}

void launch_x_operand(cudaStream_t s, const Graph& g, int32_t sb, const float* x,
                      __nv_bfloat16* xh, int64_t n) {
  if (n <= 0) return;
  if (sb == QH_SB_DISCRETE)  // CSR storage keeps the state vertex-major
    k_x_to_sign_bf16<<<::qh::counted(nblk(n)), 256, 0, s>>>(
        x, xh, n, g.n_pad, g.csr_mode ? (int32_t)(n / g.n_pad) : 0, g.pad_node);
  else
    k_f32_to_bf16<<<::qh::counted(nblk(n)), 256, 0, s>>>(x, xh, n);
}

void launch_f32_to_bf16(cudaStream_t s, const float* x, __nv_bfloat16* xh, int64_t n) {
  if (n > 0) k_f32_to_bf16<<<::qh::counted(nblk(n)), 256, 0, s>>>(x, xh, n);
}

void launch_step_f32(cudaStream_t s, const Graph& g, const StepArgs& a) {
  if (g.n_row_tiles == 0) return;
  dim3 grid(g.n_row_tiles, (a.R + F_RT - 1) / F_RT);
  k_step_f32<<<::qh::counted(grid), 256, 0, s>>>(a);
}

const char* csr_variant_name(int v, bool bf16) {
  if (v == CSR_BAND8) return "csr-band8-bf16";
  if (v == CSR_LANE8) return bf16 ? "csr-lane8-bf16" : "csr-lane8-fp32";
  return bf16 ? "csr-lane4-bf16" : "csr-lane4-fp32";
}

void launch_step_csr(cudaStream_t s, const Graph& g, const StepArgs& a, const float* pval,
                     const __nv_bfloat16* xh_in, int variant, bool remainder) {
  if (g.n_pad == 0) return;
  // a warp per vertex, CSR_CTA threads per CTA
  const unsigned grid = (unsigned)(((int64_t)g.n_pad * 32 + CSR_CTA - 1) / CSR_CTA);
  const int64_t* rowp = remainder ? g.rrow_ptr : g.prow_ptr;
  const int32_t* colp = remainder ? g.rcol : g.pcol;
  const bool disc = a.sb == QH_SB_DISCRETE;  // FP32 operands: sgn of the gathered x
  if ((variant == CSR_LANE8 || variant == CSR_BAND8) && a.R % 8 == 0) {
    // lanes per neighbour row: 8 replicas each, at most a warp
    const int lanes = a.R >= 256 ? 32 : a.R >= 128 ? 16 : a.R >= 64 ? 8 : 4;
#define QH_CSR8(P)                                                                               \
  (xh_in == nullptr && disc                                                                      \
       ? k_step_csr8<false, P, false, true><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, \
                                                                          pval, nullptr)         \
   : xh_in == nullptr                                                                            \
       ? k_step_csr8<false, P, false, false><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, \
                                                                          pval, nullptr)         \
   : a.zb != nullptr                                                                             \
       ? k_step_csr8<true, P, true, false><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, \
                                                                          pval, xh_in)           \
       : k_step_csr8<true, P, false, false><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, \
                                                                          pval, xh_in))
    switch (lanes) {
      case 32: QH_CSR8(1); break;
      case 16: QH_CSR8(2); break;
      case 8: QH_CSR8(4); break;
      default: QH_CSR8(8); break;
    }
#undef QH_CSR8
    return;
  }
  if (xh_in != nullptr)
    k_step_csr<true, false><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, pval, xh_in);
  else if (disc)
    k_step_csr<false, true><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, pval, nullptr);
  else
    k_step_csr<false, false><<<::qh::counted(grid), CSR_CTA, 0, s>>>(a, rowp, colp, pval, nullptr);
}

void launch_transpose(cudaStream_t s, const float* in, float* out, int64_t rows, int64_t cols) {
  if (rows == 0 || cols == 0) return;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  k_transpose<<<::qh::counted(grid), 256, 0, s>>>(in, out, rows, cols);
}

void launch_signs(cudaStream_t s, const Graph& g, int32_t R, const float* x, int8_t* signs_t) {
  if (g.n_pad == 0) return;
  if (g.csr_mode) {  // state already vertex-major
    const int64_t n = (int64_t)g.n_pad * R;
    k_signs_vm<<<::qh::counted(nblk(n)), 256, 0, s>>>(x, n, signs_t);
    return;
  }
  dim3 grid((g.n_pad + 31) / 32, (R + 31) / 32);
  k_signs_t<<<::qh::counted(grid), 256, 0, s>>>(x, g.n_pad, R, signs_t);
}

void launch_cut(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t, const double* w,
                const double* sum_w, double* node_val, double* cuts, const int32_t* active) {
  if (g.n_blocks == 0) return;
  // replicas per lane: a multiple of 4 in [4, 32] so that one warp pass spans R
  int32_t per = (((R + 31) / 32) + 3) / 4 * 4;
  per = per < 4 ? 4 : (per > 32 ? 32 : per);
  // integer weights: exact int32; real weights: FP64 for a few replicas (the final
  // parity cut), compensated FP32 for the many-replica pick
  if (g.integer_weights)
    k_cut_nodes<<<::qh::counted(nblk((int64_t)g.n_nodes * 32)), 256, 0, s>>>(
        g.n_nodes, g.row_ptr, g.col, w, g.block_of, g.pad_index, signs_t, R, per, node_val, active);
  else if (R <= 4)
    k_cut_nodes_few<<<::qh::counted(nblk((int64_t)g.n_nodes * 32)), 256, 0, s>>>(
        g.n_nodes, g.row_ptr, g.col, w, g.block_of, g.pad_index, signs_t, R, node_val, active);
  else  // at most 8 replicas per lane: 16 accumulators, more warps in flight
    k_cut_nodes_df<8><<<::qh::counted(nblk((int64_t)g.n_nodes * 32)), 256, 0, s>>>(
        g.n_nodes, g.row_ptr, g.col, w, g.block_of, g.pad_index, signs_t, R, per < 8 ? per : 8,
        node_val, active);
  dim3 grid((R + 31) / 32, g.n_blocks);
  k_cut_reduce<<<::qh::counted(grid), 1024, 0, s>>>(g.n_blocks, g.pad_off, g.block_ptr, R, node_val, sum_w, cuts,
                                     active);
}

void launch_cut_from_product(cudaStream_t s, const Graph& g, int32_t R, const float* z,
                             const __nv_bfloat16* signs, const double* sum_w, double* acc,
                             double* cuts, const int32_t* active) {
  if (g.n_blocks == 0) return;
  int32_t max_n = 0;
  for (int32_t b = 0; b < g.n_blocks; ++b) max_n = std::max(max_n, g.h_block_size[b]);
  cudaMemsetAsync(acc, 0, (size_t)g.n_blocks * R * 8, s);
  dim3 grid((R + 31) / 32, (max_n + CUT_CHUNK - 1) / CUT_CHUNK, g.n_blocks);
  k_cut_from_product<<<::qh::counted(grid), 1024, 0, s>>>(g.pad_off, g.block_ptr, R, g.n_pad, z,
                                                          signs, acc, active);
  k_cut_finish<<<::qh::counted(nblk((int64_t)g.n_blocks * R)), 256, 0, s>>>(g.n_blocks, R, acc,
                                                                          sum_w, cuts, active);
}

void launch_pick_best(cudaStream_t s, int32_t n_blocks, int32_t R, const double* cuts,
                      int32_t* best_r, double* best_cut, const int32_t* active) {
  if (n_blocks > 0) k_pick_best<<<::qh::counted(n_blocks), 256, 0, s>>>(n_blocks, R, cuts, best_r, best_cut, active);
}

// One row of the energy-check trace: each block's best cut over the replicas at the check
// after t_done steps, NaN for a block that is not running (stopped early, or not solved)
// or whose schedule has ended (the checks inside the multi-step launch skip those too).
__global__ void k_trace_check(int32_t n_blocks, const double* __restrict__ best_cut,
                              const int32_t* __restrict__ running, int32_t t_done,
                              const int32_t* __restrict__ steps_b, double* row) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_blocks)
    row[b] = running[b] && t_done < steps_b[b] ? best_cut[b] : __longlong_as_double(-1ll);
}

void launch_trace_check(cudaStream_t s, int32_t n_blocks, const double* best_cut,
                        const int32_t* running, int32_t t_done, const int32_t* steps_b,
                        double* row) {
  if (n_blocks > 0)
    k_trace_check<<<::qh::counted(nblk(n_blocks)), 256, 0, s>>>(n_blocks, best_cut, running,
                                                                t_done, steps_b, row);
}

void launch_early_stop(cudaStream_t s, int32_t n_blocks, const double* best_cut, double* best_seen,
                       int32_t* stall, int32_t* active, int32_t* steps_run, int32_t patience,
                       int32_t t_done, const int32_t* steps_b) {
  if (n_blocks > 0)
    k_early_stop<<<::qh::counted(nblk(n_blocks)), 256, 0, s>>>(n_blocks, best_cut, best_seen, stall, active,
                                               steps_run, patience, t_done, steps_b);
}

void launch_track_check(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t,
                        const double* best_cut, const int32_t* best_r, const int32_t* active,
                        int32_t t_done, const int32_t* steps_b, double* kept_cut, int32_t* kept_r,
                        int32_t* flag, int8_t* kept_spins) {
  if (g.n_blocks == 0) return;
  k_track_check<<<::qh::counted(nblk(g.n_blocks)), 256, 0, s>>>(g.n_blocks, best_cut, best_r, active,
                                                   t_done, steps_b, kept_cut, kept_r, flag);
  launch_extract_spins(s, g, R, signs_t, best_r, kept_spins, flag);
}

void launch_track_final(cudaStream_t s, const Graph& g, double* best_cut, int32_t* best_r,
                        const int32_t* active, const double* kept_cut, const int32_t* kept_r,
                        int32_t* flag, const int8_t* kept_spins, int8_t* spins) {
  if (g.n_blocks == 0) return;
  k_track_final<<<::qh::counted(nblk(g.n_blocks)), 256, 0, s>>>(g.n_blocks, best_cut, best_r, active,
                                                   kept_cut, kept_r, flag);
  if (g.n_nodes > 0)
    k_copy_spins<<<::qh::counted(nblk(g.n_nodes)), 256, 0, s>>>(g.n_nodes, g.block_of, flag,
                                                   kept_spins, spins);
}

void launch_extract_spins(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t,
                          const int32_t* best_r, int8_t* spins, const int32_t* active) {
  if (g.n_nodes > 0)
    k_extract_spins<<<::qh::counted(nblk(g.n_nodes)), 256, 0, s>>>(g.n_nodes, g.block_of, g.pad_index, signs_t, R,
                                                    best_r, spins, active);
}

void launch_block_sums(cudaStream_t s, const Graph& g, const double* w, double* sum_w,
                       double* sum_j2, double* node_tmp) {
  if (g.n_blocks == 0) return;
  k_node_sums<<<::qh::counted(nblk(g.n_nodes)), 256, 0, s>>>(g.n_nodes, g.row_ptr, w, node_tmp,
                                              node_tmp + g.n_nodes);
  k_block_sums<<<::qh::counted(g.n_blocks), 256, 0, s>>>(g.n_blocks, g.block_ptr, g.perm, node_tmp,
                                          node_tmp + g.n_nodes, sum_w, sum_j2);
}

void launch_refine_prepare(cudaStream_t s, const Graph& g, const int8_t* spins,
                           const double* best_cut, int32_t* active, int32_t* C, float* deform,
                           int32_t* tries, float deform_h, int32_t deform_tries) {
  if (g.n_blocks > 0)
    k_refine_prepare<<<::qh::counted((unsigned)g.n_blocks), 256, 0, s>>>(
        g.n_blocks, g.block_ptr, g.perm, spins, best_cut, active, C, deform, tries, deform_h,
        deform_tries);
}

void launch_gauge(cudaStream_t s, const Graph& g, const int8_t* spins, double* w,
                  const int32_t* active, const float* deform, int8_t* gauge) {
  if (g.n_nodes > 0)
    k_gauge<<<::qh::counted(nblk((int64_t)g.n_nodes * 32)), 256, 0, s>>>(
        g.n_nodes, g.row_ptr, g.col, g.block_of, spins, w, active, deform, gauge);
}

void launch_apply_gauge(cudaStream_t s, const Graph& g, const double* w0, const int8_t* gauge,
                        double* w) {
  if (g.n_nodes > 0)
    k_apply_gauge<<<::qh::counted(nblk((int64_t)g.n_nodes * 32)), 256, 0, s>>>(
        g.n_nodes, g.row_ptr, g.col, w0, gauge, w);
}

void launch_vote(cudaStream_t s, const Graph& g, const int8_t* spins, int8_t* hap1, int8_t* hap2,
                 int32_t* block_id) {
  if (g.n_snps > 0)
    k_vote<<<::qh::counted(nblk(g.n_snps)), 256, 0, s>>>(g.n_snps, g.cov_ptr, g.cov_frag, g.cov_allele,
                                          g.block_of, spins, hap1, hap2, block_id);
}

void launch_parity(cudaStream_t s, const Graph& g, const int32_t* C, int8_t* hap1, int8_t* hap2,
                   int32_t* block_id) {
  if (g.n_snps > 0)
    k_parity<<<::qh::counted(nblk(g.n_snps)), 256, 0, s>>>(g.n_snps, g.block_of, C, hap1, hap2, block_id);
}

}  // namespace qh
