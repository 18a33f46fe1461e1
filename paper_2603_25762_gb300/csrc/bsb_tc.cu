// Fused bSB step on the 5th-generation tensor cores (sm_103a): one CTA per
// (128-row tile of J, BN replicas).  For each nonzero 128 x 128 J tile of its
// row slab, TMA stages the J tile and the matching X_hat tile (BF16, 128-byte
// swizzle) into shared memory; one thread issues tcgen05.mma (BF16 x BF16 ->
// FP32) into a TMEM accumulator; then all four warps read Z = J_hat X_hat back
// with tcgen05.ld and apply the bSB update of the SB algorithm solution:
//   y <- y + dt * ( -(a0 - a(t)) x + c0 * Z ),  x <- x + dt * a0 * y,
//   |x| > 1 => x <- sgn(x), y <- 0,            X_hat_{t+1} <- bf16(x)
// State x, y stays FP32 in HBM ([R][n_pad], vertex-contiguous, so each warp's
// accesses are 128-byte coalesced).  Every mbarrier wait is bounded: on expiry
// the kernel sets ERR_TIMEOUT in the error word and skips its update.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include "qh_internal.cuh"
#include "tc_ptx.cuh"

namespace qh {

namespace {

template <int BN, int STAGES>
struct TcSmem {
  static constexpr uint32_t B_BYTES = BN * 64 * 2;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t BAR_OFF = STAGES * STAGE;
  static constexpr uint32_t BYTES = BAR_OFF + 8 * (2 * STAGES + 1) + 16 + 1024;  // + align slack
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(128) k_step_tc(const __grid_constant__ CUtensorMap tmJ,
                                                 const __grid_constant__ CUtensorMap tmX,
                                                 StepArgs a) {
  using L = TcSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 accb = smem_u32(bars + 2 * STAGES);

  const RowTile rt = a.rt[blockIdx.x];
  const int32_t sb = a.steps_b[rt.block];
  if ((a.active != nullptr && !a.active[rt.block]) || a.t >= sb) return;  // CTA-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (a.use_lo ? rt.n_all : rt.n_hi) * 2;  // 64-wide K slices

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), (uint32_t)BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nk > 0) {
    // producer: TMA J slice and X_hat slice per stage
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err)) break;
      uint8_t* sa = smem + s * L::STAGE;
      mbar_expect_tx(full0 + 8 * s, L::STAGE);
      const int e = kb >> 1, half = kb & 1;
      tma_load_2d(smem_u32(sa), &tmJ, full0 + 8 * s, half * 64, (rt.tile_begin + e) * TILE);
      tma_load_2d(smem_u32(sa + A_BYTES), &tmX, full0 + 8 * s,
                  a.tile_col[rt.tile_begin + e] * TILE + half * 64, (int32_t)blockIdx.y * BN);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer: 4 x (K = 16) per 64-wide slice
    constexpr uint32_t idesc = idesc_bf16<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph, a.err)) break;
      tc_fence_after();
      uint8_t* sa = smem + s * L::STAGE;
      const uint64_t ad = sdesc_sw128(smem_u32(sa));
      const uint64_t bd = sdesc_sw128(smem_u32(sa + A_BYTES));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma_bf16(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                 (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(accb);
  }
  __syncwarp();

  // epilogue: thread <-> accumulator row (TMEM lane), 32 replica columns at a time
  const bool ok = nk > 0 ? mbar_wait(accb, 0, a.err) : true;
  tc_fence_after();
  const int row = warp * 32 + lane;
  const bool vrow = ok && row < rt.valid;
  const double at = (double)a.a0 * (double)a.t / (double)sb;
  const float coef_x = (float)(-((double)a.a0 - at));
  const float c0 = a.c0[rt.block];
  const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
  const size_t base = (size_t)blockIdx.y * BN * a.n_pad + rt.row0 + row;
#pragma unroll
  for (int c = 0; c < BN / 32; ++c) {
    uint32_t v[32];
    __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the row guard below
    if (nk > 0) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0u;
    }
    if (!vrow) continue;
    const size_t b0 = base + (size_t)(c * 32) * a.n_pad;
    if (a.z_out != nullptr) {
#pragma unroll
      for (int j = 0; j < 32; ++j) a.z_out[b0 + (size_t)j * a.n_pad] = __uint_as_float(v[j]);
      continue;
    }
    float xs[32], ys[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      xs[j] = a.x[b0 + (size_t)j * a.n_pad];
      ys[j] = a.y[b0 + (size_t)j * a.n_pad];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float x = xs[j], y = ys[j];
      sb_update(a.sb, __uint_as_float(v[j]), x, y, a.dt, coef_x, a.dta0, c0, fe);
      const size_t idx = b0 + (size_t)j * a.n_pad;
      a.x[idx] = x;
      a.y[idx] = y;
      a.xh_out[idx] = __float2bfloat16_rn(sb_operand(a.sb, x));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)BN);
  }
}

// ---------------------------------------------------------------------------
// Launch-bounded variant of the step kernel for the solver: MINB CTAs per SM share
// the SM (one CTA's epilogue overlaps another's TMA / MMA phase).  The first 32
// replica columns of the state are loaded before the accumulator is ready and the
// next 32 are in flight while the current 32 are updated.
template <int BN, int STAGES, int MINB>
__global__ void __launch_bounds__(128, MINB) k_step_tc_v(const __grid_constant__ CUtensorMap tmJ,
                                                         const __grid_constant__ CUtensorMap tmX,
                                                         StepArgs a) {
  using L = TcSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 accb = smem_u32(bars + 2 * STAGES);

  const RowTile rt = a.rt[blockIdx.x];
  const int32_t sb = a.steps_b[rt.block];
  if ((a.active != nullptr && !a.active[rt.block]) || a.t >= sb) return;  // CTA-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (a.use_lo ? rt.n_all : rt.n_hi) * 2;
  const int row = warp * 32 + lane;
  const bool vrow = row < rt.valid;
  const size_t base = (size_t)blockIdx.y * BN * a.n_pad + rt.row0 + row;
  constexpr int CH = 16;  // replica columns per epilogue chunk
  float xs[CH], ys[CH];
  if (vrow) {  // chunk 0 of the state: independent of the product, start it now
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      xs[j] = a.x[base + (size_t)j * a.n_pad];
      ys[j] = a.y[base + (size_t)j * a.n_pad];
    }
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), (uint32_t)BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nk > 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err)) break;
      uint8_t* sa = smem + s * L::STAGE;
      mbar_expect_tx(full0 + 8 * s, L::STAGE);
      const int e = kb >> 1, half = kb & 1;
      tma_load_2d(smem_u32(sa), &tmJ, full0 + 8 * s, half * 64, (rt.tile_begin + e) * TILE);
      tma_load_2d(smem_u32(sa + A_BYTES), &tmX, full0 + 8 * s,
                  a.tile_col[rt.tile_begin + e] * TILE + half * 64, (int32_t)blockIdx.y * BN);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    constexpr uint32_t idesc = idesc_bf16<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph, a.err)) break;
      tc_fence_after();
      uint8_t* sa = smem + s * L::STAGE;
      const uint64_t ad = sdesc_sw128(smem_u32(sa));
      const uint64_t bd = sdesc_sw128(smem_u32(sa + A_BYTES));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma_bf16(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                 (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(accb);
  }
  __syncwarp();

  const bool ok = nk > 0 ? mbar_wait(accb, 0, a.err) : true;
  tc_fence_after();
  const double at = a.a0 * (double)a.t / (double)sb;
  const float coef_x = (float)(-(a.a0 - at));
  const float c0 = a.c0[rt.block];
  const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
#pragma unroll
  for (int c = 0; c < BN / CH; ++c) {
    uint32_t v[CH];
    __syncwarp();
    if (nk > 0) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * CH), v);
    } else {
#pragma unroll
      for (int j = 0; j < CH; ++j) v[j] = 0u;
    }
    const size_t b0 = base + (size_t)(c * CH) * a.n_pad;
    const bool more = c + 1 < BN / CH;
    float xn[CH], yn[CH];
    if (vrow && more) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        xn[j] = a.x[b0 + (size_t)(CH + j) * a.n_pad];
        yn[j] = a.y[b0 + (size_t)(CH + j) * a.n_pad];
      }
    }
    if (vrow && ok) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        float x = xs[j], y = ys[j];
        sb_update(a.sb, __uint_as_float(v[j]), x, y, a.dt, coef_x, a.dta0, c0, fe);
        const size_t idx = b0 + (size_t)j * a.n_pad;
        a.x[idx] = x;
        a.y[idx] = y;
        a.xh_out[idx] = __float2bfloat16_rn(sb_operand(a.sb, x));
      }
    }
    if (more) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        xs[j] = xn[j];
        ys[j] = yn[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)BN);
  }
}

// ---------------------------------------------------------------------------
// FP8 (e4m3) variant.  With J' = s J split as J' = Jh + Jl and x = xh + xl (all e4m3,
// s a power of two), each nonzero tile contributes the slices (Jh, Xh), (Jh, Xl) and,
// when J' has a remainder, (Jl, Xh) -- the dropped Jl Xl term is ~2^-8 relative.  A
// slice is one 128 x 128-byte K-slice of A and B (four K = 32 kind::f8f6f4 MMAs), so
// stages, descriptors and smem layout are those of the BF16 kernel.  Z = acc / s.
__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major, M = 128.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_e4m3() {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void split_e4m3(float x, uint8_t& h, uint8_t& l) {
  __nv_fp8_e4m3 hi(x);
  __nv_fp8_e4m3 lo(x - static_cast<float>(hi));
  h = hi.__x;
  l = lo.__x;
}

template <int BN, int STAGES, int MINB>
__global__ void __launch_bounds__(128, MINB)
    k_step_tc_f8(const __grid_constant__ CUtensorMap tmJh, const __grid_constant__ CUtensorMap tmJl,
                 const __grid_constant__ CUtensorMap tmXh, const __grid_constant__ CUtensorMap tmXl,
                 StepArgs a, int32_t n_slices) {
  using L = TcSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 accb = smem_u32(bars + 2 * STAGES);

  const RowTile rt = a.rt[blockIdx.x];
  const int32_t sb = a.steps_b[rt.block];
  if ((a.active != nullptr && !a.active[rt.block]) || a.t >= sb) return;  // CTA-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = rt.n_hi * n_slices;
  const int row = warp * 32 + lane;
  const bool vrow = row < rt.valid;
  const size_t base = (size_t)blockIdx.y * BN * a.n_pad + rt.row0 + row;
  constexpr int CH = 16;
  float xs[CH], ys[CH];
  if (vrow && a.z_out == nullptr) {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      xs[j] = a.x[base + (size_t)j * a.n_pad];
      ys[j] = a.y[base + (size_t)j * a.n_pad];
    }
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), (uint32_t)BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nk > 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err)) break;
      uint8_t* sa = smem + s * L::STAGE;
      mbar_expect_tx(full0 + 8 * s, L::STAGE);
      const int e = kb / n_slices, sl = kb % n_slices;  // slice: 0 (Jh,Xh) 1 (Jh,Xl) 2 (Jl,Xh)
      const CUtensorMap* mj = sl == 2 ? &tmJl : &tmJh;
      const CUtensorMap* mx = sl == 1 ? &tmXl : &tmXh;
      tma_load_2d(smem_u32(sa), mj, full0 + 8 * s, 0, (rt.f32_begin + e) * TILE);
      tma_load_2d(smem_u32(sa + A_BYTES), mx, full0 + 8 * s,
                  a.tile_col[rt.tile_begin + e] * TILE, (int32_t)blockIdx.y * BN);
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    constexpr uint32_t idesc = idesc_e4m3<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph, a.err)) break;
      tc_fence_after();
      uint8_t* sa = smem + s * L::STAGE;
      const uint64_t ad = sdesc_sw128(smem_u32(sa));
      const uint64_t bd = sdesc_sw128(smem_u32(sa + A_BYTES));
#pragma unroll
      for (int k = 0; k < 4; ++k)  // K = 32 e4m3 = 32 bytes per MMA
        mma_f8(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
               (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(accb);
  }
  __syncwarp();

  const bool ok = nk > 0 ? mbar_wait(accb, 0, a.err) : true;
  tc_fence_after();
  const double at = a.a0 * (double)a.t / (double)sb;
  const float coef_x = (float)(-(a.a0 - at));
  const float c0 = a.c0[rt.block];
  const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
  const float inv_s = a.inv_scale;
#pragma unroll
  for (int c = 0; c < BN / CH; ++c) {
    uint32_t v[CH];
    __syncwarp();
    if (nk > 0) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * CH), v);
    } else {
#pragma unroll
      for (int j = 0; j < CH; ++j) v[j] = 0u;
    }
    const size_t b0 = base + (size_t)(c * CH) * a.n_pad;
    if (a.z_out != nullptr) {
      if (vrow && ok)
#pragma unroll
        for (int j = 0; j < CH; ++j)
          a.z_out[b0 + (size_t)j * a.n_pad] = __uint_as_float(v[j]) * inv_s;
      continue;
    }
    const bool more = c + 1 < BN / CH;
    float xn[CH], yn[CH];
    if (vrow && more) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        xn[j] = a.x[b0 + (size_t)(CH + j) * a.n_pad];
        yn[j] = a.y[b0 + (size_t)(CH + j) * a.n_pad];
      }
    }
    if (vrow && ok) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        float x = xs[j], y = ys[j];
        sb_update(a.sb, __uint_as_float(v[j]) * inv_s, x, y, a.dt, coef_x, a.dta0, c0, fe);
        const size_t idx = b0 + (size_t)j * a.n_pad;
        a.x[idx] = x;
        a.y[idx] = y;
        uint8_t h8, l8;  // the variant's operand: for discrete SB sgn(x), lo = 0
        split_e4m3(sb_operand(a.sb, x), h8, l8);
        a.x8h_out[idx] = h8;
        a.x8l_out[idx] = l8;
      }
    }
    if (more) {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        xs[j] = xn[j];
        ys[j] = yn[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)BN);
  }
}

// J' = s J (FP32 tiles) -> e4m3 hi / lo tiles; flag = 1 if any remainder is nonzero.
__global__ void k_tiles_to_e4m3(const float* __restrict__ tf, int64_t n, float s, uint8_t* th,
                                uint8_t* tl, int32_t* has_lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint8_t h, l;
  split_e4m3(tf[i] * s, h, l);
  th[i] = h;
  tl[i] = l;
  if (l != 0 && (l & 0x7f) != 0) atomicOr(has_lo, 1);
}

// x -> e4m3 hi / lo.  pad_node != nullptr: the operand of SB variant sb at real
// vertices (state [R][n_pad]), 0 at padding.
__global__ void k_x_to_e4m3(const float* __restrict__ x, int64_t n, uint8_t* h, uint8_t* l,
                            int32_t sb, int32_t n_pad, const int32_t* __restrict__ pad_node) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = pad_node == nullptr      ? x[i]
                  : pad_node[i % n_pad] >= 0 ? sb_operand(sb, x[i])
                                             : 0.f;
  split_e4m3(v, h[i], l[i]);
}

// ---------------------------------------------------------------------------
// Persistent variant: one CTA per SM walks the (row tile, BN replicas) work items
// of the step.  Warp 0 (one thread) issues TMA: the item's FP32 x and y state
// tiles ([BN][128], double-buffered) and the J / X_hat K-slices (operand ring).
// Warp 1 (one thread) issues tcgen05.mma into one of two TMEM accumulators.
// Warps 2-5 read the accumulator (TMEM lane quarter = warp % 4), update x, y in
// shared memory, store X_hat_{t+1} directly and hand the tiles back to TMA for the
// store.  Loads of the next item overlap the update and stores of the current one.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int32_t c0,
                                             int32_t c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void epi_barrier() {  // named barrier 1: the 4 epilogue warps
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

template <int BN, int OSTAGES>
struct PSmem {
  static constexpr uint32_t B_BYTES = BN * 64 * 2;
  static constexpr uint32_t OSTAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t STILE = BN * TILE * 4;        // one FP32 state tile
  static constexpr uint32_t STATE_OFF = OSTAGES * OSTAGE; // 2 buffers x (x tile, y tile)
  static constexpr uint32_t BAR_OFF = STATE_OFF + 4 * STILE;
  static constexpr uint32_t N_BARS = 2 * OSTAGES + 8;
  static constexpr uint32_t BYTES = BAR_OFF + 8 * N_BARS + 16 + 1024;
};

__device__ __forceinline__ bool item_live(const StepArgs& a, const RowTile& rt) {
  return (a.active == nullptr || a.active[rt.block]) && a.t < a.steps_b[rt.block];
}

template <int BN, int OSTAGES>
__global__ void __launch_bounds__(192, 1)
    k_step_tc_p(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmX,
                const __grid_constant__ CUtensorMap tmSx, const __grid_constant__ CUtensorMap tmSy,
                StepArgs a, int32_t n_items, int32_t n_rep) {
  using L = PSmem<BN, OSTAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::N_BARS);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + OSTAGES);
  const uint32_t sfull0 = smem_u32(bars + 2 * OSTAGES), sempty0 = sfull0 + 16;
  const uint32_t afull0 = sfull0 + 32, aempty0 = sfull0 + 48;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OSTAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(sfull0 + 8 * s, 1);
      mbar_init(sempty0 + 8 * s, 1);
      mbar_init(afull0 + 8 * s, 1);
      mbar_init(aempty0 + 8 * s, 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), (uint32_t)(2 * BN));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0, kg = 0;
      bool ok = true;
      for (int32_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const int32_t rti = item / n_rep, rn = item % n_rep;
        const RowTile rt = a.rt[rti];
        if (!item_live(a, rt)) continue;
        const uint32_t sb = it & 1u, sph = (it >> 1) & 1u;
        if (!(ok = mbar_wait(sempty0 + 8 * sb, sph ^ 1u, a.err))) break;
        uint8_t* sx = smem + L::STATE_OFF + sb * 2 * L::STILE;
        mbar_expect_tx(sfull0 + 8 * sb, 2 * L::STILE);
        tma_load_2d(smem_u32(sx), &tmSx, sfull0 + 8 * sb, rt.row0, rn * BN);
        tma_load_2d(smem_u32(sx + L::STILE), &tmSy, sfull0 + 8 * sb, rt.row0, rn * BN);
        const int nk = (a.use_lo ? rt.n_all : rt.n_hi) * 2;
        for (int kb = 0; kb < nk; ++kb, ++kg) {
          const uint32_t st = kg % OSTAGES, ph = (kg / OSTAGES) & 1u;
          if (!(ok = mbar_wait(empty0 + 8 * st, ph ^ 1u, a.err))) break;
          uint8_t* sa = smem + st * L::OSTAGE;
          mbar_expect_tx(full0 + 8 * st, L::OSTAGE);
          const int e = kb >> 1, half = kb & 1;
          tma_load_2d(smem_u32(sa), &tmJ, full0 + 8 * st, half * 64, (rt.tile_begin + e) * TILE);
          tma_load_2d(smem_u32(sa + A_BYTES), &tmX, full0 + 8 * st,
                      a.tile_col[rt.tile_begin + e] * TILE + half * 64, rn * BN);
        }
        ++it;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      uint32_t it = 0, kg = 0;
      bool ok = true;
      for (int32_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const RowTile rt = a.rt[item / n_rep];
        if (!item_live(a, rt)) continue;
        const uint32_t ab = it & 1u, aph = (it >> 1) & 1u;
        if (!(ok = mbar_wait(aempty0 + 8 * ab, aph ^ 1u, a.err))) break;
        tc_fence_after();
        const uint32_t dcol = tmem + ab * BN;
        const int nk = (a.use_lo ? rt.n_all : rt.n_hi) * 2;
        for (int kb = 0; kb < nk; ++kb, ++kg) {
          const uint32_t st = kg % OSTAGES, ph = (kg / OSTAGES) & 1u;
          if (!(ok = mbar_wait(full0 + 8 * st, ph, a.err))) break;
          tc_fence_after();
          uint8_t* sa = smem + st * L::OSTAGE;
          const uint64_t ad = sdesc_sw128(smem_u32(sa));
          const uint64_t bd = sdesc_sw128(smem_u32(sa + A_BYTES));
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_bf16(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                     (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(empty0 + 8 * st);
        }
        mma_commit(afull0 + 8 * ab);
        ++it;
      }
    }
  } else {
    // epilogue warps 2..5
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;     // accumulator row = vertex within the row tile
    const bool leader = (warp == 2 && lane == 0);
    uint32_t it = 0;
    for (int32_t item = blockIdx.x; item < n_items; item += gridDim.x) {
      const int32_t rti = item / n_rep, rn = item % n_rep;
      const RowTile rt = a.rt[rti];
      if (!item_live(a, rt)) continue;
      const uint32_t b = it & 1u, ph = (it >> 1) & 1u;
      bool ok = mbar_wait(afull0 + 8 * b, ph, a.err);
      ok = mbar_wait(sfull0 + 8 * b, ph, a.err) && ok;
      tc_fence_after();
      float* sx = reinterpret_cast<float*>(smem + L::STATE_OFF + b * 2 * L::STILE);
      float* sy = sx + BN * TILE;
      const double at = a.a0 * (double)a.t / (double)a.steps_b[rt.block];
      const float coef_x = (float)(-(a.a0 - at));
      const float c0 = a.c0[rt.block];
      const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
      const bool vrow = ok && row < rt.valid;
      __nv_bfloat16* xh = a.xh_out + (size_t)rn * BN * a.n_pad + rt.row0 + row;
#pragma unroll
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(tmem + b * BN + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32), v);
        if (vrow) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int r = c * 32 + j;
            float x = sx[r * TILE + row], y = sy[r * TILE + row];
            sb_update(a.sb, __uint_as_float(v[j]), x, y, a.dt, coef_x, a.dta0, c0, fe);
            sx[r * TILE + row] = x;
            sy[r * TILE + row] = y;
            xh[(size_t)r * a.n_pad] = __float2bfloat16_rn(sb_operand(a.sb, x));
          }
        }
      }
      // accumulator free for the MMA warp, state tile ready for the TMA store
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty0 + 8 * b);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      epi_barrier();
      if (leader) {
        if (ok) {
          tma_store_2d(&tmSx, smem_u32(sx), rt.row0, rn * BN);
          tma_store_2d(&tmSy, smem_u32(sy), rt.row0, rn * BN);
          bulk_commit();
          bulk_wait_read0();
        }
        mbar_arrive(sempty0 + 8 * b);
      }
      ++it;
    }
    if (leader) bulk_wait0();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)(2 * BN));
  }
}

// ---------------------------------------------------------------------------
// Persistent register-epilogue variant (the solver's step kernel).  One CTA per
// SM walks the (row tile, 128 replicas) work items.  Warp 0 issues the TMA loads
// of the J and X_hat K-slices into a 4-stage ring, warp 1 issues tcgen05.mma into
// one of two TMEM accumulators (item i+1 accumulates while item i is updated).
// Warps 4..11 are the epilogue: warp w reads TMEM lane quarter w % 4 and column
// half (w - 4) / 4, so each thread owns one vertex and 64 replicas.  The FP32
// state goes HBM -> registers -> HBM with warp-coalesced 128-byte accesses; the x,
// y loads of the next 32 columns are in flight while the current ones are updated,
// and the first chunk of an item is loaded before its accumulator is ready.
constexpr int P2_BN = 128;
constexpr int P2_STAGES = 4;
constexpr int P2_MAX_TILES = 64;  // per row tile (hi + lo entries); more falls back

struct P2Smem {
  static constexpr uint32_t B_BYTES = P2_BN * 64 * 2;
  static constexpr uint32_t OSTAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t COL_OFF = P2_STAGES * OSTAGE;       // staged tile columns
  static constexpr uint32_t BAR_OFF = COL_OFF + 2 * P2_MAX_TILES * 4;
  static constexpr uint32_t N_BARS = 2 * P2_STAGES + 4;
  static constexpr uint32_t BYTES = BAR_OFF + 8 * N_BARS + 16 + 1024;
};

__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap* map, int32_t c0, int32_t c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1)
               : "memory");
}

__global__ void __launch_bounds__(384, 1)
    k_step_tc_p2(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmSx, const __grid_constant__ CUtensorMap tmSy,
                 StepArgs a, int32_t n_items, int32_t n_rep) {
  using L = P2Smem;
  constexpr int BN = P2_BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::N_BARS);
  int32_t* scol = reinterpret_cast<int32_t*>(smem + L::COL_OFF);  // [2][P2_MAX_TILES]
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + P2_STAGES);
  const uint32_t afull0 = smem_u32(bars + 2 * P2_STAGES), aempty0 = afull0 + 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P2_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(afull0 + 8 * s, 1);
      mbar_init(aempty0 + 8 * s, 8);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), (uint32_t)(2 * BN));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // stream every item's FP32 state toward L2 now: the epilogue's loads then hit
      // L2 while DRAM runs at full rate underneath
      for (int32_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const RowTile rt = a.rt[item / n_rep];
        if (!item_live(a, rt)) continue;
        tma_prefetch_l2(&tmSx, rt.row0, (item % n_rep) * P2_BN);
        tma_prefetch_l2(&tmSy, rt.row0, (item % n_rep) * P2_BN);
      }
      uint32_t kg = 0, it = 0;
      bool ok = true;
      for (int32_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const RowTile rt = a.rt[item / n_rep];
        const int32_t rn = item % n_rep;
        if (!item_live(a, rt)) continue;
        // stage this item's column tiles (independent loads, one latency)
        int32_t* cols = scol + (it & 1u) * P2_MAX_TILES;
        const int ne = a.use_lo ? rt.n_all : rt.n_hi;
        for (int e = 0; e < ne; ++e) cols[e] = a.tile_col[rt.tile_begin + e];
        const int nk = ne * 2;
        for (int kb = 0; kb < nk; ++kb, ++kg) {
          const uint32_t st = kg % P2_STAGES, ph = (kg / P2_STAGES) & 1u;
          if (!(ok = mbar_wait(empty0 + 8 * st, ph ^ 1u, a.err))) break;
          uint8_t* sa = smem + st * L::OSTAGE;
          mbar_expect_tx(full0 + 8 * st, L::OSTAGE);
          const int e = kb >> 1, half = kb & 1;
          tma_load_2d(smem_u32(sa), &tmJ, full0 + 8 * st, half * 64, (rt.tile_begin + e) * TILE);
          tma_load_2d(smem_u32(sa + A_BYTES), &tmX, full0 + 8 * st, cols[e] * TILE + half * 64,
                      rn * BN);
        }
        ++it;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      uint32_t it = 0, kg = 0;
      bool ok = true;
      for (int32_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const RowTile rt = a.rt[item / n_rep];
        if (!item_live(a, rt)) continue;
        const uint32_t ab = it & 1u, aph = (it >> 1) & 1u;
        if (!(ok = mbar_wait(aempty0 + 8 * ab, aph ^ 1u, a.err))) break;
        tc_fence_after();
        const uint32_t dcol = tmem + ab * BN;
        const int nk = (a.use_lo ? rt.n_all : rt.n_hi) * 2;
        for (int kb = 0; kb < nk; ++kb, ++kg) {
          const uint32_t st = kg % P2_STAGES, ph = (kg / P2_STAGES) & 1u;
          if (!(ok = mbar_wait(full0 + 8 * st, ph, a.err))) break;
          tc_fence_after();
          uint8_t* sa = smem + st * L::OSTAGE;
          const uint64_t ad = sdesc_sw128(smem_u32(sa));
          const uint64_t bd = sdesc_sw128(smem_u32(sa + A_BYTES));
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_bf16(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                     (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(empty0 + 8 * st);
        }
        mma_commit(afull0 + 8 * ab);
        ++it;
      }
    }
  } else if (warp >= 4) {
    const int q = warp & 3;                 // TMEM lane quarter
    const int hcol = ((warp - 4) >> 2) * 64;  // column half
    const int row = q * 32 + lane;
    uint32_t it = 0;
    for (int32_t item = blockIdx.x; item < n_items; item += gridDim.x) {
      const RowTile rt = a.rt[item / n_rep];
      const int32_t rn = item % n_rep;
      if (!item_live(a, rt)) continue;
      const uint32_t ab = it & 1u, aph = (it >> 1) & 1u;
      const bool vrow = row < rt.valid;
      const size_t base = ((size_t)rn * BN + hcol) * a.n_pad + rt.row0 + row;
      // chunk 0 of this item: state loads issued before the accumulator is ready
      float xs[32], ys[32];
      if (vrow) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          xs[j] = a.x[base + (size_t)j * a.n_pad];
          ys[j] = a.y[base + (size_t)j * a.n_pad];
        }
      }
      const bool ok = mbar_wait(afull0 + 8 * ab, aph, a.err);
      tc_fence_after();
      const double at = a.a0 * (double)a.t / (double)a.steps_b[rt.block];
      const float coef_x = (float)(-(a.a0 - at));
      const float c0 = a.c0[rt.block];
      const float fe = deform_force(a.deform, rt.block, a.t, a.steps_b[rt.block]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(tmem + ab * BN + ((uint32_t)(q * 32) << 16) + (uint32_t)(hcol + c * 32), v);
        const size_t b0 = base + (size_t)(c * 32) * a.n_pad;
        float xn[32], yn[32];
        if (vrow && c == 0) {  // next chunk's loads overlap this chunk's update
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            xn[j] = a.x[b0 + (size_t)(32 + j) * a.n_pad];
            yn[j] = a.y[b0 + (size_t)(32 + j) * a.n_pad];
          }
        }
        if (vrow && ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float x = xs[j], y = ys[j];
            sb_update(a.sb, __uint_as_float(v[j]), x, y, a.dt, coef_x, a.dta0, c0, fe);
            const size_t idx = b0 + (size_t)j * a.n_pad;
            a.x[idx] = x;
            a.y[idx] = y;
            a.xh_out[idx] = __float2bfloat16_rn(sb_operand(a.sb, x));
          }
        }
        if (c == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            xs[j] = xn[j];
            ys[j] = yn[j];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty0 + 8 * ab);
      ++it;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)(2 * BN));
  }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D tensor map over a row-major [outer][inner] array with a box of
// box_inner x box_rows elements (BF16 operands: 64-wide boxes with the 128-byte
// swizzle that sdesc_sw128 describes; FP32 state tiles: 128-wide, unswizzled).
bool make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
              uint32_t box_rows, bool fp32, bool bytes) {
  auto enc = get_encode();
  if (!enc) return false;
  const uint32_t esz = fp32 ? 4 : (bytes ? 1 : 2);
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {fp32 ? 128u : (bytes ? 128u : 64u), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map,
                   fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                        : (bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16),
                   2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   fp32 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

template <int BN, int STAGES, int MINB>
qh_status launch_variant(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* xh_in) {
  CUtensorMap mJ, mX;
  if (!make_map(&mJ, g.tile_bf16, TILE, (uint64_t)g.n_tiles * TILE, TILE) ||
      !make_map(&mX, xh_in, (uint64_t)g.n_pad, (uint64_t)a.R, BN))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed");
  dim3 grid(g.n_row_tiles, a.R / BN);
  k_step_tc_v<BN, STAGES, MINB><<<::qh::counted(grid), 128, TcSmem<BN, STAGES>::BYTES, ctx->stream>>>(mJ, mX, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_step_tc_v launch");
  return QH_OK;
}

template <int BN, int STAGES, int MINB>
cudaError_t set_attr_v() {
  return cudaFuncSetAttribute(k_step_tc_v<BN, STAGES, MINB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcSmem<BN, STAGES>::BYTES);
}

template <int BN, int STAGES, int MINB>
cudaError_t set_attr_f8() {
  return cudaFuncSetAttribute(k_step_tc_f8<BN, STAGES, MINB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcSmem<BN, STAGES>::BYTES);
}

template <int BN, int STAGES, int MINB>
qh_status launch_f8_impl(Ctx* ctx, const Graph& g, const StepArgs& a, const Fp8Operands& op) {
  CUtensorMap mJh, mJl, mXh, mXl;
  const uint64_t jrows = (uint64_t)std::max<int64_t>(g.n_tiles_hi, 1) * TILE;
  if (!make_map(&mJh, op.jh, TILE, jrows, TILE, false, true) ||
      !make_map(&mJl, op.jl, TILE, jrows, TILE, false, true) ||
      !make_map(&mXh, op.xh_in, (uint64_t)g.n_pad, (uint64_t)a.R, BN, false, true) ||
      !make_map(&mXl, op.xl_in, (uint64_t)g.n_pad, (uint64_t)a.R, BN, false, true))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed (e4m3)");
  dim3 grid(g.n_row_tiles, a.R / BN);
  k_step_tc_f8<BN, STAGES, MINB><<<::qh::counted(grid), 128, TcSmem<BN, STAGES>::BYTES,
                                   ctx->stream>>>(mJh, mJl, mXh, mXl, a, op.n_slices);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_step_tc_f8 launch");
  return QH_OK;
}

qh_status launch_persistent2(Ctx* ctx, const Graph& g, const StepArgs& a,
                             const __nv_bfloat16* xh_in) {
  CUtensorMap mJ, mX, mSx, mSy;
  if (!make_map(&mJ, g.tile_bf16, TILE, (uint64_t)g.n_tiles * TILE, TILE) ||
      !make_map(&mX, xh_in, (uint64_t)g.n_pad, (uint64_t)a.R, P2_BN) ||
      !make_map(&mSx, a.x, (uint64_t)g.n_pad, (uint64_t)a.R, P2_BN, true) ||
      !make_map(&mSy, a.y, (uint64_t)g.n_pad, (uint64_t)a.R, P2_BN, true))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed");
  const int32_t n_rep = a.R / P2_BN;
  const int32_t n_items = g.n_row_tiles * n_rep;
  const int grid = std::min(n_items, ctx->n_sm);
  k_step_tc_p2<<<::qh::counted(grid), 384, P2Smem::BYTES, ctx->stream>>>(mJ, mX, mSx, mSy, a, n_items, n_rep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_step_tc_p2 launch");
  return QH_OK;
}

template <int BN, int OSTAGES>
qh_status launch_persistent(Ctx* ctx, const Graph& g, const StepArgs& a,
                            const __nv_bfloat16* xh_in) {
  using L = PSmem<BN, OSTAGES>;
  CUtensorMap mJ, mX, mSx, mSy;
  if (!make_map(&mJ, g.tile_bf16, TILE, (uint64_t)g.n_tiles * TILE, TILE) ||
      !make_map(&mX, xh_in, (uint64_t)g.n_pad, (uint64_t)a.R, BN) ||
      !make_map(&mSx, a.x, (uint64_t)g.n_pad, (uint64_t)a.R, BN, true) ||
      !make_map(&mSy, a.y, (uint64_t)g.n_pad, (uint64_t)a.R, BN, true))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed");
  const int32_t n_rep = a.R / BN;
  const int32_t n_items = g.n_row_tiles * n_rep;
  const int grid = std::min(n_items, ctx->n_sm);
  k_step_tc_p<BN, OSTAGES><<<::qh::counted(grid), 192, L::BYTES, ctx->stream>>>(mJ, mX, mSx, mSy, a, n_items,
                                                                  n_rep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_step_tc_p launch");
  return QH_OK;
}

template <int BN, int STAGES>
qh_status launch_impl(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* xh_in) {
  using L = TcSmem<BN, STAGES>;
  CUtensorMap mJ, mX;
  if (!make_map(&mJ, g.tile_bf16, TILE, (uint64_t)g.n_tiles * TILE, TILE) ||
      !make_map(&mX, xh_in, (uint64_t)g.n_pad, (uint64_t)a.R, BN))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed");
  dim3 grid(g.n_row_tiles, a.R / BN);
  k_step_tc<BN, STAGES><<<::qh::counted(grid), 128, L::BYTES, ctx->stream>>>(mJ, mX, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_step_tc launch");
  return QH_OK;
}

template <int BN, int OSTAGES>
cudaError_t set_attr_p() {
  return cudaFuncSetAttribute(k_step_tc_p<BN, OSTAGES>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PSmem<BN, OSTAGES>::BYTES);
}

template <int BN, int STAGES>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_step_tc<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcSmem<BN, STAGES>::BYTES);
}

}  // namespace

// Once per process and device, outside any stream capture: shared-memory opt-in of
// every kernel variant and the CUDA driver entry point for tensor-map encoding.
qh_status tc_prepare(Ctx* ctx) {
  cudaError_t e = set_attr<64, 4>();
  if (e == cudaSuccess) e = set_attr<128, 3>();
  if (e == cudaSuccess) e = set_attr<256, 2>();
  if (e == cudaSuccess) e = set_attr_p<64, 3>();
  if (e == cudaSuccess) e = set_attr_v<128, 3, 1>();
  if (e == cudaSuccess) e = set_attr_v<128, 2, 3>();
  if (e == cudaSuccess) e = set_attr_v<64, 2, 4>();
  if (e == cudaSuccess) e = set_attr_v<256, 2, 2>();
  if (e == cudaSuccess) e = set_attr_f8<128, 2, 3>();
  if (e == cudaSuccess) e = set_attr_f8<64, 2, 4>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_tc_p2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P2Smem::BYTES);
  if (e == cudaSuccess) e = run_set_attrs();
  if (e == cudaSuccess) e = band_set_attrs();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(k_step_tc)");
  if (!get_encode()) return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled entry point not found");
  return QH_OK;
}

qh_status launch_step_f8(Ctx* ctx, const Graph& g, const StepArgs& a, const Fp8Operands& op) {
  if (g.n_row_tiles == 0) return QH_OK;
  if (a.R % 128 == 0) return launch_f8_impl<128, 2, 3>(ctx, g, a, op);
  return launch_f8_impl<64, 2, 4>(ctx, g, a, op);
}

void launch_tiles_to_e4m3(cudaStream_t s, const float* tf, int64_t n, float scale, uint8_t* th,
                          uint8_t* tl, int32_t* has_lo) {
  if (n > 0)
    k_tiles_to_e4m3<<<::qh::counted((unsigned)((n + 255) / 256)), 256, 0, s>>>(tf, n, scale, th,
                                                                              tl, has_lo);
}

void launch_x_to_e4m3(cudaStream_t s, const float* x, int64_t n, uint8_t* h, uint8_t* l) {
  if (n > 0)
    k_x_to_e4m3<<<::qh::counted((unsigned)((n + 255) / 256)), 256, 0, s>>>(x, n, h, l, 0, 1,
                                                                          nullptr);
}

void launch_x_operand_e4m3(cudaStream_t s, const Graph& g, int32_t sb, const float* x, int64_t n,
                           uint8_t* h, uint8_t* l) {
  if (n > 0 && g.n_pad > 0)
    k_x_to_e4m3<<<::qh::counted((unsigned)((n + 255) / 256)), 256, 0, s>>>(x, n, h, l, sb, g.n_pad,
                                                                          g.pad_node);
}

bool tc_plan_ok(int R, const TcPlan& plan) {
  if (plan.bn != 64 && plan.bn != 128 && plan.bn != 256) return false;
  return R > 0 && R % plan.bn == 0;
}

// Solver-step kernel variants the autotuner chooses from.
int tc_n_variants() { return 10; }
const char* tc_variant_name(int v) {
  static const char* names[] = {"cta-bn128-s3",          "cta-bn128-s2-x3",
                                "cta-bn64-s2-x4",        "cta-bn256-s2-x2",
                                "persistent-bn128",      "persistent-bn64-tma-state",
                                "multistep-jres-group",  "multistep-stream-tile",
                                "multistep-jres-tile",   "multistep-stream-group"};
  return (v >= 0 && v < 10) ? names[v] : "none";
}
bool tc_variant_ok(int v, const Graph& g, int R, int n_sm, bool use_lo) {
  switch (v) {
    case 0: case 1: case 4: return R % 128 == 0 && (v != 4 || g.max_tiles_per_row <= P2_MAX_TILES);
    case 2: case 5: return R % 64 == 0;
    case 3: return R % 256 == 0;
    case 6: case 7: case 8: case 9:
      return run_plan(g, R, n_sm, v, use_lo, nullptr);
    default: return false;
  }
}

qh_status launch_step_tc(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* xh_in,
                         const TcPlan& plan) {
  if (g.n_row_tiles == 0) return QH_OK;
  if (a.z_out == nullptr && plan.variant >= 0) {
    switch (plan.variant) {
      case 0: return launch_variant<128, 3, 1>(ctx, g, a, xh_in);
      case 1: return launch_variant<128, 2, 3>(ctx, g, a, xh_in);
      case 2: return launch_variant<64, 2, 4>(ctx, g, a, xh_in);
      case 3: return launch_variant<256, 2, 2>(ctx, g, a, xh_in);
      case 4: return launch_persistent2(ctx, g, a, xh_in);
      case 5: return launch_persistent<64, 3>(ctx, g, a, xh_in);
      case 6: case 7: case 8: case 9:
        return set_err(ctx, QH_EUNSUPPORTED, "the multi-step kernel runs step ranges (launch_run)");
      default: break;
    }
  }
  if (plan.bn == 64) return launch_impl<64, 4>(ctx, g, a, xh_in);
  if (plan.bn == 128) return launch_impl<128, 3>(ctx, g, a, xh_in);
  return launch_impl<256, 2>(ctx, g, a, xh_in);
}

}  // namespace qh
