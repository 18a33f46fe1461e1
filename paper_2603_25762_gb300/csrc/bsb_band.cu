// Band product of a CSR-mode graph on the tensor cores (SB algorithm solution, the
// per-step coupling J X_hat restricted to the band: the entries whose column lies in
// the row's 128-vertex tile or in one of its two neighbour tiles).
//
// The CSR step keeps its state vertex-major ([n_pad][R], the replicas of a vertex
// contiguous), so X_hat enters the product as an MN-major B operand: a TMA box of
// 64 replicas x 64 vertices lands as 64 rows of 128 bytes (one vertex per row) with
// the 128-byte swizzle, which is the canonical MN-major layout of tcgen05 (64 MN
// elements per row, 8 K rows per 1024-byte atom).  One CTA per (row tile, 128
// replicas): the three band tiles (A, K-major) and the matching X_hat rows are loaded
// at once, 24 MMAs (M = 128, N = 128, K = 16) accumulate Z in TMEM, and the epilogue
// writes Z[v][r] (FP32, vertex-major) for the CSR step, which adds the remainder.
#include "tc_ptx.cuh"

namespace qh {
namespace {

constexpr uint32_t BAND_A = TILE * 64 * 2;   // 128 rows x 64 K of a band tile (16 KB)
constexpr uint32_t BAND_B = 64 * 128 * 2;    // 64 K (vertices) x 128 replicas (16 KB)
constexpr uint32_t BAND_B_OFF = 6 * BAND_A;  // A: 3 tiles x 2 K-slices, then B likewise
constexpr uint32_t BAND_BAR_OFF = BAND_B_OFF + 6 * BAND_B;
constexpr uint32_t BAND_SMEM = BAND_BAR_OFF + 2 * 8 + 16 + 1024;  // + alignment slack

// MN-major operand with 128-byte swizzle: rows of 128 bytes hold 64 consecutive MN
// elements (replicas) of one K index (vertex); 8 K rows form a 1024-byte atom.
// Leading byte offset: to the next 64 MN elements (the second TMA box, 8 KB on);
// stride byte offset: to the next 8 K rows.
__device__ __forceinline__ uint64_t sdesc_sw128_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(8192 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16: D = F32, A = B = BF16, A K-major, B MN-major (bit 16), N = 128, M = 128.
constexpr uint32_t IDESC_BAND =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(128 >> 3) << 17) |
    ((uint32_t)(128 >> 4) << 24);

__global__ void __launch_bounds__(128, 1) k_band_mma(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB,
                                                     const RowTile* __restrict__ rts,
                                                     int32_t n_row_tiles, int32_t R,
                                                     const int32_t* __restrict__ active,
                                                     const int32_t* __restrict__ steps_b,
                                                     int32_t t, float* __restrict__ z,
                                                     int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAND_BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const uint32_t full = smem_u32(bars), done = smem_u32(bars + 1);

  const int32_t V = blockIdx.x;
  const RowTile rt = rts[V];
  if ((active != nullptr && !active[rt.block]) || (steps_b != nullptr && t >= steps_b[rt.block]))
    return;  // CTA-uniform: the CSR step does not read Z of a frozen block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t r0 = (int32_t)blockIdx.y * 128;
  // band tile d (offset d - 1) exists when the neighbour row tile is in range and in
  // the same block (entries never cross blocks)
  uint32_t dmask = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t U = V + d - 1;
    if (U >= 0 && U < n_row_tiles && (d == 1 || rts[U].block == rt.block)) dmask |= 1u << d;
  }

  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 128u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    uint32_t bytes = 0;
    for (int d = 0; d < 3; ++d)
      if (dmask >> d & 1u) bytes += 2 * (BAND_A + BAND_B);
    mbar_expect_tx(full, bytes);
    for (int d = 0; d < 3; ++d) {
      if (!(dmask >> d & 1u)) continue;
      const int32_t U = V + d - 1;
      for (int s = 0; s < 2; ++s) {
        const uint32_t slot = (uint32_t)(2 * d + s);
        tma_load_2d(smem_u32(smem + slot * BAND_A), &tmA, full, s * 64, (3 * V + d) * TILE);
        for (int h = 0; h < 2; ++h)
          tma_load_2d(smem_u32(smem + BAND_B_OFF + slot * BAND_B + h * (BAND_B / 2)), &tmB, full,
                      r0 + h * 64, U * TILE + s * 64);
      }
    }
    bool ok = mbar_wait(full, 0, err);
    tc_fence_after();
    if (ok) {
      uint32_t acc = 0;
      for (int d = 0; d < 3; ++d) {
        if (!(dmask >> d & 1u)) continue;
        for (int s = 0; s < 2; ++s) {
          const uint32_t slot = (uint32_t)(2 * d + s);
          const uint64_t ad = sdesc_sw128(smem_u32(smem + slot * BAND_A));
          const uint64_t bd = sdesc_sw128_mn(smem_u32(smem + BAND_B_OFF + slot * BAND_B));
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // K = 16 per MMA: A +32 B, B +2 atoms (2048 B)
            mma_bf16(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(128 * k), IDESC_BAND, acc);
            acc = 1u;
          }
        }
      }
    }
    mma_commit(done);  // arrives when the MMAs above (if any) have completed
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0, err);
  tc_fence_after();
  const int row = warp * 32 + lane;
  const bool vrow = ok && row < rt.valid;
  float* zr = z + (size_t)(rt.row0 + row) * R + r0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t v[16];
    __syncwarp();
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
    if (vrow) {
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(zr + c * 16 + j) =
            make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                        __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 128u);
  }
}

}  // namespace

cudaError_t band_set_attrs() {
  return cudaFuncSetAttribute(k_band_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)BAND_SMEM);
}

qh_status launch_band_mma(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* band,
                          const __nv_bfloat16* xh_vm, float* z) {
  if (g.n_row_tiles == 0) return QH_OK;
  if (a.R % 128 != 0) return set_err(ctx, QH_EINVAL, "band product needs R to be a multiple of 128");
  if (a.R / 128 > 65535)  // replica tiles index the grid's y dimension
    return set_err(ctx, QH_EUNSUPPORTED, "band product: more than 65,535 replica tiles");
  CUtensorMap mA, mB;
  if (!make_map(&mA, band, TILE, (uint64_t)3 * g.n_row_tiles * TILE, TILE) ||
      !make_map(&mB, xh_vm, (uint64_t)a.R, (uint64_t)g.n_pad, 64))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed (band product)");
  dim3 grid((unsigned)g.n_row_tiles, (unsigned)(a.R / 128));
  k_band_mma<<<::qh::counted(grid), 128, BAND_SMEM, ctx->stream>>>(
      mA, mB, g.rt, g.n_row_tiles, a.R, a.active, a.z_out != nullptr ? nullptr : a.steps_b, a.t, z,
      a.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_band_mma launch");
  return QH_OK;
}

}  // namespace qh
