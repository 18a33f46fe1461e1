// Band product of a CSR-mode graph on the tensor cores (SB algorithm solution, the
// per-step coupling J X_hat restricted to the band: the entries whose column lies in
// the row's 128-vertex tile or in one of its two neighbour tiles).
//
// The CSR step keeps its state vertex-major ([n_pad][R], the replicas of a vertex
// contiguous), so X_hat enters the product as an MN-major B operand: a TMA box of
// 64 replicas x 64 vertices lands as 64 rows of 128 bytes (one vertex per row) with
// the 128-byte swizzle, which is the canonical MN-major layout of tcgen05 (64 MN
// elements per row, 8 K rows per 1024-byte atom).  A persistent, warp-specialised
// kernel (one CTA per SM) streams the band tiles (A, K-major) and the matching X_hat
// rows; 8 MMAs per band tile (M = 128, N = 128, K = 16) accumulate Z in TMEM, and the
// epilogue writes Z[v][r] (FP32, vertex-major) for the CSR step, which adds the
// remainder.
#include "tc_ptx.cuh"

namespace qh {
namespace {

constexpr uint32_t BAND_A = TILE * 64 * 2;   // 128 rows x 64 K of a band tile (16 KB)
constexpr uint32_t BAND_B = 64 * 128 * 2;    // 64 K (vertices) x 128 replicas (16 KB)

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

// ---------------------------------------------------------------------------
// One CTA per SM walks (row tile, 128 replicas) items.  A TMA
// warp streams one band tile per stage through a 3-stage ring, an MMA warp
// accumulates an item's tiles into one of two TMEM buffers, and four epilogue warps
// drain the other buffer to Z, so loads, MMAs and stores of successive items overlap.
constexpr int PST = 3;
constexpr uint32_t PSTAGE = 2 * BAND_A + 2 * BAND_B;  // A K-slices 0 / 1, then B K-slices
constexpr uint32_t P_BAR_OFF = PST * PSTAGE;
constexpr uint32_t P_SMEM = P_BAR_OFF + 11 * 8 + 16 + 1024;

// Bounded wait that also gives up once another role of the CTA has given up.
__device__ __forceinline__ bool bwait(uint32_t bar, uint32_t parity, int32_t* err,
                                      volatile int32_t* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (abort != nullptr && *abort) return false;
    if (clock64() - t0 > (1ll << 31)) {
      atomicOr(err, ERR_TIMEOUT);
      if (abort != nullptr) *abort = 1;
      return false;
    }
  }
  return true;
}

__global__ void __launch_bounds__(192, 1) k_band_mma(const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB,
                                                       const RowTile* __restrict__ rts,
                                                       int32_t n_row_tiles, int32_t nrep,
                                                       int32_t R,
                                                       const int32_t* __restrict__ active,
                                                       const int32_t* __restrict__ steps_b,
                                                       int32_t t, float* __restrict__ z,
                                                       int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P_BAR_OFF);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + PST),
                 accf0 = smem_u32(bars + 2 * PST), acce0 = smem_u32(bars + 2 * PST + 2),
                 drain = smem_u32(bars + 2 * PST + 4);
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < PST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);  // the four epilogue warps
    }
    mbar_init(drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_slot), 256u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int32_t* abort = &abort_flag;
  const int32_t n_items = n_row_tiles * nrep;
  // every role walks the same items and tiles: live row tiles, present band tiles
  auto item = [&](int32_t w, int32_t& V, int32_t& rep, uint32_t& dmask) -> bool {
    V = w / nrep;
    rep = w % nrep;
    const RowTile rt = rts[V];
    if ((active != nullptr && !active[rt.block]) ||
        (steps_b != nullptr && t >= steps_b[rt.block]))
      return false;
    dmask = 0;
    for (int d = 0; d < 3; ++d) {
      const int32_t U = V + d - 1;
      if (U >= 0 && U < n_row_tiles && (d == 1 || rts[U].block == rt.block)) dmask |= 1u << d;
    }
    return true;
  };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      uint32_t cnt = 0;
      bool ok = true;
      for (int32_t w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        int32_t V, rep;
        uint32_t dmask;
        if (!item(w, V, rep, dmask)) continue;
        for (int d = 0; d < 3 && ok; ++d) {
          if (!(dmask >> d & 1u)) continue;
          const uint32_t s = cnt % PST, ph = (cnt / PST) & 1u;
          ok = bwait(empty0 + 8 * s, ph ^ 1u, err, abort);
          if (!ok) break;
          uint8_t* sa = smem + s * PSTAGE;
          mbar_expect_tx(full0 + 8 * s, PSTAGE);
          const int32_t U = V + d - 1;
          for (int k = 0; k < 2; ++k) {
            tma_load_2d(smem_u32(sa + k * BAND_A), &tmA, full0 + 8 * s, k * 64, (3 * V + d) * TILE);
            for (int h = 0; h < 2; ++h)
              tma_load_2d(smem_u32(sa + 2 * BAND_A + k * BAND_B + h * (BAND_B / 2)), &tmB,
                          full0 + 8 * s, rep * 128 + h * 64, U * TILE + k * 64);
          }
          ++cnt;
        }
      }
      // copies still in flight land before the CTA leaves
      for (uint32_t c = cnt > (uint32_t)PST ? cnt - PST : 0; c < cnt; ++c)
        bwait(full0 + 8 * (c % PST), (c / PST) & 1u, err, nullptr);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      uint32_t cnt = 0, icount = 0;
      bool ok = true;
      for (int32_t w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        int32_t V, rep;
        uint32_t dmask;
        if (!item(w, V, rep, dmask)) continue;
        const uint32_t ab = icount & 1u, aph = (icount >> 1) & 1u;
        ok = bwait(acce0 + 8 * ab, aph ^ 1u, err, abort);
        if (!ok) break;
        tc_fence_after();
        uint32_t acc = 0;
        for (int d = 0; d < 3 && ok; ++d) {
          if (!(dmask >> d & 1u)) continue;
          const uint32_t s = cnt % PST, ph = (cnt / PST) & 1u;
          ok = bwait(full0 + 8 * s, ph, err, abort);
          if (!ok) break;
          tc_fence_after();
          uint8_t* sa = smem + s * PSTAGE;
          for (int k = 0; k < 2; ++k) {
            const uint64_t ad = sdesc_sw128(smem_u32(sa + k * BAND_A));
            const uint64_t bd = sdesc_sw128_mn(smem_u32(sa + 2 * BAND_A + k * BAND_B));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              mma_bf16(tmem + ab * 128, ad + (uint64_t)(2 * j), bd + (uint64_t)(128 * j),
                       IDESC_BAND, acc);
              acc = 1u;
            }
          }
          mma_commit(empty0 + 8 * s);
          ++cnt;
        }
        if (!ok) break;
        mma_commit(accf0 + 8 * ab);
        ++icount;
      }
      // the tensor cores finish before TMEM is released
      mma_commit(drain);
      bwait(drain, 0, err, nullptr);
    }
  } else {  // ---- epilogue: warps 2..5, TMEM lane quarter warp % 4
    const int q = warp & 3;
    uint32_t icount = 0;
    for (int32_t w = blockIdx.x; w < n_items; w += gridDim.x) {
      int32_t V, rep;
      uint32_t dmask;
      if (!item(w, V, rep, dmask)) continue;
      const uint32_t ab = icount & 1u, aph = (icount >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, bwait(accf0 + 8 * ab, aph, err, abort));
      if (!ok) break;
      tc_fence_after();
      const RowTile rt = rts[V];
      const int row = q * 32 + lane;
      const bool vrow = row < rt.valid;
      float* zr = z + (size_t)(rt.row0 + row) * R + rep * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t v[16];
        __syncwarp();
        tmem_ld16(tmem + ab * 128 + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 16), v);
        if (vrow) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(zr + c * 16 + j) =
                make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * ab);
      ++icount;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 256u);
  }
}

}  // namespace

cudaError_t band_set_attrs() {
  return cudaFuncSetAttribute(k_band_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)P_SMEM);
}

qh_status launch_band_mma(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* band,
                          const __nv_bfloat16* xh_vm, float* z) {
  if (g.n_row_tiles == 0) return QH_OK;
  if (a.R % 128 != 0) return set_err(ctx, QH_EINVAL, "band product needs R to be a multiple of 128");
  if ((int64_t)g.n_row_tiles * (a.R / 128) > INT32_MAX)  // items are counted in int32
    return set_err(ctx, QH_EUNSUPPORTED, "band product: too many (row tile, replica tile) items");
  CUtensorMap mA, mB;
  if (!make_map(&mA, band, TILE, (uint64_t)3 * g.n_row_tiles * TILE, TILE) ||
      !make_map(&mB, xh_vm, (uint64_t)a.R, (uint64_t)g.n_pad, 64))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed (band product)");
  const int32_t nrep = a.R / 128;
  const int64_t n_items = (int64_t)g.n_row_tiles * nrep;
  const unsigned grid = (unsigned)std::min<int64_t>(n_items, ctx->n_sm);
  k_band_mma<<<::qh::counted(grid), 192, P_SMEM, ctx->stream>>>(
      mA, mB, g.rt, g.n_row_tiles, nrep, a.R, a.active, a.z_out != nullptr ? nullptr : a.steps_b,
      a.t, z, a.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_band_mma launch");
  return QH_OK;
}

}  // namespace qh
