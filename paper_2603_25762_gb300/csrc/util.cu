// Scans and a bitonic sort used by the graph build (single-pass, deterministic).
#include <atomic>

#include "qh_internal.cuh"
#include "util.cuh"

namespace qh {

static std::atomic<int64_t> g_launches{0};
void note_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Scans in three passes over tiles of 2,048 elements (coalesced loads): the total (or
// maximum) of each tile, an exclusive scan of those in one CTA, then each tile's own
// scan from its offset.
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <bool MAX>
__device__ __forceinline__ int64_t scan_op(int64_t a, int64_t b) {
  return MAX ? (a > b ? a : b) : a + b;
}

// Block-wide exclusive scan of one value per thread (and the block total).
template <bool MAX>
__device__ __forceinline__ int64_t block_excl(int64_t v, int64_t ident, int64_t* total) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl = scan_op<MAX>(incl, u);
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int64_t before = ident, all = ident;
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    if (w < warp) before = scan_op<MAX>(before, warp_tot[w]);
    all = scan_op<MAX>(all, warp_tot[w]);
  }
  __syncthreads();
  const int64_t excl_in_warp = __shfl_up_sync(0xffffffffu, incl, 1);
  *total = all;
  return lane == 0 ? before : scan_op<MAX>(before, excl_in_warp);
}

template <typename TIn, bool MAX>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_total(const TIn* __restrict__ in,
                                                             int64_t* __restrict__ part, int64_t n,
                                                             int64_t ident) {
  const int64_t b = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t acc = ident;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS)
    if (b + i < n) acc = scan_op<MAX>(acc, (int64_t)in[b + i]);
  int64_t total;
  block_excl<MAX>(acc, ident, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One CTA: part[0..nt) <- exclusive scan; part[nt] <- the grand total.
template <bool MAX>
__global__ void __launch_bounds__(SCAN_THREADS) k_part_scan(int64_t* part, int64_t nt,
                                                            int64_t ident) {
  int64_t carry = ident;
  for (int64_t b = 0; b < nt; b += SCAN_THREADS) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < nt ? part[i] : ident;
    int64_t total;
    const int64_t ex = block_excl<MAX>(v, ident, &total);
    if (i < nt) part[i] = scan_op<MAX>(carry, ex);
    carry = scan_op<MAX>(carry, total);
  }
  if (threadIdx.x == 0) part[nt] = carry;
}

// Each tile from its offset: exclusive (sum, int64 out, out[n] = total) or inclusive
// (max, int32 out).
template <typename TIn, typename TOut, bool MAX>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const TIn* __restrict__ in,
                                                            const int64_t* __restrict__ part,
                                                            TOut* __restrict__ out, int64_t n,
                                                            int64_t nt, int64_t ident) {
  __shared__ int64_t s[SCAN_TILE];
  const int64_t b = (int64_t)blockIdx.x * SCAN_TILE;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS)
    s[i] = b + i < n ? (int64_t)in[b + i] : ident;
  __syncthreads();
  int64_t loc = ident;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) loc = scan_op<MAX>(loc, s[threadIdx.x * SCAN_ITEMS + j]);
  int64_t total;
  int64_t run = scan_op<MAX>(part[blockIdx.x], block_excl<MAX>(loc, ident, &total));
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    const int i = threadIdx.x * SCAN_ITEMS + j;
    const int64_t v = s[i];
    if (MAX) run = scan_op<MAX>(run, v);  // inclusive
    if (b + i < n) out[b + i] = (TOut)run;
    if (!MAX) run += v;  // exclusive
  }
  if (!MAX && blockIdx.x == 0 && threadIdx.x == 0) out[n] = (TOut)part[nt];
}

template <typename TIn, typename TOut, bool MAX>
bool scan3(Ctx* ctx, cudaStream_t s, const TIn* in, TOut* out, int64_t n, int64_t ident) {
  if (n <= 0) {
    if (!MAX) return cudaMemsetAsync(out, 0, sizeof(TOut), s) == cudaSuccess;
    return true;
  }
  const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* part = (int64_t*)ctx->scratch(sizeof(int64_t) * (nt + 1), 24);
  if (part == nullptr) return false;
  k_tile_total<TIn, MAX><<<::qh::counted((unsigned)nt), SCAN_THREADS, 0, s>>>(in, part, n, ident);
  k_part_scan<MAX><<<::qh::counted(1), SCAN_THREADS, 0, s>>>(part, nt, ident);
  k_tile_scan<TIn, TOut, MAX><<<::qh::counted((unsigned)nt), SCAN_THREADS, 0, s>>>(in, part, out, n,
                                                                                  nt, ident);
  return true;
}

// Bitonic sort: global compare-exchange for strides >= 1024, shared-memory
// passes for the inner strides.
__global__ void k_bitonic_global(uint64_t* keys, int64_t n, int64_t k, int64_t j) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t l = i ^ j;
  if (l > i) {
    uint64_t a = keys[i], b = keys[l];
    bool up = (i & k) == 0;
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

constexpr int BSORT_LOCAL = 2048;

__global__ void k_bitonic_local(uint64_t* keys, int64_t n, int64_t k, int64_t jstart) {
  __shared__ uint64_t s[BSORT_LOCAL];
  int64_t base = (int64_t)blockIdx.x * BSORT_LOCAL;
  for (int t = threadIdx.x; t < BSORT_LOCAL; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  for (int64_t kk = (k == 0 ? 2 : k); kk <= (k == 0 ? BSORT_LOCAL : k); kk <<= 1) {
    for (int64_t j = (k == 0 ? kk >> 1 : jstart); j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < BSORT_LOCAL; t += blockDim.x) {
        int l = t ^ (int)j;
        if (l > t) {
          uint64_t a = s[t], b = s[l];
          bool up = ((base + t) & kk) == 0;
          if ((a > b) == up) {
            s[t] = b;
            s[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < BSORT_LOCAL; t += blockDim.x) keys[base + t] = s[t];
}

__global__ void k_fill_u64(uint64_t* p, int64_t b, int64_t e, uint64_t v) {
  int64_t i = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < e) p[i] = v;
}

}  // namespace

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

bool scan_i64(Ctx* ctx, cudaStream_t s, const int64_t* in, int64_t* out, int64_t n) {
  return scan3<int64_t, int64_t, false>(ctx, s, in, out, n, 0);
}
bool scan_i32_to_i64(Ctx* ctx, cudaStream_t s, const int32_t* in, int64_t* out, int64_t n) {
  return scan3<int32_t, int64_t, false>(ctx, s, in, out, n, 0);
}
bool scan_max_i32(Ctx* ctx, cudaStream_t s, const int32_t* in, int32_t* out, int64_t n) {
  return scan3<int32_t, int32_t, true>(ctx, s, in, out, n, (int64_t)INT32_MIN);
}

void sort_u64(cudaStream_t s, uint64_t* keys, int64_t n, int64_t cap) {
  if (n <= 1) return;
  int64_t N = next_pow2(n < BSORT_LOCAL ? BSORT_LOCAL : n);
  (void)cap;
  if (N > n) k_fill_u64<<<::qh::counted((unsigned)((N - n + 255) / 256)), 256, 0, s>>>(keys, n, N, ~0ull);
  unsigned nb_local = (unsigned)(N / BSORT_LOCAL);
  // all stages with k <= BSORT_LOCAL in shared memory
  k_bitonic_local<<<::qh::counted(nb_local), 512, 0, s>>>(keys, N, 0, 0);
  for (int64_t k = 2 * BSORT_LOCAL; k <= N; k <<= 1) {
    for (int64_t j = k >> 1; j >= BSORT_LOCAL; j >>= 1)
      k_bitonic_global<<<::qh::counted((unsigned)((N + 255) / 256)), 256, 0, s>>>(keys, N, k, j);
    k_bitonic_local<<<::qh::counted(nb_local), 512, 0, s>>>(keys, N, k, BSORT_LOCAL >> 1);
  }
}

}  // namespace qh
