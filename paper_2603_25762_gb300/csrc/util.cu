// Scans and a bitonic sort used by the graph build (single-pass, deterministic).
#include <atomic>

#include "qh_internal.cuh"
#include "util.cuh"

namespace qh {

static std::atomic<int64_t> g_launches{0};
void note_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int SCAN_THREADS = 1024;

// One CTA, each thread owns a contiguous chunk: local sums, block scan, write-back.
template <typename TIn>
__global__ void k_scan_excl(const TIn* __restrict__ in, int64_t* __restrict__ out, int64_t n) {
  __shared__ int64_t part[SCAN_THREADS];
  int64_t chunk = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  int64_t b = (int64_t)threadIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += (int64_t)in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t i = b; i < e; ++i) {
    int64_t v = (int64_t)in[i];
    out[i] = run;
    run += v;
  }
  if (threadIdx.x == SCAN_THREADS - 1) out[n] = part[SCAN_THREADS - 1];
}

__global__ void k_scan_max(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  __shared__ int32_t part[SCAN_THREADS];
  int64_t chunk = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  int64_t b = (int64_t)threadIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  int32_t m = INT32_MIN;
  for (int64_t i = b; i < e; ++i) m = max(m, in[i]);
  part[threadIdx.x] = m;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : INT32_MIN;
    __syncthreads();
    part[threadIdx.x] = max(part[threadIdx.x], v);
    __syncthreads();
  }
  int32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : INT32_MIN;
  for (int64_t i = b; i < e; ++i) {
    run = max(run, in[i]);
    out[i] = run;
  }
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

void scan_i64(cudaStream_t s, const int64_t* in, int64_t* out, int64_t n) {
  k_scan_excl<int64_t><<<::qh::counted(1), SCAN_THREADS, 0, s>>>(in, out, n);
}
void scan_i32_to_i64(cudaStream_t s, const int32_t* in, int64_t* out, int64_t n) {
  k_scan_excl<int32_t><<<::qh::counted(1), SCAN_THREADS, 0, s>>>(in, out, n);
}
void scan_max_i32(cudaStream_t s, const int32_t* in, int32_t* out, int64_t n) {
  if (n > 0) k_scan_max<<<::qh::counted(1), SCAN_THREADS, 0, s>>>(in, out, n);
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
