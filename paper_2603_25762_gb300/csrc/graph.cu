// Graph construction (read graph and SNP graph), connected
// components (phase blocks) and the padded 128 x 128 J tile layout.
//
// Read graph (read-based Max-Cut graph construction, Eqs. delta / w_ab): for
// every pair of fragments whose SNP ranges intersect, walk the shared SNPs;
// CONFLICT counts opposing alleles, SIGNED sums -M_aj M_bj (W = -M M^T).
// Integer weights, exact.
// SNP graph (SNP-based graph construction, Eq. edge_weight_SNP, Pore-C alpha,
// linkage depth k/10): each SNP row gathers the terms of every fragment that
// covers it, sorts them by (partner SNP, fragment) in shared memory and sums
// each edge in fragment order in FP64 (deterministic, no atomics).
// Components: lock-free union-find hooking the larger root under the smaller,
// so every root is its component's smallest vertex (blocks are numbered in
// that order; singletons are dropped).
#include <algorithm>
#include <cmath>

#include "qh_internal.cuh"
#include "util.cuh"

namespace qh {

namespace {

// ------------------------------------------------------------------ validate
// Warp per fragment, the lanes striding over its entries (each compares its SNP with the
// entry before it).  A fragment range outside [0, nnz] is flagged before any entry of it
// is read.
__global__ void k_validate(int32_t m, int32_t n, int64_t nnz, const int64_t* __restrict__ fp,
                           const int32_t* __restrict__ snp, const int8_t* __restrict__ allele,
                           const uint8_t* __restrict__ qual, int check_qual, int32_t* err) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  int64_t b = fp[i], e = fp[i + 1];
  if (e < b || b < 0 || e > nnz) {
    if (lane == 0) atomicOr(err, ERR_INPUT);
    return;
  }
  for (int64_t k = b + lane; k < e; k += 32) {
    int32_t s = snp[k];
    int8_t a = allele[k];
    if (s < 0 || s >= n || (k > b && s <= snp[k - 1]) || (a != 1 && a != -1))
      atomicOr(err, ERR_INPUT);
    if (check_qual) {
      uint8_t q = qual[k];
      if (q < 4 || q > 93) atomicOr(err, ERR_QUAL);
    }
  }
}

// ------------------------------------------------------------------ coverage (SNP -> fragments)
__global__ void k_cov_count(int64_t nnz, const int32_t* __restrict__ snp, int32_t* cnt) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nnz) atomicAdd(&cnt[snp[k]], 1);
}

// Warp per fragment, the lanes taking its entries in parallel: the order within a SNP's
// list is set afterwards by k_cov_sort.
__global__ void k_cov_fill(int32_t m, const int64_t* __restrict__ fp, const int32_t* __restrict__ snp,
                           const int8_t* __restrict__ allele, const int64_t* __restrict__ cov_ptr,
                           int32_t* cursor, int32_t* cov_frag, int8_t* cov_allele) {
  const int64_t i64 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i64 >= m) return;
  const int32_t i = (int32_t)i64;
  for (int64_t k = fp[i] + (threadIdx.x & 31); k < fp[i + 1]; k += 32) {
    int32_t s = snp[k];
    int64_t slot = cov_ptr[s] + atomicAdd(&cursor[s], 1);
    cov_frag[slot] = i;
    cov_allele[slot] = allele[k];
  }
}

// Sort each SNP's covering list by fragment index.  Warp per SNP: lists of up to
// 256 entries are sorted in the warp's shared-memory slice (bitonic, keys
// fragment << 8 | allele); longer ones (rare) by lane 0 in place.
constexpr int COV_SORT_MAX = 256;

__global__ void __launch_bounds__(256) k_cov_sort(int32_t n, const int64_t* __restrict__ cov_ptr,
                                                  int32_t* cov_frag, int8_t* cov_allele) {
  __shared__ int64_t keys[8][COV_SORT_MAX];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= n) return;
  int64_t b = cov_ptr[s], e = cov_ptr[s + 1];
  int32_t len = (int32_t)(e - b);
  if (len <= 1) return;
  if (len <= COV_SORT_MAX) {
    int32_t N = 2;
    while (N < len) N <<= 1;
    int64_t* k = keys[w];
    for (int i = lane; i < N; i += 32)
      k[i] = i < len ? (((int64_t)cov_frag[b + i] << 8) | (int64_t)(uint8_t)(cov_allele[b + i] + 1))
                     : INT64_MAX;
    __syncwarp();
    for (int kk = 2; kk <= N; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < N; i += 32) {
          int l = i ^ j;
          if (l > i) {
            int64_t a0 = k[i], a1 = k[l];
            bool up = (i & kk) == 0;
            if ((a0 > a1) == up) {
              k[i] = a1;
              k[l] = a0;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int i = lane; i < len; i += 32) {
      cov_frag[b + i] = (int32_t)(k[i] >> 8);
      cov_allele[b + i] = (int8_t)((int32_t)(k[i] & 0xff) - 1);
    }
    return;
  }
  if (lane != 0) return;
  for (int64_t i = b + 1; i < e; ++i) {
    int32_t f = cov_frag[i];
    int8_t a = cov_allele[i];
    int64_t j = i - 1;
    while (j >= b && cov_frag[j] > f) {
      cov_frag[j + 1] = cov_frag[j];
      cov_allele[j + 1] = cov_allele[j];
      --j;
    }
    cov_frag[j + 1] = f;
    cov_allele[j + 1] = a;
  }
}

// ------------------------------------------------------------------ read graph
__global__ void k_first_last(int32_t m, const int64_t* __restrict__ fp, const int32_t* __restrict__ snp,
                             int32_t* first, int32_t* last, uint64_t* keys) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t b = fp[i], e = fp[i + 1];
  int32_t f = (e > b) ? snp[b] : INT32_MAX;
  int32_t l = (e > b) ? snp[e - 1] : -1;
  first[i] = f;
  last[i] = l;
  keys[i] = ((uint64_t)(uint32_t)f << 32) | (uint32_t)i;
}

__global__ void k_unpack_order(int32_t m, const uint64_t* __restrict__ keys, const int32_t* __restrict__ last,
                               int32_t* order, int32_t* sfirst, int32_t* slast) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  int32_t i = (int32_t)(keys[p] & 0xffffffffu);
  order[p] = i;
  sfirst[p] = (int32_t)(keys[p] >> 32);
  slast[p] = last[i];
}

// Exact weight of one fragment pair by walking both sorted SNP lists.
__device__ __forceinline__ int32_t pair_weight(const int32_t* __restrict__ snp,
                                               const int8_t* __restrict__ allele, int64_t ab,
                                               int64_t ae, int64_t bb, int64_t be, int mode) {
  int32_t w = 0;
  while (ab < ae && bb < be) {
    int32_t sa = snp[ab], sb = snp[bb];
    if (sa < sb) {
      ++ab;
    } else if (sa > sb) {
      ++bb;
    } else {
      int prod = (int)allele[ab] * (int)allele[bb];
      w += (mode == QH_WEIGHT_CONFLICT) ? (prod == -1 ? 1 : 0) : -prod;
      ++ab;
      ++bb;
    }
  }
  return w;
}

// Candidate range of fragment a in first-SNP order: q in [lo, hi) with
// sfirst[q] <= last_a (upper bound) and running max of slast >= first_a.
__device__ __forceinline__ void cand_range(int32_t m, const int32_t* sfirst, const int32_t* pmax_last,
                                           int32_t fa, int32_t la, int32_t* lo, int32_t* hi) {
  int32_t l = 0, h = m;
  while (l < h) {
    int32_t mid = (l + h) >> 1;
    if (sfirst[mid] <= la) l = mid + 1; else h = mid;
  }
  *hi = l;
  l = 0;
  h = m;
  while (l < h) {
    int32_t mid = (l + h) >> 1;
    if (pmax_last[mid] >= fa) h = mid; else l = mid + 1;
  }
  *lo = l;
}

// Warp per fragment a: pass 0 counts w != 0 partners, pass 1 writes them in
// first-SNP order (deterministic positions from warp ballots).
// Fragment a's alleles as a dense window over its SNP range (0 where a has no allele),
// in shared memory, when the range spans at most READ_WIN SNPs: a pair's weight is then
// one walk over the other fragment's SNP list with a lookup per SNP, in place of a
// merge of both lists.
constexpr int READ_WIN = 1024;

// Exact weight of the pair (a, b) from a's allele window (SNPs fa .. fa + READ_WIN - 1).
__device__ __forceinline__ int32_t pair_weight_win(const int32_t* __restrict__ snp,
                                                   const int8_t* __restrict__ allele,
                                                   const int8_t* win, int32_t fa, int32_t la,
                                                   int64_t bb, int64_t be, int mode) {
  int32_t w = 0;
  for (int64_t k = bb; k < be; ++k) {
    const int32_t j = snp[k];
    if (j > la) break;  // b's list is sorted
    if (j < fa) continue;
    const int prod = (int)win[j - fa] * (int)allele[k];
    w += (mode == QH_WEIGHT_CONFLICT) ? (prod == -1 ? 1 : 0) : -prod;
  }
  return w;
}

template <int PASS>
__global__ void k_read_edges(int32_t m, const int64_t* __restrict__ fp, const int32_t* __restrict__ snp,
                             const int8_t* __restrict__ allele, const int32_t* __restrict__ first,
                             const int32_t* __restrict__ last, const int32_t* __restrict__ order,
                             const int32_t* __restrict__ sfirst, const int32_t* __restrict__ slast,
                             const int32_t* __restrict__ pmax_last, int mode, int64_t* cnt,
                             const int64_t* __restrict__ row_ptr, int32_t* col, double* w) {
  __shared__ int8_t win_all[256 / 32][READ_WIN];
  int32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= m) return;
  int64_t ab = fp[a], ae = fp[a + 1];
  if (ae == ab) {
    if (PASS == 0 && lane == 0) cnt[a] = 0;
    return;
  }
  int32_t fa = first[a], la = last[a];
  int8_t* win = win_all[threadIdx.x >> 5];
  const bool use_win = la - fa < READ_WIN;  // warp-uniform
  if (use_win) {
    for (int32_t j = lane; j <= la - fa; j += 32) win[j] = 0;
    __syncwarp();
    for (int64_t k = ab + lane; k < ae; k += 32) win[snp[k] - fa] = allele[k];
    __syncwarp();
  }
  int32_t lo, hi;
  cand_range(m, sfirst, pmax_last, fa, la, &lo, &hi);
  int64_t count = 0;
  int64_t out = PASS == 1 ? row_ptr[a] : 0;
  for (int32_t q0 = lo; q0 < hi; q0 += 32) {
    int32_t q = q0 + lane;
    int32_t wv = 0;
    int32_t b = -1;
    if (q < hi) {
      b = order[q];
      if (b != a && slast[q] >= fa && sfirst[q] <= la)
        wv = use_win ? pair_weight_win(snp, allele, win, fa, la, fp[b], fp[b + 1], mode)
                     : pair_weight(snp, allele, ab, ae, fp[b], fp[b + 1], mode);
    }
    unsigned mask = __ballot_sync(0xffffffffu, wv != 0);
    if (PASS == 1 && wv != 0) {
      int64_t pos = out + __popc(mask & ((1u << lane) - 1));
      col[pos] = b;
      w[pos] = (double)wv;
    }
    out += __popc(mask);
    count += __popc(mask);
  }
  if (PASS == 0 && lane == 0) cnt[a] = count;
}

// ------------------------------------------------------------------ SNP graph
__global__ void k_llr_table(double* L) {
  int qa = blockIdx.x, qb = threadIdx.x;
  if (qa > 93 || qb > 93) return;
  double ua = 1.0 - exp10(-(double)qa / 10.0);
  double ub = 1.0 - exp10(-(double)qb / 10.0);
  double pcis = ua * ub + (1.0 - ua) * (1.0 - ub);
  double ptrans = ua * (1.0 - ub) + (1.0 - ua) * ub;
  L[qa * 94 + qb] = log10(pcis / ptrans);
}

struct SnpRowSmem {
  uint64_t key[SNP_ROW_CAP];   // (partner SNP << 32) | fragment
  double val[SNP_ROW_CAP];
};

// The small kernel's capacities: a dense window of this many SNPs, else this many
// fragment terms on the sorted path (both fit its 32 KB of shared memory).
constexpr int SNP_SMALL_CAP = 2048;
constexpr int SNP_SMALL_TERMS = 2048;
constexpr size_t SNP_SMALL_SMEM = (size_t)SNP_SMALL_TERMS * 16;

// CTA per SNP row u.  PASS 0: count distinct partners; PASS 1: write (v, w_uv).
// A row with a narrow window of covered SNPs sums into a dense window; otherwise its
// fragment terms are gathered and sorted by (partner, fragment).  SMALL: capacities
// SNP_SMALL_CAP / SNP_SMALL_TERMS in a small shared-memory footprint (many CTAs per
// SM); a row over them is appended to `defer` in PASS 0 and left to the large kernel
// (SNP_DENSE_CAP / SNP_ROW_CAP), which walks the deferred rows (`rows`, `n_list` of
// them).  Every path sums a partner's terms in fragment order: the same weights.
template <int PASS, bool SMALL>
__global__ void __launch_bounds__(SMALL ? 256 : 512) k_snp_rows(
    int32_t n, const int64_t* __restrict__ fp, const int32_t* __restrict__ snp,
    const int8_t* __restrict__ allele, const uint8_t* __restrict__ qual,
    const uint8_t* __restrict__ is_porec, const int64_t* __restrict__ cov_ptr,
    const int32_t* __restrict__ cov_frag, const double* __restrict__ L, double alpha,
    int linkage_k, int64_t* cnt, const int64_t* __restrict__ row_ptr, int32_t* col, double* w,
    int32_t* err, const int32_t* __restrict__ rows, const int32_t* __restrict__ n_list,
    int32_t* defer, int32_t* n_defer) {
  constexpr int DCAP = SMALL ? SNP_SMALL_CAP : SNP_DENSE_CAP;
  constexpr int TCAP = SMALL ? SNP_SMALL_TERMS : SNP_ROW_CAP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int32_t s_total;
  __shared__ int32_t s_runs[32];
  __shared__ int32_t s_w0, s_w1;
  __shared__ int32_t s_off[1025];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem_raw);       // sorted path: TCAP keys
  double* sval = reinterpret_cast<double*>(smem_raw) + TCAP;    // and their terms
  const int32_t count = rows != nullptr ? *n_list : n;
  for (int32_t ri = blockIdx.x; ri < count; ri += gridDim.x) {
    const int32_t u = rows != nullptr ? rows[ri] : ri;
    int64_t cb = cov_ptr[u], ce = cov_ptr[u + 1];
    int32_t ncov = (int32_t)(ce - cb);
    // SNP window spanned by the covering fragments
    if (threadIdx.x == 0) {
      s_w0 = INT32_MAX;
      s_w1 = -1;
      s_total = 0;
    }
    __syncthreads();
    {
      int32_t w0 = INT32_MAX, w1 = -1;
      for (int32_t c = threadIdx.x; c < ncov; c += blockDim.x) {
        int32_t i = cov_frag[cb + c];
        w0 = min(w0, snp[fp[i]]);
        w1 = max(w1, snp[fp[i + 1] - 1]);
      }
      if (w1 >= 0) {
        atomicMin(&s_w0, w0);
        atomicMax(&s_w1, w1);
      }
    }
    __syncthreads();
    const int32_t w0 = s_w0, W = s_w1 - s_w0 + 1;
    if (ncov > 0 && W <= DCAP) {
      // Dense window: acc[v - w0] summed fragment by fragment in fragment order (the
      // partners of one fragment are distinct, so its terms go in parallel).  The
      // counting pass needs only which partners occur.
      double* acc = reinterpret_cast<double*>(smem_raw);
      uint8_t* touched = reinterpret_cast<uint8_t*>(acc + DCAP);
      for (int32_t t = threadIdx.x; t < W; t += blockDim.x) {
        acc[t] = 0.0;
        touched[t] = 0;
      }
      __syncthreads();
      for (int32_t c = 0; c < ncov; ++c) {
        const int32_t i = cov_frag[cb + c];
        const int64_t fb = fp[i], fe = fp[i + 1];
        const int32_t S = (int32_t)(fe - fb);
        const int32_t depth = (int32_t)(((int64_t)linkage_k * (S - 1)) / 10);
        int64_t l = fb, h = fe;
        while (l < h) {
          int64_t mid = (l + h) >> 1;
          if (snp[mid] < u) l = mid + 1; else h = mid;
        }
        const int32_t p = (int32_t)(l - fb);
        const int32_t lo = max(0, p - depth), hi = min(S - 1, p + depth);
        const int64_t eu = fb + p;
        const double a = (is_porec != nullptr && is_porec[i]) ? alpha : 1.0;
        for (int32_t pp = lo + threadIdx.x; pp <= hi; pp += blockDim.x) {
          if (pp == p) continue;
          const int64_t ev = fb + pp;
          const int32_t k = snp[ev] - w0;
          touched[k] = 1;
          if (PASS == 0) continue;
          const double lv = L[(int)qual[eu] * 94 + (int)qual[ev]];
          const double sg = ((int)allele[eu] * (int)allele[ev] > 0) ? 1.0 : -1.0;
          const double term = -(a * (sg * lv)) / (double)(S - 1);
          acc[k] += term;
        }
        __syncthreads();
      }
      // compaction in ascending partner order: per-thread contiguous chunk + block scan
      const int32_t chunk = (W + blockDim.x - 1) / blockDim.x;
      const int32_t t0 = threadIdx.x * chunk, t1 = min(W, t0 + chunk);
      int32_t mine = 0;
      for (int32_t t = t0; t < t1; ++t) mine += touched[t];
      // block exclusive scan of `mine` (warp shuffles, then the warp totals)
      int32_t incl = mine;
      for (int off = 1; off < 32; off <<= 1) {
        int32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if ((threadIdx.x & 31) >= off) incl += v;
      }
      if ((threadIdx.x & 31) == 31) s_runs[threadIdx.x >> 5] = incl;
      __syncthreads();
      int32_t warp_before = 0, total = 0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
        if (wi < (int)(threadIdx.x >> 5)) warp_before += s_runs[wi];
        total += s_runs[wi];
      }
      if (PASS == 1) {
        int64_t out = row_ptr[u] + warp_before + incl - mine;
        for (int32_t t = t0; t < t1; ++t)
          if (touched[t]) {
            col[out] = w0 + t;
            w[out] = acc[t];
            ++out;
          }
      } else if (threadIdx.x == 0) {
        cnt[u] = total;
      }
      __syncthreads();
      continue;
    }
    // per covering fragment: number of partners inside the linkage window
    int32_t base = 0;
    for (int32_t c0 = 0; c0 < ncov; c0 += 1024) {
      int32_t cn = min(1024, ncov - c0);
      for (int32_t c = threadIdx.x; c < cn; c += blockDim.x) {
        int32_t i = cov_frag[cb + c0 + c];
        int64_t fb = fp[i], fe = fp[i + 1];
        int32_t S = (int32_t)(fe - fb);
        int32_t depth = (int32_t)(((int64_t)linkage_k * (S - 1)) / 10);
        // position of u inside fragment i (binary search, SNPs ascending)
        int64_t l = fb, h = fe;
        while (l < h) {
          int64_t mid = (l + h) >> 1;
          if (snp[mid] < u) l = mid + 1; else h = mid;
        }
        int32_t p = (int32_t)(l - fb);
        int32_t lo = max(0, p - depth), hi = min(S - 1, p + depth);
        s_off[c + 1] = hi - lo;  // partners (window minus u itself)
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_off[0] = 0;
        for (int32_t c = 0; c < cn; ++c) s_off[c + 1] += s_off[c];
      }
      __syncthreads();
      int32_t tot = s_off[cn];
      if (base + tot > TCAP) {  // small kernel: the large kernel's row; large: error
        if (threadIdx.x == 0 && !SMALL) atomicOr(err, ERR_ROWCAP);
        base = TCAP + 1;
        __syncthreads();
        break;
      }
      // fill terms: thread per (fragment, partner)
      for (int32_t t = threadIdx.x; t < tot; t += blockDim.x) {
        int32_t lo = 0, hi = cn;
        while (hi - lo > 1) {
          int32_t mid = (lo + hi) >> 1;
          if (s_off[mid] <= t) lo = mid; else hi = mid;
        }
        int32_t c = lo, k = t - s_off[c];
        int32_t i = cov_frag[cb + c0 + c];
        int64_t fb = fp[i], fe = fp[i + 1];
        int32_t S = (int32_t)(fe - fb);
        int32_t depth = (int32_t)(((int64_t)linkage_k * (S - 1)) / 10);
        int64_t l = fb, h = fe;
        while (l < h) {
          int64_t mid = (l + h) >> 1;
          if (snp[mid] < u) l = mid + 1; else h = mid;
        }
        int32_t p = (int32_t)(l - fb);
        int32_t wlo = max(0, p - depth);
        int32_t pp = wlo + k;
        if (pp >= p) ++pp;  // skip u itself
        int64_t eu = fb + p, ev = fb + pp;
        int32_t v = snp[ev];
        double lv = L[(int)qual[eu] * 94 + (int)qual[ev]];
        double sg = ((int)allele[eu] * (int)allele[ev] > 0) ? 1.0 : -1.0;
        double a = (is_porec != nullptr && is_porec[i]) ? alpha : 1.0;
        double term = -(a * (sg * lv)) / (double)(S - 1);
        skey[base + t] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)i;
        sval[base + t] = term;
      }
      base += tot;
      __syncthreads();
    }
    if (base > TCAP) {
      if (SMALL) {
        if (PASS == 0 && threadIdx.x == 0) defer[atomicAdd(n_defer, 1)] = u;
      } else if (PASS == 0 && threadIdx.x == 0) {
        cnt[u] = 0;
      }
      __syncthreads();
      continue;
    }
    int32_t total = base;
    int32_t N = 1;
    while (N < total) N <<= 1;
    for (int32_t t = total + threadIdx.x; t < N; t += blockDim.x) {
      skey[t] = ~0ull;
      sval[t] = 0.0;
    }
    __syncthreads();
    // bitonic sort of (key, val) by key
    for (int32_t k = 2; k <= N; k <<= 1) {
      for (int32_t j = k >> 1; j > 0; j >>= 1) {
        for (int32_t t = threadIdx.x; t < N; t += blockDim.x) {
          int32_t l = t ^ j;
          if (l > t) {
            uint64_t ka = skey[t], kb = skey[l];
            bool up = (t & k) == 0;
            if ((ka > kb) == up) {
              skey[t] = kb;
              skey[l] = ka;
              double va = sval[t];
              sval[t] = sval[l];
              sval[l] = va;
            }
          }
        }
        __syncthreads();
      }
    }
    // runs of equal partner: run starts, counted in order
    int64_t out = PASS == 1 ? row_ptr[u] : 0;
    int32_t done = 0;
    for (int32_t t0 = 0; t0 < total; t0 += blockDim.x) {
      int32_t t = t0 + threadIdx.x;
      bool start = t < total && (t == 0 || (skey[t] >> 32) != (skey[t - 1] >> 32));
      unsigned bal = __ballot_sync(0xffffffffu, start);
      if ((threadIdx.x & 31) == 0) s_runs[threadIdx.x >> 5] = __popc(bal);
      __syncthreads();
      int32_t before = 0, chunk_runs = 0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
        if (wi < (int)(threadIdx.x >> 5)) before += s_runs[wi];
        chunk_runs += s_runs[wi];
      }
      before += __popc(bal & ((1u << (threadIdx.x & 31)) - 1));
      if (PASS == 1 && start) {
        double acc = 0.0;
        uint32_t v = (uint32_t)(skey[t] >> 32);
        for (int32_t q = t; q < total && (uint32_t)(skey[q] >> 32) == v; ++q) acc += sval[q];
        col[out + done + before] = (int32_t)v;
        w[out + done + before] = acc;
      }
      done += chunk_runs;
      __syncthreads();
    }
    if (PASS == 0 && threadIdx.x == 0) cnt[u] = done;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ components
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
  while (true) {
    int32_t p = parent[x];
    if (p == x) return x;
    int32_t gp = parent[p];
    if (gp != p) parent[x] = gp;  // path halving; gp is an ancestor, never larger
    x = p;
  }
}

__global__ void k_uf_init(int32_t n, int32_t* parent) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) parent[v] = v;
}

// Union of the sets of x and y: the larger root is hooked under the smaller, so every
// component ends with its smallest vertex as root, whatever order the unions run in.
__device__ __forceinline__ void uf_union(int32_t* parent, int32_t x, int32_t y) {
  while (true) {
    x = uf_find(parent, x);
    y = uf_find(parent, y);
    if (x == y) return;
    if (x < y) {
      int32_t t = x;
      x = y;
      y = t;
    }
    // x > y: hook root x under y.  A failed CAS returns x's current parent, read at
    // L2: continue from there, so that a stale root cached in this SM's L1 cannot make
    // the loop retry forever (each retry starts from a strictly smaller vertex).
    const int32_t old = atomicCAS(&parent[x], x, y);
    if (old == x) return;
    x = old;
  }
}

// Components by subgraph sampling (Sutton, Ben-Nun & Barak, "Optimizing parallel graph
// connectivity computation via subgraph sampling", IPDPS 2018): each vertex first links
// its first UF_LINK_FIRST adjacency entries; a sample of the vertices then names the
// largest component so far; only vertices outside it go through their other entries.
// An entry (a, b) past a's first ones is taken by a when b > a or b is in the sampled
// component, so every edge not already inside that component is taken by at least one
// endpoint (or by a phase-one link), and the partition is the one all edges give.
constexpr int UF_LINK_FIRST = 2;
constexpr int UF_SAMPLES = 256;

__global__ void k_uf_link_first(int32_t n, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const double* __restrict__ w,
                                int32_t* parent) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int64_t e1 = min(rp[a] + UF_LINK_FIRST, rp[a + 1]);
  for (int64_t e = rp[a]; e < e1; ++e) {
    const int32_t b = col[e];
    if (b != a && w[e] != 0.0) uf_union(parent, a, b);
  }
}

// One block of UF_SAMPLES threads: the root that most of the evenly spaced sample
// vertices reach (ties to the larger root; any choice is correct).
__global__ void __launch_bounds__(UF_SAMPLES) k_uf_sample(int32_t n, int32_t* parent,
                                                          int32_t* giant) {
  __shared__ int32_t roots[UF_SAMPLES];
  __shared__ unsigned long long best;
  const int i = threadIdx.x;
  const int64_t v = n >= UF_SAMPLES ? (int64_t)i * n / UF_SAMPLES : (i < n ? i : -1);
  const int32_t r = v >= 0 ? uf_find(parent, (int32_t)v) : -1;
  roots[i] = r;
  if (i == 0) best = 0ull;
  __syncthreads();
  if (r >= 0) {
    uint32_t c = 0;
    for (int j = 0; j < UF_SAMPLES; ++j) c += roots[j] == r ? 1u : 0u;
    atomicMax(&best, ((unsigned long long)c << 32) | (uint32_t)r);
  }
  __syncthreads();
  if (i == 0) giant[0] = best != 0ull ? (int32_t)(best & 0xFFFFFFFFull) : -1;
}

__global__ void k_uf_flag(int32_t n, int32_t* parent, const int32_t* __restrict__ giant,
                          int32_t* in_giant) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) in_giant[v] = uf_find(parent, v) == giant[0] ? 1 : 0;
}

__global__ void k_uf_link_rest(int32_t n, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ col, const double* __restrict__ w,
                               const int32_t* __restrict__ in_giant, int32_t* parent) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n || in_giant[a]) return;
  const int64_t e1 = rp[a + 1];
  for (int64_t e = rp[a] + UF_LINK_FIRST; e < e1; ++e) {
    const int32_t b = col[e];
    if (b == a || (b < a && !in_giant[b]) || w[e] == 0.0) continue;
    uf_union(parent, a, b);
  }
}

__global__ void k_uf_compress(int32_t n, int32_t* parent, int32_t* label, int32_t* size) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t r = uf_find(parent, v);
  label[v] = r;
  atomicAdd(&size[r], 1);
}

__global__ void k_block_roots(int32_t n, const int32_t* __restrict__ label, const int32_t* __restrict__ size,
                              int32_t* is_root) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) is_root[v] = (label[v] == v && size[v] >= 2) ? 1 : 0;
}

__global__ void k_block_of(int32_t n, const int32_t* __restrict__ label, const int32_t* __restrict__ size,
                           const int64_t* __restrict__ root_rank, int32_t* block_of,
                           uint64_t* keys) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t r = label[v];
  int32_t b = size[r] >= 2 ? (int32_t)root_rank[r] : -1;
  block_of[v] = b;
  keys[v] = b >= 0 ? (((uint64_t)(uint32_t)b << 32) | (uint32_t)v) : ~0ull;
}

__global__ void k_block_sizes(int32_t n, const int32_t* __restrict__ label, const int32_t* __restrict__ size,
                              const int64_t* __restrict__ root_rank, int32_t* bsize) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && label[v] == v && size[v] >= 2) bsize[root_rank[v]] = size[v];
}

__global__ void k_perm_local(int64_t total, const uint64_t* __restrict__ keys,
                             const int64_t* __restrict__ block_ptr, const int32_t* __restrict__ pad_off,
                             int32_t* perm, int32_t* local, int32_t* pad_index, int32_t* pad_node) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= total) return;
  int32_t v = (int32_t)(keys[k] & 0xffffffffu);
  int32_t b = (int32_t)(keys[k] >> 32);
  int32_t l = (int32_t)(k - block_ptr[b]);
  perm[k] = v;
  local[v] = l;
  pad_index[v] = pad_off[b] + l;
  pad_node[pad_off[b] + l] = v;
}

// ------------------------------------------------------------------ tiles
__global__ void k_tile_flags(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double* __restrict__ w, const int32_t* __restrict__ block_of,
                             const int32_t* __restrict__ local, const int64_t* __restrict__ slot_off,
                             const int32_t* __restrict__ tiles_per_block, int32_t* flags) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0) return;
  int32_t T = tiles_per_block[b];
  int32_t ra = local[a] / TILE;
  for (int64_t e = rp[a]; e < rp[a + 1]; ++e) {
    if (w[e] == 0.0) continue;
    int32_t cb = local[col[e]] / TILE;
    flags[slot_off[b] + (int64_t)ra * T + cb] = 1;
  }
}

}  // namespace

// Padded CSR of J = -w: rows in padded order, columns as padded indices.
__global__ void k_pcsr_count(int32_t n, const int64_t* __restrict__ rp, const double* __restrict__ w,
                             const int32_t* __restrict__ pad_index, int64_t* cnt) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;  // warp per vertex
  const int lane = threadIdx.x & 31;
  if (a >= n || pad_index[a] < 0) return;  // warp-uniform
  int64_t c = 0;
  const int64_t e1 = rp[a + 1];
  for (int64_t e0 = rp[a]; e0 < e1; e0 += 32)
    c += __popc(__ballot_sync(0xffffffffu, e0 + lane < e1 && w[e0 + lane] != 0.0));
  if (lane == 0) cnt[pad_index[a]] = c;
}

// Warp per vertex: the lanes take 32 entries of the row at a time and write its nonzeros
// in row order (a ballot gives each lane its place among them), so the stores coalesce.
__global__ void k_pcsr_fill(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ pad_index,
                            const int64_t* __restrict__ prow, int32_t* pcol, float* pval) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n || pad_index[a] < 0) return;  // warp-uniform
  int64_t o = prow[pad_index[a]];
  const int64_t e1 = rp[a + 1];
  for (int64_t e0 = rp[a]; e0 < e1; e0 += 32) {
    const int64_t e = e0 + lane;
    const double wv = e < e1 ? w[e] : 0.0;
    const uint32_t nz = __ballot_sync(0xffffffffu, wv != 0.0);
    if (wv != 0.0) {
      const int64_t q = o + __popc(nz & ((1u << lane) - 1u));
      if (pcol != nullptr) pcol[q] = pad_index[col[e]];
      pval[q] = (float)(-wv);
    }
    o += __popc(nz);
  }
}

// Band / remainder split of the padded CSR (CSR mode): entry (v, u) lies in the band
// when the column tile of u is the row tile of v or one of its two neighbours.
__device__ __forceinline__ int band_offset(int32_t v, int32_t u) { return u / TILE - v / TILE; }

// The band / remainder kernels below run a warp per vertex, the lanes taking 32 entries
// of the row at a time; the remainder keeps the row order through a ballot.
__global__ void k_rem_count(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ pad_index,
                            int64_t* cnt) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n || pad_index[a] < 0) return;  // warp-uniform
  const int32_t v = pad_index[a];
  int64_t c = 0;
  const int64_t e1 = rp[a + 1];
  for (int64_t e0 = rp[a]; e0 < e1; e0 += 32) {
    const int64_t e = e0 + lane;
    bool rem = false;
    if (e < e1 && w[e] != 0.0) {
      const int d = band_offset(v, pad_index[col[e]]);
      rem = d < -1 || d > 1;
    }
    c += __popc(__ballot_sync(0xffffffffu, rem));
  }
  if (lane == 0) cnt[v] = c;
}

__global__ void k_rem_fill(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ w, const int32_t* __restrict__ pad_index,
                           const int64_t* __restrict__ rrow, int32_t* rcol, float* rval) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n || pad_index[a] < 0) return;  // warp-uniform
  const int32_t v = pad_index[a];
  int64_t o = rrow[v];
  const int64_t e1 = rp[a + 1];
  for (int64_t e0 = rp[a]; e0 < e1; e0 += 32) {
    const int64_t e = e0 + lane;
    bool rem = false;
    int32_t u = 0;
    double wv = 0.0;
    if (e < e1) {
      wv = w[e];
      if (wv != 0.0) {
        u = pad_index[col[e]];
        const int d = band_offset(v, u);
        rem = d < -1 || d > 1;
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, rem);
    if (rem) {
      const int64_t q = o + __popc(m & ((1u << lane) - 1u));
      if (rcol != nullptr) rcol[q] = u;
      rval[q] = (float)(-wv);
    }
    o += __popc(m);
  }
}

// band[(rt * 3 + d + 1)][v % 128][u % 128] = BF16(-w) for band entries (zeroed before)
__global__ void k_band_fill(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ pad_index,
                            __nv_bfloat16* band) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n || pad_index[a] < 0) return;
  const int32_t v = pad_index[a];
  for (int64_t e = rp[a] + lane; e < rp[a + 1]; e += 32) {
    if (w[e] == 0.0) continue;
    const int32_t u = pad_index[col[e]];
    const int d = band_offset(v, u);
    if (d < -1 || d > 1) continue;
    const int64_t t = (int64_t)(v / TILE) * 3 + (d + 1);
    band[t * TILE * TILE + (int64_t)(v % TILE) * TILE + (u % TILE)] = __float2bfloat16_rn((float)(-w[e]));
  }
}

// Tile fill (also used after a refinement sign inversion): J = -w into the
// FP32 tiles and the BF16 hi (+ lo remainder) tiles.
// Warp per vertex, the lanes striding over the row: neighbouring entries of a row land
// in neighbouring columns of a tile row, so the stores of a warp coalesce.
__global__ void k_tile_fill(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ block_of,
                            const int32_t* __restrict__ local, const int64_t* __restrict__ slot_off,
                            const int32_t* __restrict__ tiles_per_block,
                            const int64_t* __restrict__ slot_tile, const RowTile* __restrict__ rt,
                            const int32_t* __restrict__ rt_of_block, int has_lo,
                            __nv_bfloat16* tb, float* tf) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= n) return;
  int32_t b = block_of[a];
  if (b < 0) return;
  int32_t T = tiles_per_block[b];
  int32_t la = local[a];
  int32_t ra = la / TILE;
  const RowTile& r = rt[rt_of_block[b] + ra];
  for (int64_t e = rp[a] + lane; e < rp[a + 1]; e += 32) {
    double wv = w[e];
    if (wv == 0.0) continue;
    int32_t lb = local[col[e]];
    int64_t slot = slot_off[b] + (int64_t)ra * T + lb / TILE;
    int64_t h = slot_tile[slot];                  // hi tile id (FP32 tiles)
    int64_t j = h - slot_tile[slot_off[b] + (int64_t)ra * T];  // index inside the row
    int64_t off = (int64_t)(la % TILE) * TILE + (lb % TILE);
    double J = -wv;
    tf[h * (int64_t)(TILE * TILE) + off] = (float)J;
    __nv_bfloat16 hi = __double2bfloat16(J);
    tb[(r.tile_begin + j) * (int64_t)(TILE * TILE) + off] = hi;
    if (has_lo) {
      __nv_bfloat16 lo = __double2bfloat16(J - (double)__bfloat162float(hi));
      tb[(r.tile_begin + r.n_hi + j) * (int64_t)(TILE * TILE) + off] = lo;
    }
  }
}

namespace {

// Largest |w| and whether any weight is non-integer: block reduction, one atomic per CTA.
__global__ void k_abs_max(int64_t nnz, const double* __restrict__ w, unsigned long long* out,
                          int32_t* nonint) {
  __shared__ double sm[256];
  __shared__ int32_t sn;
  if (threadIdx.x == 0) sn = 0;
  double m = 0.0;
  int32_t ni = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = fabs(w[e]);
    m = fmax(m, v);
    ni |= (v != floor(v)) ? 1 : 0;
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  if (ni) sn = 1;
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));  // non-negative doubles order as ints
    if (sn) atomicOr(nonint, 1);
  }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

qh_status build_graph_device(Ctx* ctx, const qh_fragments* f, const qh_graph_opts* o, Graph* g) {
  cudaStream_t s = ctx->stream;
  const int32_t m = f->n_frags, n = f->n_snps;
  g->mode = o->mode;
  g->weight_mode = o->weight_mode;
  g->linkage_k = o->linkage_k;
  g->porec_alpha = o->porec_alpha;
  g->n_frags = m;
  g->n_snps = n;
  // ---- copy fragments to the device
  cudaMemcpyKind kind = f->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int64_t nnz_f = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&nnz_f, f->frag_ptr + m, sizeof(int64_t),
                              f->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  int64_t fp0 = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&fp0, f->frag_ptr, sizeof(int64_t),
                              f->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  if (fp0 != 0 || nnz_f < 0) return set_err(ctx, QH_EINVAL, "frag_ptr[0] must be 0 and frag_ptr[m] >= 0");
  g->nnz_frag = nnz_f;
  g->frag_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (m + 1));
  g->snp = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(nnz_f, 1));
  g->allele = (int8_t*)dalloc(*g, std::max<int64_t>(nnz_f, 1));
  g->qual = (uint8_t*)dalloc(*g, std::max<int64_t>(nnz_f, 1));
  g->is_porec = (uint8_t*)dalloc(*g, std::max<int32_t>(m, 1));
  if (!g->frag_ptr || !g->snp || !g->allele || !g->qual || !g->is_porec)
    return set_err(ctx, QH_ENOMEM, "device allocation failed (fragments)");
  QH_CUDA_TRY(cudaMemcpyAsync(g->frag_ptr, f->frag_ptr, sizeof(int64_t) * (m + 1), kind, s));
  if (nnz_f > 0) {
    QH_CUDA_TRY(cudaMemcpyAsync(g->snp, f->snp, sizeof(int32_t) * nnz_f, kind, s));
    QH_CUDA_TRY(cudaMemcpyAsync(g->allele, f->allele, nnz_f, kind, s));
    if (f->qual)
      QH_CUDA_TRY(cudaMemcpyAsync(g->qual, f->qual, nnz_f, kind, s));
    else
      QH_CUDA_TRY(cudaMemsetAsync(g->qual, 30, nnz_f, s));
  }
  if (f->is_porec && m > 0)
    QH_CUDA_TRY(cudaMemcpyAsync(g->is_porec, f->is_porec, m, kind, s));
  else
    QH_CUDA_TRY(cudaMemsetAsync(g->is_porec, 0, std::max<int32_t>(m, 1), s));
  // ---- validate
  QH_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
  if (m > 0)
    k_validate<<<::qh::counted(nblk((int64_t)m * 32)), 256, 0, s>>>(m, n, nnz_f, g->frag_ptr, g->snp, g->allele, g->qual,
                                       o->mode == QH_MODE_SNP && f->qual != nullptr ? 1 : 0,
                                       ctx->d_err);
  int32_t herr = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr & ERR_INPUT)
    return set_err(ctx, QH_EINVAL,
                   "malformed fragments (SNP out of range, not strictly increasing, or allele not +-1)");
  if (herr & ERR_QUAL) return set_err(ctx, QH_EINVAL, "Phred quality outside [4, 93]");
  QH_STAGE_CHECK("graph build: validate");
  // ---- SNP -> fragment coverage lists (used by SNP rows and by voting)
  {
    int32_t* cnt = (int32_t*)ctx->scratch(sizeof(int32_t) * (n + 1), 0);
    if (!cnt) return set_err(ctx, QH_ENOMEM, "allocation failed (coverage)");
    QH_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s));
    if (nnz_f > 0) k_cov_count<<<::qh::counted(nblk(nnz_f)), 256, 0, s>>>(nnz_f, g->snp, cnt);
    g->cov_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (n + 1));
    g->cov_frag = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(nnz_f, 1));
    g->cov_allele = (int8_t*)dalloc(*g, std::max<int64_t>(nnz_f, 1));
    if (!g->cov_ptr || !g->cov_frag || !g->cov_allele) return set_err(ctx, QH_ENOMEM, "allocation failed (coverage)");
    if (!scan_i32_to_i64(ctx, s, cnt, g->cov_ptr, n)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
    QH_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s));
    if (m > 0)
      k_cov_fill<<<::qh::counted(nblk((int64_t)m * 32)), 256, 0, s>>>(m, g->frag_ptr, g->snp, g->allele, g->cov_ptr, cnt,
                                         g->cov_frag, g->cov_allele);
    if (n > 0) k_cov_sort<<<::qh::counted(nblk((int64_t)n * 32)), 256, 0, s>>>(n, g->cov_ptr, g->cov_frag, g->cov_allele);
  }
  QH_STAGE_CHECK("graph build: coverage lists");
  // ---- edges
  if (o->mode == QH_MODE_READ) {
    g->n_nodes = m;
    int64_t cap = next_pow2(std::max<int64_t>(m, 2048));
    int32_t* first = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 1);
    int32_t* last = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 2);
    uint64_t* keys = (uint64_t*)ctx->scratch(sizeof(uint64_t) * cap, 3);
    int32_t* order = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 4);
    int32_t* sfirst = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 5);
    int32_t* slast = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 6);
    int32_t* pmax = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(m, 1), 7);
    int64_t* cnt = (int64_t*)ctx->scratch(sizeof(int64_t) * (m + 1), 8);
    if (!first || !last || !keys || !order || !sfirst || !slast || !pmax || !cnt)
      return set_err(ctx, QH_ENOMEM, "allocation failed (read graph scratch)");
    g->row_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (m + 1));
    if (!g->row_ptr) return set_err(ctx, QH_ENOMEM, "allocation failed (edges)");
    if (m > 0) {
      k_first_last<<<::qh::counted(nblk(m)), 256, 0, s>>>(m, g->frag_ptr, g->snp, first, last, keys);
      sort_u64(s, keys, m, cap);
      k_unpack_order<<<::qh::counted(nblk(m)), 256, 0, s>>>(m, keys, last, order, sfirst, slast);
      if (!scan_max_i32(ctx, s, slast, pmax, m)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
      k_read_edges<0><<<::qh::counted(nblk((int64_t)m * 32)), 256, 0, s>>>(
          m, g->frag_ptr, g->snp, g->allele, first, last, order, sfirst, slast, pmax,
          o->weight_mode, cnt, nullptr, nullptr, nullptr);
    }
    if (!scan_i64(ctx, s, cnt, g->row_ptr, m)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
    QH_CUDA_TRY(cudaMemcpyAsync(&g->nnz, g->row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    g->col = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
    g->w = (double*)dalloc(*g, sizeof(double) * std::max<int64_t>(g->nnz, 1));
    if (!g->col || !g->w) return set_err(ctx, QH_ENOMEM, "allocation failed (edges)");
    if (m > 0 && g->nnz > 0)
      k_read_edges<1><<<::qh::counted(nblk((int64_t)m * 32)), 256, 0, s>>>(
          m, g->frag_ptr, g->snp, g->allele, first, last, order, sfirst, slast, pmax,
          o->weight_mode, nullptr, g->row_ptr, g->col, g->w);
  } else {
    g->n_nodes = n;
    double* L = (double*)ctx->scratch(sizeof(double) * 94 * 94, 1);
    int64_t* cnt = (int64_t*)ctx->scratch(sizeof(int64_t) * (n + 1), 2);
    if (!L || !cnt) return set_err(ctx, QH_ENOMEM, "allocation failed (SNP graph scratch)");
    k_llr_table<<<::qh::counted(94), 94, 0, s>>>(L);
    QH_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
    // rows whose covered window is narrow go to the small-footprint kernel (many CTAs
    // per SM); the others are deferred to the large kernel
    const size_t smem = sizeof(SnpRowSmem);
    const size_t smem_s = SNP_SMALL_SMEM;
    QH_CUDA_TRY(cudaFuncSetAttribute(k_snp_rows<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s));
    QH_CUDA_TRY(cudaFuncSetAttribute(k_snp_rows<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s));
    QH_CUDA_TRY(cudaFuncSetAttribute(k_snp_rows<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QH_CUDA_TRY(cudaFuncSetAttribute(k_snp_rows<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::max(1, std::min(n, ctx->n_sm * 4));
    const unsigned grid_s = (unsigned)std::max(1, std::min(n, ctx->n_sm * 16));
    int32_t* defer = (int32_t*)ctx->scratch(sizeof(int32_t) * (n + 1), 23);
    g->row_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (n + 1));
    if (!g->row_ptr || !defer) return set_err(ctx, QH_ENOMEM, "allocation failed (edges)");
    int32_t* n_defer = defer + n;
    QH_CUDA_TRY(cudaMemsetAsync(n_defer, 0, sizeof(int32_t), s));
    if (n > 0) {
      k_snp_rows<0, true><<<::qh::counted(grid_s), 256, smem_s, s>>>(
          n, g->frag_ptr, g->snp, g->allele, g->qual, g->is_porec, g->cov_ptr, g->cov_frag, L,
          o->porec_alpha, o->linkage_k, cnt, nullptr, nullptr, nullptr, ctx->d_err, nullptr,
          nullptr, defer, n_defer);
      k_snp_rows<0, false><<<::qh::counted(grid), 512, smem, s>>>(
          n, g->frag_ptr, g->snp, g->allele, g->qual, g->is_porec, g->cov_ptr, g->cov_frag, L,
          o->porec_alpha, o->linkage_k, cnt, nullptr, nullptr, nullptr, ctx->d_err, defer,
          n_defer, nullptr, nullptr);
    }
    if (!scan_i64(ctx, s, cnt, g->row_ptr, n)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
    QH_CUDA_TRY(cudaMemcpyAsync(&g->nnz, g->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr & ERR_ROWCAP)
      return set_err(ctx, QH_EUNSUPPORTED, "an SNP row gathers more than 8192 fragment terms");
    g->col = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
    g->w = (double*)dalloc(*g, sizeof(double) * std::max<int64_t>(g->nnz, 1));
    if (!g->col || !g->w) return set_err(ctx, QH_ENOMEM, "allocation failed (edges)");
    if (n > 0 && g->nnz > 0) {
      k_snp_rows<1, true><<<::qh::counted(grid_s), 256, smem_s, s>>>(
          n, g->frag_ptr, g->snp, g->allele, g->qual, g->is_porec, g->cov_ptr, g->cov_frag, L,
          o->porec_alpha, o->linkage_k, nullptr, g->row_ptr, g->col, g->w, ctx->d_err, nullptr,
          nullptr, nullptr, nullptr);
      k_snp_rows<1, false><<<::qh::counted(grid), 512, smem, s>>>(
          n, g->frag_ptr, g->snp, g->allele, g->qual, g->is_porec, g->cov_ptr, g->cov_frag, L,
          o->porec_alpha, o->linkage_k, nullptr, g->row_ptr, g->col, g->w, ctx->d_err, defer,
          n_defer, nullptr, nullptr);
    }
  }
  const int32_t N = g->n_nodes;
  QH_STAGE_CHECK("graph build: edges");
  // ---- weight range: integer weights up to 256 are exact in one BF16 operand
  {
    unsigned long long* amax = (unsigned long long*)ctx->scratch(16, 9);
    if (!amax) return set_err(ctx, QH_ENOMEM, "allocation failed (weight range)");
    int32_t* nonint = (int32_t*)(amax + 1);
    QH_CUDA_TRY(cudaMemsetAsync(amax, 0, 16, s));
    if (g->nnz > 0)
      k_abs_max<<<::qh::counted((unsigned)std::min<int64_t>(nblk(g->nnz), ctx->n_sm * 4)), 256, 0, s>>>(g->nnz, g->w, amax, nonint);
    unsigned long long hv[2] = {0, 0};
    QH_CUDA_TRY(cudaMemcpyAsync(hv, amax, 16, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    double mx;
    memcpy(&mx, &hv[0], sizeof(double));
    g->max_abs_w = mx;
    g->integer_weights = ((int32_t)hv[1] == 0);
    g->has_lo = !(g->integer_weights && mx <= 256.0);
  }
  QH_STAGE_CHECK("graph build: weight range");
  // ---- components
  int32_t* parent = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(N, 1), 10);
  int32_t* label = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(N, 1), 11);
  int32_t* csize = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(N, 1), 12);
  int32_t* isroot = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(N, 1), 13);
  int64_t* rrank = (int64_t*)ctx->scratch(sizeof(int64_t) * (N + 1), 14);
  int64_t kcap = next_pow2(std::max<int64_t>(N, 2048));
  uint64_t* bkeys = (uint64_t*)ctx->scratch(sizeof(uint64_t) * kcap, 15);
  if (!parent || !label || !csize || !isroot || !rrank || !bkeys)
    return set_err(ctx, QH_ENOMEM, "allocation failed (components)");
  g->block_of = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(N, 1));
  g->local = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(N, 1));
  g->pad_index = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(N, 1));
  if (!g->block_of || !g->local || !g->pad_index) return set_err(ctx, QH_ENOMEM, "allocation failed (blocks)");
  QH_CUDA_TRY(cudaMemsetAsync(csize, 0, sizeof(int32_t) * std::max(N, 1), s));
  QH_CUDA_TRY(cudaMemsetAsync(g->local, 0xff, sizeof(int32_t) * std::max(N, 1), s));
  QH_CUDA_TRY(cudaMemsetAsync(g->pad_index, 0xff, sizeof(int32_t) * std::max(N, 1), s));
  if (N > 0) {
    k_uf_init<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, parent);
    // label holds the sampled-component flags and isroot[0] the sampled root until
    // the compression and the root marks below overwrite them
    k_uf_link_first<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, parent);
    k_uf_sample<<<::qh::counted(1), UF_SAMPLES, 0, s>>>(N, parent, isroot);
    k_uf_flag<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, parent, isroot, label);
    k_uf_link_rest<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, label,
                                                           parent);
    k_uf_compress<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, parent, label, csize);
    k_block_roots<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, label, csize, isroot);
  }
  if (!scan_i32_to_i64(ctx, s, isroot, rrank, N)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
  int64_t nb64 = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&nb64, rrank + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  const int32_t nb = (int32_t)nb64;
  g->n_blocks = nb;
  int32_t* bsize = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(nb, 1), 16);
  if (!bsize) return set_err(ctx, QH_ENOMEM, "allocation failed (block sizes)");
  if (N > 0) {
    k_block_of<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, label, csize, rrank, g->block_of, bkeys);
    k_block_sizes<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, label, csize, rrank, bsize);
    sort_u64(s, bkeys, N, kcap);
  }
  g->h_block_size.assign(nb, 0);
  if (nb > 0)
    QH_CUDA_TRY(cudaMemcpyAsync(g->h_block_size.data(), bsize, sizeof(int32_t) * nb,
                                cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  // host: block offsets, padded offsets, row tiles, tile slots
  std::vector<int64_t> h_block_ptr(nb + 1, 0);
  g->h_pad_off.assign(nb + 1, 0);
  std::vector<int64_t> h_slot_off(nb + 1, 0);
  std::vector<int32_t> h_T(std::max(nb, 1), 0);
  for (int32_t b = 0; b < nb; ++b) {
    int32_t sz = g->h_block_size[b];
    int32_t T = (sz + TILE - 1) / TILE;
    h_T[b] = T;
    h_block_ptr[b + 1] = h_block_ptr[b] + sz;
    g->h_pad_off[b + 1] = g->h_pad_off[b] + T * TILE;
    h_slot_off[b + 1] = h_slot_off[b] + (int64_t)T * T;
  }
  g->n_pad = g->h_pad_off[nb];
  const int64_t n_slots = h_slot_off[nb];
  const int64_t total_in_blocks = h_block_ptr[nb];
  g->block_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (nb + 1));
  g->pad_off = (int32_t*)dalloc(*g, sizeof(int32_t) * (nb + 1));
  g->perm = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(total_in_blocks, 1));
  g->pad_node = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(g->n_pad, 1));
  int64_t* d_slot_off = (int64_t*)ctx->scratch(sizeof(int64_t) * (nb + 1), 17);
  int32_t* d_T = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max(nb, 1), 18);
  int32_t* flags = (int32_t*)ctx->scratch(sizeof(int32_t) * std::max<int64_t>(n_slots, 1), 19);
  int64_t* slot_tile = (int64_t*)ctx->scratch(sizeof(int64_t) * (n_slots + 1), 20);
  if (!g->block_ptr || !g->pad_off || !g->perm || !g->pad_node || !d_slot_off || !d_T || !flags ||
      !slot_tile)
    return set_err(ctx, QH_ENOMEM, "allocation failed (layout)");
  QH_CUDA_TRY(cudaMemcpyAsync(g->block_ptr, h_block_ptr.data(), sizeof(int64_t) * (nb + 1),
                              cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(g->pad_off, g->h_pad_off.data(), sizeof(int32_t) * (nb + 1),
                              cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(d_slot_off, h_slot_off.data(), sizeof(int64_t) * (nb + 1),
                              cudaMemcpyHostToDevice, s));
  if (nb > 0)
    QH_CUDA_TRY(cudaMemcpyAsync(d_T, h_T.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemsetAsync(g->pad_node, 0xff, sizeof(int32_t) * std::max(g->n_pad, 1), s));
  if (total_in_blocks > 0)
    k_perm_local<<<::qh::counted(nblk(total_in_blocks)), 256, 0, s>>>(total_in_blocks, bkeys, g->block_ptr,
                                                        g->pad_off, g->perm, g->local,
                                                        g->pad_index, g->pad_node);
  QH_STAGE_CHECK("graph build: components and layout");
  // ---- tile slots: flag nonzero 128 x 128 tiles (all of them in dense mode)
  if (o->dense) {
    std::vector<int32_t> ones(std::max<int64_t>(n_slots, 1), 1);
    QH_CUDA_TRY(cudaMemcpyAsync(flags, ones.data(), sizeof(int32_t) * std::max<int64_t>(n_slots, 1),
                                cudaMemcpyHostToDevice, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    QH_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * std::max<int64_t>(n_slots, 1), s));
    if (N > 0)
      k_tile_flags<<<::qh::counted(nblk(N)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, g->block_of, g->local,
                                          d_slot_off, d_T, flags);
  }
  if (!scan_i32_to_i64(ctx, s, flags, slot_tile, n_slots)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
  std::vector<int64_t> h_slot_tile(n_slots + 1);
  QH_CUDA_TRY(cudaMemcpyAsync(h_slot_tile.data(), slot_tile, sizeof(int64_t) * (n_slots + 1),
                              cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  g->n_tiles_hi = h_slot_tile[n_slots];
  // storage: CSR when the nonzero tiles would be mostly empty and numerous
  g->csr_mode = o->storage == QH_STORAGE_CSR ||
                (o->storage == QH_STORAGE_AUTO && !o->dense && g->n_tiles_hi > 4096 &&
                 g->n_tiles_hi * (int64_t)TILE * TILE > 64 * std::max<int64_t>(g->nnz, 1));
  if (g->csr_mode) {
    g->n_tiles_hi = 0;
    g->has_lo = false;
    std::fill(h_slot_tile.begin(), h_slot_tile.end(), 0);
  }
  // row tiles: hi entries then (if needed) lo entries, contiguous per row tile
  g->h_rt.clear();
  std::vector<int32_t> h_rt_of_block(std::max(nb, 1), 0);
  std::vector<int32_t> h_tile_col;
  int64_t entry = 0;
  for (int32_t b = 0; b < nb; ++b) {
    h_rt_of_block[b] = (int32_t)g->h_rt.size();
    int32_t T = h_T[b];
    for (int32_t r = 0; r < T; ++r) {
      int64_t s0 = h_slot_off[b] + (int64_t)r * T;
      RowTile rt;
      rt.block = b;
      rt.row0 = g->h_pad_off[b] + r * TILE;
      rt.valid = std::min(TILE, g->h_block_size[b] - r * TILE);
      rt.tile_begin = (int32_t)entry;
      rt.n_hi = (int32_t)(h_slot_tile[s0 + T] - h_slot_tile[s0]);
      rt.n_all = g->has_lo ? 2 * rt.n_hi : rt.n_hi;
      rt.f32_begin = (int32_t)h_slot_tile[s0];
      int32_t ct0 = g->h_pad_off[b] / TILE;
      std::vector<int32_t> cols;
      for (int32_t c = 0; c < T; ++c)
        if (h_slot_tile[s0 + c + 1] > h_slot_tile[s0 + c]) cols.push_back(ct0 + c);
      for (int rep = 0; rep < (g->has_lo ? 2 : 1); ++rep)
        h_tile_col.insert(h_tile_col.end(), cols.begin(), cols.end());
      entry += rt.n_all;
      g->max_tiles_per_row = std::max(g->max_tiles_per_row, rt.n_all);
      g->h_rt.push_back(rt);
    }
  }
  g->n_tiles = entry;
  g->n_row_tiles = (int32_t)g->h_rt.size();
  g->rt = (RowTile*)dalloc(*g, sizeof(RowTile) * std::max(g->n_row_tiles, 1));
  g->tile_col = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(g->n_tiles, 1));
  g->tile_bf16 = (__nv_bfloat16*)dalloc(*g, sizeof(__nv_bfloat16) * TILE * TILE * std::max<int64_t>(g->n_tiles, 1));
  g->tile_f32 = (float*)dalloc(*g, sizeof(float) * TILE * TILE * std::max<int64_t>(g->n_tiles_hi, 1));
  g->rt_of_block = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(nb, 1));
  g->slot_off = (int64_t*)dalloc(*g, sizeof(int64_t) * (nb + 1));
  g->tiles_per_block = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max(nb, 1));
  g->slot_tile = (int64_t*)dalloc(*g, sizeof(int64_t) * (n_slots + 1));
  if (!g->rt || !g->tile_col || !g->tile_bf16 || !g->tile_f32 || !g->rt_of_block || !g->slot_off ||
      !g->tiles_per_block || !g->slot_tile)
    return set_err(ctx, QH_ENOMEM, "allocation failed (tiles)");
  if (g->n_row_tiles > 0)
    QH_CUDA_TRY(cudaMemcpyAsync(g->rt, g->h_rt.data(), sizeof(RowTile) * g->n_row_tiles,
                                cudaMemcpyHostToDevice, s));
  if (g->n_tiles > 0)
    QH_CUDA_TRY(cudaMemcpyAsync(g->tile_col, h_tile_col.data(), sizeof(int32_t) * g->n_tiles,
                                cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(g->rt_of_block, h_rt_of_block.data(), sizeof(int32_t) * std::max(nb, 1),
                              cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(g->slot_off, d_slot_off, sizeof(int64_t) * (nb + 1),
                              cudaMemcpyDeviceToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(g->tiles_per_block, d_T, sizeof(int32_t) * std::max(nb, 1),
                              cudaMemcpyDeviceToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(g->slot_tile, slot_tile, sizeof(int64_t) * (n_slots + 1),
                              cudaMemcpyDeviceToDevice, s));
  // padded CSR of J
  {
    int64_t* pcnt = (int64_t*)ctx->scratch(sizeof(int64_t) * (g->n_pad + 1), 22);
    g->prow_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (g->n_pad + 1));
    if (!pcnt || !g->prow_ptr) return set_err(ctx, QH_ENOMEM, "allocation failed (padded CSR)");
    QH_CUDA_TRY(cudaMemsetAsync(pcnt, 0, sizeof(int64_t) * (g->n_pad + 1), s));
    if (N > 0)
      k_pcsr_count<<<::qh::counted(nblk((int64_t)N * 32)), 256, 0, s>>>(N, g->row_ptr, g->w, g->pad_index, pcnt);
    if (!scan_i64(ctx, s, pcnt, g->prow_ptr, g->n_pad)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
    int64_t pnnz = 0;
    QH_CUDA_TRY(cudaMemcpyAsync(&pnnz, g->prow_ptr + g->n_pad, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    g->pnnz = pnnz;
    g->pcol = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(pnnz, 1));
    g->pval = (float*)dalloc(*g, sizeof(float) * std::max<int64_t>(pnnz, 1));
    if (!g->pcol || !g->pval) return set_err(ctx, QH_ENOMEM, "allocation failed (padded CSR)");
    if (N > 0)
      k_pcsr_fill<<<::qh::counted(nblk((int64_t)N * 32)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, g->pad_index,
                                                         g->prow_ptr, g->pcol, g->pval);
  }
  // CSR mode: band tiles and the remainder CSR
  if (g->csr_mode) {
    int64_t* rcnt = (int64_t*)ctx->scratch(sizeof(int64_t) * (g->n_pad + 1), 22);
    g->rrow_ptr = (int64_t*)dalloc(*g, sizeof(int64_t) * (g->n_pad + 1));
    g->band = (__nv_bfloat16*)dalloc(*g, sizeof(__nv_bfloat16) * TILE * TILE * 3 *
                                             std::max<int64_t>(g->n_row_tiles, 1));
    if (!rcnt || !g->rrow_ptr || !g->band) return set_err(ctx, QH_ENOMEM, "allocation failed (band)");
    QH_CUDA_TRY(cudaMemsetAsync(rcnt, 0, sizeof(int64_t) * (g->n_pad + 1), s));
    if (N > 0)
      k_rem_count<<<::qh::counted(nblk((int64_t)N * 32)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, g->pad_index, rcnt);
    if (!scan_i64(ctx, s, rcnt, g->rrow_ptr, g->n_pad)) return set_err(ctx, QH_ENOMEM, "allocation failed (scan)");
    int64_t rnnz = 0;
    QH_CUDA_TRY(cudaMemcpyAsync(&rnnz, g->rrow_ptr + g->n_pad, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    g->rnnz = rnnz;
    g->rcol = (int32_t*)dalloc(*g, sizeof(int32_t) * std::max<int64_t>(rnnz, 1));
    g->rval = (float*)dalloc(*g, sizeof(float) * std::max<int64_t>(rnnz, 1));
    if (!g->rcol || !g->rval) return set_err(ctx, QH_ENOMEM, "allocation failed (band)");
    if (N > 0)
      k_rem_fill<<<::qh::counted(nblk((int64_t)N * 32)), 256, 0, s>>>(N, g->row_ptr, g->col, g->w, g->pad_index,
                                                        g->rrow_ptr, g->rcol, g->rval);
    qh_status st = reband(ctx, g, g->w, g->band, nullptr);
    if (st != QH_OK) return st;
  }
  {
    qh_status st = retile(ctx, g, g->w, g->tile_bf16, g->tile_f32, nullptr);
    if (st != QH_OK) return st;
  }
  QH_STAGE_CHECK("graph build: tiles and padded CSR");
  // ---- per-block sums (sum of w over both triangles, sum of J^2) and default c0
  g->sum_w = (double*)dalloc(*g, sizeof(double) * std::max(nb, 1));
  g->sum_j2 = (double*)dalloc(*g, sizeof(double) * std::max(nb, 1));
  double* node_tmp = (double*)ctx->scratch(sizeof(double) * 2 * std::max(N, 1), 21);
  if (!g->sum_w || !g->sum_j2 || !node_tmp) return set_err(ctx, QH_ENOMEM, "allocation failed (block sums)");
  launch_block_sums(s, *g, g->w, g->sum_w, g->sum_j2, node_tmp);
  std::vector<double> sj2(std::max(nb, 1));
  g->h_sum_w.assign(std::max(nb, 1), 0.0);
  if (nb > 0) {
    QH_CUDA_TRY(cudaMemcpyAsync(sj2.data(), g->sum_j2, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaMemcpyAsync(g->h_sum_w.data(), g->sum_w, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  }
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  g->h_c0.assign(std::max(nb, 1), 0.0);
  for (int32_t b = 0; b < nb; ++b) {
    double Nb = (double)g->h_block_size[b];
    double sigma = std::sqrt(sj2[b] / (Nb * (Nb - 1.0)));
    g->h_c0[b] = sigma > 0 ? 0.5 / (sigma * std::sqrt(Nb)) : 0.0;
  }
  g->h_block_ptr = h_block_ptr;
  QH_STAGE_CHECK("graph build: block sums");
  return QH_OK;
}

qh_status reband(Ctx* ctx, const Graph* g, const double* w, __nv_bfloat16* band, float* rval) {
  cudaStream_t s = ctx->stream;
  if (!g->csr_mode || g->n_row_tiles == 0) return QH_OK;
  if (band != nullptr) {
    QH_CUDA_TRY(cudaMemsetAsync(band, 0, sizeof(__nv_bfloat16) * TILE * TILE * 3 * g->n_row_tiles, s));
    if (g->n_nodes > 0)
      k_band_fill<<<::qh::counted(nblk((int64_t)g->n_nodes * 32)), 256, 0, s>>>(g->n_nodes, g->row_ptr, g->col, w,
                                                                g->pad_index, band);
  }
  if (rval != nullptr && g->n_nodes > 0)
    k_rem_fill<<<::qh::counted(nblk((int64_t)g->n_nodes * 32)), 256, 0, s>>>(g->n_nodes, g->row_ptr, g->col, w,
                                                             g->pad_index, g->rrow_ptr, nullptr, rval);
  QH_CUDA_TRY(cudaGetLastError());
  return QH_OK;
}

qh_status retile(Ctx* ctx, Graph* g, const double* w, __nv_bfloat16* tb, float* tf, float* pval) {
  cudaStream_t s = ctx->stream;
  if (pval != nullptr && g->n_nodes > 0)  // padded CSR values (pattern unchanged)
    k_pcsr_fill<<<::qh::counted(nblk((int64_t)g->n_nodes * 32)), 256, 0, s>>>(g->n_nodes, g->row_ptr, g->col, w,
                                                              g->pad_index, g->prow_ptr, nullptr,
                                                              pval);
  if (g->n_tiles > 0)
    QH_CUDA_TRY(cudaMemsetAsync(tb, 0, sizeof(__nv_bfloat16) * TILE * TILE * g->n_tiles, s));
  if (g->n_tiles_hi > 0)
    QH_CUDA_TRY(cudaMemsetAsync(tf, 0, sizeof(float) * TILE * TILE * g->n_tiles_hi, s));
  if (g->n_nodes > 0 && g->n_tiles > 0)
    k_tile_fill<<<::qh::counted(nblk((int64_t)g->n_nodes * 32)), 256, 0, s>>>(g->n_nodes, g->row_ptr, g->col, w, g->block_of,
                                                 g->local, g->slot_off, g->tiles_per_block,
                                                 g->slot_tile, g->rt, g->rt_of_block,
                                                 g->has_lo ? 1 : 0, tb, tf);
  QH_CUDA_TRY(cudaGetLastError());
  return QH_OK;
}

}  // namespace qh
