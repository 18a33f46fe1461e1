// Multi-step bSB on the tensor cores: one persistent launch runs steps t0 .. t1-1
// of the SB algorithm solution's update
//   y <- y + dt * ( -(a0 - a(t)) x + c0 * J_hat X_hat ),  x <- x + dt * a0 * y,
//   |x| > 1 => x <- sgn(x), y <- 0,                       X_hat_{t+1} <- bf16(x)
// with the momentum y held on chip for the whole launch.
//
// Work item = (128-row tile of J, 128 replicas).  A CTA owns up to four items and
// gives each its own 128 TMEM columns.  Those columns are the MMA accumulator and
// hold y / (dt c0) between steps: every MMA accumulates J_hat X_hat onto it, so
//   dt c0 * acc = y + dt c0 Z,   y_{t+1} = dt c0 * acc - dt (a0 - a(t)) x.
// y therefore never leaves the SM between t0 and t1: it is read from HBM before the
// first step and written back after the last one.  Per spin-update the state costs
// 4 + 4 bytes (x) + 2 bytes (X_hat) of memory traffic instead of 16 + 2.
//
// Hand-off between steps, through release counters in global memory that a dedicated
// warp releases (gpu scope) after each item's epilogue and the TMA producer acquires
// before it loads X_hat of the next step.  Two modes:
//  * tile: item (row tile r, replica tile k) reads X_hat only in the column tiles of
//    r's nonzero J tiles; per item a counter counts its finished steps, and column
//    tile c of X_hat_t is loaded once counter (c, k) reaches the steps done.
//  * group: one counter per (block, k) counts the finished items of all row tiles of
//    the block; step t+1 of any of them starts when all have finished step t.
// J's tile pattern is symmetric, so in both modes the same waits also guarantee that
// every reader of r's column has finished step t-1 before item r overwrites the
// buffer that held X_hat_{t-1} with X_hat_{t+1}.
// All CTAs are co-resident (cooperative launch), so these waits always end; every
// wait is nevertheless bounded and sets ERR_TIMEOUT in the error word when it
// expires, after which all CTAs stop and drain their copies in flight.
//
// Early-stop checks inside the launch (read graphs: integer weights; at most three items
// per CTA).  At a check step t (a multiple of check_every, 0 < t < steps_b) the
// epilogue of step t-1 also writes S_t = sgn(x_t) in BF16 (exact +-1) next to X_hat_t,
// under the same release.  Step t's producer loads the (J, S_t) K-slices after the
// item's usual ones, the MMA issuer multiplies them into the spare TMEM columns
// 384..511, and the epilogue reduces s_i (J S)_i over its rows into exact per-replica
// integer sums E = S^T J S of the block (the cut is (sum W + E) / 4, J = -W).  The last
// contributing warp of the block takes the decision of the Results' stopping rule (a
// best cut above the best seen resets the stall count, else it grows; the block stops
// when it reaches patience) and publishes it; every item waits for that decision one
// check later, so a stopped block runs at most check_every steps past its stop, and its
// spins at the stop stay in the S buffer of that check's parity.  The checks are a
// separate instantiation (CHECK = true): the kernel without them carries none of their
// code.
//
// Roles (384 threads): warp 0 = TMA producer (six lanes), warp 1 = MMA issuer (one
// thread), warps 2-9 = epilogue (TMEM lane quarter = warp % 4 = 32 vertices, two warps
// per quarter split the 128 replicas), warp 10 = signal, warp 11 = J producer.  With JRES
// the J tiles of the CTA's single row tile stay in shared memory for the whole launch and
// only X_hat streams.  Otherwise J and X_hat K-slices stream through the ring: copied
// together by warp 0, or (jsplit: the kernel without checks, rows wider than the ring)
// J by warp 11 as soon as a slot frees, X_hat by warp 0 once its release is seen.
#include <algorithm>
#include <vector>

#include "qh_internal.cuh"
#include "tc_ptx.cuh"

namespace qh {

namespace {

constexpr int RB = 128;          // replicas per item (MMA N)
constexpr int MAX_ITEMS = 4;     // 4 items x 128 TMEM columns = 512
constexpr int EPI_WARPS = 8;
constexpr int RUN_THREADS = 32 * (4 + EPI_WARPS);
constexpr int SIGNAL_WARP = 2 + EPI_WARPS;
constexpr int JPROD_WARP = SIGNAL_WARP + 1;  // J K-slices into their own ring (stream mode)
constexpr uint32_t SLICE = TILE * 64 * 2;  // a 128 x 64 BF16 K-slice (16 KB)
constexpr int JRES_TILES = 4;              // resident J tiles (hi + lo entries) per CTA

struct ItemInfo {
  int32_t row0, valid, tile_begin, nk;  // nk = K-slices (2 per J tile entry)
  int32_t block, k, last_t, steps_b;    // last_t < t0: nothing to do this launch
  int32_t rt;                           // row tile index (= its column tile index)
  uint32_t rows_b;                      // row tiles of the block
  float dtc0, inv_dtc0;                 // dt * c0 and its reciprocal
  float dth;                            // dt * deformation field strength (0: none)
  double inv_steps;                     // 1 / steps_b
};

template <bool JRES>
struct RunSmem {
  static constexpr int ST = 6;                                  // operand ring slots
  static constexpr uint32_t SLOT = JRES ? SLICE : 2 * SLICE;    // X_hat (+ J) per slot
  static constexpr uint32_t RING_OFF = JRES ? JRES_TILES * 2 * SLICE : 0;
  static constexpr uint32_t BAR_OFF = RING_OFF + ST * SLOT;
  // full (X_hat), empty, full (J) (ring); accf, edone, decision (per item); jbar, drain,
  // sfull, sfree
  static constexpr int N_BARS = 3 * ST + 3 * MAX_ITEMS + 4;
  static constexpr uint32_t INFO_OFF = BAR_OFF + 8 * N_BARS;
  static constexpr uint32_t STOP_OFF = INFO_OFF + sizeof(ItemInfo) * MAX_ITEMS;
  static constexpr uint32_t BYTES = STOP_OFF + 4 * MAX_ITEMS + 16 + 1024;
};

struct RunArgs {
  const RowTile* rt;
  const int32_t* tile_col;
  float* x;                 // [R][n_pad]: read before the first step, written after the last
  float* y;                 // [R][n_pad]: likewise
  float4* xq;               // [R/4][n_pad] working copy of x between the first and the last
                            // step: xq[(rho/4) n_pad + v] holds replicas rho..rho+3 of v
  __nv_bfloat16* xh0;       // X_hat_t for even t
  __nv_bfloat16* xh1;       // X_hat_t for odd t
  const float* c0;          // [n_blocks]
  const int32_t* active;    // [n_blocks] or nullptr
  const int32_t* steps_b;   // [n_blocks]
  uint32_t* done;           // tile: [n_row_tiles][n_kt] steps finished; group:
                            // [n_blocks][n_kt] items finished; zero at launch
  const int32_t* rows_b;    // [n_blocks] row tiles per block
  int32_t group_sync;       // hand-off mode: 0 = tile, 1 = group
  int32_t jsplit;           // stream mode without checks: J K-slices copied by their own warp
  const int2* work;         // [grid] {first position, item count} in the wave's item list
  const int32_t* items;     // the wave's items (row tile * n_kt + replica tile)
  int32_t item_stride;      // a CTA's items sit at positions first, first + stride, ...
  int32_t n_pad, n_kt, n_blocks, t0, t1, use_lo;
  float dt, dta0;
  double a0;
  int32_t* err;
  const float* deform;      // [n_blocks] deformation field strength, or nullptr
  // early-stop checks inside the launch (check_every = 0: none)
  int32_t check_every, patience;
  __nv_bfloat16* s0;        // [R][n_pad] S_t = sgn(x_t) for even t / check_every
  __nv_bfloat16* s1;        //            and for odd
  const double* sum_w;      // [n_blocks] sum of W over both directions
  unsigned long long* e_sum;  // [2][n_blocks][R] S^T J S per replica (two's complement)
  uint32_t* e_cnt;          // [2][n_blocks] epilogue warps that have added their share
  uint32_t* decided;        // [n_blocks] checks decided (released after each decision)
  double* seen;             // [n_blocks] best cut seen at a check
  int32_t* stall;           // [n_blocks] checks since it last improved
  int32_t* stop_t;          // [n_blocks] the step count the block stopped at, or -1
  double* check_trace;      // [checks][n_blocks] best cut of each check, or nullptr
  // step timeline (test hook; nullptr in the solver): per CTA, traced step u0 + j and
  // item slot i, TRACE_EVENTS global-timer stamps followed by TRACE_EVENTS SM-clock
  // stamps at trace[((cta * trace_nu + j) * MAX_ITEMS + i) * 2 * TRACE_EVENTS + ...]
  unsigned long long* trace;
  int32_t trace_u0, trace_nu;
};

// Step-timeline events of one (step, item): the hand-off points of the pipeline.
enum : int {
  TR_DEPS = 0,      // producer: the item's inputs of this step are released
  TR_LOADED = 1,    // producer: the item's last operand load is issued
  TR_ACC_FREE = 2,  // MMA issuer: the epilogue of the previous step left the accumulator
  TR_FIRST_OP = 3,  // MMA issuer: the first operand slice has landed
  TR_MMA_DONE = 4,  // MMA issuer: every MMA of the item is issued (stamped before its commit)
  TR_EPI_START = 5, // epilogue (warp 2): the accumulator is ready
  TR_EPI_END = 6,   // epilogue (warp 2): its share of the update is stored (before it arrives)
  TR_RELEASE = 7,   // signal warp: X_hat of the next step is released to the other CTAs
  TR_PROD_START = 8,  // producer: reaches the item (before any of its waits)
  TR_OWN = 9,       // producer: the item's own previous step is released (tile mode)
  TR_SLOT = 10,     // producer: the first ring slot for the item is free
  TR_SLOT1 = 11,    // producer: the ring slots of K-slices 1 .. 5 are free (5 events)
  TRACE_EVENTS = 16
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// One stamp of the step timeline (no-op unless tracing and u is a traced step).
__device__ __forceinline__ void trace_at(const RunArgs& a, int u, int i, int ev) {
  if (a.trace == nullptr) return;
  const int j = u - a.trace_u0;
  if (j < 0 || j >= a.trace_nu) return;
  unsigned long long* p =
      a.trace + (((size_t)blockIdx.x * a.trace_nu + j) * MAX_ITEMS + i) * (2 * TRACE_EVENTS);
  p[ev] = global_ns();
  p[TRACE_EVENTS + ev] = (unsigned long long)clock64();
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Issue a 32-lane x 16-column TMEM load without waiting for it.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
// Wait for outstanding TMEM loads; the registers are threaded through so that no
// use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}
// The same for FP32 values (x of an item kept in TMEM): .b32 TMEM accesses take any
// 32-bit register.  The loads are ordered with the other TMEM accesses (volatile).
__device__ __forceinline__ void tmem_ld16f(uint32_t taddr, float (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
        "=f"(v[14]), "=f"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld_f(float (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                 "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]),
                 "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st16f(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15])
      : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acq_rel_gpu(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Relaxed gpu-scope accesses: L2-coherent, never a stale L1 line.
__device__ __forceinline__ int32_t ld_relaxed_s32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_s32(int32_t* p, int32_t v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
// Orders generic-proxy global accesses against later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

constexpr long long WAIT_LIMIT = 1ll << 31;  // SM cycles, about one second

// Bounded mbarrier wait that also gives up when another role has aborted.
__device__ __forceinline__ bool rwait(uint32_t bar, uint32_t parity, int32_t* err,
                                      volatile int32_t* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicOr(err, ERR_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Bounded wait until a release counter reaches `target`; gives up on an abort of
// this CTA or a timeout reported by any other CTA.
// Polls back off for 32 ns, and the error word is read every 64th poll only, so a
// waiting producer takes few issue slots and little L2 bandwidth.
__device__ __forceinline__ bool wait_count(const uint32_t* p, uint32_t target, int32_t* err,
                                           volatile int32_t* abort) {
  if (ld_acquire_gpu(p) >= target) return true;
  const long long t0 = clock64();
  for (uint32_t n = 1; ld_acquire_gpu(p) < target; ++n) {
    __nanosleep(32);
    if (*abort) return false;
    if ((n & 63u) == 0 && (*reinterpret_cast<volatile int32_t*>(err) & ERR_TIMEOUT)) {
      *abort = 1;
      return false;
    }
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicOr(err, ERR_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Failure-detection probe: one of the step kernels' bounded waits on something that
// nothing will complete (which = 0: an mbarrier phase; 1: a release counter).  The wait
// expires after about a second, sets ERR_TIMEOUT and the kernel returns.
__global__ void k_wait_probe(int which, const uint32_t* counter, int32_t* err) {
  __shared__ uint64_t bar;
  __shared__ int32_t abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (which == 0)
      rwait(smem_u32(&bar), 0, err, &abort_flag);
    else
      wait_count(counter, 1u, err, &abort_flag);
  }
}

// Position in the CTA's sequence of (step, item) pairs that have work; `dead` masks the
// items whose block stopped early.
struct Cursor {
  int u, i;
};
__device__ __forceinline__ Cursor next_live(Cursor c, const ItemInfo* info, int n_items,
                                            int t0, int n_steps, uint32_t dead) {
  while (true) {
    if (++c.i == n_items) {
      c.i = 0;
      if (++c.u >= n_steps) return Cursor{n_steps, 0};
    }
    if (t0 + c.u <= info[c.i].last_t && !((dead >> c.i) & 1u)) return c;
  }
}

// Step t of a block is a check step: its product also runs on S_t = sgn(x_t).  The
// kernel without checks (CHECK = false) compiles none of their code: the roles' loops
// stay as small as before, which their instruction caches need.
template <bool CHECK>
__device__ __forceinline__ bool check_step(const RunArgs& a, int t, int steps_b) {
  return CHECK && t > 0 && t < steps_b && t % a.check_every == 0;
}
// A check step that first waits for the decision of the previous check.
template <bool CHECK>
__device__ __forceinline__ bool decision_step(const RunArgs& a, int t, int steps_b) {
  return check_step<CHECK>(a, t, steps_b) && t >= 2 * a.check_every;
}

// S = sgn(x) of one epilogue thread's vertex and 64 replicas, read back from its x
// working copy (q0: float4 m of chunk c at q0[(4c + m) np]; sc: replica j at sc[j np]).
__device__ __forceinline__ void write_signs(const float4* __restrict__ q0, uint32_t np,
                                         __nv_bfloat16* __restrict__ sc) {
  const __nv_bfloat16 one = __float2bfloat16_rn(1.f), neg = __float2bfloat16_rn(-1.f);
#pragma unroll 1
  for (int m = 0; m < 16; ++m) {
    const float4 v = q0[(size_t)m * np];
    sc[(size_t)(4 * m) * np] = v.x >= 0.f ? one : neg;
    sc[(size_t)(4 * m + 1) * np] = v.y >= 0.f ? one : neg;
    sc[(size_t)(4 * m + 2) * np] = v.z >= 0.f ? one : neg;
    sc[(size_t)(4 * m + 3) * np] = v.w >= 0.f ? one : neg;
  }
}

// The energy of one check product, by one epilogue warp, and the block's decision when
// this warp is the block's last contributor.  E = S^T J S per replica: this thread's
// row contributes s_i (J S)_{i,rho} for its 64 replicas (s_own: its own S_t values,
// replica j at s_own[j np]), the warp sums its 32 rows.  The products are integers
// (integer J, +-1 S), summed exactly by the MMA in FP32.  False when a wait gave up.
__device__ __forceinline__ bool check_energy(
    uint32_t scol, const __nv_bfloat16* __restrict__ s_own, uint32_t np,
    const unsigned long long* e_blk, unsigned long long* e_mine,
    unsigned long long* e_next, uint32_t* cnt, uint32_t* cnt_next, uint32_t total, int32_t R,
    double sum_w, double* seen, int32_t* stall, int32_t* stop_t, uint32_t* decided, int t,
    int check_every, int patience, uint32_t sfull, uint32_t sfree, uint32_t n_chk,
    int32_t* err, volatile int32_t* abort, int lane, double* trace_slot) {
  if (!__all_sync(0xffffffffu, rwait(sfull, n_chk & 1u, err, abort))) return false;
  tc_fence_after();
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    uint32_t v[16];
    __syncwarp();
    tmem_ld16(scol + (uint32_t)(c * 16), v);
    int p[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {  // s_i of this thread's row, as written at step t - 1
      const int iv = __float2int_rn(__uint_as_float(v[j]));
      p[j] = __bfloat162float(s_own[(size_t)(16 * c + j) * np]) < 0.f ? -iv : iv;
    }
    // butterfly over the lanes: after the four halving rounds lane l holds 16 lanes'
    // sums for replica (l >> 1) & 15; the last round adds its neighbour's
#pragma unroll
    for (int w = 8, o = 16; w >= 1; w >>= 1, o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int m = 0; m < w; ++m) {
        const int keep = up ? p[m + w] : p[m], send = up ? p[m] : p[m + w];
        p[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    const int tot = p[0] + __shfl_xor_sync(0xffffffffu, p[0], 1);
    if ((lane & 1) == 0)
      atomicAdd(e_mine + c * 16 + ((lane >> 1) & 15), (unsigned long long)(long long)tot);
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(sfree);
  // this warp's share is in; the block's last warp takes the decision
  __threadfence();
  __syncwarp();
  uint32_t old = 0;
  if (lane == 0) old = atom_add_acq_rel_gpu(cnt, 1u);
  old = __shfl_sync(0xffffffffu, old, 0);
  if (old + 1 != total) return true;
  __threadfence();
  double best = -INFINITY;
  for (int rho = lane; rho < R; rho += 32)  // cut = (sum W + S^T J S) / 4, J = -W
    best = fmax(best, 0.25 * (sum_w + (double)(long long)ld_relaxed_u64(e_blk + rho)));
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  // the next check uses the other parity: clear it (its last reader, the previous
  // decision, is done: every contributor above waited for it)
  for (int rho = lane; rho < R; rho += 32) st_relaxed_u64(e_next + rho, 0ull);
  if (lane == 0) {
    if (trace_slot != nullptr) st_relaxed_f64(trace_slot, best);  // the check's best cut
    if (best > ld_relaxed_f64(seen)) {
      st_relaxed_f64(seen, best);
      st_relaxed_s32(stall, 0);
    } else {
      const int32_t st = ld_relaxed_s32(stall) + 1;
      st_relaxed_s32(stall, st);
      if (st >= patience) st_relaxed_s32(stop_t, t);
    }
    st_relaxed_s32(reinterpret_cast<int32_t*>(cnt_next), 0);
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release_gpu(decided, (uint32_t)(t / check_every));
  return true;
}

template <bool JRES, int SB, bool CHECK, bool XT>
__global__ void __launch_bounds__(RUN_THREADS, 1)
    k_bsb_run(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmX0,
              const __grid_constant__ CUtensorMap tmX1, const __grid_constant__ CUtensorMap tmS0,
              const __grid_constant__ CUtensorMap tmS1, RunArgs a) {
  using L = RunSmem<JRES>;
  constexpr int ST = L::ST;
  // J K-slices in a ring of their own, filled by the J producer warp (stream mode without
  // checks, chosen by the host when row tiles span more K-slices than the ring holds);
  // otherwise the TMA producer copies J and X_hat of a K-slice together
  const bool jsplit = !JRES && !CHECK && a.jsplit != 0;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  ItemInfo* info = reinterpret_cast<ItemInfo*>(smem + L::INFO_OFF);
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t abort_s;
  volatile int32_t* abort_flag = &abort_s;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * ST, fullj0 = empty0 + 8 * ST,
                 accf0 = fullj0 + 8 * ST,
                 edone0 = accf0 + 8 * MAX_ITEMS, decb0 = edone0 + 8 * MAX_ITEMS,
                 jbar = decb0 + 8 * MAX_ITEMS, drain = jbar + 8, sfull = drain + 8,
                 sfree = sfull + 8;
  // first step an item does not run because its block stopped (written by the producer
  // before it arrives on the item's decision barrier)
  volatile int32_t* stop_u = reinterpret_cast<volatile int32_t*>(smem + L::STOP_OFF);
  // TMEM columns of the check product (free when a CTA holds at most three items)
  constexpr uint32_t SPARE_COL = 3 * RB;

  const int2 wk = a.work[blockIdx.x];
  // the check product needs the spare TMEM columns and S_t written in this launch:
  // a CTA given more items, or a launch not starting at step 0, does nothing
  const bool refused = CHECK && (a.check_every < 1 || wk.y > 3 || a.t0 != 0);
  const int n_items = refused ? 0 : wk.y;
  const int n_steps = a.t1 - a.t0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 2 && lane < n_items) {
    const int item = a.items[wk.x + lane * a.item_stride];
    const RowTile rt = a.rt[item / a.n_kt];
    ItemInfo it;
    it.row0 = rt.row0;
    it.valid = rt.valid;
    it.tile_begin = rt.tile_begin;
    it.nk = 2 * (a.use_lo ? rt.n_all : rt.n_hi);
    it.block = rt.block;
    it.k = item % a.n_kt;
    it.steps_b = a.steps_b[rt.block];
    const bool on = a.active == nullptr || a.active[rt.block] != 0;
    it.last_t = on ? min(a.t1, it.steps_b) - 1 : a.t0 - 1;
    it.rt = item / a.n_kt;
    it.rows_b = (uint32_t)a.rows_b[rt.block];
    it.dtc0 = a.dt * a.c0[rt.block];
    it.inv_dtc0 = 1.0f / it.dtc0;
    it.inv_steps = 1.0 / (double)it.steps_b;
    it.dth = a.deform ? a.dt * a.deform[rt.block] : 0.f;
    info[lane] = it;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(fullj0 + 8 * s, 1);
    }
    for (int i = 0; i < MAX_ITEMS; ++i) {
      mbar_init(accf0 + 8 * i, 1);
      mbar_init(edone0 + 8 * i, EPI_WARPS);
      mbar_init(decb0 + 8 * i, 1);
      stop_u[i] = 0x7fffffff;
    }
    mbar_init(jbar, 1);
    mbar_init(drain, 1);
    mbar_init(sfull, 1);
    mbar_init(sfree, EPI_WARPS);
    abort_s = 0;
    if (refused) atomicOr(a.err, ERR_CONFIG);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_slot), 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // Lanes 0 .. ST-1 fill up to ST ring slots at once, one K-slice (X_hat and J
    // copies) per lane: the bulk copies of one thread complete one after the other, so
    // parallel lanes multiply the bytes in flight.  The MMA issuer consumes the slots
    // in order.
    if (n_items > 0) {
      const bool lead = lane == 0;
      uint32_t q = 0;
      bool jissued = false;
      if (JRES && lead) {  // all items of the CTA share one row tile
        const ItemInfo& it = info[0];
        mbar_expect_tx(jbar, (uint32_t)it.nk * SLICE);
        for (int kb = 0; kb < it.nk; ++kb)
          tma_load_2d(smem_u32(smem + kb * SLICE), &tmJ, jbar, (kb & 1) * 64,
                      (it.tile_begin + (kb >> 1)) * TILE);
        jissued = true;
      }
      bool ok = true;
      uint32_t dead = 0;  // items whose block stopped early
      for (int u = 0; ok && u < n_steps; ++u) {
        const int t = a.t0 + u;
        const CUtensorMap* mx = (t & 1) ? &tmX1 : &tmX0;
        for (int i = 0; ok && i < n_items; ++i) {
          const ItemInfo& it = info[i];
          if (t > it.last_t || ((dead >> i) & 1u)) continue;
          const bool chk = check_step<CHECK>(a, t, it.steps_b);
          if (chk && t >= 2 * a.check_every) {
            // the previous check's decision: the items of a stopped block end here; the
            // other roles learn it from stop_u after the item's decision barrier
            int verdict = 0;  // 0: go on, 1: stopped, -1: the wait gave up
            if (lead) {
              if (wait_count(a.decided + it.block, (uint32_t)(t / a.check_every - 1), a.err,
                             abort_flag)) {
                if (ld_relaxed_s32(a.stop_t + it.block) >= 0) {
                  stop_u[i] = u;
                  verdict = 1;
                }
                mbar_arrive(decb0 + 8 * i);
              } else {
                verdict = -1;
              }
            }
            verdict = __shfl_sync(0xffffffffu, verdict, 0);
            if (verdict < 0) {
              ok = false;
              break;
            }
            if (verdict > 0) {
              dead |= 1u << i;
              continue;
            }
          }
          // Dependencies, waited in parallel by the lanes (acquire loads of one thread
          // would serialise, a round trip each).  Tile mode: lane 0 waits for the item's
          // own previous step, every loading lane for the column tile of its K-slice
          // (both halves of a column check its counter).  Group mode: lane 0 waits until
          // every row tile of the block has finished step t-1.  Then the lanes fill up to
          // ST ring slots, one K-slice each.
          if (lead) trace_at(a, u, i, TR_PROD_START);
          // pass 0: X_hat_t and J; pass 1 (check steps): S_t and J for the check product.
          // S_t is released together with X_hat_t, so pass 1 needs no waits of its own:
          // each lane's acquire and proxy fence of pass 0 covered its K-slices.
          for (int pass = 0; ok && pass < (chk ? 2 : 1); ++pass) {
            const CUtensorMap* mp =
                pass == 0 ? mx : (((t / a.check_every) & 1) ? &tmS1 : &tmS0);
            for (int kb0 = 0; ok && kb0 < it.nk; kb0 += ST) {
              const int kb = kb0 + lane;
              const bool mine = lane < ST && kb < it.nk;
              const int e = kb >> 1, half = kb & 1;
              const int32_t ct = mine ? a.tile_col[it.tile_begin + e] : 0;
              bool lok = true;
              if (pass == 0) {
                if (u > 0 && kb0 == 0 && lead && !a.group_sync) {
                  lok = wait_count(a.done + (size_t)it.rt * a.n_kt + it.k, (uint32_t)u, a.err,
                                   abort_flag);
                  if (lok) trace_at(a, u, i, TR_OWN);
                }
                // every loading lane acquires the release its own copies depend on
                if (lok && mine && u > 0)
                  lok = a.group_sync
                            ? wait_count(a.done + (size_t)it.block * a.n_kt + it.k,
                                         (uint32_t)u * it.rows_b, a.err, abort_flag)
                            : wait_count(a.done + (size_t)ct * a.n_kt + it.k, (uint32_t)u,
                                         a.err, abort_flag);
                if (lok && lead && (u == 0 || a.group_sync) && kb0 == 0)
                  trace_at(a, u, i, TR_OWN);
                if (!__all_sync(0xffffffffu, lok)) {
                  ok = false;
                  break;
                }
                if (u > 0 && mine) fence_proxy_async_global();
                if (kb0 + ST >= it.nk && lead) trace_at(a, u, i, TR_DEPS);
              }
              if (mine) {
                const int s = (int)((q + kb) % ST);
                const uint32_t ph = ((q + kb) / ST) & 1u;
                lok = rwait(empty0 + 8 * s, ph ^ 1u, a.err, abort_flag);
                if (lok) {
                  if (pass == 0 && kb == 0) trace_at(a, u, i, TR_SLOT);
                  if (pass == 0 && kb >= 1 && kb <= 5) trace_at(a, u, i, TR_SLOT1 + kb - 1);
                  uint8_t* slot = smem + L::RING_OFF + s * L::SLOT;
                  mbar_expect_tx(full0 + 8 * s, jsplit ? SLICE : L::SLOT);
                  const uint32_t xdst = JRES ? smem_u32(slot) : smem_u32(slot + SLICE);
                  tma_load_2d(xdst, mp, full0 + 8 * s, ct * TILE + half * 64, it.k * RB);
                  if (!JRES && !jsplit)
                    tma_load_2d(smem_u32(slot), &tmJ, full0 + 8 * s, half * 64,
                                (it.tile_begin + e) * TILE);
                }
              }
              if (!__all_sync(0xffffffffu, lok)) ok = false;
            }
            if (!ok) break;
            q += (uint32_t)it.nk;
          }
          if (!ok) break;
          if (lead) trace_at(a, u, i, TR_LOADED);
        }
      }
      // copies still in flight must land before the CTA exits: the last load of
      // every ring slot, and the resident J tiles
      if (lead) {
        for (uint32_t jq = q > (uint32_t)ST ? q - ST : 0u; jq < q; ++jq)
          mbar_wait(full0 + 8 * (jq % ST), (jq / ST) & 1u, a.err);
        if (jissued) mbar_wait(jbar, 0, a.err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && n_items > 0) {
      constexpr uint32_t idesc = idesc_bf16<RB>();
      bool ok = true;
      if (JRES) ok = rwait(jbar, 0, a.err, abort_flag);
      uint32_t q = 0, dead = 0, n_chk = 0;
      for (int u = 0; ok && u < n_steps; ++u) {
        const int t = a.t0 + u;
        for (int i = 0; ok && i < n_items; ++i) {
          const ItemInfo& it = info[i];
          if (t > it.last_t || ((dead >> i) & 1u)) continue;
          const bool chk = check_step<CHECK>(a, t, it.steps_b);
          if (chk && t >= 2 * a.check_every) {
            if (!(ok = rwait(decb0 + 8 * i, (uint32_t)(t / a.check_every) & 1u, a.err,
                             abort_flag)))
              break;
            if (u >= stop_u[i]) {
              dead |= 1u << i;
              continue;
            }
          }
          // the epilogue has stored y / (dt c0) of the previous step into the columns
          if (!(ok = rwait(edone0 + 8 * i, (uint32_t)u & 1u, a.err, abort_flag))) break;
          tc_fence_after();
          trace_at(a, u, i, TR_ACC_FREE);
          // pass 0: the step's product onto y / (dt c0); pass 1 (check steps): J S_t into
          // the spare columns, once the epilogue has read the last check product
          for (int pass = 0; ok && pass < (chk ? 2 : 1); ++pass) {
            if (pass == 1) {
              if (!(ok = rwait(sfree, (n_chk & 1u) ^ 1u, a.err, abort_flag))) break;
              tc_fence_after();
            }
            const uint32_t d = pass == 0 ? tmem + (uint32_t)(i * RB) : tmem + SPARE_COL;
            for (int kb = 0; kb < it.nk; ++kb) {
              const int s = (int)(q % ST);
              const uint32_t ph = (q / ST) & 1u;
              if (!(ok = rwait(full0 + 8 * s, ph, a.err, abort_flag))) break;
              if (jsplit && !(ok = rwait(fullj0 + 8 * s, ph, a.err, abort_flag))) break;
              tc_fence_after();
              if (pass == 0 && kb == 0) trace_at(a, u, i, TR_FIRST_OP);
              uint8_t* slot = smem + L::RING_OFF + s * L::SLOT;
              // D (vertices x replicas) += J slice (A) x X_hat (or S) slice (B)^T
              const uint64_t jd = sdesc_sw128(JRES ? smem_u32(smem + kb * SLICE) : smem_u32(slot));
              const uint64_t xd = sdesc_sw128(JRES ? smem_u32(slot) : smem_u32(slot + SLICE));
#pragma unroll
              for (int k = 0; k < 4; ++k)
                mma_bf16(d, jd + (uint64_t)(2 * k), xd + (uint64_t)(2 * k), idesc,
                         (pass == 0 || kb > 0 || k > 0) ? 1u : 0u);
              mma_commit(empty0 + 8 * s);
              ++q;
            }
            if (!ok) break;
            if (pass == 0) {
              trace_at(a, u, i, TR_MMA_DONE);
              mma_commit(accf0 + 8 * i);
            } else {
              mma_commit(sfull);
              ++n_chk;
            }
          }
        }
      }
      mma_commit(drain);  // every MMA of this thread has completed once this fires
      mbar_wait(drain, 0, a.err);
    }
  } else if (warp < SIGNAL_WARP) {
    // ------------------------------------------------------------ epilogue
    // The accumulator is (vertex x replica): TMEM lane = vertex of the row tile,
    // column = replica of the item.  A thread owns one vertex and 64 replicas (half hh
    // of the item) in four chunks of 16; for each replica the 32 lanes of a warp touch
    // 32 consecutive vertices, one coalesced 128-byte line of x ([R][n_pad]).
    // Element indices fit 32 bits: R * n_pad <= MAX_ITEMS * 128 * 128 * CTAs.
    const int qd = warp & 3, hh = (warp - 2) >> 2;
    const int r = qd * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(hh * 64);
    float* __restrict__ xs = a.x;
    float* __restrict__ ys = a.y;
    const uint32_t np = (uint32_t)a.n_pad;
    // index of (replica k*128 + hh*64 + 16*chunk, vertex row0 + r)
    auto elem0 = [&](const ItemInfo& it, int chunk) -> uint32_t {
      return (uint32_t)(it.k * RB + hh * 64 + chunk * 16) * np + (uint32_t)(it.row0 + r);
    };
    // float4 index of replicas 4m .. 4m+3 of this chunk's 16 (m = 0..3), vertex row0 + r
    auto quad0 = [&](const ItemInfo& it, int chunk) -> uint32_t {
      return (uint32_t)(it.k * (RB / 4) + hh * 16 + chunk * 4) * np + (uint32_t)(it.row0 + r);
    };
    // XT (kernel without checks, waves of at most three items per CTA): the TMEM columns
    // that no accumulator uses hold x of the first items, item i when i + n_items <= 3, at
    // columns (n_items + i) * 128 (one item of three, two of two, one of one).  The others
    // keep x in the blocked working copy.  A separate instantiation: the branches cost
    // waves of four-item CTAs about 3% of their step time.
    auto xt = [&](int i) { return XT && i + n_items <= 3; };
    auto xt_col = [&](int i) { return lane_base + (uint32_t)((n_items + i) * RB); };
    // y -> y / (dt c0) into the item's TMEM columns; x into TMEM or the working copy
    for (int i = 0; i < n_items; ++i) {
      const ItemInfo it = info[i];
      if (a.t0 > it.last_t) continue;
      const bool vr = r < it.valid;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float* yc = ys + elem0(it, c);
        const float* xc = xs + elem0(it, c);
        uint32_t v[16];
        float xv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = vr ? __float_as_uint(yc[j * np] * it.inv_dtc0) : 0u;
          xv[j] = vr ? xc[j * np] : 0.f;
        }
        if (!xt(i)) {
          float4* qc = a.xq + quad0(it, c);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            qc[m * np] = make_float4(xv[4 * m], xv[4 * m + 1], xv[4 * m + 2], xv[4 * m + 3]);
        }
        __syncwarp();
        if (xt(i)) tmem_st16f(xt_col(i) + (uint32_t)(c * 16), xv);
        tmem_st16(lane_base + (uint32_t)(i * RB + c * 16), v);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(edone0 + 8 * i);
    }
    // x is prefetched three 16-replica chunks ahead along the (step, item) sequence;
    // chunk c of any item always lands in xb[c]
    float xb[4][16];
    uint32_t dead = 0, n_chk = 0;  // items whose block stopped; check products read
    Cursor cur{0, -1};
    cur = next_live(cur, info, n_items, a.t0, n_steps, dead);
    ItemInfo nit = info[cur.i < n_items ? cur.i : 0];
    auto load_x = [&](float (&dst)[16], const ItemInfo& it, bool on, int chunk) {
      if (!on) return;
      // the prefetch may read what this thread stored one chunk earlier (a CTA with a
      // single item): both go through a.xq, so program order keeps it behind the store
      const float4* src = a.xq + quad0(it, chunk);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float4 q = src[m * np];
        dst[4 * m] = q.x;
        dst[4 * m + 1] = q.y;
        dst[4 * m + 2] = q.z;
        dst[4 * m + 3] = q.w;
      }
    };
    bool fresh = true;  // xb holds nothing for the cursor's item yet
    while (cur.u < n_steps) {
      if (fresh) {
        const bool gx = !xt(cur.i);
        load_x(xb[0], nit, gx, 0);
        load_x(xb[1], nit, gx, 1);
        load_x(xb[2], nit, gx, 2);
        fresh = false;
      }
      if (decision_step<CHECK>(a, a.t0 + cur.u, nit.steps_b)) {
        const bool dok = __all_sync(
            0xffffffffu, rwait(decb0 + 8 * cur.i, (uint32_t)((a.t0 + cur.u) / a.check_every) & 1u,
                               a.err, abort_flag));
        if (!dok) break;
        if (cur.u >= stop_u[cur.i]) {
          // the block stopped at the previous check: drop the item, and the x prefetched
          // for it
          dead |= 1u << cur.i;
          cur = next_live(cur, info, n_items, a.t0, n_steps, dead);
          nit = info[cur.u < n_steps ? cur.i : 0];
          fresh = true;
          continue;
        }
      }
      const ItemInfo it = nit;  // registers: the loop's stores cannot alias it
      const int t = a.t0 + cur.u;
      const Cursor nxt = next_live(cur, info, n_items, a.t0, n_steps, dead);
      const bool non = nxt.u < n_steps, gxn = non && !xt(nxt.i);
      // a check step: the energy of S_t after the update; the step before a check step
      // writes S_{t+1}
      const bool chk = check_step<CHECK>(a, t, it.steps_b), wchk = check_step<CHECK>(a, t + 1, it.steps_b);
      nit = info[non ? nxt.i : cur.i];
      const bool vr = r < it.valid, last = t == it.last_t;
      __nv_bfloat16* __restrict__ xh_out = (t & 1) ? a.xh0 : a.xh1;  // X_hat_{t+1}
      // -(a0 - a(t)) in FP64 as in the other step kernels (a(t) = a0 t / steps_b, with
      // the reciprocal taken once per item), by one lane, shared with the warp
      // and the deformation force dt h (1 - t / steps_b) (0 without deformation)
      float coef = 0.f, dtfe = 0.f;
      if (lane == 0) {
        coef = (float)(-(a.a0 - a.a0 * (double)t * it.inv_steps));
        dtfe = it.dth * (float)(1.0 - (double)t * it.inv_steps);
      }
      const float dtcx = a.dt * __shfl_sync(0xffffffffu, coef, 0);
      const float dtfe_s = __shfl_sync(0xffffffffu, dtfe, 0);
      const float dtc0 = it.dtc0, inv = it.inv_dtc0, dta0 = a.dta0;
      const bool ok = __all_sync(0xffffffffu, rwait(accf0 + 8 * cur.i, (uint32_t)cur.u & 1u,
                                                    a.err, abort_flag));
      if (!ok) break;
      tc_fence_after();
      if (warp == 2 && lane == 0) trace_at(a, cur.u, cur.i, TR_EPI_START);
      const uint32_t col0 = lane_base + (uint32_t)(cur.i * RB);
      const bool xti = xt(cur.i);
      const uint32_t xcol = xt_col(cur.i);
      uint32_t va[16], vb[16];
      __syncwarp();
      if (xti) {  // x of all four chunks from TMEM, awaited with the first product chunk
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16f(xcol + (uint32_t)(c * 16), xb[c]);
      }
      tmem_ld16_async(col0, va);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t(&v)[16] = (c & 1) ? vb : va;
        uint32_t(&vn)[16] = (c & 1) ? va : vb;
        tmem_wait_ld(v);
        if (c == 0 && xti) {  // nothing is in flight now: these waits return at once
          tmem_wait_ld_f(xb[0]);
          tmem_wait_ld_f(xb[1]);
          tmem_wait_ld_f(xb[2]);
          tmem_wait_ld_f(xb[3]);
        }
        if (c < 3) {
          __syncwarp();
          tmem_ld16_async(col0 + (uint32_t)((c + 1) * 16), vn);
        }
        // chunk c + 3 of the sequence: chunk 3 of this item, else 0..2 of the next
        if (c == 0)
          load_x(xb[3], it, !xti, 3);
        else
          load_x(xb[c - 1], nit, gxn, c - 1);
        const uint32_t e0 = elem0(it, c);
        float* xc = xs + e0;
        float* yc = ys + e0;
        __nv_bfloat16* hc = xh_out + e0;
        float4* qc = a.xq + quad0(it, c);
        uint32_t out[16];
        float xo[16], yo[16];
        const float2 dtc0_2 = make_float2(dtc0, dtc0), dta0_2 = make_float2(dta0, dta0);
        const float2 inv_2 = make_float2(inv, inv), dtcx_2 = make_float2(dtcx, dtcx);
        const float2 dtfe_2 = make_float2(dtfe_s, dtfe_s);
#pragma unroll
        for (int j = 0; j < 16; j += 2) {  // element pairs on the packed FP32x2 pipe
          const float2 x0 = make_float2(xb[c][j], xb[c][j + 1]);
          const float2 acc = make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1]));
          // adiabatic SB: -(x^2 + a0 - a(t)); no walls
          float2 cx = dtcx_2;
          if (SB == QH_SB_ADIABATIC)
            cx = __ffma2_rn(make_float2(-a.dt * x0.x, -a.dt * x0.y), x0, dtcx_2);
          const float2 y1 = __ffma2_rn(dtc0_2, acc, __ffma2_rn(cx, x0, dtfe_2));
          const float2 x1 = __ffma2_rn(dta0_2, y1, x0);
          const bool w0 = SB != QH_SB_ADIABATIC && fabsf(x1.x) > 1.f;
          const bool w1 = SB != QH_SB_ADIABATIC && fabsf(x1.y) > 1.f;
          xo[j] = w0 ? copysignf(1.f, x1.x) : x1.x;
          xo[j + 1] = w1 ? copysignf(1.f, x1.y) : x1.y;
          yo[j] = w0 ? 0.f : y1.x;
          yo[j + 1] = w1 ? 0.f : y1.y;
          // padding vertices (J rows of zeros) may drift under the deformation field,
          // in TMEM only: their x, y and X_hat are never stored (vr)
          const float2 ys = __fmul2_rn(make_float2(yo[j], yo[j + 1]), inv_2);
          out[j] = __float_as_uint(ys.x);
          out[j + 1] = __float_as_uint(ys.y);
        }
        if (vr) {
#pragma unroll
          for (int j = 0; j < 16; ++j) hc[j * np] = __float2bfloat16_rn(sb_operand(SB, xo[j]));
          if (!last) {
            if (!xti) {
#pragma unroll
              for (int m = 0; m < 4; ++m)
                qc[m * np] = make_float4(xo[4 * m], xo[4 * m + 1], xo[4 * m + 2], xo[4 * m + 3]);
            }
          } else {  // the launch's last step: state back into the solver's layout
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              xc[j * np] = xo[j];
              yc[j * np] = yo[j];
            }
          }
        }
        if (!last) {
          __syncwarp();
          if (xti) tmem_st16f(xcol + (uint32_t)(c * 16), xo);
          tmem_st16(col0 + (uint32_t)(c * 16), out);
        }
      }
      if (!last) tmem_wait_st();
      // S_{t+1} = sgn(x_{t+1}) before the arrive, so that the release covers it
      if (wchk && vr)
        write_signs(a.xq + quad0(it, 0), np,
                    ((((t + 1) / a.check_every) & 1) ? a.s1 : a.s0) + elem0(it, 0));
      tc_fence_before();
      __syncwarp();
      if (warp == 2 && lane == 0) trace_at(a, cur.u, cur.i, TR_EPI_END);
      if (lane == 0) mbar_arrive(edone0 + 8 * cur.i);
      if (chk) {
        const int par = (t / a.check_every) & 1;
        const int32_t R = a.n_kt * RB;
        const size_t eo = ((size_t)par * a.n_blocks + it.block) * R;
        const size_t eo1 = ((size_t)(par ^ 1) * a.n_blocks + it.block) * R;
        const bool cok = check_energy(
            tmem + ((uint32_t)(qd * 32) << 16) + SPARE_COL + (uint32_t)(hh * 64),
            (par ? a.s1 : a.s0) + elem0(it, 0), np,
            a.e_sum + eo, a.e_sum + eo + it.k * RB + hh * 64, a.e_sum + eo1,
            a.e_cnt + (size_t)par * a.n_blocks + it.block,
            a.e_cnt + (size_t)(par ^ 1) * a.n_blocks + it.block,
            it.rows_b * (uint32_t)a.n_kt * EPI_WARPS, R, a.sum_w[it.block], a.seen + it.block,
            a.stall + it.block, a.stop_t + it.block, a.decided + it.block, t, a.check_every,
            a.patience, sfull, sfree, n_chk, a.err, abort_flag, lane,
            a.check_trace ? a.check_trace + (size_t)(t / a.check_every - 1) * a.n_blocks + it.block
                          : nullptr);
        if (!cok) break;
        ++n_chk;
      }
      cur = nxt;
    }
  } else if (warp == JPROD_WARP) {
    // ------------------------------------------------------------ J producer
    // Stream mode without checks, when the host asks for it: the J K-slices depend on no
    // other CTA, so they go into a ring of their own as soon as the MMAs free a slot,
    // ahead of the X_hat copies that wait for the neighbours' releases.  The warp walks
    // the MMA issuer's sequence of (step, item, K-slice), lanes 0 .. ST-1 one K-slice
    // each.  Lane s < ST keeps the latest use of ring slot s, so that the copies still in
    // flight land before the exit.
    if (jsplit && n_items > 0) {
      uint32_t q = 0;
      int32_t last_use = -1;
      bool ok = true;
      for (int u = 0; ok && u < n_steps; ++u) {
        const int t = a.t0 + u;
        for (int i = 0; ok && i < n_items; ++i) {
          const ItemInfo& it = info[i];
          if (t > it.last_t) continue;
          for (int kb0 = 0; ok && kb0 < it.nk; kb0 += ST) {
            const int kb = kb0 + lane;
            const bool mine = lane < ST && kb < it.nk;
            bool lok = true;
            if (mine) {
              const int s = (int)((q + kb) % ST);
              const uint32_t ph = ((q + kb) / ST) & 1u;
              lok = rwait(empty0 + 8 * s, ph ^ 1u, a.err, abort_flag);
              if (lok) {
                mbar_expect_tx(fullj0 + 8 * s, SLICE);
                tma_load_2d(smem_u32(smem + L::RING_OFF + s * L::SLOT), &tmJ, fullj0 + 8 * s,
                            (kb & 1) * 64, (it.tile_begin + (kb >> 1)) * TILE);
              }
            }
            const uint32_t issued = __ballot_sync(0xffffffffu, mine && lok);
            if (lane < ST) {  // this round's use of slot `lane`, if it was issued
              const int kbs = kb0 + (int)(((uint32_t)lane + 2u * ST - (q + kb0) % ST) % ST);
              if ((issued >> (kbs - kb0)) & 1u) last_use = (int32_t)(q + kbs);
            }
            if (!__all_sync(0xffffffffu, !mine || lok)) ok = false;
          }
          q += (uint32_t)it.nk;
        }
      }
      if (last_use >= 0) mbar_wait(fullj0 + 8 * lane, ((uint32_t)last_use / ST) & 1u, a.err);
    }
  } else {
    // ------------------------------------------------------------ signal
    // After the epilogue of an item, release its X_hat_{t+1} to the other CTAs.
    if (lane == 0) {
      // A parity wait also succeeds on the previous phase of that parity, so every
      // phase of edone is observed in order: first phase 0 (the initial y store).
      bool ok = true;
      for (int i = 0; ok && i < n_items; ++i)
        if (a.t0 <= info[i].last_t) ok = rwait(edone0 + 8 * i, 0u, a.err, abort_flag);
      uint32_t dead = 0;
      for (int u = 0; ok && u < n_steps; ++u) {
        const int t = a.t0 + u;
        for (int i = 0; i < n_items; ++i) {
          const ItemInfo& it = info[i];
          if (t > it.last_t || ((dead >> i) & 1u)) continue;
          if (decision_step<CHECK>(a, t, it.steps_b)) {
            if (!(ok = rwait(decb0 + 8 * i, (uint32_t)(t / a.check_every) & 1u, a.err,
                             abort_flag)))
              break;
            if (u >= stop_u[i]) {
              dead |= 1u << i;
              continue;
            }
          }
          // phase 0 of edone is the initial y store; step u completes phase u + 1
          if (!(ok = rwait(edone0 + 8 * i, (uint32_t)(u + 1) & 1u, a.err, abort_flag))) break;
          if (t == it.last_t) continue;  // nobody waits for X_hat beyond this launch
          // the epilogue's stores happen-before this thread's edone acquire (mbarrier,
          // CTA scope); the gpu-scope release below is cumulative over them
          fence_proxy_async_global();
          red_release_gpu_add(
              a.done + (size_t)(a.group_sync ? it.block : it.rt) * a.n_kt + it.k, 1u);
          trace_at(a, u, i, TR_RELEASE);
        }
        if (!ok) break;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// A block stopped at check step t keeps the signs it had there: x <- S of t's parity
// (exactly +-1, so sgn(x) is that check's spin pattern), steps_run <- t.
__global__ void k_stop_fixup(int64_t n, int32_t n_pad, const int32_t* __restrict__ pad_node,
                             const int32_t* __restrict__ block_of,
                             const int32_t* __restrict__ stop_t, int32_t check_every,
                             const __nv_bfloat16* __restrict__ s0,
                             const __nv_bfloat16* __restrict__ s1, float* x) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t node = pad_node[e % n_pad];
  if (node < 0) return;
  const int32_t t = stop_t[block_of[node]];
  if (t < 0) return;
  x[e] = __bfloat162float((((t / check_every) & 1) ? s1 : s0)[e]);
}

__global__ void k_stop_steps(int32_t nb, const int32_t* __restrict__ stop_t, int32_t* steps_run) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb && stop_t[b] >= 0) steps_run[b] = stop_t[b];
}

}  // namespace

void launch_stop_fixup(cudaStream_t s, const Graph& g, int32_t R, const RunCheck& c, float* x,
                       int32_t* steps_run) {
  const int64_t n = (int64_t)R * g.n_pad;
  if (n > 0)
    k_stop_fixup<<<::qh::counted((unsigned)((n + 255) / 256)), 256, 0, s>>>(
        n, g.n_pad, g.pad_node, g.block_of, c.stop_t, c.check_every, c.s,
        c.s + (size_t)R * g.n_pad, x);
  if (g.n_blocks > 0)
    k_stop_steps<<<::qh::counted((unsigned)((g.n_blocks + 255) / 256)), 256, 0, s>>>(
        g.n_blocks, c.stop_t, steps_run);
}

// ---------------------------------------------------------------------------
// Host side.

bool run_variant(int v) { return v >= RUN_VARIANT_FIRST && v < RUN_VARIANT_FIRST + 4; }
static bool run_jres(int v) { return v == RUN_VARIANT_FIRST || v == RUN_VARIANT_FIRST + 2; }
static bool run_group(int v) { return v == RUN_VARIANT_FIRST || v == RUN_VARIANT_FIRST + 3; }

// Work split.  Items are numbered row-tile-major (item = row_tile * n_kt + k), and
// the blocks' row tiles are contiguous.  Blocks (all, or those of a partial solve)
// are packed into waves whose items fit on chip (at most MAX_ITEMS per SM); a wave
// lists its items row-tile-major and is one launch over the step range, and the
// waves run one after the other.
// Within a wave a CTA processes its items in a fixed order every step, and the split
// puts the row-tile neighbours of an item (item -+ n_kt, same k) at the same position
// in their CTAs, so an item's inputs for step t+1 are finished a whole step period
// before it needs them.  JRES: every CTA takes up to MAX_ITEMS consecutive replica
// tiles of ONE row tile (its J tiles stay resident), the same k ranges in every row.
// Stream: CTA c of the wave's G CTAs takes the wave's items c, c + G, c + 2G, ...
// False when some block does not fit one wave.
bool run_plan(const Graph& g, int R, int n_sm, int variant, bool use_lo, RunPlan* plan,
              const std::vector<int32_t>* mask, int max_items) {
  if (!run_variant(variant) || max_items < 1 || max_items > MAX_ITEMS) return false;
  const bool jres = run_jres(variant);
  if (R % RB != 0 || g.n_row_tiles == 0 || g.csr_mode || n_sm < 1) return false;
  const int n_kt = R / RB;
  const int cpr = (n_kt + max_items - 1) / max_items;  // JRES: CTAs per row tile
  if (jres)
    for (const RowTile& rt : g.h_rt)
      if ((use_lo ? rt.n_all : rt.n_hi) > JRES_TILES) return false;
  // row-tile range of every block (blocks appear in order in the row-tile list)
  std::vector<int32_t> first(std::max(g.n_blocks, 1), -1), count(std::max(g.n_blocks, 1), 0);
  for (int32_t r = 0; r < g.n_row_tiles; ++r) {
    const int32_t b = g.h_rt[r].block;
    if (mask && !(*mask)[b]) continue;
    if (first[b] < 0) first[b] = r;
    count[b] += 1;
  }
  // a block's load on one wave: CTAs (JRES) or items (stream)
  const int64_t cap = jres ? n_sm : (int64_t)max_items * n_sm;
  auto load = [&](int32_t b) -> int64_t { return (int64_t)count[b] * (jres ? cpr : n_kt); };
  int64_t total = 0;
  for (int32_t b = 0; b < g.n_blocks; ++b) {
    if (load(b) > cap) return false;
    total += load(b);
  }
  const int64_t n_waves = (total + cap - 1) / cap;
  const int64_t target = (total + n_waves - 1) / n_waves;
  RunPlan p;
  // a wave's items: those of its row tiles, row-tile-major; work entries index this list
  auto emit = [&](const std::vector<int32_t>& rows) {
    RunWave w;
    w.work_off = (int)p.work.size();
    w.item_off = (int)p.items.size();
    for (int32_t r : rows)
      for (int k = 0; k < n_kt; ++k) p.items.push_back(r * n_kt + k);
    if (jres) {
      for (size_t j = 0; j < rows.size(); ++j)
        for (int c = 0; c < cpr; ++c) {
          const int b = (int)((int64_t)n_kt * c / cpr), e = (int)((int64_t)n_kt * (c + 1) / cpr);
          p.work.push_back(make_int2((int)j * n_kt + b, e - b));
        }
      w.stride = 1;
    } else {
      const int64_t n = (int64_t)rows.size() * n_kt;
      const int64_t grid = std::min<int64_t>(n_sm, n);
      for (int64_t c = 0; c < grid; ++c)
        p.work.push_back(make_int2((int)c, (int)((n - c + grid - 1) / grid)));
      w.stride = (int)grid;
    }
    w.grid = (int)p.work.size() - w.work_off;
    for (int c = w.work_off; c < (int)p.work.size(); ++c) w.max_items = std::max(w.max_items, p.work[c].y);
    p.waves.push_back(w);
  };
  std::vector<int32_t> rows;
  int64_t cur = 0;
  for (int32_t b = 0; b < g.n_blocks; ++b) {
    if (count[b] == 0) continue;
    if (!rows.empty() && cur + load(b) > target) {  // target <= cap
      emit(rows);
      rows.clear();
      cur = 0;
    }
    for (int32_t r = first[b]; r < first[b] + count[b]; ++r) rows.push_back(r);
    cur += load(b);
  }
  if (!rows.empty()) emit(rows);
  if (plan) *plan = std::move(p);
  return true;
}

// Items per CTA for a solve: three or four, whichever gives the fewer step-periods of
// waves.  A CTA runs its items' epilogues one after another, so four items make the step
// period epilogue-bound: measured on batched-blocks (R = 256, 11,048 items), 13.5 µs per
// step at four items per CTA (20 waves) against 9.44 µs at three (27 waves, x of one item
// in TMEM), a ratio of 0.70.  Three items win unless they need more than 1/0.70 times
// the waves (a graph that fits one wave at four but not at three keeps four).
int run_items(const Graph& g, int R, int n_sm, int variant, bool use_lo,
              const std::vector<int32_t>* mask) {
  RunPlan p3, p4;
  if (!run_plan(g, R, n_sm, variant, use_lo, &p3, mask, 3)) return MAX_ITEMS;
  if (!run_plan(g, R, n_sm, variant, use_lo, &p4, mask, MAX_ITEMS)) return 3;
  return 100 * (int64_t)p3.waves.size() <= 143 * (int64_t)p4.waves.size() ? 3 : MAX_ITEMS;
}

qh_status run_prepare(Ctx* ctx, const Graph& g, int R, int variant, bool use_lo, RunBufs* rb,
                      const std::vector<int32_t>* mask, int max_items) {
  RunPlan plan;
  if (!run_plan(g, R, ctx->n_sm, variant, use_lo, &plan, mask, max_items))
    return set_err(ctx, QH_EINVAL, "multi-step kernel: a block does not fit one wave");
  const int n_kt = R / RB;
  rb->jres = run_jres(variant);
  rb->group_sync = run_group(variant);
  // J copies run ahead in their own ring when most row tiles span more K-slices (2 per
  // stored tile entry) than the operand ring holds: the copies of their later K-slices
  // wait for ring slots, and without the split the J copies wait with them.  Rows that
  // fit the ring measured slower with the split (one more wait per K-slice).
  int64_t wide = 0;
  for (const RowTile& rt : g.h_rt)
    if (2 * (use_lo ? rt.n_all : rt.n_hi) > RunSmem<false>::ST) ++wide;
  rb->jsplit = 2 * wide > (int64_t)g.h_rt.size();
  rb->waves = plan.waves;
  std::vector<int32_t> rows(std::max(g.n_blocks, 1), 0);
  for (const RowTile& rt : g.h_rt) rows[rt.block] += 1;
  rb->n_done = (int64_t)(rb->group_sync ? (int64_t)rows.size() : g.n_row_tiles) * n_kt;
  rb->work = (int2*)ctx->scratch(std::max<size_t>(plan.work.size(), 1) * sizeof(int2), S_RUN_WORK);
  rb->items = (int32_t*)ctx->scratch(std::max<size_t>(plan.items.size(), 1) * 4, S_RUN_ITEMS);
  rb->rows_b = (int32_t*)ctx->scratch(rows.size() * 4, S_RUN_ROWS);
  rb->done = (uint32_t*)ctx->scratch((size_t)rb->n_done * 4, S_RUN_DONE);
  rb->xq = (float4*)ctx->scratch((size_t)R * g.n_pad * 4, S_RUN_XQ);
  if (!rb->work || !rb->items || !rb->rows_b || !rb->done || !rb->xq)
    return set_err(ctx, QH_ENOMEM, "allocation failed (multi-step kernel)");
  QH_CUDA_TRY(cudaMemcpyAsync(rb->work, plan.work.data(), plan.work.size() * sizeof(int2),
                              cudaMemcpyHostToDevice, ctx->stream));
  QH_CUDA_TRY(cudaMemcpyAsync(rb->items, plan.items.data(), plan.items.size() * 4,
                              cudaMemcpyHostToDevice, ctx->stream));
  QH_CUDA_TRY(cudaMemcpyAsync(rb->rows_b, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice,
                              ctx->stream));
  return QH_OK;
}

template <bool JRES, int SB>
qh_status launch_run_impl(Ctx* ctx, const Graph& g, const StepArgs& s, const RunBufs& rb,
                          __nv_bfloat16* xh0, __nv_bfloat16* xh1, int t0, int t1,
                          unsigned long long* trace, int trace_u0, int trace_nu,
                          const RunCheck* chk) {
  using L = RunSmem<JRES>;
  CUtensorMap mJ, mX0, mX1, mS0, mS1;
  // without checks the S maps repeat the X_hat ones (never loaded)
  __nv_bfloat16* s0 = chk ? chk->s : xh0;
  __nv_bfloat16* s1 = chk ? chk->s + (size_t)s.R * g.n_pad : xh1;
  if (!make_map(&mJ, g.tile_bf16, TILE, (uint64_t)std::max<int64_t>(g.n_tiles, 1) * TILE, TILE) ||
      !make_map(&mX0, xh0, (uint64_t)g.n_pad, (uint64_t)s.R, RB) ||
      !make_map(&mX1, xh1, (uint64_t)g.n_pad, (uint64_t)s.R, RB) ||
      !make_map(&mS0, s0, (uint64_t)g.n_pad, (uint64_t)s.R, RB) ||
      !make_map(&mS1, s1, (uint64_t)g.n_pad, (uint64_t)s.R, RB))
    return set_err(ctx, QH_ECUDA, "cuTensorMapEncodeTiled failed (multi-step kernel)");
  RunArgs a{};
  a.rt = s.rt;
  a.tile_col = s.tile_col;
  a.x = s.x;
  a.y = s.y;
  a.xq = rb.xq;
  a.xh0 = xh0;
  a.xh1 = xh1;
  a.c0 = s.c0;
  a.active = s.active;
  a.steps_b = s.steps_b;
  a.done = rb.done;
  a.work = rb.work;
  a.rows_b = rb.rows_b;
  a.group_sync = rb.group_sync ? 1 : 0;
  a.jsplit = (!JRES && chk == nullptr && rb.jsplit) ? 1 : 0;
  a.n_pad = s.n_pad;
  a.n_kt = s.R / RB;
  a.n_blocks = g.n_blocks;
  a.t0 = t0;
  a.t1 = t1;
  a.use_lo = s.use_lo;
  a.dt = s.dt;
  a.dta0 = s.dta0;
  a.a0 = s.a0;
  a.err = s.err;
  a.deform = s.deform;
  a.trace = trace;
  a.trace_u0 = trace_u0;
  a.trace_nu = trace_nu;
  if (chk) {
    a.check_every = chk->check_every;
    a.patience = chk->patience;
    a.s0 = s0;
    a.s1 = s1;
    a.sum_w = chk->sum_w;
    a.e_sum = chk->e_sum;
    a.e_cnt = chk->e_cnt;
    a.decided = chk->decided;
    a.seen = chk->seen;
    a.stall = chk->stall;
    a.stop_t = chk->stop_t;
    a.check_trace = chk->trace;
  }
  // every wave's counters start from zero; waves use disjoint counters
  QH_CUDA_TRY(cudaMemsetAsync(rb.done, 0, (size_t)rb.n_done * 4, ctx->stream));
  for (const RunWave& w : rb.waves) {
    a.work = rb.work + w.work_off;
    a.items = rb.items + w.item_off;
    a.item_stride = w.stride;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)w.grid);
    cfg.blockDim = dim3(RUN_THREADS);
    cfg.dynamicSmemBytes = L::BYTES;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the waits always end
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch(1);
    cudaError_t e =
        chk         ? cudaLaunchKernelEx(&cfg, k_bsb_run<JRES, SB, true, false>, mJ, mX0, mX1, mS0,
                                         mS1, a)
        : w.max_items <= 3
            ? cudaLaunchKernelEx(&cfg, k_bsb_run<JRES, SB, false, true>, mJ, mX0, mX1, mS0, mS1, a)
            : cudaLaunchKernelEx(&cfg, k_bsb_run<JRES, SB, false, false>, mJ, mX0, mX1, mS0, mS1,
                                 a);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_bsb_run launch");
  }
  return QH_OK;
}

qh_status launch_run(Ctx* ctx, const Graph& g, const StepArgs& s, const RunBufs& rb,
                     __nv_bfloat16* xh0, __nv_bfloat16* xh1, int t0, int t1,
                     unsigned long long* trace, int trace_u0, int trace_nu,
                     const RunCheck* check) {
  if (g.n_row_tiles == 0 || t1 <= t0) return QH_OK;
  if (check && (check->check_every < 1 || check->patience < 1 || t0 != 0))
    return set_err(ctx, QH_EINVAL, "multi-step checks need check_every, patience >= 1 from step 0");
#define QH_RUN_CASE(J, V) \
  launch_run_impl<J, V>(ctx, g, s, rb, xh0, xh1, t0, t1, trace, trace_u0, trace_nu, check)
  switch (s.sb * 2 + (rb.jres ? 1 : 0)) {
    case 0: return QH_RUN_CASE(false, QH_SB_BALLISTIC);
    case 1: return QH_RUN_CASE(true, QH_SB_BALLISTIC);
    case 2: return QH_RUN_CASE(false, QH_SB_DISCRETE);
    case 3: return QH_RUN_CASE(true, QH_SB_DISCRETE);
    case 4: return QH_RUN_CASE(false, QH_SB_ADIABATIC);
    case 5: return QH_RUN_CASE(true, QH_SB_ADIABATIC);
    default: return set_err(ctx, QH_EINVAL, "bad SB variant");
  }
#undef QH_RUN_CASE
}

int run_trace_events() { return TRACE_EVENTS; }
int run_max_items() { return MAX_ITEMS; }
int run_item_mask() { return 0x7fffffff; }

template <bool JRES, int SB>
static cudaError_t run_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_bsb_run<JRES, SB, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)RunSmem<JRES>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bsb_run<JRES, SB, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RunSmem<JRES>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bsb_run<JRES, SB, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RunSmem<JRES>::BYTES);
  return e;
}

qh_status launch_wait_probe(Ctx* ctx, int which) {
  uint32_t* counter = (uint32_t*)ctx->scratch(16, S_WAIT_PROBE);
  if (!counter) return set_err(ctx, QH_ENOMEM, "allocation failed (wait probe)");
  QH_CUDA_TRY(cudaMemsetAsync(counter, 0, 16, ctx->stream));
  k_wait_probe<<<::qh::counted(1), 32, 0, ctx->stream>>>(which, counter, ctx->d_err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_wait_probe launch");
  return QH_OK;
}

cudaError_t run_set_attrs() {
  cudaError_t e = run_attr<true, QH_SB_BALLISTIC>();
  if (e == cudaSuccess) e = run_attr<false, QH_SB_BALLISTIC>();
  if (e == cudaSuccess) e = run_attr<true, QH_SB_DISCRETE>();
  if (e == cudaSuccess) e = run_attr<false, QH_SB_DISCRETE>();
  if (e == cudaSuccess) e = run_attr<true, QH_SB_ADIABATIC>();
  if (e == cudaSuccess) e = run_attr<false, QH_SB_ADIABATIC>();
  return e;
}

}  // namespace qh
