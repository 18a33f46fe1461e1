// Internal declarations shared by the CUDA translation units of libqhap.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string.h>

#include <memory>
#include <string>
#include <vector>

#include "qhap.h"

namespace qh {

// Kernel-launch counter of this process (every launch site wraps its grid in
// counted(); replays of a captured step loop add the loop's kernel count).
void note_launch(int64_t n = 1);
int64_t launches();
template <class G>
inline G counted(G grid) {
  note_launch();
  return grid;
}

constexpr int TILE = 128;           // J tile edge (rows = MMA M, columns = 2 x 64 K-slices)
constexpr int SNP_ROW_CAP = 8192;   // max fragment terms gathered for one SNP row (sort path)
constexpr int SNP_DENSE_CAP = 12288;  // max SNP window of one row for the dense path

// Device error word bits (set by kernels, read back by the host).
enum : int32_t {
  ERR_INPUT = 1,        // malformed fragments
  ERR_QUAL = 2,         // Phred quality outside [4, 93]
  ERR_ROWCAP = 4,       // SNP row over SNP_ROW_CAP terms
  ERR_TIMEOUT = 8,      // bounded wait expired (mbarrier)
  ERR_CONFIG = 16,      // a kernel refused the launch's arguments (host-side slip)
};

struct RowTile {           // one 128-row slab of a block in the padded layout
  int32_t block;           // phase block
  int32_t row0;            // first padded row (multiple of 128)
  int32_t valid;           // rows < valid are real vertices
  int32_t tile_begin;      // first entry in tile_col / BF16 tile data
  int32_t n_hi;            // entries carrying J (FP32 path uses these only)
  int32_t n_all;           // hi entries followed by lo (BF16 remainder) entries
  int32_t f32_begin;       // first FP32 tile of this row tile
  int32_t pad_;
};

// Device memory of graphs and solutions comes from the owning context's stream-ordered
// pool: allocation and release need no device synchronisation.  A handle may outlive
// its context; `alive` tells whether the context (its stream and pool) still exists.
struct PoolRef {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  std::shared_ptr<bool> alive;
  // Allocation-failure injection (test hook): device allocations left before every
  // further one fails; -1 = off.  Shared by the context's scratch and its graphs.
  std::shared_ptr<int64_t> fail_after;
};
// false when the injected failure point is reached (counts the allocation otherwise)
bool alloc_permitted(const PoolRef& m);
void* pool_alloc(const PoolRef& m, size_t bytes, std::vector<void*>* owner);
void pool_free_all(const PoolRef& m, std::vector<void*>* owned);

struct Graph {
  int mode = 0, weight_mode = 1, linkage_k = 10;
  double porec_alpha = 0.1;
  int32_t n_frags = 0, n_snps = 0, n_nodes = 0;
  int64_t nnz_frag = 0;
  // fragments (device)
  int64_t* frag_ptr = nullptr;
  int32_t* snp = nullptr;
  int8_t* allele = nullptr;
  uint8_t* qual = nullptr;
  uint8_t* is_porec = nullptr;
  // SNP -> covering fragments (device), fragments ascending per SNP
  int64_t* cov_ptr = nullptr;
  int32_t* cov_frag = nullptr;
  int8_t* cov_allele = nullptr;
  // edges (device), both directions
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* w = nullptr;         // weights A (exact integers in READ mode)
  bool integer_weights = true;
  double max_abs_w = 0.0;
  // components / blocks
  int32_t n_blocks = 0;
  int32_t* block_of = nullptr;    // [n_nodes], -1 = dropped
  int32_t* local = nullptr;       // [n_nodes]
  int32_t* pad_index = nullptr;   // [n_nodes], -1 = dropped
  int32_t* pad_node = nullptr;    // [n_pad] -> vertex or -1
  int64_t* block_ptr = nullptr;   // [n_blocks+1] into perm
  int32_t* perm = nullptr;        // vertices of each block, ascending
  int32_t* pad_off = nullptr;     // [n_blocks+1] padded offsets (device)
  std::vector<int32_t> h_block_size, h_pad_off;
  std::vector<int64_t> h_block_ptr;
  int32_t n_pad = 0;
  // tiles
  int32_t n_row_tiles = 0;
  int64_t n_tiles = 0;            // all BF16 entries (hi + lo)
  int64_t n_tiles_hi = 0;         // FP32 tiles
  bool has_lo = false;
  int32_t max_tiles_per_row = 0;  // largest n_all over row tiles
  RowTile* rt = nullptr;          // [n_row_tiles]
  int32_t* rt_of_block = nullptr; // [n_blocks] first row tile of the block
  int32_t* tile_col = nullptr;    // [n_tiles] column tile (padded col / 128)
  int64_t* slot_off = nullptr;    // [n_blocks+1] tile-slot offsets (T_b^2 slots per block)
  int32_t* tiles_per_block = nullptr;  // [n_blocks] T_b
  int64_t* slot_tile = nullptr;   // [slots+1] exclusive scan of nonzero slots
  __nv_bfloat16* tile_bf16 = nullptr;  // [n_tiles][128][128] row-major
  float* tile_f32 = nullptr;           // [n_tiles_hi][128][128] row-major
  std::vector<RowTile> h_rt;
  // padded CSR of J (always built; the solver's operand when csr_mode)
  bool csr_mode = false;
  int64_t pnnz = 0;             // stored entries (w != 0 only)
  int64_t* prow_ptr = nullptr;  // [n_pad+1]
  int32_t* pcol = nullptr;      // [nnz] padded column
  float* pval = nullptr;        // [nnz] J = -w (FP32)
  // CSR mode: J split into a band and a remainder for the BF16 band-tile step.  The
  // band holds the entries whose padded column lies in the row's tile or in one of its
  // two neighbour tiles, as three dense 128 x 128 BF16 tiles per row tile (offsets -1,
  // 0, +1); the remainder CSR holds every other stored entry (FP32).
  __nv_bfloat16* band = nullptr;  // [n_row_tiles][3][128][128] row-major, J = -w
  int64_t rnnz = 0;
  int64_t* rrow_ptr = nullptr;    // [n_pad+1]
  int32_t* rcol = nullptr;        // [rnnz] padded column
  float* rval = nullptr;          // [rnnz] J = -w (FP32)
  // per-block constants
  double* sum_w = nullptr;        // [n_blocks] sum_{a,b} w_ab (both triangles)
  double* sum_j2 = nullptr;       // [n_blocks]
  std::vector<double> h_c0;       // default c0 per block
  std::vector<double> h_sum_w;
  // all device allocations of this graph, freed together
  std::vector<void*> allocs;
  PoolRef mem;
};

struct Solution {
  int mode = 0;
  int32_t n_blocks = 0, R = 0, replica_base = 0, n_nodes = 0;
  std::vector<int32_t> best_r, steps_run, iters;
  std::vector<double> best_cut;
  std::vector<double> cuts_first;        // [n_blocks * R]
  std::vector<int8_t> spins;             // [n_nodes] best spins by vertex (0 = dropped)
  std::vector<int32_t> C;                // SNP mode flip counts [n_nodes] (-1: block not solved)
  std::vector<uint8_t> solved;           // [n_blocks] 1 = solved here or imported
  // SNP refinement state after the last solve, for a later call that continues it:
  // solves run over the graph, and per block whether it still refines, its deformation
  // field and re-solves used; per vertex the gauge the next solve starts from
  int32_t refine_done = 0;
  // energy checks of the first solve: [checks][n_blocks] best cut per check (NaN: the
  // block was not running), checks every check_every steps
  std::vector<double> check_trace;
  int32_t check_every = 0;
  std::vector<int32_t> refining, refine_tries;
  std::vector<float> refine_deform;
  std::vector<int8_t> refine_gauge;
  mutable bool device_stale = false;     // host spins / C changed after the device copies
  double solve_ms = 0, step_ms = 0, spin_updates = 0;
  int64_t n_step_launches = 0;
  std::string kernel;                    // step kernel that ran
  std::vector<int32_t> block_size;
  std::vector<int64_t> block_ptr;        // host copy for per-block extraction
  std::vector<int32_t> perm;             // vertices of each block, ascending (host copy)
  int8_t* d_spins = nullptr;             // device [n_nodes]
  int32_t* d_C = nullptr;                // device [n_nodes]
  std::vector<void*> allocs;
  PoolRef mem;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  PoolRef mem;  // pool for graph and solution memory (on this context's stream)
  int n_sm = 148;
  std::string err;
  int32_t* d_err = nullptr;
  std::vector<void*> slots;         // grow-only scratch buffers
  std::vector<size_t> slot_bytes;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // one captured step loop, replayed while its shape is unchanged
  cudaGraphExec_t loop_exec = nullptr;
  std::string loop_key;
  int64_t loop_kernels = 0;  // kernels launched by one replay of loop_exec
  // step-kernel autotuning: shape key -> chosen variant, and the last report
  std::vector<std::pair<std::string, int>> tuned;
  std::string tune_report;
  void* scratch(size_t bytes, int slot);
};

// Device-side view handed to the step kernels.
struct StepArgs {
  const RowTile* rt;
  const int32_t* tile_col;
  const float* tile_f32;
  float* x;               // [R][n_pad]  (BF16 path: in place)
  float* y;               // [R][n_pad]
  const float* xin;       // FP32 path: x_t operand (double-buffered)
  float* xout;            // FP32 path: x_{t+1}
  __nv_bfloat16* xh_out;  // BF16 path: X_hat_{t+1}
  float* z_out;           // debug matvec: Z output (nullptr in solver steps)
  const float* c0;        // [n_blocks]
  const int32_t* active;  // [n_blocks] or nullptr
  const int32_t* steps_b;  // [n_blocks] schedule length per block (a(t) = a0 t / steps_b)
  int32_t n_pad, R;
  int32_t t;              // step index
  int32_t use_lo;         // BF16 paths: also accumulate the lo (remainder) tiles
  uint8_t* x8h_out;       // FP8 path: e4m3 hi / lo parts of X_{t+1}
  uint8_t* x8l_out;
  float inv_scale;        // FP8 path: 1 / s of the scaled J tiles
  float dt, dta0;         // dta0 = dt * a0
  double a0;
  int32_t* err;
  int32_t sb;             // SB variant: QH_SB_BALLISTIC, QH_SB_DISCRETE, QH_SB_ADIABATIC
  const float* zb;        // CSR step: band product Z = J_band X_hat ([n_pad][R], FP32) to
                          // start the accumulation from, or nullptr
  const float* deform;    // [n_blocks] deformation field strength h_b of this solve, or
                          // nullptr: y gains dt h_b (1 - t / steps_b) (uniform field
                          // along the incumbent, all +1 in the refinement's gauged frame)
};

// The deformation field's force at step t of a block with schedule length sb.
__device__ __forceinline__ float deform_force(const float* deform, int32_t block, int32_t t,
                                              int32_t sb) {
  return deform ? deform[block] * (1.f - (float)t / (float)sb) : 0.f;
}

// One element of the SB update, after the coupling z (= J x_hat) is known.
// coef_x = -(a0 - a(t)); the adiabatic variant adds -x^2 and has no walls.
// fe: the deformation field's force (0 without deformation).
__device__ __forceinline__ void sb_update(int sb, float z, float& x, float& y, float dt,
                                          float coef_x, float dta0, float c0, float fe = 0.f) {
  const float cx = sb == QH_SB_ADIABATIC ? coef_x - x * x : coef_x;
  y = y + dt * (cx * x + c0 * z + fe);
  x = x + dta0 * y;
  if (sb != QH_SB_ADIABATIC && fabsf(x) > 1.f) {
    x = x > 0.f ? 1.f : -1.f;
    y = 0.f;
  }
}
// The product's operand for the next step: x, or sgn(x) (sgn(0) = +1) for discrete SB.
__device__ __forceinline__ float sb_operand(int sb, float x) {
  return sb == QH_SB_DISCRETE ? (x >= 0.f ? 1.f : -1.f) : x;
}

// Tensor-core precisions use the BF16 hi tiles; the lo (remainder) tiles join when
// asked for (QH_PREC_BF16X2) or when integer weights above 256 need them to stay exact.
inline bool is_tc_precision(int p) { return p == QH_PREC_BF16 || p == QH_PREC_BF16X2; }
// Power-of-two scale of J for e4m3 tiles: 1 for integer weights below 256 (exact as
// hi + lo), else the largest 2^k with max|J| * 2^k <= 240.
inline float fp8_scale(const Graph& g) {
  if (g.integer_weights && g.max_abs_w < 256.0) return 1.f;
  if (!(g.max_abs_w > 0.0)) return 1.f;
  float s = 1.f;
  while (g.max_abs_w * s * 2.0 <= 240.0) s *= 2.f;
  while (g.max_abs_w * s > 240.0) s *= 0.5f;
  return s;
}
inline int32_t use_lo_for(const Graph& g, int precision) {
  return g.has_lo && (precision == QH_PREC_BF16X2 || g.integer_weights) ? 1 : 0;
}

qh_status set_err(Ctx* ctx, qh_status st, const std::string& msg);
qh_status cuda_fail(Ctx* ctx, cudaError_t e, const char* what);
void* dalloc(Graph& g, size_t bytes);
qh_status retile(Ctx* ctx, Graph* g, const double* w, __nv_bfloat16* tb, float* tf, float* pval);
qh_status build_graph_device(Ctx* ctx, const qh_fragments* f, const qh_graph_opts* o, Graph* g);

// ---- launchers (bsb_simt.cu)
void launch_init_state(cudaStream_t s, const Graph& g, int32_t R, int32_t replica_base,
                       uint64_t seed, int32_t iter, float* x, float* y, __nv_bfloat16* xh,
                       const int32_t* active, int32_t sb = QH_SB_BALLISTIC);
// X_hat of a state for the given SB variant: bf16(x), or sgn(x) at real vertices.
void launch_x_operand(cudaStream_t s, const Graph& g, int32_t sb, const float* x,
                      __nv_bfloat16* xh, int64_t n);
void launch_step_f32(cudaStream_t s, const Graph& g, const StepArgs& a);
// CSR storage: warp per padded vertex, state [n_pad][R]; xh_in != nullptr selects the
// BF16 X_hat operand, otherwise a.xin (FP32).  variant: CSR_LANE4 (4 replicas per lane,
// any R that is a multiple of 4) or CSR_LANE8 (8 per lane, several neighbours per warp
// at once; R a multiple of 8).
// CSR_BAND8: the band on the tensor cores (launch_band_mma, BF16 operands, R a multiple
// of 128), then the lane-8 CSR step over the remainder, starting from the band product.
constexpr int CSR_LANE4 = 10;
constexpr int CSR_LANE8 = 11;
constexpr int CSR_BAND8 = 12;
inline bool csr_variant_ok(int v, int R, int precision) {
  return v == CSR_LANE4   ? R % 4 == 0
         : v == CSR_LANE8 ? R % 8 == 0
         : v == CSR_BAND8 ? R % 128 == 0 && precision != QH_PREC_FP32
                          : false;
}
// Default: the band on the tensor cores when it holds at least a quarter of the
// entries (BF16 operands, R a multiple of 128); else 8 replicas per lane for BF16
// operands (fewer instructions per gathered neighbour), 4 per lane for FP32 operands
// (fewer registers, more warps in flight).
inline int csr_default_variant(const Graph& g, int precision, int R) {
  if (precision != QH_PREC_FP32 && R % 128 == 0 && g.band != nullptr &&
      4 * (g.pnnz - g.rnnz) >= g.pnnz && g.pnnz > 0)
    return CSR_BAND8;
  return (precision != QH_PREC_FP32 && R % 8 == 0) ? CSR_LANE8 : CSR_LANE4;
}
const char* csr_variant_name(int v, bool bf16);
// remainder = true: walk the remainder CSR (rrow_ptr / rcol with values pval), adding
// to a.zb; otherwise the full padded CSR (prow_ptr / pcol).
void launch_step_csr(cudaStream_t s, const Graph& g, const StepArgs& a, const float* pval,
                     const __nv_bfloat16* xh_in, int variant, bool remainder = false);
cudaError_t band_set_attrs();
// Failure-detection probe (bsb_run.cu): a bounded device wait that expires.
qh_status launch_wait_probe(Ctx* ctx, int which);
// Z = J_band X_hat for the live blocks (X_hat vertex-major, [n_pad][R]); the band tiles
// `band` as built by the graph (or a working copy).
qh_status launch_band_mma(Ctx* ctx, const Graph& g, const StepArgs& a, const __nv_bfloat16* band,
                          const __nv_bfloat16* xh_vm, float* z);
void launch_transpose(cudaStream_t s, const float* in, float* out, int64_t rows, int64_t cols);
void launch_signs(cudaStream_t s, const Graph& g, int32_t R, const float* x, int8_t* signs_t);
void launch_cut(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t, const double* w,
                const double* sum_w, double* node_val, double* cuts, const int32_t* active);
void launch_pick_best(cudaStream_t s, int32_t n_blocks, int32_t R, const double* cuts,
                      int32_t* best_r, double* best_cut, const int32_t* active);
// row[b] = best_cut[b] where running[b] and t_done < steps_b[b], else NaN (one check of
// Per-replica cuts from z = J S (S = the replicas' signs in BF16, both [R][n_pad]):
// cut = (sum_w + sum_a s_a z_a) / 4, exact for integer weights (row sums of |J| < 2^24).
// acc: n_blocks * R doubles of scratch.
void launch_cut_from_product(cudaStream_t s, const Graph& g, int32_t R, const float* z,
                             const __nv_bfloat16* signs, const double* sum_w, double* acc,
                             double* cuts, const int32_t* active);
// the energy trace)
void launch_trace_check(cudaStream_t s, int32_t n_blocks, const double* best_cut,
                        const int32_t* running, int32_t t_done, const int32_t* steps_b,
                        double* row);
void launch_early_stop(cudaStream_t s, int32_t n_blocks, const double* best_cut, double* best_seen,
                       int32_t* stall, int32_t* active, int32_t* steps_run, int32_t patience,
                       int32_t t_done, const int32_t* steps_b);
// Best during the run (track_best): after a check (signs, cut and pick of that state)
// keep each running block's better result; at the end let the kept result replace the
// final one unless the final is strictly better.
void launch_track_check(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t,
                        const double* best_cut, const int32_t* best_r, const int32_t* active,
                        int32_t t_done, const int32_t* steps_b, double* kept_cut, int32_t* kept_r,
                        int32_t* flag, int8_t* kept_spins);
void launch_track_final(cudaStream_t s, const Graph& g, double* best_cut, int32_t* best_r,
                        const int32_t* active, const double* kept_cut, const int32_t* kept_r,
                        int32_t* flag, const int8_t* kept_spins, int8_t* spins);
void launch_extract_spins(cudaStream_t s, const Graph& g, int32_t R, const int8_t* signs_t,
                          const int32_t* best_r, int8_t* spins, const int32_t* active);
void launch_block_sums(cudaStream_t s, const Graph& g, const double* w, double* sum_w,
                       double* sum_j2, double* node_tmp /* 2 * n_nodes */);
// Refill the band tiles and the remainder CSR values of a CSR-mode graph from weights
// w (after a refinement sign inversion; the pattern is unchanged).
qh_status reband(Ctx* ctx, const Graph* g, const double* w, __nv_bfloat16* band, float* rval);
void launch_refine_prepare(cudaStream_t s, const Graph& g, const int8_t* spins,
                           const double* best_cut, int32_t* active, int32_t* C, float* deform,
                           int32_t* tries, float deform_h, int32_t deform_tries);
// w <- D_s w D_s on the active, undeformed blocks; gauge (or nullptr) *= s there
void launch_gauge(cudaStream_t s, const Graph& g, const int8_t* spins, double* w,
                  const int32_t* active, const float* deform, int8_t* gauge);
// w = D_g w0 D_g (g = +-1 per vertex)
void launch_apply_gauge(cudaStream_t s, const Graph& g, const double* w0, const int8_t* gauge,
                        double* w);
void launch_vote(cudaStream_t s, const Graph& g, const int8_t* spins, int8_t* hap1, int8_t* hap2,
                 int32_t* block_id);
void launch_parity(cudaStream_t s, const Graph& g, const int32_t* C, int8_t* hap1, int8_t* hap2,
                   int32_t* block_id);
void launch_f32_to_bf16(cudaStream_t s, const float* x, __nv_bfloat16* xh, int64_t n);

// ---- launchers (bsb_tc.cu)
struct TcPlan {
  int bn = 128;     // replicas per CTA (MMA N)
  int stages = 3;   // TMA/MMA pipeline depth
  int variant = -1;  // solver-step kernel variant (autotuned); -1 = the plain kernel
};
qh_status launch_step_tc(Ctx* ctx, const Graph& g, const StepArgs& a,
                         const __nv_bfloat16* xh_in, const TcPlan& plan);
bool tc_plan_ok(int R, const TcPlan& plan);
struct Fp8Operands {
  const uint8_t* jh;      // e4m3 hi / lo tiles of s*J, indexed like the FP32 tiles
  const uint8_t* jl;
  const uint8_t* xh_in;   // e4m3 hi / lo parts of X_t, [R][n_pad]
  const uint8_t* xl_in;
  int32_t n_slices;       // 2, or 3 when s*J has a nonzero remainder
};
qh_status launch_step_f8(Ctx* ctx, const Graph& g, const StepArgs& a, const Fp8Operands& op);
void launch_tiles_to_e4m3(cudaStream_t s, const float* tf, int64_t n, float scale, uint8_t* th,
                          uint8_t* tl, int32_t* has_lo);
void launch_x_to_e4m3(cudaStream_t s, const float* x, int64_t n, uint8_t* h, uint8_t* l);
// The FP8 product operand of a state [R][n_pad] for SB variant sb (sgn(x) for discrete
// SB, x otherwise) at real vertices, 0 at padding, as e4m3 hi / lo.
void launch_x_operand_e4m3(cudaStream_t s, const Graph& g, int32_t sb, const float* x, int64_t n,
                           uint8_t* h, uint8_t* l);
int tc_n_variants();
const char* tc_variant_name(int v);
bool tc_variant_ok(int v, const Graph& g, int R, int n_sm, bool use_lo);
qh_status tc_prepare(Ctx* ctx);

// Multi-step tensor-core kernel (bsb_run.cu): one launch runs a range of steps with
// the momentum y held in TMEM.  Four of the autotuner's variants select it:
//   6: J resident in smem, group hand-off   7: J streamed, tile hand-off
//   8: J resident in smem, tile hand-off    9: J streamed, group hand-off
constexpr int RUN_VARIANT_FIRST = 6;
constexpr int S_RUN_WORK = 96, S_RUN_ROWS = 97, S_RUN_DONE = 98, S_RUN_XQ = 99;  // scratch slots
constexpr int S_WAIT_PROBE = 100, S_RUN_ITEMS = 101, S_RUN_S = 102, S_RUN_E = 103, S_RUN_EC = 104;
struct RunWave {              // one launch: whole blocks whose items fit on chip
  int work_off = 0;           // first entry of the wave in RunBufs::work
  int item_off = 0;           // first entry of the wave in RunBufs::items
  int grid = 0;               // CTAs
  int stride = 1;             // a CTA's items: first, first + stride, ...
  int max_items = 0;          // most items of one CTA
};
struct RunPlan {
  std::vector<int2> work;     // per CTA of every wave: {first position, item count}
  std::vector<int32_t> items; // per wave: its items, row-tile-major
  std::vector<RunWave> waves;
};
struct RunBufs {
  int2* work = nullptr;       // device copy of RunPlan::work
  int32_t* items = nullptr;   // device copy of RunPlan::items
  int32_t* rows_b = nullptr;  // [n_blocks] row tiles per block
  uint32_t* done = nullptr;   // release counters (per item or per block x replica tile)
  float4* xq = nullptr;       // [R/4][n_pad] blocked working copy of x
  std::vector<RunWave> waves;
  int64_t n_done = 0;
  bool jres = false;
  bool group_sync = false;
  bool jsplit = false;  // stream mode: J K-slices in a ring of their own (rows of > 6 slices)
};
bool run_variant(int v);
// mask (n_blocks flags, or nullptr = every block): blocks left out take no items
// max_items: items per CTA at most (run_max_items(), or 3 for checks inside the launch)
bool run_plan(const Graph& g, int R, int n_sm, int variant, bool use_lo, RunPlan* plan,
              const std::vector<int32_t>* mask = nullptr, int max_items = 4);
// items per CTA (3 or 4) that minimise the waves' step periods (see bsb_run.cu)
int run_items(const Graph& g, int R, int n_sm, int variant, bool use_lo,
              const std::vector<int32_t>* mask = nullptr);
qh_status run_prepare(Ctx* ctx, const Graph& g, int R, int variant, bool use_lo, RunBufs* rb,
                      const std::vector<int32_t>* mask = nullptr, int max_items = 4);
// Early-stop checks inside one multi-step launch over steps 0 .. t1 (integer weights;
// the plan must hold at most three items per CTA).  All device buffers, zeroed by the
// caller except seen (-inf) and stop_t (-1).
struct RunCheck {
  int32_t check_every = 0, patience = 0;
  __nv_bfloat16* s = nullptr;        // two [R][n_pad] buffers of S = sgn(x), zero at start
  const double* sum_w = nullptr;     // [n_blocks]
  unsigned long long* e_sum = nullptr;  // [2][n_blocks][R]
  uint32_t* e_cnt = nullptr;         // [2][n_blocks]
  uint32_t* decided = nullptr;       // [n_blocks]
  double* seen = nullptr;            // [n_blocks]
  int32_t* stall = nullptr;          // [n_blocks]
  int32_t* stop_t = nullptr;         // [n_blocks]
  double* trace = nullptr;           // [checks][n_blocks] best cut per check, or nullptr
};
// Steps t0 .. t1-1 in one launch.  X_hat_t is read from xh0 (t even) or xh1 (t odd);
// x, y of `s` are updated in place.
// trace (test hook, else nullptr): step-timeline stamps of steps trace_u0 ..
// trace_u0 + trace_nu - 1 (relative to t0), run_trace_events() global-timer and as many
// SM-clock stamps per (CTA, step, item slot of run_max_items()).
qh_status launch_run(Ctx* ctx, const Graph& g, const StepArgs& s, const RunBufs& rb,
                     __nv_bfloat16* xh0, __nv_bfloat16* xh1, int t0, int t1,
                     unsigned long long* trace = nullptr, int trace_u0 = 0, int trace_nu = 0,
                     const RunCheck* check = nullptr);
// After a launch with checks: a block that stopped at check step t takes the signs it had
// there (S of that check's parity) as its x, and t as its steps_run.
void launch_stop_fixup(cudaStream_t s, const Graph& g, int32_t R, const RunCheck& c,
                       float* x, int32_t* steps_run);
int run_trace_events();
int run_max_items();
int run_item_mask();  // the item-id bits of a wave's item list entries
cudaError_t run_set_attrs();

}  // namespace qh

// Opaque handles of the C ABI.
struct qh_ctx {
  qh::Ctx c;
};
struct qh_graph {
  qh::Graph g;
  qh_ctx* owner;
};
struct qh_solution {
  qh::Solution s;
};

// NVTX range over a scope (host timeline for nsys / ncu range filters; a no-op
// unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Launch-error check at a stage boundary (kernel launches are not checked one by one).
#define QH_STAGE_CHECK(name)                                      \
  do {                                                            \
    cudaError_t _e = cudaGetLastError();                          \
    if (_e != cudaSuccess) return qh::cuda_fail(ctx, _e, name);   \
  } while (0)

#define QH_CUDA_TRY(expr)                                        \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return qh::cuda_fail(ctx, _e, #expr); \
  } while (0)
