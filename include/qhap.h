/*
 * qhap.h -- C ABI of the GB300 (sm_103a) QHap phasing hot path.
 *
 * QHap ("Quantum-Inspired Haplotype Phasing") phases diploid haplotypes by
 * turning read evidence into a weighted graph and solving Max-Cut on it with
 * ballistic simulated bifurcation (bSB).  This library runs that path on one
 * GPU with hand-written CUDA kernels:
 *
 *   qh_build_graph : fragments -> read graph or SNP graph (the coupling J = -A)
 *                    -> connected components (phase blocks) -> J tiles
 *   qh_bsb_solve   : multi-replica bSB on every block at once -> spins, cut
 *                    (SNP graphs: iterative refinement with sign inversion)
 *   qh_phase       : spins -> haplotypes (read voting or flip-count parity)
 *
 * Conventions for every call
 *  - Status: every call returns qh_status; none aborts the process.  On error
 *    qh_last_error(ctx) holds a one-line description.
 *  - Streams: work is issued on the context's CUDA stream.  Calls that return
 *    host data synchronise that stream before returning.
 *  - Ownership: input arrays stay owned by the caller and are copied (host or
 *    device) before the call returns.  Opaque handles (qh_ctx, qh_graph,
 *    qh_solution) are owned by the library and released by their *_free /
 *    qh_destroy call.  Output arrays are caller-allocated with the lengths
 *    stated per argument.
 *  - Pointers marked "host or device" are read from device memory when the
 *    call's `on_device` flag is 1, from host memory otherwise.
 *  - Thread safety: one context must not be used by two host threads at once.
 */
#ifndef QHAP_H
#define QHAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QH_OK = 0,
  QH_EINVAL = 1,       /* invalid argument or malformed input */
  QH_ENOMEM = 2,       /* device or host allocation failed */
  QH_ECUDA = 3,        /* a CUDA runtime/driver call failed */
  QH_ETIMEOUT = 4,     /* a bounded device-side wait expired; context stays usable */
  QH_EUNSUPPORTED = 5  /* valid request outside this build's limits */
} qh_status;

typedef struct qh_ctx qh_ctx;
typedef struct qh_graph qh_graph;
typedef struct qh_solution qh_solution;

/* Graph modes (read-based / SNP-based method, Methods). */
enum { QH_MODE_READ = 0, QH_MODE_SNP = 1 };
/* Read-graph weights: CONFLICT = count of shared SNPs with opposing alleles
 * (Eqs. delta and w_ab); SIGNED = conflicts - agreements, W = -M M^T. */
enum { QH_WEIGHT_CONFLICT = 0, QH_WEIGHT_SIGNED = 1 };
/* J x X product precision in the bSB step.  State x, y is FP32 in all modes.
 * FP32: SIMT FP32 product.
 * BF16: tcgen05 BF16 x BF16 -> FP32 accumulate, X_hat = bf16(x).  J is rounded to
 *   BF16 (exact for integer |w| <= 256; larger integers are split J = hi + lo,
 *   both BF16, in the same accumulator, so integer J stays exact).
 * BF16X2: as BF16, with real weights also split into hi + lo (J to ~2^-17).
 * FP8: tcgen05 kind::f8f6f4 (e4m3) with FP32 accumulate: s*J = Jh + Jl and
 *   x = xh + xl in e4m3 (s a power of two: 1 for integer |w| < 256, else scaled to
 *   240), Z = (Jh Xh + Jh Xl + Jl Xh) / s (tile storage only). */
enum { QH_PREC_FP32 = 0, QH_PREC_BF16 = 1, QH_PREC_BF16X2 = 2, QH_PREC_FP8 = 3 };
/* Schedules: LINEAR = a(t) = a0 * t / steps with the given steps;
 * AUTO = steps chosen from the block size as in the paper's SNP-based runs
 * (500 iterations for < 5,000 nodes, 1,000 otherwise). */
enum { QH_SCHED_LINEAR = 0, QH_SCHED_AUTO = 1 };
/* Simulated-bifurcation variants (the three the paper compares, in their standard
 * formulations; a(t) as above, symplectic Euler: y from x_t, then x from y_{t+1}):
 * BALLISTIC: y += dt(-(a0 - a(t)) x + c0 J x), x += dt a0 y, |x| > 1 => x = sgn x, y = 0
 * DISCRETE:  as BALLISTIC with J sgn(x) (sgn(0) = +1) in place of J x
 * ADIABATIC: y += dt(-(x^2 + a0 - a(t)) x + c0 J x), x += dt a0 y, no walls
 * All three run on every precision, storage and step kernel. */
enum { QH_SB_BALLISTIC = 0, QH_SB_DISCRETE = 1, QH_SB_ADIABATIC = 2 };

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on, or NULL to let the context create (and own) one.
 * Errors: QH_EINVAL (out is NULL, bad device), QH_ECUDA. */
qh_status qh_create(qh_ctx** out, int device, void* cuda_stream);
/* Release the context (waits for its stream).  NULL is a no-op. */
void qh_destroy(qh_ctx* ctx);
/* Static English name of a status code. */
const char* qh_status_str(int status);
/* Description of the last error on this context ("" if none).  Valid until
 * the next call on the context. */
const char* qh_last_error(const qh_ctx* ctx);

/* ---------------------------------------------------------------- inputs */

/* Fragments: per read, the heterozygous sites it covers, the allele seen at each
 * and its base quality (Methods, input preprocessing), stored as CSR.
 *  n_frags, n_snps : m fragments over n heterozygous SNPs
 *  frag_ptr  int64[m+1]  fragment i owns entries frag_ptr[i] .. frag_ptr[i+1]-1;
 *                        frag_ptr[0] = 0, non-decreasing
 *  snp       int32[nnz]  SNP index in [0, n), strictly increasing in a fragment
 *  allele    int8[nnz]   +1 = allele of the initial H1, -1 = of the initial H2
 *                        (ternary matrix M, read-based matrix construction)
 *  qual      uint8[nnz]  Phred base quality Q in [4, 93]; required in SNP mode,
 *                        may be NULL in read mode
 *  is_porec  uint8[m]    1 = Pore-C fragment; NULL = none
 * Fragment order matters only for speed: reads sorted by first SNP give banded
 * J tiles. */
typedef struct {
  int32_t n_frags;
  int32_t n_snps;
  const int64_t* frag_ptr;
  const int32_t* snp;
  const int8_t* allele;
  const uint8_t* qual;
  const uint8_t* is_porec;
  int32_t on_device; /* 1: the five arrays are device pointers */
} qh_fragments;

typedef struct {
  int32_t mode;        /* QH_MODE_READ | QH_MODE_SNP */
  int32_t weight_mode; /* READ mode: QH_WEIGHT_CONFLICT | QH_WEIGHT_SIGNED */
  int32_t linkage_k;   /* SNP mode: linkage depth k/10, 1..10 (10 = all pairs) */
  int32_t dense;       /* 1: store every J tile of each block (no zero-tile skipping) */
  int32_t storage;     /* J for the solver: QH_STORAGE_AUTO | _TILES | _CSR */
  double porec_alpha;  /* SNP mode: Pore-C contribution factor (paper default 0.1) */
} qh_graph_opts;

/* J storage for the solver.  TILES: nonzero 128 x 128 tiles, tensor-core steps,
 * state [R][n_pad].  CSR: one row per padded vertex, warp-per-vertex gather steps,
 * state [n_pad][R] (graphs whose edges scatter over most tiles, e.g. long-range
 * Pore-C contacts).  AUTO picks CSR when the nonzero tiles would hold more than
 * 64 stored entries per edge and exceed 4,096 tiles, TILES otherwise. */
enum { QH_STORAGE_AUTO = 0, QH_STORAGE_TILES = 1, QH_STORAGE_CSR = 2 };

/* Build the phasing graph and its phase blocks.
 * READ mode: vertices = fragments; w_ab per weight_mode (read-based Max-Cut
 * graph construction).  SNP mode: vertices = SNPs; w_uv = -sum_i alpha_i *
 * sgn(W_iu W_iv) log10(P_cis / P_trans) / (|S_i| - 1) accumulated in FP64 in
 * fragment order, with q~ = 1 - 10^(-Q/10) (SNP-based matrix and graph
 * construction; Pore-C data support).  Edges are the pairs with w != 0;
 * connected components with >= 2 vertices become phase blocks, numbered by
 * their smallest vertex; single-vertex components are dropped.
 * Errors: QH_EINVAL (malformed fragments, Q outside [4, 93] in SNP mode,
 * bad options), QH_ENOMEM, QH_ECUDA, QH_EUNSUPPORTED (an SNP row whose covering
 * fragments span more than 12,288 SNPs and gather more than 8,192 terms). */
qh_status qh_build_graph(qh_ctx* ctx, const qh_fragments* frags, const qh_graph_opts* opts,
                         qh_graph** out);

/* Graph summary.  Any output pointer may be NULL.
 *  n_nodes     : vertices (fragments or SNPs)
 *  n_blocks    : phase blocks
 *  block_sizes : int32[cap] filled with min(cap, n_blocks) block sizes
 *  nnz         : stored directed edges (2 per undirected edge)
 *  n_tiles     : stored 128 x 128 J tiles */
qh_status qh_graph_info(const qh_graph* g, int32_t* n_nodes, int32_t* n_blocks,
                        int32_t* block_sizes, int32_t cap, int64_t* nnz, int64_t* n_tiles);

/* Copy the edge list of the graph to host arrays (test and inspection hook).
 * row_ptr int64[n_nodes+1], col int32[nnz], w float64[nnz] (exact integers in
 * READ mode).  Rows list each vertex's neighbours. */
qh_status qh_graph_edges(qh_ctx* ctx, const qh_graph* g, int64_t* row_ptr, int32_t* col,
                         double* w);

/* Block membership: block_of int32[n_nodes] (-1 for dropped singletons) and
 * local int32[n_nodes] (index of the vertex inside its block, ascending vertex
 * order).  Either may be NULL. */
qh_status qh_graph_blocks(qh_ctx* ctx, const qh_graph* g, int32_t* block_of, int32_t* local);

void qh_graph_free(qh_graph* g);

/* ---------------------------------------------------------------- solver */

/* bSB options (SB algorithm solution).  Each step, for every replica:
 *   y <- y + dt * ( -(a0 - a(t)) x + c0 * J x ),   x <- x + dt * a0 * y,
 *   |x| > 1  =>  x <- sgn(x), y <- 0,              a(t) = a0 * t / steps,
 * with x, y drawn uniform on [-0.1, 0.1] from SplitMix64 keyed by
 * (seed, block, refinement iteration, replica index, local vertex, x|y).
 * Spins are s = sgn(x) with sgn(0) = +1. */
typedef struct {
  int32_t replicas;     /* R >= 1 (multiple of 16 for QH_PREC_BF16) */
  int32_t steps;        /* >= 1 (LINEAR schedule) */
  int32_t schedule;     /* QH_SCHED_LINEAR | QH_SCHED_AUTO */
  int32_t precision;    /* QH_PREC_FP32 | QH_PREC_BF16 | QH_PREC_BF16X2 | QH_PREC_FP8 */
  double dt;            /* time step (1.0) */
  double a0;            /* bifurcation parameter target (1.0) */
  double c0;            /* coupling scale; <= 0 selects 0.5 / (sigma sqrt(N)) per
                           block, sigma^2 = sum_{a != b} J_ab^2 / (N (N - 1)) */
  uint64_t seed;        /* RNG seed */
  int32_t replica_base; /* first replica index (replicas are base .. base+R-1) */
  int32_t check_every;  /* energy check period in steps for early stop (0 = off) */
  int32_t patience;     /* stop a block after this many checks without a better
                           best-replica energy (0 = never stop early) */
  int32_t refine_max;   /* SNP mode: maximum refinement iterations (>= 1) */
  int32_t step_kernel;  /* -1 = default.  Tile storage, BF16: autotuned by default,
                           else a variant index 0..9 (see qh_solution_kernel for
                           names; 6..9 are the multi-step kernels that keep y on
                           chip and launch once per step range).  CSR storage
                           (FP32 or BF16): 10 = 4 replicas per lane (R a multiple
                           of 4), 11 = 8 replicas per lane, several neighbours per
                           warp at once (R a multiple of 8); BF16 only: 12 = the
                           band (entries within a row tile's neighbourhood) on the
                           tensor cores, then 11 over the remaining entries (R a
                           multiple of 128).  Default for CSR: 12 when R allows and
                           the band holds at least a quarter of the entries, else
                           11 for BF16 when R allows, else 10.  Invalid choices ->
                           QH_EINVAL */
  int32_t sb_variant;   /* QH_SB_BALLISTIC (0, the paper's solver), QH_SB_DISCRETE,
                           QH_SB_ADIABATIC; every precision, storage and step
                           kernel.  Discrete SB multiplies J by sgn(x), which FP8
                           and BF16 hold exactly.  Other values -> QH_EINVAL */
  double deform_h;      /* SNP mode: the adaptive deformation of the refinement
                           (0 = off, the plain refinement).  When a solve of a block
                           ends with a cut <= 0 or with all vertices in one subset,
                           the block is solved again, up to deform_tries times, with
                           the force dt h_k (1 - t / steps) added to y along the
                           incumbent partition (h_k = deform_h 2^(k-1) on the k-th
                           re-solve); a positive cut is accepted as usual.  Every
                           solve counts toward refine_max.  The paper names a
                           deformation h for components whose cut keeps coming
                           out negative but gives no formula: this is the
                           library's reading of it.  Must be finite and >= 0. */
  int32_t deform_tries; /* re-solves with deformation after a failed solve (>= 0) */
  int32_t check_mode;   /* where the early-stop checks run (with check_every and
                           patience > 0): 0 = inside the multi-step launch when it
                           applies (a multi-step step kernel, integer weights, at
                           most three items per SM fit every block) and pays
                           (check_every <= 128), else between launches; 1 = always
                           between launches, with the separate cut kernels.  Both
                           give the same steps_run, cuts and spins.  Other values
                           -> QH_EINVAL */
  int32_t track_best;   /* 1 = report the best value reached during the run (Results):
                           with check_every > 0, the best cut over the replicas at
                           any check or at the end, with its replica and spins (ties:
                           the earliest check, the end last; the lowest replica).
                           qh_solution_cuts still gives the final state's cuts.  The
                           checks then run between launches, and also without early
                           stop (patience 0).  0 = the final state (default) */
} qh_bsb_opts;

/* Run multi-replica bSB on every block of the graph in one batched launch per
 * step (the step loop is replayed from a CUDA graph), or, with the multi-step
 * kernels, in one launch per range of steps (per early-stop check period).  Each replica's final
 * spins are cut-evaluated exactly (FP64 reduction; exact for integer weights);
 * the best replica per block wins, ties to the lowest replica index.
 * SNP mode additionally runs the iterative refinement (flip counter C on the
 * smaller subset, sign inversion of edges crossing the partition) until the
 * cut is <= 0, the partition has a single subset, or refine_max iterations.
 * Errors: QH_EINVAL, QH_ENOMEM, QH_ECUDA, QH_ETIMEOUT. */
qh_status qh_bsb_solve(qh_ctx* ctx, const qh_graph* g, const qh_bsb_opts* opts,
                       qh_solution** out);

/* qh_bsb_solve on the listed blocks only (block indices as numbered by the graph,
 * each at most once): the unit of block sharding, where the blocks of one graph are
 * split across processes or GPUs (connected components are independent subproblems,
 * SB algorithm solution).  The listed blocks get exactly the result qh_bsb_solve gives
 * them (same draws, keyed by block and replica); the others stay unsolved: best cut 0,
 * best replica -1, steps_run 0, iterations 0, spins 0, zero rows in qh_solution_cuts,
 * and qh_phase leaves their SNPs unphased.  n_blocks = 0 solves nothing.
 * Errors: as qh_bsb_solve, and QH_EINVAL for an index out of range or listed twice. */
qh_status qh_bsb_solve_blocks(qh_ctx* ctx, const qh_graph* g, const qh_bsb_opts* opts,
                              const int32_t* blocks, int32_t n_blocks, qh_solution** out);

/* Checkpoint of the SNP refinement (SB algorithm solution, the refinement loop: flip
 * counts C on the smaller subset, sign inversion of the edges crossing each solve's
 * partition).  The state after a solve is what the next solve of the loop starts from;
 * host arrays, caller-owned:
 *  iterations_done : solves of the loop run over the graph so far (>= 1); the next
 *                    solve's random draws are keyed by this iteration index
 *  flips    int32[n_nodes] : C, the times each vertex was in the smaller subset
 *                            (-1 for a vertex in no block or in an unsolved block)
 *  gauge    int8[n_nodes]  : +1 / -1, the product of the partitions whose sign
 *                            inversions the next solve's weights carry: its graph is
 *                            w'_ab = g_a w_ab g_b (+1 outside the blocks)
 *  refining int32[n_blocks]: 1 while the block's refinement goes on
 *  solves   int32[n_blocks]: solves the block has run
 *  deform   float[n_blocks]: the field strength of the block's next (deformed) solve,
 *                            0 for none (qh_bsb_opts.deform_h)
 *  tries    int32[n_blocks]: deformed re-solves the block has used */
typedef struct {
  int32_t iterations_done;
  int32_t* flips;
  int8_t* gauge;
  int32_t* refining;
  int32_t* solves;
  float* deform;
  int32_t* tries;
} qh_refine_state;

/* Save: write a SNP-mode solution's refinement state into the caller's arrays (every
 * pointer non-NULL, lengths as above).  A solve with refine_max = k followed by
 * qh_bsb_solve_resume with refine_max = K > k from this state gives the same flip
 * counts, parity partition, final cuts and haplotypes as one solve with refine_max = K.
 * Errors: QH_EINVAL (READ-mode solution, NULL pointer, a solution imported block by
 * block). */
qh_status qh_solution_refine_state(const qh_solution* sol, qh_refine_state* state);

/* Resume: continue the SNP refinement of `g` from a saved state, for the solves
 * iterations_done .. opts->refine_max - 1 (refine_max counts every solve of the loop,
 * those before the checkpoint included), with the same options as the solve that made
 * the state (replicas, steps, seed, precision, deform_h, ...).  The blocks that are no
 * longer refining keep their flip counts.  The result is a solution as qh_bsb_solve
 * returns it, except that qh_solution_cuts, the best replica and steps_run describe the
 * first solve of this call.  Errors: as qh_bsb_solve; QH_EINVAL for a READ-mode graph,
 * a NULL array, iterations_done < 1 or >= refine_max, a gauge value other than +-1, a
 * negative count, or a deformation field in the state without opts->deform_h > 0. */
qh_status qh_bsb_solve_resume(qh_ctx* ctx, const qh_graph* g, const qh_bsb_opts* opts,
                              const qh_refine_state* state, qh_solution** out);

/* Import one block's result into a solution, e.g. a block solved by another process
 * of a sharded run (host values as qh_solution_block returns them there).
 *  spins        : int8[block size], +1 / -1 in local vertex order (SNP mode: the
 *                 parity partition, +1 where the flip count is even)
 *  best_cut, best_replica (>= 0, a global replica index), steps_run (>= 0),
 *  iterations (>= 1) : reported back by qh_solution_block
 * The block's row of qh_solution_cuts becomes zeros.  qh_phase uses the imported
 * spins (read voting, or the SNP parity).  Errors: QH_EINVAL. */
qh_status qh_solution_set_block(qh_ctx* ctx, qh_solution* sol, int32_t block, const int8_t* spins,
                                double best_cut, int32_t best_replica, int32_t steps_run,
                                int32_t iterations);

/* Per-block result.  Any output pointer may be NULL.
 *  spins        : int8[block size], best replica's spins in local vertex order
 *  best_cut     : cut of those spins on the block's original (ungauged) graph
 *  best_replica : replica index (replica_base + r) of the winner; -1 for a block
 *                 that a partial solve (qh_bsb_solve_blocks) left unsolved
 *  steps_run    : bSB steps actually run (early stop may shorten it)
 *  iterations   : refinement iterations (1 in READ mode)
 * Errors: QH_EINVAL (block out of range). */
qh_status qh_solution_block(qh_ctx* ctx, const qh_solution* sol, int32_t block, int8_t* spins,
                            double* best_cut, int32_t* best_replica, int32_t* steps_run,
                            int32_t* iterations);

/* Spins of the solution by vertex: int8[n_nodes], +1 / -1 for vertices in a
 * block (READ mode: best replica; SNP mode: the flip-count parity partition,
 * +1 where C is even), 0 for dropped singletons. */
qh_status qh_solution_spins(qh_ctx* ctx, const qh_solution* sol, int8_t* spins);

/* All replicas' final cuts of the first refinement iteration:
 * cuts float64[n_blocks * R], row b = block b (values on the block's graph). */
qh_status qh_solution_cuts(qh_ctx* ctx, const qh_solution* sol, double* cuts);

/* Energy-check trace of the first solve (Results: the energy against the iterations;
 * the checks of qh_bsb_opts.check_every, with early stop or track_best on): the best
 * cut over the replicas of each block at steps check_every, 2 check_every, ... below
 * the longest block schedule.
 *  n_checks     : the number of checks (0 when no checks ran)
 *  check_every  : their period in steps (may be NULL)
 *  trace float64[n_checks * n_blocks] (may be NULL): row c = check c + 1; NaN for a
 *                 block that was not running at that check (it had stopped early, its
 *                 schedule had ended, or it was not solved)
 * Errors: QH_EINVAL (NULL solution or n_checks). */
qh_status qh_solution_check_trace(const qh_solution* sol, int32_t* n_checks, int32_t* check_every,
                                  double* trace);

/* Timing of the last solve in milliseconds (CUDA events on the context stream):
 *  solve_ms : whole qh_bsb_solve device time
 *  step_ms  : the bSB step launches only; n_step_launches launches
 *  spin_updates : sum over blocks of N_b * R * steps_run_b (all iterations) */
qh_status qh_solution_timing(const qh_solution* sol, double* solve_ms, double* step_ms,
                             int64_t* n_step_launches, double* spin_updates);

/* Name of the bSB step kernel the solve ran ("k_step_f32" for FP32; for BF16 the
 * tensor-core variant the autotuner chose for this graph shape). */
const char* qh_solution_kernel(const qh_solution* sol);

/* Step-kernel autotuning of the context's latest new graph shape, as
 * "variant=microseconds;..." ("" until a BF16 solve has tuned).  Tuning runs once
 * per (replicas, tile layout) shape and context: each valid variant runs a few
 * steps on the solve's own state, which is then re-initialised. */
const char* qh_tuning_report(const qh_ctx* ctx);

/* Number of CUDA kernels this library has launched in the process so far (every
 * context; each replay of a captured step loop counts all of its kernels). */
int64_t qh_kernel_launches(void);

void qh_solution_free(qh_solution* sol);

/* ---------------------------------------------------------------- phase */

/* Haplotypes from the solution (consistency processing / SNP parity swap).
 * READ mode: each SNP is voted on by the block holding the most reads that
 * cover it (ties: lower block); with d_l = c_l^(+) - c_l^(-) for S_1 = {s=+1}
 * and S_2 = {s=-1}: opposing majorities give S_1 the sign of d_1; otherwise the
 * subset with the larger |d_l| (tie: S_1) keeps its majority and the other
 * takes the complement; zero coverage or d_1 = d_2 = 0 leaves it unphased.
 * SNP mode: H1' = H1 where C is even, swapped where C is odd.
 * Outputs (host or device per on_device), each of length n_snps:
 *  hap1 int8 : +1 = H1' carries the initial-H1 allele, -1 = the initial-H2
 *              allele, 0 = unphased;   hap2 = -hap1 (0 where unphased)
 *  block_id int32 : phase block of the SNP, -1 if unphased
 * Errors: QH_EINVAL. */
qh_status qh_phase(qh_ctx* ctx, const qh_graph* g, const qh_solution* sol, int8_t* hap1,
                   int8_t* hap2, int32_t* block_id, int32_t on_device);

/* ---------------------------------------------------------------- test hooks */

/* One J x X product with the solver's operands, for precision checks.
 * x  float32[R][n_pad] (device) : state, padded vertex layout (for CSR storage
 *    the hook transposes to the solver's [n_pad][R] layout and back)
 * z  float32[R][n_pad] (device) : output J_hat x X_hat (FP32 accumulate), where
 *    J_hat, X_hat are the precision's operands (BF16 rounds x to BF16).
 * n_pad is qh_debug_layout's value.  R multiple of 16 for BF16.
 * Errors: QH_EINVAL, QH_ECUDA, QH_ETIMEOUT. */
qh_status qh_debug_matvec(qh_ctx* ctx, const qh_graph* g, int32_t precision, int32_t R,
                          const float* x, float* z);

/* Run `nsteps` solver steps t0 .. t0+nsteps-1 of a `steps`-step schedule from a
 * given state, in place: x, y float32[R][n_pad] (device), same layout.
 * c0_per_block float64[n_blocks] (host) or NULL for the default c0.
 * Resume: the state (x, y, t) is all a step range needs.  The product operand is
 * rebuilt from x exactly as the kernels write it, so running t0 .. t0+n and then
 * t0+n .. t0+2n gives the same bits as one call over t0 .. t0+2n. */
qh_status qh_debug_steps(qh_ctx* ctx, const qh_graph* g, int32_t precision, int32_t R,
                         float* x, float* y, int32_t t0, int32_t nsteps, int32_t steps, double dt,
                         double a0, const double* c0_per_block);

/* qh_debug_steps with an explicit step kernel (BF16 / BF16X2 tile storage: 0..9;
 * CSR storage, FP32 or BF16: 10 or 11; CSR storage, BF16: 12) and SB variant (QH_SB_*):
 * step_kernel = -1 is the default; otherwise an index into the solver's kernel
 * variants (qh_bsb_opts.step_kernel).  The multi-step variants run all `nsteps`
 * steps in ONE launch, the momentum y held on chip between steps.  QH_EINVAL when
 * the variant does not fit the graph, precision or R.  field_per_block (host,
 * n_blocks values, or NULL): the refinement's deformation field strength h_b of each
 * block; every step then adds dt h_b (1 - t / steps) to y on every vertex. */
qh_status qh_debug_steps_v(qh_ctx* ctx, const qh_graph* g, int32_t precision, int32_t R,
                           float* x, float* y, int32_t t0, int32_t nsteps, int32_t steps,
                           double dt, double a0, const double* c0_per_block, int32_t step_kernel,
                           int32_t sb_variant, const double* field_per_block);

/* Test hook of the failure detection (not part of the paper's method): runs one of the
 * step kernels' bounded device waits on something that nothing completes (which = 0:
 * an mbarrier phase; 1: a release counter of the multi-step kernel).  The wait gives
 * up after about one second and the call returns QH_ETIMEOUT; the context stays
 * usable for the next call.  QH_EINVAL for another `which`. */
qh_status qh_debug_wait_timeout(qh_ctx* ctx, int32_t which);

/* Test hook of the error paths (not part of the paper's method): allocation-failure
 * injection on the host.  after >= 0: the context's next `after` device allocations
 * (graph and solution memory, grown scratch buffers) succeed and every later one
 * fails as if the device were out of memory, so the call that meets it returns
 * QH_ENOMEM (graphs and solutions it had begun are freed); after = -1 turns the
 * injection off.  Allocations that an earlier call left in place are reused and not
 * counted.  QH_EINVAL for after < -1.  No device work. */
qh_status qh_debug_fail_alloc(qh_ctx* ctx, int64_t after);

/* The solver's initial state (SB algorithm solution: random starts of the replicas),
 * for checks of the random draws.  Writes x, y float32[R][n_pad] (device, padded
 * layout, zero at padding columns) exactly as qh_bsb_solve draws them for replicas
 * replica_base .. replica_base + R - 1 of refinement iteration `iter`: SplitMix64 keyed
 * by (seed, block << 16 | iter), draw ((replica << 24) | local vertex) * 2 + {0: x, 1: y},
 * value ((v >> 40) 2^-24) 0.2 - 0.1 computed in FP64 and rounded once to FP32.
 * Errors: QH_EINVAL (R < 1, iter < 0, replica index >= 65536), QH_ENOMEM, QH_ECUDA. */
qh_status qh_debug_init_state(qh_ctx* ctx, const qh_graph* g, int32_t R, int32_t replica_base,
                              uint64_t seed, int32_t iter, float* x, float* y);

/* Step timeline of the multi-step kernel (tracing hook, not part of the paper's
 * method).  Runs steps 0 .. steps-1 of bSB (BF16, seed 1, default c0, dt = a0 = 1) as
 * ONE launch of multi-step variant `step_kernel` (6..9) with R replicas, and records
 * for the steps u0 .. u0+nu-1 of every CTA and item slot the hand-off points of its
 * pipeline: [0] inputs released, [1] last operand load issued, [2] accumulator free,
 * [3] first operand landed, [4] MMAs committed, [5] epilogue start, [6] epilogue end,
 * [7] X_hat released, [8] producer reaches the item, [9] its own previous step is
 * released, [10] its first ring slot is free, [11..15] the ring slots of its K-slices
 * 1..5 are free.  stamps (host) uint64[n_ctas][nu][4][32]: columns 0..15 the events as
 * global-timer nanoseconds, 16..31 the same events as SM clock cycles (0 = event not
 * reached or not recorded).
 * items (host, may be NULL) int32[n_ctas][4]: the item (row tile * R/128 + replica
 * tile) of each slot, -1 for none.  stamps = NULL only returns n_ctas.
 * Errors: QH_EINVAL (not a multi-step variant for this graph, or more than one wave),
 * QH_ENOMEM, QH_ECUDA, QH_ETIMEOUT. */
qh_status qh_debug_run_trace(qh_ctx* ctx, const qh_graph* g, int32_t R, int32_t step_kernel,
                             int32_t steps, int32_t u0, int32_t nu, uint64_t* stamps,
                             int32_t* items, int32_t* n_ctas);

/* Padded layout: n_pad and padded_index int32[n_nodes] (-1 for vertices in no
 * block): vertex v of block b sits at padded column pad_off[b] + local[v]. */
qh_status qh_debug_layout(qh_ctx* ctx, const qh_graph* g, int32_t* n_pad, int32_t* padded_index,
                          double* c0_default);

/* ---------------------------------------------------------------- no device allocation */

/* J_hat x X_hat with the BF16 tensor cores, exactly as qh_debug_matvec(...,
 * QH_PREC_BF16, ...) computes it, but without allocating any device memory.
 * The paper has no counterpart.  It serves callers that are not free to allocate
 * GPU memory: a host whose allocator already owns the device memory (a framework
 * or serving process that reserves the GPU's memory up front and hands it out
 * itself, where an extra cudaMalloc fails or escapes its accounting), and a
 * process held to a fixed device-memory budget.  Such callers pass their own
 * input and output buffers; the library adds nothing to the device's allocations.
 * x  float32[R][n_pad] (device, caller-owned): state in the padded layout
 * z  float32[R][n_pad] (device, caller-owned): output; set to zero, then every
 *    vertex of every block receives sum_b J_hat_ab X_hat_b in FP32
 * Working memory (the BF16 copy of x and two per-block parameter arrays) lives
 * in one fixed array of 8.5 MiB compiled into the library, which every GPU that
 * loads the library keeps until the process exits.  Limits: R a multiple of 64,
 * R * n_pad <= 4,194,304 and at most 65,536 blocks, otherwise QH_EINVAL with a
 * message.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use the library across a
 * cudaDeviceReset of the device.  All calls share the one array and each call
 * overwrites it in full, so two calls whose work overlaps on the GPU (different
 * streams or contexts) race on it.  The call synchronises the context stream and
 * reads back the context's error word before it returns.
 * Errors: QH_EINVAL, QH_ECUDA, QH_ETIMEOUT. */
qh_status qh_matvec_bf16_noalloc(qh_ctx* ctx, const qh_graph* g, int32_t R, const float* x,
                                 float* z);

#ifdef __cplusplus
}
#endif

#endif /* QHAP_H */
