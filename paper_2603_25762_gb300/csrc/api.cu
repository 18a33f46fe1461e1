// C ABI of libqhap: contexts, graph handles, the batched bSB solve (step loop
// captured once into a CUDA graph and replayed), phasing and test hooks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>

#include "qh_internal.cuh"
#include "util.cuh"

namespace qh {

qh_status set_err(Ctx* ctx, qh_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

qh_status cuda_fail(Ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (ctx) ctx->err = m;
  return e == cudaErrorMemoryAllocation ? QH_ENOMEM : QH_ECUDA;
}

bool alloc_permitted(const PoolRef& m) {
  if (!m.fail_after || *m.fail_after < 0) return true;
  if (*m.fail_after == 0) return false;
  --*m.fail_after;
  return true;
}

void* pool_alloc(const PoolRef& m, size_t bytes, std::vector<void*>* owner) {
  if (!alloc_permitted(m)) return nullptr;
  void* p = nullptr;
  cudaError_t e = m.pool ? cudaMallocFromPoolAsync(&p, bytes, m.pool, m.stream)
                         : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  owner->push_back(p);
  return p;
}

void pool_free_all(const PoolRef& m, std::vector<void*>* owned) {
  const bool ordered = m.pool && m.alive && *m.alive;
  for (void* p : *owned) {
    if (ordered)
      cudaFreeAsync(p, m.stream);  // after the work already queued on the stream
    else
      cudaFree(p);  // the context is gone: release synchronously
  }
  owned->clear();
}

void* dalloc(Graph& g, size_t bytes) { return pool_alloc(g.mem, bytes, &g.allocs); }

void* Ctx::scratch(size_t bytes, int slot) {
  if (slot >= (int)slots.size()) {
    slots.resize(slot + 1, nullptr);
    slot_bytes.resize(slot + 1, 0);
  }
  if (bytes == 0) bytes = 16;
  if (slot_bytes[slot] < bytes) {
    if (slots[slot]) {
      cudaStreamSynchronize(stream);
      cudaFree(slots[slot]);
      slots[slot] = nullptr;
      slot_bytes[slot] = 0;
      if (loop_exec) {  // captured pointers may dangle now
        cudaGraphExecDestroy(loop_exec);
        loop_exec = nullptr;
        loop_key.clear();
      }
    }
    void* p = nullptr;
    size_t want = bytes + bytes / 8;
    if (!alloc_permitted(mem)) return nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    slots[slot] = p;
    slot_bytes[slot] = want;
  }
  return slots[slot];
}

namespace {

// Scratch slot ids used by the solver (graph build uses 0..20).
enum {
  S_X = 32, S_Y, S_X1, S_XH0, S_XH1, S_SIGNS, S_NODEVAL, S_CUTS, S_BESTR, S_BESTCUT, S_ACTIVE,
  S_STEPSB, S_C0, S_SEEN, S_STALL, S_STEPSRUN, S_SPINS, S_C, S_WWORK, S_TBWORK, S_TFWORK,
  S_SUMW, S_SUMJ2, S_NODETMP, S_SIGNS1, S_NODEVAL1, S_CUT1, S_DBG0, S_DBG1, S_DBG2, S_RUNNING,
  S_PVWORK, S_TR0, S_TR1, S_F8H, S_F8L, S_F8FLAG, S_X8, S_DEFORM, S_TRIES, S_DBGDEF,
  S_ZBAND, S_BANDWORK, S_RVWORK, S_TRACE, S_KCUT, S_KR, S_KFLAG, S_KSPINS, S_GAUGE, S_CTRACE,
  S_CUTS_S, S_CUTS_Z
};

struct SolveBufs {
  float *x, *y, *x1;
  __nv_bfloat16 *xh0, *xh1;
  int8_t* signs;
  double *node_val, *cuts, *best_cut, *seen;
  int32_t *best_r, *active, *running, *steps_b, *stall, *steps_run;
  float* c0;
  int8_t* spins;
  int32_t* C;
  float* deform;    // nullptr without the refinement's deformation
  int32_t* tries;
  float* zband;     // CSR band-tile step: the band product Z ([n_pad][R]), else nullptr
  // track_best: the best result kept over the checks (cut, replica, copy flag, spins)
  double* kept_cut;
  int32_t *kept_r, *kept_flag;
  int8_t* kept_spins;
  int8_t* gauge;    // SNP mode: product of the partitions the weights are inverted by
  double* trace;    // energy checks: [checks][n_blocks] best cut of each check (NaN: none)
  // per-replica cuts on the tensor cores: the signs S in BF16 and z = J S, [R][n_pad]
  __nv_bfloat16* cut_s;
  float* cut_z;
};

qh_status run_step(Ctx* ctx, const Graph& g, int precision, const TcPlan& plan, StepArgs a,
                   const float* x_cur_f32, float* x_next_f32, const __nv_bfloat16* xh_cur,
                   __nv_bfloat16* xh_next, const Fp8Operands* f8 = nullptr, int64_t ns = 0,
                   float* zband = nullptr) {
  if (precision == QH_PREC_FP8) {  // X_hat buffers hold the e4m3 hi part, then the lo part
    Fp8Operands op = *f8;
    op.xh_in = reinterpret_cast<const uint8_t*>(xh_cur);
    op.xl_in = op.xh_in + ns;
    a.x8h_out = reinterpret_cast<uint8_t*>(xh_next);
    a.x8l_out = a.x8h_out + ns;
    return launch_step_f8(ctx, g, a, op);
  }
  if (precision == QH_PREC_FP32) {
    a.xin = x_cur_f32;
    a.xout = x_next_f32;
    if (g.csr_mode)
      launch_step_csr(ctx->stream, g, a, g.pval, nullptr, plan.variant);
    else
      launch_step_f32(ctx->stream, g, a);
    return QH_OK;
  }
  a.xh_out = xh_next;
  if (g.csr_mode) {
    if (plan.variant == CSR_BAND8) {  // band on the tensor cores, then the remainder
      qh_status st = launch_band_mma(ctx, g, a, g.band, xh_cur, zband);
      if (st != QH_OK) return st;
      a.zb = zband;
      launch_step_csr(ctx->stream, g, a, g.rval, xh_cur, plan.variant, true);
      return QH_OK;
    }
    launch_step_csr(ctx->stream, g, a, g.pval, xh_cur, plan.variant);
    return QH_OK;
  }
  return launch_step_tc(ctx, g, a, xh_cur, plan);
}

// The CUDA runtime is shared with the host application (for example PyTorch): its
// per-thread last-error slot may hold an error from someone else's call.  Entry
// points clear it so that stage checks report only this library's launches; the
// cleared error is kept in the context's message for diagnosis.
void clear_foreign_error(Ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) ctx->err = std::string("cleared a pending error from an earlier call: ") +
                                   cudaGetErrorString(e);
}

qh_status check_err_word(Ctx* ctx) {
  int32_t herr = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  QH_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (herr & ERR_TIMEOUT) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), ctx->stream);
    return set_err(ctx, QH_ETIMEOUT, "a bounded device wait expired in the bSB step kernel");
  }
  if (herr & ERR_CONFIG) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), ctx->stream);
    return set_err(ctx, QH_EINVAL, "the multi-step kernel refused its launch arguments");
  }
  return QH_OK;
}

// Time every valid step-kernel variant on the live state for a few steps and keep
// the fastest for this graph shape.  The state is re-initialised afterwards.
std::string tune_key(const Graph& g, int R, int use_lo, int sb) {
  char kb[160];
  snprintf(kb, sizeof kb, "%d|%d|%lld|%d|%d|%d|%d", R, g.n_row_tiles, (long long)g.n_tiles,
           g.max_tiles_per_row, g.n_pad, use_lo, sb);
  return kb;
}


bool tuned_variant(Ctx* ctx, const Graph& g, int R, int sb, TcPlan* plan) {
  const std::string kb = tune_key(g, R, 0, sb);
  for (auto& kv : ctx->tuned)
    if (kv.first == kb) {
      plan->variant = kv.second;
      return true;
    }
  return false;
}

// The multi-step kernel keeps y / (dt c0) on chip: every block's dt * c0 must be a
// normal float with a finite reciprocal.
bool run_c0_ok(const float* c0, int32_t nb, float dt) {
  for (int32_t b = 0; b < nb; ++b) {
    const float d = dt * c0[b];
    if (!std::isnormal(d) || !std::isfinite(1.0f / d)) return false;
  }
  return true;
}

qh_status autotune(Ctx* ctx, const Graph& g, StepArgs a, const SolveBufs& B, int R, TcPlan* plan,
                   bool allow_run) {
  const std::string kb = tune_key(g, R, 0, a.sb);
  cudaStream_t s = ctx->stream;
  float best = 1e30f;
  int best_v = -1;
  std::string rep;
  for (int v = 0; v < tc_n_variants(); ++v) {
    if (!tc_variant_ok(v, g, R, ctx->n_sm, a.use_lo != 0)) continue;
    if (run_variant(v) && !allow_run) continue;
    TcPlan p = *plan;
    p.variant = v;
    RunBufs rb;
    if (run_variant(v)) {
      qh_status st = run_prepare(ctx, g, R, v, a.use_lo != 0, &rb, nullptr,
                                 run_items(g, R, ctx->n_sm, v, a.use_lo != 0));
      if (st != QH_OK) return st;
    }
    float ms = 0.f;
    for (int rep_i = 0; rep_i < 2; ++rep_i) {  // warm-up pass, then the timed pass
      QH_CUDA_TRY(cudaEventRecord(ctx->ev[2], s));
      if (run_variant(v)) {  // the six steps in one launch
        qh_status st = launch_run(ctx, g, a, rb, B.xh0, B.xh1, 0, 6);
        if (st != QH_OK) return st;
      }
      for (int k = 0; k < 6 && !run_variant(v); ++k) {
        a.t = k;
        a.xh_out = (k % 2 == 0) ? B.xh1 : B.xh0;
        qh_status st = launch_step_tc(ctx, g, a, (k % 2 == 0) ? B.xh0 : B.xh1, p);
        if (st != QH_OK) return st;
      }
      QH_CUDA_TRY(cudaEventRecord(ctx->ev[3], s));
      QH_CUDA_TRY(cudaEventSynchronize(ctx->ev[3]));
      QH_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
    }
    ms /= 6.f;
    char line[96];
    snprintf(line, sizeof line, "%s%s=%.2fus", rep.empty() ? "" : ";", tc_variant_name(v), ms * 1e3f);
    rep += line;
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  qh_status st = check_err_word(ctx);
  if (st != QH_OK) return st;
  plan->variant = best_v;
  ctx->tuned.emplace_back(kb, best_v);
  ctx->tune_report = rep;
  return QH_OK;
}

TcPlan pick_plan(int R) {
  TcPlan p;
  p.bn = (R % 128 == 0) ? 128 : 64;
  p.stages = 3;
  return p;
}

}  // namespace
}  // namespace qh

using namespace qh;

extern "C" {

const char* qh_status_str(int st) {
  switch (st) {
    case QH_OK: return "QH_OK";
    case QH_EINVAL: return "QH_EINVAL";
    case QH_ENOMEM: return "QH_ENOMEM";
    case QH_ECUDA: return "QH_ECUDA";
    case QH_ETIMEOUT: return "QH_ETIMEOUT";
    case QH_EUNSUPPORTED: return "QH_EUNSUPPORTED";
    default: return "QH_UNKNOWN";
  }
}

const char* qh_last_error(const qh_ctx* ctx) { return ctx ? ctx->c.err.c_str() : ""; }

qh_status qh_create(qh_ctx** out, int device, void* stream) {
  if (!out) return QH_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return QH_EINVAL;
  }
  qh_ctx* h = new (std::nothrow) qh_ctx;
  if (!h) return QH_ENOMEM;
  Ctx* ctx = &h->c;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete h;
    return QH_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return QH_ECUDA;
    }
    ctx->own_stream = true;
  }
  {  // stream-ordered pool for graph and solution memory; keeps what it has reserved
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->mem.pool, &props) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(ctx->mem.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      (void)cudaGetLastError();
      ctx->mem.pool = nullptr;  // plain cudaMalloc / cudaFree
    }
    ctx->mem.stream = ctx->stream;
    ctx->mem.alive = std::make_shared<bool>(true);
    ctx->mem.fail_after = std::make_shared<int64_t>(-1);
  }
  if (cudaMalloc(&ctx->d_err, sizeof(int32_t)) != cudaSuccess ||
      cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), ctx->stream) != cudaSuccess) {
    delete h;
    return QH_ECUDA;
  }
  for (auto& e : ctx->ev) cudaEventCreate(&e);
  if (tc_prepare(ctx) != QH_OK) {
    qh_status st = QH_ECUDA;
    qh_destroy(h);
    return st;
  }
  *out = h;
  return QH_OK;
}

void qh_destroy(qh_ctx* h) {
  if (!h) return;
  Ctx* ctx = &h->c;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
  for (void* p : ctx->slots)
    if (p) cudaFree(p);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->mem.alive) *ctx->mem.alive = false;  // graphs and solutions left behind free synchronously
  if (ctx->mem.pool) cudaMemPoolDestroy(ctx->mem.pool);  // released once they are freed
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete h;
}

void qh_graph_free(qh_graph* g) {
  if (!g) return;
  // the owning context may already be gone: only the graph's own pool reference
  // (which knows whether it is) is used here
  pool_free_all(g->g.mem, &g->g.allocs);
  delete g;
}

qh_status qh_build_graph(qh_ctx* h, const qh_fragments* f, const qh_graph_opts* o, qh_graph** out) {
  NvtxRange nvtx_range("qh_build_graph");
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  clear_foreign_error(ctx);
  if (!f || !o || !out) return set_err(ctx, QH_EINVAL, "NULL argument");
  *out = nullptr;
  if (f->n_frags < 0 || f->n_snps < 0 || !f->frag_ptr)
    return set_err(ctx, QH_EINVAL, "bad fragment sizes or NULL frag_ptr");
  if (o->mode != QH_MODE_READ && o->mode != QH_MODE_SNP) return set_err(ctx, QH_EINVAL, "bad mode");
  if (o->mode == QH_MODE_READ && o->weight_mode != QH_WEIGHT_CONFLICT && o->weight_mode != QH_WEIGHT_SIGNED)
    return set_err(ctx, QH_EINVAL, "bad weight_mode");
  if (o->mode == QH_MODE_SNP) {
    if (o->linkage_k < 1 || o->linkage_k > 10) return set_err(ctx, QH_EINVAL, "linkage_k must be 1..10");
    if (!f->qual) return set_err(ctx, QH_EINVAL, "SNP mode needs qualities");
    if (!(o->porec_alpha >= 0.0)) return set_err(ctx, QH_EINVAL, "porec_alpha must be >= 0");
  }
  cudaSetDevice(ctx->device);
  qh_graph* gh = new (std::nothrow) qh_graph;
  if (!gh) return QH_ENOMEM;
  gh->owner = h;
  gh->g.mem = ctx->mem;
  qh_status st = build_graph_device(ctx, f, o, &gh->g);
  if (st != QH_OK) {
    cudaStreamSynchronize(ctx->stream);
    (void)cudaGetLastError();
    qh_graph_free(gh);
    return st;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    qh_graph_free(gh);
    return cuda_fail(ctx, e, "graph build");
  }
  *out = gh;
  return QH_OK;
}

qh_status qh_graph_info(const qh_graph* gh, int32_t* n_nodes, int32_t* n_blocks, int32_t* sizes,
                        int32_t cap, int64_t* nnz, int64_t* n_tiles) {
  if (!gh) return QH_EINVAL;
  const Graph& g = gh->g;
  if (n_nodes) *n_nodes = g.n_nodes;
  if (n_blocks) *n_blocks = g.n_blocks;
  if (sizes)
    for (int32_t b = 0; b < std::min(cap, g.n_blocks); ++b) sizes[b] = g.h_block_size[b];
  if (nnz) *nnz = g.nnz;
  if (n_tiles) *n_tiles = g.n_tiles;
  return QH_OK;
}

qh_status qh_graph_edges(qh_ctx* h, const qh_graph* gh, int64_t* rp, int32_t* col, double* w) {
  if (!h || !gh) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Graph& g = gh->g;
  cudaStream_t s = ctx->stream;
  if (rp) QH_CUDA_TRY(cudaMemcpyAsync(rp, g.row_ptr, sizeof(int64_t) * (g.n_nodes + 1), cudaMemcpyDeviceToHost, s));
  if (col && g.nnz) QH_CUDA_TRY(cudaMemcpyAsync(col, g.col, sizeof(int32_t) * g.nnz, cudaMemcpyDeviceToHost, s));
  if (w && g.nnz) QH_CUDA_TRY(cudaMemcpyAsync(w, g.w, sizeof(double) * g.nnz, cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  return QH_OK;
}

qh_status qh_graph_blocks(qh_ctx* h, const qh_graph* gh, int32_t* block_of, int32_t* local) {
  if (!h || !gh) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Graph& g = gh->g;
  cudaStream_t s = ctx->stream;
  if (block_of && g.n_nodes)
    QH_CUDA_TRY(cudaMemcpyAsync(block_of, g.block_of, sizeof(int32_t) * g.n_nodes, cudaMemcpyDeviceToHost, s));
  if (local && g.n_nodes)
    QH_CUDA_TRY(cudaMemcpyAsync(local, g.local, sizeof(int32_t) * g.n_nodes, cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  return QH_OK;
}

// The solve of every block (sel == nullptr) or of the listed blocks only.
static qh_status solve_impl(qh_ctx* h, const qh_graph* gh, const qh_bsb_opts* o,
                            const int32_t* sel, int32_t n_sel, qh_solution** out,
                            const qh_refine_state* rs = nullptr) {
  NvtxRange nvtx_range("qh_bsb_solve");
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  clear_foreign_error(ctx);
  if (!gh || !o || !out) return set_err(ctx, QH_EINVAL, "NULL argument");
  *out = nullptr;
  const Graph& G = gh->g;
  const int32_t R = o->replicas, nb = G.n_blocks;
  // blocks to solve: all, or the listed ones (each at most once)
  std::vector<int32_t> sel_mask(std::max(nb, 1), sel ? 0 : 1);
  if (sel) {
    if (n_sel < 0) return set_err(ctx, QH_EINVAL, "negative block count");
    for (int32_t k = 0; k < n_sel; ++k) {
      if (sel[k] < 0 || sel[k] >= nb) return set_err(ctx, QH_EINVAL, "block index out of range");
      if (sel_mask[sel[k]]) return set_err(ctx, QH_EINVAL, "block listed twice");
      sel_mask[sel[k]] = 1;
    }
  }
  if (R < 1) return set_err(ctx, QH_EINVAL, "replicas must be >= 1");
  if (o->schedule != QH_SCHED_LINEAR && o->schedule != QH_SCHED_AUTO) return set_err(ctx, QH_EINVAL, "bad schedule");
  if (o->schedule == QH_SCHED_LINEAR && o->steps < 1) return set_err(ctx, QH_EINVAL, "steps must be >= 1");
  if (o->precision != QH_PREC_FP32 && !is_tc_precision(o->precision) && o->precision != QH_PREC_FP8)
    return set_err(ctx, QH_EINVAL, "bad precision");
  if (o->sb_variant < QH_SB_BALLISTIC || o->sb_variant > QH_SB_ADIABATIC)
    return set_err(ctx, QH_EINVAL, "bad sb_variant");
  if (o->precision == QH_PREC_FP8 && G.csr_mode)
    return set_err(ctx, QH_EUNSUPPORTED, "FP8 needs tile storage (the graph is stored as CSR)");
  if (o->precision == QH_PREC_FP8 && R % 64 != 0)
    return set_err(ctx, QH_EINVAL, "FP8 precision needs replicas to be a multiple of 64");
  if (!(o->dt > 0.0) || !(o->a0 > 0.0)) return set_err(ctx, QH_EINVAL, "dt and a0 must be > 0");
  if (!(o->deform_h >= 0.0) || !std::isfinite(o->deform_h) || o->deform_tries < 0 ||
      o->check_mode < 0 || o->check_mode > 1 || o->track_best < 0 || o->track_best > 1)
    return set_err(ctx, QH_EINVAL,
                   "deform_h must be finite and >= 0, deform_tries >= 0, check_mode and track_best 0 or 1");
  if (o->check_every < 0 || o->patience < 0 || o->replica_base < 0) return set_err(ctx, QH_EINVAL, "negative option");
  if ((int64_t)o->replica_base + R > (1 << 16)) return set_err(ctx, QH_EINVAL, "replica indices must stay below 65536");
  if (is_tc_precision(o->precision) && o->step_kernel >= 0 && !G.csr_mode &&
      (o->step_kernel >= tc_n_variants() ||
       !tc_variant_ok(o->step_kernel, G, R, ctx->n_sm, use_lo_for(G, o->precision))))
    return set_err(ctx, QH_EINVAL, "step_kernel variant not valid for this graph and replica count");
  const bool snp = G.mode == QH_MODE_SNP;
  const int32_t refine_max = snp ? o->refine_max : 1;
  if (refine_max < 1) return set_err(ctx, QH_EINVAL, "refine_max must be >= 1");
  // a resumed refinement: the saved state must fit the graph and the options
  const int32_t it0 = rs ? rs->iterations_done : 0;
  if (rs) {
    if (!snp) return set_err(ctx, QH_EINVAL, "only a SNP-mode refinement can be resumed");
    if (!rs->flips || !rs->gauge || !rs->refining || !rs->solves || !rs->deform || !rs->tries)
      return set_err(ctx, QH_EINVAL, "NULL array in the refinement state");
    if (it0 < 1 || it0 >= refine_max)
      return set_err(ctx, QH_EINVAL, "iterations_done must be >= 1 and below refine_max");
    const bool dfm = o->deform_h > 0.0 && o->deform_tries > 0;
    for (int32_t v = 0; v < G.n_nodes; ++v)
      if (rs->gauge[v] != 1 && rs->gauge[v] != -1)
        return set_err(ctx, QH_EINVAL, "gauge values must be +1 or -1");
    for (int32_t b = 0; b < nb; ++b)
      if (rs->solves[b] < 0 || rs->tries[b] < 0 || !(rs->deform[b] >= 0.f) ||
          !std::isfinite(rs->deform[b]) || (!dfm && (rs->deform[b] != 0.f || rs->tries[b] != 0)))
        return set_err(ctx, QH_EINVAL,
                       "negative count or deformation in the refinement state (a deformation "
                       "needs deform_h > 0 and deform_tries > 0)");
  }
  const TcPlan plan = pick_plan(R);
  if (G.csr_mode && R % 4 != 0)
    return set_err(ctx, QH_EINVAL, "CSR storage needs replicas to be a multiple of 4");
  if (o->step_kernel >= 0 && (G.csr_mode != (o->step_kernel >= CSR_LANE4) ||
                              (G.csr_mode && !csr_variant_ok(o->step_kernel, R, o->precision))))
    return set_err(ctx, QH_EINVAL, "step_kernel variant not valid for this graph storage and R");
  if (is_tc_precision(o->precision) && !G.csr_mode && !tc_plan_ok(R, plan))
    return set_err(ctx, QH_EINVAL, "BF16 precision needs replicas to be a multiple of 64");
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  qh_solution* sh = new (std::nothrow) qh_solution;
  if (!sh) return QH_ENOMEM;
  // every return that does not hand the solution out frees it (with any device memory)
  struct SolutionGuard {
    qh_solution*& p;
    ~SolutionGuard() {
      if (p) qh_solution_free(p);
    }
  } sol_guard{sh};
  Solution& sol = sh->s;
  sol.mode = G.mode;
  sol.n_blocks = nb;
  sol.R = R;
  sol.replica_base = o->replica_base;
  sol.n_nodes = G.n_nodes;
  sol.block_size = G.h_block_size;
  sol.block_ptr = G.h_block_ptr;
  sol.best_r.assign(nb, 0);
  sol.steps_run.assign(nb, 0);
  sol.iters.assign(nb, 0);
  sol.best_cut.assign(nb, 0.0);
  sol.cuts_first.assign((size_t)nb * R, 0.0);
  sol.spins.assign(G.n_nodes, 0);
  sol.C.assign(G.n_nodes, 0);
  sol.solved.assign(std::max(nb, 1), 0);
  int32_t n_solve = 0;
  for (int32_t b = 0; b < nb; ++b) {
    sol.solved[b] = (uint8_t)sel_mask[b];
    n_solve += sel_mask[b];
  }
  if (n_solve == 0) {  // no block, or an empty selection: nothing to solve
    for (int32_t v = 0; v < G.n_nodes; ++v) sol.C[v] = -1;
    sol.mem = ctx->mem;
    sol.d_spins = (int8_t*)pool_alloc(sol.mem, std::max(G.n_nodes, 1), &sol.allocs);
    sol.d_C = (int32_t*)pool_alloc(sol.mem, (size_t)std::max(G.n_nodes, 1) * 4, &sol.allocs);
    if (!sol.d_spins || !sol.d_C) return set_err(ctx, QH_ENOMEM, "allocation failed (solution)");
    sol.device_stale = true;
    *out = sh;
    sh = nullptr;
    return QH_OK;
  }
  // ---- per-block schedule and coupling scale
  std::vector<int32_t> h_steps(nb);
  int32_t max_steps = 0;
  for (int32_t b = 0; b < nb; ++b) {
    h_steps[b] = o->schedule == QH_SCHED_AUTO ? (G.h_block_size[b] < 5000 ? 500 : 1000) : o->steps;
    max_steps = std::max(max_steps, h_steps[b]);
  }
  std::vector<float> h_c0(nb);
  for (int32_t b = 0; b < nb; ++b) h_c0[b] = (float)(o->c0 > 0.0 ? o->c0 : G.h_c0[b]);
  // ---- buffers
  const size_t NS = (size_t)R * G.n_pad;
  SolveBufs B{};
  auto sc = [&](size_t bytes, int slot) { return ctx->scratch(bytes, slot); };
  B.x = (float*)sc(NS * 4, S_X);
  B.y = (float*)sc(NS * 4, S_Y);
  if (o->precision == QH_PREC_FP32) {
    B.x1 = (float*)sc(NS * 4, S_X1);
  } else {
    B.xh0 = (__nv_bfloat16*)sc(NS * 2, S_XH0);
    B.xh1 = (__nv_bfloat16*)sc(NS * 2, S_XH1);
  }
  B.signs = (int8_t*)sc(NS, S_SIGNS);
  B.node_val = (double*)sc(NS * 8, S_NODEVAL);
  B.cuts = (double*)sc((size_t)nb * R * 8, S_CUTS);
  B.best_r = (int32_t*)sc(nb * 4, S_BESTR);
  B.best_cut = (double*)sc(nb * 8, S_BESTCUT);
  B.active = (int32_t*)sc(nb * 4, S_ACTIVE);
  B.running = (int32_t*)sc(nb * 4, S_RUNNING);
  B.steps_b = (int32_t*)sc(nb * 4, S_STEPSB);
  B.c0 = (float*)sc(nb * 4, S_C0);
  B.seen = (double*)sc(nb * 8, S_SEEN);
  B.stall = (int32_t*)sc(nb * 4, S_STALL);
  B.steps_run = (int32_t*)sc(nb * 4, S_STEPSRUN);
  B.spins = (int8_t*)sc(G.n_nodes + 16, S_SPINS);
  B.C = (int32_t*)sc((G.n_nodes + 1) * 4, S_C);
  B.gauge = snp ? (int8_t*)sc((size_t)G.n_nodes + 16, S_GAUGE) : nullptr;
  // the refinement's adaptive deformation: per-block field strength and re-solve count
  const bool deform_on = snp && o->deform_h > 0.0 && o->deform_tries > 0;
  // CSR storage: the step variant (the band-tile step needs the band product buffer and,
  // in SNP mode, working copies of the band tiles and remainder values)
  const int csr_v = !G.csr_mode ? -1
                    : o->step_kernel >= 0 ? o->step_kernel
                                          : csr_default_variant(G, o->precision, R);
  const bool band_on = csr_v == CSR_BAND8;
  B.zband = band_on ? (float*)sc(NS * 4, S_ZBAND) : nullptr;
  B.deform = deform_on ? (float*)sc(nb * 4, S_DEFORM) : nullptr;
  B.tries = deform_on ? (int32_t*)sc(nb * 4, S_TRIES) : nullptr;
  const bool track = o->track_best != 0 && o->check_every > 0;
  B.kept_cut = track ? (double*)sc(nb * 8, S_KCUT) : nullptr;
  B.kept_r = track ? (int32_t*)sc(nb * 4, S_KR) : nullptr;
  B.kept_flag = track ? (int32_t*)sc(nb * 4, S_KFLAG) : nullptr;
  B.kept_spins = track ? (int8_t*)sc(G.n_nodes + 16, S_KSPINS) : nullptr;
  bool okb = B.x && B.y && B.signs && B.node_val && B.cuts && B.best_r && B.best_cut && B.active && B.running &&
             B.steps_b && B.c0 && B.seen && B.stall && B.steps_run && B.spins && B.C &&
             (!snp || B.gauge) &&
             (!deform_on || (B.deform && B.tries)) && (!band_on || B.zband) &&
             (!track || (B.kept_cut && B.kept_r && B.kept_flag && B.kept_spins)) &&
             (o->precision == QH_PREC_FP32 ? B.x1 != nullptr : (B.xh0 && B.xh1));
  // working copy of the graph for the SNP refinement (weights, tiles, sums are gauged)
  Graph W = G;
  W.allocs.clear();
  double* sum_w_work = G.sum_w;
  if (snp && okb) {
    W.w = (double*)sc(std::max<int64_t>(G.nnz, 1) * 8, S_WWORK);
    W.tile_bf16 = (__nv_bfloat16*)sc(std::max<int64_t>(G.n_tiles, 1) * TILE * TILE * 2, S_TBWORK);
    W.tile_f32 = (float*)sc(std::max<int64_t>(G.n_tiles_hi, 1) * TILE * TILE * 4, S_TFWORK);
    if (G.csr_mode) {
      W.pval = (float*)sc(std::max<int64_t>(G.pnnz, 1) * 4, S_PVWORK);
      if (W.pval && G.pnnz)
        QH_CUDA_TRY(cudaMemcpyAsync(W.pval, G.pval, G.pnnz * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (band_on) {
      const size_t bb = (size_t)3 * G.n_row_tiles * TILE * TILE * 2;
      W.band = (__nv_bfloat16*)sc(std::max<size_t>(bb, 2), S_BANDWORK);
      W.rval = (float*)sc(std::max<int64_t>(G.rnnz, 1) * 4, S_RVWORK);
      if (!W.band || !W.rval) okb = false;
      if (okb && bb) QH_CUDA_TRY(cudaMemcpyAsync(W.band, G.band, bb, cudaMemcpyDeviceToDevice, s));
      if (okb && G.rnnz)
        QH_CUDA_TRY(cudaMemcpyAsync(W.rval, G.rval, G.rnnz * 4, cudaMemcpyDeviceToDevice, s));
    }
    sum_w_work = (double*)sc(nb * 8, S_SUMW);
    double* sj2 = (double*)sc(nb * 8, S_SUMJ2);
    double* ntmp = (double*)sc((size_t)std::max(G.n_nodes, 1) * 16, S_NODETMP);
    okb = W.w && W.tile_bf16 && W.tile_f32 && sum_w_work && sj2 && ntmp && W.pval &&
          (!band_on || (W.band && W.rval));
    if (okb) {
      if (G.nnz) QH_CUDA_TRY(cudaMemcpyAsync(W.w, G.w, G.nnz * 8, cudaMemcpyDeviceToDevice, s));
      if (G.n_tiles)
        QH_CUDA_TRY(cudaMemcpyAsync(W.tile_bf16, G.tile_bf16, G.n_tiles * TILE * TILE * 2,
                                    cudaMemcpyDeviceToDevice, s));
      if (G.n_tiles_hi)
        QH_CUDA_TRY(cudaMemcpyAsync(W.tile_f32, G.tile_f32, G.n_tiles_hi * TILE * TILE * 4,
                                    cudaMemcpyDeviceToDevice, s));
      QH_CUDA_TRY(cudaMemcpyAsync(sum_w_work, G.sum_w, nb * 8, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (!okb) return set_err(ctx, QH_ENOMEM, "device allocation failed (solver state)");
  // FP8: e4m3 hi / lo tiles of s*J from the (working) FP32 tiles
  const bool fp8 = o->precision == QH_PREC_FP8;
  Fp8Operands f8{};
  const float f8_s = fp8 ? fp8_scale(G) : 1.f;
  uint8_t *f8_jh = nullptr, *f8_jl = nullptr;
  int32_t* f8_flag = nullptr;
  const int64_t f8_n = G.n_tiles_hi * (int64_t)TILE * TILE;
  auto convert_fp8_tiles = [&]() -> qh_status {
    QH_CUDA_TRY(cudaMemsetAsync(f8_flag, 0, 4, s));
    launch_tiles_to_e4m3(s, W.tile_f32, f8_n, f8_s, f8_jh, f8_jl, f8_flag);
    int32_t hl = 0;
    QH_CUDA_TRY(cudaMemcpyAsync(&hl, f8_flag, 4, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    f8.n_slices = hl ? 3 : 2;
    return QH_OK;
  };
  if (fp8) {
    f8_jh = (uint8_t*)sc(std::max<int64_t>(f8_n, 1), S_F8H);
    f8_jl = (uint8_t*)sc(std::max<int64_t>(f8_n, 1), S_F8L);
    f8_flag = (int32_t*)sc(16, S_F8FLAG);
    if (!f8_jh || !f8_jl || !f8_flag) {
      return set_err(ctx, QH_ENOMEM, "device allocation failed (FP8 tiles)");
    }
    qh_status st = convert_fp8_tiles();
    if (st != QH_OK) return st;
    f8.jh = f8_jh;
    f8.jl = f8_jl;
  }
  QH_CUDA_TRY(cudaMemcpyAsync(B.steps_b, h_steps.data(), nb * 4, cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemcpyAsync(B.c0, h_c0.data(), nb * 4, cudaMemcpyHostToDevice, s));
  QH_CUDA_TRY(cudaMemsetAsync(B.C, 0, (G.n_nodes + 1) * 4, s));
  if (B.deform) {
    QH_CUDA_TRY(cudaMemsetAsync(B.deform, 0, nb * 4, s));
    QH_CUDA_TRY(cudaMemsetAsync(B.tries, 0, nb * 4, s));
  }
  // the second operand buffer is written at real vertices only: its padding columns
  // must hold zeros (they meet the zero columns of J, and 0 * NaN would not vanish)
  if (o->precision == QH_PREC_FP32)
    QH_CUDA_TRY(cudaMemsetAsync(B.x1, 0, NS * 4, s));
  else
    QH_CUDA_TRY(cudaMemsetAsync(B.xh1, 0, NS * 2, s));
  QH_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 4, s));
  // blocks left out of a partial solve keep zero cuts, picks and spins
  QH_CUDA_TRY(cudaMemsetAsync(B.cuts, 0, (size_t)nb * R * 8, s));
  QH_CUDA_TRY(cudaMemsetAsync(B.best_r, 0, nb * 4, s));
  QH_CUDA_TRY(cudaMemsetAsync(B.best_cut, 0, nb * 8, s));
  QH_CUDA_TRY(cudaMemsetAsync(B.spins, 0, G.n_nodes + 16, s));
  QH_CUDA_TRY(cudaMemcpyAsync(B.active, sel_mask.data(), nb * 4, cudaMemcpyHostToDevice, s));
  if (snp) QH_CUDA_TRY(cudaMemsetAsync(B.gauge, 1, (size_t)G.n_nodes + 16, s));
  std::vector<int32_t> h_active0(sel_mask.begin(), sel_mask.begin() + nb);
  if (rs) {
    // the saved flip counts, gauge, refining blocks and deformation; the working graph
    // becomes the gauged one, as the solve after the checkpoint would have found it
    std::vector<int32_t> hC(std::max(G.n_nodes, 1), 0);
    for (int32_t v = 0; v < G.n_nodes; ++v) hC[v] = std::max(rs->flips[v], 0);
    for (int32_t b = 0; b < nb; ++b) {
      h_active0[b] = sel_mask[b] && rs->refining[b] ? 1 : 0;
      if (sel_mask[b]) sol.iters[b] = rs->solves[b];
    }
    if (G.n_nodes) {
      QH_CUDA_TRY(cudaMemcpyAsync(B.C, hC.data(), (size_t)G.n_nodes * 4, cudaMemcpyHostToDevice, s));
      QH_CUDA_TRY(cudaMemcpyAsync(B.gauge, rs->gauge, G.n_nodes, cudaMemcpyHostToDevice, s));
    }
    QH_CUDA_TRY(cudaMemcpyAsync(B.active, h_active0.data(), nb * 4, cudaMemcpyHostToDevice, s));
    if (B.deform) {
      QH_CUDA_TRY(cudaMemcpyAsync(B.deform, rs->deform, nb * 4, cudaMemcpyHostToDevice, s));
      QH_CUDA_TRY(cudaMemcpyAsync(B.tries, rs->tries, nb * 4, cudaMemcpyHostToDevice, s));
    }
    launch_apply_gauge(s, W, G.w, B.gauge, W.w);
    qh_status st = retile(ctx, &W, W.w, W.tile_bf16, W.tile_f32, W.csr_mode ? W.pval : nullptr);
    if (st == QH_OK && band_on) st = reband(ctx, &W, W.w, W.band, W.rval);
    if (st == QH_OK && fp8) st = convert_fp8_tiles();
    if (st != QH_OK) return st;
    launch_block_sums(s, W, W.w, sum_w_work, (double*)ctx->scratch(nb * 8, S_SUMJ2),
                      (double*)ctx->scratch((size_t)std::max(G.n_nodes, 1) * 16, S_NODETMP));
    // the host's copies of these arrays must not change before the copies above ran
    QH_CUDA_TRY(cudaStreamSynchronize(s));
  }
  QH_CUDA_TRY(cudaEventRecord(ctx->ev[0], s));

  // energy checks every check_every steps: for the early stop (patience > 0) and for
  // the best result during the run (track_best)
  const bool early = o->check_every > 0 && o->patience > 0;
  const bool checking = early || track;
  // the energy-check trace of each solve: the best cut over the replicas per block at
  // each check t = check_every, 2 check_every, ... < max_steps
  const int32_t n_checks = checking ? (max_steps - 1) / o->check_every : 0;
  B.trace = n_checks > 0 ? (double*)ctx->scratch((size_t)n_checks * nb * 8, S_CTRACE) : nullptr;
  if (n_checks > 0 && !B.trace) return set_err(ctx, QH_ENOMEM, "allocation failed (check trace)");
  // The replicas' cuts (every check and the end of each solve) as one product z = J S on
  // the tensor cores, S = sgn(x) in BF16, instead of a gather per edge: exact when the
  // weights are integers and every row sum of |J| stays below 2^24 (FP32 accumulation),
  // on tile storage with R a multiple of 64.
  bool tc_cut = !W.csr_mode && W.integer_weights && W.n_tiles > 0 && R % 64 == 0;
  if (tc_cut) {
    int32_t max_n = 0;
    for (int32_t b = 0; b < nb; ++b) max_n = std::max(max_n, W.h_block_size[b]);
    tc_cut = W.max_abs_w * (double)max_n < 16777216.0;
  }
  B.cut_s = tc_cut ? (__nv_bfloat16*)ctx->scratch(NS * 2, S_CUTS_S) : nullptr;
  B.cut_z = tc_cut ? (float*)ctx->scratch(NS * 4, S_CUTS_Z) : nullptr;
  if (tc_cut && (!B.cut_s || !B.cut_z))
    return set_err(ctx, QH_ENOMEM, "allocation failed (tensor-core cuts)");
  // ---- the step loop, captured once per shape and replayed
  // The captured step loop bakes in pointers and sizes; it is replayed only when every
  // one of them is unchanged (a rebuilt graph at other addresses is captured anew).
  std::string skey;
  {
    auto add = [&skey](const void* p) { skey += std::to_string((uintptr_t)p) + "|"; };
    auto addi = [&skey](long long v) { skey += std::to_string(v) + "|"; };
    addi(o->precision); addi(R); addi(max_steps); addi(checking ? o->check_every : 0);
    addi(o->sb_variant);
    addi(o->patience);
    addi(track ? 1 : 0);
    char d[64];
    snprintf(d, sizeof d, "%.17g|%.17g|", o->dt, o->a0);
    skey += d;
    addi(G.n_nodes); addi(G.n_pad); addi(G.n_blocks); addi(G.n_row_tiles); addi(G.n_tiles);
    addi(G.n_tiles_hi); addi(G.has_lo); addi(G.csr_mode); addi(G.integer_weights);
    addi(G.max_tiles_per_row); addi(G.pnnz); addi(G.nnz);
    addi(f8.n_slices); add(f8_jh); add(f8_jl);
    skey += std::to_string(f8_s) + "|";
    for (const void* p : {(const void*)G.rt, (const void*)G.tile_col, (const void*)W.tile_bf16,
                          (const void*)W.tile_f32, (const void*)G.prow_ptr, (const void*)G.pcol,
                          (const void*)W.pval, (const void*)W.band, (const void*)W.rval,
                          (const void*)G.rrow_ptr, (const void*)G.rcol, (const void*)B.zband,
                          (const void*)G.row_ptr, (const void*)G.col,
                          (const void*)W.w, (const void*)G.block_of, (const void*)G.pad_index,
                          (const void*)G.pad_node, (const void*)G.local, (const void*)G.pad_off,
                          (const void*)G.block_ptr, (const void*)G.perm, (const void*)sum_w_work})
      add(p);
    for (const void* p : {(const void*)B.x, (const void*)B.y, (const void*)B.x1, (const void*)B.xh0,
                          (const void*)B.xh1, (const void*)B.signs, (const void*)B.node_val,
                          (const void*)B.cuts, (const void*)B.best_r, (const void*)B.best_cut,
                          (const void*)B.running, (const void*)B.steps_b, (const void*)B.c0,
                          (const void*)B.seen, (const void*)B.stall, (const void*)B.steps_run,
                          (const void*)ctx->d_err, (const void*)B.deform, (const void*)B.trace,
                          (const void*)B.cut_s, (const void*)B.cut_z})
      add(p);
  }
  StepArgs a{};
  a.rt = G.rt;
  a.tile_col = G.tile_col;
  a.tile_f32 = W.tile_f32;
  a.x = B.x;
  a.y = B.y;
  a.c0 = B.c0;
  a.deform = B.deform;
  a.active = B.running;
  a.steps_b = B.steps_b;
  a.n_pad = G.n_pad;
  a.R = R;
  a.dt = (float)o->dt;
  a.a0 = o->a0;
  a.dta0 = (float)(o->dt * o->a0);
  a.err = ctx->d_err;
  a.sb = o->sb_variant;
  const float* x_final = B.x;
  if (o->precision == QH_PREC_FP32 && (max_steps % 2 == 1)) x_final = B.x1;
  TcPlan tplan = plan;
  a.use_lo = use_lo_for(G, o->precision);
  a.inv_scale = 1.f / f8_s;
  if (is_tc_precision(o->precision)) {
    qh_status st = QH_OK;
    if (o->step_kernel >= 0 && !G.csr_mode) {
      tplan.variant = o->step_kernel;
    } else if (!G.csr_mode) {
      if (!tuned_variant(ctx, G, R, o->sb_variant, &tplan)) {  // first solve of this shape: time the variants
        QH_CUDA_TRY(cudaMemcpyAsync(B.running, B.active, nb * 4, cudaMemcpyDeviceToDevice, s));
        launch_init_state(s, W, R, o->replica_base, o->seed, 0, B.x, B.y, B.xh0, B.active,
                          o->sb_variant);
        QH_STAGE_CHECK("solve: state init (tuning)");
        st = autotune(ctx, W, a, B, R, &tplan, run_c0_ok(h_c0.data(), nb, a.dt));
      }
    }
    if (st != QH_OK) return st;
  }
  if (G.csr_mode) tplan.variant = csr_v;
  sol.kernel = G.csr_mode ? csr_variant_name(tplan.variant, is_tc_precision(o->precision))
              : fp8 ? (R % 128 == 0 ? "e4m3-bn128-s2-x3" : "e4m3-bn64-s2-x4")
              : is_tc_precision(o->precision) ? tc_variant_name(tplan.variant) : "k_step_f32";
  skey += "|v" + std::to_string(tplan.variant);
  // the multi-step kernel runs whole step ranges: a few direct launches, no capture
  const bool multistep = is_tc_precision(o->precision) && !G.csr_mode && run_variant(tplan.variant);
  RunBufs rb;
  if (multistep && !run_c0_ok(h_c0.data(), nb, a.dt)) {
    return set_err(ctx, QH_EINVAL, "multi-step kernel needs dt * c0 to be a normal float in every block");
  }
  // Early-stop checks inside the multi-step launch: integer weights, so that the tensor
  // cores give the energies exactly (every row sum of |J| below 2^24), and every block
  // in one wave at three items per SM (the fourth item's TMEM holds the check product).
  // The kernel with checks runs its steps about 20% slower than the one without, and a
  // check between launches costs about 30 step times (hifi-region, 1,024 replicas), so
  // the checks move inside the launch when they come at least every FUSED_CHECK_MAX
  // steps.
  constexpr int32_t FUSED_CHECK_MAX = 128;
  bool fused = multistep && early && !track && o->check_mode == 0 && W.integer_weights &&
               o->check_every <= FUSED_CHECK_MAX;
  if (fused) {
    int32_t max_n = 0;
    for (int32_t b = 0; b < nb; ++b) max_n = std::max(max_n, W.h_block_size[b]);
    fused = W.max_abs_w * (double)max_n < 16777216.0 &&
            run_plan(W, R, ctx->n_sm, tplan.variant, a.use_lo != 0, nullptr,
                     sel ? &sel_mask : nullptr, 3);
  }
  RunCheck chk;
  if (multistep) {
    qh_status st = run_prepare(ctx, W, R, tplan.variant, a.use_lo != 0, &rb,
                               sel ? &sel_mask : nullptr,
                               fused ? 3
                                     : run_items(W, R, ctx->n_sm, tplan.variant, a.use_lo != 0,
                                                 sel ? &sel_mask : nullptr));
    if (st != QH_OK) return st;
  }
  if (fused) {
    chk.check_every = o->check_every;
    chk.patience = o->patience;
    chk.s = (__nv_bfloat16*)ctx->scratch((size_t)2 * NS * 2, S_RUN_S);
    chk.sum_w = sum_w_work;
    chk.e_sum = (unsigned long long*)ctx->scratch((size_t)2 * nb * R * 8, S_RUN_E);
    chk.e_cnt = (uint32_t*)ctx->scratch((size_t)4 * nb * 4, S_RUN_EC);  // e_cnt, decided, stop_t
    chk.seen = B.seen;
    chk.stall = B.stall;
    chk.trace = B.trace;
    if (!chk.s || !chk.e_sum || !chk.e_cnt)
      return set_err(ctx, QH_ENOMEM, "allocation failed (early-stop checks)");
    chk.decided = chk.e_cnt + 2 * nb;
    chk.stop_t = reinterpret_cast<int32_t*>(chk.e_cnt + 3 * nb);
  }
  // every replica's cut of the state x (signs into B.signs for the picks and spins)
  auto replica_cuts = [&](const float* xc, const int32_t* act) -> qh_status {
    launch_signs(s, W, R, xc, B.signs);
    if (!tc_cut) {
      launch_cut(s, W, R, B.signs, W.w, sum_w_work, B.node_val, B.cuts, act);
      return QH_OK;
    }
    launch_x_operand(s, W, QH_SB_DISCRETE, xc, B.cut_s, (int64_t)NS);
    StepArgs az = a;
    az.z_out = B.cut_z;
    az.t = 0;
    az.active = act;
    az.use_lo = W.has_lo ? 1 : 0;
    qh_status st = launch_step_tc(ctx, W, az, B.cut_s, pick_plan(R));
    if (st != QH_OK) return st;
    launch_cut_from_product(s, W, R, B.cut_z, B.cut_s, sum_w_work, B.node_val, B.cuts, act);
    return QH_OK;
  };
  if (!multistep && (ctx->loop_key != skey || !ctx->loop_exec)) {
    if (ctx->loop_exec) {
      cudaGraphExecDestroy(ctx->loop_exec);
      ctx->loop_exec = nullptr;
    }
    ctx->loop_key.clear();
    cudaGraph_t graph;
    const int64_t before = launches();
    QH_STAGE_CHECK("solve: before step-loop capture");
    QH_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    qh_status st = QH_OK;
    for (int32_t t = 0; t < max_steps && st == QH_OK; ++t) {
      a.t = t;
      const bool even = (t % 2) == 0;
      st = run_step(ctx, W, o->precision, tplan, a, even ? B.x : B.x1, even ? B.x1 : B.x,
                    even ? B.xh0 : B.xh1, even ? B.xh1 : B.xh0, &f8, (int64_t)NS, B.zband);
      if (checking && (t + 1) % o->check_every == 0 && t + 1 < max_steps) {
        const float* xc = (o->precision == QH_PREC_FP32 && even) ? B.x1 : B.x;
        if (st == QH_OK) st = replica_cuts(xc, B.running);
        launch_pick_best(s, nb, R, B.cuts, B.best_r, B.best_cut, B.running);
        launch_trace_check(s, nb, B.best_cut, B.running, t + 1, B.steps_b,
                           B.trace + (size_t)((t + 1) / o->check_every - 1) * nb);
        if (track)
          launch_track_check(s, W, R, B.signs, B.best_cut, B.best_r, B.running, t + 1, B.steps_b,
                             B.kept_cut, B.kept_r, B.kept_flag, B.kept_spins);
        if (early)
          launch_early_stop(s, nb, B.best_cut, B.seen, B.stall, B.running, B.steps_run,
                            o->patience, t + 1, B.steps_b);
      }
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != QH_OK) {
      if (ce == cudaSuccess) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&ctx->loop_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      ctx->loop_exec = nullptr;
      return cuda_fail(ctx, ce, "cudaGraphInstantiate");
    }
    ctx->loop_key = skey;
    // the captured launches run on each replay, not at capture time
    ctx->loop_kernels = launches() - before;
    note_launch(-ctx->loop_kernels);
  }
  double step_ms_total = 0.0, spin_updates = 0.0;
  int64_t launches = 0;
  std::vector<int32_t> h_active(h_active0), h_steps_run(nb);
  int32_t it_last = it0 - 1;
  bool any0 = false;
  for (int32_t b = 0; b < nb; ++b) any0 = any0 || h_active0[b];
  for (int32_t it = it0; it < refine_max && any0; ++it) {
    it_last = it;
    NvtxRange nvtx_iter("qh_bsb_solve: solve of every active block");
    for (int32_t b = 0; b < nb; ++b)
      if (h_active[b]) sol.iters[b] += 1;
    // steps_run defaults to the block's schedule length; early stop lowers it
    QH_CUDA_TRY(cudaMemcpyAsync(B.steps_run, h_steps.data(), nb * 4, cudaMemcpyHostToDevice, s));
    if (early) {
      std::vector<double> neg(nb, -INFINITY);
      QH_CUDA_TRY(cudaMemcpyAsync(B.seen, neg.data(), nb * 8, cudaMemcpyHostToDevice, s));
      QH_CUDA_TRY(cudaMemsetAsync(B.stall, 0, nb * 4, s));
    }
    if (track) {  // nothing kept yet
      std::vector<double> neg(nb, -INFINITY);
      QH_CUDA_TRY(cudaMemcpyAsync(B.kept_cut, neg.data(), nb * 8, cudaMemcpyHostToDevice, s));
      QH_CUDA_TRY(cudaMemsetAsync(B.kept_r, 0xff, nb * 4, s));
    }
    QH_CUDA_TRY(cudaMemcpyAsync(B.running, B.active, nb * 4, cudaMemcpyDeviceToDevice, s));
    if (B.trace)  // NaN until a check records a block
      QH_CUDA_TRY(cudaMemsetAsync(B.trace, 0xff, (size_t)n_checks * nb * 8, s));
    launch_init_state(s, W, R, o->replica_base, o->seed, it, B.x, B.y,
                      is_tc_precision(o->precision) ? B.xh0 : nullptr, B.active, o->sb_variant);
    if (fp8)
      launch_x_operand_e4m3(s, W, o->sb_variant, B.x, (int64_t)NS,
                            reinterpret_cast<uint8_t*>(B.xh0), reinterpret_cast<uint8_t*>(B.xh0) + NS);
    QH_STAGE_CHECK("solve: state init");
    QH_CUDA_TRY(cudaEventRecord(ctx->ev[2], s));
    if (fused) {
      // one launch over all steps; the blocks stop inside it
      QH_CUDA_TRY(cudaMemsetAsync(chk.s, 0, (size_t)2 * NS * 2, s));
      QH_CUDA_TRY(cudaMemsetAsync(chk.e_sum, 0, (size_t)2 * nb * R * 8, s));
      QH_CUDA_TRY(cudaMemsetAsync(chk.e_cnt, 0, (size_t)3 * nb * 4, s));
      QH_CUDA_TRY(cudaMemsetAsync(chk.stop_t, 0xff, (size_t)nb * 4, s));
      qh_status st = launch_run(ctx, W, a, rb, B.xh0, B.xh1, 0, max_steps, nullptr, 0, 0, &chk);
      if (st != QH_OK) return st;
      launch_stop_fixup(s, W, R, chk, B.x, B.steps_run);
    } else if (multistep) {
      const int32_t chunk = checking ? o->check_every : max_steps;
      for (int32_t t0 = 0; t0 < max_steps; t0 += chunk) {
        const int32_t t1 = std::min(max_steps, t0 + chunk);
        qh_status st = launch_run(ctx, W, a, rb, B.xh0, B.xh1, t0, t1);
        if (st != QH_OK) return st;
        if (checking && t1 < max_steps) {
          st = replica_cuts(B.x, B.running);
          if (st != QH_OK) return st;
          launch_pick_best(s, nb, R, B.cuts, B.best_r, B.best_cut, B.running);
          launch_trace_check(s, nb, B.best_cut, B.running, t1, B.steps_b,
                             B.trace + (size_t)(t1 / o->check_every - 1) * nb);
          if (track)
            launch_track_check(s, W, R, B.signs, B.best_cut, B.best_r, B.running, t1, B.steps_b,
                               B.kept_cut, B.kept_r, B.kept_flag, B.kept_spins);
          if (early)
            launch_early_stop(s, nb, B.best_cut, B.seen, B.stall, B.running, B.steps_run,
                              o->patience, t1, B.steps_b);
        }
      }
    } else {
      QH_CUDA_TRY(cudaGraphLaunch(ctx->loop_exec, s));
      note_launch(ctx->loop_kernels);
    }
    QH_CUDA_TRY(cudaEventRecord(ctx->ev[3], s));
    {
      qh_status st = replica_cuts(x_final, B.active);
      if (st != QH_OK) return st;
    }
    launch_pick_best(s, nb, R, B.cuts, B.best_r, B.best_cut, B.active);
    launch_extract_spins(s, W, R, B.signs, B.best_r, B.spins, B.active);
    if (track)  // the best result during the run, unless the final one is strictly better
      launch_track_final(s, W, B.best_cut, B.best_r, B.active, B.kept_cut, B.kept_r, B.kept_flag,
                         B.kept_spins, B.spins);
    QH_STAGE_CHECK("solve: signs, cut, replica pick");
    if (it == it0)
      QH_CUDA_TRY(cudaMemcpyAsync(sol.cuts_first.data(), B.cuts, (size_t)nb * R * 8, cudaMemcpyDeviceToHost, s));
    if (it == it0 && B.trace) {
      sol.check_every = o->check_every;
      sol.check_trace.assign((size_t)n_checks * nb, 0.0);
      QH_CUDA_TRY(cudaMemcpyAsync(sol.check_trace.data(), B.trace, (size_t)n_checks * nb * 8,
                                  cudaMemcpyDeviceToHost, s));
    }
    QH_CUDA_TRY(cudaMemcpyAsync(h_steps_run.data(), B.steps_run, nb * 4, cudaMemcpyDeviceToHost, s));
    if (it == it0 || !snp) {
      QH_CUDA_TRY(cudaMemcpyAsync(sol.best_r.data(), B.best_r, nb * 4, cudaMemcpyDeviceToHost, s));
      QH_CUDA_TRY(cudaMemcpyAsync(sol.best_cut.data(), B.best_cut, nb * 8, cudaMemcpyDeviceToHost, s));
    }
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    {
      qh_status st = check_err_word(ctx);
      if (st != QH_OK) return st;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    step_ms_total += ms;
    launches += fused ? (int64_t)rb.waves.size()
                : multistep ? (int64_t)rb.waves.size() *
                                  (checking ? (max_steps + o->check_every - 1) / o->check_every : 1)
                            : max_steps;
    for (int32_t b = 0; b < nb; ++b)
      if (h_active[b]) {
        spin_updates += (double)G.h_block_size[b] * R * h_steps_run[b];
        if (it == it0 || !snp) sol.steps_run[b] = h_steps_run[b];
      }
    if (!snp) break;
    // ---- SNP refinement: termination test, flip counter, sign inversion
    launch_refine_prepare(s, W, B.spins, B.best_cut, B.active, B.C, B.deform, B.tries,
                          (float)o->deform_h, o->deform_tries);
    QH_STAGE_CHECK("solve: refinement test");
    QH_CUDA_TRY(cudaMemcpyAsync(h_active.data(), B.active, nb * 4, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t n_active = 0;
    for (int32_t b = 0; b < nb; ++b) n_active += h_active[b] != 0;
    if (n_active == 0 || it + 1 == refine_max) break;
    launch_gauge(s, W, B.spins, W.w, B.active, B.deform, B.gauge);
    {
      qh_status st = retile(ctx, &W, W.w, W.tile_bf16, W.tile_f32, W.csr_mode ? W.pval : nullptr);
      if (st == QH_OK && band_on) st = reband(ctx, &W, W.w, W.band, W.rval);
      if (st == QH_OK && fp8) st = convert_fp8_tiles();
      if (st != QH_OK) return st;
    }
    launch_block_sums(s, W, W.w, sum_w_work, (double*)ctx->scratch(nb * 8, S_SUMJ2),
                      (double*)ctx->scratch((size_t)std::max(G.n_nodes, 1) * 16, S_NODETMP));
  }
  // ---- the refinement state after the last solve, for a call that continues the loop:
  // the gauge the next solve would start from applies the last partition to the blocks
  // that go on refining without a deformed re-solve (as launch_gauge would)
  if (snp) {
    const size_t nn = (size_t)std::max(G.n_nodes, 1);
    std::vector<int8_t> hg(nn, 1), hs(nn, 0);
    std::vector<int32_t> ha(nb, 0), ht(nb, 0), hb(nn, -1);
    std::vector<float> hd(nb, 0.f);
    if (G.n_nodes) {
      QH_CUDA_TRY(cudaMemcpyAsync(hg.data(), B.gauge, G.n_nodes, cudaMemcpyDeviceToHost, s));
      QH_CUDA_TRY(cudaMemcpyAsync(hs.data(), B.spins, G.n_nodes, cudaMemcpyDeviceToHost, s));
      QH_CUDA_TRY(cudaMemcpyAsync(hb.data(), G.block_of, (size_t)G.n_nodes * 4,
                                  cudaMemcpyDeviceToHost, s));
    }
    QH_CUDA_TRY(cudaMemcpyAsync(ha.data(), B.active, nb * 4, cudaMemcpyDeviceToHost, s));
    if (B.deform) {
      QH_CUDA_TRY(cudaMemcpyAsync(hd.data(), B.deform, nb * 4, cudaMemcpyDeviceToHost, s));
      QH_CUDA_TRY(cudaMemcpyAsync(ht.data(), B.tries, nb * 4, cudaMemcpyDeviceToHost, s));
    }
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t b = 0; b < nb; ++b) ha[b] = ha[b] && sel_mask[b] ? 1 : 0;
    sol.refine_gauge.assign(G.n_nodes, 1);
    for (int32_t v = 0; v < G.n_nodes; ++v) {
      const int32_t b = hb[v];
      const bool flip = b >= 0 && ha[b] && hd[b] == 0.f && hs[v] < 0;
      sol.refine_gauge[v] = (int8_t)(flip ? -hg[v] : hg[v]);
    }
    sol.refine_done = it_last + 1;
    sol.refining = ha;
    sol.refine_deform = hd;
    sol.refine_tries = ht;
  }
  // ---- final spins and cut on the original graph
  if (snp) {
    // partition from the flip-count parity: +1 where C is even
    std::vector<int32_t> hC(G.n_nodes);
    std::vector<int32_t> blk(G.n_nodes);
    if (G.n_nodes) {
      QH_CUDA_TRY(cudaMemcpyAsync(hC.data(), B.C, G.n_nodes * 4, cudaMemcpyDeviceToHost, s));
      QH_CUDA_TRY(cudaMemcpyAsync(blk.data(), G.block_of, G.n_nodes * 4, cudaMemcpyDeviceToHost, s));
    }
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    // vertices of blocks left out of a partial solve: spin 0, flip count -1 (unphased)
    for (int32_t v = 0; v < G.n_nodes; ++v) {
      const bool on = blk[v] >= 0 && sel_mask[blk[v]];
      sol.C[v] = on ? hC[v] : -1;
      sol.spins[v] = on ? ((hC[v] % 2 == 0) ? 1 : -1) : 0;
    }
    // cut of the parity partition on the ungauged weights (one pseudo-replica)
    int8_t* st1 = (int8_t*)ctx->scratch((size_t)std::max(G.n_pad, 1) + 16, S_SIGNS1);
    double* nv1 = (double*)ctx->scratch((size_t)std::max(G.n_pad, 1) * 8, S_NODEVAL1);
    double* cut1 = (double*)ctx->scratch((size_t)nb * 8, S_CUT1);
    int32_t* pidx = (int32_t*)ctx->scratch((size_t)std::max(G.n_nodes, 1) * 4, S_DBG0);
    if (!st1 || !nv1 || !cut1 || !pidx) {
      return set_err(ctx, QH_ENOMEM, "allocation failed (final cut)");
    }
    std::vector<int32_t> hp(G.n_nodes);
    if (G.n_nodes)
      QH_CUDA_TRY(cudaMemcpyAsync(hp.data(), G.pad_index, G.n_nodes * 4, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int8_t> hs(std::max(G.n_pad, 1), 1);
    for (int32_t v = 0; v < G.n_nodes; ++v)
      if (hp[v] >= 0 && sol.spins[v] != 0) hs[hp[v]] = sol.spins[v];
    QH_CUDA_TRY(cudaMemcpyAsync(st1, hs.data(), G.n_pad, cudaMemcpyHostToDevice, s));
    launch_cut(s, G, 1, st1, G.w, G.sum_w, nv1, cut1, nullptr);
    QH_STAGE_CHECK("solve: final parity cut");
    QH_CUDA_TRY(cudaMemcpyAsync(sol.best_cut.data(), cut1, nb * 8, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t b = 0; b < nb; ++b)
      if (!sel_mask[b]) sol.best_cut[b] = 0.0;
  } else {
    if (G.n_nodes)
      QH_CUDA_TRY(cudaMemcpyAsync(sol.spins.data(), B.spins, G.n_nodes, cudaMemcpyDeviceToHost, s));
  }
  QH_CUDA_TRY(cudaEventRecord(ctx->ev[1], s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  // device copies of the spins / counts for qh_phase
  sol.d_spins = (int8_t*)nullptr;
  {
    sol.mem = ctx->mem;
    sol.d_spins = (int8_t*)pool_alloc(sol.mem, std::max(G.n_nodes, 1), &sol.allocs);
    sol.d_C = (int32_t*)pool_alloc(sol.mem, (size_t)std::max(G.n_nodes, 1) * 4, &sol.allocs);
    if (!sol.d_spins || !sol.d_C) {
      return set_err(ctx, QH_ENOMEM, "allocation failed (solution)");
    }
    if (G.n_nodes) {
      QH_CUDA_TRY(cudaMemcpyAsync(sol.d_spins, sol.spins.data(), G.n_nodes, cudaMemcpyHostToDevice, s));
      if (snp)
        QH_CUDA_TRY(cudaMemcpyAsync(sol.d_C, sol.C.data(), G.n_nodes * 4, cudaMemcpyHostToDevice, s));
      else
        QH_CUDA_TRY(cudaMemcpyAsync(sol.d_C, B.C, G.n_nodes * 4, cudaMemcpyDeviceToDevice, s));
    }
    QH_CUDA_TRY(cudaStreamSynchronize(s));
  }
  sol.perm.assign(G.h_block_ptr[nb], 0);
  if (!sol.perm.empty()) {
    QH_CUDA_TRY(cudaMemcpyAsync(sol.perm.data(), G.perm, sol.perm.size() * 4, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
  }
  float total = 0.f;
  cudaEventElapsedTime(&total, ctx->ev[0], ctx->ev[1]);
  sol.solve_ms = total;
  sol.step_ms = step_ms_total;
  sol.n_step_launches = launches;
  sol.spin_updates = spin_updates;
  *out = sh;
  sh = nullptr;
  return QH_OK;
}

qh_status qh_bsb_solve(qh_ctx* h, const qh_graph* gh, const qh_bsb_opts* o, qh_solution** out) {
  return solve_impl(h, gh, o, nullptr, -1, out);
}

qh_status qh_bsb_solve_resume(qh_ctx* h, const qh_graph* gh, const qh_bsb_opts* o,
                              const qh_refine_state* state, qh_solution** out) {
  if (h && !state) return set_err(&h->c, QH_EINVAL, "NULL refinement state");
  return solve_impl(h, gh, o, nullptr, -1, out, state);
}

qh_status qh_solution_check_trace(const qh_solution* sh, int32_t* n_checks, int32_t* check_every,
                                  double* trace) {
  if (!sh || !n_checks) return QH_EINVAL;
  const Solution& s = sh->s;
  const int32_t nb = std::max(s.n_blocks, 1);
  *n_checks = (int32_t)(s.check_trace.size() / (size_t)nb);
  if (check_every) *check_every = s.check_every;
  if (trace && !s.check_trace.empty())
    memcpy(trace, s.check_trace.data(), s.check_trace.size() * sizeof(double));
  return QH_OK;
}

qh_status qh_solution_refine_state(const qh_solution* sh, qh_refine_state* st) {
  if (!sh || !st || !st->flips || !st->gauge || !st->refining || !st->solves || !st->deform ||
      !st->tries)
    return QH_EINVAL;
  const Solution& s = sh->s;
  if (s.mode != QH_MODE_SNP || s.refine_done < 1 ||
      (int32_t)s.refine_gauge.size() != s.n_nodes)
    return QH_EINVAL;
  st->iterations_done = s.refine_done;
  for (int32_t v = 0; v < s.n_nodes; ++v) {
    st->flips[v] = s.C[v];
    st->gauge[v] = s.refine_gauge[v];
  }
  for (int32_t b = 0; b < s.n_blocks; ++b) {
    st->refining[b] = s.refining[b];
    st->solves[b] = s.iters[b];
    st->deform[b] = s.refine_deform[b];
    st->tries[b] = s.refine_tries[b];
  }
  return QH_OK;
}

qh_status qh_bsb_solve_blocks(qh_ctx* h, const qh_graph* gh, const qh_bsb_opts* o,
                              const int32_t* blocks, int32_t n_blocks, qh_solution** out) {
  if (h && !blocks && n_blocks > 0) return set_err(&h->c, QH_EINVAL, "NULL block list");
  static const int32_t none = 0;
  return solve_impl(h, gh, o, blocks ? blocks : &none, blocks ? n_blocks : 0, out);
}

qh_status qh_solution_set_block(qh_ctx* h, qh_solution* sh, int32_t b, const int8_t* spins,
                                double best_cut, int32_t best_replica, int32_t steps_run,
                                int32_t iterations) {
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  if (!sh || !spins) return set_err(ctx, QH_EINVAL, "NULL argument");
  Solution& s = sh->s;
  if (b < 0 || b >= s.n_blocks) return set_err(ctx, QH_EINVAL, "block out of range");
  if (best_replica < 0 || steps_run < 0 || iterations < 1 || !std::isfinite(best_cut))
    return set_err(ctx, QH_EINVAL, "best_replica, steps_run >= 0, iterations >= 1, finite cut");
  const int64_t k0 = s.block_ptr[b], k1 = s.block_ptr[b + 1];
  for (int64_t k = k0; k < k1; ++k)
    if (spins[k - k0] != 1 && spins[k - k0] != -1) return set_err(ctx, QH_EINVAL, "spins must be +1 or -1");
  for (int64_t k = k0; k < k1; ++k) {
    const int32_t v = s.perm[k];
    s.spins[v] = spins[k - k0];
    // SNP mode: the parity partition, +1 where the flip count is even
    s.C[v] = spins[k - k0] > 0 ? 0 : 1;
  }
  s.best_cut[b] = best_cut;
  s.best_r[b] = best_replica - s.replica_base;
  s.steps_run[b] = steps_run;
  s.iters[b] = iterations;
  for (int32_t r = 0; r < s.R; ++r) s.cuts_first[(size_t)b * s.R + r] = 0.0;
  s.solved[b] = 1;
  s.device_stale = true;
  s.refine_done = 0;  // an imported block carries no refinement state
  return QH_OK;
}

qh_status qh_solution_block(qh_ctx* h, const qh_solution* sh, int32_t b, int8_t* spins,
                            double* best_cut, int32_t* best_replica, int32_t* steps_run,
                            int32_t* iterations) {
  if (!h || !sh) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Solution& s = sh->s;
  if (b < 0 || b >= s.n_blocks) return set_err(ctx, QH_EINVAL, "block out of range");
  if (spins)
    for (int64_t k = s.block_ptr[b]; k < s.block_ptr[b + 1]; ++k)
      spins[k - s.block_ptr[b]] = s.spins[s.perm[k]];
  if (best_cut) *best_cut = s.best_cut[b];
  if (best_replica) *best_replica = s.solved[b] ? s.replica_base + s.best_r[b] : -1;
  if (steps_run) *steps_run = s.steps_run[b];
  if (iterations) *iterations = s.iters[b];
  return QH_OK;
}

qh_status qh_solution_spins(qh_ctx* h, const qh_solution* sh, int8_t* spins) {
  if (!h || !sh || !spins) return QH_EINVAL;
  const Solution& s = sh->s;
  if (s.n_nodes) memcpy(spins, s.spins.data(), s.n_nodes);
  return QH_OK;
}

qh_status qh_solution_cuts(qh_ctx* h, const qh_solution* sh, double* cuts) {
  if (!h || !sh || !cuts) return QH_EINVAL;
  const Solution& s = sh->s;
  memcpy(cuts, s.cuts_first.data(), s.cuts_first.size() * sizeof(double));
  return QH_OK;
}

qh_status qh_solution_timing(const qh_solution* sh, double* solve_ms, double* step_ms,
                             int64_t* n_step_launches, double* spin_updates) {
  if (!sh) return QH_EINVAL;
  const Solution& s = sh->s;
  if (solve_ms) *solve_ms = s.solve_ms;
  if (step_ms) *step_ms = s.step_ms;
  if (n_step_launches) *n_step_launches = s.n_step_launches;
  if (spin_updates) *spin_updates = s.spin_updates;
  return QH_OK;
}

const char* qh_solution_kernel(const qh_solution* sh) { return sh ? sh->s.kernel.c_str() : ""; }

int64_t qh_kernel_launches(void) { return launches(); }

const char* qh_tuning_report(const qh_ctx* h) { return h ? h->c.tune_report.c_str() : ""; }

void qh_solution_free(qh_solution* sh) {
  if (!sh) return;
  pool_free_all(sh->s.mem, &sh->s.allocs);
  delete sh;
}

qh_status qh_phase(qh_ctx* h, const qh_graph* gh, const qh_solution* sh, int8_t* hap1, int8_t* hap2,
                   int32_t* block_id, int32_t on_device) {
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  NvtxRange nvtx_range("qh_phase");
  ctx->err.clear();
  clear_foreign_error(ctx);
  if (!gh || !sh || !hap1 || !hap2 || !block_id) return set_err(ctx, QH_EINVAL, "NULL argument");
  const Graph& g = gh->g;
  const Solution& sol = sh->s;
  if (sol.n_nodes != g.n_nodes || sol.mode != g.mode)
    return set_err(ctx, QH_EINVAL, "solution does not belong to this graph");
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  if (sol.device_stale && g.n_nodes) {  // blocks imported by qh_solution_set_block
    QH_CUDA_TRY(cudaMemcpyAsync(sol.d_spins, sol.spins.data(), g.n_nodes, cudaMemcpyHostToDevice, s));
    QH_CUDA_TRY(cudaMemcpyAsync(sol.d_C, sol.C.data(), (size_t)g.n_nodes * 4, cudaMemcpyHostToDevice, s));
    QH_CUDA_TRY(cudaStreamSynchronize(s));
    sol.device_stale = false;
  }
  const int32_t n = g.n_snps;
  int8_t *d1 = hap1, *d2 = hap2;
  int32_t* db = block_id;
  if (!on_device) {
    d1 = (int8_t*)ctx->scratch(std::max(n, 1), S_DBG0);
    d2 = (int8_t*)ctx->scratch(std::max(n, 1), S_DBG1);
    db = (int32_t*)ctx->scratch((size_t)std::max(n, 1) * 4, S_DBG2);
    if (!d1 || !d2 || !db) return set_err(ctx, QH_ENOMEM, "allocation failed (phase)");
  }
  if (g.mode == QH_MODE_READ)
    launch_vote(s, g, sol.d_spins, d1, d2, db);
  else
    launch_parity(s, g, sol.d_C, d1, d2, db);
  QH_CUDA_TRY(cudaGetLastError());
  if (!on_device && n > 0) {
    QH_CUDA_TRY(cudaMemcpyAsync(hap1, d1, n, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaMemcpyAsync(hap2, d2, n, cudaMemcpyDeviceToHost, s));
    QH_CUDA_TRY(cudaMemcpyAsync(block_id, db, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  }
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  return QH_OK;
}

// ------------------------------------------------------------------ test hooks
qh_status qh_debug_wait_timeout(qh_ctx* h, int32_t which) {
  if (!h || which < 0 || which > 1) return QH_EINVAL;
  Ctx* ctx = &h->c;
  cudaSetDevice(ctx->device);
  clear_foreign_error(ctx);
  qh_status st = launch_wait_probe(ctx, which);
  if (st != QH_OK) return st;
  return check_err_word(ctx);
}

qh_status qh_debug_fail_alloc(qh_ctx* h, int64_t after) {
  if (!h || after < -1 || !h->c.mem.fail_after) return QH_EINVAL;
  *h->c.mem.fail_after = after;
  return QH_OK;
}

qh_status qh_debug_init_state(qh_ctx* h, const qh_graph* gh, int32_t R, int32_t replica_base,
                              uint64_t seed, int32_t iter, float* x, float* y) {
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  clear_foreign_error(ctx);
  if (!gh || !x || !y) return set_err(ctx, QH_EINVAL, "NULL argument");
  if (R < 1 || replica_base < 0 || (int64_t)replica_base + R > (1 << 16) || iter < 0)
    return set_err(ctx, QH_EINVAL, "R >= 1, iter >= 0 and replica indices below 65536 required");
  const Graph& g = gh->g;
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  const size_t NS = (size_t)R * g.n_pad;
  if (NS == 0) return QH_OK;
  if (g.csr_mode) {  // the solver's vertex-major layout, transposed to [R][n_pad]
    float* xt = (float*)ctx->scratch(NS * 4, S_TR0);
    float* yt = (float*)ctx->scratch(NS * 4, S_TR1);
    if (!xt || !yt) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    launch_init_state(s, g, R, replica_base, seed, iter, xt, yt, nullptr, nullptr);
    launch_transpose(s, xt, x, g.n_pad, R);
    launch_transpose(s, yt, y, g.n_pad, R);
  } else {
    launch_init_state(s, g, R, replica_base, seed, iter, x, y, nullptr, nullptr);
  }
  QH_STAGE_CHECK("debug: state init");
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  return QH_OK;
}

qh_status qh_debug_layout(qh_ctx* h, const qh_graph* gh, int32_t* n_pad, int32_t* padded_index,
                          double* c0_default) {
  if (!h || !gh) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Graph& g = gh->g;
  if (n_pad) *n_pad = g.n_pad;
  if (padded_index && g.n_nodes) {
    QH_CUDA_TRY(cudaMemcpyAsync(padded_index, g.pad_index, g.n_nodes * 4, cudaMemcpyDeviceToHost, ctx->stream));
    QH_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  if (c0_default)
    for (int32_t b = 0; b < g.n_blocks; ++b) c0_default[b] = g.h_c0[b];
  return QH_OK;
}

static qh_status debug_fp8_tiles(Ctx* ctx, const Graph& g, Fp8Operands* f8, float* scale) {
  const int64_t n = g.n_tiles_hi * (int64_t)TILE * TILE;
  uint8_t* jh = (uint8_t*)ctx->scratch(std::max<int64_t>(n, 1), S_F8H);
  uint8_t* jl = (uint8_t*)ctx->scratch(std::max<int64_t>(n, 1), S_F8L);
  int32_t* flag = (int32_t*)ctx->scratch(16, S_F8FLAG);
  if (!jh || !jl || !flag) return set_err(ctx, QH_ENOMEM, "allocation failed (FP8 tiles)");
  *scale = fp8_scale(g);
  QH_CUDA_TRY(cudaMemsetAsync(flag, 0, 4, ctx->stream));
  launch_tiles_to_e4m3(ctx->stream, g.tile_f32, n, *scale, jh, jl, flag);
  int32_t hl = 0;
  QH_CUDA_TRY(cudaMemcpyAsync(&hl, flag, 4, cudaMemcpyDeviceToHost, ctx->stream));
  QH_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  f8->jh = jh;
  f8->jl = jl;
  f8->n_slices = hl ? 3 : 2;
  return QH_OK;
}

static qh_status debug_common(Ctx* ctx, const Graph& g, int precision, int32_t R, StepArgs& a,
                              const double* c0_per_block, int32_t steps,
                              std::vector<float>* c0_out = nullptr) {
  if (precision != QH_PREC_FP32 && !is_tc_precision(precision) && precision != QH_PREC_FP8)
    return set_err(ctx, QH_EINVAL, "bad precision");
  if (precision == QH_PREC_FP8 && (g.csr_mode || R % 64 != 0))
    return set_err(ctx, QH_EINVAL, "FP8 needs tile storage and R a multiple of 64");
  if (R < 1) return set_err(ctx, QH_EINVAL, "R must be >= 1");
  if (is_tc_precision(precision) && !g.csr_mode && !tc_plan_ok(R, pick_plan(R)))
    return set_err(ctx, QH_EINVAL, "BF16 precision needs R to be a multiple of 64");
  const int32_t nb = std::max(g.n_blocks, 1);
  std::vector<float> c0(nb);
  std::vector<int32_t> sb(nb, steps);
  for (int32_t b = 0; b < g.n_blocks; ++b) c0[b] = (float)(c0_per_block ? c0_per_block[b] : g.h_c0[b]);
  float* dc0 = (float*)ctx->scratch(nb * 4, S_C0);
  int32_t* dsb = (int32_t*)ctx->scratch(nb * 4, S_STEPSB);
  if (!dc0 || !dsb) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
  QH_CUDA_TRY(cudaMemcpyAsync(dc0, c0.data(), nb * 4, cudaMemcpyHostToDevice, ctx->stream));
  QH_CUDA_TRY(cudaMemcpyAsync(dsb, sb.data(), nb * 4, cudaMemcpyHostToDevice, ctx->stream));
  QH_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
  a = StepArgs{};
  a.rt = g.rt;
  a.tile_col = g.tile_col;
  a.tile_f32 = g.tile_f32;
  a.c0 = dc0;
  a.active = nullptr;
  a.steps_b = dsb;
  a.n_pad = g.n_pad;
  a.R = R;
  a.err = ctx->d_err;
  a.use_lo = use_lo_for(g, precision);
  if (c0_out) *c0_out = c0;
  return QH_OK;
}

qh_status qh_debug_run_trace(qh_ctx* h, const qh_graph* gh, int32_t R, int32_t step_kernel,
                             int32_t steps, int32_t u0, int32_t nu, uint64_t* stamps,
                             int32_t* items, int32_t* n_ctas) {
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  clear_foreign_error(ctx);
  if (!gh || !n_ctas) return set_err(ctx, QH_EINVAL, "NULL argument");
  const Graph& g = gh->g;
  if (steps < 1 || u0 < 0 || nu < 1 || u0 + nu > steps)
    return set_err(ctx, QH_EINVAL, "steps >= 1 and 0 <= u0 < u0 + nu <= steps required");
  const bool use_lo = use_lo_for(g, QH_PREC_BF16) != 0;
  if (!run_variant(step_kernel) || !tc_variant_ok(step_kernel, g, R, ctx->n_sm, use_lo))
    return set_err(ctx, QH_EINVAL, "step_kernel must be a multi-step variant valid for this graph");
  RunPlan plan;
  if (!run_plan(g, R, ctx->n_sm, step_kernel, use_lo, &plan) || plan.waves.size() != 1)
    return set_err(ctx, QH_EINVAL, "the traced launch must be a single wave");
  const RunWave& w = plan.waves[0];
  *n_ctas = w.grid;
  if (!stamps) return QH_OK;
  const int EV = run_trace_events(), MI = run_max_items();
  constexpr int SLOTS = 4, COLS = 32;  // item slots per CTA, stamps per slot in the caller's arrays
  if (2 * EV > COLS) return set_err(ctx, QH_EUNSUPPORTED, "more trace events than the layout holds");
  if (MI > SLOTS) return set_err(ctx, QH_EUNSUPPORTED, "more item slots than the trace layout holds");
  if (items)
    for (int c = 0; c < w.grid; ++c) {
      const int2 wk = plan.work[w.work_off + c];
      for (int j = 0; j < SLOTS; ++j)
        items[c * SLOTS + j] =
            j < std::min(wk.y, MI) ? plan.items[w.item_off + wk.x + j * w.stride] & run_item_mask()
                                   : -1;
    }
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  StepArgs a;
  qh_status st = debug_common(ctx, g, QH_PREC_BF16, R, a, nullptr, steps);
  if (st) return st;
  const size_t NS = (size_t)R * g.n_pad;
  const size_t n_stamps = (size_t)w.grid * nu * MI * 2 * EV;
  float* x = (float*)ctx->scratch(NS * 4, S_X);
  float* y = (float*)ctx->scratch(NS * 4, S_Y);
  __nv_bfloat16* xh0 = (__nv_bfloat16*)ctx->scratch(NS * 2, S_XH0);
  __nv_bfloat16* xh1 = (__nv_bfloat16*)ctx->scratch(NS * 2, S_XH1);
  unsigned long long* tr = (unsigned long long*)ctx->scratch(n_stamps * 8, S_TRACE);
  if (!x || !y || !xh0 || !xh1 || !tr) return set_err(ctx, QH_ENOMEM, "allocation failed (trace)");
  std::vector<float> c0h(std::max(g.n_blocks, 1));
  for (int32_t b = 0; b < g.n_blocks; ++b) c0h[b] = (float)g.h_c0[b];
  if (!run_c0_ok(c0h.data(), g.n_blocks, 1.f))
    return set_err(ctx, QH_EINVAL, "multi-step kernel needs dt * c0 to be a normal float in every block");
  a.x = x;
  a.y = y;
  a.dt = 1.f;
  a.a0 = 1.0;
  a.dta0 = 1.f;
  a.sb = QH_SB_BALLISTIC;
  QH_CUDA_TRY(cudaMemsetAsync(xh1, 0, NS * 2, s));
  QH_CUDA_TRY(cudaMemsetAsync(tr, 0, n_stamps * 8, s));
  launch_init_state(s, g, R, 0, 1, 0, x, y, xh0, nullptr);
  RunBufs rb;
  st = run_prepare(ctx, g, R, step_kernel, use_lo, &rb);
  if (st) return st;
  st = launch_run(ctx, g, a, rb, xh0, xh1, 0, steps, tr, u0, nu);
  if (st) return st;
  QH_STAGE_CHECK("debug: traced multi-step launch");
  std::vector<unsigned long long> hs(n_stamps);
  QH_CUDA_TRY(cudaMemcpyAsync(hs.data(), tr, n_stamps * 8, cudaMemcpyDeviceToHost, s));
  QH_CUDA_TRY(cudaStreamSynchronize(s));
  // [cta][step][MI][EV global, EV clock] -> [cta][step][SLOTS][16 global, 16 clock]
  memset(stamps, 0, (size_t)w.grid * nu * SLOTS * COLS * 8);
  for (size_t cs = 0; cs < (size_t)w.grid * nu; ++cs)
    for (int j = 0; j < MI; ++j)
      for (int e = 0; e < EV; ++e) {
        stamps[(cs * SLOTS + j) * COLS + e] = hs[(cs * MI + j) * 2 * EV + e];
        stamps[(cs * SLOTS + j) * COLS + COLS / 2 + e] = hs[(cs * MI + j) * 2 * EV + EV + e];
      }
  return check_err_word(ctx);
}

qh_status qh_debug_matvec(qh_ctx* h, const qh_graph* gh, int32_t precision, int32_t R, const float* x,
                          float* z) {
  if (!h || !gh || !x || !z) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Graph& g = gh->g;
  cudaSetDevice(ctx->device);
  StepArgs a;
  qh_status st = debug_common(ctx, g, precision, R, a, nullptr, 1 << 30);
  if (st) return st;
  a.z_out = z;
  a.t = 0;
  a.a0 = 1.0;
  QH_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)R * g.n_pad * 4, ctx->stream));
  if (g.csr_mode) {  // API layout [R][n_pad] <-> solver layout [n_pad][R]
    if (R % 4 != 0) return set_err(ctx, QH_EINVAL, "CSR storage needs R to be a multiple of 4");
    const size_t NS = (size_t)R * g.n_pad;
    float* xt = (float*)ctx->scratch(NS * 4, S_TR0);
    float* zt = (float*)ctx->scratch(NS * 4, S_TR1);
    __nv_bfloat16* xh = (__nv_bfloat16*)ctx->scratch(NS * 2, S_XH0);
    if (!xt || !zt || !xh) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    QH_CUDA_TRY(cudaMemsetAsync(zt, 0, NS * 4, ctx->stream));
    launch_transpose(ctx->stream, x, xt, R, g.n_pad);
    a.z_out = zt;
    const int cv = csr_default_variant(g, precision, R);
    if (precision == QH_PREC_FP32) {
      a.xin = xt;
      launch_step_csr(ctx->stream, g, a, g.pval, nullptr, cv);
    } else if (cv == CSR_BAND8) {  // band product on the tensor cores + the remainder
      launch_f32_to_bf16(ctx->stream, xt, xh, (int64_t)NS);
      float* zb = (float*)ctx->scratch(NS * 4, S_ZBAND);
      if (!zb) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
      st = launch_band_mma(ctx, g, a, g.band, xh, zb);
      if (st) return st;
      a.zb = zb;
      launch_step_csr(ctx->stream, g, a, g.rval, xh, cv, true);
    } else {
      launch_f32_to_bf16(ctx->stream, xt, xh, (int64_t)NS);
      launch_step_csr(ctx->stream, g, a, g.pval, xh, cv);
    }
    launch_transpose(ctx->stream, zt, z, g.n_pad, R);
    QH_CUDA_TRY(cudaGetLastError());
    return check_err_word(ctx);
  }
  if (precision == QH_PREC_FP8) {
    Fp8Operands f8{};
    float sc8 = 1.f;
    st = debug_fp8_tiles(ctx, g, &f8, &sc8);
    if (st) return st;
    const int64_t NS = (int64_t)R * g.n_pad;
    uint8_t* x8 = (uint8_t*)ctx->scratch((size_t)NS * 2, S_X8);
    if (!x8) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    launch_x_to_e4m3(ctx->stream, x, NS, x8, x8 + NS);
    f8.xh_in = x8;
    f8.xl_in = x8 + NS;
    a.inv_scale = 1.f / sc8;
    st = launch_step_f8(ctx, g, a, f8);
    if (st) return st;
  } else if (precision == QH_PREC_FP32) {
    a.xin = x;
    a.xout = nullptr;
    launch_step_f32(ctx->stream, g, a);
  } else {
    __nv_bfloat16* xh = (__nv_bfloat16*)ctx->scratch((size_t)R * g.n_pad * 2, S_XH0);
    if (!xh) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    launch_f32_to_bf16(ctx->stream, x, xh, (int64_t)R * g.n_pad);
    st = launch_step_tc(ctx, g, a, xh, pick_plan(R));
    if (st) return st;
  }
  QH_CUDA_TRY(cudaGetLastError());
  return check_err_word(ctx);
}

qh_status qh_debug_steps(qh_ctx* h, const qh_graph* gh, int32_t precision, int32_t R, float* x,
                         float* y, int32_t t0, int32_t nsteps, int32_t steps, double dt, double a0,
                         const double* c0_per_block) {
  return qh_debug_steps_v(h, gh, precision, R, x, y, t0, nsteps, steps, dt, a0, c0_per_block, -1,
                          QH_SB_BALLISTIC, nullptr);
}

qh_status qh_debug_steps_v(qh_ctx* h, const qh_graph* gh, int32_t precision, int32_t R, float* x,
                           float* y, int32_t t0, int32_t nsteps, int32_t steps, double dt,
                           double a0, const double* c0_per_block, int32_t step_kernel,
                           int32_t sb_variant, const double* field_per_block) {
  if (!h || !gh || !x || !y || nsteps < 0 || steps < 1 || t0 < 0) return QH_EINVAL;
  if (sb_variant < QH_SB_BALLISTIC || sb_variant > QH_SB_ADIABATIC) return QH_EINVAL;
  Ctx* ctx = &h->c;
  const Graph& g = gh->g;
  cudaSetDevice(ctx->device);
  StepArgs a;
  std::vector<float> c0h;
  qh_status st = debug_common(ctx, g, precision, R, a, c0_per_block, steps, &c0h);
  if (st) return st;
  a.sb = sb_variant;
  a.deform = nullptr;
  if (field_per_block != nullptr && g.n_blocks > 0) {
    std::vector<float> hf(g.n_blocks);
    for (int32_t b = 0; b < g.n_blocks; ++b) {
      if (!std::isfinite(field_per_block[b]))
        return set_err(ctx, QH_EINVAL, "deformation field strengths must be finite");
      hf[b] = (float)field_per_block[b];
    }
    float* d = (float*)ctx->scratch((size_t)g.n_blocks * 4, S_DBGDEF);
    if (!d) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    QH_CUDA_TRY(cudaMemcpy(d, hf.data(), (size_t)g.n_blocks * 4, cudaMemcpyHostToDevice));
    a.deform = d;
  }
  if (step_kernel >= 0 && g.csr_mode) {
    if (!csr_variant_ok(step_kernel, R, precision))
      return set_err(ctx, QH_EINVAL, "step_kernel variant not valid for this graph, precision and R");
  } else if (step_kernel >= 0) {
    if (!is_tc_precision(precision) || g.csr_mode || step_kernel >= tc_n_variants() ||
        !tc_variant_ok(step_kernel, g, R, ctx->n_sm, a.use_lo != 0))
      return set_err(ctx, QH_EINVAL, "step_kernel variant not valid for this graph, precision and R");
    if (run_variant(step_kernel) && !run_c0_ok(c0h.data(), g.n_blocks, (float)dt))
      return set_err(ctx, QH_EINVAL, "multi-step kernel needs dt * c0 to be a normal float in every block");
  }
  a.x = x;
  a.y = y;
  a.dt = (float)dt;
  a.a0 = a0;
  a.dta0 = (float)(dt * a0);
  const size_t NS = (size_t)R * g.n_pad;
  cudaStream_t s = ctx->stream;
  float* xu = x;  // user buffers in [R][n_pad]
  float* yu = y;
  const int csr_v = step_kernel >= 0 ? step_kernel : csr_default_variant(g, precision, R);
  if (g.csr_mode) {
    if (R % 4 != 0) return set_err(ctx, QH_EINVAL, "CSR storage needs R to be a multiple of 4");
    x = (float*)ctx->scratch(NS * 4, S_TR0);
    y = (float*)ctx->scratch(NS * 4, S_TR1);
    if (!x || !y) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    launch_transpose(s, xu, x, R, g.n_pad);
    launch_transpose(s, yu, y, R, g.n_pad);
    a.x = x;
    a.y = y;
  }
  if (precision == QH_PREC_FP32) {
    float* x1 = (float*)ctx->scratch(NS * 4, S_X1);
    if (!x1) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    QH_CUDA_TRY(cudaMemcpyAsync(x1, x, NS * 4, cudaMemcpyDeviceToDevice, s));
    for (int32_t k = 0; k < nsteps; ++k) {
      a.t = t0 + k;
      a.xin = (k % 2 == 0) ? x : x1;
      a.xout = (k % 2 == 0) ? x1 : x;
      if (g.csr_mode)
        launch_step_csr(s, g, a, g.pval, nullptr, csr_v);
      else
        launch_step_f32(s, g, a);
    }
    if (nsteps % 2 == 1) QH_CUDA_TRY(cudaMemcpyAsync(x, x1, NS * 4, cudaMemcpyDeviceToDevice, s));
  } else {
    __nv_bfloat16* xh0 = (__nv_bfloat16*)ctx->scratch(NS * 2, S_XH0);
    __nv_bfloat16* xh1 = (__nv_bfloat16*)ctx->scratch(NS * 2, S_XH1);
    if (!xh0 || !xh1) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
    QH_CUDA_TRY(cudaMemsetAsync(xh1, 0, NS * 2, s));
    if (precision == QH_PREC_FP8) {
      Fp8Operands f8{};
      float sc8 = 1.f;
      st = debug_fp8_tiles(ctx, g, &f8, &sc8);
      if (st) return st;
      a.inv_scale = 1.f / sc8;
      uint8_t* b0 = reinterpret_cast<uint8_t*>(xh0);
      uint8_t* b1 = reinterpret_cast<uint8_t*>(xh1);
      launch_x_operand_e4m3(s, g, sb_variant, x, (int64_t)NS, b0, b0 + NS);
      for (int32_t k = 0; k < nsteps; ++k) {
        a.t = t0 + k;
        uint8_t* cur = (k % 2 == 0) ? b0 : b1;
        uint8_t* nxt = (k % 2 == 0) ? b1 : b0;
        f8.xh_in = cur;
        f8.xl_in = cur + NS;
        a.x8h_out = nxt;
        a.x8l_out = nxt + NS;
        st = launch_step_f8(ctx, g, a, f8);
        if (st) return st;
      }
      QH_CUDA_TRY(cudaGetLastError());
      return check_err_word(ctx);
    }
    if (step_kernel >= 0 && run_variant(step_kernel)) {  // one launch for all nsteps
      RunBufs rb;
      st = run_prepare(ctx, g, R, step_kernel, a.use_lo != 0, &rb);
      if (st) return st;
      if (t0 % 2 == 1) {  // X_hat_t lives in xh0 for even t, xh1 for odd t
        QH_CUDA_TRY(cudaMemsetAsync(xh0, 0, NS * 2, s));
        launch_x_operand(s, g, sb_variant, x, xh1, (int64_t)NS);
      } else {
        launch_x_operand(s, g, sb_variant, x, xh0, (int64_t)NS);
      }
      st = launch_run(ctx, g, a, rb, xh0, xh1, t0, t0 + nsteps);
      if (st) return st;
      QH_CUDA_TRY(cudaGetLastError());
      return check_err_word(ctx);
    }
    TcPlan plan = pick_plan(R);
    if (step_kernel >= 0) plan.variant = step_kernel;
    launch_x_operand(s, g, sb_variant, x, xh0, (int64_t)NS);
    for (int32_t k = 0; k < nsteps; ++k) {
      a.t = t0 + k;
      a.xh_out = (k % 2 == 0) ? xh1 : xh0;
      if (g.csr_mode) {
        const __nv_bfloat16* xc = (k % 2 == 0) ? xh0 : xh1;
        if (csr_v == CSR_BAND8) {
          float* zb = (float*)ctx->scratch(NS * 4, S_ZBAND);
          if (!zb) return set_err(ctx, QH_ENOMEM, "allocation failed (debug)");
          st = launch_band_mma(ctx, g, a, g.band, xc, zb);
          if (st) return st;
          StepArgs ab = a;
          ab.zb = zb;
          launch_step_csr(s, g, ab, g.rval, xc, csr_v, true);
        } else {
          launch_step_csr(s, g, a, g.pval, xc, csr_v);
        }
        continue;
      }
      st = launch_step_tc(ctx, g, a, (k % 2 == 0) ? xh0 : xh1, plan);
      if (st) return st;
    }
  }
  if (g.csr_mode) {
    launch_transpose(s, x, xu, g.n_pad, R);
    launch_transpose(s, y, yu, g.n_pad, R);
  }
  QH_CUDA_TRY(cudaGetLastError());
  return check_err_word(ctx);
}

}  // extern "C"
