// J x X product on the BF16 tensor cores for callers that must not allocate device
// memory: hosts whose own allocator already owns the GPU's memory, or processes held
// to a fixed device-memory budget (see qh_matvec_bf16_noalloc in qhap.h).
//
// The only working memory beyond the caller's input and output is the BF16 copy of
// X and two small per-block parameter arrays.  Instead of coming from cudaMalloc or
// the context's grow-on-demand buffers, they live in the file-scope array below,
// which every GPU that loads this library holds until the process exits.  Its device
// address is looked up once per device and kept for the life of the process, so the
// library must not be used across a cudaDeviceReset of that device.
#include <mutex>

#include "qh_internal.cuh"

namespace qh {

namespace {

// Layout of the static scratch: [BF16 X_hat : NOALLOC_MAX_ELEMS x 2 B]
//                               [per-block steps : NOALLOC_MAX_BLOCKS x 4 B]
//                               [per-block c0    : NOALLOC_MAX_BLOCKS x 4 B]
constexpr int64_t NOALLOC_MAX_ELEMS = int64_t(1) << 22;   // R * n_pad <= 4,194,304
constexpr int64_t NOALLOC_MAX_BLOCKS = int64_t(1) << 16;  // phase blocks <= 65,536
constexpr size_t NOALLOC_XH_BYTES = size_t(NOALLOC_MAX_ELEMS) * 2;
constexpr size_t NOALLOC_BYTES = NOALLOC_XH_BYTES + size_t(NOALLOC_MAX_BLOCKS) * 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (host code cannot use
// the symbol itself: on the host it names a stand-in, not device memory).
qh_status scratch_address(Ctx* ctx, unsigned char** out) {
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return set_err(ctx, QH_EUNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
    g_scratch_addr[ctx->device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[ctx->device]);
  return QH_OK;
}

__global__ void k_fill_block_params(int32_t nb, int32_t* steps_b, float* c0) {
  int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) {
    steps_b[b] = 1 << 30;  // "step 0 of a very long schedule": every block is live
    c0[b] = 0.f;           // unused when the kernel writes Z instead of updating x, y
  }
}

}  // namespace
}  // namespace qh

using namespace qh;

extern "C" qh_status qh_matvec_bf16_noalloc(qh_ctx* h, const qh_graph* gh, int32_t R,
                                            const float* x, float* z) {
  if (!h) return QH_EINVAL;
  Ctx* ctx = &h->c;
  ctx->err.clear();
  if (!gh || !x || !z) return set_err(ctx, QH_EINVAL, "NULL argument");
  const Graph& g = gh->g;
  if (g.csr_mode) return set_err(ctx, QH_EUNSUPPORTED, "the graph is stored as CSR, not as J tiles");
  if (R < 1 || !tc_plan_ok(R, TcPlan{R % 128 == 0 ? 128 : 64, 3}))
    return set_err(ctx, QH_EINVAL, "R must be a positive multiple of 64");
  const int64_t elems = (int64_t)R * g.n_pad;
  if (elems > NOALLOC_MAX_ELEMS)
    return set_err(ctx, QH_EINVAL,
                   "R * n_pad exceeds 4,194,304 elements (the static scratch holds 8 MiB of BF16 X)");
  if ((int64_t)g.n_blocks > NOALLOC_MAX_BLOCKS)
    return set_err(ctx, QH_EINVAL, "more than 65,536 phase blocks");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  unsigned char* base = nullptr;
  qh_status st = scratch_address(ctx, &base);
  if (st != QH_OK) return st;
  __nv_bfloat16* xh = reinterpret_cast<__nv_bfloat16*>(base);
  int32_t* steps_b = reinterpret_cast<int32_t*>(base + NOALLOC_XH_BYTES);
  float* c0 = reinterpret_cast<float*>(base + NOALLOC_XH_BYTES + NOALLOC_MAX_BLOCKS * 4);
  cudaStream_t s = ctx->stream;
  // Z rows outside the blocks are never written by the kernel: start Z at zero
  e = cudaMemsetAsync(z, 0, (size_t)elems * 4, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(z)");
  e = cudaMemsetAsync(ctx->d_err, 0, 4, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(err)");
  if (g.n_blocks > 0)
    k_fill_block_params<<<::qh::counted((g.n_blocks + 255) / 256), 256, 0, s>>>(g.n_blocks, steps_b, c0);
  // X_hat = bf16(x) over the whole R x n_pad extent: nothing of a previous call survives
  launch_f32_to_bf16(s, x, xh, elems);
  StepArgs a{};
  a.rt = g.rt;
  a.tile_col = g.tile_col;
  a.tile_f32 = g.tile_f32;
  a.c0 = c0;
  a.active = nullptr;
  a.steps_b = steps_b;
  a.n_pad = g.n_pad;
  a.R = R;
  a.t = 0;
  a.a0 = 1.0;
  a.z_out = z;
  a.err = ctx->d_err;
  a.use_lo = use_lo_for(g, QH_PREC_BF16);
  st = launch_step_tc(ctx, g, a, xh, TcPlan{R % 128 == 0 ? 128 : 64, 3});
  if (st != QH_OK) return st;
  int32_t herr = 0;
  e = cudaMemcpyAsync(&herr, ctx->d_err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "qh_matvec_bf16_noalloc");
  if (herr & ERR_TIMEOUT) return set_err(ctx, QH_ETIMEOUT, "a bounded device wait expired");
  return QH_OK;
}
