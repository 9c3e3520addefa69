// sfr_solve_noalloc: FR-ADM for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc when they solve: processes whose device memory is
// handed out by a fixed pool or by a framework allocator that must own every byte, and
// latency-critical paths that may not take the allocator's locks or risk its
// fragmentation.  For them this entry point runs the same FR-ADM kernels as sfr_solve,
// but takes every byte of workspace (multiplier buffers, Delta, thin products, reduction
// partials, r x r matrices and the iteration state) from one file-scope __device__ array
// of fixed size, so a call allocates nothing: no cudaMalloc, cudaFree, graph
// instantiation, event or pinned buffer.
//
// The array lives in the module image, so every GPU that loads libsfr holds
// kStaticScratchBytes of it until the process exits.  All calls share it and it keeps the
// previous call's contents; the solve clears what must start at zero.  Calls whose work
// overlaps on the GPU (two host threads, or two contexts on one device) race on it.
// The array's device address is looked up on every call, so a device reset
// (cudaDeviceReset), which reloads the module at a new address, leaves no stale address.
#include <cstring>

#include "sfr_internal.h"

namespace sfr {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  In host code the symbol's name is
// only a host-side stand-in, not a device address, so it is looked up on every call: the lookup
// is a host query, not a stream operation, and a cached address would outlive a device reset
// (the module reloads and the array may move).
cudaError_t scratch_base(void** out) { return cudaGetSymbolAddress(out, g_static_scratch); }

struct NoAllocFail {
  sfr_status code;
  std::string msg;
};

#define NA_CUDA(call)                                                                                          \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) throw NoAllocFail{SFR_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// One FR-ADM iteration (same kernels and order as sfr_solve), launched eagerly.
void iteration(const Shape& s, Buffers& b, bool fp64, bool first, cudaStream_t st) {
  if (first) {
    NA_CUDA(launch_init_p(s, b, fp64, st));
    NA_CUDA(launch_gram_p(s, b, fp64, false, st));
  }
  NA_CUDA(launch_rxr(s, b, false, st));
  NA_CUDA(launch_apply_u(s, b, fp64, first, st));
  const int u_new = 1 - b.u_cur;
  const bool wp = !first && mx_path(s, fp64);  // W = (Delta^T P) T_U + C_old H, as sfr_solve forms it
  NA_CUDA(launch_wpass(s, b, fp64, first, u_new, st, wp));
  NA_CUDA(launch_wfinal(s, b, fp64, first, st, wp));
  NA_CUDA(launch_rxr(s, b, true, st));
  NA_CUDA(launch_apply_v(s, b, fp64, st));
  NA_CUDA(launch_sweep(s, b, fp64, u_new, st));
  NA_CUDA(launch_iter_end(s, b, fp64, st));
  NA_CUDA(launch_gram_p(s, b, fp64, true, st));
  b.u_cur = u_new;
  std::swap(b.Y[0], b.Y[1]);
}

}  // namespace
}  // namespace sfr

using namespace sfr;

extern "C" sfr_status sfr_solve_noalloc(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res) {
  if (!ctx) return SFR_E_INVAL;
  std::string why;
  sfr_status v = validate(prob, res, &why);
  if (v == SFR_OK && prob->nys_l != 0) v = SFR_E_INVAL, why = "sfr_solve_noalloc solves FR-ADM only (nys_l must be 0)";
  if (v == SFR_OK && prob->mem != SFR_MEM_DEVICE) v = SFR_E_INVAL, why = "sfr_solve_noalloc needs device buffers";
  if (v != SFR_OK) {
    ctx_set_error(ctx, why);
    if (res) res->status = v;
    return v;
  }
  const sfr_problem& p = *prob;
  const bool fp64 = p.precision == SFR_PREC_FP64;
  const int device = ctx_device(ctx);
  cudaStream_t st = ctx_stream(ctx);
  try {
    NA_CUDA(cudaSetDevice(device));
    const Shape s = plan_shape(p.m, p.n, p.ldm, p.r, ctx_num_sms(ctx));
    const size_t need = carve(s, fp64, nullptr, nullptr);
    if (need > kStaticScratchBytes) {
      char buf[200];
      snprintf(buf, sizeof buf, "problem needs %zu bytes of workspace; the no-alloc scratch holds %zu", need,
               kStaticScratchBytes);
      throw NoAllocFail{SFR_E_NOMEM, buf};
    }
    void* base = nullptr;
    NA_CUDA(scratch_base(&base));
    Buffers b{};
    carve(s, fp64, base, &b);
    b.M = p.M;
    b.m_dtype = p.m_dtype;
    b.u_cur = 0;
    // state, Y_1 = 0, B_0 = I, identity warm-start bases: the array holds the last call's values
    DevState h{};
    h.mu = p.mu0;
    h.mu_last = p.mu0;
    h.rho = p.rho;
    h.mu_max = p.mu_max;
    h.tol = p.tol;
    h.fixed = p.fixed_iters > 0;
    h.max_iter = p.fixed_iters > 0 ? p.fixed_iters : p.max_iter;
    h.status = SFR_OK;
    NA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemsetAsync(b.Y[0], 0, (fp64 ? 8 : 4) * (size_t)s.m * b.ldy, st));
    double eye[kMaxRank * kMaxRank];
    float eyef[kMaxRank * kMaxRank];
    memset(eye, 0, sizeof eye);
    memset(eyef, 0, sizeof eyef);
    for (int i = 0; i < s.rp; ++i) {
      eye[i * s.rp + i] = 1.0;
      eyef[i * s.rp + i] = 1.f;
    }
    NA_CUDA(cudaMemcpyAsync(b.B, eye, 8 * s.rp * s.rp, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(b.Qeig_u, eyef, 4 * s.rp * s.rp, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(b.Qeig_v, eyef, 4 * s.rp * s.rp, cudaMemcpyHostToDevice, st));
    NA_CUDA(launch_norm_m(s, b, st));
    iteration(s, b, fp64, true, st);
    const Buffers after_first = b;
    DevState out{};
    int launched = 1;
    const int cap = h.max_iter;
    for (;;) {
      NA_CUDA(cudaMemcpyAsync(&out, b.st, sizeof out, cudaMemcpyDeviceToHost, st));
      NA_CUDA(cudaStreamSynchronize(st));
      if (out.done || launched >= cap) break;
      for (int k = 0; k < 8 && launched < cap; ++k, ++launched) iteration(s, b, fp64, false, st);
    }
    // buffers of the last completed iteration K: iterations after the first alternate them
    const int K = out.iter;
    Buffers fin = after_first;
    if (K >= 2 && (K - 1) % 2 == 1) {
      fin.u_cur = 1 - after_first.u_cur;
      std::swap(fin.Y[0], fin.Y[1]);
    }
    std::swap(fin.Y[0], fin.Y[1]);  // Y[0] <- the multiplier the last iteration read
    if (out.status == SFR_OK || out.status == SFR_E_NOCONV) {
      NA_CUDA(launch_export_factors(s, fin, fp64, fin.u_cur, res->U, res->V, st));
      if (res->B)
        for (int i = 0; i < p.r; ++i)
          NA_CUDA(cudaMemcpyAsync(res->B + (size_t)i * p.r, fin.B + (size_t)i * s.rp, 8 * p.r,
                                  cudaMemcpyDeviceToDevice, st));
      if (res->S || res->L)
        NA_CUDA(launch_finalize(s, fin, fp64, fin.u_cur, res->S, res->s_dtype, res->lds, res->L, st));
    }
    NA_CUDA(cudaStreamSynchronize(st));
    res->iters = out.iter;
    res->rel_residual = out.res;
    res->status = (sfr_status)out.status;
    res->path = 0;  // SIMT passes only (the tensor-core path's operand copies are not in the array)
    res->lambda_min_B = NAN;
    if (res->B && (res->status == SFR_OK || res->status == SFR_E_NOCONV)) {
      std::vector<double> hb((size_t)p.r * p.r);
      NA_CUDA(cudaMemcpy(hb.data(), res->B, 8 * hb.size(), cudaMemcpyDeviceToHost));
      res->lambda_min_B = host_lambda_min(hb, p.r);
    }
    if (res->status != SFR_OK) ctx_set_error(ctx, "sfr_solve_noalloc: solve did not finish cleanly");
    return res->status;
  } catch (const NoAllocFail& f) {
    ctx_set_error(ctx, f.msg);
    res->status = f.code;
    return f.code;
  }
}
