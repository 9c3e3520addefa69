// Internal declarations shared by the libsfr translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/sfr.h"
#include "tc_sweep.h"

namespace sfr {

constexpr int kMaxRank = 64;  // r <= 64: r x r blocks live in shared memory

// Programmatic dependent launch.  The kernels of an iteration are launched with
// cudaLaunchAttributeProgrammaticStreamSerialization (launch_pdl), so that the next kernel is
// launched while the current one runs.  Every kernel of the library starts with pdl_enter():
// griddepcontrol.wait blocks until the preceding kernel has completed and its writes are
// visible (it returns at once for a kernel launched without the attribute), so no global
// memory is touched before that; then griddepcontrol.launch_dependents lets the following
// kernel be scheduled.  A grid triggers only once all its CTAs run, so waiting dependents
// never hold resources that the triggering grid still needs.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kern<<<grid, block, smem, st>>>(args...) with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace sfr

#include "launch.cuh"

namespace sfr {

// Per-problem scalars, device resident, read and written by the iteration kernels.
struct DevState {
  double mu;          // mu_k: penalty of the iteration about to run (Algorithm 1)
  double mu_last;     // mu used by the most recent S/Y step
  double rho;         // continuation factor
  double mu_max;      // mu_bar
  double tol;         // relative residual tolerance
  double norm_m;      // ||M||_F
  double res;         // ||M - L - S||_F / ||M||_F after the last iteration
  double lam_min_u;   // smallest eigenvalue of the last U-side Gram (B G_P B)
  double lam_min_v;   // smallest eigenvalue of the last V-side Gram (B G_W B)
  int32_t iter;       // completed iterations
  int32_t max_iter;   // hard cap (fixed_iters when > 0)
  int32_t fixed;      // 1: run exactly max_iter iterations
  int32_t done;       // 1: stop (converged, cap reached or failed)
  int32_t status;     // sfr_status of the solve so far
  int32_t pad;
};

// Shapes and launch parameters of one problem; plain values captured by the kernels.
struct Shape {
  int64_t m, n, ldm;
  int r, rp;            // rank and padded rank (8, 16, 32 or 64)
  int nsplit;           // column splits of the sweep (partial thin products P)
  int cols_per_split;   // multiple of the sweep's column tile
  int nchunk;           // row chunks of the W = X^T U pass
  int rows_per_chunk;   // multiple of the W pass's row tile
  int sweep_grid_x;     // ceil(m / sweep rows per CTA)
  int wpass_grid_x;     // ceil(n / W-pass columns per CTA)
  int gram_rows;        // rows per CTA in the Gram / row-transform kernels
  int gp_blocks;        // ceil(m / gram_rows)
  int gw_blocks;        // ceil(n / gram_rows)
  int resid_parts;      // residual partials written by one sweep
  int num_sms;          // SMs of the device (grid sizing of the persistent-style kernels)
  int mx_grid_x;        // row-block CTAs of the mixed-path SIMT sweep (64-row blocks, grid-stride)
  int q_ctas;           // > 0: persistent tensor-core sweep over this many CTAs, whose Q partials per
                        // 128-row block are the CTAs owning its tiles (tc_q_slots); nsplit = max slots
  int64_t mc_ld;        // > 0: the SIMT mixed passes read an aligned copy of M with this leading
                        // dimension (rows 16-byte aligned, zero padding), made once per solve
  int mc_es;            // element size of that copy
};

// Persistent tensor-core sweep: the N = R T (128-row block, 64-column tile) pairs, row-major,
// are split into G contiguous ranges; CTA c owns tiles [c N / G, (c + 1) N / G).
__host__ __device__ inline int64_t tc_tile_owner(int64_t x, int64_t N, int64_t G) { return ((x + 1) * G - 1) / N; }
// Number of CTAs (Q partial slots) that own tiles of row block rb; slot k is CTA owner(rb T) + k.
__host__ __device__ inline int tc_q_slots(int64_t rb, int64_t T, int64_t N, int64_t G) {
  return (int)(tc_tile_owner(rb * T + T - 1, N, G) - tc_tile_owner(rb * T, N, G) + 1);
}

// Device buffers of one solve.  TC is double (FP64 path) or float (mixed path);
// the pointers below are typed void* and cast by the launchers.
struct Buffers {
  const void* M;        // m x n matrix the passes read (device): the caller's, or its aligned copy Mc
  sfr_dtype m_dtype;
  void* Mc;             // aligned copy of M (Shape::mc_ld > 0), else null
  int64_t ldy;          // leading dimension of Y[] and D: n, rounded up to 4 on the SIMT mixed path
                        // (16-byte aligned rows for its vector and cp.async accesses)
  void* Y[2];           // multiplier ping-pong, m x ldy, TC
  void* D;              // Delta = X_{k+1} - L_{k+1}, m x ldy, TC
  void* P;              // m x rp, TC: X_k V_k
  void* U[2];           // m x rp, TC: U_bar ping-pong
  void* W;              // n x rp, TC: X_k^T U_bar
  void* V;              // n x rp, TC
  void* C;              // n x rp, TC: C = V_bar B_bar (so L = U C^T)
  void* Qpart;          // nsplit x m x rp, TC
  void* Wpart;          // nchunk x n x rp, TC
  double* GPpart;       // gp_blocks x rp x rp
  double* GWpart;       // gw_blocks x rp x rp
  double* Hpart;        // gp_blocks x rp x rp : U_old^T U_new partials
  double* Gsum;         // rp x rp : summed Gram (input of the r x r projector)
  double* resid_part;   // sweep CTAs
  double* normm_part;   // ||M||^2 partials
  double* B;            // rp x rp
  double* Bprev;        // rp x rp : B of the previous iteration (Algorithm 4 stopping rule)
  double* TU;           // rp x rp : U_bar = P T_U
  double* TV;           // rp x rp : V_bar = W T_V
  double* TCm;          // rp x rp : C = W T_C
  float* Qeig_u;        // rp x rp : last U-side eigenvectors (warm start)
  float* Qeig_v;        // rp x rp : last V-side eigenvectors
  DevState* st;
  int u_cur;            // which U buffer holds the current U_bar (host-side bookkeeping)
  bool tc;              // tensor-core path (mixed precision, r <= 64, bfloat16 M)
  bool full;            // Algorithm 4 on a fixed M: no multiplier or Delta buffers; the
                        // tensor-core path keeps two-term bfloat16 splits of U^T and V^T
  TcBuffers t;          // its extra buffers (Y[] above alias t.Y[] when tc)
};

// ---- kernel launchers (sweep.cu / rxr.cu) ----
// Each launcher returns the cudaError_t of its launch.

cudaError_t launch_norm_m(const Shape& s, const Buffers& b, cudaStream_t st);
cudaError_t launch_init_p(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st);
// pt: also write P^T as a two-term bfloat16 split into b.t.Ut (the tensor-core W pass operand)
cudaError_t launch_gram_p(const Shape& s, const Buffers& b, bool fp64, bool sum_parts, cudaStream_t st,
                          const void* addA = nullptr, const double* H = nullptr, bool pt = false);
// Sums the Gram partials into b.Gsum, then runs the r x r projector; fp64 = false (mixed path)
// stops Newton at the float32 resolution of its Gram.
cudaError_t launch_rxr(const Shape& s, const Buffers& b, bool v_side, cudaStream_t st, bool fp64 = true);
// out[e] = sum over c < count of parts[c * rpsq + e], in a fixed order (float64)
cudaError_t launch_reduce_parts(const double* parts, int count, int rpsq, double* out, const DevState* dst,
                                cudaStream_t st);
cudaError_t launch_apply_u(const Shape& s, const Buffers& b, bool fp64, bool first, cudaStream_t st);
// wp: the mixed SIMT path's partials of Delta^T P instead of Delta^T U_new (W = (Delta^T P) T_U + C H)
cudaError_t launch_wpass(const Shape& s, const Buffers& b, bool fp64, bool first, int u_new, cudaStream_t st,
                         bool wp = false);
cudaError_t launch_wfinal(const Shape& s, const Buffers& b, bool fp64, bool first, cudaStream_t st, bool wp = false);
cudaError_t launch_apply_v(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st);
cudaError_t launch_sweep(const Shape& s, const Buffers& b, bool fp64, int u_cur, cudaStream_t st);
cudaError_t launch_iter_end(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st);
cudaError_t launch_finalize(const Shape& s, const Buffers& b, bool fp64, int u_cur, void* S, sfr_dtype s_dtype,
                            int64_t lds, void* L, cudaStream_t st);  // Y is bfloat16 (ld t.ldy) when b.tc
// Algorithm 4 (FixedRankOptFull): Qpart = split partials of M V (SIMT), the end-of-iteration
// stopping rule on the change of B, and the float64 -> working-precision copy of V_0.
cudaError_t launch_ppass(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st);
cudaError_t launch_full_end(const Shape& s, const Buffers& b, cudaStream_t st);
cudaError_t launch_import(const Shape& s, const double* src, int64_t rows, void* dst, bool fp64, cudaStream_t st);
cudaError_t launch_export_factors(const Shape& s, const Buffers& b, bool fp64, int u_cur, double* U, double* V,
                                  cudaStream_t st);

// Tile constants shared between the launchers and the host planner.
constexpr int kSweepBM = 32;     // rows per sweep CTA
constexpr int kSweepBN = 64;     // columns per sweep tile
constexpr int kWBN = 64;         // columns per W-pass CTA
constexpr int kWBM = 32;         // rows per W-pass tile
constexpr int kGramRows = 64;    // rows per Gram / transform CTA

inline int pad_rank(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : 64; }
// The mixed path's float32 SIMT passes for r <= 32 (sweep_mx*/wpass_mx* kernels).
inline bool mx_path(const Shape& s, bool fp64) { return !fp64 && s.rp <= 32; }
// Leading dimension of the aligned copy of M that the SIMT mixed passes read when the caller's rows
// are not 16-byte aligned (0: no copy; the tensor-core path has its own alignment rule).
inline int64_t mcopy_ld(const Shape& s, bool fp64, bool tc, sfr_dtype m_dtype, const void* M) {
  if (tc || !mx_path(s, fp64)) return 0;
  const int64_t es = m_dtype == SFR_F64 ? 8 : m_dtype == SFR_F32 ? 4 : 2;
  if ((s.ldm * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(M) % 16) == 0) return 0;
  const int64_t per = 16 / es;
  return (s.n + per - 1) / per * per;
}
inline void plan_mcopy(Shape* s, bool fp64, bool tc, sfr_dtype m_dtype, const void* M) {
  s->mc_ld = mcopy_ld(*s, fp64, tc, m_dtype, M);
  s->mc_es = m_dtype == SFR_F64 ? 8 : m_dtype == SFR_F32 ? 4 : 2;
}
// M -> b.Mc (zero padding past column n); the passes then read b.Mc with leading dimension s.mc_ld.
cudaError_t launch_copy_m(const Shape& s, const void* M, int64_t ldm, void* Mc, cudaStream_t st);

// ---- host helpers shared by the entry points (solver.cu)
Shape plan_shape(int64_t m, int64_t n, int64_t ldm, int r, int num_sms);
// base == nullptr: size only.  full: the buffers of Algorithm 4 (no m x n workspace).
size_t carve(const Shape& s, bool fp64, void* base, Buffers* b, bool tc = false, bool full = false);
double host_lambda_min(std::vector<double> A, int r);

// ---- grouped serving engine (batch.cu)
// One request handed to the engine: the problem, where its results go, the workspace bytes the
// context admitted it with, and the context's handle for it.
struct BatchJob {
  sfr_problem prob;
  sfr_result* res;
  size_t bytes;
  void* token;
};
class BatchEngine;
// take(job, block): the next admissible request (block = wait for one; false when stopping with
// nothing queued); done(job, status, message): the request finished.
BatchEngine* batch_create(int device, int capacity, std::function<bool(BatchJob*, bool)> take,
                          std::function<void(BatchJob&, sfr_status, const std::string&)> done);
void batch_destroy(BatchEngine* e);  // waits until every admitted request is answered
bool batch_eligible(const sfr_problem& p);
int ctx_device(const sfr_ctx* ctx);
int ctx_num_sms(const sfr_ctx* ctx);
cudaStream_t ctx_stream(const sfr_ctx* ctx);
void ctx_set_error(sfr_ctx* ctx, const std::string& msg);

}  // namespace sfr

// Argument checks of sfr_solve / sfr_submit (solver.cu); SFR_OK or SFR_E_INVAL with a reason.
sfr_status validate(const sfr_problem* p, const sfr_result* r, std::string* why);
