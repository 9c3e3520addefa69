// Host driver of libsfr: contexts, workspace, the FR-ADM iteration schedule
// (Algorithm 1) on one stream with CUDA graphs, FR-Nys (Algorithm 2), and the
// request queue behind sfr_submit / sfr_poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sfr_internal.h"

namespace sfr {

// ---------------------------------------------------------------- errors
struct Fail {
  sfr_status code;
  std::string msg;
};

#define SFR_CUDA(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) throw Fail{SFR_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

static std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

static size_t dtype_size(sfr_dtype d) { return d == SFR_F64 ? 8 : d == SFR_F32 ? 4 : 2; }

// ---------------------------------------------------------------- device memory
// A growable device arena: one cudaMalloc per workspace, carved into aligned pieces.
struct DeviceBlock {
  void* ptr = nullptr;
  size_t bytes = 0;
  ~DeviceBlock() {
    if (ptr) cudaFree(ptr);
  }
  void release(size_t* held) {
    if (ptr) {
      cudaFree(ptr);
      *held -= bytes;
    }
    ptr = nullptr;
    bytes = 0;
  }
  void ensure(size_t want, size_t* held, size_t budget) {
    if (want <= bytes) return;
    if (budget && *held - bytes + want > budget)
      throw Fail{SFR_E_NOMEM, fmt("workspace of %zu bytes exceeds the HBM budget of %zu bytes", want, budget)};
    if (ptr) {
      cudaFree(ptr);
      *held -= bytes;
      ptr = nullptr;
      bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail{SFR_E_NOMEM, fmt("cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e))};
    }
    bytes = want;
    *held += want;
  }
};

struct Carver {
  char* base;
  size_t off = 0;
  bool dry;
  explicit Carver(void* b) : base(static_cast<char*>(b)), dry(b == nullptr) {}
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = dry ? nullptr : base + off;
    off += bytes;
    return p;
  }
};

// ---------------------------------------------------------------- planning
Shape plan_shape(int64_t m, int64_t n, int64_t ldm, int r, int num_sms) {
  Shape s{};
  s.m = m;
  s.n = n;
  s.ldm = ldm;
  s.r = r;
  s.rp = pad_rank(r);
  const int64_t target = 2LL * num_sms;
  s.sweep_grid_x = (int)((m + kSweepBM - 1) / kSweepBM);
  int64_t tiles = (n + kSweepBN - 1) / kSweepBN;
  // column splits: enough (64-row block, split) pairs for four CTAs per SM
  const int64_t nrb64 = (m + 63) / 64;
  int64_t ns = std::max<int64_t>(1, std::min<int64_t>(tiles, (4LL * num_sms + nrb64 - 1) / nrb64));
  int64_t tps = (tiles + ns - 1) / ns;
  s.cols_per_split = (int)(tps * kSweepBN);
  s.nsplit = (int)((n + s.cols_per_split - 1) / s.cols_per_split);
  s.wpass_grid_x = (int)((n + kWBN - 1) / kWBN);
  int64_t rtiles = (m + kWBM - 1) / kWBM;
  int64_t nc = std::max<int64_t>(1, std::min<int64_t>(rtiles, (target + s.wpass_grid_x - 1) / s.wpass_grid_x));
  // chunks are whole multiples of 64 rows (the tensor-core W pass loads 64-row blocks)
  int64_t rtpc = (rtiles + nc - 1) / nc;
  s.rows_per_chunk = (int)(((rtpc * kWBM) + 63) / 64 * 64);
  s.nchunk = (int)((m + s.rows_per_chunk - 1) / s.rows_per_chunk);
  s.gram_rows = kGramRows;
  // thin kernels loop over 64-row tiles with at most four CTAs per SM (latency hiding for tall
  // matrices), which bounds the number of r x r partials the projector kernels reduce
  auto thin_ctas = [&](int64_t rows) {  // one CTA per SM, four for tall thin matrices
    const int64_t tiles = (rows + kGramRows - 1) / kGramRows;
    return (int)std::min<int64_t>(tiles, tiles >= 4LL * num_sms ? 4LL * num_sms : num_sms);
  };
  s.gp_blocks = thin_ctas(m);
  s.gw_blocks = thin_ctas(n);
  s.resid_parts = s.nsplit * (int)std::max<int64_t>(s.sweep_grid_x, 8 * nrb64);  // see launch_iter_end
  s.q_ctas = 0;
  s.num_sms = num_sms;
  s.mx_grid_x = (int)std::max<int64_t>(1, std::min<int64_t>(nrb64, (8LL * num_sms + s.nsplit - 1) / s.nsplit));
  return s;
}

// Lay out every buffer of one solve inside `base` (or just size it when base == nullptr).
size_t carve(const Shape& s, bool fp64, void* base, Buffers* b, bool tc, bool full) {
  const size_t tcb = fp64 ? 8 : 4;
  const size_t rp = s.rp, rpsq = rp * rp;
  Carver c(base);
  Buffers x{};
  x.tc = tc;
  x.full = full;
  if (tc) {
    // tensor-core path: bfloat16 multiplier and transposed Delta, plus the MMA operand copies
    // (Algorithm 4 on a fixed M needs only the transposed, split thin factors)
    x.t.ldy = (s.n + 63) / 64 * 64;
    x.t.ldd = (s.m + 63) / 64 * 64;
    if (!full) {
      x.t.Y[0] = x.Y[0] = c.take(2 * s.m * x.t.ldy);
      x.t.Y[1] = x.Y[1] = c.take(2 * s.m * x.t.ldy);
      x.t.D = c.take(2 * s.m * x.t.ldy);
      x.t.Uh = static_cast<float*>(c.take(4 * s.m * 64));
      x.t.Ul = static_cast<float*>(c.take(4 * s.m * 64));
      x.t.Ch = static_cast<float*>(c.take(4 * s.n * 64));
      x.t.Cl = static_cast<float*>(c.take(4 * s.n * 64));
    }
    x.D = nullptr;
    x.t.Ut = c.take(2 * 128 * x.t.ldd);
    x.t.Vt = c.take(2 * 128 * x.t.ldy);
  } else if (!full) {
    x.ldy = mx_path(s, fp64) ? (s.n + 3) / 4 * 4 : s.n;
    x.Y[0] = c.take(tcb * s.m * x.ldy);
    x.Y[1] = c.take(tcb * s.m * x.ldy);
    x.D = c.take(tcb * s.m * x.ldy);
  }
  if (s.mc_ld > 0) x.Mc = c.take((size_t)s.mc_es * s.m * s.mc_ld);
  x.P = c.take(tcb * s.m * rp);
  x.U[0] = c.take(tcb * s.m * rp);
  x.U[1] = c.take(tcb * s.m * rp);
  x.W = c.take(tcb * s.n * rp);
  x.V = c.take(tcb * s.n * rp);
  x.C = c.take(tcb * s.n * rp);
  x.Qpart = c.take(tcb * s.nsplit * s.m * rp);
  x.Wpart = c.take(tcb * s.nchunk * s.n * rp);
  x.GPpart = static_cast<double*>(c.take(8 * rpsq * s.gp_blocks));
  x.GWpart = static_cast<double*>(c.take(8 * rpsq * s.gw_blocks));
  x.Hpart = static_cast<double*>(c.take(8 * rpsq * (s.gp_blocks + 1)));
  x.Gsum = static_cast<double*>(c.take(8 * rpsq));
  x.resid_part = static_cast<double*>(c.take(8 * (size_t)s.resid_parts));
  x.normm_part = static_cast<double*>(c.take(8 * 1024));
  x.B = static_cast<double*>(c.take(8 * rpsq));
  x.Bprev = static_cast<double*>(c.take(8 * rpsq));
  x.TU = static_cast<double*>(c.take(8 * rpsq));
  x.TV = static_cast<double*>(c.take(8 * rpsq));
  x.TCm = static_cast<double*>(c.take(8 * rpsq));
  x.Qeig_u = static_cast<float*>(c.take(4 * rpsq));
  x.Qeig_v = static_cast<float*>(c.take(4 * rpsq));
  x.st = static_cast<DevState*>(c.take(sizeof(DevState)));
  if (b) *b = x;
  return c.off + 256;
}

// ---------------------------------------------------------------- launch-shape autotuner
// The mixed-path SIMT sweep loops each CTA over 64-row blocks, so its grid is free: how many CTAs
// per SM hide latency best depends on the shape (row length, rank, storage).  The first solve of
// a size class (m and n bucketed by powers of two, padded rank, dtype of M, vector-load
// eligibility) times the sweep at 2, 4, 8 and 16 CTAs per SM before it starts and keeps the
// fastest.  The table is process-wide and an entry never changes once set, so every solve of a
// class -- through sfr_solve or any serving slot -- uses the same grid and gets the same result
// (the grid decides the order of the residual partial sums).  SFR_AUTOTUNE=0 disables it (8 per
// SM); SFR_TUNE_FILE=path loads and appends choices as a flat JSON object {"class": ctas, ...}.
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;  // size class -> CTAs per SM
bool g_tune_loaded = false;

std::string tune_file() {
  const char* f = getenv("SFR_TUNE_FILE");
  return f ? std::string(f) : std::string();
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const std::string path = tune_file();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  fclose(f);
  // "key": value pairs of a flat object
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t colon = text.find(':', end);
    if (colon == std::string::npos) break;
    const int v = atoi(text.c_str() + colon + 1);
    if (v > 0 && v <= 64) g_tune.emplace(key, v);
    pos = colon + 1;
  }
}

void tune_save_locked() {
  const std::string path = tune_file();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "w");
  if (!f) return;
  fputs("{", f);
  bool firstk = true;
  for (const auto& kv : g_tune) {
    fprintf(f, "%s\n  \"%s\": %d", firstk ? "" : ",", kv.first.c_str(), kv.second);
    firstk = false;
  }
  fputs("\n}\n", f);
  fclose(f);
}

int ilog2(int64_t v) {
  int k = 0;
  while (v > 1) {
    v >>= 1;
    ++k;
  }
  return k;
}
}  // namespace

std::string tune_class(const Shape& s, sfr_dtype m_dtype, bool vec) {
  return fmt("mx_sweep/m2^%d/n2^%d/rp%d/dt%d/v%d", ilog2(s.m), ilog2(s.n), s.rp, (int)m_dtype, (int)vec);
}

int mx_grid_for(const Shape& s, int ctas_per_sm) {
  const int64_t nrb64 = (s.m + 63) / 64;
  return (int)std::max<int64_t>(1, std::min<int64_t>(nrb64, ((int64_t)ctas_per_sm * s.num_sms + s.nsplit - 1) / s.nsplit));
}

// Sets s.mx_grid_x for the mixed SIMT sweep from the process-wide table, timing the candidates on
// b (on stream st) when the size class is new; true when it launched timing sweeps.
bool tune_mx_grid(Shape& s, Buffers& b, sfr_dtype m_dtype, cudaStream_t st) {
  const char* env = getenv("SFR_AUTOTUNE");
  const bool vec = (b.ldy % 4 == 0) &&
                   ((size_t)s.ldm * (m_dtype == SFR_F64 ? 8 : m_dtype == SFR_F32 ? 4 : 2)) % 16 == 0 &&
                   (reinterpret_cast<uintptr_t>(b.M) % 16) == 0;
  const std::string cls = tune_class(s, m_dtype, vec);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(cls);
  if (it != g_tune.end()) {
    s.mx_grid_x = mx_grid_for(s, it->second);
    return false;
  }
  int best = 8;
  bool timed = false;
  if (!(env && env[0] == '0')) {
    cudaEvent_t e0, e1;
    SFR_CUDA(cudaEventCreate(&e0));
    SFR_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int c : {2, 4, 8, 16}) {
      Shape t = s;
      t.mx_grid_x = mx_grid_for(s, c);
      SFR_CUDA(launch_sweep(t, b, false, 0, st));  // warm-up
      SFR_CUDA(cudaEventRecord(e0, st));
      for (int k = 0; k < 3; ++k) SFR_CUDA(launch_sweep(t, b, false, 0, st));
      SFR_CUDA(cudaEventRecord(e1, st));
      SFR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      SFR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms * 0.97f) {  // prefer the earlier (smaller) grid unless clearly faster
        best_ms = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    timed = true;
  }
  g_tune.emplace(cls, best);
  tune_save_locked();
  s.mx_grid_x = mx_grid_for(s, best);
  return timed;
}

// ---------------------------------------------------------------- one FR-ADM solve
struct Solver {
  int device = 0;
  int num_sms = 152;
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // the auxiliary solver's stream is created and destroyed by it
  size_t budget = 0;
  size_t held = 0;
  DeviceBlock work;
  DeviceBlock staging;  // host-memory mode: device copies of M / S / L / perm
  DeviceBlock nys;      // FR-Nys: gathered blocks and block factors
  DevState* host_state = nullptr;  // pinned
  // graph cache, keyed by the buffer layout it was captured with
  cudaGraphExec_t graph = nullptr;    // two iterations, event slots 1-2
  cudaGraphExec_t graph_b = nullptr;  // the same two iterations, event slots 3-4
  std::string graph_key;
  int graph_kernels = 0;
  TcMaps maps;          // tensor maps of the current tensor-core solve (captured by value in graphs)
  bool last_tc = false; // whether the last solve took the tensor-core path
  // profiling: kernel counters and events (slot 0: eager iteration, slots 1-2: the graph's two)
  bool profile = false;
  bool profile_pass_only = false;  // time only the m x n pass (sweep or P pass), not W pass / r x r
  bool count_stats = false;
  bool capturing = false;
  int64_t launches[SFR_STAT_COUNT] = {};
  int64_t timed[SFR_STAT_COUNT] = {};
  double total_ms[SFR_STAT_COUNT] = {};
  double bytes[SFR_STAT_COUNT] = {};
  double sweep_bytes = 0, wpass_bytes = 0, wpass_first_bytes = 0;  // per launch, set per solve
  int pass_kind = SFR_STAT_SWEEP;  // class of the m x n pass timed in event slot 0 (sweep or P pass)
  cudaEvent_t ev[5][4][2] = {};       // slot 0: eager iteration; 1-2: graph A; 3-4: graph B
  cudaEvent_t done_ev[2] = {};        // completion of the last launch of graph A / B
  DevState* host_state2 = nullptr;    // pinned state copies taken after graph A / B
  std::unique_ptr<Solver> aux;        // FR-Nys: solves the second block concurrently (own stream)
  cudaStream_t side = nullptr;        // tensor-core path: the W pass, beside the U-side projector
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

  ~Solver() {
    if (aux) aux.reset();
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_b) cudaGraphExecDestroy(graph_b);
    if (host_state) cudaFreeHost(host_state);
    if (host_state2) cudaFreeHost(host_state2);
    if (own_stream && stream) cudaStreamDestroy(stream);
    for (auto& e : done_ev)
      if (e) cudaEventDestroy(e);
    for (auto& a : ev)
      for (auto& b : a)
        for (auto& e : b)
          if (e) cudaEventDestroy(e);
  }

  void make_done_events() {
    for (auto& e : done_ev)
      if (!e) SFR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!host_state2) SFR_CUDA(cudaMallocHost(&host_state2, 2 * sizeof(DevState)));
  }

  void ensure_side() {
    if (!side) SFR_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    if (!fork_ev) SFR_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    if (!join_ev) SFR_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
  }

  void make_events() {
    for (auto& a : ev)
      for (auto& b : a)
        for (auto& e : b)
          if (!e) SFR_CUDA(cudaEventCreate(&e));
  }

  // Timed launch of one kernel class: events around it when profiling.
  template <typename F>
  void timed_launch(int slot, int k, F&& f) {
    timed_launch_on(stream, slot, k, f);
  }
  template <typename F>
  void timed_launch_on(cudaStream_t on, int slot, int k, F&& f) {
    // inside stream capture an event record becomes a graph node only with the external flag,
    // and that flag is refused outside capture
    const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    // profile 2: the sweep of the eager first iteration (slot 0) and of the first iteration of
    // each replay of graph A (slot 1), one iteration in four
    const bool timed = profile && (!profile_pass_only || (k == 0 && slot <= 1));
    if (timed) SFR_CUDA(cudaEventRecordWithFlags(ev[slot][k][0], on, flags));
    SFR_CUDA(f());
    if (timed) SFR_CUDA(cudaEventRecordWithFlags(ev[slot][k][1], on, flags));
  }

  // Accumulate the event durations of the iterations that ran in `slot`s [first, first + count).
  void harvest(int first, int count) {
    if (!profile || !count_stats) return;
    for (int sl = first; sl < first + count; ++sl) {
      if (profile_pass_only && sl > 1) break;  // see timed_launch_on
      float ms;
      SFR_CUDA(cudaEventElapsedTime(&ms, ev[sl][0][0], ev[sl][0][1]));
      total_ms[pass_kind] += ms;
      timed[pass_kind] += 1;
      bytes[pass_kind] += sweep_bytes;
      if (profile_pass_only) continue;
      SFR_CUDA(cudaEventElapsedTime(&ms, ev[sl][1][0], ev[sl][1][1]));
      total_ms[SFR_STAT_WPASS] += ms;
      timed[SFR_STAT_WPASS] += 1;
      bytes[SFR_STAT_WPASS] += sl == 0 ? wpass_first_bytes : wpass_bytes;
      for (int k = 2; k < 4; ++k) {
        SFR_CUDA(cudaEventElapsedTime(&ms, ev[sl][k][0], ev[sl][k][1]));
        total_ms[SFR_STAT_RXR] += ms;
        timed[SFR_STAT_RXR] += 1;
      }
    }
  }

  void count(int kind, int64_t n) {
    if (count_stats) launches[kind] += n;
  }

  // Enqueue one FR-ADM iteration; returns the number of kernels it launches.
  int enqueue_iteration(const Shape& s, Buffers& b, bool fp64, bool first, int slot) {
    if (b.tc) return enqueue_iteration_tc(s, b, first, slot);
    cudaStream_t st = stream;
    int kernels = 0;
    if (first) {
      SFR_CUDA(launch_init_p(s, b, fp64, st));
      SFR_CUDA(launch_gram_p(s, b, fp64, false, st));
      kernels += 2;
    }
    const int u_new = 1 - b.u_cur;
    if (!first && mx_path(s, fp64)) {
      // as on the tensor-core path: the W pass forms Delta^T P beside the U-side projector, and
      // W = (Delta^T P) T_U + C_old H after both
      ensure_side();
      SFR_CUDA(cudaEventRecord(fork_ev, st));
      SFR_CUDA(cudaStreamWaitEvent(side, fork_ev, 0));
      timed_launch_on(side, slot, 1, [&] { return launch_wpass(s, b, fp64, false, u_new, side, true); });
      SFR_CUDA(cudaEventRecord(join_ev, side));
      timed_launch(slot, 2, [&] { return launch_rxr(s, b, false, st, fp64); });  // T_U
      SFR_CUDA(launch_apply_u(s, b, fp64, false, st));                          // U_bar = P T_U, H partials
      SFR_CUDA(cudaStreamWaitEvent(st, join_ev, 0));
      SFR_CUDA(launch_wfinal(s, b, fp64, false, st, true));                     // W, G_W partials
    } else {
      timed_launch(slot, 2, [&] { return launch_rxr(s, b, false, st, fp64); });  // T_U = B (B G_P B)^{-1/2}
      SFR_CUDA(launch_apply_u(s, b, fp64, first, st));                          // U_bar = P T_U
      timed_launch(slot, 1, [&] { return launch_wpass(s, b, fp64, first, u_new, st); });  // X^T U_bar partials
      SFR_CUDA(launch_wfinal(s, b, fp64, first, st));                           // W, G_W partials
    }
    timed_launch(slot, 3, [&] { return launch_rxr(s, b, true, st, fp64); });   // T_V, B_bar, T_C
    SFR_CUDA(launch_apply_v(s, b, fp64, st));                                 // V_bar, C
    timed_launch(slot, 0, [&] { return launch_sweep(s, b, fp64, u_new, st); });  // S/Y steps, Delta, next P
    SFR_CUDA(launch_iter_end(s, b, fp64, st));                                // residual, mu, stop test
    SFR_CUDA(launch_gram_p(s, b, fp64, true, st));                            // P = sum of partials, G_P
    kernels += (first ? 11 : 12) + (s.nchunk >= 32 ? 1 : 0);  // as on the tensor-core path below (+ W pre-sum)
    b.u_cur = u_new;
    std::swap(b.Y[0], b.Y[1]);
    return kernels;
  }

  // The same iteration on the tensor-core path (mixed precision, bfloat16 storage, r <= 64).
  int enqueue_iteration_tc(const Shape& s, Buffers& b, bool first, int slot) {
    cudaStream_t st = stream;
    int kernels = 0;
    if (first) {
      SFR_CUDA(launch_init_p(s, b, false, st));
      SFR_CUDA(launch_gram_p(s, b, false, false, st));
      kernels += 2;
    }
    const int u_new = 1 - b.u_cur;
    if (first) {  // W = M^T U_bar
      timed_launch(slot, 2, [&] { return launch_rxr(s, b, false, st, false); });  // T_U
      SFR_CUDA(launch_apply_u(s, b, false, first, st));  // U_bar = P T_U, its TF32 split and U^T
      timed_launch(slot, 1, [&] { return tc_launch_wpass(s, maps, true, static_cast<float*>(b.Wpart), b.st, st); });
      SFR_CUDA(launch_wfinal(s, b, false, true, st));  // W, G_W partials
    } else {
      // W = X^T U_bar = X^T P T_U = (C_old (U_old^T P) + Delta^T P) T_U: the W pass forms
      // Delta^T P, which does not wait for the U-side projector, so it runs on the side stream
      // beside it; W = (Delta^T P) T_U + C_old H (H = U_old^T U_bar) after both.  (Issuing the
      // projector on a high-priority side stream instead measured slower.)
      ensure_side();
      SFR_CUDA(cudaEventRecord(fork_ev, st));
      SFR_CUDA(cudaStreamWaitEvent(side, fork_ev, 0));
      timed_launch_on(side, slot, 1,
                      [&] { return tc_launch_wpass_p(s, maps, static_cast<float*>(b.Wpart), b.st, side); });
      SFR_CUDA(cudaEventRecord(join_ev, side));
      timed_launch(slot, 2, [&] { return launch_rxr(s, b, false, st, false); });  // T_U
      SFR_CUDA(launch_apply_u(s, b, false, false, st));  // U_bar = P T_U, its TF32 split, H partials
      SFR_CUDA(cudaStreamWaitEvent(st, join_ev, 0));
      SFR_CUDA(launch_wfinal(s, b, false, false, st, true));  // W, G_W partials
    }
    timed_launch(slot, 3, [&] { return launch_rxr(s, b, true, st, false); });  // T_V, B_bar, T_C
    SFR_CUDA(launch_apply_v(s, b, false, st));  // V_bar, C, with the TF32 split of C and V^T
    const int y_in = b.Y[0] == b.t.Y[0] ? 0 : 1;
    timed_launch(slot, 0, [&] {
      return tc_launch_sweep(s, maps, b.t, y_in, static_cast<float*>(b.Qpart), b.resid_part, b.st, st);
    });
    SFR_CUDA(launch_iter_end(s, b, false, st));
    // P_{k+1} = U_bar B_bar + Delta V_bar  (L V_bar = U_bar B_bar since V_bar^T V_bar = I), with
    // P^T for the next W pass
    SFR_CUDA(launch_gram_p(s, b, false, true, st, b.U[u_new], b.B, true));
    // launches: projector 2 + 2 (partial sums, cluster kernel), transforms 2, W pass 1, W final
    // 1 (+1 H sum after the first, +1 wide pre-sum of many W partials), sweep 1, iteration end 1,
    // P / Gram 1
    kernels += (first ? 11 : 12) + (s.nchunk >= 32 ? 1 : 0);
    b.u_cur = u_new;
    std::swap(b.Y[0], b.Y[1]);
    return kernels;
  }

  // Iterations 2, 3, ... after an eager first one: two graphs (A, B) of two iterations each,
  // captured from `after_first` once per buffer layout (`key`) and replayed alternately until the
  // device state says done.  The host reads the state copied after the previous launch while the
  // next one already runs, so the GPU does not wait for the host; a launch issued after
  // convergence finds the stop flag set and costs only its launches.  `iter(b, slot)` enqueues
  // one iteration (event slot `slot`) and returns its kernel count.  On return host_state holds
  // the final device state.
  template <typename F>
  void drive(const Buffers& after_first, const std::string& key, int cap, bool timed_first, F&& iter) {
    Buffers b = after_first;
    if (graph_key != key + (profile ? "/p" : "")) {
      for (cudaGraphExec_t* gp : {&graph, &graph_b})
        if (*gp) {
          cudaGraphExecDestroy(*gp);
          *gp = nullptr;
        }
      for (int which = 0; which < 2; ++which) {
        b = after_first;
        cudaGraph_t g;
        SFR_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed));
        capturing = true;
        try {
          graph_kernels = iter(b, 1 + 2 * which);
          graph_kernels += iter(b, 2 + 2 * which);
        } catch (...) {
          capturing = false;
          cudaStreamEndCapture(stream, &g);
          throw;
        }
        capturing = false;
        SFR_CUDA(cudaStreamEndCapture(stream, &g));
        // node priorities honoured: the projector's cluster launches carry the top priority
        cudaError_t e = cudaGraphInstantiate(which ? &graph_b : &graph, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        SFR_CUDA(e);
      }
      graph_key = key + (profile ? "/p" : "");
    }
    make_done_events();
    SFR_CUDA(cudaMemcpyAsync(host_state, after_first.st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
    SFR_CUDA(cudaStreamSynchronize(stream));
    if (timed_first) harvest(0, host_state->iter >= 1 ? 1 : 0);
    int launched = 1, last_iter = host_state->iter, which = 0;
    int queue[2], queued = 0;  // launched graphs whose state has not been read yet (oldest first)
    bool stop = host_state->done != 0;
    while (!stop) {
      if (launched < cap) {
        SFR_CUDA(cudaGraphLaunch(which ? graph_b : graph, stream));
        SFR_CUDA(cudaMemcpyAsync(host_state2 + which, after_first.st, sizeof(DevState), cudaMemcpyDeviceToHost,
                                 stream));
        SFR_CUDA(cudaEventRecord(done_ev[which], stream));
        launched += 2;
        count(SFR_STAT_ALL, graph_kernels);
        count(pass_kind, 2);
        count(SFR_STAT_WPASS, 2);
        count(SFR_STAT_RXR, 4);
        queue[queued++] = which;
        which ^= 1;
      }
      if (queued == 2 || (launched >= cap && queued > 0)) {
        const int y = queue[0];
        queue[0] = queue[1];
        --queued;
        SFR_CUDA(cudaEventSynchronize(done_ev[y]));
        const DevState& hs = host_state2[y];
        harvest(1 + 2 * y, hs.iter - last_iter);
        last_iter = hs.iter;
        *host_state = hs;
        stop = hs.done != 0;
      }
      if (launched >= cap && queued == 0) stop = true;
    }
    SFR_CUDA(cudaMemcpyAsync(host_state, after_first.st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
    SFR_CUDA(cudaStreamSynchronize(stream));
  }

  // Picks the mixed SIMT sweep's grid for this size class (see the autotuner above).  Runs before
  // the first iteration: the sweep reads Y_1 = 0 and whatever U, C, V hold, and writes buffers the
  // first iteration overwrites, so timing it changes nothing.
  void tune_mx(Shape& s, Buffers& b, sfr_dtype m_dtype) {
    if (tune_mx_grid(s, b, m_dtype, stream)) count(SFR_STAT_ALL, 16);
  }

  // Runs Algorithm 1 on a device-resident M.  Returns the final host copy of the state and
  // fills U/V/B/S/L (device pointers) as requested.
  DevState run(const sfr_problem& p, const void* Mdev, double* Udev, double* Bdev, double* Vdev, void* Sdev,
               sfr_dtype s_dtype, int64_t lds, void* Ldev) {
    const bool fp64 = p.precision == SFR_PREC_FP64;
    const Shape s0 = plan_shape(p.m, p.n, p.ldm, p.r, num_sms);
    const bool tc = !fp64 && tc_supported(s0, p.m_dtype, p.ldm) && ((uintptr_t)Mdev % 16) == 0;
    last_tc = tc;
    Shape s = s0;
    if (tc) tc_plan(&s, num_sms);  // persistent sweep over the SMs
    plan_mcopy(&s, fp64, tc, p.m_dtype, Mdev);
    Buffers b{};
    const size_t bytes = carve(s, fp64, nullptr, nullptr, tc);
    work.ensure(bytes, &held, budget);
    carve(s, fp64, work.ptr, &b, tc);
    if (tc) SFR_CUDA(tc_make_maps(s, b.t, Mdev, p.ldm, &maps));
    pass_kind = SFR_STAT_SWEEP;
    {
      // algorithmic bytes per element: sweep reads M and Y_k, writes Y_{k+1} and Delta; the W pass
      // reads Delta (iteration 1: M, or M^T on the tensor-core path)
      const double mn = (double)s.m * s.n, bm = (double)dtype_size(p.m_dtype);
      const double by = tc ? 2 : (fp64 ? 8 : 4), bd = tc ? 2 : (fp64 ? 8 : 4);
      sweep_bytes = mn * (bm + 2 * by + bd);
      wpass_bytes = mn * bd;
      wpass_first_bytes = mn * bm;
    }
    b.M = Mdev;
    if (s.mc_ld > 0) {  // rows of M not 16-byte aligned: the passes read an aligned copy
      SFR_CUDA(launch_copy_m(s, Mdev, p.ldm, b.Mc, stream));
      b.M = b.Mc;
      s.ldm = s.mc_ld;
    }
    b.m_dtype = p.m_dtype;
    b.u_cur = 0;

    DevState h{};
    h.mu = p.mu0;
    h.mu_last = p.mu0;
    h.rho = p.rho;
    h.mu_max = p.mu_max;
    h.tol = p.tol;
    h.fixed = p.fixed_iters > 0;
    h.max_iter = p.fixed_iters > 0 ? p.fixed_iters : p.max_iter;
    h.status = SFR_OK;
    SFR_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, stream));
    const size_t ybytes = tc ? 2 * (size_t)s.m * b.t.ldy : (fp64 ? 8 : 4) * (size_t)s.m * b.ldy;
    SFR_CUDA(cudaMemsetAsync(b.Y[0], 0, ybytes, stream));  // Y_1 = 0
    std::vector<double> eye(s.rp * s.rp, 0.0);
    std::vector<float> eyef(s.rp * s.rp, 0.f);
    for (int i = 0; i < s.rp; ++i) {
      eye[i * s.rp + i] = 1.0;
      eyef[i * s.rp + i] = 1.f;
    }
    SFR_CUDA(cudaMemcpyAsync(b.B, eye.data(), 8 * eye.size(), cudaMemcpyHostToDevice, stream));  // B_0 = I_r
    SFR_CUDA(cudaMemcpyAsync(b.Qeig_u, eyef.data(), 4 * eyef.size(), cudaMemcpyHostToDevice, stream));
    SFR_CUDA(cudaMemcpyAsync(b.Qeig_v, eyef.data(), 4 * eyef.size(), cudaMemcpyHostToDevice, stream));
    SFR_CUDA(launch_norm_m(s, b, stream));
    count(SFR_STAT_ALL, 2);
    if (profile) make_events();
    if (!tc && mx_path(s, fp64)) tune_mx(s, b, p.m_dtype);

    // iteration 1 (X_1 = M, V_1 = I_{n x r}), eager
    count(SFR_STAT_ALL, enqueue_iteration(s, b, fp64, true, 0));
    count(SFR_STAT_SWEEP, 1);
    count(SFR_STAT_WPASS, 1);
    count(SFR_STAT_RXR, 2);
    const Buffers after_first = b;
    const std::string key = fmt("%p/%lld/%lld/%lld/%d/%d/%p", work.ptr, (long long)s.m, (long long)s.n,
                                (long long)s.ldm, s.r, (int)fp64, Mdev) +
                            fmt("/%d/%d/%d", (int)p.m_dtype, (int)tc, s.mx_grid_x);
    drive(after_first, key, h.max_iter, true,
          [&](Buffers& bb, int slot) { return enqueue_iteration(s, bb, fp64, false, slot); });
    DevState out = *host_state;
    const int K = out.iter;
    // buffers of the last completed iteration (see the graph's two-iteration period)
    Buffers fin = after_first;
    if (K >= 2 && K % 2 == 0) {
      fin.u_cur = 1 - after_first.u_cur;  // U written by the first iteration of a pair
      // that iteration read after_first.Y[0]
    } else {
      fin.Y[0] = after_first.Y[1];  // the second iteration of a pair (or iteration 1) read Y[1]
      fin.Y[1] = after_first.Y[0];
    }
    if (out.status == SFR_OK || out.status == SFR_E_NOCONV) {
      SFR_CUDA(launch_export_factors(s, fin, fp64, fin.u_cur, Udev, Vdev, stream));
      count(SFR_STAT_ALL, (Udev ? 1 : 0) + (Vdev ? 1 : 0) + ((Sdev || Ldev) ? 1 : 0));
      if (Bdev)  // the leading r x r block of the padded B, in one strided copy
        SFR_CUDA(cudaMemcpy2DAsync(Bdev, 8 * p.r, fin.B, 8 * s.rp, 8 * p.r, p.r, cudaMemcpyDeviceToDevice, stream));
      if ((Sdev || Ldev) && fin.tc)
        SFR_CUDA(tc_launch_finalize(s, maps, fin.t, fin.Y[0] == fin.t.Y[0] ? 0 : 1, Sdev, (int)s_dtype, lds, Ldev,
                                    fin.st, stream));
      else if (Sdev || Ldev)
        SFR_CUDA(launch_finalize(s, fin, fp64, fin.u_cur, Sdev, s_dtype, lds, Ldev, stream));
    }
    SFR_CUDA(cudaStreamSynchronize(stream));
    return out;
  }
  // One iteration of Algorithm 4: FixedRankOptStep (Algorithm 3) with X = M fixed, so both thin
  // products read M itself: P = M V_i (init_p: the first r columns of M, for V_0 = I_{n x r}),
  // U = P T_U, W = M^T U, V = W T_V, B = Sym(G_W T_V); then the stopping rule on the change of B.
  int enqueue_full(const Shape& s, Buffers& b, bool fp64, bool init_p, int slot) {
    cudaStream_t st = stream;
    if (init_p) {
      SFR_CUDA(launch_init_p(s, b, fp64, st));
    } else {
      timed_launch(slot, 0, [&] {
        return b.tc ? tc_launch_full_ppass(s, maps, static_cast<float*>(b.Qpart), b.st, st) : launch_ppass(s, b, fp64, st);
      });
    }
    SFR_CUDA(launch_gram_p(s, b, fp64, !init_p, st));                          // P, G_P partials
    timed_launch(slot, 2, [&] { return launch_rxr(s, b, false, st, fp64); });  // T_U = B (B G_P B)^{-1/2}
    SFR_CUDA(launch_apply_u(s, b, fp64, true, st));                            // U = P T_U
    const int u_new = 1 - b.u_cur;
    timed_launch(slot, 1, [&] {
      return b.tc ? tc_launch_full_wpass(s, maps, static_cast<float*>(b.Wpart), b.st, st)
                  : launch_wpass(s, b, fp64, true, u_new, st);
    });
    SFR_CUDA(launch_wfinal(s, b, fp64, true, st));                             // W = M^T U, G_W partials
    timed_launch(slot, 3, [&] { return launch_rxr(s, b, true, st, fp64); });   // T_V, B = Sym(G_W T_V)
    SFR_CUDA(launch_apply_v(s, b, fp64, st));                                  // V = W T_V
    SFR_CUDA(launch_full_end(s, b, st));
    b.u_cur = u_new;
    // P pass (or init_p) 1, P sum / Gram 1, projectors 2 + 2, transforms 2, W pass 1, W sum 1 (+1 wide
    // pre-sum of many W partials), end 1
    return 11 + (!b.tc && s.nchunk >= 32 ? 1 : 0);
  }

  // Runs Algorithm 4 (FixedRankOptFull) on a device-resident M from V_0 (NULL: I_{n x r}) and
  // B_0 (NULL: I_r), both device float64; writes U, B, V (device, float64) where non-null.
  DevState run_full(const sfr_opt_full_problem& p, const void* Mdev, const double* V0, const double* B0, double* Udev,
                    double* Bdev, double* Vdev) {
    const bool fp64 = p.precision == SFR_PREC_FP64;
    const Shape s0 = plan_shape(p.m, p.n, p.ldm, p.r, num_sms);
    const bool tc = !fp64 && tc_supported(s0, p.m_dtype, p.ldm) && ((uintptr_t)Mdev % 16) == 0;
    last_tc = tc;
    Shape s = s0;
    if (tc) tc_plan(&s, num_sms);  // the P pass uses the sweep's persistent partition
    Buffers b{};
    work.ensure(carve(s, fp64, nullptr, nullptr, tc, true), &held, budget);
    carve(s, fp64, work.ptr, &b, tc, true);
    if (tc) SFR_CUDA(tc_make_full_maps(s, b.t, Mdev, p.ldm, &maps));
    pass_kind = SFR_STAT_PPASS;
    {
      // algorithmic bytes per element: each of the two passes reads M once
      const double mn = (double)s.m * s.n, bm = (double)dtype_size(p.m_dtype);
      sweep_bytes = wpass_bytes = wpass_first_bytes = mn * bm;
    }
    b.M = Mdev;
    b.m_dtype = p.m_dtype;
    b.u_cur = 0;

    DevState h{};
    h.tol = p.tol;
    h.fixed = p.tol == 0.0;
    h.max_iter = p.max_iter;
    h.status = SFR_OK;
    SFR_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, stream));
    std::vector<double> eye(s.rp * s.rp, 0.0);
    std::vector<float> eyef(s.rp * s.rp, 0.f);
    for (int i = 0; i < s.rp; ++i) {
      eye[i * s.rp + i] = 1.0;
      eyef[i * s.rp + i] = 1.f;
    }
    SFR_CUDA(cudaMemcpyAsync(b.B, eye.data(), 8 * eye.size(), cudaMemcpyHostToDevice, stream));
    if (B0)  // B_0 in the leading r x r block, identity in the padding
      SFR_CUDA(cudaMemcpy2DAsync(b.B, 8 * s.rp, B0, 8 * p.r, 8 * p.r, p.r, cudaMemcpyDeviceToDevice, stream));
    SFR_CUDA(cudaMemcpyAsync(b.Bprev, b.B, 8 * eye.size(), cudaMemcpyDeviceToDevice, stream));
    SFR_CUDA(cudaMemcpyAsync(b.Qeig_u, eyef.data(), 4 * eyef.size(), cudaMemcpyHostToDevice, stream));
    SFR_CUDA(cudaMemcpyAsync(b.Qeig_v, eyef.data(), 4 * eyef.size(), cudaMemcpyHostToDevice, stream));
    if (profile) make_events();

    // iteration 1, eager
    if (V0) {
      // V = V_0 in working precision (with its split transpose on the tensor-core path): the
      // V-side row transform of W = V_0 with T_V = I (and C = V_0 B_0)
      SFR_CUDA(launch_import(s, V0, s.n, b.W, fp64, stream));
      SFR_CUDA(cudaMemcpyAsync(b.TV, eye.data(), 8 * eye.size(), cudaMemcpyHostToDevice, stream));
      SFR_CUDA(cudaMemcpyAsync(b.TCm, b.B, 8 * eye.size(), cudaMemcpyDeviceToDevice, stream));
      SFR_CUDA(launch_apply_v(s, b, fp64, stream));
      count(SFR_STAT_ALL, 2);
    }
    count(SFR_STAT_ALL, enqueue_full(s, b, fp64, V0 == nullptr, 0));
    count(SFR_STAT_PPASS, V0 ? 1 : 0);
    count(SFR_STAT_WPASS, 1);
    count(SFR_STAT_RXR, 2);
    const Buffers after_first = b;
    const std::string key = fmt("full/%p/%lld/%lld/%lld/%d/%d/%p", work.ptr, (long long)s.m, (long long)s.n,
                                (long long)s.ldm, s.r, (int)fp64, Mdev) +
                            fmt("/%d/%d", (int)p.m_dtype, (int)tc);
    drive(after_first, key, h.max_iter, V0 != nullptr,
          [&](Buffers& bb, int slot) { return enqueue_full(s, bb, fp64, false, slot); });
    DevState out = *host_state;
    const int K = out.iter;
    Buffers fin = after_first;
    if (K >= 2 && K % 2 == 0) fin.u_cur = 1 - after_first.u_cur;  // U of the first iteration of a pair
    if (out.status == SFR_OK || out.status == SFR_E_NOCONV) {
      SFR_CUDA(launch_export_factors(s, fin, fp64, fin.u_cur, Udev, Vdev, stream));
      count(SFR_STAT_ALL, (Udev ? 1 : 0) + (Vdev ? 1 : 0));
      if (Bdev)
        SFR_CUDA(cudaMemcpy2DAsync(Bdev, 8 * p.r, fin.B, 8 * s.rp, 8 * p.r, p.r, cudaMemcpyDeviceToDevice, stream));
    }
    SFR_CUDA(cudaStreamSynchronize(stream));
    return out;
  }
};


// Smallest eigenvalue of a symmetric r x r matrix (host, float64): Householder reduction to
// tridiagonal form, then bisection on the Sturm count (the number of negative pivots of
// T - x I, which equals the number of eigenvalues below x).  O(r^3) once, O(r) per probe.
double host_lambda_min(std::vector<double> A, int r) {
  if (r <= 0) return NAN;
  std::vector<double> v(r), pv(r), d(r), e(r, 0.0);
  for (int k = 0; k + 2 < r; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < r; ++i) alpha += A[i * r + k] * A[i * r + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (A[(k + 1) * r + k] > 0) alpha = -alpha;
    double vv = 0.0;
    for (int i = k + 1; i < r; ++i) {
      v[i] = A[i * r + k] - (i == k + 1 ? alpha : 0.0);
      vv += v[i] * v[i];
    }
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // trailing block: A <- H A H, H = I - beta v v^T, as A - v w^T - w v^T
    double pv_dot = 0.0;
    for (int i = k + 1; i < r; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < r; ++j) s += A[i * r + j] * v[j];
      pv[i] = beta * s;
      pv_dot += pv[i] * v[i];
    }
    const double c = 0.5 * beta * pv_dot;
    for (int i = k + 1; i < r; ++i) pv[i] -= c * v[i];  // w
    for (int i = k + 1; i < r; ++i)
      for (int j = k + 1; j < r; ++j) A[i * r + j] -= v[i] * pv[j] + pv[i] * v[j];
    A[(k + 1) * r + k] = A[k * r + k + 1] = alpha;
    for (int i = k + 2; i < r; ++i) A[i * r + k] = A[k * r + i] = 0.0;
  }
  for (int i = 0; i < r; ++i) d[i] = A[i * r + i];
  for (int i = 0; i + 1 < r; ++i) e[i] = A[(i + 1) * r + i];
  auto below = [&](double x) {  // eigenvalues of the tridiagonal matrix below x
    int count = 0;
    double q = d[0] - x;
    for (int i = 0;; ++i) {
      if (q < 0) ++count;
      if (i + 1 == r) break;
      if (q == 0.0) q = 1e-300;
      q = d[i + 1] - x - e[i] * e[i] / q;
    }
    return count;
  };
  double lo = d[0], hi = d[0];
  for (int i = 0; i < r; ++i) {  // Gershgorin interval
    const double rad = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < r ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - rad);
    hi = std::max(hi, d[i] + rad);
  }
  if (!(lo == lo) || !(hi == hi)) return NAN;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (below(mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

DevState solver_run(Solver& sv, const sfr_problem& p, const void* Mdev, double* U, double* B, double* V, void* S,
                    sfr_dtype s_dtype, int64_t lds, void* L) {
  return sv.run(p, Mdev, U, B, V, S, s_dtype, lds, L);
}
void* solver_nys_block(Solver& sv, size_t bytes) {
  sv.nys.ensure(bytes, &sv.held, sv.budget);
  return sv.nys.ptr;
}
cudaStream_t solver_stream(Solver& sv) { return sv.stream; }
bool solver_last_tc(const Solver& sv) { return sv.last_tc; }

// The auxiliary solver of sv (created on first use): its own stream, workspace and graph cache.
Solver* solver_aux(Solver& sv) {
  if (!sv.aux) {
    auto a = std::make_unique<Solver>();
    a->device = sv.device;
    a->num_sms = sv.num_sms;
    SFR_CUDA(cudaStreamCreateWithFlags(&a->stream, cudaStreamNonBlocking));
    a->own_stream = true;
    SFR_CUDA(cudaMallocHost(&a->host_state, sizeof(DevState)));
    sv.aux = std::move(a);
  }
  return sv.aux.get();
}

// Reserves, from the calling thread, the workspace that `sv.run` will need for problem p on the
// device matrix at Mdev, counted against the holder's budget (`held` / `budget`).  False when the
// budget or the device refuses it.
bool solver_reserve(Solver& sv, const sfr_problem& p, const void* Mdev, size_t* held, size_t budget) {
  const bool fp64 = p.precision == SFR_PREC_FP64;
  Shape s = plan_shape(p.m, p.n, p.ldm, p.r, sv.num_sms);
  const bool tc = !fp64 && tc_supported(s, p.m_dtype, p.ldm) && ((uintptr_t)Mdev % 16) == 0;
  if (tc) tc_plan(&s, sv.num_sms);
  plan_mcopy(&s, fp64, tc, p.m_dtype, Mdev);
  try {
    sv.work.ensure(carve(s, fp64, nullptr, nullptr, tc), held, budget);
  } catch (const Fail&) {
    return false;
  }
  return true;
}
size_t* solver_held(Solver& sv) { return &sv.held; }
size_t solver_budget(const Solver& sv) { return sv.budget; }

sfr_status nys_solve_device(Solver& sv, const sfr_problem& p, const void* Mdev, const int64_t* perm_dev,
                            sfr_result* res, void* Sdev, void* Ldev, double* Udev, double* Bdev, double* Vdev,
                            std::string* err);

// FR-Nys entry: stage host buffers when needed, then run on the device.
sfr_status sfr_nys_solve(Solver& sv, const sfr_problem& p, sfr_result* res, std::string* err) {
  const size_t mbytes = dtype_size(p.m_dtype) * (size_t)((p.m - 1) * p.ldm + p.n);
  const size_t outbytes = dtype_size(res->s_dtype) * (size_t)((p.m - 1) * res->lds + p.n);
  if (p.mem == SFR_MEM_DEVICE)
    return nys_solve_device(sv, p, p.M, p.nys_perm, res, res->S, res->L, res->U, res->B, res->V, err);
  size_t need = 0;
  auto add = [&](size_t bytes) { need = (need + 255) & ~size_t(255); size_t o = need; need += bytes; return o; };
  const size_t offM = add(mbytes), offP = add(8 * (size_t)p.m);
  const size_t offS = res->S ? add(outbytes) : 0, offL = res->L ? add(outbytes) : 0;
  const size_t ub = 8 * (size_t)p.m * p.r, vb = 8 * (size_t)p.n * p.r, bb = 8 * (size_t)p.r * p.r;
  const size_t offU = res->U ? add(ub) : 0, offV = res->V ? add(vb) : 0, offB = res->B ? add(bb) : 0;
  sv.staging.ensure(need + 256, &sv.held, sv.budget);
  char* st = static_cast<char*>(sv.staging.ptr);
  SFR_CUDA(cudaMemcpyAsync(st + offM, p.M, mbytes, cudaMemcpyHostToDevice, sv.stream));
  SFR_CUDA(cudaMemcpyAsync(st + offP, p.nys_perm, 8 * (size_t)p.m, cudaMemcpyHostToDevice, sv.stream));
  sfr_status s = nys_solve_device(sv, p, st + offM, reinterpret_cast<const int64_t*>(st + offP), res,
                                  res->S ? st + offS : nullptr, res->L ? st + offL : nullptr,
                                  res->U ? reinterpret_cast<double*>(st + offU) : nullptr,
                                  res->B ? reinterpret_cast<double*>(st + offB) : nullptr,
                                  res->V ? reinterpret_cast<double*>(st + offV) : nullptr, err);
  if (s == SFR_OK) {
    if (res->S) SFR_CUDA(cudaMemcpyAsync(res->S, st + offS, outbytes, cudaMemcpyDeviceToHost, sv.stream));
    if (res->L) SFR_CUDA(cudaMemcpyAsync(res->L, st + offL, outbytes, cudaMemcpyDeviceToHost, sv.stream));
    if (res->U) SFR_CUDA(cudaMemcpyAsync(res->U, st + offU, ub, cudaMemcpyDeviceToHost, sv.stream));
    if (res->V) SFR_CUDA(cudaMemcpyAsync(res->V, st + offV, vb, cudaMemcpyDeviceToHost, sv.stream));
    if (res->B) SFR_CUDA(cudaMemcpyAsync(res->B, st + offB, bb, cudaMemcpyDeviceToHost, sv.stream));
    SFR_CUDA(cudaStreamSynchronize(sv.stream));
  }
  return s;
}

}  // namespace sfr

// ---------------------------------------------------------------- C ABI
using namespace sfr;

struct Request {
  uint64_t ticket;
  sfr_problem prob;
  sfr_result* res;
  bool finished = false;
  sfr_status status = SFR_PENDING;
  int passed_over = 0;  // times a later request was admitted ahead of this one
};

struct sfr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  std::unique_ptr<Solver> solver;
  // request queue (sfr_submit / sfr_poll): `max_slots` slots, each a host thread with its own
  // stream, workspace and graph cache, so admitted requests run concurrently on the device
  int max_slots = 8;
  size_t budget = 0;      // cap on the summed workspace of running requests (0 = none)
  size_t in_use = 0;      // workspace bytes of running requests
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> live;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<std::unique_ptr<Solver>> slot_solvers;
  std::vector<cudaStream_t> slot_streams;
  // grouped engine (max_batch > 0): its own queue of the requests it can run
  int max_batch = 0;
  std::deque<std::shared_ptr<Request>> bqueue;
  BatchEngine* batch = nullptr;
};

static thread_local std::string g_create_error;

namespace sfr {
int ctx_device(const sfr_ctx* ctx) { return ctx->device; }
int ctx_num_sms(const sfr_ctx* ctx) { return ctx->solver->num_sms; }
cudaStream_t ctx_stream(const sfr_ctx* ctx) { return ctx->stream; }
void ctx_set_error(sfr_ctx* ctx, const std::string& msg) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->last_error = msg;
}
}  // namespace sfr

sfr_status validate(const sfr_problem* p, const sfr_result* r, std::string* why) {
  if (!p || !r) return *why = "null problem or result", SFR_E_INVAL;
  if (p->m <= 0 || p->n <= 0) return *why = "m and n must be positive", SFR_E_INVAL;
  if (p->ldm < p->n) return *why = "ldm must be >= n", SFR_E_INVAL;
  if (p->r < 1 || p->r > kMaxRank || p->r > p->m || p->r > p->n)
    return *why = fmt("need 1 <= r <= min(m, n, %d)", kMaxRank), SFR_E_INVAL;
  if (!p->M) return *why = "M is null", SFR_E_INVAL;
  if (p->m_dtype != SFR_F64 && p->m_dtype != SFR_F32 && p->m_dtype != SFR_BF16) return *why = "bad m_dtype", SFR_E_INVAL;
  if (!(p->rho > 1.0)) return *why = "rho must exceed 1", SFR_E_INVAL;
  if (!(p->mu0 > 0.0) || !(p->mu_max >= p->mu0)) return *why = "need 0 < mu0 <= mu_max", SFR_E_INVAL;
  if (p->fixed_iters <= 0 && (p->max_iter <= 0 || !(p->tol >= 0.0))) return *why = "need max_iter > 0 and tol >= 0", SFR_E_INVAL;
  if (p->precision != SFR_PREC_FP64 && p->precision != SFR_PREC_MIXED) return *why = "bad precision", SFR_E_INVAL;
  if (p->mem != SFR_MEM_DEVICE && p->mem != SFR_MEM_HOST) return *why = "bad mem", SFR_E_INVAL;
  if ((r->S || r->L) && (r->s_dtype != SFR_F64 && r->s_dtype != SFR_F32)) return *why = "s_dtype must be F64 or F32", SFR_E_INVAL;
  if ((r->S || r->L) && r->lds < p->n) return *why = "lds must be >= n", SFR_E_INVAL;
  if (p->nys_l != 0) {
    if (p->nys_l < p->r || p->nys_l > p->m || p->nys_l > p->n) return *why = "need r <= nys_l <= min(m, n)", SFR_E_INVAL;
    if (!p->nys_perm) return *why = "FR-Nys needs nys_perm", SFR_E_INVAL;
  }
  if ((int64_t)p->m * p->n > (int64_t)1 << 40) return *why = "matrix too large", SFR_E_INVAL;
  return SFR_OK;
}

// Solve on `sv`, staging host buffers when p.mem == SFR_MEM_HOST.
static sfr_status solve_with(Solver& sv, const sfr_problem& p, sfr_result* res, std::string* err) {
  try {
    res->path = 0;
    SFR_CUDA(cudaSetDevice(sv.device));
    if (p.nys_l != 0) {
      res->status = sfr_nys_solve(sv, p, res, err);
      return res->status;
    }
    const void* Mdev = p.M;
    double *U = res->U, *B = res->B, *V = res->V;
    void *S = res->S, *L = res->L;
    const size_t sb = dtype_size(res->s_dtype);
    const size_t mbytes = dtype_size(p.m_dtype) * (size_t)((p.m - 1) * p.ldm + p.n);
    const size_t outbytes = sb * (size_t)((p.m - 1) * res->lds + p.n);
    char* st = nullptr;
    size_t offU = 0, offV = 0, offB = 0, offS = 0, offL = 0;
    if (p.mem == SFR_MEM_HOST) {
      size_t need = 0;
      auto add = [&](size_t bytes) { need = (need + 255) & ~size_t(255); size_t o = need; need += bytes; return o; };
      const size_t offM = add(mbytes);
      if (U) offU = add(8 * (size_t)p.m * p.r);
      if (V) offV = add(8 * (size_t)p.n * p.r);
      if (B) offB = add(8 * (size_t)p.r * p.r);
      if (S) offS = add(outbytes);
      if (L) offL = add(outbytes);
      sv.staging.ensure(need + 256, &sv.held, sv.budget);
      st = static_cast<char*>(sv.staging.ptr);
      SFR_CUDA(cudaMemcpyAsync(st + offM, p.M, mbytes, cudaMemcpyHostToDevice, sv.stream));
      Mdev = st + offM;
      if (U) U = reinterpret_cast<double*>(st + offU);
      if (V) V = reinterpret_cast<double*>(st + offV);
      if (B) B = reinterpret_cast<double*>(st + offB);
      if (S) S = st + offS;
      if (L) L = st + offL;
    }
    DevState out = sv.run(p, Mdev, U, B, V, S, res->s_dtype, res->lds, L);
    res->path = sv.last_tc ? SFR_PATH_TC : 0;
    if (p.mem == SFR_MEM_HOST) {
      if (res->U) SFR_CUDA(cudaMemcpyAsync(res->U, U, 8 * (size_t)p.m * p.r, cudaMemcpyDeviceToHost, sv.stream));
      if (res->V) SFR_CUDA(cudaMemcpyAsync(res->V, V, 8 * (size_t)p.n * p.r, cudaMemcpyDeviceToHost, sv.stream));
      if (res->B) SFR_CUDA(cudaMemcpyAsync(res->B, B, 8 * (size_t)p.r * p.r, cudaMemcpyDeviceToHost, sv.stream));
      if (res->S) SFR_CUDA(cudaMemcpyAsync(res->S, S, outbytes, cudaMemcpyDeviceToHost, sv.stream));
      if (res->L) SFR_CUDA(cudaMemcpyAsync(res->L, L, outbytes, cudaMemcpyDeviceToHost, sv.stream));
      SFR_CUDA(cudaStreamSynchronize(sv.stream));
    }
    res->iters = out.iter;
    res->rel_residual = out.res;
    res->status = (sfr_status)out.status;
    res->lambda_min_B = NAN;
    if (res->status == SFR_OK || res->status == SFR_E_NOCONV) {
      // lambda_min of the returned B (SPD diagnostic, Appendix): from the device copy of B
      std::vector<double> hb((size_t)p.r * p.r);
      if (res->B && p.mem == SFR_MEM_HOST) {
        memcpy(hb.data(), res->B, 8 * hb.size());
      } else if (res->B) {
        SFR_CUDA(cudaMemcpy(hb.data(), res->B, 8 * hb.size(), cudaMemcpyDeviceToHost));
      }
      if (res->B) res->lambda_min_B = host_lambda_min(hb, p.r);
    }
    if (res->status != SFR_OK) {
      *err = res->status == SFR_E_NOCONV  ? fmt("no convergence after %d iterations (residual %.3e)", out.iter, out.res)
             : res->status == SFR_E_RANK ? fmt("rank-deficient thin product at iteration %d", out.iter + 1)
             : res->status == SFR_E_NAN  ? fmt("non-finite value at iteration %d", out.iter + 1)
                                         : fmt("solve failed with status %d", (int)res->status);
    }
    return res->status;
  } catch (const Fail& f) {
    *err = f.msg;
    res->status = f.code;
    return f.code;
  }
}

static sfr_status validate_full(const sfr_opt_full_problem* p, const sfr_opt_full_result* r, std::string* why) {
  if (!p || !r) return *why = "null problem or result", SFR_E_INVAL;
  if (p->m <= 0 || p->n <= 0) return *why = "m and n must be positive", SFR_E_INVAL;
  if (p->ldm < p->n) return *why = "ldm must be >= n", SFR_E_INVAL;
  if (p->r < 1 || p->r > kMaxRank || p->r > p->m || p->r > p->n)
    return *why = fmt("need 1 <= r <= min(m, n, %d)", kMaxRank), SFR_E_INVAL;
  if (!p->M) return *why = "M is null", SFR_E_INVAL;
  if (p->m_dtype != SFR_F64 && p->m_dtype != SFR_F32 && p->m_dtype != SFR_BF16) return *why = "bad m_dtype", SFR_E_INVAL;
  if (p->max_iter <= 0 || !(p->tol >= 0.0)) return *why = "need max_iter > 0 and tol >= 0", SFR_E_INVAL;
  if (p->precision != SFR_PREC_FP64 && p->precision != SFR_PREC_MIXED) return *why = "bad precision", SFR_E_INVAL;
  if (p->mem != SFR_MEM_DEVICE && p->mem != SFR_MEM_HOST) return *why = "bad mem", SFR_E_INVAL;
  if ((int64_t)p->m * p->n > (int64_t)1 << 40) return *why = "matrix too large", SFR_E_INVAL;
  return SFR_OK;
}

// Algorithm 4 on `sv`, staging host buffers when p.mem == SFR_MEM_HOST.
static sfr_status full_with(Solver& sv, const sfr_opt_full_problem& p, sfr_opt_full_result* res, std::string* err) {
  try {
    SFR_CUDA(cudaSetDevice(sv.device));
    const void* Mdev = p.M;
    const double *V0 = p.V0, *B0 = p.B0;
    double *U = res->U, *B = res->B, *V = res->V;
    const size_t mbytes = dtype_size(p.m_dtype) * (size_t)((p.m - 1) * p.ldm + p.n);
    const size_t ub = 8 * (size_t)p.m * p.r, vb = 8 * (size_t)p.n * p.r, bb = 8 * (size_t)p.r * p.r;
    if (p.mem == SFR_MEM_HOST) {
      size_t need = 0;
      auto add = [&](size_t bytes) { need = (need + 255) & ~size_t(255); size_t o = need; need += bytes; return o; };
      const size_t offM = add(mbytes), offV0 = V0 ? add(vb) : 0, offB0 = B0 ? add(bb) : 0;
      const size_t offU = U ? add(ub) : 0, offV = V ? add(vb) : 0, offB = B ? add(bb) : 0;
      sv.staging.ensure(need + 256, &sv.held, sv.budget);
      char* st = static_cast<char*>(sv.staging.ptr);
      SFR_CUDA(cudaMemcpyAsync(st + offM, p.M, mbytes, cudaMemcpyHostToDevice, sv.stream));
      Mdev = st + offM;
      if (V0) {
        SFR_CUDA(cudaMemcpyAsync(st + offV0, p.V0, vb, cudaMemcpyHostToDevice, sv.stream));
        V0 = reinterpret_cast<const double*>(st + offV0);
      }
      if (B0) {
        SFR_CUDA(cudaMemcpyAsync(st + offB0, p.B0, bb, cudaMemcpyHostToDevice, sv.stream));
        B0 = reinterpret_cast<const double*>(st + offB0);
      }
      if (U) U = reinterpret_cast<double*>(st + offU);
      if (V) V = reinterpret_cast<double*>(st + offV);
      if (B) B = reinterpret_cast<double*>(st + offB);
    }
    if (p.B0) {
      // the projector forms (B G B)^{-1/2}, i.e. it needs B = B^T (Algorithm 4 takes B_0 in SPD_r;
      // Lemma 1 needs only rank(B_0) = r, so an indefinite symmetric B_0 is accepted)
      std::vector<double> hb((size_t)p.r * p.r);
      if (p.mem == SFR_MEM_HOST) memcpy(hb.data(), p.B0, bb);
      else SFR_CUDA(cudaMemcpy(hb.data(), p.B0, bb, cudaMemcpyDeviceToHost));
      double amax = 0.0, asym = 0.0;
      for (int i = 0; i < p.r; ++i)
        for (int j = 0; j < p.r; ++j) {
          amax = std::max(amax, std::fabs(hb[i * p.r + j]));
          asym = std::max(asym, std::fabs(hb[i * p.r + j] - hb[j * p.r + i]));
        }
      if (!(amax > 0.0 && amax < 1e300) || asym > 1e-12 * amax) {
        *err = "B0 must be a finite, nonzero symmetric matrix";
        res->status = SFR_E_INVAL;
        return SFR_E_INVAL;
      }
    }
    DevState out = sv.run_full(p, Mdev, V0, B0, U, B, V);
    res->iters = out.iter;
    res->rel_change = out.res;
    res->status = (sfr_status)out.status;
    res->lambda_min_B = NAN;
    const bool ok = res->status == SFR_OK || res->status == SFR_E_NOCONV;
    if (p.mem == SFR_MEM_HOST && ok) {
      if (res->U) SFR_CUDA(cudaMemcpyAsync(res->U, U, ub, cudaMemcpyDeviceToHost, sv.stream));
      if (res->V) SFR_CUDA(cudaMemcpyAsync(res->V, V, vb, cudaMemcpyDeviceToHost, sv.stream));
      if (res->B) SFR_CUDA(cudaMemcpyAsync(res->B, B, bb, cudaMemcpyDeviceToHost, sv.stream));
      SFR_CUDA(cudaStreamSynchronize(sv.stream));
    }
    if (ok && res->B) {
      std::vector<double> hb((size_t)p.r * p.r);
      if (p.mem == SFR_MEM_HOST) memcpy(hb.data(), res->B, bb);
      else SFR_CUDA(cudaMemcpy(hb.data(), res->B, bb, cudaMemcpyDeviceToHost));
      res->lambda_min_B = host_lambda_min(hb, p.r);
    }
    if (res->status != SFR_OK) {
      *err = res->status == SFR_E_NOCONV  ? fmt("B still changing by %.3e after %d iterations", out.res, out.iter)
             : res->status == SFR_E_RANK ? fmt("rank-deficient thin product at iteration %d", out.iter + 1)
             : res->status == SFR_E_NAN  ? fmt("non-finite value at iteration %d", out.iter + 1)
                                         : fmt("FixedRankOptFull failed with status %d", (int)res->status);
    }
    return res->status;
  } catch (const Fail& f) {
    *err = f.msg;
    res->status = f.code;
    return f.code;
  }
}

// Device bytes one request needs while it runs (workspace, plus staging for host buffers and
// the FR-Nys block buffers), from the same planner the solve uses.
static size_t request_bytes(const sfr_problem& p, int num_sms) {
  const bool fp64 = p.precision == SFR_PREC_FP64;
  size_t total = 0;
  // (the aligned copy of M is planned from M's own rows where the solve reads them in place)
  auto one = [&](int64_t m, int64_t n, int64_t ldm, const void* M) {
    Shape s = plan_shape(m, n, ldm, p.r, num_sms);
    const bool tc = !fp64 && tc_supported(s, p.m_dtype, ldm);
    if (tc) tc_plan(&s, num_sms);
    plan_mcopy(&s, fp64, tc, p.m_dtype, M);
    return carve(s, fp64, nullptr, nullptr, tc);
  };
  if (p.nys_l) {  // the two block solves run concurrently on gathered (dense) blocks
    total = one(p.m, p.nys_l, p.nys_l, nullptr) + one(p.nys_l, p.n, p.n, nullptr);
    total += dtype_size(p.m_dtype) * (size_t)(p.m * p.nys_l + p.nys_l * p.n) + 8 * (size_t)(2 * p.m + 2 * p.nys_l + p.n) * p.r;
  } else if (p.mem == SFR_MEM_DEVICE) {
    total = one(p.m, p.n, p.ldm, p.M);
  } else {
    total = one(p.m, p.n, p.ldm, nullptr);  // the staging copy keeps ldm
  }
  if (p.mem == SFR_MEM_HOST) total += dtype_size(p.m_dtype) * (size_t)(p.m * p.ldm) + 16 * (size_t)p.m * p.n;
  return total;
}

// The grouped engine's side of the queue: the oldest batched request that the free budget admits
// (passing over one that does not fit yet at most kMaxPassOver times, as the slots do).
static bool batch_take(sfr_ctx* ctx, BatchJob* job, bool block, int num_sms) {
  constexpr int kMaxPassOver = 64;
  std::unique_lock<std::mutex> lk(ctx->mu);
  for (;;) {
    auto pick = ctx->bqueue.end();
    size_t need = 0;
    for (auto it = ctx->bqueue.begin(); it != ctx->bqueue.end(); ++it) {
      const size_t want = request_bytes((*it)->prob, num_sms);
      if (!ctx->budget || ctx->in_use + want <= ctx->budget) {
        pick = it;
        need = want;
        break;
      }
      if ((*it)->passed_over >= kMaxPassOver) break;
    }
    if (pick != ctx->bqueue.end()) {
      for (auto it = ctx->bqueue.begin(); it != pick; ++it) ++(*it)->passed_over;
      std::shared_ptr<Request> rq = *pick;
      ctx->bqueue.erase(pick);
      ctx->in_use += need;
      job->prob = rq->prob;
      job->res = rq->res;
      job->bytes = need;
      job->token = rq.get();  // kept alive by ctx->live until polled
      return true;
    }
    if (!block) return false;
    if (ctx->stopping && ctx->bqueue.empty()) return false;
    ctx->cv_work.wait(lk);
  }
}

static void batch_done(sfr_ctx* ctx, BatchJob& job, sfr_status st, const std::string& msg) {
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->in_use -= job.bytes;
    Request* rq = static_cast<Request*>(job.token);
    job.res->status = st;
    rq->status = st;
    rq->finished = true;
    if (st < 0) ctx->last_error = msg;
  }
  ctx->cv_done.notify_all();
  ctx->cv_work.notify_all();
}

// One slot: take the oldest request once the HBM budget admits it, solve it on this slot's
// stream, release its workspace share, take the next (continuous batching of independent solves).
static void worker_main(sfr_ctx* ctx, int slot) {
  cudaSetDevice(ctx->device);
  Solver& sv = *ctx->slot_solvers[slot];
  for (;;) {
    std::shared_ptr<Request> rq;
    size_t need = 0;
    {
      std::unique_lock<std::mutex> lk(ctx->mu);
      for (;;) {
        if (ctx->queue.empty()) {
          if (ctx->stopping) return;
          ctx->cv_work.wait(lk);
          continue;
        }
        // requests that can never fit the budget fail at once
        bool refused = false;
        for (auto it = ctx->queue.begin(); it != ctx->queue.end(); ++it) {
          const size_t want = request_bytes((*it)->prob, sv.num_sms);
          if (ctx->budget && want > ctx->budget) {
            std::shared_ptr<Request> bad = *it;
            ctx->queue.erase(it);
            bad->status = SFR_E_NOMEM;
            bad->res->status = SFR_E_NOMEM;
            bad->finished = true;
            ctx->last_error = fmt("request needs %zu bytes; the HBM budget is %zu", want, ctx->budget);
            refused = true;
            break;
          }
        }
        if (refused) {
          ctx->cv_done.notify_all();
          continue;
        }
        // the oldest request that fits the free budget; a request that does not fit yet is passed
        // over by later, smaller ones at most kMaxPassOver times, after which admission waits for it
        // (so a large request cannot be starved by a stream of small ones)
        constexpr int kMaxPassOver = 64;
        auto pick = ctx->queue.end();
        for (auto it = ctx->queue.begin(); it != ctx->queue.end(); ++it) {
          const size_t want = request_bytes((*it)->prob, sv.num_sms);
          if (!ctx->budget || ctx->in_use + want <= ctx->budget) {
            pick = it;
            need = want;
            break;
          }
          if ((*it)->passed_over >= kMaxPassOver) break;  // this one goes next: wait for memory
        }
        if (pick == ctx->queue.end()) {
          ctx->cv_work.wait(lk);  // wait for a running request to release memory
          continue;
        }
        for (auto it = ctx->queue.begin(); it != pick; ++it) ++(*it)->passed_over;
        rq = *pick;
        ctx->queue.erase(pick);
        break;
      }
      ctx->in_use += need;
    }
    std::string err;
    sfr_status st = solve_with(sv, rq->prob, rq->res, &err);
    if (ctx->budget) {  // with a budget the slot keeps no memory between requests
      sv.graph_key.clear();
      if (sv.graph) {
        cudaGraphExecDestroy(sv.graph);
        sv.graph = nullptr;
      }
      sv.work.release(&sv.held);
      sv.staging.release(&sv.held);
      sv.nys.release(&sv.held);
      if (sv.aux) {
        sv.aux->graph_key.clear();
        sv.aux->work.release(&sv.held);  // reserved against this slot's count
      }
    }
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->in_use -= need;
      rq->status = st;
      rq->finished = true;
      if (st < 0) ctx->last_error = err;
    }
    ctx->cv_done.notify_all();
    ctx->cv_work.notify_all();
  }
}

extern "C" {

const char* sfr_version(void) { return "libsfr 0.1 (sm_103a)"; }

const char* sfr_last_error(const sfr_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  // serving slots write the message from their threads: hand out a copy taken under the lock,
  // valid until this thread's next call
  static thread_local std::string copy;
  {
    std::lock_guard<std::mutex> lk(const_cast<sfr_ctx*>(ctx)->mu);
    copy = ctx->last_error;
  }
  return copy.c_str();
}

sfr_status sfr_create(sfr_ctx** out, const sfr_config* cfg) {
  if (!out || !cfg) {
    g_create_error = "null argument";
    return SFR_E_INVAL;
  }
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    g_create_error = fmt("no CUDA device %d (%s)", cfg->device, cudaGetErrorString(e));
    cudaGetLastError();
    return e != cudaSuccess ? SFR_E_CUDA : SFR_E_INVAL;
  }
  auto ctx = std::make_unique<sfr_ctx>();
  ctx->device = cfg->device;
  ctx->max_slots = cfg->max_slots > 0 ? std::min(cfg->max_slots, 64) : 8;
  try {
    SFR_CUDA(cudaSetDevice(cfg->device));
    cudaDeviceProp prop;
    SFR_CUDA(cudaGetDeviceProperties(&prop, cfg->device));
    if (cfg->cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
      SFR_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    ctx->budget = cfg->hbm_budget_bytes;
    auto make_solver = [&](cudaStream_t stream, bool main) {
      auto sv = std::make_unique<Solver>();
      sv->device = cfg->device;
      sv->num_sms = prop.multiProcessorCount;
      sv->stream = stream;
      sv->budget = main ? cfg->hbm_budget_bytes : 0;  // slots are admitted by the context's budget
      sv->profile = main && cfg->profile != 0;
      sv->profile_pass_only = cfg->profile == 2;
      sv->count_stats = main;
      SFR_CUDA(cudaMallocHost(&sv->host_state, sizeof(DevState)));
      return sv;
    };
    ctx->solver = make_solver(ctx->stream, true);
    for (int w = 0; w < ctx->max_slots; ++w) {
      cudaStream_t st;
      SFR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      ctx->slot_streams.push_back(st);
      ctx->slot_solvers.push_back(make_solver(st, false));
    }
  } catch (const Fail& f) {
    g_create_error = f.msg;
    return f.code;
  }
  sfr_ctx* raw = ctx.release();
  for (int w = 0; w < raw->max_slots; ++w) raw->workers.emplace_back(worker_main, raw, w);
  if (cfg->max_batch > 0) {
    raw->max_batch = std::min(cfg->max_batch, 1024);
    const int sms = raw->solver->num_sms;
    raw->batch = batch_create(
        raw->device, raw->max_batch, [raw, sms](BatchJob* j, bool block) { return batch_take(raw, j, block, sms); },
        [raw](BatchJob& j, sfr_status st, const std::string& m) { batch_done(raw, j, st, m); });
  }
  *out = raw;
  return SFR_OK;
}

sfr_status sfr_solve(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res) {
  if (!ctx) return SFR_E_INVAL;
  std::string why;
  sfr_status v = validate(prob, res, &why);
  if (v != SFR_OK) {
    ctx_set_error(ctx, why);
    if (res) res->status = v;
    return v;
  }
  std::string err;
  sfr_status s = solve_with(*ctx->solver, *prob, res, &err);
  if (s < 0) ctx_set_error(ctx, err);
  return s;
}

sfr_status sfr_fixed_rank_opt_full(sfr_ctx* ctx, const sfr_opt_full_problem* prob, sfr_opt_full_result* res) {
  if (!ctx) return SFR_E_INVAL;
  std::string why;
  sfr_status v = validate_full(prob, res, &why);
  if (v != SFR_OK) {
    ctx_set_error(ctx, why);
    if (res) res->status = v;
    return v;
  }
  std::string err;
  sfr_status s = full_with(*ctx->solver, *prob, res, &err);
  if (s < 0) ctx_set_error(ctx, err);
  return s;
}

sfr_status sfr_submit(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res, uint64_t* ticket) {
  if (!ctx || !ticket) return SFR_E_INVAL;
  std::string why;
  sfr_status v = validate(prob, res, &why);
  if (v != SFR_OK) {
    ctx_set_error(ctx, why);
    if (res) res->status = v;
    return v;
  }
  auto rq = std::make_shared<Request>();
  rq->prob = *prob;
  rq->res = res;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    const bool batched = ctx->batch && batch_eligible(*prob);
    auto& q = batched ? ctx->bqueue : ctx->queue;
    const int limit = batched ? 4 * ctx->max_batch : 64 * ctx->max_slots;
    if ((int)q.size() >= limit) {
      ctx->last_error = "request queue full";
      return SFR_E_BUSY;
    }
    rq->ticket = ctx->next_ticket++;
    res->status = SFR_PENDING;
    q.push_back(rq);
    ctx->live[rq->ticket] = rq;
    *ticket = rq->ticket;
  }
  ctx->cv_work.notify_all();
  return SFR_OK;
}

sfr_status sfr_poll(sfr_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
  if (!ctx) return SFR_E_INVAL;
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto it = ctx->live.find(ticket);
  if (it == ctx->live.end()) {
    ctx->last_error = fmt("unknown ticket %llu", (unsigned long long)ticket);
    return SFR_E_INVAL;
  }
  std::shared_ptr<Request> rq = it->second;
  auto ready = [&] { return rq->finished; };
  if (timeout_us < 0) {
    ctx->cv_done.wait(lk, ready);
  } else if (timeout_us > 0) {
    if (!ctx->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return SFR_E_TIMEOUT;
  } else if (!rq->finished) {
    return SFR_PENDING;
  }
  ctx->live.erase(ticket);
  return rq->status;
}

sfr_status sfr_stats(sfr_ctx* ctx, sfr_kernel_stat* out, int32_t count, int32_t reset) {
  if (!ctx || (count > 0 && !out)) return SFR_E_INVAL;
  Solver& sv = *ctx->solver;
  for (int k = 0; k < count && k < SFR_STAT_COUNT; ++k) {
    out[k].launches = sv.launches[k];
    out[k].timed = sv.timed[k];
    out[k].total_ms = sv.total_ms[k];
    out[k].bytes = sv.bytes[k];
  }
  if (reset)
    for (int k = 0; k < SFR_STAT_COUNT; ++k) {
      sv.launches[k] = 0;
      sv.timed[k] = 0;
      sv.total_ms[k] = 0.0;
      sv.bytes[k] = 0.0;
    }
  return SFR_OK;
}

sfr_status sfr_destroy(sfr_ctx* ctx) {
  if (!ctx) return SFR_E_INVAL;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stopping = true;
  }
  ctx->cv_work.notify_all();
  for (auto& w : ctx->workers)
    if (w.joinable()) w.join();
  if (ctx->batch) batch_destroy(ctx->batch);  // answers every request it holds first
  cudaSetDevice(ctx->device);
  ctx->solver.reset();
  ctx->slot_solvers.clear();
  for (cudaStream_t st : ctx->slot_streams) cudaStreamDestroy(st);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return SFR_OK;
}

}  // extern "C"
