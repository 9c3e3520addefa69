// Grouped serving engine (sfr_config.max_batch > 0).
//
// Requests that run the mixed-precision SIMT passes (FR-ADM, device buffers, padded rank <= 32)
// are solved together: every step advances each live problem by one FR-ADM iteration
// (Algorithm 1), and each kernel of the iteration is launched once for all of them.  The engine
// records every problem's launches (launch_k with a LaunchRecorder installed), merges the records
// stage by stage into grouped launches (one per kernel instantiation present), copies the
// per-problem argument tables to the device in one transfer and launches the grouped kernels,
// which run every problem's own grid with its own arguments: each problem computes exactly what
// sfr_solve computes for it, whatever else is in the batch.
//
// Between steps the engine admits queued requests as memory and capacity allow (their first
// iteration runs as one grouped "first" step of its own), reads all problems' device states with
// one copy (pipelined one step behind, so the GPU is not idle while the host decides), retires
// the converged ones (their factors, S and L are written by their own output kernels) and hands
// the results back.  Each problem's workspace comes from the stream-ordered allocator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "sfr_internal.h"

namespace sfr {

namespace {

struct BatchFail {
  std::string msg;
};

#define BT_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) throw BatchFail{std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// Start state of one problem: DevState, B_0 = I, both warm-start eigenbases = I (Algorithm 1's
// initial values; Y_1 = 0 is a memset).
__global__ void batch_init_kernel(DevState* st, DevState init, double* B, float* Qu, float* Qv, int rp) {
  pdl_enter();
  if (threadIdx.x == 0) *st = init;
  for (int e = threadIdx.x; e < rp * rp; e += blockDim.x) {
    const bool d = (e / rp) == (e % rp);
    B[e] = d ? 1.0 : 0.0;
    Qu[e] = d ? 1.f : 0.f;
    Qv[e] = d ? 1.f : 0.f;
  }
}

struct BProblem {
  BatchJob job;
  Shape s{};
  Buffers b{}, after_first{};
  void* mem = nullptr;
  int slot = -1;
  uint64_t admitted_at = 0;  // snapshot sequence number when admitted
  bool first_done = false;   // its first iteration has been launched
  int steps = 0;             // iterations launched for it
  cudaEvent_t fin = nullptr; // its output kernels have finished
  DevState last{};           // the state it retired with
};

constexpr int kStages = 11;
using StageRecs = std::vector<std::vector<RecordedLaunch>>;  // [stage] -> launches in order

}  // namespace

class BatchEngine {
 public:
  BatchEngine(int device, int capacity, std::function<bool(BatchJob*, bool)> take,
              std::function<void(BatchJob&, sfr_status, const std::string&)> done)
      : device_(device), cap_(capacity), take_(std::move(take)), done_(std::move(done)) {
    thr_ = std::thread([this] { run(); });
  }
  ~BatchEngine() {
    if (thr_.joinable()) thr_.join();
  }

 private:
  int device_, cap_;
  std::function<bool(BatchJob*, bool)> take_;
  std::function<void(BatchJob&, sfr_status, const std::string&)> done_;
  std::thread thr_;
  cudaStream_t st_ = nullptr;
  DevState* d_states_ = nullptr;
  DevState* h_states_[2] = {};
  cudaEvent_t st_ev_[2] = {};
  uint64_t snap_seq_[2] = {};
  bool snap_valid_[2] = {};
  uint64_t seq_ = 0;
  double* h_B_ = nullptr;  // pinned r x r B of each slot (lambda_min on the host)
  unsigned char* h_tab_[2] = {};
  unsigned char* d_tab_[2] = {};
  size_t tab_cap_ = 0;
  cudaEvent_t tab_ev_[2] = {};
  int parity_ = 0;
  int num_sms_ = 152;
  std::vector<int> free_slots_;
  std::vector<std::unique_ptr<BProblem>> live_, finishing_;

  void setup() {
    BT_CUDA(cudaSetDevice(device_));
    cudaDeviceProp prop;
    BT_CUDA(cudaGetDeviceProperties(&prop, device_));
    num_sms_ = prop.multiProcessorCount;
    BT_CUDA(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    BT_CUDA(cudaMalloc(&d_states_, sizeof(DevState) * cap_));
    for (int i = 0; i < 2; ++i) {
      BT_CUDA(cudaMallocHost(&h_states_[i], sizeof(DevState) * cap_));
      BT_CUDA(cudaEventCreateWithFlags(&st_ev_[i], cudaEventDisableTiming));
      BT_CUDA(cudaEventCreateWithFlags(&tab_ev_[i], cudaEventDisableTiming));
    }
    BT_CUDA(cudaMallocHost(&h_B_, sizeof(double) * kMaxRank * kMaxRank * cap_));
    cudaMemPool_t pool;  // keep freed workspace in the pool instead of returning it at each sync
    if (cudaDeviceGetDefaultMemPool(&pool, device_) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    for (int i = cap_ - 1; i >= 0; --i) free_slots_.push_back(i);
  }

  void teardown() {
    cudaSetDevice(device_);
    if (st_) cudaStreamSynchronize(st_);
    for (int i = 0; i < 2; ++i) {
      if (h_states_[i]) cudaFreeHost(h_states_[i]);
      if (h_tab_[i]) cudaFreeHost(h_tab_[i]);
      if (d_tab_[i]) cudaFree(d_tab_[i]);
      if (st_ev_[i]) cudaEventDestroy(st_ev_[i]);
      if (tab_ev_[i]) cudaEventDestroy(tab_ev_[i]);
    }
    if (h_B_) cudaFreeHost(h_B_);
    if (d_states_) cudaFree(d_states_);
    if (st_) cudaStreamDestroy(st_);
  }

  // Workspace, start state, ||M||, P = M[:, :r]; nullptr when the problem could not be set up
  // (it has been answered already).
  BProblem* admit(BatchJob& job) {
    try {
      return admit_or_throw(job);
    } catch (const BatchFail& f) {
      cudaGetLastError();
      done_(job, SFR_E_CUDA, f.msg);
      return nullptr;
    }
  }

  BProblem* admit_or_throw(BatchJob& job) {
    auto q = std::make_unique<BProblem>();
    q->job = job;
    const sfr_problem& p = job.prob;
    q->s = plan_shape(p.m, p.n, p.ldm, p.r, num_sms_);
    plan_mcopy(&q->s, false, false, p.m_dtype, p.M);
    const size_t bytes = carve(q->s, false, nullptr, nullptr);
    if (cudaMallocAsync(&q->mem, bytes, st_) != cudaSuccess) {
      cudaGetLastError();
      done_(q->job, SFR_E_NOMEM, "cudaMallocAsync failed for a batched request's workspace");
      return nullptr;
    }
    q->slot = free_slots_.back();
    free_slots_.pop_back();
    struct Undo {  // give the slot and the workspace back unless the problem goes live
      BatchEngine* e;
      BProblem* q;
      bool armed = true;
      ~Undo() {
        if (!armed) return;
        e->free_slots_.push_back(q->slot);
        cudaFreeAsync(q->mem, e->st_);
        cudaGetLastError();
      }
    } undo{this, q.get()};
    Buffers& b = q->b;
    carve(q->s, false, q->mem, &b);
    b.st = d_states_ + q->slot;
    b.M = p.M;
    if (q->s.mc_ld > 0) {  // rows of M not 16-byte aligned: the passes read an aligned copy
      BT_CUDA(launch_copy_m(q->s, p.M, p.ldm, b.Mc, st_));
      b.M = b.Mc;
      q->s.ldm = q->s.mc_ld;
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
    BT_CUDA(launch_pdl(batch_init_kernel, 1, 256, 0, st_, b.st, h, b.B, b.Qeig_u, b.Qeig_v, q->s.rp));
    BT_CUDA(cudaMemsetAsync(b.Y[0], 0, 4 * (size_t)q->s.m * b.ldy, st_));  // Y_1 = 0
    BT_CUDA(launch_norm_m(q->s, b, st_));
    // Sweep grid: with many problems per launch, each CTA takes 8 row blocks of its column split
    // (the cp.async pipeline then runs over them) instead of the one-problem grid sfr_solve tunes.
    // The sweep's partials are per row block and split, so its results do not depend on this.
    q->s.mx_grid_x = (int)std::max<int64_t>(1, ((q->s.m + 63) / 64 + 7) / 8);
    BT_CUDA(launch_init_p(q->s, b, false, st_));  // X_1 = M, V_1 = I_{n x r}: P = M[:, :r]
    q->admitted_at = seq_;
    BProblem* raw = q.get();
    live_.push_back(std::move(q));
    undo.armed = false;
    return raw;
  }

  // The launches of one iteration of q (the first, or a later one), recorded stage by stage;
  // then q's buffer bookkeeping advances as after a launch (same order as sfr_solve).
  void record_iteration(BProblem& q, bool first, StageRecs& out) {
    out.assign(kStages, {});
    Shape& s = q.s;
    Buffers& b = q.b;
    LaunchRecorder rec;
    auto stage = [&](int k, auto&& f) {
      rec.recs.clear();
      g_recorder = &rec;
      const cudaError_t e = f();
      g_recorder = nullptr;
      if (e != cudaSuccess) throw BatchFail{std::string("recording a batched launch: ") + cudaGetErrorString(e)};
      out[k] = std::move(rec.recs);
    };
    if (first) stage(1, [&] { return launch_gram_p(s, b, false, false, st_); });
    stage(2, [&] { return launch_rxr(s, b, false, st_, false); });   // T_U = B (B G_P B)^{-1/2}
    stage(3, [&] { return launch_apply_u(s, b, false, first, st_); });  // U = P T_U
    const int u_new = 1 - b.u_cur;
    // W = (Delta^T P) T_U + C_old H after the first iteration, as sfr_solve forms it
    stage(4, [&] { return launch_wpass(s, b, false, first, u_new, st_, !first); });
    stage(5, [&] { return launch_wfinal(s, b, false, first, st_, !first); });
    stage(6, [&] { return launch_rxr(s, b, true, st_, false); });    // T_V, B, T_C
    stage(7, [&] { return launch_apply_v(s, b, false, st_); });
    stage(8, [&] { return launch_sweep(s, b, false, u_new, st_); });
    stage(9, [&] { return launch_iter_end(s, b, false, st_); });
    stage(10, [&] { return launch_gram_p(s, b, false, true, st_); });
    b.u_cur = u_new;
    std::swap(b.Y[0], b.Y[1]);
    ++q.steps;
  }

  // Launches the recorded iterations of all problems as grouped kernels: for each stage and
  // position j in it, one grouped launch per (kernel, block size, shared memory) present.
  void launch_merged(std::vector<StageRecs>& recs) {
    if (recs.empty()) return;
    struct Group {
      const RecordedLaunch* first;
      std::vector<const RecordedLaunch*> items;
    };
    std::vector<Group> groups;
    for (int k = 0; k < kStages; ++k) {
      size_t jmax = 0;
      for (auto& r : recs) jmax = std::max(jmax, r[k].size());
      for (size_t j = 0; j < jmax; ++j) {
        const size_t g0 = groups.size();
        for (auto& r : recs) {
          if (j >= r[k].size()) continue;
          const RecordedLaunch& x = r[k][j];
          size_t g = g0;
          for (; g < groups.size(); ++g)
            if (groups[g].first->kind == x.kind && groups[g].first->block == x.block && groups[g].first->smem == x.smem)
              break;
          if (g == groups.size()) groups.push_back(Group{&x, {}});
          groups[g].items.push_back(&x);
        }
      }
    }
    // table layout per group: starts[count + 1] (int), then the entries, each part 256-aligned
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t total = 0;
    std::vector<size_t> off(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) {
      off[g] = total;
      total += al(sizeof(int) * (groups[g].items.size() + 1)) + al(groups[g].first->entry_size * groups[g].items.size());
    }
    const int par = parity_;
    if (total > tab_cap_) {
      BT_CUDA(cudaStreamSynchronize(st_));
      for (int i = 0; i < 2; ++i) {
        if (h_tab_[i]) cudaFreeHost(h_tab_[i]);
        if (d_tab_[i]) cudaFree(d_tab_[i]);
        h_tab_[i] = nullptr;
        d_tab_[i] = nullptr;
      }
      tab_cap_ = std::max(total * 2, size_t(1) << 20);
      for (int i = 0; i < 2; ++i) {
        BT_CUDA(cudaMallocHost(&h_tab_[i], tab_cap_));
        BT_CUDA(cudaMalloc(&d_tab_[i], tab_cap_));
      }
    } else {
      BT_CUDA(cudaEventSynchronize(tab_ev_[par]));  // the copy that last read this host buffer is done
    }
    unsigned char* h = h_tab_[par];
    std::vector<unsigned> totals(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) {
      int* starts = reinterpret_cast<int*>(h + off[g]);
      unsigned char* ent = h + off[g] + al(sizeof(int) * (groups[g].items.size() + 1));
      int acc = 0;
      const size_t es = groups[g].first->entry_size;
      for (size_t i = 0; i < groups[g].items.size(); ++i) {
        const RecordedLaunch& x = *groups[g].items[i];
        starts[i] = acc;
        acc += (int)(x.grid.x * x.grid.y);
        std::memcpy(ent + i * es, x.entry.data(), es);
      }
      starts[groups[g].items.size()] = acc;
      totals[g] = (unsigned)acc;
    }
    BT_CUDA(cudaMemcpyAsync(d_tab_[par], h, total, cudaMemcpyHostToDevice, st_));
    BT_CUDA(cudaEventRecord(tab_ev_[par], st_));
    for (size_t g = 0; g < groups.size(); ++g) {
      const int* starts = reinterpret_cast<const int*>(d_tab_[par] + off[g]);
      const void* ent = d_tab_[par] + off[g] + al(sizeof(int) * (groups[g].items.size() + 1));
      if (totals[g] == 0) continue;
      BT_CUDA(groups[g].first->launch_grouped(starts, ent, (int)groups[g].items.size(), totals[g],
                                              groups[g].first->block, groups[g].first->smem, st_));
    }
    parity_ ^= 1;
  }

  // Output of a converged (or failed) problem: U, V, B, S / L from the buffers of its last
  // iteration, B also to the host for lambda_min; completion is signalled by q.fin.
  void retire(BProblem& q, const DevState& ds) {
    q.last = ds;
    const int K = ds.iter;
    Buffers fin = q.after_first;  // the buffers of iteration K (two iterations alternate them)
    if (K >= 2 && K % 2 == 0) fin.u_cur = 1 - q.after_first.u_cur;
    else std::swap(fin.Y[0], fin.Y[1]);
    sfr_result* res = q.job.res;
    const int r = q.s.r;
    if (ds.status == SFR_OK || ds.status == SFR_E_NOCONV) {
      BT_CUDA(launch_export_factors(q.s, fin, false, fin.u_cur, res->U, res->V, st_));
      double* hB = h_B_ + (size_t)q.slot * kMaxRank * kMaxRank;
      BT_CUDA(cudaMemcpy2DAsync(hB, 8 * r, fin.B, 8 * q.s.rp, 8 * r, r, cudaMemcpyDeviceToHost, st_));
      if (res->B)
        BT_CUDA(cudaMemcpy2DAsync(res->B, 8 * r, fin.B, 8 * q.s.rp, 8 * r, r, cudaMemcpyDeviceToDevice, st_));
      if (res->S || res->L)
        BT_CUDA(launch_finalize(q.s, fin, false, fin.u_cur, res->S, res->s_dtype, res->lds, res->L, st_));
    }
    BT_CUDA(cudaEventCreateWithFlags(&q.fin, cudaEventDisableTiming));
    BT_CUDA(cudaEventRecord(q.fin, st_));
  }

  // Answers the retired problems whose output kernels have finished; frees their workspace.
  void reap(bool wait) {
    for (size_t i = 0; i < finishing_.size();) {
      BProblem& q = *finishing_[i];
      if (wait) BT_CUDA(cudaEventSynchronize(q.fin));
      else if (cudaEventQuery(q.fin) != cudaSuccess) {
        cudaGetLastError();
        ++i;
        continue;
      }
      cudaEventDestroy(q.fin);
      sfr_result* res = q.job.res;
      const DevState& ds = q.last;
      res->iters = ds.iter;
      res->rel_residual = ds.res;
      res->status = (sfr_status)ds.status;
      res->path = 0;
      res->lambda_min_B = NAN;
      if (ds.status == SFR_OK || ds.status == SFR_E_NOCONV) {
        const int r = q.s.r;
        std::vector<double> hb(h_B_ + (size_t)q.slot * kMaxRank * kMaxRank,
                               h_B_ + (size_t)q.slot * kMaxRank * kMaxRank + (size_t)r * r);
        res->lambda_min_B = host_lambda_min(hb, r);
      }
      cudaFreeAsync(q.mem, st_);
      free_slots_.push_back(q.slot);
      const sfr_status stt = (sfr_status)ds.status;
      std::string msg;
      if (stt == SFR_E_NOCONV) msg = "batched request: no convergence within max_iter";
      else if (stt == SFR_E_RANK) msg = "batched request: rank-deficient thin product";
      else if (stt == SFR_E_NAN) msg = "batched request: non-finite value";
      else if (stt == SFR_E_CUDA) msg = "batched request: the device state never reported a stop";
      else if (stt != SFR_OK) msg = "batched request failed";
      done_(q.job, stt, msg);
      finishing_.erase(finishing_.begin() + i);
    }
  }

  // Reads a snapshot of the states (taken after an earlier step) and retires what it shows done.
  void process_snapshot(int which) {
    if (!snap_valid_[which]) return;
    BT_CUDA(cudaEventSynchronize(st_ev_[which]));
    snap_valid_[which] = false;
    const DevState* hs = h_states_[which];
    for (size_t i = 0; i < live_.size();) {
      BProblem& q = *live_[i];
      const sfr_problem& p = q.job.prob;
      const int budget = (p.fixed_iters > 0 ? p.fixed_iters : p.max_iter) + 8;
      const bool seen = q.first_done && q.admitted_at < snap_seq_[which];
      if (seen && (hs[q.slot].done || q.steps > budget)) {
        DevState ds = hs[q.slot];
        if (!ds.done) ds.status = SFR_E_CUDA;  // its iteration count never reached the stop rule
        retire(q, ds);
        finishing_.push_back(std::move(live_[i]));
        live_.erase(live_.begin() + i);
      } else {
        ++i;
      }
    }
  }

  void fail_all(const std::string& msg) {
    cudaGetLastError();
    cudaStreamSynchronize(st_);
    cudaGetLastError();
    for (auto* v : {&live_, &finishing_})
      for (auto& q : *v) {
        q->job.res->status = SFR_E_CUDA;
        if (q->mem) cudaFree(q->mem);
        free_slots_.push_back(q->slot);
        done_(q->job, SFR_E_CUDA, msg);
      }
    live_.clear();
    finishing_.clear();
  }

  void run() {
    try {
      setup();
    } catch (const BatchFail& f) {
      BatchJob job;  // answer every request with the failure
      while (take_(&job, true)) done_(job, SFR_E_CUDA, f.msg);
      return;
    }
    for (;;) {
      try {
        std::vector<BProblem*> fresh;  // admitted now: their first iteration is still to run
        if (live_.empty() && finishing_.empty()) {
          BatchJob job;
          if (!take_(&job, true)) break;  // stopping and nothing queued
          if (BProblem* q = admit(job)) fresh.push_back(q);
        }
        while ((int)(live_.size() + finishing_.size()) < cap_) {
          BatchJob job;
          if (!take_(&job, false)) break;
          if (BProblem* q = admit(job)) fresh.push_back(q);
        }
        if (live_.empty() && finishing_.empty()) continue;  // nothing could be admitted
        // one grouped step: the first iteration of the newly admitted problems, then one
        // iteration of every problem already running
        std::vector<StageRecs> recs;
        for (BProblem* q : fresh) {
          recs.emplace_back();
          record_iteration(*q, true, recs.back());
          q->after_first = q->b;
        }
        launch_merged(recs);
        recs.clear();
        for (auto& q : live_)
          if (q->first_done) {
            recs.emplace_back();
            record_iteration(*q, false, recs.back());
          }
        launch_merged(recs);
        for (BProblem* q : fresh) q->first_done = true;
        // snapshot of every slot's state after this step; decide on the previous one meanwhile
        const int w = (int)(seq_ & 1);
        ++seq_;
        BT_CUDA(cudaMemcpyAsync(h_states_[w], d_states_, sizeof(DevState) * cap_, cudaMemcpyDeviceToHost, st_));
        BT_CUDA(cudaEventRecord(st_ev_[w], st_));
        snap_seq_[w] = seq_;
        snap_valid_[w] = true;
        process_snapshot(w ^ 1);
        reap(live_.empty());  // nothing left to step: wait for the output kernels instead of spinning
      } catch (const BatchFail& f) {
        fail_all(f.msg);
      }
    }
    // drain: every admitted problem finishes (the loop above only ends with nothing live)
    try {
      reap(true);
    } catch (const BatchFail& f) {
      fail_all(f.msg);
    }
    teardown();
  }
};

BatchEngine* batch_create(int device, int capacity, std::function<bool(BatchJob*, bool)> take,
                          std::function<void(BatchJob&, sfr_status, const std::string&)> done) {
  return new BatchEngine(device, capacity, std::move(take), std::move(done));
}

void batch_destroy(BatchEngine* e) { delete e; }

bool batch_eligible(const sfr_problem& p) {
  return p.precision == SFR_PREC_MIXED && p.nys_l == 0 && p.mem == SFR_MEM_DEVICE && pad_rank(p.r) <= 32;
}

}  // namespace sfr
