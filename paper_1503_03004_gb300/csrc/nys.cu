// FR-Nys (Algorithm 2): Nystrom sub-sampling around two FR-ADM solves.
//
//   M~ = rows of M shuffled by perm (M~[i] = M[perm[i]]),
//   (L_L, S_L) = FR-ADM(M~[:, :l], r),   (L_T, S_T) = FR-ADM(M~[:l, :], r),
//   L = L_L (L_L[:l, :l])^+ L_T,   S = M~ - L   (returned in M's row order).
//
// Both block solves return their factors L_L = U_L B_L V_L^T, L_T = U_T B_T V_T^T.
// With A = U_L[:l] B_L (l x r, full column rank) and V_L orthonormal,
//   (L_L[:l, :l])^+ = (A V_L^T)^+ = V_L (A^T A)^{-1} A^T,
// so L = U_L B_L (A^T A)^{-1} B_L (U_L[:l]^T U_T) B_T V_T^T = U_L Core V_T^T,
// an r x r core; no l x l pseudo-inverse is formed.  The m x n pass then writes
// S = M - (U_L Core) V_T^T row by row in M's original order.  With the SVD
// Core = A diag(sigma) C^T (r x r, one-sided Jacobi on the host), L = (U_L A) diag(sigma) (V_T C)^T
// is returned in the polar form of the other entry points: U = U_L A, B = diag(sigma),
// V = V_T C, U and V orthonormal.  The two block solves run concurrently, the second on an
// auxiliary solver with its own stream and workspace.
#include <algorithm>
#include <cmath>
#include <thread>
#include <string>
#include <vector>

#include "sfr_internal.h"

namespace sfr {

struct Solver;
DevState solver_run(Solver& sv, const sfr_problem& p, const void* Mdev, double* U, double* B, double* V, void* S,
                    sfr_dtype s_dtype, int64_t lds, void* L);
void* solver_nys_block(Solver& sv, size_t bytes);
cudaStream_t solver_stream(Solver& sv);
bool solver_last_tc(const Solver& sv);
Solver* solver_aux(Solver& sv);
bool solver_reserve(Solver& sv, const sfr_problem& p, const void* Mdev, size_t* held, size_t budget);
size_t* solver_held(Solver& sv);
size_t solver_budget(const Solver& sv);

namespace {

template <typename T>
__global__ void gather_cols_kernel(const T* __restrict__ M, int64_t ldm, const int64_t* __restrict__ perm, int64_t m,
                                   int64_t l, T* __restrict__ out) {
  pdl_enter();
  // out[i][j] = M[perm[i]][j], j < l   (left block of M~, m x l, dense)
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * l) return;
  int64_t i = idx / l, j = idx % l;
  out[idx] = M[perm[i] * ldm + j];
}

template <typename T>
__global__ void gather_rows_kernel(const T* __restrict__ M, int64_t ldm, const int64_t* __restrict__ perm, int64_t l,
                                   int64_t n, T* __restrict__ out) {
  pdl_enter();
  // out[i][j] = M[perm[i]][j], i < l   (top block of M~, l x n, dense)
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * n) return;
  int64_t i = idx / n, j = idx % n;
  out[idx] = M[perm[i] * ldm + j];
}

// flag = 1 when some perm[i] lies outside [0, m): checked before any gather or scatter.
__global__ void check_perm_kernel(const int64_t* __restrict__ perm, int64_t m, int* __restrict__ flag) {
  pdl_enter();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (perm[i] < 0 || perm[i] >= m) atomicExch(flag, 1);
}

constexpr int CR = kMaxRank;
constexpr int CLD = CR + 1;

// One CTA: Core = B_L (A^T A)^{-1} B_L (U_L[:l]^T U_T) B_T with A = U_L[:l] B_L.
__global__ void nys_core_kernel(const double* __restrict__ UL, const double* __restrict__ BL,
                                const double* __restrict__ UT, const double* __restrict__ BT, int64_t l, int r,
                                double* __restrict__ core, int* __restrict__ bad) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* G1 = reinterpret_cast<double*>(smem_raw);
  double* G2 = G1 + CR * CLD;
  double* T = G2 + CR * CLD;
  double* Bl = T + CR * CLD;
  const int tid = threadIdx.x;
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double g1 = 0.0, g2 = 0.0;
    for (int64_t i = 0; i < l; ++i) {
      g1 = fma(UL[i * r + a], UL[i * r + b], g1);
      g2 = fma(UL[i * r + a], UT[i * r + b], g2);
    }
    G1[a * CLD + b] = g1;
    G2[a * CLD + b] = g2;
    Bl[a * CLD + b] = BL[a * r + b];
  }
  __syncthreads();
  // T = G1 B_L ; G1 <- B_L T = A^T A
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v = fma(G1[a * CLD + k], Bl[k * CLD + b], v);
    T[a * CLD + b] = v;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v = fma(Bl[a * CLD + k], T[k * CLD + b], v);
    G1[a * CLD + b] = v;
  }
  __syncthreads();
  // T = G2 B_T ; G2 <- B_L T  (right-hand side)
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v = fma(G2[a * CLD + k], BT[k * r + b], v);
    T[a * CLD + b] = v;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v = fma(Bl[a * CLD + k], T[k * CLD + b], v);
    G2[a * CLD + b] = v;
  }
  __syncthreads();
  // Solve (A^T A) X = rhs by Gauss-Jordan with partial pivoting (single thread picks the pivot)
  __shared__ int piv;
  __shared__ int singular;
  if (tid == 0) singular = 0;
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      int p = k;
      double best = fabs(G1[k * CLD + k]);
      for (int i = k + 1; i < r; ++i)
        if (fabs(G1[i * CLD + k]) > best) { best = fabs(G1[i * CLD + k]); p = i; }
      piv = p;
      if (!(best > 1e-300)) singular = 1;
    }
    __syncthreads();
    if (singular) break;
    const int p = piv;
    if (p != k)
      for (int j = tid; j < r; j += blockDim.x) {
        double t = G1[k * CLD + j]; G1[k * CLD + j] = G1[p * CLD + j]; G1[p * CLD + j] = t;
        t = G2[k * CLD + j]; G2[k * CLD + j] = G2[p * CLD + j]; G2[p * CLD + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / G1[k * CLD + k];
    for (int i = tid; i < r; i += blockDim.x) T[i] = G1[i * CLD + k];
    __syncthreads();
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      if (i == k) continue;
      const double f = T[i] * inv;
      G1[i * CLD + j] -= f * G1[k * CLD + j];
      G2[i * CLD + j] -= f * G2[k * CLD + j];
    }
    __syncthreads();
    for (int j = tid; j < r; j += blockDim.x) {
      G1[k * CLD + j] *= inv;
      G2[k * CLD + j] *= inv;
    }
    __syncthreads();
  }
  if (singular) {
    if (tid == 0) *bad = 1;
    return;
  }
  // Core = B_L X
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v = fma(Bl[a * CLD + k], G2[k * CLD + b], v);
    core[a * r + b] = v;
  }
  if (tid == 0) *bad = 0;
}

// Uo[perm[i]][:] = U_L[i][:] Core   (m x r, dense, M's row order; perm == nullptr: identity)
__global__ void nys_rows_kernel(const double* __restrict__ UL, const double* __restrict__ core,
                                const int64_t* __restrict__ perm, int64_t m, int r, double* __restrict__ Uo) {
  pdl_enter();
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * r) return;
  int64_t i = idx / r;
  int b = (int)(idx % r);
  double v = 0.0;
  for (int a = 0; a < r; ++a) v = fma(UL[i * r + a], core[a * r + b], v);
  Uo[(perm ? perm[i] : i) * r + b] = v;
}

// S = M - Uo V_T^T (and optionally L), Algorithm 2's S = M~ - L in M's row order.
template <typename TC, typename TMs, typename TSo>
__global__ void __launch_bounds__(256) nys_residual_kernel(const TMs* __restrict__ M, int64_t m, int64_t n,
                                                           int64_t ldm, const double* __restrict__ Uo,
                                                           const double* __restrict__ VT, int r, TSo* __restrict__ S,
                                                           TSo* __restrict__ L, int64_t lds) {
  pdl_enter();
  __shared__ TC us[8][CR];
  __shared__ TC vs[32][CR + 1];
  const int64_t nbx = (n + 31) / 32;  // 1-D grid over (8-row, 32-column) blocks, columns fastest
  const int64_t i0 = ((int64_t)blockIdx.x / nbx) * 8, j0 = ((int64_t)blockIdx.x % nbx) * 32;
  const int tj = threadIdx.x & 31, ti = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < 8 * r; e += blockDim.x) {
    int ii = e / r, a = e % r;
    us[ii][a] = i0 + ii < m ? (TC)Uo[(i0 + ii) * r + a] : (TC)0;
  }
  for (int e = threadIdx.x; e < 32 * r; e += blockDim.x) {
    int jj = e / r, a = e % r;
    vs[jj][a] = j0 + jj < n ? (TC)VT[(j0 + jj) * r + a] : (TC)0;
  }
  __syncthreads();
  const int64_t i = i0 + ti, j = j0 + tj;
  if (i >= m || j >= n) return;
  TC lv = 0;
  for (int a = 0; a < r; ++a) lv += us[ti][a] * vs[tj][a];
  TC mv;
  if constexpr (std::is_same<TMs, __nv_bfloat16>::value) mv = (TC)__bfloat162float(M[i * ldm + j]);
  else mv = (TC)M[i * ldm + j];
  if (S) S[i * lds + j] = (TSo)(mv - lv);
  if (L) L[i * lds + j] = (TSo)lv;
}

template <typename F>
cudaError_t by_mtype(sfr_dtype dt, const void* M, F&& f) {
  switch (dt) {
    case SFR_F64: return f(static_cast<const double*>(M));
    case SFR_F32: return f(static_cast<const float*>(M));
    case SFR_BF16: return f(static_cast<const __nv_bfloat16*>(M));
    default: return cudaErrorInvalidValue;
  }
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// SVD of the r x r core, K = A diag(sigma) C^T (host, float64), by one-sided (Hestenes) Jacobi:
// plane rotations J applied to the columns of W = K until they are mutually orthogonal, so that
// K C = W with C the product of the rotations; then sigma_j = ||w_j||, a_j = w_j / sigma_j.
// Columns come out sorted by decreasing sigma; a column with sigma = 0 gets a unit vector
// orthogonal to the others, so that A is orthogonal in every case.
void core_svd(const std::vector<double>& K, int r, std::vector<double>& A, std::vector<double>& sig,
              std::vector<double>& C) {
  std::vector<double> W = K;  // row-major r x r
  C.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) C[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < r - 1; ++p)
      for (int q = p + 1; q < r; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < r; ++i) {
          const double wp = W[(size_t)i * r + p], wq = W[(size_t)i * r + q];
          alpha += wp * wp;
          beta += wq * wq;
          gamma += wp * wq;
        }
        if (gamma == 0.0 || std::fabs(gamma) <= 1e-17 * std::sqrt(alpha * beta)) continue;
        off = std::max(off, std::fabs(gamma) / std::sqrt(alpha * beta));
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < r; ++i) {
          double* w = &W[(size_t)i * r];
          const double wp = w[p], wq = w[q];
          w[p] = c * wp - sn * wq;
          w[q] = sn * wp + c * wq;
          double* cc = &C[(size_t)i * r];
          const double cp = cc[p], cq = cc[q];
          cc[p] = c * cp - sn * cq;
          cc[q] = sn * cp + c * cq;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> norms(r);
  for (int j = 0; j < r; ++j) {
    double v = 0.0;
    for (int i = 0; i < r; ++i) v += W[(size_t)i * r + j] * W[(size_t)i * r + j];
    norms[j] = std::sqrt(v);
  }
  std::vector<int> order(r);
  for (int j = 0; j < r; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return norms[a] > norms[b]; });
  const double big = norms[order[0]];
  A.assign((size_t)r * r, 0.0);
  sig.assign(r, 0.0);
  std::vector<double> Cs((size_t)r * r);
  for (int jj = 0; jj < r; ++jj) {
    const int j = order[jj];
    sig[jj] = norms[j];
    for (int i = 0; i < r; ++i) Cs[(size_t)i * r + jj] = C[(size_t)i * r + j];
    if (norms[j] > 1e-300 && norms[j] > 1e-15 * big) {
      for (int i = 0; i < r; ++i) A[(size_t)i * r + jj] = W[(size_t)i * r + j] / norms[j];
    } else {
      sig[jj] = 0.0;
      for (int e = 0; e < r; ++e) {  // first unit vector not in the span of the columns so far
        std::vector<double> v(r, 0.0);
        v[e] = 1.0;
        for (int k = 0; k < jj; ++k) {
          double d = 0.0;
          for (int i = 0; i < r; ++i) d += A[(size_t)i * r + k] * v[i];
          for (int i = 0; i < r; ++i) v[i] -= d * A[(size_t)i * r + k];
        }
        double nv = 0.0;
        for (int i = 0; i < r; ++i) nv += v[i] * v[i];
        nv = std::sqrt(nv);
        if (nv > 0.5) {
          for (int i = 0; i < r; ++i) A[(size_t)i * r + jj] = v[i] / nv;
          break;
        }
      }
    }
  }
  C = Cs;
}

}  // namespace

// Returns SFR status; fills res (iterations, residual, lambda_min_B) and writes S, L and the
// factors U, B, V where the device pointers are non-null.
sfr_status nys_solve_device(Solver& sv, const sfr_problem& p, const void* Mdev, const int64_t* perm_dev,
                            sfr_result* res, void* Sdev, void* Ldev, double* Udev, double* Bdev, double* Vdev,
                            std::string* err) {
  cudaStream_t st = solver_stream(sv);
  const int64_t m = p.m, n = p.n, l = p.nys_l;
  const int r = p.r;
  const size_t es = p.m_dtype == SFR_F64 ? 8 : p.m_dtype == SFR_F32 ? 4 : 2;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t bL = al(es * m * l), bT = al(es * l * n);
  const size_t bUL = al(8 * m * r), bVL = al(8 * l * r), bUT = al(8 * l * r), bVT = al(8 * n * r), bB = al(8 * r * r);
  const size_t total = bL + bT + bUL + bVL + bUT + bVT + 2 * bB + 3 * al(8 * r * r) + al(8 * m * r) + 512;
  char* base = static_cast<char*>(solver_nys_block(sv, total));
  char* q = base;
  void* Mleft = q; q += bL;
  void* Mtop = q; q += bT;
  double* UL = reinterpret_cast<double*>(q); q += bUL;
  double* VL = reinterpret_cast<double*>(q); q += bVL;
  double* UT = reinterpret_cast<double*>(q); q += bUT;
  double* VT = reinterpret_cast<double*>(q); q += bVT;
  double* BL = reinterpret_cast<double*>(q); q += bB;
  double* BT = reinterpret_cast<double*>(q); q += bB;
  double* core = reinterpret_cast<double*>(q); q += al(8 * r * r);
  double* Asvd = reinterpret_cast<double*>(q); q += al(8 * r * r);   // left singular vectors of the core
  double* Csvd = reinterpret_cast<double*>(q); q += al(8 * r * r);   // right singular vectors
  double* Uo = reinterpret_cast<double*>(q); q += al(8 * m * r);
  int* flag = reinterpret_cast<int*>(q);

  int hflag = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    launch_pdl(check_perm_kernel, 256, 256, 0, st, perm_dev, m, flag);
    e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
  if (hflag) { *err = "FR-Nys: nys_perm has an entry outside [0, m)"; return SFR_E_INVAL; }
  e = by_mtype(p.m_dtype, Mdev, [&](auto M) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
    launch_pdl(gather_cols_kernel<T>, cdiv(m * l, 256), 256, 0, st, M, p.ldm, perm_dev, m, l, static_cast<T*>(Mleft));
    launch_pdl(gather_rows_kernel<T>, cdiv(l * n, 256), 256, 0, st, M, p.ldm, perm_dev, l, n, static_cast<T*>(Mtop));
    return cudaGetLastError();
  });
  if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }

  sfr_problem pl = p;
  pl.nys_l = 0;
  pl.nys_perm = nullptr;
  pl.mem = SFR_MEM_DEVICE;
  pl.m = m; pl.n = l; pl.ldm = l; pl.M = Mleft;
  sfr_problem pt = pl;
  pt.m = l; pt.n = n; pt.ldm = n; pt.M = Mtop;
  // The two block solves (Algorithm 2) are independent: the top block runs on the auxiliary
  // solver in a second host thread while this one solves the left block, when the budget holds
  // both workspaces (their memory is reserved here, before either starts); else one after the
  // other.
  Solver* aux = solver_aux(sv);
  bool concurrent = solver_reserve(sv, pl, Mleft, solver_held(sv), solver_budget(sv)) &&
                    solver_reserve(*aux, pt, Mtop, solver_held(sv), solver_budget(sv));
  cudaEvent_t gathered = nullptr;
  if (concurrent) {
    e = cudaEventCreateWithFlags(&gathered, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(gathered, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(solver_stream(*aux), gathered, 0);
    if (gathered) cudaEventDestroy(gathered);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
  }
  DevState a{}, b{};
  bool top_tc = false, top_failed = false;
  std::string top_err;
  std::thread top;
  if (concurrent) {
    int dev = 0;
    cudaGetDevice(&dev);
    top = std::thread([&, dev] {
      cudaSetDevice(dev);
      try {
        b = solver_run(*aux, pt, Mtop, UT, BT, VT, nullptr, SFR_F64, 0, nullptr);
        top_tc = solver_last_tc(*aux);
      } catch (...) {
        top_failed = true;
        top_err = "FR-Nys: the top block solve failed";
      }
    });
  }
  try {
    a = solver_run(sv, pl, Mleft, UL, BL, VL, nullptr, SFR_F64, 0, nullptr);
  } catch (...) {
    if (top.joinable()) top.join();
    throw;
  }
  res->path |= solver_last_tc(sv) ? SFR_PATH_TC : 0;
  if (concurrent) {
    top.join();
    if (top_failed) { *err = top_err; return SFR_E_CUDA; }
  } else {
    b = solver_run(sv, pt, Mtop, UT, BT, VT, nullptr, SFR_F64, 0, nullptr);
    top_tc = solver_last_tc(sv);
  }
  res->path |= top_tc ? SFR_PATH_TC : 0;
  res->iters = a.iter + b.iter;
  res->rel_residual = std::max(a.res, b.res);
  res->lambda_min_B = NAN;
  for (const DevState* s : {&a, &b}) {
    if (s->status != SFR_OK) {
      *err = "FR-Nys block solve failed";
      return (sfr_status)s->status;
    }
  }
  const int core_smem = (int)(4 * sizeof(double) * CR * CLD);
  e = cudaFuncSetAttribute(nys_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, core_smem);
  if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
  launch_pdl(nys_core_kernel, 1, 256, core_smem, st, UL, BL, UT, BT, l, r, core, flag);
  launch_pdl(nys_rows_kernel, cdiv(m * r, 256), 256, 0, st, UL, core, perm_dev, m, r, Uo);
  cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
  if (hflag) { *err = "FR-Nys: singular l x l block"; return SFR_E_RANK; }
  {
    // polar factors of L = U_L Core V_T^T from the SVD of the r x r core (host)
    std::vector<double> hk((size_t)r * r), A, sig, C;
    e = cudaMemcpy(hk.data(), core, 8 * hk.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
    core_svd(hk, r, A, sig, C);
    res->lambda_min_B = sig[r - 1];
    if (Udev || Vdev) {
      e = cudaMemcpyAsync(Asvd, A.data(), 8 * A.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Csvd, C.data(), 8 * C.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && Udev) e = launch_pdl(nys_rows_kernel, cdiv(m * r, 256), 256, 0, st, UL, Asvd, perm_dev, m, r, Udev);
      if (e == cudaSuccess && Vdev)
        e = launch_pdl(nys_rows_kernel, cdiv(n * r, 256), 256, 0, st, VT, Csvd, (const int64_t*)nullptr, n, r, Vdev);
      if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
    }
    if (Bdev) {
      std::vector<double> hb((size_t)r * r, 0.0);
      for (int i = 0; i < r; ++i) hb[(size_t)i * r + i] = sig[i];
      e = cudaMemcpyAsync(Bdev, hb.data(), 8 * hb.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // hb is a stack buffer
      if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
    }
  }
  if (Sdev || Ldev) {
    const int64_t nblk = (int64_t)cdiv(n, 32) * cdiv(m, 8);
    if (nblk > 0x7fffffffLL) { *err = "FR-Nys output: m x n too large for one launch"; return SFR_E_INVAL; }
    const unsigned grid = (unsigned)nblk;
    const bool fp64 = p.precision == SFR_PREC_FP64;
    e = by_mtype(p.m_dtype, Mdev, [&](auto M) {
      using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
      if (res->s_dtype == SFR_F64) {
        if (fp64) launch_pdl(nys_residual_kernel<double, TMs, double>, grid, 256, 0, st, M, m, n, p.ldm, Uo, VT, r, (double*)Sdev, (double*)Ldev, res->lds);
        else launch_pdl(nys_residual_kernel<float, TMs, double>, grid, 256, 0, st, M, m, n, p.ldm, Uo, VT, r, (double*)Sdev, (double*)Ldev, res->lds);
      } else {
        if (fp64) launch_pdl(nys_residual_kernel<double, TMs, float>, grid, 256, 0, st, M, m, n, p.ldm, Uo, VT, r, (float*)Sdev, (float*)Ldev, res->lds);
        else launch_pdl(nys_residual_kernel<float, TMs, float>, grid, 256, 0, st, M, m, n, p.ldm, Uo, VT, r, (float*)Sdev, (float*)Ldev, res->lds);
      }
      return cudaGetLastError();
    });
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return SFR_E_CUDA; }
  }
  return SFR_OK;
}

}  // namespace sfr
