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
// S = M - (U_L Core) V_T^T row by row in M's original order.
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

// Uo[perm[i]][:] = U_L[i][:] Core   (m x r, dense, M's row order)
__global__ void nys_rows_kernel(const double* __restrict__ UL, const double* __restrict__ core,
                                const int64_t* __restrict__ perm, int64_t m, int r, double* __restrict__ Uo) {
  pdl_enter();
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * r) return;
  int64_t i = idx / r;
  int b = (int)(idx % r);
  double v = 0.0;
  for (int a = 0; a < r; ++a) v = fma(UL[i * r + a], core[a * r + b], v);
  Uo[perm[i] * r + b] = v;
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

}  // namespace

// Returns SFR status; fills res (S, L; factors are not returned for FR-Nys).
sfr_status nys_solve_device(Solver& sv, const sfr_problem& p, const void* Mdev, const int64_t* perm_dev,
                            sfr_result* res, void* Sdev, void* Ldev, std::string* err) {
  cudaStream_t st = solver_stream(sv);
  const int64_t m = p.m, n = p.n, l = p.nys_l;
  const int r = p.r;
  const size_t es = p.m_dtype == SFR_F64 ? 8 : p.m_dtype == SFR_F32 ? 4 : 2;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t bL = al(es * m * l), bT = al(es * l * n);
  const size_t bUL = al(8 * m * r), bVL = al(8 * l * r), bUT = al(8 * l * r), bVT = al(8 * n * r), bB = al(8 * r * r);
  const size_t total = bL + bT + bUL + bVL + bUT + bVT + 2 * bB + al(8 * r * r) + al(8 * m * r) + 512;
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
  DevState a = solver_run(sv, pl, Mleft, UL, BL, VL, nullptr, SFR_F64, 0, nullptr);
  res->path |= solver_last_tc(sv) ? SFR_PATH_TC : 0;
  sfr_problem pt = pl;
  pt.m = l; pt.n = n; pt.ldm = n; pt.M = Mtop;
  DevState b = solver_run(sv, pt, Mtop, UT, BT, VT, nullptr, SFR_F64, 0, nullptr);
  res->path |= solver_last_tc(sv) ? SFR_PATH_TC : 0;
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
