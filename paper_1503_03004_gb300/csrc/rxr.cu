// r x r steps of FixedRankOptStep (Algorithm 3), one CTA per problem.
//
// Stiefel projector (Sec. 4.1.1, Eq. 9): P_O[A] = A (A^T A)^{-1/2} for a full-rank
// m x r matrix A.  With A = P B (U side, P = X V) or A = W B (V side, W = X^T U),
//     A^T A = B G B,   G = P^T P  or  W^T W,
// so P_O[A] = P T with T = B (B G B)^{-1/2}: only r x r work, applied row-wise later.
// SPD projector (Sec. 4.1.2, Eq. 10): B_bar = Sym(U_bar^T X V_bar) = Sym(W^T V_bar)
//     = Sym(G_W T_V), and C = V_bar B_bar = W (T_V B_bar) so that L = U_bar C^T.
//
// The inverse square root Z = K^{-1/2} of K = B G B is computed in two stages:
//  1. cyclic parallel Jacobi in float32 (warm-started from the previous call's
//     eigenvectors) gives an approximate eigenbasis Q and eigenvalues lambda;
//  2. Newton's method for the symmetric solution of Z K Z = I in float64:
//     with R = I - Z K Z, the correction Delta solves Delta K Z + Z K Delta = R;
//     in the approximate eigenbasis K Z ~ Q diag(sqrt(lambda)) Q^T, so
//     Delta = Q [ (Q^T R Q)_pq / (sqrt(lambda_p) + sqrt(lambda_q)) ] Q^T.
//     The residual R is formed in float64; the small correction may be formed
//     in float32.  Each step contracts the error by roughly the eigenbasis error,
//     so two or three steps reach float64 round-off.
//
// GB300 runs float64 at about 2 FMA per clock per SM, so one r = 64 product (262k FMA)
// takes ~60 us on one SM.  The kernel therefore runs as a thread-block cluster: every
// CTA keeps full copies of the r x r matrices in shared memory, computes a slice of rows
// of each float64 product, and pushes its rows to the other CTAs through distributed
// shared memory.  Everything else (float32 Jacobi, element-wise steps, scalar decisions)
// is computed redundantly and identically by every CTA, so control flow stays uniform
// across the cluster; only rank 0 writes to global memory.
#include <cooperative_groups.h>

#include "sfr_internal.h"

namespace cg = cooperative_groups;

namespace sfr {
namespace {

constexpr int RPMAX = kMaxRank;
constexpr int LD = RPMAX + 1;
constexpr int kThreads = 256;

__device__ __forceinline__ bool stopped(const DevState* st) { return *(volatile const int32_t*)&st->done != 0; }

// C = op(A) op(B) on the leading r x r blocks of [RPMAX][LD] shared arrays.
template <typename T, bool TA, bool TB>
__device__ void mm(const T* A, const T* B, T* C, int r) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    T acc = 0;
    for (int k = 0; k < r; ++k) {
      const T a = TA ? A[k * LD + i] : A[i * LD + k];
      const T b = TB ? B[j * LD + k] : B[k * LD + j];
      acc = fma(a, b, acc);
    }
    C[i * LD + j] = acc;
  }
  __syncthreads();
}

// C = op(A) op(B) for float64, rows split across the cluster and broadcast through DSMEM.
// C must not alias A or B.  On return every CTA holds the full product.
template <bool TA, bool TB>
__device__ void mm_dist(const double* A, const double* B, double* C, int r) {
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int rpc = (r + cs - 1) / cs, i0 = min(r, rank * rpc), i1 = min(r, i0 + rpc);
  const int nloc = (i1 - i0) * r;
  for (int e = threadIdx.x; e < nloc; e += blockDim.x) {
    const int i = i0 + e / r, j = e % r;
    // four independent chains (k mod 4) keep the float64 pipe busy with 8 warps per SM
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int k = 0;
    for (; k + 4 <= r; k += 4)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double a = TA ? A[(k + q) * LD + i] : A[i * LD + k + q];
        const double b = TB ? B[j * LD + k + q] : B[(k + q) * LD + j];
        acc[q] = fma(a, b, acc[q]);
      }
    for (; k < r; ++k) {
      const double a = TA ? A[k * LD + i] : A[i * LD + k];
      const double b = TB ? B[j * LD + k] : B[k * LD + j];
      acc[0] = fma(a, b, acc[0]);
    }
    C[i * LD + j] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
  __syncthreads();
  if (cs > 1) {
    cl.sync();  // every CTA is past its earlier reads of C
    for (int q = 1; q < cs; ++q) {
      double* Cq = cl.map_shared_rank(C, (rank + q) % cs);
      for (int e = threadIdx.x; e < nloc; e += blockDim.x) {
        const int i = i0 + e / r, j = e % r;
        Cq[i * LD + j] = C[i * LD + j];
      }
    }
    cl.sync();  // all rows have arrived everywhere
  }
}

// C = op(A) op(B) in float32 on the leading r x r blocks, 4 x 4 outputs per thread (register
// blocking keeps the shared-memory traffic at 8 loads per 16 FMAs).  Reads may touch rows and
// columns beyond r (inside the RPMAX x LD arrays); only outputs inside r x r are written.
template <bool TA, bool TB>
__device__ void mmf(const float* A, const float* B, float* C, int r) {
  const int nb = (r + 3) / 4;
  for (int blk = threadIdx.x; blk < nb * nb; blk += blockDim.x) {
    const int i0 = 4 * (blk / nb), j0 = 4 * (blk % nb);
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int k = 0; k < r; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = TA ? A[k * LD + i0 + q] : A[(i0 + q) * LD + k];
        b[q] = TB ? B[(j0 + q) * LD + k] : B[k * LD + j0 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (i0 + x < r && j0 + y < r) C[(i0 + x) * LD + j0 + y] = acc[x][y];
  }
  __syncthreads();
}

__device__ double block_reduce(double v, double* red, bool take_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmax(v, w) : v + w;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = take_max ? 0.0 : 0.0;
  for (int i = 0; i < nw; ++i) t = take_max ? fmax(t, red[i]) : t + red[i];
  __syncthreads();
  return t;
}

// Cyclic two-sided Jacobi on the symmetric n2 x n2 float matrix A (n2 even; rows/cols
// beyond r are zero), accumulating the rotations into Q (A_final = Q^T A_init Q).
// Round-robin ordering: n2/2 disjoint rotations per step, n2-1 steps per sweep.
__device__ void jacobi_f32(float* A, float* Q, int n2, int max_sweeps, double* red, float* cs, float* sn, int* pp,
                           int* qq) {
  const int np = n2 / 2;
  const bool pow2 = (np & (np - 1)) == 0;
  const int lg = 31 - __clz(np);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
      const int i = e / n2, j = e % n2;
      const double v = (double)A[i * LD + j];
      if (i == j) dia += v * v; else off += v * v;
    }
    off = block_reduce(off, red, false);
    dia = block_reduce(dia, red, false);
    // off-diagonal mass below (3e-5)^2 of the diagonal: the float64 Newton steps that follow
    // contract the remaining error by about this factor per step, so stop here
    if (!(off > 1e-9 * dia)) break;
    for (int step = 0; step < n2 - 1; ++step) {
      if (threadIdx.x < np) {
        const int k = threadIdx.x;
        int p, q;
        if (k == 0) { p = n2 - 1; q = step; }
        else { p = (step + k) % (n2 - 1); q = (step - k + n2 - 1) % (n2 - 1); }
        const float apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq)) && apq != 0.f) {
          const float th = (aqq - app) / (2.f * apq);
          float t;
          if (fabsf(th) > 1e15f) t = 0.5f / th;
          else t = copysignf(1.f, th) / (fabsf(th) + sqrtf(1.f + th * th));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
      }
      __syncthreads();
      // A <- J^T A J in one phase: the pairs partition the indices, so each 2 x 2 block
      // (rows {p1, q1}, columns {p2, q2}) is touched by exactly one row and one column rotation
      for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int k1 = pow2 ? (e >> lg) : e / np, k2 = pow2 ? (e & (np - 1)) : e % np;
        const float c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
        if (s1 == 0.f && s2 == 0.f) continue;
        const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
        const float a = A[p1 * LD + p2], b = A[p1 * LD + q2], c = A[q1 * LD + p2], d = A[q1 * LD + q2];
        const float ra = c1 * a - s1 * c, rb = c1 * b - s1 * d, rc = s1 * a + c1 * c, rd = s1 * b + c1 * d;
        A[p1 * LD + p2] = c2 * ra - s2 * rb;
        A[p1 * LD + q2] = s2 * ra + c2 * rb;
        A[q1 * LD + p2] = c2 * rc - s2 * rd;
        A[q1 * LD + q2] = s2 * rc + c2 * rd;
      }
      // Q <- Q J
      for (int e = threadIdx.x; e < np * n2; e += blockDim.x) {
        const int k = pow2 ? (e & (np - 1)) : e % np, j = pow2 ? (e >> lg) : e / np;
        const float c = cs[k], s = sn[k];
        if (s == 0.f) continue;
        const int p = pp[k], q = qq[k];
        const float xp = Q[j * LD + p], xq = Q[j * LD + q];
        Q[j * LD + p] = c * xp - s * xq;
        Q[j * LD + q] = s * xp + c * xq;
      }
      __syncthreads();
    }
  }
}

// One first-order eigenbasis refinement round for a nearly diagonal A = Q^T K Q (float32):
// Q <- Q (I + E), E_pq = A_pq / (A_qq - A_pp) for p != q (the small-angle Jacobi rotation of
// every pair at once), then one Newton-Schulz re-orthonormalisation and A <- Q^T K Q.
// Returns false (leaving Q, A unchanged) when some |E_pq| > 0.25, i.e. A is not close enough
// to diagonal for the first-order step; pairs with (relative) gaps below 1e-5 are left alone,
// since any basis of a cluster serves the Newton preconditioner.
__device__ bool refine_basis(const float* Kf, float* Q, float* A, float* F1, float* F2, int r, double* red) {
  float big = 0.f;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e % r;
    float v = 0.f;
    if (p != q) {
      const float gap = A[q * LD + q] - A[p * LD + p];
      const float scl = fmaxf(fabsf(A[p * LD + p]), fabsf(A[q * LD + q]));
      if (fabsf(gap) > 1e-5f * scl) v = A[p * LD + q] / gap;
    }
    F1[p * LD + q] = v;
    big = fmaxf(big, fabsf(v));
  }
  big = (float)block_reduce((double)big, red, true);
  if (!(big <= 0.25f)) return false;
  mmf<false, false>(Q, F1, F2, r);                  // Q E
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    Q[i * LD + j] += F2[i * LD + j];
  }
  __syncthreads();
  mmf<true, false>(Q, Q, F1, r);                    // Q^T Q
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    F1[i * LD + j] = 0.5f * ((i == j ? 3.f : 0.f) - F1[i * LD + j]);
  }
  __syncthreads();
  mmf<false, false>(Q, F1, F2, r);                  // Q (3I - Q^T Q) / 2
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Q[(e / r) * LD + e % r] = F2[(e / r) * LD + e % r];
  __syncthreads();
  mmf<false, false>(Kf, Q, F1, r);                  // A = Q^T K Q
  mmf<true, false>(Q, F1, A, r);
  return true;
}

__device__ bool near_diagonal(const float* A, int r, double* red) {
  double off = 0.0, dia = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    const double v = (double)A[i * LD + j];
    if (i == j) dia += v * v; else off += v * v;
  }
  off = block_reduce(off, red, false);
  dia = block_reduce(dia, red, false);
  return !(off > 1e-9 * dia);
}

struct RxrSmem {
  double K[RPMAX * LD];    // B G B / s
  double B[RPMAX * LD];
  double Z[RPMAX * LD];    // K^{-1/2} iterate
  double T1[RPMAX * LD];   // scratch; also holds two float scratch arrays
  double T2[RPMAX * LD];   // scratch
  float Af[RPMAX * LD];    // Jacobi matrix / float scratch
  float Qf[RPMAX * LD];    // approximate eigenbasis
  double lam[RPMAX];
  double sq[RPMAX];
  double red[32];
  float cs[RPMAX / 2], sn[RPMAX / 2];
  int pp[RPMAX / 2], qq[RPMAX / 2];
  double scale;
  int bad;
};

// dst = the summed r x r Gram G (rp x rp float64 in global memory; every CTA reads all of it).
__device__ void load_gram(const double* __restrict__ G, int rp, int r, double* dst) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    dst[i * LD + j] = G[i * rp + j];
  }
  __syncthreads();
}

__device__ void fail(DevState* st, int code) {
  if (threadIdx.x == 0 && cg::this_cluster().block_rank() == 0) { st->status = code; st->done = 1; }
}

// v_side = false: T_U = B (B G_P B)^{-1/2}.
// v_side = true:  T_V = B (B G_W B)^{-1/2}, B <- Sym(G_W T_V), T_C = T_V B.
// float64: K = B G B, the Newton residual, T, B_bar, T_C (G: the float64 sum of the partials).
// float32: the eigenbasis, eigenvalue estimates, Z0 and the Newton corrections, which only
// steer the iteration (their error shrinks with each Newton step).
__global__ void __launch_bounds__(kThreads) rxr_kernel(const double* __restrict__ G, int rp, int r,
                                                       double* __restrict__ Bg, double* __restrict__ Tout,
                                                       double* __restrict__ TCout, float* __restrict__ Qeig,
                                                       int v_side, int mixed, DevState* st) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RxrSmem& S = *reinterpret_cast<RxrSmem*>(smem_raw);
  float* F1 = reinterpret_cast<float*>(S.T1);            // float scratch inside T1
  float* F2 = F1 + RPMAX * LD;
  float* Kf = reinterpret_cast<float*>(S.T2);            // float copy of K inside T2 (until Z0)
  float* lamf = reinterpret_cast<float*>(S.lam);         // float eigenvalue estimates
  float* sqf = lamf + RPMAX;                             // sqrt(lambda)
  float* isqf = reinterpret_cast<float*>(S.sq);          // 1 / sqrt(lambda)
  const int tid = threadIdx.x;
  const int rpsq = rp * rp;
  const bool writer = cg::this_cluster().block_rank() == 0;
  // 1. Gram of the thin matrix and B; K = B G B (symmetrised) scaled by s = trace / r
  load_gram(G, rp, r, S.T2);
  for (int e = tid; e < r * r; e += blockDim.x) S.B[(e / r) * LD + e % r] = Bg[(e / r) * rp + e % r];
  __syncthreads();
  mm_dist<false, false>(S.T2, S.B, S.T1, r);
  mm_dist<false, false>(S.B, S.T1, S.Z, r);
  double tr = 0.0;
  for (int i = tid; i < r; i += blockDim.x) tr += S.Z[i * LD + i];
  tr = block_reduce(tr, S.red, false);
  const double scale = tr / r;
  if (!(scale > 0.0) || !(scale < 1e300)) { fail(st, SFR_E_NAN); return; }
  const double inv_s = 1.0 / scale;
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    const double v = 0.5 * (S.Z[i * LD + j] + S.Z[j * LD + i]) * inv_s;
    S.K[i * LD + j] = v;
    Kf[i * LD + j] = (float)v;
  }
  // 2. float32 Jacobi, warm-started from the previous eigenbasis Qw: A = Qw^T K Qw
  const int n2 = (r + 1) & ~1;
  for (int e = tid; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    const bool in = i < r && j < r;
    if (!in) Kf[i * LD + j] = 0.f;
    S.Qf[i * LD + j] = in ? Qeig[i * rp + j] : (i == j ? 1.f : 0.f);
  }
  __syncthreads();
  mmf<false, false>(Kf, S.Qf, F2, n2);
  mmf<true, false>(S.Qf, F2, S.Af, n2);
  // the basis of the previous call is usually close: refine it to first order (cheap), and fall
  // back to Jacobi sweeps only when that does not converge
  bool diag = near_diagonal(S.Af, n2, S.red);
  for (int round = 0; round < 3 && !diag; ++round) {
    if (!refine_basis(Kf, S.Qf, S.Af, F1, F2, n2, S.red)) break;
    diag = near_diagonal(S.Af, n2, S.red);
  }
  if (!diag) jacobi_f32(S.Af, S.Qf, n2, 10, S.red, S.cs, S.sn, S.pp, S.qq);
  // re-orthonormalise the float basis: Q <- Q (3I - Q^T Q) / 2
  mmf<true, false>(S.Qf, S.Qf, F1, r);
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    F1[i * LD + j] = 0.5f * ((i == j ? 3.f : 0.f) - F1[i * LD + j]);
  }
  __syncthreads();
  mmf<false, false>(S.Qf, F1, F2, r);
  for (int e = tid; e < r * r; e += blockDim.x) S.Qf[(e / r) * LD + e % r] = F2[(e / r) * LD + e % r];
  __syncthreads();
  // 3. eigenvalue estimates lambda_p = q_p^T K q_p / q_p^T q_p in float32; those far below the
  //    largest are recomputed in float64 for the rank test (Eq. 9 needs rank r)
  mmf<false, false>(Kf, S.Qf, F1, r);
  for (int p = tid; p < r; p += blockDim.x) {
    float num = 0.f, den = 0.f;
    for (int i = 0; i < r; ++i) {
      num = fmaf(S.Qf[i * LD + p], F1[i * LD + p], num);
      den = fmaf(S.Qf[i * LD + p], S.Qf[i * LD + p], den);
    }
    lamf[p] = num / den;
  }
  __syncthreads();
  float hi = 0.f;
  for (int p = 0; p < r; ++p) hi = fmaxf(hi, lamf[p]);
  for (int p = tid; p < r; p += blockDim.x) {
    if (lamf[p] < 1e-3f * hi) {
      double num = 0.0, den = 0.0;
      for (int i = 0; i < r; ++i) {
        double kq = 0.0;
        for (int k = 0; k < r; ++k) kq = fma(S.K[i * LD + k], (double)S.Qf[k * LD + p], kq);
        num = fma((double)S.Qf[i * LD + p], kq, num);
        den = fma((double)S.Qf[i * LD + p], (double)S.Qf[i * LD + p], den);
      }
      lamf[p] = (float)(num / den);
    }
  }
  __syncthreads();
  bool bad = false;
  float lo = hi;
  for (int p = 0; p < r; ++p) {
    lo = fminf(lo, lamf[p]);
    bad |= !(lamf[p] > 1e-14f * hi);
  }
  bad |= !(hi > 0.f);
  __syncthreads();
  if (writer && tid == 0) {
    if (v_side) st->lam_min_v = (double)lo * scale; else st->lam_min_u = (double)lo * scale;
  }
  if (bad) { fail(st, SFR_E_RANK); return; }
  for (int p = tid; p < r; p += blockDim.x) {
    const float sq = sqrtf(lamf[p]);
    sqf[p] = sq;
    isqf[p] = 1.f / sq;
  }
  __syncthreads();
  // 4. Z0 = Q diag(lambda^{-1/2}) Q^T (float32 start; Newton below brings it to float64 accuracy)
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    F2[i * LD + j] = S.Qf[i * LD + j] * isqf[j];
  }
  __syncthreads();
  mmf<false, true>(F2, S.Qf, F1, r);
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S.Z[i * LD + j] = 0.5 * ((double)F1[i * LD + j] + (double)F1[j * LD + i]);
  }
  __syncthreads();
  // 5. Newton steps on Z K Z = I (residual in float64, correction in float32)
  for (int it = 0; it < 6; ++it) {
    mm_dist<false, false>(S.K, S.Z, S.T1, r);
    mm_dist<false, false>(S.Z, S.T1, S.T2, r);
    float rmax = 0.f;
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      const float v = (float)((i == j ? 1.0 : 0.0) - 0.5 * (S.T2[i * LD + j] + S.T2[j * LD + i]));
      F1[i * LD + j] = v;
      rmax = fmaxf(rmax, fabsf(v));
    }
    const double rm = block_reduce((double)rmax, S.red, true);
    if (!(rm == rm)) { fail(st, SFR_E_NAN); return; }
    if (rm < 4e-16 * r) break;
    mmf<false, false>(F1, S.Qf, F2, r);     // R Q
    mmf<true, false>(S.Qf, F2, S.Af, r);    // Q^T R Q
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int p = e / r, q = e % r;
      S.Af[p * LD + q] = S.Af[p * LD + q] / (sqf[p] + sqf[q]);
    }
    __syncthreads();
    mmf<false, true>(S.Af, S.Qf, F2, r);    // Dt Q^T
    mmf<false, false>(S.Qf, F2, F1, r);     // Q Dt Q^T
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.Z[i * LD + j] += 0.5 * ((double)F1[i * LD + j] + (double)F1[j * LD + i]);
    }
    __syncthreads();
    // The step just taken leaves a residual of about (eigenbasis error + float32 rounding of the
    // correction) x rm + O(rm^2): from rm < 3e-6 about 1e-11 (mixed path, whose Gram carries
    // float32 rounding), from rm < 1e-7 about 1e-14 (float64 path), so stop without forming it again.
    if (rm < (mixed ? 3e-6 : 1e-7)) break;
  }
  // 6. (B G B)^{-1/2} = Z / sqrt(s); T = B (B G B)^{-1/2}
  const double zs = 1.0 / sqrt(scale);
  for (int e = tid; e < r * r; e += blockDim.x) S.Z[(e / r) * LD + e % r] *= zs;
  __syncthreads();
  mm_dist<false, false>(S.B, S.Z, S.T1, r);
  if (writer)
    for (int e = tid; e < rpsq; e += blockDim.x) {
      const int i = e / rp, j = e % rp;
      const bool in = i < r && j < r;
      Tout[e] = in ? S.T1[i * LD + j] : 0.0;
      Qeig[e] = in ? S.Qf[i * LD + j] : (i == j ? 1.f : 0.f);
    }
  if (!v_side) return;
  // 7. B_bar = Sym(G_W T_V) (Eq. 10 with W = X^T U_bar), T_C = T_V B_bar
  load_gram(G, rp, r, S.K);
  mm_dist<false, false>(S.K, S.T1, S.T2, r);
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S.Z[i * LD + j] = 0.5 * (S.T2[i * LD + j] + S.T2[j * LD + i]);
  }
  __syncthreads();
  mm_dist<false, false>(S.T1, S.Z, S.T2, r);
  if (writer)
    for (int e = tid; e < rpsq; e += blockDim.x) {
      const int i = e / rp, j = e % rp;
      const bool in = i < r && j < r;
      Bg[e] = in ? S.Z[i * LD + j] : 0.0;
      TCout[e] = in ? S.T2[i * LD + j] : 0.0;
    }
}


}  // namespace

// Cluster size for the r x r kernel: 16 CTAs (non-portable size) when the device accepts it
// with this kernel's shared memory, else 8, else a single CTA.
static int rxr_cluster_size(size_t smem) {
  static int cached = 0;
  if (cached) return cached;
  int best = 1;
  if (cudaFuncSetAttribute(rxr_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    cudaGetLastError();
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cs;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, rxr_kernel, &cfg) == cudaSuccess && nclusters > 0) {
      best = cs;
      break;
    }
    cudaGetLastError();
  }
  cached = best;
  return best;
}

cudaError_t launch_rxr(const Shape& s, const Buffers& b, bool v_side, cudaStream_t st, bool fp64) {
  const double* parts = v_side ? b.GWpart : b.GPpart;
  const int count = v_side ? s.gw_blocks : s.gp_blocks;
  cudaError_t e = launch_reduce_parts(parts, count, s.rp * s.rp, b.Gsum, b.st, st);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(RxrSmem);
  e = cudaFuncSetAttribute(rxr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int cs = rxr_cluster_size(smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = cs;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, rxr_kernel, (const double*)b.Gsum, s.rp, s.r, b.B, v_side ? b.TV : b.TU,
                            v_side ? b.TCm : (double*)nullptr, v_side ? b.Qeig_v : b.Qeig_u, v_side ? 1 : 0,
                            fp64 ? 0 : 1, b.st);
}

}  // namespace sfr
