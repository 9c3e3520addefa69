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
constexpr int LD = RPMAX + 4;  // row stride of the r x r arrays: 16-byte aligned float rows
constexpr int kThreads = 512;

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
__device__ void mm_dist(const double* A, const double* B, double* C, int r, double scale = 1.0) {
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
    C[i * LD + j] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * scale;
  }
  __syncthreads();
  if (cs > 1) {
    cl.sync();  // every CTA is past its earlier reads of C
    // push this CTA's rows to the other CTAs in 16-byte pieces (column pairs; with r odd the
    // last pair carries column r, which no product reads)
    const int np2 = (r + 1) / 2, per = (i1 - i0) * np2;
    for (int e = threadIdx.x; e < (cs - 1) * per; e += blockDim.x) {
      const int q = 1 + e / per, w = e % per;
      const int i = i0 + w / np2, j = 2 * (w % np2);
      double* Cq = cl.map_shared_rank(C, (rank + q) % cs);
      *reinterpret_cast<double2*>(Cq + i * LD + j) = *reinterpret_cast<const double2*>(C + i * LD + j);
    }
    cl.sync();  // all rows have arrived everywhere
  }
}

// C = op(A) op(B) in float32 on the leading r x r blocks, 4 x 4 outputs per thread.  Operands
// move in 16-byte loads, 4 x 4 blocks of A and B per 4 steps of k (8 loads per 64 FMAs); the
// sum over k runs in order.  Reads may touch rows and columns beyond r (inside the RPMAX x LD
// arrays); only outputs inside r x r are written.
template <bool TA, bool TB>
__device__ void mmf(const float* A, const float* B, float* C, int r) {
  const int nb = (r + 3) / 4, r4 = r & ~3;
  for (int blk = threadIdx.x; blk < nb * nb; blk += blockDim.x) {
    const int i0 = 4 * (blk / nb), j0 = 4 * (blk % nb);
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    for (int k = 0; k < r4; k += 4) {
      float a[4][4], b[4][4];  // a[x][q] = op(A)(i0 + x, k + q), b[q][y] = op(B)(k + q, j0 + y)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 va = TA ? *reinterpret_cast<const float4*>(A + (k + q) * LD + i0)
                             : *reinterpret_cast<const float4*>(A + (i0 + q) * LD + k);
        const float4 vb = TB ? *reinterpret_cast<const float4*>(B + (j0 + q) * LD + k)
                             : *reinterpret_cast<const float4*>(B + (k + q) * LD + j0);
        const float fa[4] = {va.x, va.y, va.z, va.w}, fb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (TA) a[w][q] = fa[w]; else a[q][w] = fa[w];
          if (TB) b[w][q] = fb[w]; else b[q][w] = fb[w];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x][q], b[q][y], acc[x][y]);
    }
    for (int k = r4; k < r; ++k) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const float av = TA ? A[k * LD + i0 + x] : A[(i0 + x) * LD + k];
          const float bv = TB ? B[(j0 + y) * LD + k] : B[k * LD + j0 + y];
          acc[x][y] = fmaf(av, bv, acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (i0 + x < r && j0 + y < r) C[(i0 + x) * LD + j0 + y] = acc[x][y];
  }
  __syncthreads();
}

// dst[i * LD + j] = src[i * rp + j] for i, j < r; for r <= i, j < n the identity's entries
// (pad_diag on the diagonal, 0 elsewhere).  Every load of a thread is issued before any store.
template <typename TS, typename TD>
__device__ __forceinline__ void load_sq(const TS* __restrict__ src, int rp, int r, int n, TD* dst, TD pad_diag) {
  constexpr int PER = RPMAX * RPMAX / kThreads;
  TS v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * kThreads, i = e / RPMAX, j = e % RPMAX;
    v[q] = (i < r && j < r) ? src[i * rp + j] : (TS)0;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * kThreads, i = e / RPMAX, j = e % RPMAX;
    if (i < n && j < n) dst[i * LD + j] = (i < r && j < r) ? (TD)v[q] : (i == j ? pad_diag : (TD)0);
  }
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
  double t = red[0];
  for (int i = 1; i < nw; ++i) t = take_max ? fmax(t, red[i]) : t + red[i];
  __syncthreads();
  return t;
}

// float version (the sums and maxima it serves steer decisions only)
__device__ float block_reduce_f(float v, float* red, bool take_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmaxf(v, w) : v + w;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = red[0];
  for (int i = 1; i < nw; ++i) t = take_max ? fmaxf(t, red[i]) : t + red[i];
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
    float off = 0.f, dia = 0.f;
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
      const int i = e / n2, j = e % n2;
      const float v = A[i * LD + j];
      if (i == j) dia = fmaf(v, v, dia); else off = fmaf(v, v, off);
    }
    off = block_reduce_f(off, reinterpret_cast<float*>(red), false);
    dia = block_reduce_f(dia, reinterpret_cast<float*>(red), false);
    // off-diagonal mass below (1e-3)^2 of the diagonal: each float64 Newton step that follows
    // contracts the residual by about this factor (the next call refines the basis further)
    if (!(off > 1e-6 * dia)) break;
    if (n2 == 64 && blockDim.x == kThreads) {
      // 32 pairs: every warp computes all 32 rotations itself (lane k: pair k) and takes the
      // ones it needs by shuffles, so a step needs a single barrier; a thread rotates the two
      // 2 x 2 blocks (pair w + 16u, pair lane) of A and the four (row w + 16u v, pair lane)
      // entries pairs of Q, all loads first
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      constexpr int NW = kThreads / 32;
      for (int step = 0; step < 63; ++step) {
        const int p = lane == 0 ? 63 : (step + lane) % 63, q = lane == 0 ? step : (step - lane + 63) % 63;
        const float apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
        float c = 1.f, sn_ = 0.f;
        if (fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq)) && apq != 0.f) {
          const float th = __fdividef(aqq - app, 2.f * apq);
          const float t = fabsf(th) > 1e15f ? __fdividef(0.5f, th)
                                           : copysignf(1.f, th) * __frcp_rn(fabsf(th) + sqrtf(1.f + th * th));
          c = rsqrtf(1.f + t * t);
          sn_ = t * c;
        }
        float v[2][4], x[4][2];
        int k1p[2], k1q[2];
        float c1[2], s1[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k1 = warp + NW * u;
          c1[u] = __shfl_sync(0xffffffffu, c, k1);
          s1[u] = __shfl_sync(0xffffffffu, sn_, k1);
          k1p[u] = __shfl_sync(0xffffffffu, p, k1);
          k1q[u] = __shfl_sync(0xffffffffu, q, k1);
        }
        __syncthreads();  // every warp has read the pivots of this step
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          v[u][0] = A[k1p[u] * LD + p]; v[u][1] = A[k1p[u] * LD + q];
          v[u][2] = A[k1q[u] * LD + p]; v[u][3] = A[k1q[u] * LD + q];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = warp + NW * u;
          x[u][0] = Q[j * LD + p];
          x[u][1] = Q[j * LD + q];
        }
        if (sn_ != 0.f || s1[0] != 0.f || s1[1] != 0.f) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float ra = c1[u] * v[u][0] - s1[u] * v[u][2], rb = c1[u] * v[u][1] - s1[u] * v[u][3];
            const float rc = s1[u] * v[u][0] + c1[u] * v[u][2], rd = s1[u] * v[u][1] + c1[u] * v[u][3];
            A[k1p[u] * LD + p] = c * ra - sn_ * rb;
            A[k1p[u] * LD + q] = sn_ * ra + c * rb;
            A[k1q[u] * LD + p] = c * rc - sn_ * rd;
            A[k1q[u] * LD + q] = sn_ * rc + c * rd;
          }
        }
        if (sn_ != 0.f) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = warp + NW * u;
            Q[j * LD + p] = c * x[u][0] - sn_ * x[u][1];
            Q[j * LD + q] = sn_ * x[u][0] + c * x[u][1];
          }
        }
        __syncthreads();
      }
      continue;
    }
    for (int step = 0; step < n2 - 1; ++step) {
      if (threadIdx.x < np) {
        const int k = threadIdx.x;
        int p, q;
        if (k == 0) { p = n2 - 1; q = step; }
        else { p = (step + k) % (n2 - 1); q = (step - k + n2 - 1) % (n2 - 1); }
        const float apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq)) && apq != 0.f) {
          const float th = __fdividef(aqq - app, 2.f * apq);
          float t;
          if (fabsf(th) > 1e15f) t = __fdividef(0.5f, th);
          else t = copysignf(1.f, th) * __frcp_rn(fabsf(th) + sqrtf(1.f + th * th));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
      }
      __syncthreads();
      // A <- J^T A J in one phase: the pairs partition the indices, so each 2 x 2 block
      // (rows {p1, q1}, columns {p2, q2}) is touched by exactly one row and one column rotation.
      // Each thread takes up to four blocks, loads all of them, then rotates and stores.
      {
        constexpr int MB = (RPMAX / 2) * (RPMAX / 2) / kThreads;
        float v[MB][4];
        int pos[MB][4];
        float rc[MB][4];
        bool act[MB];
        // with 32 pairs a thread's column pair k2 is its lane for every u: load it once
        const bool lanepair = np == 32;
        const int kl = threadIdx.x & 31;
        const float cl = cs[kl], sl = sn[kl];
        const int pl = pp[kl], ql = qq[kl];
#pragma unroll
        for (int u = 0; u < MB; ++u) {
          const int e = threadIdx.x + u * kThreads;
          act[u] = e < np * np;
          if (!act[u]) continue;
          const int k1 = pow2 ? (e >> lg) : e / np, k2 = pow2 ? (e & (np - 1)) : e % np;
          rc[u][0] = cs[k1]; rc[u][1] = sn[k1];
          rc[u][2] = lanepair ? cl : cs[k2];
          rc[u][3] = lanepair ? sl : sn[k2];
          act[u] = !(rc[u][1] == 0.f && rc[u][3] == 0.f);
          const int p1 = pp[k1], q1 = qq[k1], p2 = lanepair ? pl : pp[k2], q2 = lanepair ? ql : qq[k2];
          pos[u][0] = p1 * LD + p2; pos[u][1] = p1 * LD + q2; pos[u][2] = q1 * LD + p2; pos[u][3] = q1 * LD + q2;
#pragma unroll
          for (int w = 0; w < 4; ++w) v[u][w] = A[pos[u][w]];
        }
#pragma unroll
        for (int u = 0; u < MB; ++u) {
          if (!act[u]) continue;
          const float c1 = rc[u][0], s1 = rc[u][1], c2 = rc[u][2], s2 = rc[u][3];
          const float ra = c1 * v[u][0] - s1 * v[u][2], rb = c1 * v[u][1] - s1 * v[u][3];
          const float rcc = s1 * v[u][0] + c1 * v[u][2], rd = s1 * v[u][1] + c1 * v[u][3];
          A[pos[u][0]] = c2 * ra - s2 * rb;
          A[pos[u][1]] = s2 * ra + c2 * rb;
          A[pos[u][2]] = c2 * rcc - s2 * rd;
          A[pos[u][3]] = s2 * rcc + c2 * rd;
        }
      }
      // Q <- Q J, up to eight (row, pair) items per thread, loads first
      {
        constexpr int MQ = (RPMAX / 2) * RPMAX / kThreads;
        float x2[MQ][2], cq[MQ][2];
        int qp[MQ][2];
        bool act[MQ];
        const bool lanepair = np == 32;
        const int kl = threadIdx.x & 31;
        const float cl = cs[kl], sl = sn[kl];
        const int pl = pp[kl], ql = qq[kl];
#pragma unroll
        for (int u = 0; u < MQ; ++u) {
          const int e = threadIdx.x + u * kThreads;
          act[u] = e < np * n2;
          if (!act[u]) continue;
          const int k = pow2 ? (e & (np - 1)) : e % np, j = pow2 ? (e >> lg) : e / np;
          cq[u][0] = lanepair ? cl : cs[k];
          cq[u][1] = lanepair ? sl : sn[k];
          act[u] = cq[u][1] != 0.f;
          qp[u][0] = j * LD + (lanepair ? pl : pp[k]);
          qp[u][1] = j * LD + (lanepair ? ql : qq[k]);
          x2[u][0] = Q[qp[u][0]]; x2[u][1] = Q[qp[u][1]];
        }
#pragma unroll
        for (int u = 0; u < MQ; ++u) {
          if (!act[u]) continue;
          const float c = cq[u][0], sv = cq[u][1];
          Q[qp[u][0]] = c * x2[u][0] - sv * x2[u][1];
          Q[qp[u][1]] = sv * x2[u][0] + c * x2[u][1];
        }
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
      if (fabsf(gap) > 1e-5f * scl) v = __fdividef(A[p * LD + q], gap);  // first-order term: 2 ulp is ample
    }
    F1[p * LD + q] = v;
    big = fmaxf(big, fabsf(v));
  }
  big = block_reduce_f(big, reinterpret_cast<float*>(red), true);
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

// Off-diagonal mass of A below tol^2 of its diagonal mass (Frobenius), float32 sums.
__device__ bool near_diagonal(const float* A, int r, double* red, double tol2 = 1e-9) {
  float off = 0.f, dia = 0.f;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    const float v = A[i * LD + j];
    if (i == j) dia = fmaf(v, v, dia); else off = fmaf(v, v, off);
  }
  const float o = block_reduce_f(off, reinterpret_cast<float*>(red), false);
  const float d = block_reduce_f(dia, reinterpret_cast<float*>(red), false);
  return !((double)o > tol2 * (double)d);
}

struct RxrSmem {
  double K[RPMAX * LD];    // B G B / s
  double B[RPMAX * LD];
  double Z[RPMAX * LD];    // K^{-1/2} iterate
  double T1[RPMAX * LD];   // scratch; also holds two float scratch arrays
  double T2[RPMAX * LD];   // scratch
  float Af[RPMAX * LD];    // Jacobi matrix / float scratch
  float Qf[RPMAX * LD];    // approximate eigenbasis
  float QT[RPMAX * LD];    // its transpose (keeps every float32 product in the conflict-free forms)
  double lam[RPMAX];
  double sq[RPMAX];
  double red[32];
  float cs[RPMAX / 2], sn[RPMAX / 2];
  int pp[RPMAX / 2], qq[RPMAX / 2];
  double scale;
  int bad;
};

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
  load_sq(G, rp, r, r, S.T2, 0.0);
  load_sq(Bg, rp, r, r, S.B, 0.0);
  __syncthreads();
  mm_dist<false, false>(S.T2, S.B, S.T1, r);
  mm_dist<false, false>(S.B, S.T1, S.Z, r);
  double tr = 0.0;  // trace of B G B: float64 sums within the first two warps (r <= 64)
  if (tid < 64) {
    tr = tid < r ? S.Z[tid * LD + tid] : 0.0;
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = tr;
  }
  __syncthreads();
  tr = S.red[0] + S.red[1];
  __syncthreads();
  const double scale = tr / r;
  if (!(scale > 0.0) || !(scale < 1e300)) { fail(st, SFR_E_NAN); return; }
  const double inv_s = 1.0 / scale;
  for (int e = tid; e < r * r; e += blockDim.x) {  // B (G B) is symmetric to float64 rounding
    const int i = e / r, j = e % r;
    const double v = S.Z[i * LD + j] * inv_s;
    S.K[i * LD + j] = v;
    Kf[i * LD + j] = (float)v;
  }
  // 2. float32 Jacobi, warm-started from the previous eigenbasis Qw: A = Qw^T K Qw
  const int n2 = (r + 1) & ~1;
  for (int e = tid; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    if (i >= r || j >= r) Kf[i * LD + j] = 0.f;
  }
  load_sq(Qeig, rp, r, n2, S.Qf, 1.f);
  __syncthreads();
  mmf<false, false>(Kf, S.Qf, F2, n2);
  mmf<true, false>(S.Qf, F2, S.Af, n2);
  // the basis of the previous call is usually close: refine it to first order (cheap), and fall
  // back to Jacobi sweeps only when that does not converge
  // at least one refinement round: a basis accurate to float32 rounding lets one Newton step
  // (two float64 products) replace two
  bool diag = false;
  for (int round = 0; round < 3; ++round) {
    if (!refine_basis(Kf, S.Qf, S.Af, F1, F2, n2, S.red)) break;
    diag = near_diagonal(S.Af, n2, S.red);
    if (diag) break;
  }
  const bool rotated = !diag;
  if (rotated) jacobi_f32(S.Af, S.Qf, n2, 10, S.red, S.cs, S.sn, S.pp, S.qq);
  if (rotated) {
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
  }
  for (int e = tid; e < r * r; e += blockDim.x) S.QT[(e % r) * LD + e / r] = S.Qf[(e / r) * LD + e % r];
  // 3. eigenvalue estimates: the diagonal of A = Q^T K Q (Rayleigh quotients of the basis, to
  //    float32 rounding); those far below the largest are recomputed in float64 for the rank
  //    test (Eq. 9 needs rank r)
  for (int p = tid; p < r; p += blockDim.x) lamf[p] = S.Af[p * LD + p];
  __syncthreads();
  float* redf = reinterpret_cast<float*>(S.red);
  float hi = 0.f;
  for (int p = tid; p < r; p += blockDim.x) hi = fmaxf(hi, lamf[p]);
  hi = block_reduce_f(hi, redf, true);
  // the float32 estimates carry errors near 1e-7 hi: below 1e-6 hi, recompute q_p^T K q_p in
  // float64 (every thread takes one row of K q_p, then a block sum)
  float anysmall = 0.f;
  for (int p = tid; p < r; p += blockDim.x)
    if (lamf[p] < 1e-6f * hi) anysmall = 1.f;
  anysmall = block_reduce_f(anysmall, redf, true);
  if (anysmall > 0.f && rotated) {
    // Jacobi stopped at a 1e-3 off-diagonal, so a basis vector of a tiny eigenvalue still mixes
    // ~1e-3 of the large ones and its Rayleigh quotient sits near 1e-6 hi: two first-order rounds
    // (near-degenerate pairs are skipped) bring the mixing down to float32 rounding first.
    for (int round = 0; round < 2; ++round)
      if (!refine_basis(Kf, S.Qf, S.Af, F1, F2, n2, S.red)) break;
    for (int e = tid; e < r * r; e += blockDim.x) S.QT[(e % r) * LD + e / r] = S.Qf[(e / r) * LD + e % r];
    for (int p = tid; p < r; p += blockDim.x) lamf[p] = S.Af[p * LD + p];
    __syncthreads();
    hi = 0.f;
    for (int p = tid; p < r; p += blockDim.x) hi = fmaxf(hi, lamf[p]);
    hi = block_reduce_f(hi, redf, true);
  }
  // A float32 eigenvector carries components of about 1e-7 along the large eigenvectors, which
  // alone would add ~1e-14 hi to its Rayleigh quotient (the rank threshold): project them out in
  // float64 first (q <- q - Q_L Q_L^T q over the columns of large eigenvalues).
  double* qs = S.Z;       // the vector (Z is free until step 4)
  double* cf = S.Z + LD;  // its coefficients on the large eigenvectors
  for (int p = 0; anysmall > 0.f && p < r; ++p) {
    if (!(lamf[p] < 1e-6f * hi)) continue;  // uniform: lamf is in shared memory
    if (tid < r) qs[tid] = (double)S.Qf[tid * LD + p];
    __syncthreads();
    if (tid < r) {
      double c = 0.0;
      if (!(lamf[tid] < 1e-6f * hi))
        for (int k = 0; k < r; ++k) c = fma((double)S.Qf[k * LD + tid], qs[k], c);
      cf[tid] = c;
    }
    __syncthreads();
    double qi = 0.0;
    if (tid < r) {
      qi = qs[tid];
      for (int q2 = 0; q2 < r; ++q2) qi = fma(-cf[q2], (double)S.Qf[tid * LD + q2], qi);
    }
    __syncthreads();
    if (tid < r) qs[tid] = qi;
    __syncthreads();
    double num = 0.0, den = 0.0;
    if (tid < r) {
      double kq = 0.0;
      for (int k = 0; k < r; ++k) kq = fma(S.K[tid * LD + k], qs[k], kq);
      num = qi * kq;
      den = qi * qi;
    }
    num = block_reduce(num, S.red, false);
    den = block_reduce(den, S.red, false);
    if (tid == 0) lamf[p] = (float)(num / den);
    __syncthreads();
  }
  float nlo = -hi, badf = 0.f;  // max of -lambda and of the rank-failure flag
  for (int p = tid; p < r; p += blockDim.x) {
    nlo = fmaxf(nlo, -lamf[p]);
    if (!(lamf[p] > 1e-14f * hi)) badf = 1.f;
  }
  const float lo = -block_reduce_f(nlo, redf, true);
  const bool bad = block_reduce_f(badf, redf, true) > 0.f || !(hi > 0.f);
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
  mmf<false, false>(F2, S.QT, F1, r);
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S.Z[i * LD + j] = (double)(0.5f * (F1[i * LD + j] + F1[j * LD + i]));
  }
  __syncthreads();
  // 5. Newton steps on Z K Z = I (residual in float64, correction in float32)
  for (int it = 0; it < 6; ++it) {
    mm_dist<false, false>(S.K, S.Z, S.T1, r);
    mm_dist<false, false>(S.Z, S.T1, S.T2, r);
    float rmax = 0.f;
    for (int e = tid; e < r * r; e += blockDim.x) {  // I - Z K Z, rounded to float32
      const int i = e / r, j = e % r;
      const float v = (float)((i == j ? 1.0 : 0.0) - S.T2[i * LD + j]);
      F1[i * LD + j] = v;
      rmax = fmaxf(rmax, fabsf(v));
    }
    const float rm = block_reduce_f(rmax, redf, true);
    if (!(rm == rm)) { fail(st, SFR_E_NAN); return; }
    if (rm < 4e-16f * r) break;
    for (int e = tid; e < r * r; e += blockDim.x) {  // R = Sym(I - Z K Z)
      const int i = e / r, j = e % r;
      F2[i * LD + j] = 0.5f * (F1[i * LD + j] + F1[j * LD + i]);
    }
    __syncthreads();
    mmf<false, false>(F2, S.Qf, F1, r);     // R Q
    mmf<true, false>(S.Qf, F1, S.Af, r);    // Q^T R Q
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int p = e / r, q = e % r;
      S.Af[p * LD + q] = __fdividef(S.Af[p * LD + q], sqf[p] + sqf[q]);
    }
    __syncthreads();
    mmf<false, false>(S.Af, S.QT, F2, r);   // Dt Q^T
    mmf<false, false>(S.Qf, F2, F1, r);     // Q Dt Q^T
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.Z[i * LD + j] += (double)(0.5f * (F1[i * LD + j] + F1[j * LD + i]));
    }
    __syncthreads();
    // The step just taken leaves a residual of about (eigenbasis error + float32 rounding of the
    // correction) x rm + O(rm^2): from rm < 3e-6 about 1e-11 (mixed path, whose Gram carries
    // float32 rounding), from rm < 1e-7 about 1e-14 (float64 path), so stop without forming it again.
    if (rm < (mixed ? 3e-6 : 1e-7)) break;
  }
  // 6. (B G B)^{-1/2} = Z / sqrt(s); T = B (B G B)^{-1/2}
  mm_dist<false, false>(S.B, S.Z, S.T1, r, 1.0 / sqrt(scale));
  if (writer)
    for (int e = tid; e < rpsq; e += blockDim.x) {
      const int i = e / rp, j = e % rp;
      const bool in = i < r && j < r;
      Tout[e] = in ? S.T1[i * LD + j] : 0.0;
      Qeig[e] = in ? S.Qf[i * LD + j] : (i == j ? 1.f : 0.f);
    }
  if (!v_side) return;
  // 7. B_bar = Sym(G_W T_V) (Eq. 10 with W = X^T U_bar), T_C = T_V B_bar
  load_sq(G, rp, r, r, S.K, 0.0);
  __syncthreads();
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
