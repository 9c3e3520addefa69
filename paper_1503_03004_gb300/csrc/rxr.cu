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
constexpr int LD = RPMAX + 4;  // row stride of the float r x r arrays: 16-byte aligned rows
constexpr int LDD = RPMAX;     // row stride of the float64 r x r arrays (read along rows only)
constexpr int kThreads = 512;

__device__ __forceinline__ bool stopped(const DevState* st) { return *(volatile const int32_t*)&st->done != 0; }

// GB300 issues float64 arithmetic at about two operations per clock per SM, so every float64
// instruction that all 512 threads execute costs ~0.1 us.  The kernel therefore keeps float64 to
// the products and the few element-wise steps that need it, takes scalar float64 math on one
// thread, and does comparisons and float64 <-> float32 conversions with integer operations.

// |x| as an integer (ordered like |x| for non-NaN values; NaN sorts above +inf).
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
constexpr long long kInfBits = 0x7ff0000000000000LL;

// float32 value of x 2^-e, rounded to nearest even, for |x 2^-e| < 2; results below the float32
// normal range flush to zero.  Integer operations only.
__device__ __forceinline__ float f64_to_f32_shift(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7ff) - 1023 - e + 127;
  if (ex <= 0 || ((b >> 52) & 0x7ff) == 0) return __uint_as_float(sign);
  const unsigned long long mant = b & 0xfffffffffffffULL;
  const unsigned long long rest = mant & ((1ULL << 29) - 1);
  unsigned bits = ((unsigned)ex << 23) | (unsigned)(mant >> 29);
  if (rest > (1ULL << 28) || (rest == (1ULL << 28) && (bits & 1u))) bits += 1;  // carries into the exponent
  return __uint_as_float(bits | sign);
}

// Exact float64 value of f 2^e (f a normal float32 or zero; subnormals flush to zero).  Integer
// operations only.
__device__ __forceinline__ double f32_to_f64_shift(float f, int e) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xff;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (ex == 0) return __longlong_as_double((long long)sign);
  const unsigned long long b = sign | ((unsigned long long)(ex - 127 + 1023 + e) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64_shift(x, 0); }

// C = epi(op(A) B) with float64 arithmetic, rows split across the cluster and broadcast through
// DSMEM.  A is a float64 array (row stride LDD); B is float64 (LDD) or float (LD), converted on
// load; C is float64 (LDD) or float (LD) and receives epi(i, j, (op(A) B)_ij).  C must not alias A
// or B.  On return every CTA holds the full product.
// PRE = false skips the barrier before the broadcast: allowed when no CTA has read C since the
// last cluster barrier.
template <bool TA, bool PRE = true, typename TB, typename TCo, typename Epi>
__device__ __noinline__ void mm_dist(const double* A, const TB* B, TCo* C, int r, Epi epi) {
  constexpr int ldb = sizeof(TB) == 8 ? LDD : LD;
  constexpr int ldc = sizeof(TCo) == 8 ? LDD : LD;
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
        const double a = TA ? A[(k + q) * LDD + i] : A[i * LDD + k + q];
        acc[q] = fma(a, to_f64(B[(k + q) * ldb + j]), acc[q]);
      }
    for (; k < r; ++k) {
      const double a = TA ? A[k * LDD + i] : A[i * LDD + k];
      acc[0] = fma(a, to_f64(B[k * ldb + j]), acc[0]);
    }
    C[i * ldc + j] = epi(i, j, (acc[0] + acc[1]) + (acc[2] + acc[3]));
  }
  __syncthreads();
  if (cs > 1) {
    if (PRE) cl.sync();  // every CTA is past its earlier reads of C
    // push this CTA's rows to the other CTAs in 16-byte pieces (column pairs of float64 or quads of
    // float; the last piece of a row may carry columns >= r, which no product or loop reads)
    constexpr int per16 = 16 / sizeof(TCo);
    const int npc = (r + per16 - 1) / per16, per = (i1 - i0) * npc;
    for (int e = threadIdx.x; e < (cs - 1) * per; e += blockDim.x) {
      const int q = 1 + e / per, w = e % per;
      const int i = i0 + w / npc, j = per16 * (w % npc);
      TCo* Cq = cl.map_shared_rank(C, (rank + q) % cs);
      *reinterpret_cast<float4*>(Cq + i * ldc + j) = *reinterpret_cast<const float4*>(C + i * ldc + j);
    }
    cl.sync();  // all rows have arrived everywhere
  }
}

// C = op(A) op(B) in float32 on the leading r x r blocks, 4 x 4 outputs per thread.  Operands
// move in 16-byte loads, 4 x 4 blocks of A and B per 4 steps of k (8 loads per 64 FMAs); the
// sum over k runs in order.  Reads may touch rows and columns beyond r (inside the RPMAX x LD
// arrays); only outputs inside r x r are written.
template <bool TA, bool TB>
__device__ __noinline__ void mmf(const float* A, const float* B, float* C, int r) {
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

// Block-wide maximum of 64-bit integers: shuffles within each warp, one shared slot per warp, then
// every thread reduces the (at most 32) warp values with shuffles again; the closing barrier lets
// `red` be reused at once.
__device__ __noinline__ long long block_max_ll(long long v, double* red) {
  long long* rl = reinterpret_cast<long long*>(red);
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (l == 0) rl[w] = v;
  __syncthreads();
  long long t = l < nw ? rl[l] : 0LL;
  for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
  __syncthreads();
  return t;
}

// float version (the sums and maxima it serves steer decisions only)
__device__ __noinline__ float block_reduce_f(float v, float* red, bool take_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(0xffffffffu, v, o);
    v = take_max ? fmaxf(v, w) : v + w;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = l < nw ? red[l] : (take_max ? -INFINITY : 0.f);
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_xor_sync(0xffffffffu, t, o);
    t = take_max ? fmaxf(t, u) : t + u;
  }
  __syncthreads();
  return t;
}

// Cyclic two-sided Jacobi on the symmetric n2 x n2 float matrix A (n2 even; rows/cols
// beyond r are zero), accumulating the rotations into Q (A_final = Q^T A_init Q).
// Round-robin ordering: n2/2 disjoint rotations per step, n2-1 steps per sweep.
__device__ __noinline__ void jacobi_f32(float* A, float* Q, int n2, int max_sweeps, double* red, float* cs, float* sn, int* pp,
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
        if (apq * apq > 1e-18f * fabsf(app * aqq) && apq != 0.f) {
          // the angle only steers convergence (c^2 + s^2 = 1 holds for any t): fast approximations
          const float th = __fdividef(aqq - app, 2.f * apq);
          const float h = 1.f + th * th;
          const float t = fabsf(th) > 1e15f ? __fdividef(0.5f, th)
                                           : __fdividef(copysignf(1.f, th), fabsf(th) + h * rsqrtf(h));
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
        if (apq * apq > 1e-18f * fabsf(app * aqq) && apq != 0.f) {
          const float th = __fdividef(aqq - app, 2.f * apq);
          const float h = 1.f + th * th;
          float t;
          if (fabsf(th) > 1e15f) t = __fdividef(0.5f, th);
          else t = __fdividef(copysignf(1.f, th), fabsf(th) + h * rsqrtf(h));
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

// A = (B Q)^T G (B Q) kn = kn Q^T K Q for the float32 copies Bf, Gf (three products; K itself is
// never formed).  The padding row and column r of an odd-sized Jacobi problem (n2 = r + 1) are zero.
__device__ __noinline__ void gram_in_basis(const float* Bf, const float* Gf, const float* Q, float* A, float* F1,
                                           float* F2, int r, int n2, float kn) {
  mmf<false, false>(Bf, Q, F1, r);   // B Q
  mmf<false, false>(Gf, F1, F2, r);  // G B Q
  mmf<true, false>(F1, F2, A, r);    // (B Q)^T G B Q
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    A[i * LD + j] = (i < r && j < r) ? A[i * LD + j] * kn : 0.f;
  }
  __syncthreads();
}

// One first-order eigenbasis refinement round for a nearly diagonal A = Q^T K Q / s (float32):
// Q <- Q (I + E), E_pq = A_pq / (A_qq - A_pp) for p != q (the small-angle Jacobi rotation of
// every pair at once), then one Newton-Schulz re-orthonormalisation, and the second-order
// eigenvalue estimates lam_p = A_pp - sum_q A_pq E_pq (A itself is not recomputed).  Pairs with
// (relative) gaps below 1e-5 are left alone, since any basis of a cluster serves the Newton
// preconditioner.  Returns max |E|; above 0.25 (A not close enough to diagonal for the
// first-order step) nothing is changed.
__device__ __noinline__ float refine_round(float* Q, const float* A, float* F1, float* F2, float* lam, int r,
                                           double* red) {
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
  if (!(big <= 0.25f)) return big;
  // lam_p = A_pp - sum_q A_pq E_pq: one warp per row
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int p = threadIdx.x >> 5; p < r; p += nw) {
    float acc = 0.f;
    for (int q = lane; q < r; q += 32) acc = fmaf(A[p * LD + q], F1[p * LD + q], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) lam[p] = A[p * LD + p] - acc;
  }
  mmf<false, false>(Q, F1, F2, r);                  // Q E (ends with a barrier)
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
  return big;
}

struct RxrSmem {
  double G[RPMAX * LDD];   // Gram of the thin factor (float64 sum of the partials); later B_bar
  double T[RPMAX * LDD];   // T_hat = B Z_hat (Newton iterate); scratch vectors of the rank test
  double W[RPMAX * LDD];   // B (until T_hat exists), then G T_hat
  float Gf[RPMAX * LD];    // G 2^-eg (float32; the power of two keeps K = B G B finite)
  float Bf[RPMAX * LD];    // B 2^-eb
  float QT[RPMAX * LD];    // Q^T
  float Af[RPMAX * LD];    // Q^T K Q / s (K = B G B), the Jacobi matrix, then the Newton correction in that basis
  float Qf[RPMAX * LD];    // approximate eigenbasis of K
  float F1[RPMAX * LD];    // scratch
  float F2[RPMAX * LD];    // scratch
  float lam[RPMAX], sq[RPMAX], isq[RPMAX];
  double red[32];
  float cs[RPMAX / 2], sn[RPMAX / 2];
  int pp[RPMAX / 2], qq[RPMAX / 2];
  double scale, inv_s, rs;  // s = trace(B G B) / r, 1 / s, 1 / sqrt(s)  (written by thread 0)
  float kn;                 // r / trace of the scaled float32 K
  int ok;
};

// Epilogues of mm_dist: the product itself, or I - product / s rounded to float32.
struct PlainEpi {
  __device__ double operator()(int, int, double v) const { return v; }
};
struct ResidEpi {
  double inv_s;
  __device__ float operator()(int i, int j, double v) const { return (float)((i == j ? 1.0 : 0.0) - v * inv_s); }
};

__device__ void fail(DevState* st, int code) {
  if (threadIdx.x == 0 && cg::this_cluster().block_rank() == 0) { st->status = code; st->done = 1; }
}

// Unbiased binary exponent of the largest |x| whose bits are `bits` (0 for 0).
__device__ __forceinline__ int exponent_of(long long bits) { return bits ? (int)(bits >> 52) - 1023 : 0; }

// v_side = false: T_U = B (B G_P B)^{-1/2}.
// v_side = true:  T_V = B (B G_W B)^{-1/2}, B <- Sym(G_W T_V), T_C = T_V B.
//
// With K = B G B and s = trace(K) / r, let Z be (K / s)^{-1/2}; then T = B Z / sqrt(s).  The kernel
// carries T_hat = B Z instead of Z: Newton's residual for Z K Z = I is
//     R = I - Z K Z = I - T_hat^T (G T_hat) / s,
// so float64 products form T_hat, W = G T_hat and T_hat^T W only, and K itself is needed in
// float32 alone (for the eigenbasis that preconditions Newton).  A Newton correction Delta of Z
// (float32, small) moves T_hat by B Delta and W by G B Delta, formed in float32: their rounding
// is float32-relative to the correction, and the next residual is formed in float64 again.
// float64: G, B, T_hat, W, R, B_bar, T_C.  float32: K, the eigenbasis, eigenvalue estimates, Z0
// and the Newton corrections, which only steer the iteration.  The mixed path also forms the
// starting T_hat = B Z0 and T_C in float32 (its U, V and C are float32).  Outputs are written by
// rows, each CTA of the cluster its own slice.
__device__ __forceinline__ void rxr_body(const VGrid& vg__, const double* __restrict__ Gg, int rp, int r,
                                         double* __restrict__ Bg, double* __restrict__ Tout,
                                         double* __restrict__ TCout, const float* __restrict__ Qin,
                                         float* __restrict__ Qeig, int v_side, int mixed, DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RxrSmem& S = *reinterpret_cast<RxrSmem*>(smem_raw);
  float* redf = reinterpret_cast<float*>(S.red);
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x;
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const bool writer = crank == 0;
  const int rpc = (r + cs - 1) / cs, row0 = min(r, crank * rpc), row1 = min(r, row0 + rpc);  // own rows
  const int n2 = (r + 1) & ~1;  // Jacobi works on an even size (row / column r zero when r is odd)
  // 1. G and B in float64 (B in W until T_hat exists), their power-of-two-scaled float32 copies,
  //    and the warm-start eigenbasis (Qin)
  constexpr int PER = RPMAX * RPMAX / kThreads;
  double gv[PER], bv[PER];
  long long gmax = 0, bmax = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = tid + q * kThreads, i = e / RPMAX, j = e % RPMAX;
    const bool in = i < r && j < r;
    gv[q] = in ? Gg[i * rp + j] : 0.0;
    bv[q] = in ? Bg[i * rp + j] : 0.0;
    gmax = max(gmax, abs_bits(gv[q]));
    bmax = max(bmax, abs_bits(bv[q]));
  }
  load_sq(Qin, rp, r, n2, S.Qf, 1.f);
  gmax = block_max_ll(gmax, S.red);
  bmax = block_max_ll(bmax, S.red);
  if (gmax >= kInfBits || bmax >= kInfBits || bmax == 0) { fail(st, SFR_E_NAN); return; }
  const int eg = exponent_of(gmax), eb = exponent_of(bmax);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = tid + q * kThreads, i = e / RPMAX, j = e % RPMAX;
    S.G[i * LDD + j] = gv[q];
    S.W[i * LDD + j] = bv[q];
    S.Gf[i * LD + j] = f64_to_f32_shift(gv[q], eg);
    S.Bf[i * LD + j] = f64_to_f32_shift(bv[q], eb);
  }
  __syncthreads();
  // 2. A = Q^T K Q in the previous call's basis Q (float32, from the scaled copies:
  //    K 2^-(eg + 2 eb)); s = trace(K) / r = trace(A) / r; A <- A / s
  gram_in_basis(S.Bf, S.Gf, S.Qf, S.Af, S.F1, S.F2, r, n2, 1.f);
  const float trf = block_reduce_f(tid < r ? S.Af[tid * LD + tid] : 0.f, redf, false);
  if (tid == 0) {
    // s = 2^(2k), the even power of two nearest below trace(B G B) / r (within a factor 4 of
    // it), so that 1 / s and 1 / sqrt(s) are exact and need no float64 division or square root;
    // A is scaled by K's power-of-two scale over s, exactly, so that its eigenvalues are those
    // of K / s.
    int e1 = 0;
    frexpf(trf / (float)r, &e1);  // trf / r = f 2^e1, f in [0.5, 1)
    const int tot = e1 + eg + 2 * eb, k = (tot >= 0 ? tot : tot - 1) / 2;  // floor(tot / 2)
    S.ok = trf > 0.f && trf < 3e38f && 2 * k > -1000 && 2 * k < 1000;
    auto pow2 = [](int e) { return __longlong_as_double((long long)(1023 + e) << 52); };
    S.scale = pow2(2 * k);
    S.inv_s = pow2(-2 * k);
    S.rs = pow2(-k);
    S.kn = ldexpf(1.f, eg + 2 * eb - 2 * k);
  }
  __syncthreads();
  if (!S.ok) { fail(st, SFR_E_NAN); return; }
  const float kn = S.kn;
  for (int e = tid; e < r * r; e += blockDim.x) S.Af[(e / r) * LD + e % r] *= kn;
  __syncthreads();
  // 3. eigenbasis: refine the previous basis to first order (cheap) while its rotation is small;
  //    a round whose rotation is at most 1e-3 leaves the basis accurate to ~1e-6 and is the last,
  //    a larger one is followed by a fresh A; float32 Jacobi sweeps only when that does not converge
  bool accepted = false;
  for (int round = 0; round < 3 && !accepted; ++round) {
    const float big = refine_round(S.Qf, S.Af, S.F1, S.F2, S.lam, n2, S.red);
    if (!(big <= 0.25f)) break;                      // A unchanged, Q unchanged
    accepted = big <= 1e-3f;
    if (!accepted) gram_in_basis(S.Bf, S.Gf, S.Qf, S.Af, S.F1, S.F2, r, n2, kn);
  }
  const bool rotated = !accepted;
  if (rotated) {
    jacobi_f32(S.Af, S.Qf, n2, 10, S.red, S.cs, S.sn, S.pp, S.qq);
    // re-orthonormalise the float basis: Q <- Q (3I - Q^T Q) / 2
    mmf<true, false>(S.Qf, S.Qf, S.F1, r);
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.F1[i * LD + j] = 0.5f * ((i == j ? 3.f : 0.f) - S.F1[i * LD + j]);
    }
    __syncthreads();
    mmf<false, false>(S.Qf, S.F1, S.F2, r);
    for (int e = tid; e < r * r; e += blockDim.x) S.Qf[(e / r) * LD + e % r] = S.F2[(e / r) * LD + e % r];
    __syncthreads();
    // 4. eigenvalue estimates after Jacobi: the diagonal of A (Rayleigh quotients of the basis)
    for (int p = tid; p < r; p += blockDim.x) S.lam[p] = S.Af[p * LD + p];
  }
  // (after a refinement round lam holds its second-order estimates); those far below the largest
  // are recomputed in float64 for the rank test (Eq. 9 needs rank r)
  __syncthreads();
  float hi = 0.f;
  for (int p = tid; p < r; p += blockDim.x) hi = fmaxf(hi, S.lam[p]);
  hi = block_reduce_f(hi, redf, true);
  float anysmall = 0.f;
  for (int p = tid; p < r; p += blockDim.x)
    if (S.lam[p] < 1e-6f * hi) anysmall = 1.f;
  anysmall = block_reduce_f(anysmall, redf, true);
  if (anysmall > 0.f && rotated) {
    // Jacobi stopped at a 1e-3 off-diagonal, so a basis vector of a tiny eigenvalue still mixes
    // ~1e-3 of the large ones and its Rayleigh quotient sits near 1e-6 hi: two first-order rounds
    // (near-degenerate pairs are skipped) bring the mixing down to float32 rounding first.
    for (int round = 0; round < 2; ++round) {
      gram_in_basis(S.Bf, S.Gf, S.Qf, S.Af, S.F1, S.F2, r, n2, kn);
      if (!(refine_round(S.Qf, S.Af, S.F1, S.F2, S.lam, n2, S.red) <= 0.25f)) {
        for (int p = tid; p < r; p += blockDim.x) S.lam[p] = S.Af[p * LD + p];
        break;
      }
    }
    __syncthreads();
    hi = 0.f;
    for (int p = tid; p < r; p += blockDim.x) hi = fmaxf(hi, S.lam[p]);
    hi = block_reduce_f(hi, redf, true);
  }
  // A float32 eigenvector carries components of about 1e-7 along the large eigenvectors, which
  // alone would add ~1e-14 hi to its Rayleigh quotient (the rank threshold): project them out in
  // float64 first (q <- q - Q_L Q_L^T q over the columns of large eigenvalues), then take
  // q^T K q / (s q^T q) = (B q)^T G (B q) / (s q^T q) with float64 matrix-vector products.
  double* qs = S.T;            // the vector (T_hat is free until step 6)
  double* cf = S.T + LDD;      // its coefficients on the large eigenvectors
  double* bq = S.T + 2 * LDD;  // B q
  for (int p = 0; anysmall > 0.f && p < r; ++p) {
    if (!(S.lam[p] < 1e-6f * hi)) continue;  // uniform: lam is in shared memory
    if (tid < r) qs[tid] = (double)S.Qf[tid * LD + p];
    __syncthreads();
    if (tid < r) {
      double c = 0.0;
      if (!(S.lam[tid] < 1e-6f * hi))
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
    if (tid < r) {
      double v = 0.0;
      for (int k = 0; k < r; ++k) v = fma(S.W[tid * LDD + k], qs[k], v);  // (B q)_tid
      bq[tid] = v;
    }
    __syncthreads();
    double num = 0.0, den = 0.0;
    if (tid < r) {
      double gq = 0.0;
      for (int k = 0; k < r; ++k) gq = fma(S.G[tid * LDD + k], bq[k], gq);  // (G B q)_tid
      num = bq[tid] * gq;
      den = qi * qi;
    }
    if (tid >= 64) num = den = 0.0;  // r <= 64: the first two warps hold every term
    if (tid < 64) {
      for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
      }
    }
    if (tid == 0) S.red[0] = num, S.red[1] = den;
    __syncthreads();
    if (tid == 32) S.red[2] = num, S.red[3] = den;
    __syncthreads();
    if (tid == 0) S.lam[p] = (float)((S.red[0] + S.red[2]) / (S.red[1] + S.red[3]) * S.inv_s);
    __syncthreads();
  }
  float nlo = -hi, badf = 0.f;  // max of -lambda and of the rank-failure flag
  for (int p = tid; p < r; p += blockDim.x) {
    nlo = fmaxf(nlo, -S.lam[p]);
    if (!(S.lam[p] > 1e-14f * hi)) badf = 1.f;
  }
  const float lo = -block_reduce_f(nlo, redf, true);
  const bool bad = block_reduce_f(badf, redf, true) > 0.f || !(hi > 0.f);
  if (writer && tid == 0) {
    if (v_side) st->lam_min_v = (double)lo * S.scale; else st->lam_min_u = (double)lo * S.scale;
  }
  if (bad) { fail(st, SFR_E_RANK); return; }
  for (int p = tid; p < r; p += blockDim.x) {
    const float sq = sqrtf(S.lam[p]);
    S.sq[p] = sq;
    S.isq[p] = 1.f / sq;
  }
  float* QT = S.QT;
  for (int e = tid; e < r * r; e += blockDim.x) QT[(e % r) * LD + e / r] = S.Qf[(e / r) * LD + e % r];
  __syncthreads();
  // 5. Z0 = Q diag(lambda^{-1/2}) Q^T (float32 start; Newton below brings it to float64 accuracy)
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S.F2[i * LD + j] = S.Qf[i * LD + j] * S.isq[j];
  }
  __syncthreads();
  mmf<false, false>(S.F2, QT, S.F1, r);
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    S.F2[i * LD + j] = 0.5f * (S.F1[i * LD + j] + S.F1[j * LD + i]);
  }
  __syncthreads();
  // 6. T_hat = B Z0.  Float64 path: float64 products of B with the float32 values of Z0, rows
  //    split across the cluster.  Mixed path: a float32 product of the scaled copy of B, in every
  //    CTA.  Newton below corrects the symmetric part of Z only, so the float32 rounding of T_hat
  //    stays as a rotation of the polar factor of about 1e-7, the size of the mixed path's own
  //    rounding of U and V.
  const PlainEpi plain;
  if (mixed) {
    mmf<false, false>(S.Bf, S.F2, S.F1, r);  // B Z0 2^-eb
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.T[i * LDD + j] = f32_to_f64_shift(S.F1[i * LD + j], eb);
    }
    __syncthreads();
    if (cs > 1) cl.sync();  // every CTA is past its reads of W (still B) before W rows arrive
  } else {
    mm_dist<false>(S.W, S.F2, S.T, r, plain);
  }
  // 7. Newton steps on Z K Z = I: R = I - T_hat^T (G T_hat) / s in float64, correction in float32
  bool w_stale = false;  // W lags T_hat by G (B Delta)
  for (int it = 0; it < 6; ++it) {
    // W was last read by the previous product (T_hat0 = B Z0 or the residual), F1 by this CTA
    // alone before that product's closing barrier: neither needs a barrier before its broadcast
    mm_dist<false, false>(S.G, S.T, S.W, r, plain);               // W = G T_hat
    mm_dist<true, false>(S.T, S.W, S.F1, r, ResidEpi{S.inv_s});  // I - Z K Z, rounded to float32
    w_stale = false;
    float rmax = 0.f;
    for (int e = tid; e < r * r; e += blockDim.x) rmax = fmaxf(rmax, fabsf(S.F1[(e / r) * LD + e % r]));
    const float rm = block_reduce_f(rmax, redf, true);
    if (!(rm == rm)) { fail(st, SFR_E_NAN); return; }
    if (rm < 4e-16f * r) break;
    for (int e = tid; e < r * r; e += blockDim.x) {  // R = Sym(I - Z K Z)
      const int i = e / r, j = e % r;
      S.F2[i * LD + j] = 0.5f * (S.F1[i * LD + j] + S.F1[j * LD + i]);
    }
    __syncthreads();
    mmf<false, false>(S.F2, S.Qf, S.F1, r);    // R Q
    mmf<true, false>(S.Qf, S.F1, S.Af, r);     // Q^T R Q
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int p = e / r, q = e % r;
      S.Af[p * LD + q] = __fdividef(S.Af[p * LD + q], S.sq[p] + S.sq[q]);
    }
    __syncthreads();
    mmf<false, false>(S.Af, QT, S.F2, r);      // Dt Q^T
    mmf<false, false>(S.Qf, S.F2, S.F1, r);    // Q Dt Q^T
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.F2[i * LD + j] = 0.5f * (S.F1[i * LD + j] + S.F1[j * LD + i]);  // Delta (symmetric)
    }
    __syncthreads();
    mmf<false, false>(S.Bf, S.F2, S.F1, r);    // B Delta 2^-eb
    // The step just taken leaves a residual of about (eigenbasis error + float32 rounding of the
    // correction) x rm + O(rm^2): from rm < 3e-6 about 1e-11 (mixed path, whose Gram carries
    // float32 rounding), from rm < 1e-7 about 1e-14 (float64 path), so stop without forming it again
    // and update only this CTA's rows of T_hat (the rows it writes).
    const bool last = rm < (mixed ? 3e-6f : 1e-7f) || it == 5;
    const int e0 = last ? row0 * r : 0, e1 = last ? row1 * r : r * r;
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.T[i * LDD + j] += f32_to_f64_shift(S.F1[i * LD + j], eb);
    }
    __syncthreads();
    w_stale = true;
    if (last) break;
  }
  // 8. T = B (B G B)^{-1/2} = T_hat / sqrt(s): this CTA's rows, and its rows of the basis
  const double rs = S.rs;
  for (int e = row0 * rp + tid; e < row1 * rp; e += blockDim.x) {
    const int i = e / rp, j = e % rp;
    Tout[e] = j < r ? S.T[i * LDD + j] * rs : 0.0;
    Qeig[e] = j < r ? S.Qf[i * LD + j] : (i == j ? 1.f : 0.f);
  }
  if (writer)
    for (int e = r * rp + tid; e < rp * rp; e += blockDim.x) {  // padding rows
      const int i = e / rp, j = e % rp;
      Tout[e] = 0.0;
      Qeig[e] = i == j ? 1.f : 0.f;
    }
  if (!v_side) return;
  // 9. B_bar = Sym(G_W T_V) (Eq. 10 with W = X^T U_bar) = Sym(G T_hat) / sqrt(s), T_C = T_V B_bar.
  //    W lags T_hat by the last correction: W + G (B Delta), the latter in float32.  Every CTA forms
  //    its rows of B_bar and sends them to the others (nobody reads G after the last W product).
  if (w_stale) mmf<false, false>(S.Gf, S.F1, S.F2, r);  // G B Delta 2^-(eg + eb)
  for (int e = row0 * r + tid; e < row1 * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double v = S.W[i * LDD + j] + S.W[j * LDD + i];
    if (w_stale) v += f32_to_f64_shift(S.F2[i * LD + j] + S.F2[j * LD + i], eg + eb);
    S.G[i * LDD + j] = 0.5 * rs * v;
  }
  __syncthreads();
  if (cs > 1) {
    const int npc = (r + 1) / 2, per = (row1 - row0) * npc;
    for (int e = tid; e < (cs - 1) * per; e += blockDim.x) {
      const int q = 1 + e / per, w = e % per;
      const int i = row0 + w / npc, j = 2 * (w % npc);
      double* Gq = cl.map_shared_rank(S.G, (crank + q) % cs);
      *reinterpret_cast<double2*>(Gq + i * LDD + j) = *reinterpret_cast<const double2*>(S.G + i * LDD + j);
    }
    cl.sync();
  }
  // this CTA's rows: B_bar, and T_C = T_V B_bar = (T_hat rows) B_bar / sqrt(s).  T_C only forms
  // C = W T_C, which the mixed path stores in float32: there float32 products suffice.
  if (mixed) {
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.Af[i * LD + j] = f64_to_f32_shift(S.G[i * LDD + j], 0);
    }
    for (int e = row0 * r + tid; e < row1 * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      S.F2[i * LD + j] = f64_to_f32_shift(S.T[i * LDD + j], 0);
    }
    __syncthreads();
  }
  for (int e = row0 * rp + tid; e < row1 * rp; e += blockDim.x) {
    const int i = e / rp, j = e % rp;
    double tc = 0.0;
    if (j < r && mixed) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int k = 0;
      for (; k + 4 <= r; k += 4)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(S.F2[i * LD + k + q], S.Af[(k + q) * LD + j], acc[q]);
      for (; k < r; ++k) acc[0] = fmaf(S.F2[i * LD + k], S.Af[k * LD + j], acc[0]);
      tc = f32_to_f64_shift((acc[0] + acc[1]) + (acc[2] + acc[3]), 0);
    } else if (j < r) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int k = 0;
      for (; k + 4 <= r; k += 4)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(S.T[i * LDD + k + q], S.G[(k + q) * LDD + j], acc[q]);
      for (; k < r; ++k) acc[0] = fma(S.T[i * LDD + k], S.G[k * LDD + j], acc[0]);
      tc = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    Bg[e] = j < r ? S.G[i * LDD + j] : 0.0;
    TCout[e] = j < r ? tc * rs : 0.0;
  }
  if (writer)
    for (int e = r * rp + tid; e < rp * rp; e += blockDim.x) {
      Bg[e] = 0.0;
      TCout[e] = 0.0;
    }
}


}  // namespace

// Cluster size for the r x r kernel: 16 CTAs (non-portable size) when the device accepts it
// with this kernel's shared memory, else 8, else a single CTA.  The result does not depend on
// it (every float64 product element is one thread's loop; the float32 work is redundant).
static int rxr_cluster_size(size_t smem) {
  static int cached = 0;
  if (cached) return cached;
  auto kern = body_kernel_of<&rxr_body, kThreads>();
  int best = 1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    cudaGetLastError();
  if (set_smem_attr<body_kernel_of<&rxr_body, kThreads>()>(smem) != cudaSuccess) cudaGetLastError();
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0) {
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
  const int cs = rxr_cluster_size(smem);
  // warm start: the U side from its own basis of the previous iteration; the V side from the U
  // side's basis of this iteration (both K share B, and their eigenbases meet as the iteration
  // settles, so the V side's first-order refinement holds from the fourth iteration on)
  return launch_k_cluster<&rxr_body, kThreads>(cs, kThreads, smem, st, (const double*)b.Gsum, s.rp, s.r, b.B,
                                              v_side ? b.TV : b.TU, v_side ? b.TCm : (double*)nullptr,
                                              (const float*)b.Qeig_u, v_side ? b.Qeig_v : b.Qeig_u,
                                              v_side ? 1 : 0, fp64 ? 0 : 1, b.st);
}

}  // namespace sfr
