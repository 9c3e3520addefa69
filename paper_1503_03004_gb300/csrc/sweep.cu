// m x n and thin (m x r, n x r) kernels of one FR-ADM iteration (Algorithm 1 with
// the L-step of Algorithm 3), SIMT version for float64 (FP64 path) and float32
// (mixed path) arithmetic.
//
// Notation (Algorithm 1): X_k = M - S_k + Y_k / mu_k, the matrix handed to
// FixedRankOptStep.  The L-step computes
//     P = X_k V_k,  U_bar = P_O[P B_k],  W = X_k^T U_bar,  V_bar = P_O[W B_k],
//     B_bar = Sym(U_bar^T X_k V_bar) = Sym(W^T V_bar)                 (Algorithm 3)
// and the S/Y steps use z = M - L_{k+1} + Y_k / mu_k:
//     S_{k+1} = P_ST_{1/mu_k}(z),   Y_{k+1} = Y_k + mu_k (M - L_{k+1} - S_{k+1}).
// Since Y_k + mu_k (z - Y_k/mu_k - P_ST(z)) = mu_k (z - P_ST(z)) = clip(mu_k z, -1, 1),
// the sweep stores Y_{k+1} = clip(mu_k z, -1, 1) and never stores S (it is rebuilt
// once at the end).  The next iteration's X is
//     X_{k+1} = M - S_{k+1} + Y_{k+1}/mu_{k+1} = L_{k+1} + Delta_{k+1},
//     Delta_{k+1} = Y_{k+1} (1/mu_k + 1/mu_{k+1}) - Y_k / mu_k,
// so the sweep writes Delta and accumulates P_{k+1} = X_{k+1} V_{k+1} row by row,
// and the second pass forms X_{k+1}^T U = C (U_old^T U) + Delta^T U with L = U_old C^T.
#include <algorithm>
#include <type_traits>

#include "sfr_internal.h"

namespace sfr {
namespace {

template <typename T> __device__ __forceinline__ T from_bf16(__nv_bfloat16 v) { return (T)__bfloat162float(v); }
template <typename TC, typename TS> __device__ __forceinline__ TC ld_as(const TS* p) { return (TC)(*p); }
template <> __device__ __forceinline__ float ld_as<float, __nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ double ld_as<double, __nv_bfloat16>(const __nv_bfloat16* p) { return (double)__bfloat162float(*p); }

__device__ __forceinline__ bool stopped(const DevState* st) { return *(volatile const int32_t*)&st->done != 0; }

// Block-wide sum of a double; every thread gets the result.  blockDim.x <= 1024.
// Residual partial of one warp over one row block of a column split of the SIMT mixed sweeps:
// slot (split, row block, warp), so that the partials (and their fixed-order sum in the
// iteration end) do not depend on how many CTAs the sweep runs.
__device__ __forceinline__ void resid_store_warp(float resid, double* __restrict__ resid_part, int64_t split,
                                                 int64_t nrb, int64_t rb) {
  double v = (double)resid;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) resid_part[(split * nrb + rb) * 8 + (threadIdx.x >> 5)] = v;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];  // fixed order: deterministic
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------- ||M||_F
template <typename TMs>
__global__ void norm_m_kernel(const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm, double* part) {
  pdl_enter();
  __shared__ double red[32];
  constexpr int64_t V = 16 / sizeof(TMs);  // elements per 16-byte load
  double acc = 0.0;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const TMs* row = M + i * ldm;
    // the elements before the row's first 16-byte boundary, whole 16-byte chunks, the tail
    const int64_t head = min(n, (int64_t)(((16 - ((uintptr_t)row & 15)) & 15) / sizeof(TMs)));
    const int64_t nv = (n - head) / V;
    float a = 0.f;
    for (int64_t j = threadIdx.x; j < head; j += blockDim.x) {
      const float v = ld_as<float, TMs>(row + j);
      a = fmaf(v, v, a);
    }
    const uint4* vrow = reinterpret_cast<const uint4*>(row + head);
#pragma unroll 4
    for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) {
      const uint4 w = __ldg(vrow + c);
      const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (sizeof(TMs) == 2) {  // two bfloat16 values: their bits are a float's top half
          const float lo = __uint_as_float(q[k] << 16), hi = __uint_as_float(q[k] & 0xffff0000u);
          a = fmaf(lo, lo, a);
          a = fmaf(hi, hi, a);
        } else {
          const float v = __uint_as_float(q[k]);
          a = fmaf(v, v, a);
        }
      }
    }
    for (int64_t j = head + nv * V + threadIdx.x; j < n; j += blockDim.x) {
      const float v = ld_as<float, TMs>(row + j);
      a = fmaf(v, v, a);
    }
    acc += (double)a;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <>
__global__ void norm_m_kernel<double>(const double* __restrict__ M, int64_t m, int64_t n, int64_t ldm, double* part) {
  pdl_enter();
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double v = M[i * ldm + j];
      acc = fma(v, v, acc);
    }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// ---------------------------------------------------------------- first P = M[:, :r]
// Iteration 1: X_1 = M (S = Y = 0), V_1 = I_{n x r}, so P = X_1 V_1 = M[:, 0:r].
template <typename TC, typename TMs>
__global__ void init_p_kernel(const TMs* __restrict__ M, int64_t m, int64_t ldm, int r, int rp, TC* P) {
  pdl_enter();
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * rp) return;
  int64_t i = idx / rp;
  int a = (int)(idx % rp);
  P[idx] = a < r ? ld_as<TC, TMs>(M + i * ldm + a) : (TC)0;
}

// ---------------------------------------------------------------- register-blocked small products
// C[R x N] = op(A)[R x K] B[K x N] on shared-memory operands, 4 x 4 outputs per thread:
// thread t < (R/4)(N/4) owns rows 4(t / (N/4)) .. +3 and columns 4(t % (N/4)) .. +3.
// op(A) = A (element (i, k) at A[i * lda + k]) or A^T (element (i, k) at A[k * lda + i]).
template <typename T, int R, int N, int K, bool TA>
__device__ __forceinline__ void block_mm(const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb,
                                         T (&acc)[4][4], int t) {
  constexpr int NB = N / 4;
  if (t >= (R / 4) * NB) return;
  const int i0 = 4 * (t / NB), j0 = 4 * (t % NB);
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    T a[4], bb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = TA ? A[k * lda + i0 + q] : A[(i0 + q) * lda + k];
      bb[q] = B[k * ldb + j0 + q];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * bb[y];
  }
}

template <typename T>
__device__ __forceinline__ void zero44(T (&acc)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0;
}

// The thin kernels run 256 threads; their global loads are unrolled with compile-time trip
// counts so that every load of a thread is in flight before the first shared-memory store.
constexpr int kThinThreads = 256;

// Gram-type products A^T B of two 64-row tiles (RP x RP output) with the 64-row sum split over
// all threads: thread t owns output block t % G (4 x 4, G = (RP/4)^2) and the rows congruent to
// t / G modulo 256 / G, accumulated across tiles; gram_store sums the row groups in a fixed order
// at the end.  (With one 4 x 4 block per thread only G threads would work: 4 of 256 at RP = 8.)
template <int RP> struct GramSplit {
  static constexpr int NB = RP / 4, G = NB * NB, KG = kThinThreads / G;
};

template <typename T, int RP>
__device__ __forceinline__ void gram_slice(const T* __restrict__ A, const T* __restrict__ B, int ld, T (&acc)[4][4],
                                           int t) {
  using GS = GramSplit<RP>;
  const int blk = t % GS::G, kg = t / GS::G;
  const int i0 = 4 * (blk / GS::NB), j0 = 4 * (blk % GS::NB);
#pragma unroll 4
  for (int k = kg; k < kGramRows; k += GS::KG) {
    T a[4], bb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = A[k * ld + i0 + q];
      bb[q] = B[k * ld + j0 + q];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * bb[y];
  }
}

// out[RP x RP] (float64) = the sum over row groups of the threads' gram_slice accumulators.
// `red` is shared scratch of 256 x 16 T (unused when the split is 1, RP = 64).
template <typename T, int RP>
__device__ __forceinline__ void gram_store(const T (&acc)[4][4], int t, T* red, double* __restrict__ out) {
  using GS = GramSplit<RP>;
  if constexpr (GS::KG == 1) {
    const int i0 = 4 * (t / GS::NB), j0 = 4 * (t % GS::NB);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) out[(i0 + x) * RP + j0 + y] = (double)acc[x][y];
  } else {
    __syncthreads();  // callers' last use of `red` (a tile buffer) is done
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) red[t * 16 + 4 * x + y] = acc[x][y];
    __syncthreads();
    for (int o = t; o < GS::G * 16; o += kThinThreads) {
      const int blk = o / 16, xy = o % 16;
      double v = 0.0;
      for (int kg = 0; kg < GS::KG; ++kg) v += (double)red[(kg * GS::G + blk) * 16 + xy];
      out[(4 * (blk / GS::NB) + xy / 4) * RP + 4 * (blk % GS::NB) + xy % 4] = v;
    }
  }
}

// s[RP x RP] (row stride LDT, type TC) = g[RP x RP] (float64, dense).
template <typename TC, int RP, int LDT>
__device__ __forceinline__ void load_rr(const double* __restrict__ g, TC* s, int t) {
  constexpr int PER = (RP * RP + kThinThreads - 1) / kThinThreads;
  double v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = t + q * kThinThreads;
    v[q] = e < RP * RP ? g[e] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = t + q * kThinThreads;
    if (e < RP * RP) s[(e / RP) * LDT + e % RP] = (TC)v[q];
  }
}

// Elements of a kGramRows x RP row tile owned by thread t: e = t + q * 256, q < RP / 4.
template <int RP>
struct TileIdx {
  static constexpr int PER = kGramRows * RP / kThinThreads;
  static __device__ __forceinline__ int row(int t, int q) { return (t + q * kThinThreads) / RP; }
  static __device__ __forceinline__ int col(int t, int q) { return (t + q * kThinThreads) % RP; }
};

// v[q] = src[(i0 + row) * RP + col] for the thread's elements (0 past `rows`).
template <typename TC, int RP>
__device__ __forceinline__ void load_tile(const TC* __restrict__ src, int64_t i0, int64_t rows, int t,
                                          TC (&v)[TileIdx<RP>::PER]) {
#pragma unroll
  for (int q = 0; q < TileIdx<RP>::PER; ++q) {
    const int64_t i = i0 + TileIdx<RP>::row(t, q);
    v[q] = i < rows ? src[i * RP + TileIdx<RP>::col(t, q)] : (TC)0;
  }
}

template <typename TC, int RP, int LDT>
__device__ __forceinline__ void store_tile(TC* s, int t, const TC (&v)[TileIdx<RP>::PER]) {
#pragma unroll
  for (int q = 0; q < TileIdx<RP>::PER; ++q) s[TileIdx<RP>::row(t, q) * LDT + TileIdx<RP>::col(t, q)] = v[q];
}

// ---------------------------------------------------------------- thin reduce + Gram partials
// For every 64-row tile handled by this CTA (tiles blockIdx.x, blockIdx.x + gridDim.x, ...):
// out[i][:] = sum_s parts[s][i][:] (times T2 when T2 != nullptr) (+ addA[i][:] H when
// addA != nullptr), then the CTA's Gram partial gpart[cta] = sum over its rows of
// out[i]^T out[i]  (r x r).  With `trans` (float, RP = 64), out is also written transposed as a
// two-term bfloat16 split: row a holds x rounded to bfloat16, row RP + a the rounding of the rest
// (ld ldt).  nparts == 0 leaves `out` as it is and only forms the Gram partial.  q_ctas > 0: the
// partials come from the persistent tensor-core sweep (q_tiles column tiles per 128-row block),
// and rows of block rb have tc_q_slots(rb) of them.
template <typename TC, int RP>
__device__ __forceinline__ void thin_gram_body(const VGrid& vg__, const TC* __restrict__ parts, int nparts, int64_t part_stride,
                                                        TC* __restrict__ out, int64_t rows, const TC* __restrict__ addA,
                                                        const double* __restrict__ H, double* __restrict__ gpart,
                                                        const DevState* st, int q_ctas, int64_t q_tiles,
                                                        const double* __restrict__ T2, __nv_bfloat16* __restrict__ trans,
                                                        int64_t ldt) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  constexpr int LDT = RP + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* tile = reinterpret_cast<TC*>(smem_raw);   // [kGramRows][LDT]
  TC* arow = tile + kGramRows * LDT;              // [kGramRows][LDT]  addA rows
  TC* Hs = arow + kGramRows * LDT;                // [RP][LDT]
  TC* T2s = Hs + RP * LDT;                        // [RP][LDT]
  TC* red = tile;                                 // after the tiles: 256 x 16 Gram scratch
  const int t = threadIdx.x;
  if (addA) load_rr<TC, RP, LDT>(H, Hs, t);
  if (T2) load_rr<TC, RP, LDT>(T2, T2s, t);
  TC g[4][4];
  zero44(g);
  const int64_t ntiles = (rows + kGramRows - 1) / kGramRows;
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t i0 = tl * kGramRows;
    TC v[TileIdx<RP>::PER];
    if (nparts == 0) {
      load_tile<TC, RP>(out, i0, rows, t, v);
    } else {
      int np = nparts;
      if (q_ctas > 0) {  // a 64-row tile lies in one 128-row block
        const int64_t nblk = (rows + 127) / 128;
        np = min(nparts, tc_q_slots(i0 / 128, q_tiles, nblk * q_tiles, q_ctas));
      }
      load_tile<TC, RP>(parts, i0, rows, t, v);
#pragma unroll 4
      for (int s = 1; s < np; ++s) {
        TC w[TileIdx<RP>::PER];
        load_tile<TC, RP>(parts + s * part_stride, i0, rows, t, w);
#pragma unroll
        for (int q = 0; q < TileIdx<RP>::PER; ++q) v[q] += w[q];
      }
    }
    TC av[TileIdx<RP>::PER];
    if (addA) load_tile<TC, RP>(addA, i0, rows, t, av);
    __syncthreads();  // previous tile consumed; Hs visible
    store_tile<TC, RP, LDT>(tile, t, v);
    if (addA) store_tile<TC, RP, LDT>(arow, t, av);
    __syncthreads();
    if (nparts > 0) {
      if (T2) {  // tile <- (sum of the partials) T2
        TC acc[4][4];
        zero44(acc);
        block_mm<TC, kGramRows, RP, RP, false>(tile, LDT, T2s, LDT, acc, t);
        __syncthreads();  // every read of the tile is done
        if (t < (kGramRows / 4) * (RP / 4)) {
          const int r0 = 4 * (t / (RP / 4)), c0 = 4 * (t % (RP / 4));
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) tile[(r0 + x) * LDT + c0 + y] = acc[x][y];
        }
        __syncthreads();
      }
      if (addA) {
        TC acc[4][4];
        zero44(acc);
        block_mm<TC, kGramRows, RP, RP, false>(arow, LDT, Hs, LDT, acc, t);
        if (t < (kGramRows / 4) * (RP / 4)) {
          const int r0 = 4 * (t / (RP / 4)), c0 = 4 * (t % (RP / 4));
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) tile[(r0 + x) * LDT + c0 + y] += acc[x][y];
        }
        __syncthreads();
      }
      for (int e = t; e < kGramRows * RP; e += blockDim.x) {
        const int ii = e / RP, a = e % RP;
        const int64_t i = i0 + ii;
        if (i < rows) out[i * RP + a] = tile[ii * LDT + a];
      }
    }
    if constexpr (std::is_same<TC, float>::value) {
      if (trans) {  // column a of the tile -> rows a (hi) and RP + a (lo) of the transpose
#pragma unroll
        for (int q = 0; q < TileIdx<RP>::PER; ++q) {
          const int e = t + q * kThinThreads, a = e / kGramRows, ii = e % kGramRows;
          const int64_t i = i0 + ii;
          if (i < rows) {
            const float x = tile[ii * LDT + a];
            const __nv_bfloat16 hb = __float2bfloat16_rn(x);
            trans[(int64_t)a * ldt + i] = hb;
            trans[(int64_t)(RP + a) * ldt + i] = __float2bfloat16_rn(x - __bfloat162float(hb));
          }
        }
      }
    }
    gram_slice<TC, RP>(tile, tile, LDT, g, t);
  }
  gram_store<TC, RP>(g, t, red, gpart + (int64_t)blockIdx.x * RP * RP);
}

// Sum of `count` partials of rpsq values into out, in a fixed order: warp w of a CTA of nw warps
// adds the partials w, w + nw, w + 2 nw, ... of 32 consecutive entries (four loads in flight),
// then the warp sums are added in warp order.  out may be the first partial (each entry is read
// and written by one CTA).  nw = blockDim.x / 32 <= 32.
template <typename T>
__device__ __forceinline__ void reduce_sq_body(const VGrid& vg__, const T* parts, int64_t count, int64_t rpsq, T* out,
                                                         const DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  __shared__ T red[32][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  T a = 0;
  if (e < rpsq) {
    int64_t c = warp;
    for (; c + 3 * nw < count; c += 4 * nw) {
      const T v0 = parts[c * rpsq + e], v1 = parts[(c + nw) * rpsq + e];
      const T v2 = parts[(c + 2 * nw) * rpsq + e], v3 = parts[(c + 3 * nw) * rpsq + e];
      a += v0;
      a += v1;
      a += v2;
      a += v3;
    }
    for (; c < count; c += nw) a += parts[c * rpsq + e];
  }
  red[warp][lane] = a;
  __syncthreads();
  if (warp == 0 && e < rpsq) {
    T s = red[0][lane];
    for (int w = 1; w < nw; ++w) s += red[w][lane];
    out[e] = s;
  }
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------- thin row transform
// dst[i][:] = src[i][:] T   (T rp x rp, float64 in global), optional second output
// dst2 = src T2, and optional partial hpart[cta] = sum over the CTA's rows of old[i]^T dst[i].
// Each CTA handles 64-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <typename TC, int RP>
__device__ __forceinline__ void row_transform_body(const VGrid& vg__, const TC* __restrict__ src, int64_t rows,
                                                            const double* __restrict__ T, TC* __restrict__ dst,
                                                            const double* __restrict__ T2, TC* __restrict__ dst2,
                                                            const TC* __restrict__ old, double* __restrict__ hpart,
                                                            const DevState* st, float* __restrict__ sp_hi,
                                                            float* __restrict__ sp_lo,
                                                            __nv_bfloat16* __restrict__ trans,
                                                            int64_t ldt, int trans_lo) {
  pdl_enter();
  SFR_VGRID(vg__);
  // Tensor-core path extras (float, RP = 64): sp_hi / sp_lo = TF32 split (hi = x rounded to TF32,
  // lo = x - hi) of dst2 (or of dst without T2), trans = dst transposed in bfloat16 (ld ldt);
  // trans_lo != 0: also the bfloat16 rounding of x - hi into row RP + a (a two-term split).
  if (stopped(st)) return;
  constexpr int LDT = RP + 4;
  constexpr bool kF32 = std::is_same<TC, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Ts = reinterpret_cast<TC*>(smem_raw);   // [RP][LDT]
  TC* T2s = Ts + RP * LDT;                     // [RP][LDT]
  TC* srow = T2s + RP * LDT;                   // [kGramRows][LDT]
  TC* drow = srow + kGramRows * LDT;           // [kGramRows][LDT]
  TC* orow = drow + kGramRows * LDT;           // [kGramRows][LDT]
  const int t = threadIdx.x;
  load_rr<TC, RP, LDT>(T, Ts, t);
  if (T2) load_rr<TC, RP, LDT>(T2, T2s, t);
  TC h[4][4];
  zero44(h);
  const int owner = t < (kGramRows / 4) * (RP / 4);
  const int r0 = 4 * (t / (RP / 4)), c0 = 4 * (t % (RP / 4));
  const int64_t ntiles = (rows + kGramRows - 1) / kGramRows;
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t i0 = tl * kGramRows;
    TC v[TileIdx<RP>::PER], ov[TileIdx<RP>::PER];
    load_tile<TC, RP>(src, i0, rows, t, v);
    if (hpart) load_tile<TC, RP>(old, i0, rows, t, ov);
    __syncthreads();
    store_tile<TC, RP, LDT>(srow, t, v);
    if (hpart) store_tile<TC, RP, LDT>(orow, t, ov);
    __syncthreads();
    TC acc[4][4];
    zero44(acc);
    block_mm<TC, kGramRows, RP, RP, false>(srow, LDT, Ts, LDT, acc, t);
    if (owner) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int64_t i = i0 + r0 + x;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          drow[(r0 + x) * LDT + c0 + y] = acc[x][y];
          if (i < rows) dst[i * RP + c0 + y] = acc[x][y];
          if constexpr (kF32) {
            if (!T2 && sp_hi && i < rows) {
              const float hv = to_tf32(acc[x][y]);
              sp_hi[i * RP + c0 + y] = hv;
              sp_lo[i * RP + c0 + y] = acc[x][y] - hv;
            }
          }
        }
      }
    }
    if (T2) {
      zero44(acc);
      block_mm<TC, kGramRows, RP, RP, false>(srow, LDT, T2s, LDT, acc, t);
      if (owner) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int64_t i = i0 + r0 + x;
          if (i < rows)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              dst2[i * RP + c0 + y] = acc[x][y];
              if constexpr (kF32) {
                if (sp_hi) {
                  const float hv = to_tf32(acc[x][y]);
                  sp_hi[i * RP + c0 + y] = hv;
                  sp_lo[i * RP + c0 + y] = acc[x][y] - hv;
                }
              }
            }
        }
      }
    }
    if (hpart || trans) __syncthreads();  // drow complete
    if (hpart) gram_slice<TC, RP>(orow, drow, LDT, h, t);
    if constexpr (kF32) {
      if (trans) {  // column a of the tile -> row a of the transpose, 64 consecutive rows i
#pragma unroll
        for (int q = 0; q < TileIdx<RP>::PER; ++q) {
          const int e = t + q * kThinThreads, a = e / kGramRows, ii = e % kGramRows;
          const int64_t i = i0 + ii;
          if (i < rows) {
            const float x = drow[ii * LDT + a];
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            trans[(int64_t)a * ldt + i] = hi;
            if (trans_lo) trans[(int64_t)(RP + a) * ldt + i] = __float2bfloat16_rn(x - __bfloat162float(hi));
          }
        }
      }
    }
  }
  if (hpart) gram_store<TC, RP>(h, t, srow, hpart + (int64_t)blockIdx.x * RP * RP);
}

// ---------------------------------------------------------------- W pass
// Wpart[c][j][:] = sum_{i in chunk c} src[i][j] U[i][:]   (the V-step product X^T U_bar of Algorithm 3).
// src is Delta (TC, ld n) from iteration 2 on, or M itself on iteration 1.
template <typename TC, typename TS, int RP>
__global__ void __launch_bounds__(256) wpass_kernel(const TS* __restrict__ src, int64_t lds, int64_t m, int64_t n,
                                                    int rows_per_chunk, const TC* __restrict__ U, TC* __restrict__ Wpart,
                                                    const DevState* st) {
  pdl_enter();
  if (stopped(st)) return;
  constexpr int APT = RP / 4;  // accumulators per thread
  __shared__ TC xs[kWBM][kWBN + 1];
  __shared__ TC us[kWBM][RP];
  const int64_t j0 = (int64_t)blockIdx.x * kWBN;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(m, r0 + rows_per_chunk);
  const int tj = threadIdx.x % kWBN, ta = threadIdx.x / kWBN;
  TC acc[APT];
#pragma unroll
  for (int c = 0; c < APT; ++c) acc[c] = 0;
  for (int64_t it = r0; it < r1; it += kWBM) {
    for (int e = threadIdx.x; e < kWBM * kWBN; e += blockDim.x) {
      int ii = e / kWBN, jj = e % kWBN;
      int64_t i = it + ii, j = j0 + jj;
      xs[ii][jj] = (i < r1 && j < n) ? ld_as<TC, TS>(src + i * lds + j) : (TC)0;
    }
    for (int e = threadIdx.x; e < kWBM * RP; e += blockDim.x) {
      int ii = e / RP, a = e % RP;
      int64_t i = it + ii;
      us[ii][a] = i < r1 ? U[i * RP + a] : (TC)0;
    }
    __syncthreads();
    TC part[APT];
#pragma unroll
    for (int c = 0; c < APT; ++c) part[c] = 0;
#pragma unroll 4
    for (int ii = 0; ii < kWBM; ++ii) {
      TC x = xs[ii][tj];
#pragma unroll
      for (int c = 0; c < APT; ++c) part[c] += x * us[ii][ta * APT + c];
    }
#pragma unroll
    for (int c = 0; c < APT; ++c) acc[c] += part[c];
    __syncthreads();
  }
  int64_t j = j0 + tj;
  if (j < n) {
    TC* dst = Wpart + (int64_t)blockIdx.y * n * RP + j * RP + ta * APT;
#pragma unroll
    for (int c = 0; c < APT; ++c) dst[c] = acc[c];
  }
}

// ---------------------------------------------------------------- P pass (Algorithm 4)
// Qpart[s][i][:] = sum_{j in split s} M[i][j] V[j][:]: the U-step product M V_i of Algorithm 3
// when it is iterated on a fixed M (Algorithm 4), in the layout of the sweep's Q partials
// (32-row blocks x column splits; thin_gram_kernel sums the splits).
constexpr int kPBN = 32;  // columns per P-pass tile
template <typename TC, typename TMs, int RP>
__global__ void __launch_bounds__(256) ppass_kernel(const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                                    const TC* __restrict__ V, TC* __restrict__ Qpart,
                                                    int cols_per_split, const DevState* st) {
  pdl_enter();
  if (stopped(st)) return;
  constexpr int BM = kSweepBM, QPT = RP / 8;  // 8 warps split the rank
  __shared__ TC Xs[BM][kPBN + 1];
  __shared__ TC Vs[kPBN][RP];
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t jbeg = (int64_t)blockIdx.y * cols_per_split;
  const int64_t jend = min(n, jbeg + cols_per_split);
  const int t = threadIdx.x, qi = t & 31, qg = t >> 5;
  TC q[QPT];
#pragma unroll
  for (int c = 0; c < QPT; ++c) q[c] = 0;
  for (int64_t j0 = jbeg; j0 < jend; j0 += kPBN) {
    __syncthreads();  // previous tile consumed
    for (int e = t; e < BM * kPBN; e += blockDim.x) {
      const int ii = e / kPBN, jj = e % kPBN;
      const int64_t i = i0 + ii, j = j0 + jj;
      Xs[ii][jj] = (i < m && j < jend) ? ld_as<TC, TMs>(M + i * ldm + j) : (TC)0;
    }
    for (int e = t; e < kPBN * RP; e += blockDim.x) {
      const int jj = e / RP, a = e % RP;
      const int64_t j = j0 + jj;
      Vs[jj][a] = j < jend ? V[j * RP + a] : (TC)0;
    }
    __syncthreads();
    TC part[QPT];
#pragma unroll
    for (int c = 0; c < QPT; ++c) part[c] = 0;
#pragma unroll 4
    for (int jj = 0; jj < kPBN; ++jj) {
      const TC xv = Xs[qi][jj];
#pragma unroll
      for (int c = 0; c < QPT; ++c) part[c] += xv * Vs[jj][qg * QPT + c];
    }
#pragma unroll
    for (int c = 0; c < QPT; ++c) q[c] += part[c];
  }
  const int64_t i = i0 + qi;
  if (i < m) {
    TC* dst = Qpart + (int64_t)blockIdx.y * m * RP + i * RP + qg * QPT;
#pragma unroll
    for (int c = 0; c < QPT; ++c) dst[c] = q[c];
  }
}

// ---------------------------------------------------------------- fused sweep (Algorithm 1 S/Y steps)
// One CTA owns kSweepBM rows and a range of columns (one split).  Per column tile:
//   L = U_bar C^T (rebuilt from the factors, never stored),
//   z = M - L + Y_k/mu_k,  Y_{k+1} = clip(mu_k z, -1, 1),  Delta = Y_{k+1}(1/mu_k + 1/mu_{k+1}) - Y_k/mu_k,
//   residual += (Y_{k+1} - Y_k)^2   (= mu_k^2 (M - L - S)^2),
//   Q += (L + Delta) V_bar           (partial of P_{k+1} = X_{k+1} V_{k+1}).
template <typename TC, typename TMs, int RP>
__global__ void __launch_bounds__(256) sweep_kernel(const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                                    const TC* __restrict__ Yin, TC* __restrict__ Yout,
                                                    TC* __restrict__ D, const TC* __restrict__ U,
                                                    const TC* __restrict__ C, const TC* __restrict__ V,
                                                    TC* __restrict__ Qpart, int cols_per_split,
                                                    double* __restrict__ resid_part, const DevState* st) {
  pdl_enter();
  if (stopped(st)) return;
  constexpr int BM = kSweepBM, BN = kSweepBN;
  constexpr int QPT = RP / 8;  // Q accumulators per thread (8 warps split the rank)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* UsT = reinterpret_cast<TC*>(smem_raw);  // [RP][BM]
  TC* CsT = UsT + RP * BM;                    // [RP][BN]
  TC* Vs = CsT + RP * BN;                     // [BN][RP]
  TC* Xs = Vs + BN * RP;                      // [BM][BN + 1]
  __shared__ double red[32];

  const double mu = st->mu;
  const double mu_next = fmin(st->mu_max, st->rho * mu);
  const TC tmu = (TC)mu, inv_mu = (TC)(1.0 / mu), dcoef = (TC)(1.0 / mu + 1.0 / mu_next);

  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t jbeg = (int64_t)blockIdx.y * cols_per_split;
  const int64_t jend = min(n, jbeg + cols_per_split);
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int qi = t & 31, qg = t >> 5;

  for (int e = t; e < RP * BM; e += blockDim.x) {
    int a = e / BM, ii = e % BM;
    int64_t i = i0 + ii;
    UsT[e] = i < m ? U[i * RP + a] : (TC)0;
  }
  TC q[QPT];
#pragma unroll
  for (int c = 0; c < QPT; ++c) q[c] = 0;
  double resid = 0.0;

  for (int64_t j0 = jbeg; j0 < jend; j0 += BN) {
    __syncthreads();  // previous tile's Xs / Vs fully consumed; UsT visible on the first pass
    for (int e = t; e < BN * RP; e += blockDim.x) {
      int jj = e / RP, a = e % RP;
      int64_t j = j0 + jj;
      TC cv = 0, vv = 0;
      if (j < jend) {
        cv = C[j * RP + a];
        vv = V[j * RP + a];
      }
      CsT[a * BN + jj] = cv;
      Vs[e] = vv;
    }
    __syncthreads();
    TC l[2][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int c = 0; c < 4; ++c) l[x][c] = 0;
#pragma unroll 4
    for (int a = 0; a < RP; ++a) {
      TC u0 = UsT[a * BM + ty], u1 = UsT[a * BM + ty + 16];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        TC cv = CsT[a * BN + tx * 4 + c];
        l[0][c] += u0 * cv;
        l[1][c] += u1 * cv;
      }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int ii = ty + 16 * x;
      const int64_t i = i0 + ii;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int jj = tx * 4 + c;
        const int64_t j = j0 + jj;
        TC xv = 0;
        if (i < m && j < jend) {
          const TC mv = ld_as<TC, TMs>(M + i * ldm + j);
          const TC y = Yin[i * n + j];
          const TC z = mv - l[x][c] + y * inv_mu;
          TC yn = tmu * z;
          yn = yn > (TC)1 ? (TC)1 : (yn < (TC)-1 ? (TC)-1 : yn);
          const TC d = yn * dcoef - y * inv_mu;
          const double dy = (double)(yn - y);
          resid += dy * dy;
          Yout[i * n + j] = yn;
          D[i * n + j] = d;
          xv = l[x][c] + d;
        }
        Xs[ii * (BN + 1) + jj] = xv;
      }
    }
    __syncthreads();
    TC part[QPT];
#pragma unroll
    for (int c = 0; c < QPT; ++c) part[c] = 0;
#pragma unroll 4
    for (int jj = 0; jj < BN; ++jj) {
      const TC xv = Xs[qi * (BN + 1) + jj];
#pragma unroll
      for (int c = 0; c < QPT; ++c) part[c] += xv * Vs[jj * RP + qg * QPT + c];
    }
#pragma unroll
    for (int c = 0; c < QPT; ++c) q[c] += part[c];
  }
  const int64_t i = i0 + qi;
  if (i < m) {
    TC* dst = Qpart + (int64_t)blockIdx.y * m * RP + i * RP + qg * QPT;
#pragma unroll
    for (int c = 0; c < QPT; ++c) dst[c] = q[c];
  }
  resid = block_sum(resid, red);
  if (t == 0) resid_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = resid;
}

// ---------------------------------------------------------------- mixed-path SIMT passes (r <= 32)
// Float32 versions of the sweep and the W pass for the mixed path when the tensor-core kernels do
// not apply (r <= 32, or M not bfloat16).  The work per element is small (2 r FMAs in the sweep,
// r in the W pass), so these are built for bandwidth: 128-bit loads and stores along rows, L and
// the thin products register-blocked (2 x 8 and 2 x r/8 per thread) so that shared-memory
// operands are mostly broadcasts, and CTAs that loop over row blocks (the C / V tile stays
// resident when a split is one tile wide, as for tall-skinny M).
constexpr int kMxBM = 64, kMxBN = 64, kMxLDX = kMxBN + 4;

// 4 consecutive elements of row-major storage as float, j0 a multiple of 4 (VEC: one aligned
// vector load; else scalar loads of the valid ones, 0 past `lim` columns).
template <typename T, bool VEC>
__device__ __forceinline__ void ld4(const T* __restrict__ p, int lim, float (&v)[4]) {
  if constexpr (VEC) {
    if constexpr (std::is_same<T, float>::value) {
      const float4 w = *reinterpret_cast<const float4*>(p);
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
      const uint2 w = *reinterpret_cast<const uint2*>(p);
      v[0] = __uint_as_float(w.x << 16); v[1] = __uint_as_float(w.x & 0xFFFF0000u);
      v[2] = __uint_as_float(w.y << 16); v[3] = __uint_as_float(w.y & 0xFFFF0000u);
    } else {
      const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
      v[0] = (float)a.x; v[1] = (float)a.y; v[2] = (float)b.x; v[3] = (float)b.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = c < lim ? ld_as<float, T>(p + c) : 0.f;
  }
}

__device__ __forceinline__ void st4(float* __restrict__ p, int lim, const float (&v)[4], bool vec) {
  if (vec) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < lim) p[c] = v[c];
  }
}

// Sweep (Algorithm 1 S- and Y-steps, next P), float32 arithmetic, float32 Y and Delta (ld n).
// CTA: column split blockIdx.y, 64-row blocks blockIdx.x, blockIdx.x + gridDim.x, ...
// Phase A: thread (tr, tc) = (t / 8, t % 8) forms L for rows 2 tr, 2 tr + 1 and columns
// 8 tc .. 8 tc + 7 of the tile, loads M and Y_k (vector loads issued before the L products),
// writes Y_{k+1}, Delta and X = L + Delta (into shared memory).  Phase B: thread (qr, qa) adds
// X V for rows 2 qr, 2 qr + 1 and ranks qa r/8 .. into registers; the Q partial of a row block is
// stored once.  One residual partial per (column split, row block, warp) (resid_store_warp).
template <typename TMs, int RP, bool VEC>
__device__ __forceinline__ void sweep_mx_body(const VGrid& vg__, const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                                       int64_t ldy, const float* __restrict__ Yin, float* __restrict__ Yout,
                                                       float* __restrict__ D, const float* __restrict__ U,
                                                       const float* __restrict__ C, const float* __restrict__ V,
                                                       float* __restrict__ Qpart, int cols_per_split,
                                                       double* __restrict__ resid_part, const DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  constexpr int BM = kMxBM, BN = kMxBN, QA = RP / 8;
  __shared__ __align__(16) float UsT[RP][BM];
  __shared__ __align__(16) float CsT[RP][BN];
  __shared__ __align__(16) float Vs[BN][RP];
  __shared__ __align__(16) float Xs[BM][kMxLDX];
  const double mu_d = st->mu, mu_next = fmin(st->mu_max, st->rho * mu_d);
  const float mu = (float)mu_d, inv_mu = (float)(1.0 / mu_d), dcoef = (float)(1.0 / mu_d + 1.0 / mu_next);
  const int64_t jbeg = (int64_t)blockIdx.y * cols_per_split;
  const int64_t jend = min(n, jbeg + cols_per_split);
  const bool one_tile = jend - jbeg <= BN;
  const int t = threadIdx.x, tr = t >> 3, tc = t & 7;
  const int64_t nrb = (m + BM - 1) / BM;

  auto load_cv = [&](int64_t j0) {  // C^T and V tiles of columns j0 .. j0 + 63 (0 past jend)
    for (int e = t; e < BN * RP; e += blockDim.x) {
      const int jj = e / RP, a = e % RP;
      const int64_t j = j0 + jj;
      const bool in = j < jend;
      CsT[a][jj] = in ? C[j * RP + a] : 0.f;
      Vs[jj][a] = in ? V[j * RP + a] : 0.f;
    }
  };
  if (one_tile) load_cv(jbeg);

  for (int64_t rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
    const int64_t i0 = rb * BM;
    __syncthreads();  // the previous row block's UsT / Xs readers are done
    for (int e = t; e < BM * RP; e += blockDim.x) {
      const int ii = e / RP, a = e % RP;
      const int64_t i = i0 + ii;
      UsT[a][ii] = i < m ? U[i * RP + a] : 0.f;
    }
    float q[2][QA];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int k = 0; k < QA; ++k) q[x][k] = 0.f;
    float resid = 0.f;
    for (int64_t j0 = jbeg; j0 < jend; j0 += BN) {
      if (!one_tile) {
        __syncthreads();  // previous tile's CsT / Vs / Xs consumed
        load_cv(j0);
      }
      // global loads of this thread's M and Y_k first (independent of the L products)
      float mv[2][8], yv[2][8];
      const int64_t jc = j0 + 8 * tc;
      const int lim = (int)(jend - jc < 8 ? jend - jc : 8);  // valid columns among the 8 (may be <= 0)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int64_t i = i0 + 2 * tr + x;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float a4[4], b4[4];
          if (i < m && lim > 4 * h) {
            ld4<TMs, VEC>(M + i * ldm + jc + 4 * h, lim - 4 * h, a4);
            ld4<float, VEC>(Yin + i * ldy + jc + 4 * h, lim - 4 * h, b4);
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) a4[c] = b4[c] = 0.f;
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            mv[x][4 * h + c] = a4[c];
            yv[x][4 * h + c] = b4[c];
          }
        }
      }
      __syncthreads();  // UsT (first tile) and CsT / Vs visible
      float l[2][8];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int c = 0; c < 8; ++c) l[x][c] = 0.f;
#pragma unroll 8
      for (int a = 0; a < RP; ++a) {
        const float2 u = *reinterpret_cast<const float2*>(&UsT[a][2 * tr]);
        const float4 c0 = *reinterpret_cast<const float4*>(&CsT[a][8 * tc]);
        const float4 c1 = *reinterpret_cast<const float4*>(&CsT[a][8 * tc + 4]);
        const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          l[0][c] = fmaf(u.x, cv[c], l[0][c]);
          l[1][c] = fmaf(u.y, cv[c], l[1][c]);
        }
      }
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int64_t i = i0 + 2 * tr + x;
        const bool row_ok = i < m;
        float yn[8], dd[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const bool ok = row_ok && c < lim;
          const float y = yv[x][c];
          const float z = mv[x][c] - l[x][c] + y * inv_mu;
          const float y1 = fminf(1.f, fmaxf(-1.f, mu * z));
          const float d = y1 * dcoef - y * inv_mu;
          const float dy = y1 - y;
          resid += ok ? dy * dy : 0.f;
          yn[c] = y1;
          dd[c] = d;
          l[x][c] = ok ? l[x][c] + d : 0.f;  // X = L + Delta (0 outside the matrix)
        }
        *reinterpret_cast<float4*>(&Xs[2 * tr + x][8 * tc]) = make_float4(l[x][0], l[x][1], l[x][2], l[x][3]);
        *reinterpret_cast<float4*>(&Xs[2 * tr + x][8 * tc + 4]) = make_float4(l[x][4], l[x][5], l[x][6], l[x][7]);
        if (row_ok)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (lim <= 4 * h) continue;
            const float y4[4] = {yn[4 * h], yn[4 * h + 1], yn[4 * h + 2], yn[4 * h + 3]};
            const float d4[4] = {dd[4 * h], dd[4 * h + 1], dd[4 * h + 2], dd[4 * h + 3]};
            st4(Yout + i * ldy + jc + 4 * h, lim - 4 * h, y4, VEC);
            st4(D + i * ldy + jc + 4 * h, lim - 4 * h, d4, VEC);
          }
      }
      __syncthreads();  // Xs complete
      // phase B: q += X V over the tile's columns
#pragma unroll 4
      for (int jj = 0; jj < BN; ++jj) {
        const float x0 = Xs[2 * tr][jj], x1 = Xs[2 * tr + 1][jj];
        float v[QA];
        if constexpr (QA == 4) {
          const float4 w = *reinterpret_cast<const float4*>(&Vs[jj][4 * tc]);
          v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
        } else if constexpr (QA == 2) {
          const float2 w = *reinterpret_cast<const float2*>(&Vs[jj][2 * tc]);
          v[0] = w.x; v[1] = w.y;
        } else {
          v[0] = Vs[jj][tc];
        }
#pragma unroll
        for (int k = 0; k < QA; ++k) {
          q[0][k] = fmaf(x0, v[k], q[0][k]);
          q[1][k] = fmaf(x1, v[k], q[1][k]);
        }
      }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int64_t i = i0 + 2 * tr + x;
      if (i < m)
#pragma unroll
        for (int k = 0; k < QA; ++k) Qpart[((int64_t)blockIdx.y * m + i) * RP + QA * tc + k] = q[x][k];
    }
    resid_store_warp(resid, resid_part, blockIdx.y, nrb, rb);
  }
}

// cp.async (16-byte, L2 only) global -> shared copy; src_bytes < 16 zero-fills the rest.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// The sweep above with the M and Y_k tiles double-buffered in shared memory by cp.async: the copy
// of the CTA's next (row block, column tile) pair is in flight while the current one is
// computed, so HBM latency is hidden without holding the tiles in registers.  Needs the vector
// conditions (n % 4 == 0, 16-byte aligned rows of M) and float32 or bfloat16 M.
template <typename TMs, int RP>
__device__ __forceinline__ void sweep_mxp_body(const VGrid& vg__, const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                                        int64_t ldy, const float* __restrict__ Yin, float* __restrict__ Yout,
                                                        float* __restrict__ D, const float* __restrict__ U,
                                                        const float* __restrict__ C, const float* __restrict__ V,
                                                        float* __restrict__ Qpart, int cols_per_split,
                                                        double* __restrict__ resid_part, int r, const DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  constexpr int BM = kMxBM, BN = kMxBN, QA = RP / 8, EPC = 16 / (int)sizeof(TMs);  // M elements per 16 B
  constexpr int LDU = RP + 4;  // padded U rows: the four rows a warp reads fall in different banks
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);                     // [2][BM][BN]
  TMs* Ms = reinterpret_cast<TMs*>(Ys + 2 * BM * BN);                 // [2][BM][BN]
  float* Us = reinterpret_cast<float*>(Ms + 2 * BM * BN);             // [2][BM][LDU]: U rows, by row-block parity
  float* CsT = Us + 2 * BM * LDU;                                     // [RP][BN]
  float* Vs = CsT + RP * BN;                                          // [BN][RP]
  float* Xs = Vs + BN * RP;                                           // [BM][kMxLDX]
  const double mu_d = st->mu, mu_next = fmin(st->mu_max, st->rho * mu_d);
  const float mu = (float)mu_d, inv_mu = (float)(1.0 / mu_d), dcoef = (float)(1.0 / mu_d + 1.0 / mu_next);
  const int64_t jbeg = (int64_t)blockIdx.y * cols_per_split;
  const int64_t jend = min(n, jbeg + cols_per_split);
  const int ntile = (int)((jend - jbeg + BN - 1) / BN);
  const int t = threadIdx.x, tr = t >> 3, tc = t & 7;
  const int64_t nrb = (m + BM - 1) / BM;
  const int64_t nmine = blockIdx.x < nrb ? (nrb - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = nmine * ntile;  // this CTA's (row block, tile) pairs, row block major

  auto issue = [&](int64_t k) {  // cp.async of pair k into stage k & 1 (and its U rows on tile 0)
    const int64_t rb = blockIdx.x + (k / ntile) * gridDim.x, i0 = rb * BM;
    const int64_t j0 = jbeg + (k % ntile) * BN;
    float* ys = Ys + (k & 1) * BM * BN;
    TMs* ms = Ms + (k & 1) * BM * BN;
    if (k % ntile == 0) {
      float* us = Us + ((k / ntile) & 1) * BM * LDU;
      for (int e = t; e < BM * (RP / 4); e += blockDim.x) {
        const int ii = e / (RP / 4), cc = e % (RP / 4);
        const int64_t i = i0 + ii;
        cp_async16(us + ii * LDU + 4 * cc, i < m ? (const void*)(U + i * RP + 4 * cc) : (const void*)U, i < m ? 16 : 0);
      }
    }
    for (int e = t; e < BM * (BN / 4); e += blockDim.x) {  // Y: 16-byte chunks of 4 floats
      const int ii = e / (BN / 4), cc = e % (BN / 4);
      const int64_t i = i0 + ii, j = j0 + 4 * cc;
      const bool ok = i < m && j < jend;
      cp_async16(ys + ii * BN + 4 * cc, ok ? (const void*)(Yin + i * ldy + j) : (const void*)Yin, ok ? 16 : 0);
    }
    for (int e = t; e < BM * (BN / EPC); e += blockDim.x) {  // M: 16-byte chunks
      const int ii = e / (BN / EPC), cc = e % (BN / EPC);
      const int64_t i = i0 + ii, j = j0 + EPC * cc;
      const int64_t left = i < m ? jend - j : 0;
      const int bytes = left <= 0 ? 0 : (left >= EPC ? 16 : (int)left * (int)sizeof(TMs));
      cp_async16(ms + ii * BN + EPC * cc, bytes ? (const void*)(M + i * ldm + j) : (const void*)M, bytes);
    }
    cp_async_commit();
  };
  auto load_cv = [&](int64_t j0) {
    for (int e = t; e < BN * RP; e += blockDim.x) {
      const int jj = e / RP, a = e % RP;
      const int64_t j = j0 + jj;
      const bool in = j < jend;
      CsT[a * BN + jj] = in ? C[j * RP + a] : 0.f;
      Vs[jj * RP + a] = in ? V[j * RP + a] : 0.f;
    }
  };

  if (total > 0) issue(0);
  if (ntile == 1) load_cv(jbeg);
  float q[2][QA];
  float resid = 0.f;
  for (int64_t k = 0; k < total; ++k) {
    const int64_t rb = blockIdx.x + (k / ntile) * gridDim.x, i0 = rb * BM;
    const int tile = (int)(k % ntile);
    const int64_t j0 = jbeg + (int64_t)tile * BN;
    if (k + 1 < total) issue(k + 1); else cp_async_commit();  // keep one group per iteration
    cp_async_wait1();  // pair k has landed (this thread's copies)
    __syncthreads();   // everyone's copies visible; the previous pair's Xs / Vs readers are done
    if (tile == 0) {
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int c = 0; c < QA; ++c) q[x][c] = 0.f;
      resid = 0.f;
    }
    if (ntile > 1) {
      load_cv(j0);
      __syncthreads();
    }
    const float* us = Us + ((k / ntile) & 1) * BM * LDU;
    // phase A: L for rows 2 tr, 2 tr + 1 and columns 8 tc .. 8 tc + 7 (ranks a < r)
    float l[2][8];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int c = 0; c < 8; ++c) l[x][c] = 0.f;
#pragma unroll 4
    for (int a = 0; a < r; ++a) {
      const float2 u = make_float2(us[(2 * tr) * LDU + a], us[(2 * tr + 1) * LDU + a]);
      const float4 c0 = *reinterpret_cast<const float4*>(&CsT[a * BN + 8 * tc]);
      const float4 c1 = *reinterpret_cast<const float4*>(&CsT[a * BN + 8 * tc + 4]);
      const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        l[0][c] = fmaf(u.x, cv[c], l[0][c]);
        l[1][c] = fmaf(u.y, cv[c], l[1][c]);
      }
    }
    const float* ys = Ys + (k & 1) * BM * BN;
    const TMs* ms = Ms + (k & 1) * BM * BN;
    const int64_t jc = j0 + 8 * tc;
    const int lim = (int)(jend - jc < 8 ? jend - jc : 8);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int rr = 2 * tr + x;
      const int64_t i = i0 + rr;
      float mv[8], yv[8];
      {
        const float4 a0 = *reinterpret_cast<const float4*>(ys + rr * BN + 8 * tc);
        const float4 a1 = *reinterpret_cast<const float4*>(ys + rr * BN + 8 * tc + 4);
        yv[0] = a0.x; yv[1] = a0.y; yv[2] = a0.z; yv[3] = a0.w; yv[4] = a1.x; yv[5] = a1.y; yv[6] = a1.z; yv[7] = a1.w;
      }
      if constexpr (std::is_same<TMs, float>::value) {
        const float4 a0 = *reinterpret_cast<const float4*>(ms + rr * BN + 8 * tc);
        const float4 a1 = *reinterpret_cast<const float4*>(ms + rr * BN + 8 * tc + 4);
        mv[0] = a0.x; mv[1] = a0.y; mv[2] = a0.z; mv[3] = a0.w; mv[4] = a1.x; mv[5] = a1.y; mv[6] = a1.z; mv[7] = a1.w;
      } else {
        const uint4 w = *reinterpret_cast<const uint4*>(ms + rr * BN + 8 * tc);
        const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          mv[2 * c] = __uint_as_float(wv[c] << 16);
          mv[2 * c + 1] = __uint_as_float(wv[c] & 0xFFFF0000u);
        }
      }
      const bool row_ok = i < m;
      float yn[8], dd[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const bool ok = row_ok && c < lim;
        const float y = yv[c];
        const float z = mv[c] - l[x][c] + y * inv_mu;
        const float y1 = fminf(1.f, fmaxf(-1.f, mu * z));
        const float d = y1 * dcoef - y * inv_mu;
        const float dy = y1 - y;
        resid += ok ? dy * dy : 0.f;
        yn[c] = y1;
        dd[c] = d;
        l[x][c] = ok ? l[x][c] + d : 0.f;  // X = L + Delta (0 outside the matrix)
      }
      *reinterpret_cast<float4*>(&Xs[rr * kMxLDX + 8 * tc]) = make_float4(l[x][0], l[x][1], l[x][2], l[x][3]);
      *reinterpret_cast<float4*>(&Xs[rr * kMxLDX + 8 * tc + 4]) = make_float4(l[x][4], l[x][5], l[x][6], l[x][7]);
      if (row_ok)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (lim <= 4 * h) continue;
          *reinterpret_cast<float4*>(Yout + i * ldy + jc + 4 * h) =
              make_float4(yn[4 * h], yn[4 * h + 1], yn[4 * h + 2], yn[4 * h + 3]);
          *reinterpret_cast<float4*>(D + i * ldy + jc + 4 * h) =
              make_float4(dd[4 * h], dd[4 * h + 1], dd[4 * h + 2], dd[4 * h + 3]);
        }
    }
    __syncthreads();  // Xs complete
    const int jn = (int)(jend - j0 < BN ? jend - j0 : BN);  // valid columns of the tile
#pragma unroll 4
    for (int jj = 0; jj < jn; ++jj) {
      const float x0 = Xs[(2 * tr) * kMxLDX + jj], x1 = Xs[(2 * tr + 1) * kMxLDX + jj];
      float v[QA];
      if constexpr (QA == 4) {
        const float4 w = *reinterpret_cast<const float4*>(&Vs[jj * RP + 4 * tc]);
        v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
      } else if constexpr (QA == 2) {
        const float2 w = *reinterpret_cast<const float2*>(&Vs[jj * RP + 2 * tc]);
        v[0] = w.x; v[1] = w.y;
      } else {
        v[0] = Vs[jj * RP + tc];
      }
#pragma unroll
      for (int c = 0; c < QA; ++c) {
        q[0][c] = fmaf(x0, v[c], q[0][c]);
        q[1][c] = fmaf(x1, v[c], q[1][c]);
      }
    }
    if (tile == ntile - 1) {  // row block done: its Q partial and residual
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int64_t i = i0 + 2 * tr + x;
        if (i < m)
#pragma unroll
          for (int c = 0; c < QA; ++c) Qpart[((int64_t)blockIdx.y * m + i) * RP + QA * tc + c] = q[x][c];
      }
      resid_store_warp(resid, resid_part, blockIdx.y, nrb, rb);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename TMs, int RP>
constexpr size_t mxp_smem() {
  return (size_t)2 * kMxBM * kMxBN * (4 + sizeof(TMs)) + (size_t)2 * kMxBM * (RP + 4) * 4 +
         (size_t)RP * 2 * kMxBN * 4 + (size_t)kMxBM * kMxLDX * 4;
}

// W pass, float32: Wpart[c][j][:] = sum over the rows i of chunk c of src[i][j] U[i][:].  CTA:
// 64 columns x a chunk of rows, in 32-row tiles (src and U tiles staged in shared memory with
// vector loads); thread (wc, wa) = (t / 8, t % 8) accumulates columns 2 wc, 2 wc + 1 and ranks
// wa r/8 .. in registers.
template <typename TS, int RP, bool VEC>
__device__ __forceinline__ void wpass_mx_body(const VGrid& vg__, const TS* __restrict__ src, int64_t lds, int64_t m, int64_t n,
                                                       int rows_per_chunk, const float* __restrict__ U,
                                                       float* __restrict__ Wpart, const DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  constexpr int BR = 32, BN = kMxBN, QA = RP / 8;
  __shared__ __align__(16) float Xs[BR][kMxLDX];
  __shared__ __align__(16) float Us[BR][RP];
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(m, r0 + rows_per_chunk);
  const int t = threadIdx.x, wc = t >> 3, wa = t & 7;
  const int lr = t >> 4, lq = t & 15;  // tile loads: rows lr and lr + 16, columns 4 lq .. 4 lq + 3
  const int lim = (int)(n - (j0 + 4 * lq) < 4 ? n - (j0 + 4 * lq) : 4);
  float acc[2][QA];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int k = 0; k < QA; ++k) acc[x][k] = 0.f;
  for (int64_t it = r0; it < r1; it += BR) {
    float v[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = it + lr + 16 * h;
      if (i < r1 && lim > 0) {
        ld4<TS, VEC>(src + i * lds + j0 + 4 * lq, lim, v[h]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[h][c] = 0.f;
      }
    }
    float uv[(BR * RP + 255) / 256];
#pragma unroll
    for (int q2 = 0; q2 < (BR * RP + 255) / 256; ++q2) {
      const int e = t + 256 * q2, ii = e / RP, a = e % RP;
      const int64_t i = it + ii;
      uv[q2] = (e < BR * RP && i < r1) ? U[i * RP + a] : 0.f;
    }
    __syncthreads();  // previous tile consumed
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<float4*>(&Xs[lr + 16 * h][4 * lq]) = make_float4(v[h][0], v[h][1], v[h][2], v[h][3]);
#pragma unroll
    for (int q2 = 0; q2 < (BR * RP + 255) / 256; ++q2) {
      const int e = t + 256 * q2;
      if (e < BR * RP) Us[e / RP][e % RP] = uv[q2];
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < BR; ++ii) {
      const float2 x = *reinterpret_cast<const float2*>(&Xs[ii][2 * wc]);
      float u[QA];
      if constexpr (QA == 4) {
        const float4 w = *reinterpret_cast<const float4*>(&Us[ii][4 * wa]);
        u[0] = w.x; u[1] = w.y; u[2] = w.z; u[3] = w.w;
      } else if constexpr (QA == 2) {
        const float2 w = *reinterpret_cast<const float2*>(&Us[ii][2 * wa]);
        u[0] = w.x; u[1] = w.y;
      } else {
        u[0] = Us[ii][wa];
      }
#pragma unroll
      for (int k = 0; k < QA; ++k) {
        acc[0][k] = fmaf(x.x, u[k], acc[0][k]);
        acc[1][k] = fmaf(x.y, u[k], acc[1][k]);
      }
    }
  }
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const int64_t j = j0 + 2 * wc + x;
    if (j < n)
#pragma unroll
      for (int k = 0; k < QA; ++k) Wpart[((int64_t)blockIdx.y * n + j) * RP + QA * wa + k] = acc[x][k];
  }
}

// The W pass above with cp.async staging: 32-row tiles of src and U in a 4-stage ring, three
// tiles in flight while one is accumulated.  Needs the vector conditions (src rows 16-byte
// aligned, n % 4 == 0) and float32 or bfloat16 src.
constexpr int kWxStages = 4;
template <typename TS, int RP>
__device__ __forceinline__ void wpass_mxp_body(const VGrid& vg__, const TS* __restrict__ src, int64_t lds, int64_t m, int64_t n,
                                                        int rows_per_chunk, const float* __restrict__ U,
                                                        float* __restrict__ Wpart, const DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  if (stopped(st)) return;
  constexpr int BR = 32, BN = kMxBN, QA = RP / 8, EPC = 16 / (int)sizeof(TS);
  constexpr int XS = BR * BN, US = BR * RP;  // elements per stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TS* Xs = reinterpret_cast<TS*>(smem_raw);                                  // [stages][BR][BN]
  float* Us = reinterpret_cast<float*>(Xs + kWxStages * XS);                 // [stages][BR][RP]
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(m, r0 + rows_per_chunk);
  const int ntile = r1 > r0 ? (int)((r1 - r0 + BR - 1) / BR) : 0;
  const int t = threadIdx.x, wc = t >> 3, wa = t & 7;
  auto issue = [&](int k) {
    const int64_t it = r0 + (int64_t)k * BR;
    TS* xs = Xs + (k % kWxStages) * XS;
    float* us = Us + (k % kWxStages) * US;
    for (int e = t; e < BR * (BN / EPC); e += blockDim.x) {
      const int ii = e / (BN / EPC), cc = e % (BN / EPC);
      const int64_t i = it + ii, j = j0 + EPC * cc;
      const int64_t left = i < r1 ? n - j : 0;
      const int bytes = left <= 0 ? 0 : (left >= EPC ? 16 : (int)left * (int)sizeof(TS));
      cp_async16(xs + ii * BN + EPC * cc, bytes ? (const void*)(src + i * lds + j) : (const void*)src, bytes);
    }
    for (int e = t; e < BR * (RP / 4); e += blockDim.x) {
      const int ii = e / (RP / 4), cc = e % (RP / 4);
      const int64_t i = it + ii;
      cp_async16(us + ii * RP + 4 * cc, i < r1 ? (const void*)(U + i * RP + 4 * cc) : (const void*)U, i < r1 ? 16 : 0);
    }
    cp_async_commit();
  };
  float acc[2][QA];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int c = 0; c < QA; ++c) acc[x][c] = 0.f;
  for (int k = 0; k < kWxStages - 1; ++k) {
    if (k < ntile) issue(k); else cp_async_commit();
  }
  for (int k = 0; k < ntile; ++k) {
    if (k + kWxStages - 1 < ntile) issue(k + kWxStages - 1); else cp_async_commit();
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kWxStages - 1) : "memory");
    __syncthreads();
    const TS* xs = Xs + (k % kWxStages) * XS;
    const float* us = Us + (k % kWxStages) * US;
#pragma unroll 4
    for (int ii = 0; ii < BR; ++ii) {
      float x0, x1;
      if constexpr (std::is_same<TS, float>::value) {
        const float2 w = *reinterpret_cast<const float2*>(xs + ii * BN + 2 * wc);
        x0 = w.x; x1 = w.y;
      } else {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(xs + ii * BN + 2 * wc);
        x0 = __uint_as_float(w << 16); x1 = __uint_as_float(w & 0xFFFF0000u);
      }
      float u[QA];
      if constexpr (QA == 4) {
        const float4 w = *reinterpret_cast<const float4*>(us + ii * RP + 4 * wa);
        u[0] = w.x; u[1] = w.y; u[2] = w.z; u[3] = w.w;
      } else if constexpr (QA == 2) {
        const float2 w = *reinterpret_cast<const float2*>(us + ii * RP + 2 * wa);
        u[0] = w.x; u[1] = w.y;
      } else {
        u[0] = us[ii * RP + wa];
      }
#pragma unroll
      for (int c = 0; c < QA; ++c) {
        acc[0][c] = fmaf(x0, u[c], acc[0][c]);
        acc[1][c] = fmaf(x1, u[c], acc[1][c]);
      }
    }
    __syncthreads();  // stage k % stages is refilled by the next iteration's issue
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const int64_t j = j0 + 2 * wc + x;
    if (j < n)
#pragma unroll
      for (int c = 0; c < QA; ++c) Wpart[((int64_t)blockIdx.y * n + j) * RP + QA * wa + c] = acc[x][c];
  }
}

template <typename TS, int RP>
constexpr size_t wxp_smem() { return (size_t)kWxStages * 32 * (kMxBN * sizeof(TS) + RP * 4); }

// ---------------------------------------------------------------- end of iteration (one CTA)
// ||M - L - S||_F = ||Y_{k+1} - Y_k||_F / mu_k; continuation mu_{k+1} = min(mu_bar, rho mu_k).
__device__ __forceinline__ void iter_end_body(const VGrid& vg__, const double* __restrict__ resid_part, int count, DevState* st) {
  pdl_enter();
  SFR_VGRID(vg__);
  __shared__ double red[32];
  if (stopped(st)) return;
  double v = 0.0;
#pragma unroll 8
  for (int c = threadIdx.x; c < count; c += blockDim.x) v += resid_part[c];
  // warp sums, then thread 0 adds them in warp order (the float64 pipe is narrow on this part:
  // the other threads do not repeat that sum)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    v = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) v += red[w];
    const double mu = st->mu;
    const double res = sqrt(v) / mu / st->norm_m;
    st->res = res;
    st->mu_last = mu;
    st->mu = fmin(st->mu_max, st->rho * mu);
    st->iter += 1;
    if (!(res == res) || res > 1e300) {
      st->status = SFR_E_NAN;
      st->done = 1;
    } else if (st->fixed) {
      if (st->iter >= st->max_iter) st->done = 1;
    } else if (res <= st->tol) {
      st->done = 1;
    } else if (st->iter >= st->max_iter) {
      st->status = SFR_E_NOCONV;
      st->done = 1;
    }
  }
}

__global__ void norm_finish_kernel(const double* __restrict__ part, int count, DevState* st) {
  pdl_enter();
  __shared__ double red[32];
  double v = 0.0;
  for (int c = threadIdx.x; c < count; c += blockDim.x) v += part[c];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    st->norm_m = sqrt(v);
    if (!(v > 0.0) || !(v < 1e300)) {
      st->status = (v == 0.0) ? SFR_E_INVAL : SFR_E_NAN;
      st->done = 1;
    }
  }
}

// ---------------------------------------------------------------- end of an Algorithm 4 iteration
// Stopping rule of FixedRankOptFull ("while not converged", Algorithm 4): the relative change
// of B, ||B_i - B_{i-1}||_F / ||B_i||_F, over the leading r x r block; then B_prev = B_i.
__global__ void full_end_kernel(const double* __restrict__ B, double* __restrict__ Bprev, int rp, int r,
                                DevState* st) {
  pdl_enter();
  __shared__ double red[32];
  if (stopped(st)) return;
  double d2 = 0.0, b2 = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, c = e % r;
    const double bv = B[a * rp + c], dv = bv - Bprev[a * rp + c];
    d2 += dv * dv;
    b2 += bv * bv;
  }
  d2 = block_sum(d2, red);
  b2 = block_sum(b2, red);
  for (int e = threadIdx.x; e < rp * rp; e += blockDim.x) Bprev[e] = B[e];
  if (threadIdx.x == 0) {
    const double res = sqrt(d2 / b2);
    st->res = res;
    st->iter += 1;
    if (!(res == res) || !(b2 < 1e300)) {
      st->status = SFR_E_NAN;
      st->done = 1;
    } else if (st->fixed) {
      if (st->iter >= st->max_iter) st->done = 1;
    } else if (res <= st->tol) {
      st->done = 1;
    } else if (st->iter >= st->max_iter) {
      st->status = SFR_E_NOCONV;
      st->done = 1;
    }
  }
}

// ---------------------------------------------------------------- outputs
// S = P_ST_{1/mu}(M - L + Y_prev / mu) with the mu, Y_prev and factors of the last iteration
// (Algorithm 1 returns L_k, S_k); optionally L itself.
template <typename TC, typename TMs, typename TSo, typename TY, int RP>
__global__ void __launch_bounds__(256) finalize_kernel(const TMs* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                                       const TY* __restrict__ Yprev, int64_t ldy, const TC* __restrict__ U,
                                                       const TC* __restrict__ C, TSo* __restrict__ S, TSo* __restrict__ L,
                                                       int64_t lds, const DevState* st) {
  pdl_enter();
  __shared__ TC us[8][RP];
  __shared__ TC cs[32][RP + 1];
  // 1-D grid over (8-row, 32-column) blocks, columns fastest (a 2-D grid would cap m at 65535 x 8)
  const int64_t nbx = (n + 31) / 32;
  const int64_t i0 = ((int64_t)blockIdx.x / nbx) * 8, j0 = ((int64_t)blockIdx.x % nbx) * 32;
  const int tj = threadIdx.x & 31, ti = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < 8 * RP; e += blockDim.x) {
    int ii = e / RP, a = e % RP;
    us[ii][a] = i0 + ii < m ? U[(i0 + ii) * RP + a] : (TC)0;
  }
  for (int e = threadIdx.x; e < 32 * RP; e += blockDim.x) {
    int jj = e / RP, a = e % RP;
    cs[jj][a] = j0 + jj < n ? C[(j0 + jj) * RP + a] : (TC)0;
  }
  __syncthreads();
  const int64_t i = i0 + ti, j = j0 + tj;
  if (i >= m || j >= n) return;
  TC l = 0;
#pragma unroll 8
  for (int a = 0; a < RP; ++a) l += us[ti][a] * cs[tj][a];
  const double mu = st->mu_last;
  const TC inv_mu = (TC)(1.0 / mu);
  const TC z = ld_as<TC, TMs>(M + i * ldm + j) - l + ld_as<TC, TY>(Yprev + i * ldy + j) * inv_mu;
  const TC sv = z > inv_mu ? z - inv_mu : (z < -inv_mu ? z + inv_mu : (TC)0);
  if (S) S[i * lds + j] = (TSo)sv;
  if (L) L[i * lds + j] = (TSo)l;
}

template <typename TC, int RP>
__global__ void export_kernel(const TC* __restrict__ src, int64_t rows, int r, double* __restrict__ dst) {
  pdl_enter();
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * r) return;
  int64_t i = idx / r;
  int a = (int)(idx % r);
  dst[idx] = (double)src[i * RP + a];
}

// dst (rows x RP, TC) = src (rows x r, float64), padding columns r .. RP-1 with zeros.
template <typename TC, int RP>
__global__ void import_kernel(const double* __restrict__ src, int64_t rows, int r, TC* __restrict__ dst) {
  pdl_enter();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * RP) return;
  const int64_t i = idx / RP;
  const int a = (int)(idx % RP);
  dst[idx] = a < r ? (TC)src[i * r + a] : (TC)0;
}

// ---------------------------------------------------------------- dispatch helpers
template <typename F>
cudaError_t by_rank(int rp, F&& f) {
  switch (rp) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    default: return cudaErrorInvalidValue;
  }
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

template <typename F>
cudaError_t by_prec(bool fp64, F&& f) {
  if (fp64) return f(double{});
  return f(float{});
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

template <typename TC, int RP>
size_t gram_smem() { return sizeof(TC) * std::max<size_t>((size_t)(2 * kGramRows + 2 * RP) * (RP + 4), 16 * kThinThreads); }
template <typename TC, int RP>
size_t transform_smem() {
  // the Gram scratch (256 x 16) starts at the source-row tile, 2 RP (RP + 4) elements in
  return sizeof(TC) * std::max<size_t>((size_t)(2 * RP + 3 * kGramRows) * (RP + 4),
                                       (size_t)2 * RP * (RP + 4) + 16 * kThinThreads);
}

template <typename K>
cudaError_t allow_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Mixed path, r <= 32: the float32 passes above.  Vector loads need n % 4 == 0 and M rows on
// 16-byte boundaries; otherwise the same kernels load element by element.
static bool mx_vec(const Shape& s, const Buffers& b) {
  const size_t es = b.m_dtype == SFR_F64 ? 8 : b.m_dtype == SFR_F32 ? 4 : 2;
  return b.ldy % 4 == 0 && ((size_t)s.ldm * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(b.M) % 16) == 0;
}

// Aligned copy of M: dst[i][j] = src[i][j] for j < n, 0 for n <= j < ldd (one thread per
// destination element, elements moved as raw bits).
template <typename T>
__global__ void copy_m_kernel(const T* __restrict__ src, int64_t ldm, int64_t m, int64_t n, T* __restrict__ dst,
                              int64_t ldd) {
  pdl_enter();
  const int64_t total = m * ldd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ldd, j = e % ldd;
    dst[e] = j < n ? src[i * ldm + j] : T(0);
  }
}

cudaError_t launch_copy_m(const Shape& s, const void* M, int64_t ldm, void* Mc, cudaStream_t st) {
  const int64_t total = s.m * s.mc_ld;
  const int blocks = (int)std::min<int64_t>(cdiv(total, 256), 8LL * s.num_sms);
  if (total == 0) return cudaSuccess;
  if (s.mc_es == 8)
    launch_pdl(copy_m_kernel<uint64_t>, blocks, 256, 0, st, static_cast<const uint64_t*>(M), ldm, s.m, s.n,
               static_cast<uint64_t*>(Mc), s.mc_ld);
  else if (s.mc_es == 4)
    launch_pdl(copy_m_kernel<uint32_t>, blocks, 256, 0, st, static_cast<const uint32_t*>(M), ldm, s.m, s.n,
               static_cast<uint32_t*>(Mc), s.mc_ld);
  else
    launch_pdl(copy_m_kernel<uint16_t>, blocks, 256, 0, st, static_cast<const uint16_t*>(M), ldm, s.m, s.n,
               static_cast<uint16_t*>(Mc), s.mc_ld);
  return cudaGetLastError();
}

// threads of the partial-sum kernel: 8 warps, 32 when there are many partials to walk
inline int reduce_threads(int64_t count) { return count >= 256 ? 1024 : 256; }

cudaError_t launch_reduce_parts(const double* parts, int count, int rpsq, double* out, const DevState* dst,
                                cudaStream_t st) {
  launch_k<&reduce_sq_body<double>, 1024>(cdiv(rpsq, 32), reduce_threads(count), 0, st, parts, (int64_t)count,
                                           (int64_t)rpsq, out, dst);
  return cudaGetLastError();
}

cudaError_t launch_norm_m(const Shape& s, const Buffers& b, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(s.m, 1024);
  cudaError_t e = by_mtype(b.m_dtype, b.M, [&](auto M) {
    using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
    launch_pdl(norm_m_kernel<TMs>, blocks, 256, 0, st, M, s.m, s.n, s.ldm, b.normm_part);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  launch_pdl(norm_finish_kernel, 1, 256, 0, st, b.normm_part, blocks, b.st);
  return cudaGetLastError();
}

cudaError_t launch_init_p(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st) {
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_mtype(b.m_dtype, b.M, [&](auto M) {
      using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
      launch_pdl(init_p_kernel<TC, TMs>, cdiv(s.m * s.rp, 256), 256, 0, st, M, s.m, s.ldm, s.r, s.rp, static_cast<TC*>(b.P));
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_gram_p(const Shape& s, const Buffers& b, bool fp64, bool sum_parts, cudaStream_t st,
                          const void* addA, const double* H, bool pt) {
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const size_t sm = gram_smem<TC, RP>();
      launch_k<&thin_gram_body<TC, RP>, 256>(s.gp_blocks, 256, sm, st,
          static_cast<const TC*>(b.Qpart), sum_parts ? s.nsplit : 0, s.m * RP, static_cast<TC*>(b.P), s.m,
          static_cast<const TC*>(addA), H, b.GPpart, b.st, s.q_ctas, (s.n + 63) / 64, (const double*)nullptr,
          pt ? static_cast<__nv_bfloat16*>(b.t.Ut) : nullptr, (int64_t)b.t.ldd);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_apply_u(const Shape& s, const Buffers& b, bool fp64, bool first, cudaStream_t st) {
  // U_new = P T_U into the other U buffer; H partials U_old^T U_new (iteration >= 2).
  const int u_old = b.u_cur, u_new = 1 - b.u_cur;
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const size_t sm = transform_smem<TC, RP>();
      // tensor-core path: also the TF32 split of U_new (the sweep's operand) and, for the first
      // W pass, its bfloat16 transpose (later W passes take P^T from the P / Gram kernel)
      // (Algorithm 4: the two-term bfloat16 split of U^T instead, the B operand of M^T U)
      const bool tcx = b.tc && RP == 64 && !fp64, tf = tcx && !b.full;
      launch_k<&row_transform_body<TC, RP>, 256>(s.gp_blocks, 256, sm, st,
          static_cast<const TC*>(b.P), s.m, b.TU, static_cast<TC*>(b.U[u_new]), nullptr, nullptr,
          first ? nullptr : static_cast<const TC*>(b.U[u_old]), first ? nullptr : b.Hpart, b.st,
          tf ? b.t.Uh : nullptr, tf ? b.t.Ul : nullptr,
          (tcx && (first || b.full)) ? static_cast<__nv_bfloat16*>(b.t.Ut) : nullptr, (int64_t)b.t.ldd,
          b.full ? 1 : 0);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_wpass(const Shape& s, const Buffers& b, bool fp64, bool first, int u_new, cudaStream_t st,
                         bool wp) {
  dim3 grid(s.wpass_grid_x, s.nchunk);
  if (mx_path(s, fp64)) {
    const bool vec = first ? mx_vec(s, b) : b.ldy % 4 == 0;
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      if constexpr (RP > 32) {
        return cudaErrorInvalidValue;
      } else {
        // wp (after the first iteration): Delta^T P, the operand that does not wait for T_U
        const float* U = static_cast<const float*>(wp && !first ? b.P : b.U[u_new]);
        float* Wp = static_cast<float*>(b.Wpart);
        auto go = [&](auto tag, auto src, int64_t lds) {
          return launch_k<decltype(tag)::value, 256>(grid, 256, 0, st, src, lds, s.m, s.n, s.rows_per_chunk, U, Wp,
                                                      b.st);
        };
        auto pipelined = [&](auto srcp, int64_t lds) {
          using TS = std::remove_const_t<std::remove_pointer_t<decltype(srcp)>>;
          constexpr size_t sm = wxp_smem<TS, RP>();
          return launch_k<&wpass_mxp_body<TS, RP>, 256>(grid, 256, sm, st, srcp, lds, s.m, s.n, s.rows_per_chunk, U,
                                                         Wp, b.st);
        };
        if (first)
          return by_mtype(b.m_dtype, b.M, [&](auto M) {
            using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
            if constexpr (!std::is_same<TMs, double>::value) {
              if (vec) return pipelined(M, s.ldm);
            }
            return vec ? go(BodyTag<&wpass_mx_body<TMs, RP, true>>{}, M, s.ldm)
                       : go(BodyTag<&wpass_mx_body<TMs, RP, false>>{}, M, s.ldm);
          });
        const float* Dp = static_cast<const float*>(b.D);
        return vec ? pipelined(Dp, b.ldy) : go(BodyTag<&wpass_mx_body<float, RP, false>>{}, Dp, b.ldy);
      }
    });
  }
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const TC* U = static_cast<const TC*>(b.U[u_new]);
      TC* Wp = static_cast<TC*>(b.Wpart);
      if (first) {
        return by_mtype(b.m_dtype, b.M, [&](auto M) {
          using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
          launch_pdl(wpass_kernel<TC, TMs, RP>, grid, 256, 0, st, M, s.ldm, s.m, s.n, s.rows_per_chunk, U, Wp, b.st);
          return cudaGetLastError();
        });
      }
      launch_pdl(wpass_kernel<TC, TC, RP>, grid, 256, 0, st, static_cast<const TC*>(b.D), s.n, s.m, s.n, s.rows_per_chunk, U, Wp,
                                                     b.st);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_wfinal(const Shape& s, const Buffers& b, bool fp64, bool first, cudaStream_t st, bool wp) {
  // W = sum_c Wpart[c] (+ C_old H, H = U_old^T U_new), then Gram partials of W.  wp: the partials
  // hold Delta^T P instead of Delta^T U_new, and W = (sum_c Wpart[c]) T_U + C_old H.
  // H = sum of the U_old^T U_new partials, reduced into the slot after the partials.
  if (!first) {
    launch_k<&reduce_sq_body<double>, 1024>(cdiv(s.rp * s.rp, 32), reduce_threads(s.gp_blocks), 0, st,
        b.Hpart, s.gp_blocks, s.rp * s.rp, b.Hpart + (size_t)s.gp_blocks * s.rp * s.rp, b.st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const double* H = b.Hpart + (size_t)s.gp_blocks * s.rp * s.rp;
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const size_t sm = gram_smem<TC, RP>();
      cudaError_t e;
      // many row chunks over few columns (tall M): sum the chunks' partials into the first one
      // with a wide reduction first, so the thin kernel does not add hundreds of them per element
      int nparts = s.nchunk;
      if (nparts >= 32) {
        const int64_t len = s.n * RP;
        launch_k<&reduce_sq_body<TC>, 1024>(cdiv(len, 32), reduce_threads(nparts), 0, st,
                                            static_cast<const TC*>(b.Wpart), (int64_t)nparts, len,
                                            static_cast<TC*>(b.Wpart), b.st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        nparts = 1;
      }
      launch_k<&thin_gram_body<TC, RP>, 256>(s.gw_blocks, 256, sm, st,
          static_cast<const TC*>(b.Wpart), nparts, s.n * RP, static_cast<TC*>(b.W), s.n,
          first ? nullptr : static_cast<const TC*>(b.C), first ? nullptr : H, b.GWpart, b.st, 0, (int64_t)0,
          wp ? (const double*)b.TU : (const double*)nullptr, (__nv_bfloat16*)nullptr, (int64_t)0);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_apply_v(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st) {
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const size_t sm = transform_smem<TC, RP>();
      // tensor-core path: also the TF32 split of C and the bfloat16 transpose of V
      // (Algorithm 4: the two-term bfloat16 split of V^T instead, the B operand of M V)
      const bool tcx = b.tc && RP == 64 && !fp64, tf = tcx && !b.full;
      launch_k<&row_transform_body<TC, RP>, 256>(s.gw_blocks, 256, sm, st,
          static_cast<const TC*>(b.W), s.n, b.TV, static_cast<TC*>(b.V), b.TCm, static_cast<TC*>(b.C), nullptr, nullptr,
          b.st, tf ? b.t.Ch : nullptr, tf ? b.t.Cl : nullptr, tcx ? static_cast<__nv_bfloat16*>(b.t.Vt) : nullptr,
          (int64_t)b.t.ldy, b.full ? 1 : 0);
      return cudaGetLastError();
    });
  });
}

static cudaError_t launch_sweep_mx(const Shape& s, const Buffers& b, int u_cur, cudaStream_t st) {
  dim3 grid(s.mx_grid_x, s.nsplit);
  const bool vec = mx_vec(s, b);
  return by_rank(s.rp, [&](auto rpc) {
    constexpr int RP = decltype(rpc)::value;
    if constexpr (RP > 32) {
      return cudaErrorInvalidValue;
    } else {
      return by_mtype(b.m_dtype, b.M, [&](auto M) {
        using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
        auto go = [&](auto tag) {
          return launch_k<decltype(tag)::value, 256>(grid, 256, 0, st, M, s.m, s.n, s.ldm, b.ldy,
                                                      static_cast<const float*>(b.Y[0]), static_cast<float*>(b.Y[1]),
                                                      static_cast<float*>(b.D), static_cast<const float*>(b.U[u_cur]),
                                                      static_cast<const float*>(b.C), static_cast<const float*>(b.V),
                                                      static_cast<float*>(b.Qpart), s.cols_per_split, b.resid_part,
                                                      b.st);
        };
        if constexpr (!std::is_same<TMs, double>::value) {
          if (vec) {
            constexpr size_t sm = mxp_smem<TMs, RP>();
            return launch_k<&sweep_mxp_body<TMs, RP>, 256>(
                grid, 256, sm, st, M, s.m, s.n, s.ldm, b.ldy, static_cast<const float*>(b.Y[0]), static_cast<float*>(b.Y[1]),
                static_cast<float*>(b.D), static_cast<const float*>(b.U[u_cur]), static_cast<const float*>(b.C),
                static_cast<const float*>(b.V), static_cast<float*>(b.Qpart), s.cols_per_split, b.resid_part, s.r,
                b.st);
          }
        }
        return vec ? go(BodyTag<&sweep_mx_body<TMs, RP, true>>{}) : go(BodyTag<&sweep_mx_body<TMs, RP, false>>{});
      });
    }
  });
}

cudaError_t launch_sweep(const Shape& s, const Buffers& b, bool fp64, int u_cur, cudaStream_t st) {
  // Y ping-pong: iteration k (0-based count of completed iterations) reads Y[k % 2] and writes
  // Y[(k + 1) % 2].  The host tracks k because graphs are replayed per iteration parity.
  if (mx_path(s, fp64)) return launch_sweep_mx(s, b, u_cur, st);
  dim3 grid(s.sweep_grid_x, s.nsplit);
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      const size_t smem = sizeof(TC) * ((size_t)RP * kSweepBM + (size_t)RP * kSweepBN * 2 +
                                        (size_t)kSweepBM * (kSweepBN + 1));
      return by_mtype(b.m_dtype, b.M, [&](auto M) {
        using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
        auto kern = sweep_kernel<TC, TMs, RP>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        launch_pdl(kern, grid, 256, smem, st, M, s.m, s.n, s.ldm, static_cast<const TC*>(b.Y[0]), static_cast<TC*>(b.Y[1]),
                                      static_cast<TC*>(b.D), static_cast<const TC*>(b.U[u_cur]),
                                      static_cast<const TC*>(b.C), static_cast<const TC*>(b.V),
                                      static_cast<TC*>(b.Qpart), s.cols_per_split, b.resid_part, b.st);
        return cudaGetLastError();
      });
    });
  });
}

cudaError_t launch_iter_end(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st) {
  // the mixed SIMT sweep writes one residual partial per (column split, 64-row block, warp), the
  // float64 SIMT sweep one per 32-row block and split, the tensor-core sweep one per CTA
  const int count = mx_path(s, fp64) ? s.nsplit * (int)((s.m + 63) / 64) * 8
                                     : (b.tc ? s.resid_parts : s.sweep_grid_x * s.nsplit);
  launch_k<&iter_end_body, 1024>(1, 1024, 0, st, b.resid_part, count, b.st);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Shape& s, const Buffers& b, bool fp64, int u_cur, void* S, sfr_dtype s_dtype,
                            int64_t lds, void* L, cudaStream_t st) {
  // Y_prev is the multiplier the last sweep read: Buffers::Y[0] by the host's swap convention.
  const int64_t nblk = (int64_t)cdiv(s.n, 32) * cdiv(s.m, 8);
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)nblk;
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      return by_mtype(b.m_dtype, b.M, [&](auto M) {
        using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
        auto go = [&](auto yptr, int64_t ldy) {
          using TY = std::remove_const_t<std::remove_pointer_t<decltype(yptr)>>;
          if (s_dtype == SFR_F64)
            launch_pdl(finalize_kernel<TC, TMs, double, TY, RP>, grid, 256, 0, st,
                M, s.m, s.n, s.ldm, yptr, ldy, static_cast<const TC*>(b.U[u_cur]), static_cast<const TC*>(b.C),
                static_cast<double*>(S), static_cast<double*>(L), lds, b.st);
          else
            launch_pdl(finalize_kernel<TC, TMs, float, TY, RP>, grid, 256, 0, st,
                M, s.m, s.n, s.ldm, yptr, ldy, static_cast<const TC*>(b.U[u_cur]), static_cast<const TC*>(b.C),
                static_cast<float*>(S), static_cast<float*>(L), lds, b.st);
          return cudaGetLastError();
        };
        if (b.tc) return go(static_cast<const __nv_bfloat16*>(b.Y[0]), b.t.ldy);
        return go(static_cast<const TC*>(b.Y[0]), b.ldy);
      });
    });
  });
}

cudaError_t launch_export_factors(const Shape& s, const Buffers& b, bool fp64, int u_cur, double* U, double* V,
                                  cudaStream_t st) {
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      if (U) launch_pdl(export_kernel<TC, RP>, cdiv(s.m * s.r, 256), 256, 0, st, static_cast<const TC*>(b.U[u_cur]), s.m, s.r, U);
      if (V) launch_pdl(export_kernel<TC, RP>, cdiv(s.n * s.r, 256), 256, 0, st, static_cast<const TC*>(b.V), s.n, s.r, V);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_ppass(const Shape& s, const Buffers& b, bool fp64, cudaStream_t st) {
  dim3 grid(s.sweep_grid_x, s.nsplit);
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      return by_mtype(b.m_dtype, b.M, [&](auto M) {
        using TMs = std::remove_const_t<std::remove_pointer_t<decltype(M)>>;
        launch_pdl(ppass_kernel<TC, TMs, RP>, grid, 256, 0, st, M, s.m, s.n, s.ldm, static_cast<const TC*>(b.V),
                                                         static_cast<TC*>(b.Qpart), s.cols_per_split, b.st);
        return cudaGetLastError();
      });
    });
  });
}

cudaError_t launch_full_end(const Shape& s, const Buffers& b, cudaStream_t st) {
  launch_pdl(full_end_kernel, 1, 256, 0, st, b.B, b.Bprev, s.rp, s.r, b.st);
  return cudaGetLastError();
}

cudaError_t launch_import(const Shape& s, const double* src, int64_t rows, void* dst, bool fp64, cudaStream_t st) {
  return by_prec(fp64, [&](auto tc) {
    using TC = decltype(tc);
    return by_rank(s.rp, [&](auto rpc) {
      constexpr int RP = decltype(rpc)::value;
      launch_pdl(import_kernel<TC, RP>, cdiv(rows * RP, 256), 256, 0, st, src, rows, s.r, static_cast<TC*>(dst));
      return cudaGetLastError();
    });
  });
}

}  // namespace sfr
