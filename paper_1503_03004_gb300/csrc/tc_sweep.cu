// Tensor-core (tcgen05 + TMA) version of the m x n passes of the mixed path, r <= 64.
//
// Per FR-ADM iteration (Algorithm 1 with the L-step of Algorithm 3), the two m x n passes are
//   sweep:  L = U_bar C^T, z = M - L + Y_k/mu_k, Y_{k+1} = clip(mu_k z, -1, 1),
//           Delta = Y_{k+1}(1/mu_k + 1/mu_{k+1}) - Y_k/mu_k, residual += (Y_{k+1} - Y_k)^2,
//           Q += Delta V_bar  (so that P_{k+1} = X_{k+1} V_bar = U_bar B_bar + Q, as V_bar^T V_bar = I);
//   W pass: W = X_{k+1}^T U_new = C (U_bar^T U_new) + Delta^T U_new.
// Storage: M, Y and Delta in bfloat16 (Delta also written transposed, n x m, so the W pass
// reads K-major operands), arithmetic in float32.  L is formed on the tensor cores as three
// TF32 products U_hi C_hi^T + U_hi C_lo^T + U_lo C_hi^T (hi = x rounded to TF32, lo = x - hi),
// which keeps float32-level accuracy; Delta V_bar and Delta^T U_new are bfloat16 products
// (Delta is O(1/mu), so its rounding is small against L).
//
// Sweep CTA: 128 rows x a range of 64-column tiles.  Warps 0-3 are the epilogue (one thread
// per row, TMEM lane = row), warp 4 issues TMA loads, warp 5 owns TMEM and issues MMAs.
#include <cuda.h>

#include "sfr_internal.h"
#include "tc_common.cuh"
#include "tc_sweep.h"

namespace sfr {
namespace {

using namespace tc;

constexpr int TBM = 128, TBN = 64, TR = 64;

// shared memory map of the sweep kernel (offsets from a 1024-byte aligned base)
constexpr uint32_t OFF_UH = 0;          // U_hi: 2 K-atoms x 128 rows x 128 B
constexpr uint32_t OFF_UL = 32768;      // U_lo
constexpr uint32_t OFF_CH = 65536;      // C_hi tile: 2 K-atoms x 64 rows x 128 B
constexpr uint32_t OFF_CL = 81920;      // C_lo tile
constexpr uint32_t OFF_VT = 98304;      // V^T tile (64 a-rows x 64 j bf16), 2 stages x 8 KB
constexpr uint32_t OFF_MS = 114688;     // M tile (128 x 64 bf16), 2 stages x 16 KB
constexpr uint32_t OFF_YS = 147456;     // Y tile (128 x 64 bf16), 2 stages x 16 KB; Y_{k+1} written in place
constexpr uint32_t OFF_DA = 180224;     // Delta tile, A operand of Delta V (128 x 64 bf16)
constexpr uint32_t OFF_DT = 196608;     // Delta^T staging: 2 boxes x 64 j-rows x 64 i bf16
constexpr uint32_t OFF_BAR = 212992;    // mbarriers and flags
constexpr uint32_t SWEEP_SMEM = OFF_BAR + 256 + 1024;

struct SweepBars {
  uint64_t u_full;
  uint64_t stage_full[2];
  uint64_t stage_empty[2];
  uint64_t c_full, c_empty;
  uint64_t l_full[2], l_empty[2];
  uint64_t d_full, d_empty;
  uint64_t q_full;
  uint32_t tmem_base;
  int abort;
  float red[4];
};
static_assert(sizeof(SweepBars) <= 256, "barrier block");

__device__ __forceinline__ bool stopped(const DevState* st) { return *(volatile const int32_t*)&st->done != 0; }

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(192, 1) sweep_tc_kernel(const __grid_constant__ CUtensorMap tmM,
                                                          const __grid_constant__ CUtensorMap tmYin,
                                                          const __grid_constant__ CUtensorMap tmYout,
                                                          const __grid_constant__ CUtensorMap tmDt,
                                                          const __grid_constant__ CUtensorMap tmUh,
                                                          const __grid_constant__ CUtensorMap tmUl,
                                                          const __grid_constant__ CUtensorMap tmCh,
                                                          const __grid_constant__ CUtensorMap tmCl,
                                                          const __grid_constant__ CUtensorMap tmVt, int64_t m,
                                                          int64_t n, int cols_per_split, float* __restrict__ Qpart,
                                                          double* __restrict__ resid_part, DevState* st) {
  if (stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  SweepBars& B = *reinterpret_cast<SweepBars*>(sm + OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * TBM;
  const int jbeg = blockIdx.y * cols_per_split;
  const int jend = (int)(((int64_t)jbeg + cols_per_split < n) ? (int64_t)jbeg + cols_per_split : n);
  const int ntiles = (jend - jbeg + TBN - 1) / TBN;
  volatile int* abort = &B.abort;

  if (tid == 0) {
    mbar_init(&B.u_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&B.stage_full[s], 1);
      mbar_init(&B.stage_empty[s], 2);
      mbar_init(&B.l_full[s], 1);
      mbar_init(&B.l_empty[s], 128);
    }
    mbar_init(&B.c_full, 1);
    mbar_init(&B.c_empty, 1);
    mbar_init(&B.d_full, 1);
    mbar_init(&B.d_empty, 1);
    mbar_init(&B.q_full, 1);
    B.abort = 0;
    mbar_fence_init();
  }
  if (warp == 5) tmem_alloc(&B.tmem_base, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;

  if (warp == 4) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_map(&tmM);
      prefetch_map(&tmYin);
      mbar_expect_tx(&B.u_full, 4 * 16384);
      for (int a = 0; a < 2; ++a) {
        tma_load_2d(sm + OFF_UH + a * 16384, &tmUh, 32 * a, i0, &B.u_full);
        tma_load_2d(sm + OFF_UL + a * 16384, &tmUl, 32 * a, i0, &B.u_full);
      }
      int armed_stage[2] = {-1, -1}, armed_c = -1;  // last tile whose loads were issued per barrier
      for (int t = 0; t < ntiles && !*abort; ++t) {
        const int s = t & 1, j0 = jbeg + t * TBN;
        if (t >= 2 && !mbar_wait(&B.stage_empty[s], ((t >> 1) - 1) & 1, abort)) break;
        mbar_expect_tx(&B.stage_full[s], 16384 + 16384 + 8192);
        tma_load_2d(sm + OFF_MS + s * 16384, &tmM, j0, i0, &B.stage_full[s]);
        tma_load_2d(sm + OFF_YS + s * 16384, &tmYin, j0, i0, &B.stage_full[s]);
        tma_load_2d(sm + OFF_VT + s * 8192, &tmVt, j0, 0, &B.stage_full[s]);
        armed_stage[s] = t;
        if (t >= 1 && !mbar_wait(&B.c_empty, (t - 1) & 1, abort)) break;
        mbar_expect_tx(&B.c_full, 4 * 8192);
        for (int a = 0; a < 2; ++a) {
          tma_load_2d(sm + OFF_CH + a * 8192, &tmCh, 32 * a, j0, &B.c_full);
          tma_load_2d(sm + OFF_CL + a * 8192, &tmCl, 32 * a, j0, &B.c_full);
        }
        armed_c = t;
      }
      if (*abort) {  // let the copies this thread issued land before the CTA exits
        int dummy = 0;
        mbar_wait(&B.u_full, 0, &dummy);
        for (int q = 0; q < 2; ++q)
          if (armed_stage[q] >= 0) { dummy = 0; mbar_wait(&B.stage_full[q], (armed_stage[q] >> 1) & 1, &dummy); }
        if (armed_c >= 0) { dummy = 0; mbar_wait(&B.c_full, armed_c & 1, &dummy); }
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id_l = idesc(2, TBM, TBN);   // tf32, 128 x 64
      const uint32_t id_q = idesc(1, TBM, TR);    // bf16, 128 x 64
      const uint32_t q_tmem = tmem + 128;
      auto delta_v = [&](int tt) -> bool {
        const int s = tt & 1;
        if (!mbar_wait(&B.d_full, tt & 1, abort)) return false;
        tc_fence_after();
        for (int kk = 0; kk < TBN / 16; ++kk) {
          const uint64_t a = desc_sw128(smem_u32(sm + OFF_DA) + kk * 32);
          const uint64_t b = desc_sw128(smem_u32(sm + OFF_VT + s * 8192) + kk * 32);
          mma_bf16(q_tmem, a, b, id_q, (tt > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&B.d_empty);
        mma_commit(&B.stage_empty[s]);
        return true;
      };
      bool ok = mbar_wait(&B.u_full, 0, abort);
      for (int t = 0; ok && t < ntiles; ++t) {
        const int b = t & 1;
        if (!mbar_wait(&B.c_full, t & 1, abort)) { ok = false; break; }
        if (t >= 2 && !mbar_wait(&B.l_empty[b], ((t >> 1) - 1) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + b * TBN;
        // L = U_hi C_hi^T + U_hi C_lo^T + U_lo C_hi^T, K = 64 in 8 steps of 8 (32 bytes)
        for (int term = 0; term < 3; ++term) {
          const uint32_t ua = smem_u32(sm + (term == 2 ? OFF_UL : OFF_UH));
          const uint32_t cb = smem_u32(sm + (term == 1 ? OFF_CL : OFF_CH));
          for (int ks = 0; ks < 8; ++ks) {
            const uint32_t koff = (ks >> 2) * 0 + (ks & 3) * 32;
            const uint64_t a = desc_sw128(ua + (ks >> 2) * 16384 + koff);
            const uint64_t bb = desc_sw128(cb + (ks >> 2) * 8192 + koff);
            mma_tf32(d, a, bb, id_l, (term > 0 || ks > 0) ? 1u : 0u);
          }
        }
        mma_commit(&B.l_full[b]);
        mma_commit(&B.c_empty);
        if (t >= 1 && !delta_v(t - 1)) { ok = false; break; }
      }
      if (ok && ntiles > 0) ok = delta_v(ntiles - 1);
      if (ok) mma_commit(&B.q_full);
      else {  // MMAs already issued must finish before the accumulator memory is released
        int dummy = 0;
        mma_commit(&B.q_full);
        mbar_wait(&B.q_full, 0, &dummy);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue: warps 0-3, one row per thread
    const int row = tid;                      // TMEM lane and tile row
    const int64_t gi = (int64_t)i0 + row;
    const float mu = (float)st->mu;
    const double mu_next_d = fmin(st->mu_max, st->rho * st->mu);
    const float inv_mu = (float)(1.0 / st->mu), dcoef = (float)(1.0 / st->mu + 1.0 / mu_next_d);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    float resid = 0.f;
    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t & 1, b = t & 1, j0 = jbeg + t * TBN;
      mbar_wait(&B.l_full[b], (t >> 1) & 1, abort) && mbar_wait(&B.stage_full[s], (t >> 1) & 1, abort) &&
          (t == 0 || mbar_wait(&B.d_empty, (t - 1) & 1, abort));
      named_bar(1, 128);  // the abort decision below is the same for all epilogue threads
      if (*abort) {
        ok = false;
        break;
      }
      tc_fence_after();
      float L[TBN];
#pragma unroll
      for (int c = 0; c < TBN; c += 16) tmem_ld16(tmem + lane_base + b * TBN + c, L + c);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive(&B.l_empty[b]);
      unsigned char* ms = sm + OFF_MS + s * 16384;
      unsigned char* ys = sm + OFF_YS + s * 16384;
      unsigned char* da = sm + OFF_DA;
      unsigned char* dt = sm + OFF_DT + (row >> 6) * 8192;
      const int ir = row & 63;
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // 16-byte chunk c = columns 8c .. 8c+7
        const uint32_t off = sw128(row, c);
        const uint4 mw = *reinterpret_cast<const uint4*>(ms + off);
        const uint4 yw = *reinterpret_cast<const uint4*>(ys + off);
        const uint32_t mv[4] = {mw.x, mw.y, mw.z, mw.w}, yv[4] = {yw.x, yw.y, yw.z, yw.w};
        uint32_t yo[4], dd[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float ynew[2], dnew[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int col = 8 * c + 2 * h + e;
            const float mval = e ? bf_hi(mv[h]) : bf_lo(mv[h]);
            const float y = e ? bf_hi(yv[h]) : bf_lo(yv[h]);
            const bool in = j0 + col < jend;
            const float z = mval - L[col] + y * inv_mu;
            float yn = fminf(1.f, fmaxf(-1.f, mu * z));
            yn = in ? __bfloat162float(__float2bfloat16_rn(yn)) : 0.f;  // value as stored
            const float dv = yn * dcoef - y * inv_mu;
            const float dy = yn - y;
            resid = fmaf(dy, dy, resid);
            ynew[e] = yn;
            dnew[e] = in ? dv : 0.f;
          }
          yo[h] = pack_bf2(ynew[0], ynew[1]);
          dd[h] = pack_bf2(dnew[0], dnew[1]);
        }
        *reinterpret_cast<uint4*>(ys + off) = make_uint4(yo[0], yo[1], yo[2], yo[3]);
        *reinterpret_cast<uint4*>(da + off) = make_uint4(dd[0], dd[1], dd[2], dd[3]);
        // transposed copy: element (j = 8c + q, i = row) -> box (row / 64), row j, i-chunk (ir / 8)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t w = dd[q >> 1];
          const unsigned short hv = (unsigned short)((q & 1) ? (w >> 16) : (w & 0xFFFF));
          *reinterpret_cast<unsigned short*>(dt + sw128(8 * c + q, ir >> 3) + (ir & 7) * 2) = hv;
        }
      }
      fence_async_smem();
      named_bar(1, 128);
      if (tid == 0) {
        mbar_arrive(&B.d_full);
        tma_store_2d(&tmYout, ys, j0, i0);
        tma_store_2d(&tmDt, sm + OFF_DT, i0, j0);
        tma_store_2d(&tmDt, sm + OFF_DT + 8192, i0 + 64, j0);
        tma_store_commit();
        tma_store_wait_read0();
        mbar_arrive(&B.stage_empty[s]);
      }
      named_bar(1, 128);
    }
    if (ok && ntiles > 0) mbar_wait(&B.q_full, 0, abort);
    named_bar(1, 128);  // uniform decision before the warp-collective TMEM loads
    if (ok && ntiles > 0 && !*abort) {
      tc_fence_after();
      float q[TR];
#pragma unroll
      for (int c = 0; c < TR; c += 16) tmem_ld16(tmem + lane_base + 128 + c, q + c);
      tmem_ld_wait();
      if (gi < m) {
        float4* dst = reinterpret_cast<float4*>(Qpart + ((int64_t)blockIdx.y * m + gi) * TR);
#pragma unroll
        for (int c = 0; c < TR / 4; ++c) dst[c] = make_float4(q[4 * c], q[4 * c + 1], q[4 * c + 2], q[4 * c + 3]);
      }
    }
    if (tid == 0) tma_store_wait0();
    // residual: warp sums, then thread 0 combines the four warps in a fixed order
    for (int o = 16; o > 0; o >>= 1) resid += __shfl_xor_sync(0xffffffffu, resid, o);
    if (lane == 0) B.red[warp] = resid;
    named_bar(1, 128);
    if (tid == 0)
      resid_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] =
          (double)B.red[0] + (double)B.red[1] + (double)B.red[2] + (double)B.red[3];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
  if (tid == 0 && B.abort) {
    st->status = SFR_E_TIMEOUT;
    st->done = 1;
  }
}

// ---------------------------------------------------------------- W pass: W = Delta^T U on tensor cores
// CTA: 128 columns j of Delta (rows of Delta^T) x a chunk of rows i; D (128 x 64) in TMEM.
constexpr int WSTAGES = 4;
constexpr uint32_t W_A_BYTES = 16384, W_B_BYTES = 8192, W_STAGE = W_A_BYTES + W_B_BYTES;
constexpr uint32_t W_OFF_BAR = WSTAGES * W_STAGE;
constexpr uint32_t WPASS_SMEM = W_OFF_BAR + 128 + 1024;

struct WBars {
  uint64_t full[WSTAGES], empty[WSTAGES];
  uint64_t acc_full;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(192, 1) wpass_tc_kernel(const __grid_constant__ CUtensorMap tmDt,
                                                          const __grid_constant__ CUtensorMap tmUt, int64_t m,
                                                          int64_t n, int rows_per_chunk, float* __restrict__ Wpart,
                                                          DevState* st) {
  if (stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  WBars& B = *reinterpret_cast<WBars*>(sm + W_OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * 128;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = (int)(((int64_t)r0 + rows_per_chunk < m) ? (int64_t)r0 + rows_per_chunk : m);
  const int nk = (r1 - r0 + 63) / 64;
  volatile int* abort = &B.abort;
  if (tid == 0) {
    for (int s = 0; s < WSTAGES; ++s) {
      mbar_init(&B.full[s], 1);
      mbar_init(&B.empty[s], 1);
    }
    mbar_init(&B.acc_full, 1);
    B.abort = 0;
    mbar_fence_init();
  }
  if (warp == 5) tmem_alloc(&B.tmem_base, 64);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  if (warp == 4) {
    if (lane == 0) {
      int armed[WSTAGES];
      for (int q = 0; q < WSTAGES; ++q) armed[q] = -1;
      for (int k = 0; k < nk && !*abort; ++k) {
        const int s = k % WSTAGES;
        if (k >= WSTAGES && !mbar_wait(&B.empty[s], ((k / WSTAGES) - 1) & 1, abort)) break;
        mbar_expect_tx(&B.full[s], W_STAGE);
        tma_load_2d(sm + s * W_STAGE, &tmDt, r0 + 64 * k, j0, &B.full[s]);
        tma_load_2d(sm + s * W_STAGE + W_A_BYTES, &tmUt, r0 + 64 * k, 0, &B.full[s]);
        armed[s] = k;
      }
      if (*abort)
        for (int q = 0; q < WSTAGES; ++q)
          if (armed[q] >= 0) {
            int dummy = 0;
            mbar_wait(&B.full[q], (armed[q] / WSTAGES) & 1, &dummy);
          }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t id = idesc(1, 128, TR);
      bool ok = true;
      for (int k = 0; k < nk; ++k) {
        const int s = k % WSTAGES;
        if (!mbar_wait(&B.full[s], (k / WSTAGES) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t a = desc_sw128(smem_u32(sm + s * W_STAGE) + kk * 32);
          const uint64_t b = desc_sw128(smem_u32(sm + s * W_STAGE + W_A_BYTES) + kk * 32);
          mma_bf16(tmem, a, b, id, (k > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&B.empty[s]);
      }
      mma_commit(&B.acc_full);
      if (!ok) {
        int dummy = 0;
        mbar_wait(&B.acc_full, 0, &dummy);
      }
    }
  } else {
    const int64_t gj = (int64_t)j0 + tid;
    float w[TR];
    bool have = false;
    if (nk == 0) {
#pragma unroll
      for (int c = 0; c < TR; ++c) w[c] = 0.f;
      have = true;
    } else {
      mbar_wait(&B.acc_full, 0, abort);
      named_bar(1, 128);  // uniform decision before the warp-collective TMEM loads
      if (!*abort) {
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < TR; c += 16) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, w + c);
        tmem_ld_wait();
        have = true;
      }
    }
    if (have && gj < n) {
      float4* dst = reinterpret_cast<float4*>(Wpart + ((int64_t)blockIdx.y * n + gj) * TR);
#pragma unroll
      for (int c = 0; c < TR / 4; ++c) dst[c] = make_float4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, 64);
  }
  if (tid == 0 && B.abort) {
    st->status = SFR_E_TIMEOUT;
    st->done = 1;
  }
}

// ---------------------------------------------------------------- thin preparation kernels
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// From U (rows x 64 f32): hi = tf32(U), lo = U - hi (rows x 64 f32), and U^T in bf16 (64 x ldt).
// Same routine for C (hi/lo) with V^T taken from a second input.
__global__ void split_transpose_kernel(const float* __restrict__ X, const float* __restrict__ Xt_src, int64_t rows,
                                       float* __restrict__ hi, float* __restrict__ lo, __nv_bfloat16* __restrict__ t,
                                       int64_t ldt, const DevState* st) {
  if (stopped(st)) return;
  __shared__ float tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int rr = e / 64, a = e % 64;
    const int64_t i = r0 + rr;
    if (i < rows) {
      const float x = X[i * 64 + a];
      const float h = tf32_round(x);
      hi[i * 64 + a] = h;
      lo[i * 64 + a] = x - h;
      tile[rr][a] = Xt_src[i * 64 + a];
    } else {
      tile[rr][a] = 0.f;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int a = e / 64, rr = e % 64;
    const int64_t i = r0 + rr;
    if (i < rows) t[(int64_t)a * ldt + i] = __float2bfloat16_rn(tile[rr][a]);
  }
}

// Mt = M^T (bf16), so iteration 1's W = M^T U uses the same K-major pass as later iterations.
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ M, int64_t m, int64_t n, int64_t ldm,
                                      __nv_bfloat16* __restrict__ Mt, int64_t ldt) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int ii = e / 64, jj = e % 64;
    tile[ii][jj] = (i0 + ii < m && j0 + jj < n) ? M[(i0 + ii) * ldm + j0 + jj] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int jj = e / 64, ii = e % 64;
    if (i0 + ii < m && j0 + jj < n) Mt[(j0 + jj) * ldt + i0 + ii] = tile[ii][jj];
  }
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------- tensor maps
// cuTensorMapEncodeTiled, fetched through the runtime so the library needs no -lcuda
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, CUtensorMapDataType dt, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_supported(const Shape& s, int m_dtype, int64_t ldm) {
  return s.rp == 64 && m_dtype == SFR_BF16 && ldm % 8 == 0 && s.n % 8 == 0 && s.m % 8 == 0 && encode_fn() != nullptr;
}

cudaError_t tc_make_maps(const Shape& s, const TcBuffers& t, const void* M, int64_t ldm, TcMaps* maps) {
  const auto BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  bool ok = true;
  ok &= make_map(&maps->M, M, BF, s.n, s.m, 2 * ldm, 64, 128);
  for (int q = 0; q < 2; ++q) ok &= make_map(&maps->Y[q], t.Y[q], BF, s.n, s.m, 2 * t.ldy, 64, 128);
  ok &= make_map(&maps->Dt_store, t.Dt, BF, s.m, s.n, 2 * t.ldd, 64, 64);
  ok &= make_map(&maps->Dt_load, t.Dt, BF, s.m, s.n, 2 * t.ldd, 64, 128);
  ok &= make_map(&maps->Ut, t.Ut, BF, s.m, 64, 2 * t.ldd, 64, 64);
  ok &= make_map(&maps->Uh, t.Uh, F32, 64, s.m, 256, 32, 128);
  ok &= make_map(&maps->Ul, t.Ul, F32, 64, s.m, 256, 32, 128);
  ok &= make_map(&maps->Ch, t.Ch, F32, 64, s.n, 256, 32, 64);
  ok &= make_map(&maps->Cl, t.Cl, F32, 64, s.n, 256, 32, 64);
  ok &= make_map(&maps->Vt, t.Vt, BF, s.n, 64, 2 * t.ldy, 64, 64);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_launch_transpose_m(const Shape& s, const void* M, int64_t ldm, const TcBuffers& t, cudaStream_t st) {
  dim3 grid(cdiv(s.n, 64), cdiv(s.m, 64));
  transpose_bf16_kernel<<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(M), s.m, s.n, ldm,
                                              static_cast<__nv_bfloat16*>(t.Dt), t.ldd);
  return cudaGetLastError();
}

cudaError_t tc_launch_prep_u(const Shape& s, const float* U, const TcBuffers& t, const DevState* dst, cudaStream_t st) {
  split_transpose_kernel<<<cdiv(s.m, 64), 256, 0, st>>>(U, U, s.m, t.Uh, t.Ul, static_cast<__nv_bfloat16*>(t.Ut),
                                                        t.ldd, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_prep_v(const Shape& s, const float* C, const float* V, const TcBuffers& t, const DevState* dst,
                             cudaStream_t st) {
  split_transpose_kernel<<<cdiv(s.n, 64), 256, 0, st>>>(C, V, s.n, t.Ch, t.Cl, static_cast<__nv_bfloat16*>(t.Vt),
                                                        t.ldy, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_wpass(const Shape& s, const TcMaps& mp, float* Wpart, DevState* dst, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(wpass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WPASS_SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(s.n, 128), s.nchunk);
  wpass_tc_kernel<<<grid, 192, WPASS_SMEM, st>>>(mp.Dt_load, mp.Ut, s.m, s.n, s.rows_per_chunk, Wpart, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_sweep(const Shape& s, const TcMaps& mp, int y_in, float* Qpart, double* resid_part,
                            DevState* dst, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(sweep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(s.m, TBM), s.nsplit);
  sweep_tc_kernel<<<grid, 192, SWEEP_SMEM, st>>>(mp.M, mp.Y[y_in], mp.Y[1 - y_in], mp.Dt_store, mp.Uh, mp.Ul, mp.Ch,
                                                  mp.Cl, mp.Vt, s.m, s.n, s.cols_per_split, Qpart, resid_part, dst);
  return cudaGetLastError();
}

}  // namespace sfr
