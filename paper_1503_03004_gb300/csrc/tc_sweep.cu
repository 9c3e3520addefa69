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
// Sweep CTA: 128 rows x a range of 64-column tiles.  Warps 0-7 are the epilogue (warp w reads
// TMEM lanes 32 (w % 4) .. + 31, i.e. rows, and columns 32 (w / 4) .. + 31 of each tile), warp 8
// issues TMA loads, warp 9 owns TMEM and issues MMAs.
#include <cuda.h>

#include <algorithm>

#include "sfr_internal.h"
#include "tc_common.cuh"
#include "tc_sweep.h"

namespace sfr {
namespace {

using namespace tc;

constexpr int TBM = 128, TBN = 64, TR = 64;

// shared memory map of the sweep kernel (offsets from a 1024-byte aligned base)
constexpr int NSTAGE = 2;
constexpr int NCB = 3;  // C tile buffers (they come from L2 about 3 us after issue)
constexpr uint32_t OFF_C = 0;           // C tiles, NCB buffers x 32 KB: hi (2 K-atoms x 64 rows x 128 B) then lo
constexpr uint32_t C_BUF = 32768;
constexpr uint32_t OFF_ST = NCB * 32768;      // input stages, NSTAGE x 32 KB: M tile (128 x 64 bf16), Y tile; each
constexpr uint32_t ST_BYTES = 32768;    // epilogue warp releases a stage once it has its M and Y values in registers
                                        // and the previous tile's bulk stores have read their source
constexpr uint32_t ST_Y = 16384;
constexpr int NVT = 4;                  // V^T tiles (64 x 64 bf16), a ring of 4: held until Delta V_bar is done
constexpr uint32_t OFF_VT = OFF_ST + NSTAGE * ST_BYTES;
constexpr uint32_t VT_BYTES = 8192;
constexpr uint32_t OFF_DA = OFF_VT + NVT * VT_BYTES;  // Delta tile, 16 KB: A operand of Delta V and TMA store
constexpr uint32_t DA_BYTES = 16384;                  // source; rewritten only once both are done with it
constexpr uint32_t OFF_YO = OFF_DA + DA_BYTES;        // Y_{k+1} tile, 16 KB: TMA store source
constexpr uint32_t OFF_BAR = OFF_YO + DA_BYTES;
constexpr uint32_t SWEEP_SMEM = OFF_BAR + 512 + 1024;
static_assert(OFF_BAR % 1024 == 0, "alignment");
static_assert(SWEEP_SMEM <= 232448, "shared memory per CTA");
// tensor memory columns: L double buffer; per segment s (a CTA's tiles span at most two 128-row
// blocks): Q at TM_Q + 64 s, U_hi at TM_U + 128 s, U_lo at TM_U + 128 s + 64
constexpr uint32_t TM_L = 0, TM_Q = 128, TM_U = 256, TM_COLS = 512;

struct SweepBars {
  uint64_t stage_full[NSTAGE], stage_empty[NSTAGE];
  uint64_t vt_full[NVT], vt_empty[NVT];
  uint64_t c_full[NCB], c_empty[NCB];
  uint64_t l_full[2], l_empty[2];
  uint64_t d_full, d_empty;
  uint64_t q_full;
  uint32_t tmem_base;
  int abort;
  double red[16];
};
static_assert(sizeof(SweepBars) <= 512, "barrier block");

__device__ __forceinline__ bool stopped(const DevState* st) { return *(volatile const int32_t*)&st->done != 0; }

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t id,
                                                uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(
          d_tmem),
      "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])));
}

// One 16-byte chunk (8 columns) of a row of the sweep epilogue: from M, Y_k (bfloat16 pairs) and L,
//   Y_{k+1} = clip(mu (M - L + Y_k / mu), -1, 1) rounded to bfloat16 (the stored value is the one used),
//   Delta = Y_{k+1} (1/mu + 1/mu_next) - Y_k / mu, resid += (Y_{k+1} - Y_k)^2.
// FULL: all 8 columns valid; else the first `nvalid` are (the rest give Y_{k+1} = Delta = 0).
template <bool FULL>
__device__ __forceinline__ void epi_chunk(const uint4& mw, const uint4& yw, const float* L, int nvalid, float mu,
                                          float inv_mu, float dcoef, uint4& yn_out, uint4& d_out, float& resid) {
  const uint32_t mv[4] = {mw.x, mw.y, mw.z, mw.w}, yv[4] = {yw.x, yw.y, yw.z, yw.w};
  uint32_t yn2[4], dd[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float y[2], ynr[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float mval = e ? bf_hi(mv[h]) : bf_lo(mv[h]);
      y[e] = e ? bf_hi(yv[h]) : bf_lo(yv[h]);
      const float z = mval - L[2 * h + e] + y[e] * inv_mu;
      ynr[e] = fminf(1.f, fmaxf(-1.f, mu * z));
      if (!FULL && 2 * h + e >= nvalid) ynr[e] = 0.f;
    }
    const uint32_t p = pack_bf2(ynr[0], ynr[1]);
    yn2[h] = p;
    float dv[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float yn = e ? bf_hi(p) : bf_lo(p);
      const float dy = yn - y[e];
      resid = fmaf(dy, dy, resid);
      dv[e] = yn * dcoef - y[e] * inv_mu;
      if (!FULL && 2 * h + e >= nvalid) dv[e] = 0.f;
    }
    dd[h] = pack_bf2(dv[0], dv[1]);
  }
  yn_out = make_uint4(yn2[0], yn2[1], yn2[2], yn2[3]);
  d_out = make_uint4(dd[0], dd[1], dd[2], dd[3]);
}

// Writes this thread's NC columns of a row (the first ncol of them valid): 16-byte vector stores
// when the destination allows them, else element by element.
template <typename TSo, int NC>
__device__ __forceinline__ void store_cols(TSo* dst, const float* v, int ncol, bool vec) {
  if (vec && ncol >= NC) {
    if constexpr (sizeof(TSo) == 4) {
#pragma unroll
      for (int q = 0; q < NC / 4; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < NC / 2; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(v[2 * q], v[2 * q + 1]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if (q < ncol) dst[q] = (TSo)v[q];
  }
}

// Epilogue: kEpiWarps warps; warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the
// kEpiCols columns kEpiCols (w / 4) .. of each 64-column tile.  Then the M / Y / V^T producer
// warp, the MMA warp and the C producer warp.
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kEpiCols = TBN / (kEpiWarps / 4);   // 16
constexpr int kEpiChunks = kEpiCols / 8;          // 16-byte chunks of a row per thread
constexpr int kProdWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kCProdWarp = kEpiWarps + 2;
constexpr int kSweepThreads = kEpiThreads + 96;
static_assert(kEpiCols % 16 == 0, "TMEM loads of 16 columns");

// Sweep CTA: a contiguous range of (128-row block, 64-column tile) pairs.  Warps 0-15: epilogue
// (warp w owns TMEM lanes / rows 32 (w % 4) .. + 31 and columns 16 (w / 4) .. + 15 of each tile);
// warp 16: TMA producer of M, Y and V^T; warp 17: TMEM owner and MMA issuer; warp 18: TMA
// producer of the C tiles.  U_hi / U_lo (the fixed A operand of the L
// products) live in tensor memory; M, Y and V^T tiles stream through three stages; C tiles
// are triple buffered; Y_{k+1} and Delta tiles are staged in shared memory and leave through TMA
// stores (the Delta tile is also the A operand of Delta V_bar).
// FINAL: the output pass after the last iteration instead (Algorithm 1 returns L_k, S_k):
// S = P_ST_{1/mu}(M - L + Y_k / mu) with the last iteration's mu, Y_k and factors, written
// (with L when requested) from registers; no V^T tiles, no Delta, no Y_{k+1}.
template <bool FINAL, typename TSo>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_tc_kernel(const __grid_constant__ CUtensorMap tmM,
                                                                   const __grid_constant__ CUtensorMap tmYin,
                                                                   const __grid_constant__ CUtensorMap tmYout,
                                                                   const __grid_constant__ CUtensorMap tmD,
                                                                   const __grid_constant__ CUtensorMap tmCh,
                                                                   const __grid_constant__ CUtensorMap tmCl,
                                                                   const __grid_constant__ CUtensorMap tmVt,
                                                                   const float* __restrict__ Uh,
                                                                   const float* __restrict__ Ul,
                                                                   int64_t m, int64_t n, float* __restrict__ Qpart,
                                                                   double* __restrict__ resid_part, DevState* st,
                                                                   TSo* __restrict__ Sout, TSo* __restrict__ Lout,
                                                                   int64_t lds, int vec_out) {
  pdl_enter();
  if (!FINAL && stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  SweepBars& B = *reinterpret_cast<SweepBars*>(sm + OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's tiles: [x0, x1) of the N (row block, column tile) pairs (tc_tile_owner); the host
  // keeps x1 - x0 <= T, so they span at most two row blocks: local tiles [0, kb) are segment 0
  // (row block rb0), [kb, ntiles) segment 1 (row block rb0 + 1)
  const int64_t T = (n + TBN - 1) / TBN, N = ((m + TBM - 1) / TBM) * T, G = gridDim.x;
  const int64_t x0 = (int64_t)blockIdx.x * N / G, x1 = ((int64_t)blockIdx.x + 1) * N / G;
  const int ntiles = (int)(x1 - x0);
  const int64_t rb0 = x0 / T;
  const int kb = (int)(((rb0 + 1) * T < x1 ? (rb0 + 1) * T : x1) - x0);
  const int nseg = kb < ntiles ? 2 : 1;
  auto tile_i0 = [&](int k) -> int { return (int)((rb0 + (k >= kb)) * TBM); };
  auto tile_j0 = [&](int k) -> int { return (int)((x0 + k - (rb0 + (k >= kb)) * T) * TBN); };
  volatile int* abort = &B.abort;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&B.stage_full[s], 1);
      mbar_init(&B.stage_empty[s], kEpiWarps);  // one arrival per epilogue warp
    }
    for (int v = 0; v < NVT; ++v) {
      mbar_init(&B.vt_full[v], 1);
      mbar_init(&B.vt_empty[v], 1);  // the Delta V MMAs of the tile have completed
    }
    for (int s = 0; s < NCB; ++s) {
      mbar_init(&B.c_full[s], 1);
      mbar_init(&B.c_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&B.l_full[s], 1);
      mbar_init(&B.l_empty[s], kEpiThreads);
    }
    for (int s = 0; s < 2; ++s) {
      if (s == 0) {
        mbar_init(&B.d_full, 1);
        mbar_init(&B.d_empty, 1);
      }
    }
    mbar_init(&B.q_full, 1);
    B.abort = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc(&B.tmem_base, TM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  const int quarter = warp & 3, grp = warp >> 2;
  const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
  if (warp < 8 * nseg) {
    // U_hi / U_lo rows of segment `seg` into tensor memory (lane = row, column = k)
    const int half = grp & 1, seg = warp >> 3;
    const int row = quarter * 32 + lane;
    const int64_t gi = (rb0 + seg) * TBM + row;
    float v[16];
    for (int part = 0; part < 2; ++part) {
      const float* src = part ? Ul : Uh;
      for (int c = 0; c < 32; c += 16) {
        const int k0 = half * 32 + c;
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = gi < m ? src[gi * TR + k0 + q] : 0.f;
        tmem_st16(tmem + lane_base + TM_U + 128 * seg + (part ? 64 : 0) + k0, v);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == kProdWarp) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_map(&tmM);
      prefetch_map(&tmYin);
      int armed_stage[NSTAGE], armed_vt[NVT];
      for (int q = 0; q < NSTAGE; ++q) armed_stage[q] = -1;
      for (int q = 0; q < NVT; ++q) armed_vt[q] = -1;
      for (int t = 0; t < ntiles && !*abort; ++t) {
        const int s = t % NSTAGE, i0 = tile_i0(t), j0 = tile_j0(t);
        if (t >= NSTAGE && !mbar_wait(&B.stage_empty[s], ((t / NSTAGE) - 1) & 1, abort)) break;
        unsigned char* stg = sm + OFF_ST + s * ST_BYTES;
        mbar_expect_tx(&B.stage_full[s], 16384 + 16384);
        tma_load_2d(stg, &tmM, j0, i0, &B.stage_full[s]);
        tma_load_2d(stg + ST_Y, &tmYin, j0, i0, &B.stage_full[s]);
        armed_stage[s] = t;
        if (!FINAL) {
          const int v = t % NVT;
          if (t >= NVT && !mbar_wait(&B.vt_empty[v], ((t / NVT) - 1) & 1, abort)) break;
          mbar_expect_tx(&B.vt_full[v], VT_BYTES);
          tma_load_2d(sm + OFF_VT + v * VT_BYTES, &tmVt, j0, 0, &B.vt_full[v]);
          armed_vt[v] = t;
        }
      }
      if (*abort) {  // let the copies this thread issued land before the CTA exits
        for (int q = 0; q < NSTAGE; ++q)
          if (armed_stage[q] >= 0) {
            int dummy = 0;
            mbar_wait(&B.stage_full[q], (armed_stage[q] / NSTAGE) & 1, &dummy);
          }
        for (int q = 0; q < NVT; ++q)
          if (armed_vt[q] >= 0) {
            int dummy = 0;
            mbar_wait(&B.vt_full[q], (armed_vt[q] / NVT) & 1, &dummy);
          }
      }
    }
  } else if (warp == kCProdWarp) {
    // ------------------------------------------------------------ TMA producer of the C tiles
    // (its own thread, so that waiting for a C buffer never holds back the M / Y stream)
    if (lane == 0) {
      int armed_c[NCB];
      for (int q = 0; q < NCB; ++q) armed_c[q] = -1;
      for (int t = 0; t < ntiles && !*abort; ++t) {
        const int cb = t % NCB, j0 = tile_j0(t);
        if (t >= NCB && !mbar_wait(&B.c_empty[cb], ((t / NCB) - 1) & 1, abort)) break;
        unsigned char* cbuf = sm + OFF_C + cb * C_BUF;
        mbar_expect_tx(&B.c_full[cb], 4 * 8192);
        for (int a = 0; a < 2; ++a) {
          tma_load_2d(cbuf + a * 8192, &tmCh, 32 * a, j0, &B.c_full[cb]);
          tma_load_2d(cbuf + 16384 + a * 8192, &tmCl, 32 * a, j0, &B.c_full[cb]);
        }
        armed_c[cb] = t;
      }
      if (*abort)
        for (int q = 0; q < NCB; ++q)
          if (armed_c[q] >= 0) {
            int dummy = 0;
            mbar_wait(&B.c_full[q], (armed_c[q] / NCB) & 1, &dummy);
          }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id_l = idesc(2, TBM, TBN);   // tf32, 128 x 64
      const uint32_t id_q = idesc(1, TBM, TR);    // bf16, 128 x 64
      auto delta_v = [&](int tt) -> bool {
        const int v = tt % NVT;
        if (!mbar_wait(&B.d_full, tt & 1, abort)) return false;
        if (!mbar_wait(&B.vt_full[v], (tt / NVT) & 1, abort)) return false;
        tc_fence_after();
        const uint32_t vt = smem_u32(sm + OFF_VT + v * VT_BYTES);
        for (int kk = 0; kk < TBN / 16; ++kk) {
          const uint64_t a = desc_sw128(smem_u32(sm + OFF_DA) + kk * 32);
          const uint64_t b = desc_sw128(vt + kk * 32);
          const int seg = tt >= kb, first = seg ? kb : 0;  // Q of each segment starts from zero
          mma_bf16(tmem + TM_Q + 64 * seg, a, b, id_q, (tt > first || kk > 0) ? 1u : 0u);
        }
        mma_commit(&B.d_empty);
        mma_commit(&B.vt_empty[v]);
        return true;
      };
      bool ok = true;
      for (int t = 0; ok && t < ntiles; ++t) {
        const int b = t & 1, cbi = t % NCB;
        if (!mbar_wait(&B.c_full[cbi], (t / NCB) & 1, abort)) { ok = false; break; }
        if (t >= 2 && !mbar_wait(&B.l_empty[b], ((t >> 1) - 1) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + TM_L + b * TBN;
        const uint32_t cbuf = smem_u32(sm + OFF_C + cbi * C_BUF);
        // L = U_hi C_hi^T + U_hi C_lo^T + U_lo C_hi^T, K = 64 in 8 steps of 8
        for (int term = 0; term < 3; ++term) {
          const uint32_t ua = tmem + TM_U + 128 * (t >= kb) + (term == 2 ? 64 : 0);
          const uint32_t cb = cbuf + (term == 1 ? 16384 : 0);
          for (int ks = 0; ks < 8; ++ks) {
            const uint64_t bb = desc_sw128(cb + (ks >> 2) * 8192 + (ks & 3) * 32);
            mma_tf32_tmem_a(d, ua + 8 * ks, bb, id_l, (term > 0 || ks > 0) ? 1u : 0u);
          }
        }
        mma_commit(&B.l_full[b]);
        mma_commit(&B.c_empty[cbi]);
        if (!FINAL && t >= 1 && !delta_v(t - 1)) { ok = false; break; }
      }
      if (!FINAL && ok && ntiles > 0) ok = delta_v(ntiles - 1);
      mma_commit(&B.q_full);
      if (!ok) {  // MMAs already issued must finish before the tensor memory is released
        int dummy = 0;
        mbar_wait(&B.q_full, 0, &dummy);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int row = quarter * 32 + lane;          // TMEM lane and tile row
    const int cbase = grp * kEpiCols;             // first of this warp's columns
    const float mu = (float)st->mu;
    const float inv_mu_last = (float)(1.0 / st->mu_last);
    const double mu_next_d = fmin(st->mu_max, st->rho * st->mu);
    const float inv_mu = (float)(1.0 / st->mu), dcoef = (float)(1.0 / st->mu + 1.0 / mu_next_d);
    double resid = 0.0;  // float64 sum of the per-tile float32 partials
    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % NSTAGE, b = t & 1, i0 = tile_i0(t), j0 = tile_j0(t);
      const int64_t gi = (int64_t)i0 + row;
      if constexpr (FINAL) {
        mbar_wait(&B.l_full[b], (t >> 1) & 1, abort) && mbar_wait(&B.stage_full[s], (t / NSTAGE) & 1, abort);
        named_bar(1, kEpiThreads);
        if (*abort) {
          ok = false;
          break;
        }
        const unsigned char* ms = sm + OFF_ST + s * ST_BYTES;
        uint4 mwr[kEpiChunks], ywr[kEpiChunks];
#pragma unroll
        for (int cc = 0; cc < kEpiChunks; ++cc) {
          const uint32_t off = sw128(row, grp * kEpiChunks + cc);
          mwr[cc] = *reinterpret_cast<const uint4*>(ms + off);
          ywr[cc] = *reinterpret_cast<const uint4*>(ms + ST_Y + off);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.stage_empty[s]);  // this warp is done with the stage
        tc_fence_after();
        float L[kEpiCols], sv[kEpiCols];
#pragma unroll
        for (int q = 0; q < kEpiCols / 16; ++q) tmem_ld16(tmem + lane_base + TM_L + b * TBN + cbase + 16 * q, L + 16 * q);
        tmem_ld_wait();
        tc_fence_before();
        mbar_arrive(&B.l_empty[b]);
#pragma unroll
        for (int cc = 0; cc < kEpiChunks; ++cc) {
          const uint4 mw = mwr[cc], yw = ywr[cc];
          const uint32_t mv[4] = {mw.x, mw.y, mw.z, mw.w}, yv[4] = {yw.x, yw.y, yw.z, yw.w};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float mval = (q & 1) ? bf_hi(mv[q >> 1]) : bf_lo(mv[q >> 1]);
            const float y = (q & 1) ? bf_hi(yv[q >> 1]) : bf_lo(yv[q >> 1]);
            const float z = mval - L[8 * cc + q] + y * inv_mu_last;
            sv[8 * cc + q] = z > inv_mu_last ? z - inv_mu_last : (z < -inv_mu_last ? z + inv_mu_last : 0.f);
          }
        }
        if (gi < m) {
          const int ncol = (int)(n - j0 - cbase);
          const int64_t o = gi * lds + j0 + cbase;
          if (Sout) store_cols<TSo, kEpiCols>(Sout + o, sv, ncol, vec_out != 0);
          if (Lout) store_cols<TSo, kEpiCols>(Lout + o, L, ncol, vec_out != 0);
        }
        continue;
      }
      mbar_wait(&B.l_full[b], (t >> 1) & 1, abort) && mbar_wait(&B.stage_full[s], (t / NSTAGE) & 1, abort);
      named_bar(1, kEpiThreads);  // the abort decision below is the same for all epilogue threads
      if (*abort) {
        ok = false;
        break;
      }
      const unsigned char* ms = sm + OFF_ST + s * ST_BYTES;
      uint4 mwr[kEpiChunks], ywr[kEpiChunks];
#pragma unroll
      for (int cc = 0; cc < kEpiChunks; ++cc) {
        const uint32_t off = sw128(row, grp * kEpiChunks + cc);
        mwr[cc] = *reinterpret_cast<const uint4*>(ms + off);
        ywr[cc] = *reinterpret_cast<const uint4*>(ms + ST_Y + off);
      }
      __syncwarp();
      tc_fence_after();
      float L[kEpiCols];
#pragma unroll
      for (int q = 0; q < kEpiCols / 16; ++q) tmem_ld16(tmem + lane_base + TM_L + b * TBN + cbase + 16 * q, L + 16 * q);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive(&B.l_empty[b]);
      unsigned char* da = sm + OFF_DA;
      unsigned char* yo = sm + OFF_YO;
      const int ncol = (int)(n - j0 - cbase);  // valid columns among this thread's (may be <= 0)
      uint4 yn[kEpiChunks], dd[kEpiChunks];
      float rt = 0.f;  // this thread's part of the tile (at most 64 terms)
#pragma unroll
      for (int cc = 0; cc < kEpiChunks; ++cc) {  // 16-byte chunk c = columns 8c .. 8c+7
        if (ncol >= kEpiCols) epi_chunk<true>(mwr[cc], ywr[cc], L + 8 * cc, 0, mu, inv_mu, dcoef, yn[cc], dd[cc], rt);
        else epi_chunk<false>(mwr[cc], ywr[cc], L + 8 * cc, ncol - 8 * cc, mu, inv_mu, dcoef, yn[cc], dd[cc], rt);
      }
      resid += (double)rt;
      // the single Delta / Y_{k+1} tiles are free once Delta V of tile t - 1 is done and the TMA
      // stores of tile t - 1 have read them (long done by now: the waits come after the compute)
      if (t >= 1) mbar_wait(&B.d_empty, (t - 1) & 1, abort);
      if (tid == 0 && t >= 1) tma_store_wait_read0();
      named_bar(1, kEpiThreads);
      // the stage goes back to the producer only now, after the bulk stores of tile t - 1 have
      // read their shared-memory source: with the release right after the stage reads, the
      // stage's next TMA load could overlap those stores' reads, and on GB300 about 450 of the
      // 67 M values that one 8192^2 sweep stored (upper 16-byte halves of 32-byte sectors in the
      // first rows of odd tiles) then differed from run to run
      if (lane == 0) mbar_arrive(&B.stage_empty[s]);
#pragma unroll
      for (int cc = 0; cc < kEpiChunks; ++cc) {
        const uint32_t off = sw128(row, grp * kEpiChunks + cc);
        *reinterpret_cast<uint4*>(yo + off) = yn[cc];
        *reinterpret_cast<uint4*>(da + off) = dd[cc];
      }
      fence_async_smem();
      named_bar(1, kEpiThreads);
      if (tid == 0) {
        mbar_arrive(&B.d_full);
        tma_store_2d(&tmYout, yo, j0, i0);
        tma_store_2d(&tmD, da, j0, i0);
        tma_store_commit();
      }
    }
    if (ok && ntiles > 0) mbar_wait(&B.q_full, 0, abort);
    named_bar(1, kEpiThreads);  // uniform decision before the warp-collective TMEM loads
    if (!FINAL && ok && ntiles > 0 && !*abort) {
      tc_fence_after();
      for (int seg = 0; seg < nseg; ++seg) {
        // Q partial of row block rb into slot (this CTA - the block's first owner)
        const int64_t rb = rb0 + seg, gi = rb * TBM + row;
        const int64_t slot = blockIdx.x - tc_tile_owner(rb * T, N, G);
        float q[kEpiCols];
#pragma unroll
        for (int c = 0; c < kEpiCols / 16; ++c)
          tmem_ld16(tmem + lane_base + TM_Q + 64 * seg + cbase + 16 * c, q + 16 * c);
        tmem_ld_wait();
        if (gi < m) {
          float4* dst = reinterpret_cast<float4*>(Qpart + (slot * m + gi) * TR + cbase);
#pragma unroll
          for (int c = 0; c < kEpiCols / 4; ++c)
            dst[c] = make_float4(q[4 * c], q[4 * c + 1], q[4 * c + 2], q[4 * c + 3]);
        }
      }
    }
    if (tid == 0) tma_store_wait0();
    // residual: warp sums, then thread 0 combines the epilogue warps in a fixed order
    for (int o = 16; o > 0; o >>= 1) resid += __shfl_xor_sync(0xffffffffu, resid, o);
    if (lane == 0) B.red[warp] = resid;
    named_bar(1, kEpiThreads);
    if (!FINAL && tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < kEpiWarps; ++w) tot += B.red[w];
      resid_part[blockIdx.x] = tot;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, TM_COLS);
  }
  if (tid == 0 && B.abort) {
    st->status = SFR_E_TIMEOUT;
    st->done = 1;
  }
}

// ---------------------------------------------------------------- W pass: W = X^T U on tensor cores
// CTA: 128 columns j x a chunk of rows i; D (128 x 64 NS) in TMEM.  A = the m x n source (Delta,
// or M on iteration 1 and in Algorithm 4) read row-major as an MN-major operand (M index = column
// j), B = U^T (K-major) as NS bfloat16 terms stacked in 64-row groups (NS = 2 for Algorithm 4:
// U = U_hi + U_lo, so that the product sees U at about 16 bits), summed in the epilogue.
constexpr int WSTAGES = 4;
constexpr uint32_t W_A_BYTES = 16384, W_B_BYTES = 8192;
template <int NS> __host__ __device__ constexpr uint32_t w_stage() { return W_A_BYTES + NS * W_B_BYTES; }
template <int NS> __host__ __device__ constexpr uint32_t w_off_bar() { return WSTAGES * w_stage<NS>(); }
template <int NS> __host__ __device__ constexpr uint32_t wpass_smem() { return w_off_bar<NS>() + 128 + 1024; }

// MN-major operand in the 128-byte swizzle layout: 64-element atoms along M 8 KB apart (LBO),
// 8-row groups along K 1024 bytes apart (SBO)
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(8192 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

struct WBars {
  uint64_t full[WSTAGES], empty[WSTAGES];
  uint64_t acc_full;
  uint32_t tmem_base;
  int abort;
};

template <int NS>
__global__ void __launch_bounds__(192, 1) wpass_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmUt, int64_t m,
                                                          int64_t n, int rows_per_chunk, float* __restrict__ Wpart,
                                                          DevState* st) {
  pdl_enter();
  constexpr uint32_t W_STAGE = w_stage<NS>(), TCOLS = NS == 1 ? 64 : 128;
  if (stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  WBars& B = *reinterpret_cast<WBars*>(sm + w_off_bar<NS>());
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
  if (warp == 5) tmem_alloc(&B.tmem_base, TCOLS);
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
        tma_load_2d(sm + s * W_STAGE, &tmA, j0, r0 + 64 * k, &B.full[s]);
        tma_load_2d(sm + s * W_STAGE + 8192, &tmA, j0 + 64, r0 + 64 * k, &B.full[s]);
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
      const uint32_t id = idesc(1, 128, TR * NS) | (1u << 15);  // A MN-major
      bool ok = true;
      for (int k = 0; k < nk; ++k) {
        const int s = k % WSTAGES;
        if (!mbar_wait(&B.full[s], (k / WSTAGES) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t a = desc_sw128_mn(smem_u32(sm + s * W_STAGE) + kk * 2048);
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
        const uint32_t lb = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int c = 0; c < TR; c += 16) tmem_ld16(tmem + lb + c, w + c);
        if constexpr (NS == 2) {
          float lo[16];
#pragma unroll
          for (int c = 0; c < TR; c += 16) {
            tmem_ld16(tmem + lb + TR + c, lo);
            tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 16; ++q) w[c + q] += lo[q];
          }
        }
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
    tmem_dealloc(tmem, TCOLS);
  }
  if (tid == 0 && B.abort) {
    st->status = SFR_E_TIMEOUT;
    st->done = 1;
  }
}

// ---------------------------------------------------------------- P pass of Algorithm 4: P = M V
// The sweep's persistent partition of (128-row block, 64-column tile) pairs: A = the bfloat16 M
// tile (K-major), B = V^T as two bfloat16 terms V_hi, V_lo stacked into 128 rows, so one N = 128
// MMA per K step forms M V_hi and M V_lo (M is exact in bfloat16, so the sum sees V at about
// 16 bits, below the float32 accumulation error).  Each row-block segment of the CTA
// accumulates in its own 128 TMEM columns over all its tiles; at the end the epilogue adds the
// two halves and writes the Q partial into slot (CTA - first owner of the block), the layout
// thin_gram_kernel sums.  Warps 0-3: epilogue (TMEM lanes = rows); warp 4: TMA producer;
// warp 5: TMEM owner and MMA issuer.
constexpr int PSTAGES = 6;
constexpr uint32_t P_A_BYTES = 16384, P_B_BYTES = 16384, P_STAGE = P_A_BYTES + P_B_BYTES;
constexpr uint32_t P_OFF_BAR = PSTAGES * P_STAGE;
constexpr uint32_t PPASS_SMEM = P_OFF_BAR + 128 + 1024;
static_assert(PPASS_SMEM <= 232448, "shared memory per CTA");

struct PBars {
  uint64_t full[PSTAGES], empty[PSTAGES];
  uint64_t acc_full;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(PBars) <= 128, "barrier block");

__global__ void __launch_bounds__(192, 1) ppass_tc_kernel(const __grid_constant__ CUtensorMap tmM,
                                                          const __grid_constant__ CUtensorMap tmVt, int64_t m,
                                                          int64_t n, float* __restrict__ Qpart, DevState* st) {
  pdl_enter();
  if (stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  PBars& B = *reinterpret_cast<PBars*>(sm + P_OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tiles [x0, x1) of the N (row block, column tile) pairs, at most two row blocks (tc_plan)
  const int64_t T = (n + TBN - 1) / TBN, N = ((m + TBM - 1) / TBM) * T, G = gridDim.x;
  const int64_t x0 = (int64_t)blockIdx.x * N / G, x1 = ((int64_t)blockIdx.x + 1) * N / G;
  const int ntiles = (int)(x1 - x0);
  const int64_t rb0 = x0 / T;
  const int kb = (int)(((rb0 + 1) * T < x1 ? (rb0 + 1) * T : x1) - x0);
  const int nseg = kb < ntiles ? 2 : 1;
  volatile int* abort = &B.abort;
  if (tid == 0) {
    for (int s = 0; s < PSTAGES; ++s) {
      mbar_init(&B.full[s], 1);
      mbar_init(&B.empty[s], 1);
    }
    mbar_init(&B.acc_full, 1);
    B.abort = 0;
    mbar_fence_init();
  }
  if (warp == 5) tmem_alloc(&B.tmem_base, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem_base;
  if (warp == 4) {
    if (lane == 0) {
      prefetch_map(&tmM);
      int armed[PSTAGES];
      for (int q = 0; q < PSTAGES; ++q) armed[q] = -1;
      for (int t = 0; t < ntiles && !*abort; ++t) {
        const int s = t % PSTAGES;
        const int i0 = (int)((rb0 + (t >= kb)) * TBM), j0 = (int)((x0 + t - (rb0 + (t >= kb)) * T) * TBN);
        if (t >= PSTAGES && !mbar_wait(&B.empty[s], ((t / PSTAGES) - 1) & 1, abort)) break;
        mbar_expect_tx(&B.full[s], P_STAGE);
        tma_load_2d(sm + s * P_STAGE, &tmM, j0, i0, &B.full[s]);
        tma_load_2d(sm + s * P_STAGE + P_A_BYTES, &tmVt, j0, 0, &B.full[s]);
        armed[s] = t;
      }
      if (*abort)
        for (int q = 0; q < PSTAGES; ++q)
          if (armed[q] >= 0) {
            int dummy = 0;
            mbar_wait(&B.full[q], (armed[q] / PSTAGES) & 1, &dummy);
          }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t id = idesc(1, TBM, 2 * TR);  // bf16, 128 x 128
      bool ok = true;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % PSTAGES, seg = t >= kb, first = seg ? kb : 0;
        if (!mbar_wait(&B.full[s], (t / PSTAGES) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        for (int kk = 0; kk < TBN / 16; ++kk) {
          const uint64_t a = desc_sw128(smem_u32(sm + s * P_STAGE) + kk * 32);
          const uint64_t b = desc_sw128(smem_u32(sm + s * P_STAGE + P_A_BYTES) + kk * 32);
          mma_bf16(tmem + 2 * TR * seg, a, b, id, (t > first || kk > 0) ? 1u : 0u);
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
    if (ntiles > 0) mbar_wait(&B.acc_full, 0, abort);
    named_bar(1, 128);  // uniform decision before the warp-collective TMEM loads
    if (ntiles > 0 && !*abort) {
      tc_fence_after();
      const uint32_t lb = (uint32_t)(warp * 32) << 16;
      for (int seg = 0; seg < nseg; ++seg) {
        const int64_t rb = rb0 + seg, gi = rb * TBM + warp * 32 + lane;
        const int64_t slot = blockIdx.x - tc_tile_owner(rb * T, N, G);
        for (int c = 0; c < TR; c += 16) {
          float hi[16], lo[16];
          tmem_ld16(tmem + lb + 2 * TR * seg + c, hi);
          tmem_ld16(tmem + lb + 2 * TR * seg + TR + c, lo);
          tmem_ld_wait();
          if (gi < m) {
            float4* dst = reinterpret_cast<float4*>(Qpart + (slot * m + gi) * TR + c);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              dst[q] = make_float4(hi[4 * q] + lo[4 * q], hi[4 * q + 1] + lo[4 * q + 1], hi[4 * q + 2] + lo[4 * q + 2],
                                   hi[4 * q + 3] + lo[4 * q + 3]);
          }
        }
      }
    }
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

void tc_plan(Shape* s, int num_sms) {
  const int64_t R = (s->m + TBM - 1) / TBM, T = (s->n + TBN - 1) / TBN, N = R * T;
  int64_t G = std::min<int64_t>(num_sms, N);
  if (G < R) G = R;  // then every CTA owns at most T tiles, i.e. at most two row blocks
  int slots = 1;
  for (int64_t rb = 0; rb < R; ++rb) slots = std::max(slots, tc_q_slots(rb, T, N, G));
  s->sweep_grid_x = (int)G;
  s->nsplit = slots;
  s->cols_per_split = (int)(T * TBN);
  s->resid_parts = (int)G;
  s->q_ctas = (int)G;
}

bool tc_supported(const Shape& s, int m_dtype, int64_t ldm) {
  return s.rp == 64 && m_dtype == SFR_BF16 && ldm % 8 == 0 && s.n % 8 == 0 && s.m % 8 == 0 && encode_fn() != nullptr;
}

cudaError_t tc_make_full_maps(const Shape& s, const TcBuffers& t, const void* M, int64_t ldm, TcMaps* maps) {
  const auto BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  bool ok = true;
  ok &= make_map(&maps->M, M, BF, s.n, s.m, 2 * ldm, 64, 128);
  ok &= make_map(&maps->M_w, M, BF, s.n, s.m, 2 * ldm, 64, 64);
  ok &= make_map(&maps->Ut2, t.Ut, BF, s.m, 128, 2 * t.ldd, 64, 128);
  ok &= make_map(&maps->Vt2, t.Vt, BF, s.n, 128, 2 * t.ldy, 64, 128);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_make_maps(const Shape& s, const TcBuffers& t, const void* M, int64_t ldm, TcMaps* maps) {
  const auto BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  bool ok = true;
  ok &= make_map(&maps->M, M, BF, s.n, s.m, 2 * ldm, 64, 128);
  ok &= make_map(&maps->M_w, M, BF, s.n, s.m, 2 * ldm, 64, 64);
  for (int q = 0; q < 2; ++q) ok &= make_map(&maps->Y[q], t.Y[q], BF, s.n, s.m, 2 * t.ldy, 64, 128);
  ok &= make_map(&maps->D, t.D, BF, s.n, s.m, 2 * t.ldy, 64, 128);
  ok &= make_map(&maps->D_w, t.D, BF, s.n, s.m, 2 * t.ldy, 64, 64);
  ok &= make_map(&maps->Ut, t.Ut, BF, s.m, 64, 2 * t.ldd, 64, 64);
  ok &= make_map(&maps->Ut2, t.Ut, BF, s.m, 128, 2 * t.ldd, 64, 128);  // P^T as a two-term split
  ok &= make_map(&maps->Ch, t.Ch, F32, 64, s.n, 256, 32, 64);
  ok &= make_map(&maps->Cl, t.Cl, F32, 64, s.n, 256, 32, 64);
  ok &= make_map(&maps->Vt, t.Vt, BF, s.n, 64, 2 * t.ldy, 64, 64);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_launch_wpass(const Shape& s, const TcMaps& mp, bool first, float* Wpart, DevState* dst,
                            cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(wpass_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wpass_smem<1>());
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(s.n, 128), s.nchunk);
  launch_pdl(wpass_tc_kernel<1>, grid, 192, wpass_smem<1>(), st, first ? mp.M_w : mp.D_w, mp.Ut, s.m, s.n, s.rows_per_chunk,
                                                          Wpart, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_wpass_p(const Shape& s, const TcMaps& mp, float* Wpart, DevState* dst, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(wpass_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wpass_smem<2>());
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(s.n, 128), s.nchunk);
  launch_pdl(wpass_tc_kernel<2>, grid, 192, wpass_smem<2>(), st, mp.D_w, mp.Ut2, s.m, s.n, s.rows_per_chunk, Wpart, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_full_wpass(const Shape& s, const TcMaps& mp, float* Wpart, DevState* dst, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(wpass_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wpass_smem<2>());
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(s.n, 128), s.nchunk);
  launch_pdl(wpass_tc_kernel<2>, grid, 192, wpass_smem<2>(), st, mp.M_w, mp.Ut2, s.m, s.n, s.rows_per_chunk, Wpart, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_full_ppass(const Shape& s, const TcMaps& mp, float* Qpart, DevState* dst, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(ppass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PPASS_SMEM);
  if (e != cudaSuccess) return e;
  launch_pdl(ppass_tc_kernel, s.sweep_grid_x, 192, PPASS_SMEM, st, mp.M, mp.Vt2, s.m, s.n, Qpart, dst);
  return cudaGetLastError();
}

cudaError_t tc_launch_sweep(const Shape& s, const TcMaps& mp, const TcBuffers& t, int y_in, float* Qpart,
                            double* resid_part, DevState* dst, cudaStream_t st) {
  auto kern = sweep_tc_kernel<false, float>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
  if (e != cudaSuccess) return e;
  launch_pdl(kern, s.sweep_grid_x, kSweepThreads, SWEEP_SMEM, st, mp.M, mp.Y[y_in], mp.Y[1 - y_in], mp.D, mp.Ch, mp.Cl, mp.Vt,
                                                         t.Uh, t.Ul, s.m, s.n, Qpart, resid_part, dst, nullptr,
                                                         nullptr, 0, 0);
  return cudaGetLastError();
}

cudaError_t tc_launch_finalize(const Shape& s, const TcMaps& mp, const TcBuffers& t, int y_in, void* S,
                               int s_dtype, int64_t lds, void* L, DevState* dst, cudaStream_t st) {
  const size_t es = s_dtype == SFR_F64 ? 8 : 4;
  const bool vec = ((uintptr_t)S % 16 == 0) && ((uintptr_t)L % 16 == 0) && ((size_t)lds * es) % 16 == 0;
  auto go = [&](auto zero) -> cudaError_t {
    using TSo = decltype(zero);
    auto kern = sweep_tc_kernel<true, TSo>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
    if (e != cudaSuccess) return e;
    launch_pdl(kern, s.sweep_grid_x, kSweepThreads, SWEEP_SMEM, st, mp.M, mp.Y[y_in], mp.Y[1 - y_in], mp.D, mp.Ch, mp.Cl,
                                                           mp.Vt, t.Uh, t.Ul, s.m, s.n, nullptr, nullptr, dst,
                                                           static_cast<TSo*>(S), static_cast<TSo*>(L), lds,
                                                           vec ? 1 : 0);
    return cudaGetLastError();
  };
  return s_dtype == SFR_F64 ? go(0.0) : go(0.f);
}

}  // namespace sfr
