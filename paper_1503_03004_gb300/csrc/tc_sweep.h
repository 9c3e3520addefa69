// Tensor-core (tcgen05 + TMA) passes of the mixed path: buffers, tensor maps, launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfr {

struct Shape;
struct DevState;

// Extra device buffers of the tensor-core path (bfloat16 multiplier, transposed Delta, and the
// split / transposed thin factors the MMAs read).
struct TcBuffers {
  void* Y[2];          // multiplier ping-pong, m x ldy bfloat16
  int64_t ldy;         // n rounded up to 64
  void* D;             // Delta, m x ldy bfloat16
  int64_t ldd;         // m rounded up to 64 (leading dimension of U^T)
  float* Uh;           // m x 64: U rounded to TF32
  float* Ul;           // m x 64: U - Uh
  void* Ut;            // 128 x ldd bfloat16, the B operand of the W pass: U_1^T in rows 0-63 for
                       // FR-ADM's first W pass, then P^T as a two-term split (rows 64-127 hold the
                       // bfloat16 rounding of P^T - rows 0-63); Algorithm 4: the same split of U^T
  float* Ch;           // n x 64: C rounded to TF32
  float* Cl;           // n x 64: C - Ch
  void* Vt;            // 128 x ldy bfloat16: V^T in rows 0-63 (Algorithm 4: plus its low part)
};

struct TcMaps {
  CUtensorMap M, M_w, Y[2], D, D_w, Ut, Ch, Cl, Vt;  // *_w: 64 x 64 boxes for the W pass
  CUtensorMap Ut2, Vt2;  // two-term splits, 64 x 128 boxes (FR-ADM: P^T in Ut; Algorithm 4: U^T, V^T)
};

bool tc_supported(const Shape& s, int m_dtype, int64_t ldm);
// Persistent sweep partition over the SMs: sets the sweep grid, the Q partial slots (nsplit),
// the residual partial count and q_ctas.
void tc_plan(Shape* s, int num_sms);
cudaError_t tc_make_maps(const Shape& s, const TcBuffers& t, const void* M, int64_t ldm, TcMaps* maps);
cudaError_t tc_launch_wpass(const Shape& s, const TcMaps& mp, bool first, float* Wpart, DevState* dst,
                            cudaStream_t st);
cudaError_t tc_launch_sweep(const Shape& s, const TcMaps& mp, const TcBuffers& t, int y_in, float* Qpart,
                            double* resid_part, DevState* dst, cudaStream_t st);
// Algorithm 4 (FixedRankOptFull) on a fixed bfloat16 M: the maps of M and of the split U^T, V^T;
// P = M V partials (persistent partition of tc_plan, Q-partial layout of the sweep) and
// W = M^T U partials (the W pass with the two-term split of U).
cudaError_t tc_make_full_maps(const Shape& s, const TcBuffers& t, const void* M, int64_t ldm, TcMaps* maps);
cudaError_t tc_launch_full_ppass(const Shape& s, const TcMaps& mp, float* Qpart, DevState* dst, cudaStream_t st);
// W pass partials Delta^T P from the two-term bfloat16 split of P^T (W = Delta^T P T_U + C H).
cudaError_t tc_launch_wpass_p(const Shape& s, const TcMaps& mp, float* Wpart, DevState* dst, cudaStream_t st);
cudaError_t tc_launch_full_wpass(const Shape& s, const TcMaps& mp, float* Wpart, DevState* dst, cudaStream_t st);
// S = P_ST_{1/mu}(M - L + Y / mu) (and L when non-null) from the last iteration's factors, mu
// and multiplier Y = t.Y[y_in]; S / L are m x n with leading dimension lds, float64 when
// s_dtype == SFR_F64 else float32.
cudaError_t tc_launch_finalize(const Shape& s, const TcMaps& mp, const TcBuffers& t, int y_in, void* S,
                               int s_dtype, int64_t lds, void* L, DevState* dst, cudaStream_t st);

}  // namespace sfr
