// Host-side checks of the launch planner and the workspace layout (no GPU needed).
//
// For a spread of problem sizes -- square and rectangular, ragged and tile-aligned, tall-skinny
// and short-wide -- and several SM counts this checks the properties the kernels rely on:
//   * the persistent tensor-core sweep's contiguous tile ranges cover every (128-row block,
//     64-column tile) pair once and span at most two row blocks per CTA, and the Delta V
//     partial slots of each row block are written by exactly one CTA each and are all summed
//     by the thin kernel (tc_q_slots), with no more slots than the buffer holds (nsplit);
//   * the SIMT sweep's column splits and the W pass's row chunks cover the matrix without an
//     empty split or chunk, chunks being whole multiples of 64 rows;
//   * every workspace buffer is 256-byte aligned, inside the carved block, and the multiplier
//     and Delta buffers of the tensor-core path do not overlap each other.
// Prints "ok" and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "../paper_1503_03004_gb300/csrc/sfr_internal.h"
#include "../paper_1503_03004_gb300/csrc/tc_sweep.h"

using namespace sfr;

static int fails = 0;
#define CHECK(cond, ...)                          \
  do {                                            \
    if (!(cond)) {                                \
      if (fails++ < 10) {                         \
        std::printf("FAIL %s: ", #cond);          \
        std::printf(__VA_ARGS__);                 \
        std::printf("\n");                        \
      }                                           \
    }                                             \
  } while (0)

static void check_tc(int64_t m, int64_t n, int sms) {
  Shape s = plan_shape(m, n, n, 64, sms);
  tc_plan(&s, sms);
  const int64_t R = (m + 127) / 128, T = (n + 63) / 64, N = R * T, G = s.sweep_grid_x;
  CHECK(G >= 1 && G <= N && (G <= sms || G == R), "m %lld n %lld G %lld", (long long)m, (long long)n, (long long)G);
  CHECK(s.resid_parts == G && s.q_ctas == G, "m %lld n %lld", (long long)m, (long long)n);
  // writers[rb][slot] = how many CTAs write that Delta V slot
  std::vector<std::vector<int>> writers(R);
  for (int64_t rb = 0; rb < R; ++rb) {
    const int slots = tc_q_slots(rb, T, N, G);
    CHECK(slots >= 1 && slots <= s.nsplit, "m %lld n %lld rb %lld slots %d nsplit %d", (long long)m, (long long)n,
          (long long)rb, slots, s.nsplit);
    writers[rb].assign(slots > 0 ? slots : 1, 0);
  }
  int64_t covered = 0, prev_end = 0;
  for (int64_t c = 0; c < G; ++c) {
    const int64_t x0 = c * N / G, x1 = (c + 1) * N / G;
    CHECK(x0 == prev_end && x1 >= x0, "m %lld n %lld cta %lld", (long long)m, (long long)n, (long long)c);
    prev_end = x1;
    covered += x1 - x0;
    if (x1 == x0) continue;
    CHECK(x1 - x0 <= T, "m %lld n %lld cta %lld spans %lld tiles > T %lld", (long long)m, (long long)n, (long long)c,
          (long long)(x1 - x0), (long long)T);
    // the kernel's segments: row block rb0 for local tiles [0, kb), rb0 + 1 for the rest
    const int64_t rb0 = x0 / T;
    const int64_t kb = ((rb0 + 1) * T < x1 ? (rb0 + 1) * T : x1) - x0;
    const int nseg = kb < x1 - x0 ? 2 : 1;
    for (int64_t k = 0; k < x1 - x0; ++k) {  // each local tile lies in its segment's row block
      const int64_t x = x0 + k, rb = rb0 + (k >= kb);
      CHECK(x / T == rb, "m %lld n %lld cta %lld tile %lld", (long long)m, (long long)n, (long long)c, (long long)k);
      CHECK(tc_tile_owner(x, N, G) == c, "owner of tile %lld", (long long)x);
    }
    for (int seg = 0; seg < nseg; ++seg) {
      const int64_t rb = rb0 + seg;
      const int64_t slot = c - tc_tile_owner(rb * T, N, G);
      CHECK(rb < R && slot >= 0 && slot < (int64_t)writers[rb].size(), "m %lld n %lld cta %lld seg %d slot %lld",
            (long long)m, (long long)n, (long long)c, seg, (long long)slot);
      if (rb < R && slot >= 0 && slot < (int64_t)writers[rb].size()) writers[rb][slot] += 1;
    }
  }
  CHECK(covered == N && prev_end == N, "m %lld n %lld covered %lld of %lld", (long long)m, (long long)n,
        (long long)covered, (long long)N);
  for (int64_t rb = 0; rb < R; ++rb)
    for (size_t k = 0; k < writers[rb].size(); ++k)
      CHECK(writers[rb][k] == 1, "m %lld n %lld rb %lld slot %zu written %d times", (long long)m, (long long)n,
            (long long)rb, k, writers[rb][k]);

  // workspace of the tensor-core path: aligned, inside the block, Y_k / Y_{k+1} / Delta disjoint
  const uintptr_t base = uintptr_t(1) << 40;
  Buffers b{};
  const size_t total = carve(s, false, reinterpret_cast<void*>(base), &b, true);
  const size_t ybytes = 2 * (size_t)m * (size_t)b.t.ldy;
  const uintptr_t y0 = (uintptr_t)b.t.Y[0], y1 = (uintptr_t)b.t.Y[1], d = (uintptr_t)b.t.D;
  CHECK(b.t.ldy >= n && b.t.ldy % 64 == 0 && b.t.ldd >= m && b.t.ldd % 64 == 0, "ld");
  CHECK(y1 >= y0 + ybytes && d >= y1 + ybytes, "m %lld n %lld: Y / Delta overlap", (long long)m, (long long)n);
  const void* ptrs[] = {b.t.Y[0], b.t.Y[1], b.t.D, b.t.Uh, b.t.Ul, b.t.Ch, b.t.Cl, b.t.Ut, b.t.Vt, b.P, b.U[0], b.U[1],
                        b.W, b.V, b.C, b.Qpart, b.Wpart, b.GPpart, b.GWpart, b.Hpart, b.Gsum, b.resid_part,
                        b.normm_part, b.B, b.Bprev, b.TU, b.TV, b.TCm, b.Qeig_u, b.Qeig_v, b.st};
  uintptr_t last = 0;
  for (const void* p : ptrs) {
    const uintptr_t a = (uintptr_t)p;
    CHECK(a % 256 == 0 && a >= base && a < base + total && a > last, "m %lld n %lld buffer at +%llu",
          (long long)m, (long long)n, (unsigned long long)(a - base));
    last = a;
  }
}

static void check_simt(int64_t m, int64_t n, int r, int sms) {
  const Shape s = plan_shape(m, n, n, r, sms);
  CHECK(s.rp >= r && s.rp <= 64, "rp");
  CHECK(s.cols_per_split % 64 == 0 && (int64_t)s.nsplit * s.cols_per_split >= n &&
            (int64_t)(s.nsplit - 1) * s.cols_per_split < n,
        "m %lld n %lld r %d: splits %d x %d", (long long)m, (long long)n, r, s.nsplit, s.cols_per_split);
  CHECK(s.rows_per_chunk % 64 == 0 && (int64_t)s.nchunk * s.rows_per_chunk >= m &&
            (int64_t)(s.nchunk - 1) * s.rows_per_chunk < m,
        "m %lld n %lld r %d: chunks %d x %d", (long long)m, (long long)n, r, s.nchunk, s.rows_per_chunk);
  CHECK(s.gp_blocks >= 1 && s.gp_blocks <= (m + 63) / 64 && s.gw_blocks >= 1 && s.gw_blocks <= (n + 63) / 64,
        "m %lld n %lld r %d: thin CTAs %d %d", (long long)m, (long long)n, r, s.gp_blocks, s.gw_blocks);
  for (int fp64 = 0; fp64 < 2; ++fp64) {
    const uintptr_t base = uintptr_t(1) << 40;
    Buffers b{};
    const size_t total = carve(s, fp64 != 0, reinterpret_cast<void*>(base), &b);
    const size_t es = fp64 ? 8 : 4;
    const size_t ybytes = es * (size_t)m * (size_t)b.ldy;
    CHECK(b.ldy >= n, "ldy");
    CHECK((uintptr_t)b.Y[1] >= (uintptr_t)b.Y[0] + ybytes && (uintptr_t)b.D >= (uintptr_t)b.Y[1] + ybytes,
          "m %lld n %lld r %d: Y / Delta overlap", (long long)m, (long long)n, r);
    CHECK((uintptr_t)b.st + sizeof(DevState) <= base + total, "state outside the block");
  }
}

int main() {
  const int64_t sizes[] = {8, 64, 120, 128, 136, 500, 512, 520, 1000, 1024, 2048, 2056, 4096, 8192, 16384, 32768};
  for (int sms : {152, 148, 132, 8})
    for (int64_t m : sizes)
      for (int64_t n : sizes) {
        if (m % 8 == 0 && n % 8 == 0) check_tc(m, n, sms);
        for (int r : {3, 20, 25, 64})
          if (r <= m && r <= n) check_simt(m, n, r, sms);
      }
  for (int64_t m : {int64_t(1) << 20, int64_t(1) << 16})
    for (int64_t n : {int64_t(40), int64_t(2048)}) {
      check_simt(m, n, 3, 152);
      check_tc(m, n, 152);
    }
  if (fails) {
    std::printf("%d violations\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
