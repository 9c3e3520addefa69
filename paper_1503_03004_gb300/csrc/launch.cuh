// Kernel launch plumbing for the kernels of an FR-ADM iteration.
//
// A kernel is written as a device-function body whose first parameter is its block
// coordinates (VGrid) and which names them blockIdx / gridDim as usual (SFR_VGRID shadows the
// built-ins).  The same body then runs
//   * on its own: body_kernel<Body, NT> fills VGrid from the built-ins;
//   * for many problems in one launch: grouped_kernel<Body, NT> reads a table of per-problem
//     entries (the problem's own grid and its arguments), maps (blockIdx.x, blockIdx.y) to
//     (local block, problem) and calls the body with that problem's grid and arguments, so
//     every problem computes exactly what its own launch would.
// launch_k launches a body on its own, or, while a LaunchRecorder is installed on the calling
// thread, records the launch instead (kernel identity, grid, shared memory, argument bytes) so
// that a serving engine can merge the launches of many problems into grouped launches.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <utility>
#include <vector>

namespace sfr {

struct VGrid {
  uint3 idx;
  dim3 dim;
};

// Inside a kernel body: blockIdx / gridDim of the body (shadowing the built-ins).
#define SFR_VGRID(vg)                \
  const uint3 blockIdx = (vg).idx;   \
  const dim3 gridDim = (vg).dim;     \
  (void)blockIdx;                    \
  (void)gridDim

template <auto Body, int NT, typename... T>
__global__ void __launch_bounds__(NT) body_kernel(T... a) {
  Body(VGrid{blockIdx, gridDim}, a...);
}

// One value of each type, laid out identically on host and device.
template <typename... T> struct Pack;
template <> struct Pack<> {};
template <typename H, typename... T> struct Pack<H, T...> {
  H head;
  Pack<T...> tail;
};

template <typename... T> struct PackMaker;
template <> struct PackMaker<> {
  static Pack<> make() { return {}; }
};
template <typename H, typename... T> struct PackMaker<H, T...> {
  static Pack<H, T...> make(H h, T... t) { return Pack<H, T...>{h, PackMaker<T...>::make(t...)}; }
};
template <typename... T>
Pack<T...> make_pack(T... v) {
  return PackMaker<T...>::make(v...);
}

template <size_t I, typename H, typename... T>
__device__ __forceinline__ const auto& pget(const Pack<H, T...>& p) {
  if constexpr (I == 0) return p.head;
  else return pget<I - 1>(p.tail);
}

template <auto Body, typename... T, size_t... I>
__device__ __forceinline__ void call_body(const VGrid& g, const Pack<T...>& p, std::index_sequence<I...>) {
  Body(g, pget<I>(p)...);
}

// One problem of a grouped launch: its grid (x, y) and its arguments.
template <typename... T> struct GroupEntry {
  uint2 grid;
  Pack<T...> args;
};

// The CTAs of all problems are numbered consecutively: problem p owns blocks
// [starts[p], starts[p + 1]).  The first warp finds p (starts ascending, count small), then the
// body runs with the problem's own grid and arguments.
template <auto Body, int NT, typename... T>
__global__ void __launch_bounds__(NT) grouped_kernel(const int* __restrict__ starts,
                                                     const GroupEntry<T...>* __restrict__ tab, int count) {
  // the table was copied in after the previous kernel: wait for it as every body waits for its inputs
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ int s_prob;
  const int bid = (int)blockIdx.x;
  if (threadIdx.x < 32) {
    int best = -1;
    for (int i = threadIdx.x; i < count; i += 32)
      if (starts[i] <= bid) best = i;
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) s_prob = best;
  }
  __syncthreads();
  const int p = s_prob;
  const GroupEntry<T...>& e = tab[p];
  const uint2 g = e.grid;
  const unsigned local = (unsigned)(bid - starts[p]);
  const VGrid vg{make_uint3(local % g.x, local / g.x, 0u), dim3(g.x, g.y, 1)};
  call_body<Body>(vg, e.args, std::index_sequence_for<T...>{});
}

// A launch captured by the recorder.
struct RecordedLaunch {
  const void* kind;                 // identifies the body and its launch bounds
  unsigned block;                   // threads per CTA
  size_t smem;                      // dynamic shared memory
  dim3 grid;                        // the problem's own grid
  size_t entry_size;                // sizeof(GroupEntry<...>)
  std::vector<unsigned char> entry; // the problem's GroupEntry bytes
  // launches `count` entries (device memory: starts[count + 1] block offsets, then the entries)
  // as one grouped kernel of starts[count] CTAs
  cudaError_t (*launch_grouped)(const int* starts, const void* entries, int count, unsigned total, unsigned block,
                                size_t smem, cudaStream_t st);
};

struct LaunchRecorder {
  std::vector<RecordedLaunch> recs;
};

// While non-null, launch_k records into this recorder instead of launching (per host thread).
inline thread_local LaunchRecorder* g_recorder = nullptr;

// Static shared memory of a kernel, queried once.
template <auto Kern>
size_t static_smem() {
  static const size_t v = [] {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(Kern)) == cudaSuccess) return fa.sharedSizeBytes;
    cudaGetLastError();
    return size_t(0);
  }();
  return v;
}

// The highest stream priority of the device (queried once).
inline int top_priority() {
  static const int v = [] {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return greatest;
  }();
  return v;
}

// Opts the kernel in to `smem` bytes of dynamic shared memory where static + dynamic exceed the
// default 48 KB (a grouped kernel adds a few bytes of its own to the body's static use).
template <auto Kern>
cudaError_t set_smem_attr(size_t smem) {
  if (smem == 0 || smem + static_smem<Kern>() <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(Kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <typename F> struct BodyTraits;
template <typename... T> struct BodyTraits<void (*)(const VGrid&, T...)> {
  template <auto Body, int NT>
  static constexpr auto kernel() {
    return &body_kernel<Body, NT, T...>;
  }
  template <auto Body, int NT, typename... A>
  static cudaError_t launch(dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... a) {
    static_assert(sizeof...(A) == sizeof...(T), "argument count of a kernel body");
    if (g_recorder) {
      RecordedLaunch r;
      r.kind = reinterpret_cast<const void*>(&grouped_kernel<Body, NT, T...>);
      r.block = block.x;
      r.smem = smem;
      r.grid = grid;
      GroupEntry<T...> e{make_uint2(grid.x, grid.y), make_pack<T...>(static_cast<T>(a)...)};
      r.entry_size = sizeof(e);
      r.entry.resize(sizeof(e));
      std::memcpy(r.entry.data(), &e, sizeof(e));
      r.launch_grouped = &launch_grouped<Body, NT>;
      g_recorder->recs.push_back(std::move(r));
      return cudaSuccess;
    }
    auto k = body_kernel<Body, NT, T...>;
    cudaError_t e = set_smem_attr<&body_kernel<Body, NT, T...>>(smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k, grid, block, smem, st, static_cast<T>(a)...);
  }
  // As launch, but as a thread-block cluster of `cluster` CTAs (grid = cluster); recorded as a
  // single-CTA launch (the body must give the same result for any cluster size).
  template <auto Body, int NT, typename... A>
  static cudaError_t launch_cluster(unsigned cluster, dim3 block, size_t smem, cudaStream_t st, A... a) {
    if (g_recorder) return launch<Body, NT>(dim3(1), block, smem, st, a...);
    auto k = body_kernel<Body, NT, T...>;
    cudaError_t e = set_smem_attr<&body_kernel<Body, NT, T...>>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[3];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see pdl_enter
    at[1].val.programmaticStreamSerializationAllowed = 1;
    // the highest scheduling priority: a cluster needs a group of free SMs at once, which
    // kernels of other streams would otherwise take as they free up
    at[2].id = cudaLaunchAttributePriority;
    at[2].val.priority = top_priority();
    cfg.attrs = at;
    cfg.numAttrs = 3;
    return cudaLaunchKernelEx(&cfg, k, static_cast<T>(a)...);
  }
  template <auto Body, int NT>
  static cudaError_t launch_grouped(const int* starts, const void* entries, int count, unsigned total, unsigned block,
                                    size_t smem, cudaStream_t st) {
    auto k = grouped_kernel<Body, NT, T...>;
    cudaError_t e = set_smem_attr<&grouped_kernel<Body, NT, T...>>(smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k, dim3(total), dim3(block), smem, st, starts, static_cast<const GroupEntry<T...>*>(entries),
                      count);
  }
};

template <auto Body, int NT, typename... A>
cudaError_t launch_k_cluster(unsigned cluster, dim3 block, size_t smem, cudaStream_t st, A... a) {
  return BodyTraits<decltype(Body)>::template launch_cluster<Body, NT>(cluster, block, smem, st, a...);
}

// The single-CTA kernel a body runs as (for occupancy and attribute queries).
template <auto Body, int NT>
constexpr auto body_kernel_of() {
  return BodyTraits<decltype(Body)>::template kernel<Body, NT>();
}

// A body as a value (to hand a body choice to a generic lambda).
template <auto F> struct BodyTag {
  static constexpr auto value = F;
};

// Body<<<grid, block, smem, st>>>(a...) with programmatic dependent launch, or recorded.
template <auto Body, int NT, typename... A>
cudaError_t launch_k(dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... a) {
  return BodyTraits<decltype(Body)>::template launch<Body, NT>(grid, block, smem, st, a...);
}

}  // namespace sfr
