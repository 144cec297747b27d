// Shared pieces of the temporal-blocking kernels (temporal.cu, adjoint_temporal.cu): the
// work partition of a launch and the shared-memory shape of the one-column periodic
// wavefront.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

namespace lbm {
namespace {

// Programmatic dependent launch: a kernel launched by launch_pdl may have its CTAs placed
// while the previous grid in the stream still runs.  It calls pdl_wait() before it touches
// memory (the previous grid has then completed and its writes are visible, so neither its
// output nor its input is used early) and pdl_done() when its own work is done.  Without
// the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_done() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// All-periodic domains.  Row R of level t - 1 feeds level t in three ways: its -y movers
// (planes 4, 8, 12) to row R - 1, f0 and the x movers to row R, its +y movers (2, 6, 10)
// to row R + 1.  Only the x movers cross columns, so for t - 1 >= 1 only they go through
// shared memory (two rows: the one read now and the one being written); the others stay
// in the registers of the column's thread.  Level 0 arrives by cp.async into a ring per
// plane group that holds each group as long as it is read: the -y movers 3 rows (the row
// read now plus two in flight), f0 and the x movers 4, the +y movers 5.
template <int K, int COLS>
struct PeriodicShape {
  static constexpr int A0 = 3, B0 = 4, C0 = 5;
  static constexpr int L0_FLOATS = COLS * (3 * A0 + 7 * B0 + 3 * C0);
  static constexpr int LV_FLOATS = COLS * 2 * 6;
  static constexpr size_t floats() { return static_cast<size_t>(L0_FLOATS) + (K - 1) * LV_FLOATS; }
};

// Work of one launch: the domain is cut into `strips` column strips of width w (the last
// one narrower) and each strip into `segments` row segments.  CTA b takes segment
// b / strips of strip b % strips, so the CTAs resident together work on the same rows of
// neighbouring strips and share the strips' halo columns in L2.
struct Partition {
  int w;             // output columns per strip (every strip but the last is exactly w wide)
  int strips;        // ceil(nx / w)
  int rows_per_cta;  // output rows per segment (the last segment may be shorter)
  int segments;      // row segments per strip
};

template <class F>
__device__ __forceinline__ void run_segment(const Partition& P, int ny, F&& segment) {
  const int strip = static_cast<int>(blockIdx.x % P.strips);
  const int ys = static_cast<int>(blockIdx.x / P.strips) * P.rows_per_cta;
  if (ys < ny) segment(strip, ys, min(ny, ys + P.rows_per_cta));
}

// Resident CTAs per SM of a kernel at its dynamic shared-memory size.
inline int resident_ctas(const void* fn, int threads, size_t smem) {
  int r = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fn, threads, smem) != cudaSuccess) return 1;
  return std::max(r, 1);
}

// The same, asked once per kernel and device.
inline int cached_resident(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return resident_ctas(fn, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, fn});
  if (it != cache.end()) return it->second;
  const int v = resident_ctas(fn, threads, smem);
  cache[{dev, fn}] = v;
  return v;
}

// Strips of equal width <= wmax, then row segments: about `waves` waves of the resident
// CTAs (`slots` of them), rounded down to whole segments per strip, no segment shorter
// than 2K rows (the wavefront's fill) unless the domain is.
inline Partition partition_rows(Partition P, int ny, int K, int slots, int waves) {
  const int min_rows = std::min(2 * K, ny);
  int seg = std::max(1, (waves * slots) / P.strips);
  seg = std::min(seg, std::max(1, ny / min_rows));
  P.rows_per_cta = (ny + seg - 1) / seg;
  P.segments = (ny + P.rows_per_cta - 1) / P.rows_per_cta;
  return P;
}

inline Partition partition(int nx, int ny, int wmax, int K, int slots, int waves) {
  Partition P;
  P.strips = (nx + wmax - 1) / wmax;
  P.w = (nx + P.strips - 1) / P.strips;
  return partition_rows(P, ny, K, slots, waves);
}

// Strips and row segments of the paired wavefront (COLS tile columns, K steps): strips of an
// even width of at most COLS - K - KL columns, KL = K rounded up to even being the left halo
// (K + 1 columns at odd K), so that every tile starts at an even column and its K + w + KL
// columns fit the COLS of the CTA; row segments for one wave of `slots` CTAs.
inline Partition pair_partition(int nx, int ny, int K, int COLS, int slots) {
  Partition P = partition(nx, ny, (COLS - 2 * K - (K & 1)) & ~1, K, slots, 1);
  P.w += P.w & 1;  // even strip width (the bound above is even)
  P.strips = (nx + P.w - 1) / P.w;
  return partition_rows(P, ny, K, slots, 1);
}

}  // namespace
}  // namespace lbm
