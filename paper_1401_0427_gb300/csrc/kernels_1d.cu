// D1Q3Q2 kernels (section 2): populations f0, f+, f- (mass, D1Q3) and g+, g-
// (discharge, D1Q2; h_0^* does not depend on beta, so there is no g0).  One thread
// per cell; five planes of `pitch` elements, post-collision values.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "scheme.cuh"

namespace cg = cooperative_groups;

namespace lbm {
namespace {

// Value of population p (1: f+, 2: f-, 3: g+, 4: g-) streaming into cell i.
template <class T>
__device__ __forceinline__ T pull1(const StepArgs<T>& A, int p, int i) {
  const bool plus = (p == 1 || p == 3);  // moves +lambda: comes from i - 1
  const int is = plus ? i - 1 : i + 1;
  if (is >= 0 && is < A.nx) return A.src[p * A.plane + is];
  const int side = plus ? LBM_SW_SIDE_XM : LBM_SW_SIDE_XP;
  switch (A.bc[side]) {
    case LBM_SW_BC_PERIODIC:
      return A.src[p * A.plane + (plus ? A.nx - 1 : 0)];
    case LBM_SW_BC_WALL: {  // mirror of the boundary cell: f+ <-> f-, g+ <-> -g-
      const int m = (p == 1) ? 2 : (p == 2) ? 1 : (p == 3) ? 4 : 3;
      const T v = A.src[m * A.plane + i];
      return p >= 3 ? -v : v;
    }
    case LBM_SW_BC_OUTFLOW:
      return A.src[p * A.plane + i];
    default:
      return A.inflow_feq[side * 5 + p];
  }
}

template <class T, bool MRT>
__global__ void __launch_bounds__(256) step1d(const StepArgs<T> A, const Consts<T> K) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T f[5];
    f[0] = A.src[i];
#pragma unroll
    for (int p = 1; p < 5; ++p) f[p] = pull1(A, p, i);
    collide5_any<T, MRT>(f, K);
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i] = f[p];
  }
}

// Steps per cluster barrier in step1d_cluster.
constexpr int kCluster1dBlock = 8;

// All n steps of a line of up to 16 * 1024 cells in one launch: one thread-block cluster,
// CTA r owns cells [r * chunk, (r + 1) * chunk) and keeps them in shared memory.  The steps
// go in blocks of up to kCluster1dBlock (KB): at the start of a block a CTA copies its own
// cells and KB cells on each side (from the neighbouring CTAs' shared memory, distributed
// shared memory, wrapping around on periodic sides) into a local window, advances the window
// KB steps on its own, and writes its own cells back.  After step s the window is exact
// except for s cells at each end that is not a physical boundary, which never reaches the
// owned cells.  One cluster barrier per block orders the write-back before the neighbours'
// next reads; the owned copies alternate between two buffers, so a block's writes never
// meet the same block's reads.  Every cell update is the pull + collide of the per-step
// kernel on the same values, so the results are equal bit for bit.
template <class T, bool MRT>
__global__ void __launch_bounds__(1024) step1d_cluster(const StepArgs<T> A, const Consts<T> K, int nsteps,
                                                       int chunk) {
  constexpr int KB = kCluster1dBlock;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wcap = chunk + 2 * KB;  // window capacity
  T* home = reinterpret_cast<T*>(smem_raw);
  T* other = home + 5 * chunk;
  T* const win0 = other + 5 * chunk;
  T* const win1 = win0 + 5 * wcap;
  const int nx = A.nx;
  const int i0 = rank * chunk;
  const int ncell = nx - i0 < chunk ? nx - i0 : chunk;  // <= 0 for idle trailing CTAs
  const bool per = A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC;  // periodic sides come in pairs
  for (int c = threadIdx.x; c < ncell; c += blockDim.x)
#pragma unroll
    for (int p = 0; p < 5; ++p) home[p * chunk + c] = A.src[p * A.plane + i0 + c];
  cluster.sync();
  for (int done = 0; done < nsteps; done += KB) {
    const int kb = nsteps - done < KB ? nsteps - done : KB;
    if (ncell > 0) {
      // the window holds cells [i0 - L, i0 + ncell + R)
      const int L = per ? kb : min(kb, i0);
      const int R = per ? kb : min(kb, nx - i0 - ncell);
      const int wn = L + ncell + R;
      const bool left_end = !per && i0 - L == 0;  // the window starts at the x- side
      const bool right_end = !per && i0 + ncell + R == nx;
      for (int w = threadIdx.x; w < wn; w += blockDim.x) {
        int g = i0 - L + w;
        if (per) {
          g %= nx;
          if (g < 0) g += nx;
        }
        const int r = g / chunk;
        const int c = g - r * chunk;
        const T* src = r == rank ? home : cluster.map_shared_rank(home, r);
#pragma unroll
        for (int p = 0; p < 5; ++p) win0[p * wcap + w] = src[p * chunk + c];
      }
      __syncthreads();
      T* cur = win0;
      T* nxt = win1;
      for (int s = 1; s <= kb; ++s) {
        const int lo = left_end ? 0 : s;
        const int hi = right_end ? wn : wn - s;
        for (int w = lo + threadIdx.x; w < hi; w += blockDim.x) {
          const int g = i0 - L + w;  // the cell (sides that are not periodic)
          T f[5];
          f[0] = cur[w];
#pragma unroll
          for (int p = 1; p < 5; ++p) {
            const bool plus = (p == 1 || p == 3);  // moves +lambda: comes from w - 1
            if (per || (plus ? g > 0 : g < nx - 1)) {
              f[p] = cur[p * wcap + (plus ? w - 1 : w + 1)];
            } else {
              const int side = plus ? LBM_SW_SIDE_XM : LBM_SW_SIDE_XP;
              switch (A.bc[side]) {
                case LBM_SW_BC_WALL: {  // mirror of the boundary cell: f+ <-> f-, g+ <-> -g-
                  const int m = (p == 1) ? 2 : (p == 2) ? 1 : (p == 3) ? 4 : 3;
                  const T v = cur[m * wcap + w];
                  f[p] = p >= 3 ? -v : v;
                  break;
                }
                case LBM_SW_BC_OUTFLOW:
                  f[p] = cur[p * wcap + w];
                  break;
                default:
                  f[p] = A.inflow_feq[side * 5 + p];
              }
            }
          }
          collide5_any<T, MRT>(f, K);
#pragma unroll
          for (int p = 0; p < 5; ++p) nxt[p * wcap + w] = f[p];
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
      }
      for (int c = threadIdx.x; c < ncell; c += blockDim.x)
#pragma unroll
        for (int p = 0; p < 5; ++p) other[p * chunk + c] = cur[p * wcap + L + c];
    }
    cluster.sync();
    T* t = home;
    home = other;
    other = t;
  }
  for (int c = threadIdx.x; c < ncell; c += blockDim.x)
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i0 + c] = home[p * chunk + c];
}

// Dynamic shared memory of step1d_cluster at `chunk` cells per CTA.
template <class T>
size_t cluster1d_smem(int chunk) {
  return (2 * 5 * static_cast<size_t>(chunk) + 2 * 5 * static_cast<size_t>(chunk + 2 * kCluster1dBlock)) * sizeof(T);
}

template <class T>
__global__ void init1d(const StepArgs<T> A, const Consts<T> K, const double* __restrict__ h,
                       const double* __restrict__ hu) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T e[5];
    equilibrium5(static_cast<T>(h[i]), static_cast<T>(hu[i]), K, e);
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i] = e[p];
  }
}

template <class T, bool MRT>
__global__ void collide1d_dense(const StepArgs<T> A, const Consts<T> K, const T* __restrict__ dense) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T f[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) f[p] = dense[p * static_cast<long long>(A.nx) + i];
    collide5_any<T, MRT>(f, K);
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i] = f[p];
  }
}

template <class T>
__global__ void moments1d(const StepArgs<T> A, double* __restrict__ h, double* __restrict__ hu) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T f[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) f[p] = A.src[p * A.plane + i];
    T d, q;
    moments5(f, d, q);
    h[i] = static_cast<double>(d);
    hu[i] = static_cast<double>(q);
  }
}

struct InflowStates1 {
  int bc[2];
  double w[2][2];
};

template <class T>
__global__ void inflow_feq1d(T* out, const InflowStates1 in, const Consts<T> K) {
  const int side = threadIdx.x;
  if (side >= 4) return;
  T e[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (side < 2 && in.bc[side] == LBM_SW_BC_INFLOW)
    equilibrium5(static_cast<T>(in.w[side][0]), static_cast<T>(in.w[side][1]), K, e);
#pragma unroll
  for (int p = 0; p < 5; ++p) out[side * 5 + p] = e[p];
}

unsigned blocks_for(int n, int threads) {
  const long long b = (static_cast<long long>(n) + threads - 1) / threads;
  return static_cast<unsigned>(b < 65535 ? b : 65535);
}

}  // namespace

template <class T>
Consts<T> consts1(const ConstsD& kd) {
  return kd.mrt ? make_consts_mrt<T>(kd.g, kd.lambda, kd.s, kd.a, kd.rates, 3) : make_consts<T>(kd.g, kd.lambda, kd.s, kd.a);
}

template <class T>
cudaError_t launch_step1d(const StepArgs<T>& a, const ConstsD& kd, cudaStream_t st) {
  if (kd.mrt)
    step1d<T, true><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, consts1<T>(kd));
  else
    step1d<T, false><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, consts1<T>(kd));
  return cudaGetLastError();
}

// CTAs of the largest cluster the device places for step1d_cluster: 16 where it allows
// that non-portable size with the shared memory of 1024-cell chunks, else the portable 8.
template <class T>
int cluster1d_probe_blocks() {
  int blocks = 8;
  if (cudaFuncSetAttribute(step1d_cluster<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(step1d_cluster<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(cluster1d_smem<T>(1024))) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = cluster1d_smem<T>(1024);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 16;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, step1d_cluster<T, false>, &cfg) == cudaSuccess && clusters > 0)
      blocks = 16;
  }
  cudaGetLastError();  // a refused attribute or probe leaves no error behind
  return blocks;
}

template <class T>
int cluster1d_max_cells() {
  static const int max_blocks = cluster1d_probe_blocks<T>();  // probed once (thread-safe initialisation)
  return max_blocks * 1024;
}

template <class T, bool MRT>
cudaError_t launch_cluster_t(const StepArgs<T>& a, const ConstsD& kd, int nsteps, cudaStream_t st) {
  const int max_cells = cluster1d_max_cells<T>();
  const int max_blocks = max_cells / 1024;
  int blocks = (a.nx + 63) / 64;  // at least 64 cells per CTA
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  const int chunk = (a.nx + blocks - 1) / blocks;
  const int window = chunk + 2 * kCluster1dBlock;
  const int threads = window < 1024 ? ((window + 31) / 32) * 32 : 1024;
  const size_t smem = cluster1d_smem<T>(chunk);
  cudaError_t e = cudaFuncSetAttribute(step1d_cluster<T, MRT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(cluster1d_smem<T>(1024)));
  if (e != cudaSuccess) return e;
  if (blocks > 8) {
    e = cudaFuncSetAttribute(step1d_cluster<T, MRT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = blocks;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step1d_cluster<T, MRT>, a, consts1<T>(kd), nsteps, chunk);
}

template <class T>
cudaError_t launch_step1d_cluster(const StepArgs<T>& a, const ConstsD& kd, int nsteps, cudaStream_t st) {
  return kd.mrt ? launch_cluster_t<T, true>(a, kd, nsteps, st) : launch_cluster_t<T, false>(a, kd, nsteps, st);
}

template <class T>
cudaError_t launch_init1d(const StepArgs<T>& a, const ConstsD& kd, const double* h, const double* hu,
                          cudaStream_t st) {
  init1d<T><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a), h, hu);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_collide1d_dense(const StepArgs<T>& a, const ConstsD& kd, const T* dense, cudaStream_t st) {
  if (kd.mrt)
    collide1d_dense<T, true><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, consts1<T>(kd), dense);
  else
    collide1d_dense<T, false><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, consts1<T>(kd), dense);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_moments1d(const StepArgs<T>& a, double* h, double* hu, cudaStream_t st) {
  moments1d<T><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, h, hu);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_inflow_feq1d(T* out, const int bc[4], const double inflow[4][3], const ConstsD& kd,
                                cudaStream_t st) {
  InflowStates1 in;
  for (int s = 0; s < 2; ++s) {
    in.bc[s] = bc[s];
    in.w[s][0] = inflow[s][0];
    in.w[s][1] = inflow[s][1];
  }
  inflow_feq1d<T><<<1, 32, 0, st>>>(out, in, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a));
  return cudaGetLastError();
}

#define LBM_INSTANTIATE_1D(T)                                                                               \
  template cudaError_t launch_step1d<T>(const StepArgs<T>&, const ConstsD&, cudaStream_t);                 \
  template int cluster1d_max_cells<T>();                                                                    \
  template cudaError_t launch_step1d_cluster<T>(const StepArgs<T>&, const ConstsD&, int, cudaStream_t);    \
  template cudaError_t launch_init1d<T>(const StepArgs<T>&, const ConstsD&, const double*, const double*,   \
                                        cudaStream_t);                                                      \
  template cudaError_t launch_collide1d_dense<T>(const StepArgs<T>&, const ConstsD&, const T*, cudaStream_t); \
  template cudaError_t launch_moments1d<T>(const StepArgs<T>&, double*, double*, cudaStream_t);             \
  template cudaError_t launch_inflow_feq1d<T>(T*, const int[4], const double[4][3], const ConstsD&, cudaStream_t);

LBM_INSTANTIATE_1D(float)
LBM_INSTANTIATE_1D(double)

}  // namespace lbm
