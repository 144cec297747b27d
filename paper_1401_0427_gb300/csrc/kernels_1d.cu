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

// All n steps of a line of up to 16 * 1024 cells in one launch: one thread-block cluster,
// CTA r holds cells [r * chunk, (r + 1) * chunk) in shared memory (two buffers of five
// planes); the cells next to a CTA's ends are read from the neighbouring CTAs' shared
// memory (distributed shared memory), and one cluster barrier per step separates the
// reads of one buffer from the writes of the next step.
template <class T, bool MRT>
__global__ void __launch_bounds__(1024) step1d_cluster(const StepArgs<T> A, const Consts<T> K, int nsteps,
                                                       int chunk) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf0 = reinterpret_cast<T*>(smem_raw);
  T* buf1 = buf0 + 5 * chunk;
  const int nx = A.nx;
  const int i0 = rank * chunk;
  const int ncell = nx - i0 < chunk ? nx - i0 : chunk;  // <= 0 for idle trailing CTAs
  for (int c = threadIdx.x; c < ncell; c += blockDim.x)
#pragma unroll
    for (int p = 0; p < 5; ++p) buf0[p * chunk + c] = A.src[p * A.plane + i0 + c];
  const int last_rank = (nx - 1) / chunk, last_c = (nx - 1) - last_rank * chunk;
  cluster.sync();
  T* cur = buf0;
  T* nxt = buf1;
  for (int n = 0; n < nsteps; ++n) {
    const T* left = rank > 0 ? cluster.map_shared_rank(cur, rank - 1) : nullptr;
    const T* right = rank + 1 <= last_rank ? cluster.map_shared_rank(cur, rank + 1) : nullptr;
    const T* first = cluster.map_shared_rank(cur, 0);
    const T* last = cluster.map_shared_rank(cur, last_rank);
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
      const int i = i0 + c;
      T f[5];
      f[0] = cur[c];
#pragma unroll
      for (int p = 1; p < 5; ++p) {
        const bool plus = (p == 1 || p == 3);
        if (plus ? i > 0 : i < nx - 1) {  // interior pull
          if (plus)
            f[p] = c > 0 ? cur[p * chunk + c - 1] : left[p * chunk + chunk - 1];
          else
            f[p] = c < ncell - 1 ? cur[p * chunk + c + 1] : right[p * chunk];
        } else {
          const int side = plus ? LBM_SW_SIDE_XM : LBM_SW_SIDE_XP;
          switch (A.bc[side]) {
            case LBM_SW_BC_PERIODIC:
              f[p] = plus ? last[p * chunk + last_c] : first[p * chunk];
              break;
            case LBM_SW_BC_WALL: {
              const int m = (p == 1) ? 2 : (p == 2) ? 1 : (p == 3) ? 4 : 3;
              const T v = cur[m * chunk + c];
              f[p] = p >= 3 ? -v : v;
              break;
            }
            case LBM_SW_BC_OUTFLOW:
              f[p] = cur[p * chunk + c];
              break;
            default:
              f[p] = A.inflow_feq[side * 5 + p];
          }
        }
      }
      collide5_any<T, MRT>(f, K);
#pragma unroll
      for (int p = 0; p < 5; ++p) nxt[p * chunk + c] = f[p];
    }
    cluster.sync();
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int c = threadIdx.x; c < ncell; c += blockDim.x)
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i0 + c] = cur[p * chunk + c];
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

template <class T>
int cluster1d_max_cells() {
  static int max_blocks = 0;
  if (max_blocks == 0) {
    // a 16-CTA cluster where the device allows it, else the portable 8
    max_blocks = 8;
    if (cudaFuncSetAttribute(step1d_cluster<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(step1d_cluster<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(2 * 5 * 1024 * sizeof(T))) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(1024);
      cfg.dynamicSmemBytes = 2 * 5 * 1024 * sizeof(T);
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = 16;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, step1d_cluster<T, false>, &cfg) == cudaSuccess && clusters > 0)
        max_blocks = 16;
    }
    cudaGetLastError();
  }
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
  const int threads = ((chunk + 31) / 32) * 32;
  const size_t smem = 2 * 5 * static_cast<size_t>(chunk) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(step1d_cluster<T, MRT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(2 * 5 * 1024 * sizeof(T)));
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
