// D1Q3Q2 kernels (section 2): populations f0, f+, f- (mass, D1Q3) and g+, g-
// (discharge, D1Q2; h_0^* does not depend on beta, so there is no g0).  One thread
// per cell; five planes of `pitch` elements, post-collision values.
#include <cuda_runtime.h>

#include "internal.h"
#include "scheme.cuh"

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

template <class T>
__global__ void __launch_bounds__(256) step1d(const StepArgs<T> A, const Consts<T> K) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T f[5];
    f[0] = A.src[i];
#pragma unroll
    for (int p = 1; p < 5; ++p) f[p] = pull1(A, p, i);
    collide5(f, K);
#pragma unroll
    for (int p = 0; p < 5; ++p) A.dst[p * A.plane + i] = f[p];
  }
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

template <class T>
__global__ void collide1d_dense(const StepArgs<T> A, const Consts<T> K, const T* __restrict__ dense) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nx; i += gridDim.x * blockDim.x) {
    T f[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) f[p] = dense[p * static_cast<long long>(A.nx) + i];
    collide5(f, K);
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
cudaError_t launch_step1d(const StepArgs<T>& a, const ConstsD& kd, cudaStream_t st) {
  step1d<T><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a));
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_init1d(const StepArgs<T>& a, const ConstsD& kd, const double* h, const double* hu,
                          cudaStream_t st) {
  init1d<T><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a), h, hu);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_collide1d_dense(const StepArgs<T>& a, const ConstsD& kd, const T* dense, cudaStream_t st) {
  collide1d_dense<T><<<blocks_for(a.nx, 128), 128, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a),
                                                             dense);
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
  template cudaError_t launch_init1d<T>(const StepArgs<T>&, const ConstsD&, const double*, const double*,   \
                                        cudaStream_t);                                                      \
  template cudaError_t launch_collide1d_dense<T>(const StepArgs<T>&, const ConstsD&, const T*, cudaStream_t); \
  template cudaError_t launch_moments1d<T>(const StepArgs<T>&, double*, double*, cudaStream_t);             \
  template cudaError_t launch_inflow_feq1d<T>(T*, const int[4], const double[4][3], const ConstsD&, cudaStream_t);

LBM_INSTANTIATE_1D(float)
LBM_INSTANTIATE_1D(double)

}  // namespace lbm
