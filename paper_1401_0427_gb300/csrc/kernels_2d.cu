// D2Q5Q4Q4 kernels (section 3): the fused pull-stream + collide step, state
// initialisation at equilibrium, collision of given populations, moments and the
// equilibria of the inflow sides.
//
// Storage: 13 planes (f0 f1 f2 f3 f4 gx1 gx2 gx3 gx4 gy1 gy2 gy3 gy4), each ny rows
// of `pitch` elements (pitch a multiple of 32, padding kept at zero), post-collision
// values.  A step reads the 13 planes of buffer `src` and writes the 13 planes of
// buffer `dst`: population p arriving at cell (x, y) is the post-collision value at
// (x, y) - v_p (streaming one cell per step, lambda = dx/dt), or the boundary rule's
// value when that cell is outside the domain.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "scheme.cuh"

namespace lbm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Velocity components of each population and its partner across an x- / y-wall.
__device__ __forceinline__ int ex_of(int p) {
  const int d = p == 0 ? 0 : (p - 1) % 4 + 1;
  return d == 1 ? 1 : (d == 3 ? -1 : 0);
}
__device__ __forceinline__ int ey_of(int p) {
  const int d = p == 0 ? 0 : (p - 1) % 4 + 1;
  return d == 2 ? 1 : (d == 4 ? -1 : 0);
}
// Reflected partner: x-wall swaps directions 1 <-> 3, y-wall swaps 2 <-> 4.
__device__ __forceinline__ int mirror_x(int p) {
  if (p == 0) return 0;
  const int d = (p - 1) % 4 + 1, base = p - d;
  return base + (d == 1 ? 3 : (d == 3 ? 1 : d));
}
__device__ __forceinline__ int mirror_y(int p) {
  if (p == 0) return 0;
  const int d = (p - 1) % 4 + 1, base = p - d;
  return base + (d == 2 ? 4 : (d == 4 ? 2 : d));
}

// --------------------------------------------------------------------------
// SIMPLE variant: one thread per cell, each population pulled with its own
// boundary test.  Clear rather than fast.
// --------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T pull_one(const StepArgs<T>& A, int p, int x, int y) {
  int xs = x - ex_of(p), ys = y - ey_of(p);
  const int side = xs < 0 ? LBM_SW_SIDE_XM
                 : xs >= A.nx ? LBM_SW_SIDE_XP
                 : ys < 0 ? LBM_SW_SIDE_YM
                 : ys >= A.ny ? LBM_SW_SIDE_YP : -1;
  if (side < 0) return A.src[p * A.plane + ys * A.pitch + xs];
  switch (A.bc[side]) {
    case LBM_SW_BC_PERIODIC:
      xs = (xs + A.nx) % A.nx;
      ys = (ys + A.ny) % A.ny;
      return A.src[p * A.plane + ys * A.pitch + xs];
    case LBM_SW_BC_WALL: {
      const bool xwall = side < 2;
      const int m = xwall ? mirror_x(p) : mirror_y(p);
      const bool normal = xwall ? (p >= 5 && p <= 8) : (p >= 9);
      const T v = A.src[m * A.plane + y * A.pitch + x];
      return normal ? -v : v;
    }
    case LBM_SW_BC_OUTFLOW:
      return A.src[p * A.plane + y * A.pitch + x];
    default:
      return A.inflow_feq[side * 13 + p];
  }
}

template <class T>
__global__ void __launch_bounds__(256) step2d_simple(const StepArgs<T> A, const Consts<T> K) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = pull_one(A, p, x, y);
    collide13(f, K);
#pragma unroll
    for (int p = 0; p < 13; ++p) A.dst[p * A.plane + y * A.pitch + x] = f[p];
  }
}

// --------------------------------------------------------------------------
// VEC variant: each thread owns V consecutive cells of one row (one 16-byte
// vector per plane: 4 FP32 or 2 FP64 values), a warp owns 32 V cells of a row.
// All 13 loads are aligned vectors: the y-moving families read whole vectors of
// rows y -+ 1, and the x-moving families read their own row and shift it by one
// cell with a warp shuffle (lanes 0 and 31 fetch the single cell beyond the warp).
// Boundary rules replace the values that would come from outside the domain;
// rows are warp-uniform, so only the first and last row and the warps holding
// x = 0 or x = nx - 1 take a boundary branch.
// --------------------------------------------------------------------------
template <class T>
struct V16;
template <>
struct V16<float> {
  static constexpr int n = 4;
  __device__ static void load(const float* p, float (&o)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  __device__ static void store(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <>
struct V16<double> {
  static constexpr int n = 2;
  __device__ static void load(const double* p, double (&o)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = t.x; o[1] = t.y;
  }
  __device__ static void store(double* p, const double (&o)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  }
};

template <class T, int V>
__device__ __forceinline__ T pick(const T (&a)[V], int i) {
  T r = a[0];
#pragma unroll
  for (int k = 1; k < V; ++k)
    if (i == k) r = a[k];
  return r;
}

template <class T, int BY>
__global__ void __launch_bounds__(32 * BY) step2d_vec(const StepArgs<T> A, const Consts<T> K) {
  using VV = V16<T>;
  constexpr int V = VV::n;
  const int lane = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  const long long P = A.plane;
  const T* __restrict__ S = A.src;
  const int x0 = (blockIdx.x * 32 + lane) * V;
  const bool active = x0 < nx;

  for (int y = blockIdx.y * BY + threadIdx.y; y < ny; y += gridDim.y * BY) {  // warp-uniform
    const long long row = static_cast<long long>(y) * A.pitch;
    T c0[V], xp[3][V], xm[3][V], yp[3][V], ym[3][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      c0[k] = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) xp[c][k] = xm[c][k] = yp[c][k] = ym[c][k] = T(0);
    }
    if (active) {
      VV::load(S + row + x0, c0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        VV::load(S + (1 + 4 * c) * P + row + x0, xp[c]);  // f1, gx1, gy1 (moving +x)
        VV::load(S + (3 + 4 * c) * P + row + x0, xm[c]);  // f3, gx3, gy3 (moving -x)
      }
    }
    // Populations moving +y (f2, gx2, gy2) arrive from row y - 1.
    {
      const int bcs = A.bc[LBM_SW_SIDE_YM];
      if (y > 0 || bcs == LBM_SW_BC_PERIODIC) {
        const long long r = static_cast<long long>(y > 0 ? y - 1 : ny - 1) * A.pitch;
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (2 + 4 * c) * P + r + x0, yp[c]);
      } else if (bcs == LBM_SW_BC_WALL) {  // mirror of row 0: f4, gx4, -gy4
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (4 + 4 * c) * P + row + x0, yp[c]);
#pragma unroll
        for (int k = 0; k < V; ++k) yp[2][k] = -yp[2][k];
      } else if (bcs == LBM_SW_BC_OUTFLOW) {
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (2 + 4 * c) * P + row + x0, yp[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T v = A.inflow_feq[LBM_SW_SIDE_YM * 13 + 2 + 4 * c];
#pragma unroll
          for (int k = 0; k < V; ++k) yp[c][k] = v;
        }
      }
    }
    // Populations moving -y (f4, gx4, gy4) arrive from row y + 1.
    {
      const int bcs = A.bc[LBM_SW_SIDE_YP];
      if (y < ny - 1 || bcs == LBM_SW_BC_PERIODIC) {
        const long long r = static_cast<long long>(y < ny - 1 ? y + 1 : 0) * A.pitch;
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (4 + 4 * c) * P + r + x0, ym[c]);
      } else if (bcs == LBM_SW_BC_WALL) {  // mirror of row ny-1: f2, gx2, -gy2
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (2 + 4 * c) * P + row + x0, ym[c]);
#pragma unroll
        for (int k = 0; k < V; ++k) ym[2][k] = -ym[2][k];
      } else if (bcs == LBM_SW_BC_OUTFLOW) {
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (4 + 4 * c) * P + row + x0, ym[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T v = A.inflow_feq[LBM_SW_SIDE_YP * 13 + 4 + 4 * c];
#pragma unroll
          for (int k = 0; k < V; ++k) ym[c][k] = v;
        }
      }
    }
    // x-moving families: L[c][k] = value at x0 + k - 1 (+x movers), R[c][k] = at x0 + k + 1.
    T L[3][V], R[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T up = __shfl_up_sync(kFull, xp[c][V - 1], 1);
      T dn = __shfl_down_sync(kFull, xm[c][0], 1);
      if (lane == 0) up = (active && x0 > 0) ? S[(1 + 4 * c) * P + row + x0 - 1] : T(0);
      if (lane == 31) dn = (x0 + V < nx) ? S[(3 + 4 * c) * P + row + x0 + V] : T(0);
      L[c][0] = up;
#pragma unroll
      for (int k = 1; k < V; ++k) L[c][k] = xp[c][k - 1];
#pragma unroll
      for (int k = 0; k < V - 1; ++k) R[c][k] = xm[c][k + 1];
      R[c][V - 1] = dn;
    }
    if (x0 == 0) {  // cell x = 0: +x movers come from the x- ghost
      switch (A.bc[LBM_SW_SIDE_XM]) {
        case LBM_SW_BC_PERIODIC:
#pragma unroll
          for (int c = 0; c < 3; ++c) L[c][0] = S[(1 + 4 * c) * P + row + nx - 1];
          break;
        case LBM_SW_BC_WALL:
          L[0][0] = xm[0][0];
          L[1][0] = -xm[1][0];
          L[2][0] = xm[2][0];
          break;
        case LBM_SW_BC_OUTFLOW:
#pragma unroll
          for (int c = 0; c < 3; ++c) L[c][0] = xp[c][0];
          break;
        default:
#pragma unroll
          for (int c = 0; c < 3; ++c) L[c][0] = A.inflow_feq[LBM_SW_SIDE_XM * 13 + 1 + 4 * c];
      }
    }
    const int kk = nx - 1 - x0;  // cell x = nx - 1 is this thread's cell kk
    if (kk >= 0 && kk < V) {
      T rv[3];
      switch (A.bc[LBM_SW_SIDE_XP]) {
        case LBM_SW_BC_PERIODIC:
#pragma unroll
          for (int c = 0; c < 3; ++c) rv[c] = S[(3 + 4 * c) * P + row];
          break;
        case LBM_SW_BC_WALL:
          rv[0] = pick(xp[0], kk);
          rv[1] = -pick(xp[1], kk);
          rv[2] = pick(xp[2], kk);
          break;
        case LBM_SW_BC_OUTFLOW:
#pragma unroll
          for (int c = 0; c < 3; ++c) rv[c] = pick(xm[c], kk);
          break;
        default:
#pragma unroll
          for (int c = 0; c < 3; ++c) rv[c] = A.inflow_feq[LBM_SW_SIDE_XP * 13 + 3 + 4 * c];
      }
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (k == kk)
#pragma unroll
          for (int c = 0; c < 3; ++c) R[c][k] = rv[c];
    }

    T out[13][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      T f[13] = {c0[k],    L[0][k], yp[0][k], R[0][k], ym[0][k], L[1][k], yp[1][k],
                 R[1][k], ym[1][k], L[2][k], yp[2][k], R[2][k], ym[2][k]};
      collide13(f, K);
      const bool valid = x0 + k < nx;  // padding cells are stored as zero
#pragma unroll
      for (int p = 0; p < 13; ++p) out[p][k] = valid ? f[p] : T(0);
    }
    if (active)
#pragma unroll
      for (int p = 0; p < 13; ++p) VV::store(A.dst + p * P + row + x0, out[p]);
  }
}

// --------------------------------------------------------------------------
// Helpers: equilibrium initialisation, collision of dense populations, moments,
// inflow equilibria.
// --------------------------------------------------------------------------
template <class T>
__global__ void init2d(const StepArgs<T> A, const Consts<T> K, const double* __restrict__ h,
                       const double* __restrict__ hu, const double* __restrict__ hv) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    const long long c = static_cast<long long>(y) * A.nx + x;
    T e[13];
    equilibrium13(static_cast<T>(h[c]), static_cast<T>(hu[c]), static_cast<T>(hv ? hv[c] : 0.0), K, e);
#pragma unroll
    for (int p = 0; p < 13; ++p) A.dst[p * A.plane + y * A.pitch + x] = e[p];
  }
}

template <class T>
__global__ void collide2d_dense(const StepArgs<T> A, const Consts<T> K, const T* __restrict__ dense) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = static_cast<long long>(A.nx) * A.ny;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    const long long c = static_cast<long long>(y) * A.nx + x;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = dense[p * n + c];
    collide13(f, K);
#pragma unroll
    for (int p = 0; p < 13; ++p) A.dst[p * A.plane + y * A.pitch + x] = f[p];
  }
}

template <class T>
__global__ void moments2d(const StepArgs<T> A, double* __restrict__ h, double* __restrict__ hu,
                          double* __restrict__ hv) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = A.src[p * A.plane + y * A.pitch + x];
    T d, qx, qy;
    moments13(f, d, qx, qy);
    const long long c = static_cast<long long>(y) * A.nx + x;
    h[c] = static_cast<double>(d);
    hu[c] = static_cast<double>(qx);
    if (hv) hv[c] = static_cast<double>(qy);
  }
}

struct InflowStates {
  int bc[4];
  double w[4][3];
};

template <class T>
__global__ void inflow_feq2d(T* out, const InflowStates in, const Consts<T> K) {
  const int side = threadIdx.x;
  if (side >= 4) return;
  T e[13];
  if (in.bc[side] == LBM_SW_BC_INFLOW) {
    equilibrium13(static_cast<T>(in.w[side][0]), static_cast<T>(in.w[side][1]),
                  static_cast<T>(in.w[side][2]), K, e);
  } else {
#pragma unroll
    for (int p = 0; p < 13; ++p) e[p] = T(0);
  }
#pragma unroll
  for (int p = 0; p < 13; ++p) out[side * 13 + p] = e[p];
}

dim3 cell_grid(int nx, int ny, dim3 block) {
  const unsigned gx = (nx + block.x - 1) / block.x;
  const unsigned gy = static_cast<unsigned>(std::min<long long>((ny + block.y - 1) / block.y, 65535));
  return dim3(gx, gy);
}

}  // namespace

template <class T>
cudaError_t launch_step2d(const StepArgs<T>& a, const ConstsD& kd, int variant, cudaStream_t st) {
  const Consts<T> K = make_consts<T>(kd.g, kd.lambda, kd.s, kd.a);
  if (variant == LBM_SW_KERNEL_SIMPLE) {
    const dim3 block(32, 8);
    step2d_simple<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, K);
  } else {
    constexpr int BY = 4;
    constexpr int V = V16<T>::n;
    const dim3 block(32, BY);
    const dim3 grid((a.nx + 32 * V - 1) / (32 * V),
                    static_cast<unsigned>(std::min<long long>((a.ny + BY - 1) / BY, 65535)));
    step2d_vec<T, BY><<<grid, block, 0, st>>>(a, K);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_init2d(const StepArgs<T>& a, const ConstsD& kd, const double* h, const double* hu,
                          const double* hv, cudaStream_t st) {
  const dim3 block(128, 2);
  init2d<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a),
                                                             h, hu, hv);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_collide2d_dense(const StepArgs<T>& a, const ConstsD& kd, const T* dense, cudaStream_t st) {
  const dim3 block(128, 2);
  collide2d_dense<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(
      a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a), dense);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_moments2d(const StepArgs<T>& a, double* h, double* hu, double* hv, cudaStream_t st) {
  const dim3 block(128, 2);
  moments2d<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, h, hu, hv);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_inflow_feq2d(T* out, const int bc[4], const double inflow[4][3], const ConstsD& kd,
                                cudaStream_t st) {
  InflowStates in;
  for (int s = 0; s < 4; ++s) {
    in.bc[s] = bc[s];
    for (int c = 0; c < 3; ++c) in.w[s][c] = inflow[s][c];
  }
  inflow_feq2d<T><<<1, 32, 0, st>>>(out, in, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a));
  return cudaGetLastError();
}

#define LBM_INSTANTIATE_2D(T)                                                                              \
  template cudaError_t launch_step2d<T>(const StepArgs<T>&, const ConstsD&, int, cudaStream_t);            \
  template cudaError_t launch_init2d<T>(const StepArgs<T>&, const ConstsD&, const double*, const double*,  \
                                        const double*, cudaStream_t);                                      \
  template cudaError_t launch_collide2d_dense<T>(const StepArgs<T>&, const ConstsD&, const T*, cudaStream_t); \
  template cudaError_t launch_moments2d<T>(const StepArgs<T>&, double*, double*, double*, cudaStream_t);   \
  template cudaError_t launch_inflow_feq2d<T>(T*, const int[4], const double[4][3], const ConstsD&, cudaStream_t);

LBM_INSTANTIATE_2D(float)
LBM_INSTANTIATE_2D(double)

}  // namespace lbm
