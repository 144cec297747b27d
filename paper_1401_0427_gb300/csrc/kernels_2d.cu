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
#include "step2d_vec.cuh"

namespace lbm {
namespace {

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

template <class T, bool MRT>
__global__ void __launch_bounds__(256) step2d_simple(const StepArgs<T> A, const Consts<T> K) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = pull_one(A, p, x, y);
    T h, qx, qy;
    collide13_any<T, MRT>(f, K, h, qx, qy);
#pragma unroll
    for (int p = 0; p < 13; ++p) A.dst[p * A.plane + y * A.pitch + x] = f[p];
  }
}

// --------------------------------------------------------------------------
// Obstacles: the SIMPLE step with a mask of solid cells ([ny][nx], nonzero = solid).  A
// population whose source cell is solid (inside the domain, or across a periodic side) is
// replaced by the mirror image of the cell's own population, the momentum family normal
// to the face negated: the WALL rule of a domain side applied at the fluid-solid face.
// Solid cells hold no fluid and keep their populations (copied to the new buffer).
// --------------------------------------------------------------------------
template <class T, bool MRT>
__global__ void __launch_bounds__(256)
    step2d_obstacle(const StepArgs<T> A, const Consts<T> K, const unsigned char* __restrict__ solid) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    const long long cell = static_cast<long long>(y) * A.pitch + x;
    if (solid[static_cast<long long>(y) * A.nx + x]) {
#pragma unroll
      for (int p = 0; p < 13; ++p) A.dst[p * A.plane + cell] = A.src[p * A.plane + cell];
      continue;
    }
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) {
      int xs = x - ex_of(p), ys = y - ey_of(p);
      const bool wrap_x = (xs < 0 || xs >= A.nx) && A.bc[xs < 0 ? LBM_SW_SIDE_XM : LBM_SW_SIDE_XP] == LBM_SW_BC_PERIODIC;
      const bool wrap_y = (ys < 0 || ys >= A.ny) && A.bc[ys < 0 ? LBM_SW_SIDE_YM : LBM_SW_SIDE_YP] == LBM_SW_BC_PERIODIC;
      if (wrap_x) xs = (xs + A.nx) % A.nx;
      if (wrap_y) ys = (ys + A.ny) % A.ny;
      const bool inside = xs >= 0 && xs < A.nx && ys >= 0 && ys < A.ny;
      if (p > 0 && inside && solid[static_cast<long long>(ys) * A.nx + xs]) {
        const bool xface = ex_of(p) != 0;
        const int m = xface ? mirror_x(p) : mirror_y(p);
        const bool normal = xface ? (p >= 5 && p <= 8) : (p >= 9);
        const T v = A.src[m * A.plane + cell];
        f[p] = normal ? -v : v;
      } else {
        f[p] = pull_one(A, p, x, y);
      }
    }
    T h, qx, qy;
    collide13_any<T, MRT>(f, K, h, qx, qy);
#pragma unroll
    for (int p = 0; p < 13; ++p) A.dst[p * A.plane + cell] = f[p];
  }
}

// --------------------------------------------------------------------------
// VEC variant (row body in step2d_vec.cuh): each thread owns V consecutive cells of one row (one 16-byte
// vector per plane: 4 FP32 or 2 FP64 values), a warp owns 32 V cells of a row.
// All 13 loads are aligned vectors: the y-moving families read whole vectors of
// rows y -+ 1, and the x-moving families read their own row and shift it by one
// cell with a warp shuffle (lanes 0 and 31 fetch the single cell beyond the warp).
// Boundary rules replace the values that would come from outside the domain;
// rows are warp-uniform, so only the first and last row and the warps holding
// x = 0 or x = nx - 1 take a boundary branch.
// --------------------------------------------------------------------------
//
// Launched with programmatic dependent launch: the next step's CTAs may be placed while this
// step's last CTAs run.  Each CTA first waits for the previous grid to have completed and
// its writes to be visible (griddepcontrol.wait: before any read of src or write of dst, so
// neither the previous step's output nor its input is touched early), and signals when its
// own rows are done (griddepcontrol.launch_dependents).  Launched without it, both are no-ops.
template <class T, int BY, bool MRT>
__global__ void __launch_bounds__(32 * BY) step2d_vec(const StepArgs<T> A, const Consts<T> K) {
  constexpr int V = V16<T>::n;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int x0 = (blockIdx.x * 32 + threadIdx.x) * V;
  for (int y = blockIdx.y * BY + threadIdx.y; y < A.ny; y += gridDim.y * BY)  // warp-uniform
    vec_row<T, false, MRT>(A, K, y, x0, threadIdx.x, nullptr);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The same step with solid cells inside the domain (mirror walls on their faces; OBST in
// vec_row), launched like step2d_vec.
template <class T, int BY, bool MRT>
__global__ void __launch_bounds__(32 * BY)
    step2d_vec_obstacle(const StepArgs<T> A, const Consts<T> K, const unsigned char* __restrict__ solid) {
  constexpr int V = V16<T>::n;
  const int x0 = (blockIdx.x * 32 + threadIdx.x) * V;
  for (int y = blockIdx.y * BY + threadIdx.y; y < A.ny; y += gridDim.y * BY)  // warp-uniform
    vec_row<T, false, MRT, true>(A, K, y, x0, threadIdx.x, nullptr, solid);
}

// The same step, also writing the moments (h, hu, hv) of the new state to three planes
// (used by the replay of the discrete adjoint).
template <class T, int BY>
__global__ void __launch_bounds__(32 * BY) step2d_vec_w(const StepArgs<T> A, const Consts<T> K, T* w_out) {
  constexpr int V = V16<T>::n;
  const int x0 = (blockIdx.x * 32 + threadIdx.x) * V;
  for (int y = blockIdx.y * BY + threadIdx.y; y < A.ny; y += gridDim.y * BY)
    vec_row<T, true>(A, K, y, x0, threadIdx.x, w_out);
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

// Collide dense pre-collision populations into the pitched buffer; solid cells (when a
// mask is given) are stored as they are.
template <class T, bool MRT>
__global__ void collide2d_dense(const StepArgs<T> A, const Consts<T> K, const T* __restrict__ dense,
                                const unsigned char* __restrict__ solid) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = static_cast<long long>(A.nx) * A.ny;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    const long long c = static_cast<long long>(y) * A.nx + x;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = dense[p * n + c];
    T h, qx, qy;
    if (!(solid && solid[c])) collide13_any<T, MRT>(f, K, h, qx, qy);
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

// Moments of the state in A.src into three planes of the population pitch.
template <class T>
__global__ void moments2d_planes(const StepArgs<T> A, T* __restrict__ w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) f[p] = A.src[p * A.plane + y * A.pitch + x];
    T d, qx, qy;
    moments13(f, d, qx, qy);
    const long long c = static_cast<long long>(y) * A.pitch + x;
    w[c] = d;
    w[A.plane + c] = qx;
    w[2 * A.plane + c] = qy;
  }
}

// An FP64 checkpoint back into the storage precision (A.dst, pitched planes) with the moments
// of the restored populations (summed as moments2d_planes does) in the three planes at w:
// the restore and the first moment slot of a segment replay in one pass.
template <class T>
__global__ void restore_moments2d(const double* __restrict__ ck, const StepArgs<T> A, T* __restrict__ w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    const long long c = static_cast<long long>(y) * A.pitch + x;
    T f[13];
#pragma unroll
    for (int p = 0; p < 13; ++p) {
      f[p] = static_cast<T>(ck[p * A.plane + c]);
      A.dst[p * A.plane + c] = f[p];
    }
    T d, qx, qy;
    moments13(f, d, qx, qy);
    w[c] = d;
    w[A.plane + c] = qx;
    w[2 * A.plane + c] = qy;
  }
}

template <class Tin, class Tout>
__global__ void convert_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = static_cast<Tout>(in[i]);
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
  const Consts<T> K = to_consts<T>(kd);
  if (variant == LBM_SW_KERNEL_SIMPLE) {
    const dim3 block(32, 8);
    if (kd.mrt)
      step2d_simple<T, true><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, K);
    else
      step2d_simple<T, false><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, K);
  } else {
    constexpr int BY = 4;
    constexpr int V = V16<T>::n;
    const dim3 block(32, BY);
    const dim3 grid((a.nx + 32 * V - 1) / (32 * V),
                    static_cast<unsigned>(std::min<long long>((a.ny + BY - 1) / BY, 65535)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return kd.mrt ? cudaLaunchKernelEx(&cfg, step2d_vec<T, BY, true>, a, K)
                  : cudaLaunchKernelEx(&cfg, step2d_vec<T, BY, false>, a, K);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_step2d_obstacle(const StepArgs<T>& a, const ConstsD& kd, const unsigned char* solid, int variant,
                                   cudaStream_t st) {
  const Consts<T> K = to_consts<T>(kd);
  if (variant == LBM_SW_KERNEL_SIMPLE) {  // one thread per cell
    const dim3 block(32, 8);
    if (kd.mrt)
      step2d_obstacle<T, true><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, K, solid);
    else
      step2d_obstacle<T, false><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, K, solid);
    return cudaGetLastError();
  }
  constexpr int BY = 4;
  constexpr int V = V16<T>::n;
  const dim3 block(32, BY);
  const dim3 grid((a.nx + 32 * V - 1) / (32 * V), static_cast<unsigned>(std::min<long long>((a.ny + BY - 1) / BY, 65535)));
  if (kd.mrt)
    step2d_vec_obstacle<T, BY, true><<<grid, block, 0, st>>>(a, K, solid);
  else
    step2d_vec_obstacle<T, BY, false><<<grid, block, 0, st>>>(a, K, solid);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_step2d_store_w(const StepArgs<T>& a, const ConstsD& kd, T* w_out, cudaStream_t st) {
  const Consts<T> K = make_consts<T>(kd.g, kd.lambda, kd.s, kd.a);
  constexpr int BY = 4;
  constexpr int V = V16<T>::n;
  const dim3 block(32, BY);
  const dim3 grid((a.nx + 32 * V - 1) / (32 * V),
                  static_cast<unsigned>(std::min<long long>((a.ny + BY - 1) / BY, 65535)));
  step2d_vec_w<T, BY><<<grid, block, 0, st>>>(a, K, w_out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_restore_moments2d(const double* ck, const StepArgs<T>& a, T* w_out, cudaStream_t st) {
  const dim3 block(128, 2);
  restore_moments2d<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(ck, a, w_out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_moments2d_planes(const StepArgs<T>& a, T* w_out, cudaStream_t st) {
  const dim3 block(128, 2);
  moments2d_planes<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, w_out);
  return cudaGetLastError();
}

template <class Tin, class Tout>
cudaError_t launch_convert(const Tin* in, Tout* out, long long n, cudaStream_t st) {
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  convert_kernel<Tin, Tout><<<static_cast<unsigned>(blocks > 0 ? blocks : 1), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, long long, cudaStream_t);

template <class T>
cudaError_t launch_init2d(const StepArgs<T>& a, const ConstsD& kd, const double* h, const double* hu,
                          const double* hv, cudaStream_t st) {
  const dim3 block(128, 2);
  init2d<T><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, make_consts<T>(kd.g, kd.lambda, kd.s, kd.a),
                                                             h, hu, hv);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_collide2d_dense(const StepArgs<T>& a, const ConstsD& kd, const T* dense,
                                  const unsigned char* solid, cudaStream_t st) {
  const dim3 block(128, 2);
  if (kd.mrt)
    collide2d_dense<T, true><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, to_consts<T>(kd), dense, solid);
  else
    collide2d_dense<T, false><<<cell_grid(a.nx, a.ny, block), block, 0, st>>>(a, to_consts<T>(kd), dense, solid);
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
  template cudaError_t launch_collide2d_dense<T>(const StepArgs<T>&, const ConstsD&, const T*,              \
                                                const unsigned char*, cudaStream_t);                        \
  template cudaError_t launch_step2d_obstacle<T>(const StepArgs<T>&, const ConstsD&, const unsigned char*, int, \
                                                 cudaStream_t);                                             \
  template cudaError_t launch_moments2d<T>(const StepArgs<T>&, double*, double*, double*, cudaStream_t);   \
  template cudaError_t launch_inflow_feq2d<T>(T*, const int[4], const double[4][3], const ConstsD&, cudaStream_t); \
  template cudaError_t launch_step2d_store_w<T>(const StepArgs<T>&, const ConstsD&, T*, cudaStream_t);       \
  template cudaError_t launch_moments2d_planes<T>(const StepArgs<T>&, T*, cudaStream_t);                          \
  template cudaError_t launch_restore_moments2d<T>(const double*, const StepArgs<T>&, T*, cudaStream_t);

LBM_INSTANTIATE_2D(float)
LBM_INSTANTIATE_2D(double)

}  // namespace lbm
