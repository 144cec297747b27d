// Conserved totals and health check of a population state.
//
// Pass 1: each block walks whole rows (grid-stride over rows), forms h, hu, hv of
// every cell in the storage precision (pair-symmetric sums), accumulates them in
// FP64, keeps min h and counts cells with NaN/Inf or h <= 0; warp shuffles then
// shared memory reduce the block to one partial of 5 doubles.  The handle's aligned
// planes are read with 16-byte vectors; any other pitch with scalar loads.
// Pass 2: one block folds the partials in a fixed order.  Same input, same bits.
#include <cuda_runtime.h>

#include <cfloat>
#include <type_traits>

#include "internal.h"
#include "scheme.cuh"

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1216;  // 8 per SM on a 152-SM GB300
constexpr unsigned kFull = 0xffffffffu;

struct Acc {
  double h, hu, hv, hmin, bad;
};

__device__ __forceinline__ Acc combine(Acc a, const Acc& b) {
  a.h += b.h;
  a.hu += b.hu;
  a.hv += b.hv;
  a.hmin = fmin(a.hmin, b.hmin);
  a.bad += b.bad;
  return a;
}

__device__ __forceinline__ Acc warp_reduce(Acc a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Acc o;
    o.h = __shfl_down_sync(kFull, a.h, off);
    o.hu = __shfl_down_sync(kFull, a.hu, off);
    o.hv = __shfl_down_sync(kFull, a.hv, off);
    o.hmin = __shfl_down_sync(kFull, a.hmin, off);
    o.bad = __shfl_down_sync(kFull, a.bad, off);
    a = combine(a, o);
  }
  return a;
}

// Block-wide reduction of one Acc per thread; thread 0 returns the total.
__device__ __forceinline__ Acc block_reduce(Acc a) {
  __shared__ Acc warp_part[kThreads / 32];
  a = warp_reduce(a);
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) warp_part[w] = a;
  __syncthreads();
  if (w == 0) {
    a = lane < kThreads / 32 ? warp_part[lane] : Acc{0.0, 0.0, 0.0, DBL_MAX, 0.0};
    a = warp_reduce(a);
  }
  return a;
}

template <class T, int Q>
__global__ void __launch_bounds__(kThreads) diag_partials(const StepArgs<T> A, double* __restrict__ part) {
  Acc a{0.0, 0.0, 0.0, DBL_MAX, 0.0};
  for (int y = blockIdx.x; y < A.ny; y += gridDim.x) {
    const T* row = A.src + static_cast<long long>(y) * A.pitch;
    for (int x = threadIdx.x; x < A.nx; x += kThreads) {
      T h, qx, qy = T(0);
      if constexpr (Q == 13) {
        T f[13];
#pragma unroll
        for (int p = 0; p < 13; ++p) f[p] = row[p * A.plane + x];
        moments13(f, h, qx, qy);
      } else {
        T f[5];
#pragma unroll
        for (int p = 0; p < 5; ++p) f[p] = row[p * A.plane + x];
        moments5(f, h, qx);
      }
      const double hd = static_cast<double>(h), ud = static_cast<double>(qx), vd = static_cast<double>(qy);
      a.h += hd;
      a.hu += ud;
      a.hv += vd;
      a.hmin = fmin(a.hmin, hd);
      if (!(hd > 0.0) || !isfinite(hd) || !isfinite(ud) || !isfinite(vd)) a.bad += 1.0;
    }
  }
  a = block_reduce(a);
  if (threadIdx.x == 0) {
    double* o = part + 5 * blockIdx.x;
    o[0] = a.h;
    o[1] = a.hu;
    o[2] = a.hv;
    o[3] = a.hmin;
    o[4] = a.bad;
  }
}

// Pass 1 with 16-byte vector loads (V = 4 FP32 or 2 FP64 cells per thread and plane); needs
// rows that start 16-byte aligned and a pitch that is a multiple of V (the handle's layout).
template <class T, int Q>
__global__ void __launch_bounds__(kThreads) diag_partials_vec(const StepArgs<T> A, double* __restrict__ part) {
  constexpr int V = 16 / sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  Acc a{0.0, 0.0, 0.0, DBL_MAX, 0.0};
  for (int y = blockIdx.x; y < A.ny; y += gridDim.x) {
    const T* row = A.src + static_cast<long long>(y) * A.pitch;
    for (int x0 = threadIdx.x * V; x0 < A.nx; x0 += kThreads * V) {
      T f[Q][V];
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const Vec t = __ldg(reinterpret_cast<const Vec*>(row + p * A.plane + x0));
        const T* tv = reinterpret_cast<const T*>(&t);
#pragma unroll
        for (int k = 0; k < V; ++k) f[p][k] = tv[k];
      }
#pragma unroll
      for (int k = 0; k < V; ++k) {
        if (x0 + k >= A.nx) break;
        T h, qx, qy = T(0);
        if constexpr (Q == 13) {
          T g[13];
#pragma unroll
          for (int p = 0; p < 13; ++p) g[p] = f[p][k];
          moments13(g, h, qx, qy);
        } else {
          T g[5];
#pragma unroll
          for (int p = 0; p < 5; ++p) g[p] = f[p][k];
          moments5(g, h, qx);
        }
        const double hd = static_cast<double>(h), ud = static_cast<double>(qx), vd = static_cast<double>(qy);
        a.h += hd;
        a.hu += ud;
        a.hv += vd;
        a.hmin = fmin(a.hmin, hd);
        if (!(hd > 0.0) || !isfinite(hd) || !isfinite(ud) || !isfinite(vd)) a.bad += 1.0;
      }
    }
  }
  a = block_reduce(a);
  if (threadIdx.x == 0) {
    double* o = part + 5 * blockIdx.x;
    o[0] = a.h;
    o[1] = a.hu;
    o[2] = a.hv;
    o[3] = a.hmin;
    o[4] = a.bad;
  }
}

__global__ void __launch_bounds__(kThreads) diag_final(const double* __restrict__ part, int nblocks,
                                                      double* __restrict__ out) {
  Acc a{0.0, 0.0, 0.0, DBL_MAX, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    const double* o = part + 5 * b;
    a = combine(a, Acc{o[0], o[1], o[2], o[3], o[4]});
  }
  a = block_reduce(a);
  if (threadIdx.x == 0) {
    out[0] = a.h;
    out[1] = a.hu;
    out[2] = a.hv;
    out[3] = a.hmin;
    out[4] = a.bad;
  }
}

}  // namespace

int diag_max_blocks() { return kMaxBlocks; }

template <class T>
cudaError_t launch_diagnostics(const StepArgs<T>& a, int q, double* partials, double* out, cudaStream_t st) {
  const int nblocks = a.ny < kMaxBlocks ? a.ny : kMaxBlocks;
  if (q == 13)
    diag_partials_vec<T, 13><<<nblocks, kThreads, 0, st>>>(a, partials);
  else
    diag_partials_vec<T, 5><<<nblocks, kThreads, 0, st>>>(a, partials);
  diag_final<<<1, kThreads, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_diagnostics_blocks(const StepArgs<T>& a, int q, int nblocks, double* partials, double* out,
                                      cudaStream_t st) {
  if (q == 13)
    diag_partials<T, 13><<<nblocks, kThreads, 0, st>>>(a, partials);
  else
    diag_partials<T, 5><<<nblocks, kThreads, 0, st>>>(a, partials);
  diag_final<<<1, kThreads, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}

template cudaError_t launch_diagnostics<float>(const StepArgs<float>&, int, double*, double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const StepArgs<double>&, int, double*, double*, cudaStream_t);
template cudaError_t launch_diagnostics_blocks<float>(const StepArgs<float>&, int, int, double*, double*,
                                                      cudaStream_t);
template cudaError_t launch_diagnostics_blocks<double>(const StepArgs<double>&, int, int, double*, double*,
                                                       cudaStream_t);

}  // namespace lbm
