// Row body of the vectorised fused D2Q5Q4Q4 step (pull-stream + collide), shared by the
// single-grid kernel (kernels_2d.cu) and the batched persistent kernel (batch.cu).
//
// A warp owns 32 * V consecutive cells of one row (one 16-byte vector per plane and
// thread: V = 4 FP32 or 2 FP64 values).  All 13 loads are aligned vectors: the
// y-moving families read whole vectors of rows y -+ 1, and the x-moving families read
// their own row and shift it by one cell with a warp shuffle (lanes 0 and 31 fetch the
// single cell beyond the warp).  Boundary rules replace the values that would come from
// outside the domain.  Every lane of the warp must call vec_row for the same row.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "scheme.cuh"

namespace lbm {

constexpr unsigned kFullMask = 0xffffffffu;

// Device constants of a host-side ConstsD (MRT rates included).
template <class T>
inline Consts<T> to_consts(const ConstsD& k) {
  return k.mrt ? make_consts_mrt<T>(k.g, k.lambda, k.s, k.a, k.rates, 10) : make_consts<T>(k.g, k.lambda, k.s, k.a);
}

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

// One row segment: cells x0 .. x0 + V - 1 of row y (x0 >= nx: the lane only takes part
// in the shuffles).  With STORE_W the moments (h, hu, hv) of the new state are also
// written to w_out (three planes with the population pitch).
//
// OBST: solid cells (solid[ny][nx], nonzero = solid) inside the domain.  A population that
// would be pulled from a solid cell takes the value of the fluid cell's own reflected
// population, the family normal to the face negated (the WALL rule on the face); solid
// cells keep their populations and are not collided.  A warp whose cells and their four
// neighbours are all fluid runs the plain path; the others also load their own +y and -y
// movers (the values the mirror rule and the solid cells need).  The same operations on
// the same values as the one-thread-per-cell obstacle kernel, so the same bits.
template <class T, bool STORE_W, bool MRT = false, bool OBST = false>
__device__ __forceinline__ void vec_row(const StepArgs<T>& A, const Consts<T>& K, int y, int x0, int lane,
                                        T* __restrict__ w_out, const unsigned char* __restrict__ solid = nullptr) {
  static_assert(!(STORE_W && OBST), "obstacles are not stored with moments");
  using VV = V16<T>;
  constexpr int V = VV::n;
  const int nx = A.nx, ny = A.ny;
  const long long P = A.plane;
  const T* __restrict__ S = A.src;
  const bool active = x0 < nx;
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
    T up = __shfl_up_sync(kFullMask, xp[c][V - 1], 1);
    T dn = __shfl_down_sync(kFullMask, xm[c][0], 1);
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

  // OBST: solid flags (bit k for cell x0 + k) of this segment and of rows y -+ 1, and of the
  // cells left of x0 and right of x0 + V - 1 (periodic sides wrap; beyond other sides the
  // domain rule already applies)
  unsigned ms = 0, mu = 0, md = 0, lb = 0, rb = 0, rlast = 0;
  bool obst = false;
  T o2[3][V], o4[3][V];  // own +y and -y movers (OBST warps that meet a solid cell)
  if constexpr (OBST) {
    const long long mrow = static_cast<long long>(y) * nx;
    auto bits = [&](long long r) {
      unsigned b = 0;
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (x0 + k < nx && solid[r + x0 + k]) b |= 1u << k;
      return b;
    };
    const bool has_up = y > 0 || A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
    const bool has_dn = y < ny - 1 || A.bc[LBM_SW_SIDE_YP] == LBM_SW_BC_PERIODIC;
    if (active) {
      ms = bits(mrow);
      if (has_up) mu = bits(static_cast<long long>(y > 0 ? y - 1 : ny - 1) * nx);
      if (has_dn) md = bits(static_cast<long long>(y < ny - 1 ? y + 1 : 0) * nx);
    }
    lb = __shfl_up_sync(kFullMask, (ms >> (V - 1)) & 1u, 1);  // cell x0 - 1
    rb = __shfl_down_sync(kFullMask, ms & 1u, 1);             // cell x0 + V
    if (lane == 0) lb = (active && x0 > 0) ? (solid[mrow + x0 - 1] != 0) : 0u;
    if (lane == 31) rb = (x0 + V < nx) ? (solid[mrow + x0 + V] != 0) : 0u;
    if (x0 == 0) lb = A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC ? (solid[mrow + nx - 1] != 0) : 0u;
    if (kk >= 0 && kk < V) rlast = A.bc[LBM_SW_SIDE_XP] == LBM_SW_BC_PERIODIC ? (solid[mrow] != 0) : 0u;
    obst = __any_sync(kFullMask, (ms | mu | md | lb | rb | rlast) != 0u);
    if (obst) {
#pragma unroll
      for (int k = 0; k < V; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) o2[c][k] = o4[c][k] = T(0);
      if (active)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          VV::load(S + (2 + 4 * c) * P + row + x0, o2[c]);
          VV::load(S + (4 + 4 * c) * P + row + x0, o4[c]);
        }
#pragma unroll
      for (int k = 0; k < V; ++k) {
        if ((ms >> k) & 1u) continue;  // a solid cell keeps its populations (below)
        const unsigned sl = k == 0 ? lb : (ms >> (k - 1)) & 1u;
        const unsigned sr = k == kk ? rlast : (k == V - 1 ? rb : (ms >> (k + 1)) & 1u);
        if (sl) {  // +x movers from a solid cell: own -x movers, hu family negated
          L[0][k] = xm[0][k];
          L[1][k] = -xm[1][k];
          L[2][k] = xm[2][k];
        }
        if (sr) {  // -x movers: own +x movers
          R[0][k] = xp[0][k];
          R[1][k] = -xp[1][k];
          R[2][k] = xp[2][k];
        }
        if ((mu >> k) & 1u) {  // +y movers: own -y movers, hv family negated
          yp[0][k] = o4[0][k];
          yp[1][k] = o4[1][k];
          yp[2][k] = -o4[2][k];
        }
        if ((md >> k) & 1u) {  // -y movers: own +y movers
          ym[0][k] = o2[0][k];
          ym[1][k] = o2[1][k];
          ym[2][k] = -o2[2][k];
        }
      }
    }
  }

  T out[13][V];
  T wo[3][V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    T f[13] = {c0[k],    L[0][k], yp[0][k], R[0][k], ym[0][k], L[1][k], yp[1][k],
               R[1][k], ym[1][k], L[2][k], yp[2][k], R[2][k], ym[2][k]};
    T wh, wx, wy;
    if (OBST && obst && ((ms >> k) & 1u)) {
      const T own[13] = {c0[k],    xp[0][k], o2[0][k], xm[0][k], o4[0][k], xp[1][k], o2[1][k],
                         xm[1][k], o4[1][k], xp[2][k], o2[2][k], xm[2][k], o4[2][k]};
#pragma unroll
      for (int p = 0; p < 13; ++p) f[p] = own[p];
    } else {
      collide13_any<T, MRT>(f, K, wh, wx, wy);
    }
    const bool valid = x0 + k < nx;  // padding cells are stored as zero
#pragma unroll
    for (int p = 0; p < 13; ++p) out[p][k] = valid ? f[p] : T(0);
    if (STORE_W) {
      wo[0][k] = valid ? wh : T(0);
      wo[1][k] = valid ? wx : T(0);
      wo[2][k] = valid ? wy : T(0);
    }
  }
  if (active) {
#pragma unroll
    for (int p = 0; p < 13; ++p) VV::store(A.dst + p * P + row + x0, out[p]);
    if (STORE_W)
#pragma unroll
      for (int c = 0; c < 3; ++c) VV::store(w_out + c * P + row + x0, wo[c]);
  }
}

}  // namespace lbm
