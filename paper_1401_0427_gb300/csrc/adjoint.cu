// Discrete adjoint of the fused D2Q5Q4Q4 step, with sqrt(T) checkpointing (a scalar
// one-thread-per-cell kernel for the SIMPLE kernel choice, a vectorised one otherwise).
//
// Forward (post-collision storage): F*^0 = E(W^0); for n = 1..T, F^n = S(F*^{n-1}),
// W^n = M F^n (sums of the families), F*^n = C(F^n) = F^n + s (E(W^n) - F^n), where
// S is the pull streaming with the boundary rules, E the equilibria of section 3
// and C the BGK relaxation of Eq. 2-relaxation.  For a loss L(W^T), with
// Phi^n = dL/dF^n (the adjoint of the pre-collision state):
//
//   Phi^T     = M^T dL/dW^T                       (M J_C = M: the collision conserves W)
//   Phi^{n-1} = J_C(W^{n-1})^T S^T Phi^n,  n = T .. 1
//   dL/dW^0   = D(W^0)^T Phi^0                    (D^T J_C^T = D^T because J_C D = D)
//
// with J_C(W) = (1 - s) I + s D M and D = dE/dW (13 x 3).  Per cell,
// J_C^T psi = (1 - s) psi + s M^T (D^T psi): the adjoint step pulls psi = S^T Phi^n in
// the reverse direction (the transposed boundary rules below), then applies this local
// product; it needs the moments W^{n-1} only, so the replay of a segment keeps three
// planes per step.  Checkpoints of F* every `interval` steps are stored in FP64 (exact
// for FP32 states, so the replay repeats the forward run bit for bit).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <numeric>
#include <string>

#include "internal.h"
#include "scheme.cuh"
#include "step2d_vec.cuh"

namespace lbm {
namespace {

template <class T>
struct AdjArgs {
  const T* __restrict__ phi_in;  // Phi^n (13 planes)
  T* __restrict__ phi_out;       // Phi^{n-1}
  const T* __restrict__ w;       // W^{n-1}: h, hu, hv planes
  int nx, ny;
  long long pitch, plane;
  int bc[4];
};

__device__ __forceinline__ int dir_of(int p) { return p == 0 ? 0 : (p - 1) % 4 + 1; }
__device__ __forceinline__ int ex_dir(int d) { return d == 1 ? 1 : (d == 3 ? -1 : 0); }
__device__ __forceinline__ int ey_dir(int d) { return d == 2 ? 1 : (d == 4 ? -1 : 0); }
__device__ __forceinline__ int mirror_pop(int p, bool xwall) {
  const int d = dir_of(p), base = p - d;
  if (xwall) return base + (d == 1 ? 3 : (d == 3 ? 1 : d));
  return base + (d == 2 ? 4 : (d == 4 ? 2 : d));
}
__device__ __forceinline__ int side_of(int dx, int dy) {
  return dx < 0 ? LBM_SW_SIDE_XM : dx > 0 ? LBM_SW_SIDE_XP : dy < 0 ? LBM_SW_SIDE_YM : LBM_SW_SIDE_YP;
}

// psi_q(x) = (S^T Phi)_q(x): the value of every forward pull that read F*_q(x).
//   - the cell x + v_q pulled it (interior); beyond the front side: PERIODIC wraps,
//     WALL hands it to the mirror partner at x (sign of the normal family), OUTFLOW and
//     INFLOW let it leave;
//   - an OUTFLOW ghost on the back side copied it into x itself.
template <class T>
__device__ __forceinline__ T reverse_pull(const AdjArgs<T>& A, int q, int x, int y) {
  const long long P = A.plane;
  if (q == 0) return A.phi_in[y * A.pitch + x];
  const int d = dir_of(q), ex = ex_dir(d), ey = ey_dir(d);
  int xf = x + ex, yf = y + ey;
  T v = T(0);
  if (xf >= 0 && xf < A.nx && yf >= 0 && yf < A.ny) {
    v = A.phi_in[q * P + yf * A.pitch + xf];
  } else {
    const int side = side_of(ex, ey);
    const int bc = A.bc[side];
    if (bc == LBM_SW_BC_PERIODIC) {
      xf = (xf + A.nx) % A.nx;
      yf = (yf + A.ny) % A.ny;
      v = A.phi_in[q * P + yf * A.pitch + xf];
    } else if (bc == LBM_SW_BC_WALL) {
      const bool xwall = side < 2;
      const int m = mirror_pop(q, xwall);
      const bool normal = xwall ? (q >= 5 && q <= 8) : (q >= 9);
      const T w = A.phi_in[m * P + y * A.pitch + x];
      v = normal ? -w : w;
    }
  }
  const int xb = x - ex, yb = y - ey;
  if (!(xb >= 0 && xb < A.nx && yb >= 0 && yb < A.ny) && A.bc[side_of(-ex, -ey)] == LBM_SW_BC_OUTFLOW)
    v += A.phi_in[q * P + y * A.pitch + x];
  return v;
}

template <class T>
__global__ void __launch_bounds__(256) adjoint_step(const AdjArgs<T> A, const Consts<T> K) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < A.ny; y += gridDim.y * blockDim.y) {
    if (x >= A.nx) continue;
    T psi[13];
#pragma unroll
    for (int q = 0; q < 13; ++q) psi[q] = reverse_pull(A, q, x, y);
    const long long c = static_cast<long long>(y) * A.pitch + x;
    T zh, zx, zy;
    equilibrium_vjp(A.w[c], A.w[A.plane + c], A.w[2 * A.plane + c], psi, K, zh, zx, zy);
    const T oms = T(1) - K.s;
#pragma unroll
    for (int q = 0; q < 13; ++q) {
      const T z = q < 5 ? zh : (q < 9 ? zx : zy);
      A.phi_out[q * A.plane + c] = oms * psi[q] + K.s * z;
    }
  }
}

// The adjoint step with the layout of the vectorised forward step: a thread owns V
// consecutive cells of a row, loads 16-byte vectors of Phi and W, and shifts the
// x-moving families by one cell with warp shuffles, in the reverse direction of the
// forward pull (+x movers read x + 1, -x movers x - 1, +y movers row y + 1, -y movers
// row y - 1).  Front-side rules (the side a population leaves through) are applied
// first, then the back-side OUTFLOW additions, as in reverse_pull.
template <class T, int BY>
__global__ void __launch_bounds__(32 * BY) adjoint_step_vec(const AdjArgs<T> A, const Consts<T> K) {
  using VV = V16<T>;
  constexpr int V = VV::n;
  const int lane = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  const long long P = A.plane;
  const T* __restrict__ S = A.phi_in;
  const int x0 = (blockIdx.x * 32 + lane) * V;
  const bool active = x0 < nx;
  for (int y = blockIdx.y * BY + threadIdx.y; y < ny; y += gridDim.y * BY) {  // warp-uniform
    const long long row = static_cast<long long>(y) * A.pitch;
    T c0[V], xp[3][V], xm[3][V], yp[3][V], ym[3][V], w[3][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      c0[k] = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) xp[c][k] = xm[c][k] = yp[c][k] = ym[c][k] = w[c][k] = T(0);
    }
    if (active) {
      VV::load(S + row + x0, c0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        VV::load(S + (1 + 4 * c) * P + row + x0, xp[c]);
        VV::load(S + (3 + 4 * c) * P + row + x0, xm[c]);
        VV::load(A.w + c * P + row + x0, w[c]);
      }
    }
    // +y movers (2, 6, 10) were pulled by row y + 1
    {
      const int bcs = A.bc[LBM_SW_SIDE_YP];
      if (y < ny - 1 || bcs == LBM_SW_BC_PERIODIC) {
        const long long r = static_cast<long long>(y < ny - 1 ? y + 1 : 0) * A.pitch;
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (2 + 4 * c) * P + r + x0, yp[c]);
      } else if (bcs == LBM_SW_BC_WALL) {  // handed to the mirror partners 4, 8, 12 at this row
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (4 + 4 * c) * P + row + x0, yp[c]);
#pragma unroll
        for (int k = 0; k < V; ++k) yp[2][k] = -yp[2][k];
      }
      if (y == 0 && A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_OUTFLOW && active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T o[V];
          VV::load(S + (2 + 4 * c) * P + row + x0, o);
#pragma unroll
          for (int k = 0; k < V; ++k) yp[c][k] = yp[c][k] + o[k];
        }
      }
    }
    // -y movers (4, 8, 12) were pulled by row y - 1
    {
      const int bcs = A.bc[LBM_SW_SIDE_YM];
      if (y > 0 || bcs == LBM_SW_BC_PERIODIC) {
        const long long r = static_cast<long long>(y > 0 ? y - 1 : ny - 1) * A.pitch;
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (4 + 4 * c) * P + r + x0, ym[c]);
      } else if (bcs == LBM_SW_BC_WALL) {
        if (active)
#pragma unroll
          for (int c = 0; c < 3; ++c) VV::load(S + (2 + 4 * c) * P + row + x0, ym[c]);
#pragma unroll
        for (int k = 0; k < V; ++k) ym[2][k] = -ym[2][k];
      }
      if (y == ny - 1 && A.bc[LBM_SW_SIDE_YP] == LBM_SW_BC_OUTFLOW && active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T o[V];
          VV::load(S + (4 + 4 * c) * P + row + x0, o);
#pragma unroll
          for (int k = 0; k < V; ++k) ym[c][k] = ym[c][k] + o[k];
        }
      }
    }
    // x: R[c][k] = value at x0 + k + 1 of the +x movers, L[c][k] = at x0 + k - 1 of the -x movers
    T R[3][V], L[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T dn = __shfl_down_sync(kFullMask, xp[c][0], 1);
      T up = __shfl_up_sync(kFullMask, xm[c][V - 1], 1);
      if (lane == 31) dn = (x0 + V < nx) ? S[(1 + 4 * c) * P + row + x0 + V] : T(0);
      if (lane == 0) up = (active && x0 > 0) ? S[(3 + 4 * c) * P + row + x0 - 1] : T(0);
#pragma unroll
      for (int k = 0; k < V - 1; ++k) R[c][k] = xp[c][k + 1];
      R[c][V - 1] = dn;
      L[c][0] = up;
#pragma unroll
      for (int k = 1; k < V; ++k) L[c][k] = xm[c][k - 1];
    }
    const int kk = nx - 1 - x0;
    const bool right = kk >= 0 && kk < V;
    // front sides: +x movers leave through x+, -x movers through x-
    if (right) {
      T rv[3];
      switch (A.bc[LBM_SW_SIDE_XP]) {
        case LBM_SW_BC_PERIODIC:
#pragma unroll
          for (int c = 0; c < 3; ++c) rv[c] = S[(1 + 4 * c) * P + row];
          break;
        case LBM_SW_BC_WALL:
          rv[0] = pick(xm[0], kk);
          rv[1] = -pick(xm[1], kk);
          rv[2] = pick(xm[2], kk);
          break;
        default:
          rv[0] = rv[1] = rv[2] = T(0);
      }
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (k == kk)
#pragma unroll
          for (int c = 0; c < 3; ++c) R[c][k] = rv[c];
    }
    if (x0 == 0) {
      switch (A.bc[LBM_SW_SIDE_XM]) {
        case LBM_SW_BC_PERIODIC:
#pragma unroll
          for (int c = 0; c < 3; ++c) L[c][0] = S[(3 + 4 * c) * P + row + nx - 1];
          break;
        case LBM_SW_BC_WALL:
          L[0][0] = xp[0][0];
          L[1][0] = -xp[1][0];
          L[2][0] = xp[2][0];
          break;
        default:
          L[0][0] = L[1][0] = L[2][0] = T(0);
      }
    }
    // back sides: an OUTFLOW ghost copied the cell's own value into it
    if (x0 == 0 && A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_OUTFLOW)
#pragma unroll
      for (int c = 0; c < 3; ++c) R[c][0] = R[c][0] + xp[c][0];
    if (right && A.bc[LBM_SW_SIDE_XP] == LBM_SW_BC_OUTFLOW) {
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (k == kk)
#pragma unroll
          for (int c = 0; c < 3; ++c) L[c][k] = L[c][k] + xm[c][k];
    }

    T out[13][V];
    const T oms = T(1) - K.s;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const T psi[13] = {c0[k],   R[0][k], yp[0][k], L[0][k], ym[0][k], R[1][k], yp[1][k],
                         L[1][k], ym[1][k], R[2][k], yp[2][k], L[2][k], ym[2][k]};
      const bool valid = x0 + k < nx;
      T zh = T(0), zx = T(0), zy = T(0);
      if (valid) equilibrium_vjp(w[0][k], w[1][k], w[2][k], psi, K, zh, zx, zy);
#pragma unroll
      for (int q = 0; q < 13; ++q) {
        const T z = q < 5 ? zh : (q < 9 ? zx : zy);
        out[q][k] = valid ? oms * psi[q] + K.s * z : T(0);
      }
    }
    if (active)
#pragma unroll
      for (int q = 0; q < 13; ++q) VV::store(A.phi_out + q * P + row + x0, out[q]);
  }
}

// Phi^T = M^T (dL/dh, dL/dhu, dL/dhv): every population of a family receives its field.
template <class T>
__global__ void adjoint_terminal(T* __restrict__ phi, const double* __restrict__ gh, const double* __restrict__ gu,
                                 const double* __restrict__ gv, int nx, int ny, long long pitch, long long plane) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < ny; y += gridDim.y * blockDim.y) {
    if (x >= nx) continue;
    const long long i = static_cast<long long>(y) * nx + x, c = static_cast<long long>(y) * pitch + x;
    const T a = static_cast<T>(gh[i]), b = static_cast<T>(gu ? gu[i] : 0.0), d = static_cast<T>(gv ? gv[i] : 0.0);
#pragma unroll
    for (int q = 0; q < 13; ++q) phi[q * plane + c] = q < 5 ? a : (q < 9 ? b : d);
  }
}

// dL/dW^0 = D(W^0)^T Phi^0.
template <class T>
__global__ void adjoint_gradient(const T* __restrict__ phi, const T* __restrict__ w, const Consts<T> K, int nx,
                                 int ny, long long pitch, long long plane, double* __restrict__ dh,
                                 double* __restrict__ du, double* __restrict__ dv) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < ny; y += gridDim.y * blockDim.y) {
    if (x >= nx) continue;
    const long long i = static_cast<long long>(y) * nx + x, c = static_cast<long long>(y) * pitch + x;
    T psi[13];
#pragma unroll
    for (int q = 0; q < 13; ++q) psi[q] = phi[q * plane + c];
    T zh, zx, zy;
    equilibrium_vjp(w[c], w[plane + c], w[2 * plane + c], psi, K, zh, zx, zy);
    dh[i] = static_cast<double>(zh);
    if (du) du[i] = static_cast<double>(zx);
    if (dv) dv[i] = static_cast<double>(zy);
  }
}

dim3 grid_for(int nx, int ny, dim3 block) {
  const unsigned gx = (nx + block.x - 1) / block.x;
  const long long gy = (ny + block.y - 1) / block.y;
  return dim3(gx, static_cast<unsigned>(gy < 65535 ? gy : 65535));
}

}  // namespace
}  // namespace lbm

struct lbm_sw_tape {
  const lbm_sw* owner = nullptr;
  int steps = 0, interval = 0, checkpoints = 0;
  bool recorded = false;
  size_t state_elems = 0;  // 13 * plane
  double* ckpt = nullptr;  // checkpoints * 13 * plane doubles
  void* wstore = nullptr;  // wslots * 3 * plane of T
  int wslots = 0;           // interval, plus room for the last fused replay launch to run past it
  bool last_w = false;      // the moment slots hold the last segment's W (left by the forward record)
  void* phi[2] = {nullptr, nullptr};
  void* rep[2] = {nullptr, nullptr};
  double* grad_staging = nullptr;  // 3 * nx * ny doubles (host transfers)
  std::string err;
};

namespace {

int tfail(lbm_sw_tape* t, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (t) t->err = buf;
  return code;
}

#define TAPE_CUDA(t, call, what)                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return tfail(t, e_ == cudaErrorMemoryAllocation ? LBM_SW_E_NOMEM : LBM_SW_E_CUDA, "%s: %s", what, \
                   cudaGetErrorString(e_));                                                   \
  } while (0)

// Steps per fused launch of the segment replays (the handle's K: its kernel also stores the
// moments of every level) and of the adjoint steps (at most 4: the reverse wavefront keeps
// every level's moments in shared memory as well, which at K = 6 would leave one CTA per SM);
// 0 when the handle does not fuse steps.
int replay_k(const lbm_sw* h) {
  if (h->kernel != LBM_SW_KERNEL_TEMPORAL || h->p.precision != LBM_SW_FP32 || h->temporal_k < 2) return 0;
  return h->temporal_k;
}
int adjoint_k(const lbm_sw* h) { return std::min(replay_k(h), 4); }

template <class T>
lbm::StepArgs<T> replay_args(const lbm_sw* h, const lbm_sw_tape* t, int from) {
  lbm::StepArgs<T> a = lbm::handle_args<T>(h, 0);
  a.src = static_cast<const T*>(t->rep[from]);
  a.dst = static_cast<T*>(t->rep[1 - from]);
  return a;
}

// The last segment of a forward record (len steps from the handle's state) run by the
// kernels of a replay, which also keep W^{k0} .. W^{k0 + len} in the moment slots, so the
// backward pass starts without replaying it.  The same updates as lbm_sw_step, so the same
// state; FP32 handles that fuse steps only (their slots have room for the last launch).
template <class T>
int record_last_segment(lbm_sw* h, lbm_sw_tape* t, int len) {
  cudaStream_t st = h->stream;
  const lbm::ConstsD kd = lbm::handle_consts(h);
  const long long P = h->plane;
  T* W = static_cast<T*>(t->wstore);
  TAPE_CUDA(t, lbm::launch_moments2d_planes<T>(lbm::handle_args<T>(h, h->cur), W, st), "record moments");
  int from = h->cur, j = 1;
  long long launches = 1;
  if constexpr (sizeof(T) == 4) {
    const int k = replay_k(h);
    for (; j + k - 1 <= len; j += k, from ^= 1, ++launches)
      TAPE_CUDA(t, lbm::launch_step2d_temporal_store_w(lbm::handle_args<T>(h, from), kd, k, W + 3 * P * j, 3 * P, st,
                                                       h->sm_count),
                "record launch");
  }
  for (; j <= len; ++j, from ^= 1, ++launches)
    TAPE_CUDA(t, lbm::launch_step2d_store_w<T>(lbm::handle_args<T>(h, from), kd, W + 3 * P * j, st), "record step");
  h->cur = from;
  h->steps_done += len;
  h->launches += launches;
  t->last_w = true;
  return LBM_SW_OK;
}

template <class T>
int run_adjoint(lbm_sw* h, lbm_sw_tape* t, const double* gh, const double* gu, const double* gv, double* dh,
                double* du, double* dv) {
  cudaStream_t st = h->stream;
  const lbm::Consts<T> K = lbm::make_consts<T>(h->p.g, h->p.lambda, h->p.s, h->p.a);
  const lbm::ConstsD kd = lbm::handle_consts(h);
  const int nx = h->p.nx, ny = h->p.ny;
  const long long P = h->plane, pitch = h->pitch;
  const dim3 block(128, 2), grid = lbm::grid_for(nx, ny, block);
  T* W = static_cast<T*>(t->wstore);
  int cur = 0;
  lbm::adjoint_terminal<T><<<grid, block, 0, st>>>(static_cast<T*>(t->phi[cur]), gh, gu, gv, nx, ny, pitch, P);
  TAPE_CUDA(t, cudaGetLastError(), "adjoint terminal launch");
  for (int seg = t->checkpoints - 1; seg >= 0; --seg) {
    const int k0 = seg * t->interval;
    const int k1 = (k0 + t->interval < t->steps) ? k0 + t->interval : t->steps;
    // replay the segment from its checkpoint, keeping W^{k0} .. W^{k1-1} (the forward record
    // left them for the last segment)
    if (seg == t->checkpoints - 1 && t->last_w) {
      t->last_w = false;
    } else {
    TAPE_CUDA(t, lbm::launch_restore_moments2d<T>(t->ckpt + static_cast<size_t>(seg) * t->state_elems,
                                                   replay_args<T>(h, t, 1), W, st),
              "checkpoint restore");  // into rep[0] (the dst of replay_args(.., 1)), with W^{k0}
    int from = 0, j = 1;
    if constexpr (sizeof(T) == 4) {
      // FP32: K steps per launch where the fused kernel can store every level's moments
      const int k = replay_k(h);
      const auto a0 = replay_args<T>(h, t, 0);
      // (the last launch may run past the segment into the spare moment slots)
      if (k > 1 && j + k <= t->wslots && lbm::temporal_store_w_supported(a0, k))
        for (; j < k1 - k0 && j + k <= t->wslots; j += k, from ^= 1)
          TAPE_CUDA(t, lbm::launch_step2d_temporal_store_w(replay_args<T>(h, t, from), kd, k, W + 3 * P * j, 3 * P, st,
                                                           h->sm_count),
                    "replay launch");
    }
    for (; j < k1 - k0; ++j, from ^= 1)
      TAPE_CUDA(t, lbm::launch_step2d_store_w<T>(replay_args<T>(h, t, from), kd, W + 3 * P * j, st), "replay step");
    }
    // adjoint steps n = k1 .. k0 + 1 (FP32 periodic: k reverse steps per launch while the
    // segment's stored moments cover them)
    for (int n = k1; n > k0; --n) {
      if constexpr (sizeof(T) == 4) {
        const int k = adjoint_k(h);
        lbm::StepArgs<float> a = lbm::handle_args<float>(h, 0);
        a.src = static_cast<const float*>(t->phi[cur]);
        a.dst = static_cast<float*>(t->phi[1 - cur]);
        if (k > 1 && n - k0 >= k && lbm::adjoint_temporal_supported(a, k)) {
          TAPE_CUDA(t, lbm::launch_adjoint_temporal(a, W + 3 * P * (n - 1 - k0), 3 * P, kd, k, st, h->sm_count),
                    "adjoint launch");
          cur ^= 1;
          n -= k - 1;  // with the loop's decrement: n -= k
          continue;
        }
      }
      lbm::AdjArgs<T> A;
      A.phi_in = static_cast<const T*>(t->phi[cur]);
      A.phi_out = static_cast<T*>(t->phi[1 - cur]);
      A.w = W + 3 * P * (n - 1 - k0);
      A.nx = nx;
      A.ny = ny;
      A.pitch = pitch;
      A.plane = P;
      for (int s = 0; s < 4; ++s) A.bc[s] = h->p.bc[s];
      if (h->kernel == LBM_SW_KERNEL_SIMPLE) {
        lbm::adjoint_step<T><<<grid, block, 0, st>>>(A, K);
      } else {
        constexpr int BY = 4;
        constexpr int V = lbm::V16<T>::n;
        const dim3 vb(32, BY);
        const dim3 vg((nx + 32 * V - 1) / (32 * V), static_cast<unsigned>((ny + BY - 1) / BY < 65535 ? (ny + BY - 1) / BY : 65535));
        lbm::adjoint_step_vec<T, BY><<<vg, vb, 0, st>>>(A, K);
      }
      TAPE_CUDA(t, cudaGetLastError(), "adjoint step launch");
      cur ^= 1;
    }
  }
  lbm::adjoint_gradient<T><<<grid, block, 0, st>>>(static_cast<const T*>(t->phi[cur]), W, K, nx, ny, pitch, P, dh, du,
                                                    dv);
  TAPE_CUDA(t, cudaGetLastError(), "adjoint gradient launch");
  return LBM_SW_OK;
}

}  // namespace

extern "C" {

void lbm_sw_tape_destroy(lbm_sw_tape* t) {
  if (!t) return;
  if (t->owner) cudaStreamSynchronize(t->owner->stream);
  if (t->ckpt) cudaFree(t->ckpt);
  if (t->wstore) cudaFree(t->wstore);
  for (int i = 0; i < 2; ++i) {
    if (t->phi[i]) cudaFree(t->phi[i]);
    if (t->rep[i]) cudaFree(t->rep[i]);
  }
  if (t->grad_staging) cudaFree(t->grad_staging);
  delete t;
}

int lbm_sw_tape_create(lbm_sw* h, int steps, int interval, lbm_sw_tape** out) {
  if (!out) return LBM_SW_E_ARG;
  *out = nullptr;
  if (!h) return LBM_SW_E_ARG;
  if (h->p.dim != 2) {
    h->err = "tape_create: the adjoint is available for 2D handles";
    return LBM_SW_E_ARG;
  }
  if (h->mrt) {
    h->err = "tape_create: the adjoint supports the BGK relaxation only (lbm_sw_set_relaxation(h, NULL, 0))";
    return LBM_SW_E_ARG;
  }
  if (h->has_obstacles) {
    h->err = "tape_create: the adjoint does not support obstacles (lbm_sw_set_obstacle(h, NULL, 0))";
    return LBM_SW_E_ARG;
  }
  if (steps < 1 || interval < 0 || interval > steps) {
    h->err = "tape_create: need steps >= 1 and 0 <= interval <= steps";
    return LBM_SW_E_ARG;
  }
  lbm_sw_tape* t = new (std::nothrow) lbm_sw_tape;
  if (!t) return LBM_SW_E_NOMEM;
  t->owner = h;
  t->steps = steps;
  t->interval = interval ? interval : static_cast<int>(std::ceil(std::sqrt(static_cast<double>(steps))));
  if (!interval && replay_k(h) > 1) {
    // a whole number of fused launches per interval: of the forward run and replay (the
    // handle's K) and of the adjoint steps where that at most doubles the interval, else of
    // the forward run and replay
    const int k = replay_k(h), both = std::lcm(k, adjoint_k(h)), iv = t->interval;
    const int round_both = (iv + both - 1) / both * both;
    t->interval = std::min(steps, round_both <= 2 * iv ? round_both : (iv + k - 1) / k * k);
  }
  t->checkpoints = (steps + t->interval - 1) / t->interval;
  // a replay that fuses k steps per launch may run up to k - 1 steps past its segment
  t->wslots = t->interval + replay_k(h);
  t->state_elems = static_cast<size_t>(13) * h->plane;
  const size_t n = static_cast<size_t>(h->p.nx) * h->p.ny;
  bool ok = cudaMalloc(&t->ckpt, sizeof(double) * t->state_elems * t->checkpoints) == cudaSuccess &&
            cudaMalloc(&t->wstore, h->elem * 3 * h->plane * t->wslots) == cudaSuccess &&
            cudaMalloc(&t->grad_staging, sizeof(double) * 3 * n) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaMalloc(&t->phi[i], h->elem * t->state_elems) == cudaSuccess &&
         cudaMemsetAsync(t->phi[i], 0, h->elem * t->state_elems, h->stream) == cudaSuccess &&
         cudaMalloc(&t->rep[i], h->elem * t->state_elems) == cudaSuccess &&
         cudaMemsetAsync(t->rep[i], 0, h->elem * t->state_elems, h->stream) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(t->wstore, 0, h->elem * 3 * h->plane * t->wslots, h->stream) == cudaSuccess;
  if (!ok) {
    h->err = std::string("tape_create: device allocation failed: ") + cudaGetErrorString(cudaGetLastError());
    lbm_sw_tape_destroy(t);
    return LBM_SW_E_NOMEM;
  }
  *out = t;
  return LBM_SW_OK;
}

int lbm_sw_forward_record(lbm_sw* h, lbm_sw_tape* t) {
  if (!h || !t) return LBM_SW_E_ARG;
  if (t->owner != h) return tfail(t, LBM_SW_E_ARG, "forward_record: tape belongs to another handle");
  if (!h->has_state) return tfail(t, LBM_SW_E_STATE, "forward_record: the handle has no state");
  if (h->mrt || h->has_obstacles)
    return tfail(t, LBM_SW_E_ARG, "forward_record: the adjoint supports BGK without obstacles only");
  // one lbm_sw_step call per checkpoint interval, so long intervals take the handle's
  // temporal blocking (bit-identical to single steps)
  for (int seg = 0; seg < t->checkpoints; ++seg) {
    const int k0 = seg * t->interval;
    double* dst = t->ckpt + static_cast<size_t>(seg) * t->state_elems;
    cudaError_t e = h->p.precision == LBM_SW_FP64
                        ? lbm::launch_convert<double, double>(static_cast<const double*>(h->buf[h->cur]), dst,
                                                              static_cast<long long>(t->state_elems), h->stream)
                        : lbm::launch_convert<float, double>(static_cast<const float*>(h->buf[h->cur]), dst,
                                                             static_cast<long long>(t->state_elems), h->stream);
    TAPE_CUDA(t, e, "checkpoint store");
    const int len = std::min(t->interval, t->steps - k0);
    if (seg == t->checkpoints - 1 && h->p.precision == LBM_SW_FP32 && replay_k(h) > 1 &&
        lbm::temporal_store_w_supported(lbm::handle_args<float>(h, 0), replay_k(h))) {
      const int rc = record_last_segment<float>(h, t, len);
      if (rc != LBM_SW_OK) return rc;
    } else {
      t->last_w = false;
      const int rc = lbm_sw_step(h, len);
      if (rc != LBM_SW_OK) return tfail(t, rc, "forward_record: %s", h->err.c_str());
    }
  }
  t->recorded = true;
  return LBM_SW_OK;
}

int lbm_sw_adjoint(lbm_sw* h, lbm_sw_tape* t, const double* g_h, const double* g_hu, const double* g_hv,
                   double* d_h, double* d_hu, double* d_hv, int on_device) {
  if (!h || !t) return LBM_SW_E_ARG;
  if (t->owner != h) return tfail(t, LBM_SW_E_ARG, "adjoint: tape belongs to another handle");
  if (!t->recorded) return tfail(t, LBM_SW_E_STATE, "adjoint: call lbm_sw_forward_record first");
  if (!g_h || !d_h) return tfail(t, LBM_SW_E_ARG, "adjoint: g_h and d_h are required");
  const size_t n = static_cast<size_t>(h->p.nx) * h->p.ny;
  const double *gh = g_h, *gu = g_hu, *gv = g_hv;
  double *dh = d_h, *du = d_hu, *dv = d_hv;
  double* s = t->grad_staging;
  if (!on_device) {
    TAPE_CUDA(t, cudaMemcpyAsync(s, g_h, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy g_h");
    if (g_hu) TAPE_CUDA(t, cudaMemcpyAsync(s + n, g_hu, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy g_hu");
    if (g_hv)
      TAPE_CUDA(t, cudaMemcpyAsync(s + 2 * n, g_hv, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy g_hv");
    gh = s;
    gu = g_hu ? s + n : nullptr;
    gv = g_hv ? s + 2 * n : nullptr;
    // the gradient overwrites the staging only after the terminal kernel has read it
    dh = s;
    du = d_hu ? s + n : nullptr;
    dv = d_hv ? s + 2 * n : nullptr;
  }
  const int rc = h->p.precision == LBM_SW_FP64 ? run_adjoint<double>(h, t, gh, gu, gv, dh, du, dv)
                                               : run_adjoint<float>(h, t, gh, gu, gv, dh, du, dv);
  if (rc != LBM_SW_OK) return rc;
  if (!on_device) {
    TAPE_CUDA(t, cudaMemcpyAsync(d_h, dh, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy d_h");
    if (d_hu) TAPE_CUDA(t, cudaMemcpyAsync(d_hu, du, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy d_hu");
    if (d_hv) TAPE_CUDA(t, cudaMemcpyAsync(d_hv, dv, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy d_hv");
    TAPE_CUDA(t, cudaStreamSynchronize(h->stream), "adjoint synchronize");
  }
  return LBM_SW_OK;
}

int lbm_sw_tape_get_info(const lbm_sw_tape* t, lbm_sw_tape_info* out) {
  if (!t || !out) return LBM_SW_E_ARG;
  out->steps = t->steps;
  out->interval = t->interval;
  out->checkpoints = t->checkpoints;
  out->recorded = t->recorded ? 1 : 0;
  out->checkpoint_bytes = sizeof(double) * t->state_elems * t->checkpoints;
  out->replay_bytes = t->owner->elem * (3 * t->owner->plane * t->wslots + 4 * t->state_elems);
  return LBM_SW_OK;
}

const char* lbm_sw_tape_last_error(const lbm_sw_tape* t) { return t ? t->err.c_str() : "null tape"; }

}  // extern "C"
