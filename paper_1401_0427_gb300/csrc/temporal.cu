// K fused D2Q5Q4Q4 steps per launch (temporal blocking), FP32.
//
// The domain is cut into strips of w <= COLS - 2K columns (equal widths but the last).
// One thread per column of a strip plus a K-column halo on each side sweeps a row
// wavefront down a segment of rows: at iteration j it brings one row of the launch's input
// state (level 0) into shared memory with cp.async (two rows ahead), then computes, for
// t = 1 .. K, one row of time level t from three rows of level t - 1; level K is written
// straight to HBM.  Each level loses one column on each side of the strip and one row at
// each end of the segment, so the halos are recomputed (a fraction about 2K/w of the
// columns and K/H of the rows, H the segment's length).  HBM traffic per lattice update is
// 104/K bytes plus the halo share, against 104 for one step per launch.
//
// Every cell update is the same pull + collide13 as the single-step kernels, on the same
// values, so K steps of this kernel equal K single steps bit for bit.
#include <cuda_pipeline.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include "internal.h"
#include "scheme.cuh"
#include "temporal.cuh"
#include "temporal_pair.cuh"

namespace lbm {
namespace {

template <int K, int COLS>
struct TemporalShape {
  static constexpr int L0 = 5;                // level-0 ring (prefetch distance 2)
  static constexpr int RING = 3;              // rows kept per intermediate level
  static constexpr size_t smem_floats() { return static_cast<size_t>(COLS) * 13 * (L0 + RING * (K - 1)); }
};

// Population p arriving at tile cell (c, R) at level t, from level t - 1 held in shared
// memory: base(row) gives the plane-0 address of a ring row; neighbour columns c -+ 1 and
// rows R -+ 1 are in the tile; sides of the domain that are not periodic use the boundary
// rule of the single-step kernels (the cell's own level t - 1 values or the inflow state).
template <int COLS>
__device__ __forceinline__ void pull_level(const float* row_m, const float* row_0, const float* row_p, int c,
                                           bool at_xm, bool at_xp, bool at_ym, bool at_yp, const int bc[4],
                                           const float* __restrict__ inflow_feq, float f[13]) {
  auto v = [&](const float* row, int p, int col) { return row[p * COLS + col]; };
  f[0] = v(row_0, 0, c);
#pragma unroll
  for (int fam = 0; fam < 3; ++fam) {
    const int p1 = 1 + 4 * fam, p2 = 2 + 4 * fam, p3 = 3 + 4 * fam, p4 = 4 + 4 * fam;
    // +x movers from c - 1
    if (!at_xm) {
      f[p1] = v(row_0, p1, c - 1);
    } else {
      const int b = bc[LBM_SW_SIDE_XM];
      if (b == LBM_SW_BC_WALL) f[p1] = fam == 1 ? -v(row_0, p3, c) : v(row_0, p3, c);
      else if (b == LBM_SW_BC_OUTFLOW) f[p1] = v(row_0, p1, c);
      else f[p1] = inflow_feq[LBM_SW_SIDE_XM * 13 + p1];
    }
    // -x movers from c + 1
    if (!at_xp) {
      f[p3] = v(row_0, p3, c + 1);
    } else {
      const int b = bc[LBM_SW_SIDE_XP];
      if (b == LBM_SW_BC_WALL) f[p3] = fam == 1 ? -v(row_0, p1, c) : v(row_0, p1, c);
      else if (b == LBM_SW_BC_OUTFLOW) f[p3] = v(row_0, p3, c);
      else f[p3] = inflow_feq[LBM_SW_SIDE_XP * 13 + p3];
    }
    // +y movers from row R - 1
    if (!at_ym) {
      f[p2] = v(row_m, p2, c);
    } else {
      const int b = bc[LBM_SW_SIDE_YM];
      if (b == LBM_SW_BC_WALL) f[p2] = fam == 2 ? -v(row_0, p4, c) : v(row_0, p4, c);
      else if (b == LBM_SW_BC_OUTFLOW) f[p2] = v(row_0, p2, c);
      else f[p2] = inflow_feq[LBM_SW_SIDE_YM * 13 + p2];
    }
    // -y movers from row R + 1
    if (!at_yp) {
      f[p4] = v(row_p, p4, c);
    } else {
      const int b = bc[LBM_SW_SIDE_YP];
      if (b == LBM_SW_BC_WALL) f[p4] = fam == 2 ? -v(row_0, p2, c) : v(row_0, p2, c);
      else if (b == LBM_SW_BC_OUTFLOW) f[p4] = v(row_0, p4, c);
      else f[p4] = inflow_feq[LBM_SW_SIDE_YP * 13 + p4];
    }
  }
}

template <int K, int COLS>
__global__ void __launch_bounds__(COLS, 1)
    step2d_temporal(const StepArgs<float> A, const Consts<float> Kc, const Partition P) {
  using S = TemporalShape<K, COLS>;
  extern __shared__ __align__(16) float smem[];
  const int c = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  const bool px = A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC;
  const bool py = A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;

  // level 0 ring [L0][13][COLS], level t ring [RING][13][COLS]
  auto lvl0 = [&](int slot) { return smem + static_cast<size_t>(slot) * 13 * COLS; };
  auto ring = [&](int t, int slot) {
    return smem + static_cast<size_t>(S::L0) * 13 * COLS + static_cast<size_t>(t - 1) * S::RING * 13 * COLS +
           static_cast<size_t>(slot) * 13 * COLS;
  };

  run_segment(P, ny, [&](int strip, int ys, int ye) {
    const int gx_raw = strip * P.w - K + c;
    const bool in_tile = c < P.w + 2 * K;
    const bool col_live = in_tile && (px || (gx_raw >= 0 && gx_raw < nx));
    const int gx = px ? ((gx_raw % nx) + nx) % nx : gx_raw;
    const bool at_xm = !px && gx_raw == 0;
    const bool at_xp = !px && gx_raw == nx - 1;
    const int iters = (ye - ys) + 2 * K;

    auto issue_row = [&](int j) {
      if (j < iters) {
        const int r = ys - K + j;
        const bool live = py || (r >= 0 && r < ny);
        if (live && col_live) {
          const int gr = py ? ((r % ny) + ny) % ny : r;
          const float* g = A.src + static_cast<long long>(gr) * A.pitch + gx;
          float* s = lvl0(j % S::L0) + c;
#pragma unroll
          for (int p = 0; p < 13; ++p) __pipeline_memcpy_async(s + p * COLS, g + p * A.plane, sizeof(float));
        }
      }
      __pipeline_commit();
    };

    issue_row(0);
    issue_row(1);
    for (int j = 0; j < iters; ++j) {
      issue_row(j + 2);
      __pipeline_wait_prior(2);  // row j has landed (this thread's copies)
      __syncthreads();           // ... and every thread's
#pragma unroll
      for (int t = 1; t <= K; ++t) {
        const int R = ys - K + j - t;  // row of level t computed now
        const bool row_ok = R >= ys - K + t && R < ye + K - t;
        const bool row_live = py || (R >= 0 && R < ny);
        if (row_ok && row_live && col_live && c >= t && c < P.w + 2 * K - t) {
          float f[13];
          const float *rm, *r0, *rp;
          if (t == 1) {  // level 0 rows R - 1, R, R + 1 are iterations j - 2, j - 1, j
            rm = lvl0((j + S::L0 - 2) % S::L0);
            r0 = lvl0((j + S::L0 - 1) % S::L0);
            rp = lvl0(j % S::L0);
          } else {
            const int base = ys - 2 * K;  // ring slot of row r: (r - base) % 3, r >= base
            rm = ring(t - 1, (R - 1 - base) % S::RING);
            r0 = ring(t - 1, (R - base) % S::RING);
            rp = ring(t - 1, (R + 1 - base) % S::RING);
          }
          const bool at_ym = !py && R == 0, at_yp = !py && R == ny - 1;
          pull_level<COLS>(rm, r0, rp, c, at_xm, at_xp, at_ym, at_yp, A.bc, A.inflow_feq, f);
          float h, qx, qy;
          collide13(f, Kc, h, qx, qy);
          if (t < K) {
            float* dst = ring(t, (R - (ys - 2 * K)) % S::RING) + c;
#pragma unroll
            for (int p = 0; p < 13; ++p) dst[p * COLS] = f[p];
          } else if (c >= K && c < K + P.w && gx_raw < nx) {
            float* g = A.dst + static_cast<long long>(R) * A.pitch + gx_raw;
#pragma unroll
            for (int p = 0; p < 13; ++p) g[p * A.plane] = f[p];
          }
        }
        if (t < K) __syncthreads();
      }
    }
    __pipeline_wait_prior(0);
  });
}

// The same wavefront on an all-periodic domain (every tile cell is a domain cell, no
// boundary rule), with the plane groups placed as PeriodicShape describes.  Level t + 1
// reads level t's x movers from the previous iteration's row and its other planes from
// registers, so the only barrier per iteration is the one after the input row lands; the
// next input row is issued after it, when every thread has finished the previous iteration.
// One wavefront of the periodic scheme over output columns [x0, x0 + w) and rows [ys, ye)
// of the grid A (every side periodic), K levels per input row.
template <int K, int COLS>
__device__ __forceinline__ void periodic_wave(const StepArgs<float>& A, const Consts<float>& Kc, float* smem, int x0,
                                              int w, int ys, int ye) {
  using S = PeriodicShape<K, COLS>;
  const int c = threadIdx.x;
  const int nx = A.nx, ny = A.ny;

  // level 0: group A [A0][3][COLS], B [B0][7][COLS], C [C0][3][COLS]
  float* const l0a = smem;
  float* const l0b = l0a + S::A0 * 3 * COLS;
  float* const l0c = l0b + S::B0 * 7 * COLS;
  // level t >= 1: x movers [2][6][COLS], planes 1, 3, 5, 7, 9, 11 in that order
  auto xm = [&](int t, int slot) { return smem + S::L0_FLOATS + (t - 1) * S::LV_FLOATS + slot * 6 * COLS; };

  const int gx_raw = x0 - K + c;
  const bool in_tile = c < w + 2 * K;
  const int gx = ((gx_raw % nx) + nx) % nx;
  const int iters = (ye - ys) + 2 * K;

  // Level t (1 .. K - 1) as the input of level t + 1, in the column's registers: the -y
  // movers, f0 and +y movers of the row computed in this iteration (*_now), f0 of the
  // previous row, the +y movers of the previous two rows.  Where a level was not
  // computed (halo columns and rows outside its range) they hold stale values that the
  // next level, whose range is one smaller on each side, never reads.
  float a_now[K][3], f0_now[K], c_now[K][3], f0_prev[K], c_prev1[K][3], c_prev2[K][3];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    f0_now[t] = f0_prev[t] = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) a_now[t][q] = c_now[t][q] = c_prev1[t][q] = c_prev2[t][q] = 0.0f;
  }

  auto issue_row = [&](int j) {
    if (j < iters && in_tile) {
      const int r = ys - K + j;
      const int gr = ((r % ny) + ny) % ny;
      const float* g = A.src + static_cast<long long>(gr) * A.pitch + gx;
      float* sa = l0a + (j % S::A0) * 3 * COLS + c;
      float* sb = l0b + (j % S::B0) * 7 * COLS + c;
      float* sc = l0c + (j % S::C0) * 3 * COLS + c;
#pragma unroll
      for (int p = 0; p < 13; ++p) {
        float* d = plane_group(p) == 0 ? sa : (plane_group(p) == 1 ? sb : sc);
        __pipeline_memcpy_async(d + plane_index(p) * COLS, g + p * A.plane, sizeof(float));
      }
    }
    __pipeline_commit();
  };

  issue_row(0);
  issue_row(1);
  for (int j = 0; j < iters; ++j) {
    __pipeline_wait_prior(1);  // row j has landed (this thread's copies; row j + 1 may be in flight)
    __syncthreads();           // ... and every thread's; iteration j - 1 is over everywhere
    issue_row(j + 2);
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int R = ys - K + j - t;  // row of level t computed now
      const bool row_ok = R >= ys - K + t && R < ye + K - t;
      if (row_ok && c >= t && c < w + 2 * K - t) {
        float f[13];
        if (t == 1) {
          // level 0: row R + 1 landed now (iteration j), R at j - 1, R - 1 at j - 2
          const float* ra = l0a + (j % S::A0) * 3 * COLS + c;
          const float* rb = l0b + ((j + S::B0 - 1) % S::B0) * 7 * COLS + c;
          const float* rc = l0c + ((j + S::C0 - 2) % S::C0) * 3 * COLS + c;
          f[0] = rb[0];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            f[1 + 4 * fam] = rb[(1 + 2 * fam) * COLS - 1];
            f[2 + 4 * fam] = rc[fam * COLS];
            f[3 + 4 * fam] = rb[(2 + 2 * fam) * COLS + 1];
            f[4 + 4 * fam] = ra[fam * COLS];
          }
        } else {
          const float* x = xm(t - 1, (j + 1) & 1) + c;  // level t - 1, row R (previous iteration)
          f[0] = f0_prev[t - 1];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            f[1 + 4 * fam] = x[(2 * fam) * COLS - 1];
            f[2 + 4 * fam] = c_prev2[t - 1][fam];
            f[3 + 4 * fam] = x[(2 * fam + 1) * COLS + 1];
            f[4 + 4 * fam] = a_now[t - 1][fam];
          }
        }
        float h, qx, qy;
        collide13(f, Kc, h, qx, qy);
        if (t < K) {
          float* x = xm(t, j & 1) + c;
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            x[(2 * fam) * COLS] = f[1 + 4 * fam];
            x[(2 * fam + 1) * COLS] = f[3 + 4 * fam];
            a_now[t][fam] = f[4 + 4 * fam];
            c_now[t][fam] = f[2 + 4 * fam];
          }
          f0_now[t] = f[0];
        } else if (c >= K && c < K + w && gx_raw < nx) {
          float* g = A.dst + static_cast<long long>(R) * A.pitch + gx_raw;
#pragma unroll
          for (int p = 0; p < 13; ++p) g[p * A.plane] = f[p];
        }
      }
      if (t > 1) {
        // level t - 1 is consumed for this iteration: age its rows
        f0_prev[t - 1] = f0_now[t - 1];
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          c_prev2[t - 1][fam] = c_prev1[t - 1][fam];
          c_prev1[t - 1][fam] = c_now[t - 1][fam];
        }
      }
    }
  }
  __pipeline_wait_prior(0);
}

template <int K, int COLS>
__global__ void __launch_bounds__(COLS, COLS == 192 ? 2 : (K <= 4 ? 5 : 3))
    step2d_temporal_periodic(const StepArgs<float> A, const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  run_segment(P, A.ny, [&](int strip, int ys, int ye) { periodic_wave<K, COLS>(A, Kc, smem, strip * P.w, P.w, ys, ye); });
}

// Batched instances: a list of wavefront units (instance, strip, row segment); CTA b runs
// units [first[b], first[b + 1]) one after the other, on a grid of one wave of resident
// CTAs (the host balances the units over the CTAs).
template <int K, int COLS>
__global__ void __launch_bounds__(COLS, COLS == 192 ? 2 : (K <= 4 ? 5 : 3))
    batch_temporal_periodic(const WaveUnit* __restrict__ units, const int* __restrict__ first,
                            const float* __restrict__ src, float* __restrict__ dst, const Consts<float> Kc) {
  extern __shared__ __align__(16) float smem[];
  for (int u = first[blockIdx.x]; u < first[blockIdx.x + 1]; ++u) {
    const WaveUnit U = units[u];
    StepArgs<float> A;
    A.src = src + U.offset;
    A.dst = dst + U.offset;
    A.inflow_feq = nullptr;
    A.nx = U.nx;
    A.ny = U.ny;
    A.pitch = U.pitch;
    A.plane = U.plane;
    for (int s = 0; s < 4; ++s) A.bc[s] = LBM_SW_BC_PERIODIC;
    periodic_wave<K, COLS>(A, Kc, smem, U.x0, U.w, U.ys, U.ye);
    __syncthreads();  // the next unit reuses the rings
  }
}

// The paired wavefront with the boundary rules of any sides (even nx; odd nx with ODD).
template <int K, int COLS, int PF, bool STORE_W = false, bool L0R = false>
__global__ void __launch_bounds__(COLS / 2, 2)
    step2d_temporal_x2(const StepArgs<float> A, const Consts<float> Kc, const Partition P,
                       float* __restrict__ wout = nullptr, long long wslot = 0) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    pair_wave<K, COLS, PF, STORE_W, L0R, false, false, STORE_W>(A, Kc, smem, strip * P.w, P.w, ys, ye, wout, wslot);
  });
  pdl_done();
}

// Every side periodic.  The plain kernel runs even widths; the one that also stores the
// moments of every level (the adjoint's replays) and the _odd kernels any width.  The
// branch-free steady state: the 6-step 256-column plain kernel and every replay kernel
// (-1 % per gradient at 1024^2).
template <int K, int COLS, int PF, bool STORE_W = false, bool L0R = false>
__global__ void __launch_bounds__(COLS / 2, 2)
    step2d_temporal_periodic_x2(const StepArgs<float> A, const Consts<float> Kc, const Partition P,
                                float* __restrict__ wout = nullptr, long long wslot = 0) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    pair_wave<K, COLS, PF, STORE_W, L0R, true, false, STORE_W, !STORE_W && K <= 6,
              STORE_W || (K == 6 && COLS == 256)>(A, Kc, smem, strip * P.w, P.w, ys, ye, wout, wslot);
  });
  pdl_done();
}

template <int K, int COLS, int PF, bool L0R, bool PER>
__global__ void __launch_bounds__(COLS / 2, 2)
    step2d_temporal_x2_odd(const StepArgs<float> A, const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    pair_wave<K, COLS, PF, false, L0R, PER, false, true, PER && K <= 6>(A, Kc, smem, strip * P.w, P.w, ys, ye, nullptr,
                                                                         0);
  });
  pdl_done();
}

// Sides of a batch (shared by its instances) and the inflow equilibria of its INFLOW sides.
struct BatchSides {
  int bc[4];
  const float* inflow_feq;  // [4][13] (device)
};

// The same for instances of any width with the paired wavefront (two columns per thread).
template <int K, int COLS, int PF, bool L0R>
__global__ void __launch_bounds__(COLS / 2, 2)
    batch_temporal_pairs(const WaveUnit* __restrict__ units, const int* __restrict__ first,
                         const float* __restrict__ src, float* __restrict__ dst, const Consts<float> Kc) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  for (int u = first[blockIdx.x]; u < first[blockIdx.x + 1]; ++u) {
    const WaveUnit U = units[u];
    StepArgs<float> A;
    A.src = src + U.offset;
    A.dst = dst + U.offset;
    A.inflow_feq = nullptr;
    A.nx = U.nx;
    A.ny = U.ny;
    A.pitch = U.pitch;
    A.plane = U.plane;
    for (int s = 0; s < 4; ++s) A.bc[s] = LBM_SW_BC_PERIODIC;
    pair_wave<K, COLS, PF, false, L0R, true, false, true, K <= 6>(A, Kc, smem, U.x0, U.w, U.ys, U.ye, nullptr, 0);
    __syncthreads();  // the next unit reuses the rings
  }
  pdl_done();
}

// The same with the boundary rules of sides that are not periodic (even K).
template <int K, int COLS, int PF, bool L0R>
__global__ void __launch_bounds__(COLS / 2, 2)
    batch_temporal_pairs_bounded(const WaveUnit* __restrict__ units, const int* __restrict__ first,
                                 const float* __restrict__ src, float* __restrict__ dst, const Consts<float> Kc,
                                 const BatchSides sides) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  for (int u = first[blockIdx.x]; u < first[blockIdx.x + 1]; ++u) {
    const WaveUnit U = units[u];
    StepArgs<float> A;
    A.src = src + U.offset;
    A.dst = dst + U.offset;
    A.inflow_feq = sides.inflow_feq;
    A.nx = U.nx;
    A.ny = U.ny;
    A.pitch = U.pitch;
    A.plane = U.plane;
    for (int s = 0; s < 4; ++s) A.bc[s] = sides.bc[s];
    pair_wave<K, COLS, PF, false, L0R, false, false, true, false>(A, Kc, smem, U.x0, U.w, U.ys, U.ye, nullptr, 0);
    __syncthreads();  // the next unit reuses the rings
  }
  pdl_done();
}

// Launch one kernel of K steps.  Column counts: 192 for the periodic kernel (its shared
// memory allows two CTAs per SM at K = 6 .. 8), 128 for the general one (full rings).
template <int K, bool PER>
cudaError_t launch_k(const StepArgs<float>& a, const ConstsD& kd, cudaStream_t st, int sm_count) {
  constexpr int COLS = PER ? 192 : 128;
  const size_t smem = (PER ? PeriodicShape<K, COLS>::floats() : TemporalShape<K, COLS>::smem_floats()) * sizeof(float);
  const void* fn;
  if constexpr (PER)
    fn = reinterpret_cast<const void*>(step2d_temporal_periodic<K, COLS>);
  else
    fn = reinterpret_cast<const void*>(step2d_temporal<K, COLS>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS, smem);
  // one wave of the resident CTAs for the periodic kernel, two for the other
  const Partition P = partition(a.nx, a.ny, COLS - 2 * K, K, resident * std::max(sm_count, 1), PER ? 1 : 2);
  const int grid = P.strips * P.segments;
  const Consts<float> K_ = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  if constexpr (PER)
    step2d_temporal_periodic<K, COLS><<<grid, COLS, smem, st>>>(a, K_, P);
  else
    step2d_temporal<K, COLS><<<grid, COLS, smem, st>>>(a, K_, P);
  return cudaGetLastError();
}

// The paired kernel: COLS tile columns, COLS / 2 threads, w even; PER: every side periodic.
template <int K, int COLS, int PF, bool L0R = false, bool PER = true>
cudaError_t launch_k_pairs(const StepArgs<float>& a, const ConstsD& kd, cudaStream_t st, int sm_count) {
  const size_t smem = PairShape<K, COLS, PF, L0R>::floats() * sizeof(float);
  const bool odd = a.nx & 1;
  const void* fn = odd ? reinterpret_cast<const void*>(step2d_temporal_x2_odd<K, COLS, PF, L0R, PER>)
                   : PER ? reinterpret_cast<const void*>(step2d_temporal_periodic_x2<K, COLS, PF, false, L0R>)
                         : reinterpret_cast<const void*>(step2d_temporal_x2<K, COLS, PF, false, L0R>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS / 2, smem);
  const Partition Q = pair_partition(a.nx, a.ny, K, COLS, resident * std::max(sm_count, 1));
  const Consts<float> K_ = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  const dim3 grid(Q.strips * Q.segments), block(COLS / 2);
  float* const no_w = nullptr;
  if (odd) return launch_pdl(step2d_temporal_x2_odd<K, COLS, PF, L0R, PER>, grid, block, smem, st, a, K_, Q);
  if constexpr (PER)
    return launch_pdl(step2d_temporal_periodic_x2<K, COLS, PF, false, L0R>, grid, block, smem, st, a, K_, Q, no_w, 0LL);
  else
    return launch_pdl(step2d_temporal_x2<K, COLS, PF, false, L0R>, grid, block, smem, st, a, K_, Q, no_w, 0LL);
}

template <int K, bool PER, int COLS = K <= 6 ? 256 : 192>
cudaError_t launch_k_pairs_w(const StepArgs<float>& a, const ConstsD& kd, float* wout, long long wslot,
                             cudaStream_t st, int sm_count) {
  // the configuration of the forward kernel at each K
  constexpr int PF = K <= 4 ? 2 : 1;
  constexpr bool L0R = K == 6;
  const size_t smem = PairShape<K, COLS, PF, L0R>::floats() * sizeof(float);
  const void* fn = PER ? reinterpret_cast<const void*>(step2d_temporal_periodic_x2<K, COLS, PF, true, L0R>)
                       : reinterpret_cast<const void*>(step2d_temporal_x2<K, COLS, PF, true, L0R>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS / 2, smem);
  const Partition Q = pair_partition(a.nx, a.ny, K, COLS, resident * std::max(sm_count, 1));
  const Consts<float> K_ = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  const dim3 grid(Q.strips * Q.segments), block(COLS / 2);
  if constexpr (PER)
    return launch_pdl(step2d_temporal_periodic_x2<K, COLS, PF, true, L0R>, grid, block, smem, st, a, K_, Q, wout, wslot);
  else
    return launch_pdl(step2d_temporal_x2<K, COLS, PF, true, L0R>, grid, block, smem, st, a, K_, Q, wout, wslot);
}

template <int K>
cudaError_t launch_k_pairs_w(const StepArgs<float>& a, const ConstsD& kd, float* wout, long long wslot,
                             cudaStream_t st, int sm_count) {
  const bool per = a.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC && a.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  if constexpr (K == 6)
    if (static_cast<long long>(a.nx) * a.ny < (1LL << 23))  // as the forward kernel
      return per ? launch_k_pairs_w<K, true, 128>(a, kd, wout, wslot, st, sm_count)
                 : launch_k_pairs_w<K, false, 128>(a, kd, wout, wslot, st, sm_count);
  return per ? launch_k_pairs_w<K, true>(a, kd, wout, wslot, st, sm_count)
             : launch_k_pairs_w<K, false>(a, kd, wout, wslot, st, sm_count);
}

template <int K>
cudaError_t launch_k(const StepArgs<float>& a, const ConstsD& kd, cudaStream_t st, int sm_count) {
  const bool per = a.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC && a.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  // even K: the paired kernel, the measured best at each K: 256 columns and two rows of
  // prefetch up to K = 4, with the input row's f0 and +y movers in registers (periodic
  // +1.6 % at K = 4 and +30 % at K = 2, walls +0.7 % and +31 %); at K = 6, 256 columns, one
  // row of prefetch and the same registers (two CTAs per SM); at K = 8, 192 columns and one
  // row of prefetch.  Sides that are not periodic take the same shapes with their boundary
  // rules.
  if constexpr (K % 2 == 0) {
    // 128-column strips (four CTAs per SM) on small grids, whose row segments are longer for
    // the same number of CTAs, so less of the work is the wavefront's fill: K = 6 below 2^23
    // cells (+5 % at 1024^2, +3 % at 2048^2, -2 % at 4096^2), K = 4 below 2^21 cells (+13 %
    // at 1024^2, +6 % at 868^2, +7 % at 724^2, +2 .. 4 % at 640^2)
    const long long cells = static_cast<long long>(a.nx) * a.ny;
    const bool small = cells < (1LL << 23);
    if constexpr (K == 4)
      if (cells < (1LL << 21))  // (periodic: f0 and +y movers in registers, +1.8 % at 1024^2; walls: -13 %)
        return per ? launch_k_pairs<K, 128, 2, true>(a, kd, st, sm_count)
                   : launch_k_pairs<K, 128, 2, false, false>(a, kd, st, sm_count);
    if (per) {
      if constexpr (K <= 4)
        return launch_k_pairs<K, 256, 2, true>(a, kd, st, sm_count);
      else if constexpr (K == 6)
        return small ? launch_k_pairs<K, 128, 1, true>(a, kd, st, sm_count)
                     : launch_k_pairs<K, 256, 1, true>(a, kd, st, sm_count);
      else
        return launch_k_pairs<K, 192, 1>(a, kd, st, sm_count);
    }
    if constexpr (K <= 4)
      return launch_k_pairs<K, 256, 2, true, false>(a, kd, st, sm_count);
    else if constexpr (K == 6)
      return small ? launch_k_pairs<K, 128, 1, true, false>(a, kd, st, sm_count)
                   : launch_k_pairs<K, 256, 1, true, false>(a, kd, st, sm_count);
    else
      return launch_k_pairs<K, 192, 1, false, false>(a, kd, st, sm_count);
  }
  // odd K on periodic grids of 2^21 cells or more: the paired wavefront with an even left halo
  // (K + 1 columns), 256 columns, one row of prefetch, the input row's f0 and +y movers in
  // registers (K = 5: 236.5k against 171.4k MLUPS for the one-column kernel at 4096^2; K = 3:
  // 167.9k against 133.0k)
  if constexpr (K == 3 || K == 5)
    if (per && static_cast<long long>(a.nx) * a.ny >= (1LL << 21)) return launch_k_pairs<K, 256, 1, true>(a, kd, st, sm_count);
  return per ? launch_k<K, true>(a, kd, st, sm_count) : launch_k<K, false>(a, kd, st, sm_count);
}

}  // namespace

bool temporal_steps_supported(int k) { return k >= 2 && k <= 8; }

bool temporal_store_w_supported(const StepArgs<float>&, int k) { return k == 2 || k == 4 || k == 6 || k == 8; }

cudaError_t launch_step2d_temporal_store_w(const StepArgs<float>& a, const ConstsD& kd, int k, float* wout,
                                           long long wslot, cudaStream_t st, int sm_count) {
  if (!temporal_store_w_supported(a, k)) return cudaErrorNotSupported;
  switch (k) {
    case 2: return launch_k_pairs_w<2>(a, kd, wout, wslot, st, sm_count);
    case 6: return launch_k_pairs_w<6>(a, kd, wout, wslot, st, sm_count);
    case 8: return launch_k_pairs_w<8>(a, kd, wout, wslot, st, sm_count);
    default: return launch_k_pairs_w<4>(a, kd, wout, wslot, st, sm_count);
  }
}

cudaError_t launch_step2d_temporal(const StepArgs<float>& a, const ConstsD& kd, int k, cudaStream_t st,
                                   int sm_count) {
  switch (k) {
    case 2: return launch_k<2>(a, kd, st, sm_count);
    case 3: return launch_k<3>(a, kd, st, sm_count);
    case 5: return launch_k<5>(a, kd, st, sm_count);
    case 6: return launch_k<6>(a, kd, st, sm_count);
    case 7: return launch_k<7>(a, kd, st, sm_count);
    case 8: return launch_k<8>(a, kd, st, sm_count);
    default: return launch_k<4>(a, kd, st, sm_count);
  }
}

// ---------------------------------------------------------------- batched instances
namespace {

// Configuration of the paired batch kernel at K (0 columns: no paired kernel for odd K): the
// single-grid shapes, with the small grids' 128-column strips at K = 6 (the instances are
// 64 to 1024 wide; measured 200k against 194k MLUPS with 256 columns).
struct PairCfg {
  int cols, pf;
  bool l0r;
};
constexpr PairCfg pair_cfg(int k) {
  return k % 2 ? PairCfg{0, 0, false} : (k <= 4 ? PairCfg{256, 2, false} : (k == 6 ? PairCfg{128, 1, true} : PairCfg{192, 1, false}));
}

template <int K>
size_t batch_smem() {
  return PeriodicShape<K, 192>::floats() * sizeof(float);
}

template <int K>
size_t batch_pair_smem() {
  constexpr PairCfg c = pair_cfg(K);
  if constexpr (c.cols == 0)
    return 0;
  else
    return PairShape<K, c.cols, c.pf, c.l0r>::floats() * sizeof(float);
}

template <int K, bool PER = true>
const void* batch_pair_fn() {
  constexpr PairCfg c = pair_cfg(K);
  if constexpr (c.cols == 0)
    return nullptr;
  else if constexpr (PER)
    return reinterpret_cast<const void*>(batch_temporal_pairs<K, c.cols, c.pf, c.l0r>);
  else
    return reinterpret_cast<const void*>(batch_temporal_pairs_bounded<K, c.cols, c.pf, c.l0r>);
}

// Shared-memory attributes of both kernels on this device; resident CTAs per SM of each
// (0 for the paired kernel at odd K).
template <int K>
cudaError_t batch_prepare(int* resident, int* resident_pairs) {
  const void* fn = reinterpret_cast<const void*>(batch_temporal_periodic<K, 192>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(batch_smem<K>()));
  if (e != cudaSuccess) return e;
  *resident = cached_resident(fn, 192, batch_smem<K>());
  *resident_pairs = 0;
  if (const void* pf = batch_pair_fn<K>()) {
    e = cudaFuncSetAttribute(pf, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(batch_pair_smem<K>()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_pair_fn<K, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(batch_pair_smem<K>()));
    if (e != cudaSuccess) return e;
    // (the bounded form has the same shape; its list is balanced over the same CTAs)
    *resident_pairs = cached_resident(pf, pair_cfg(K).cols / 2, batch_pair_smem<K>());
  }
  return cudaSuccess;
}

cudaError_t batch_prepare_k(int k, int* resident, int* resident_pairs) {
  switch (k) {
    case 2: return batch_prepare<2>(resident, resident_pairs);
    case 3: return batch_prepare<3>(resident, resident_pairs);
    case 5: return batch_prepare<5>(resident, resident_pairs);
    case 6: return batch_prepare<6>(resident, resident_pairs);
    case 7: return batch_prepare<7>(resident, resident_pairs);
    case 8: return batch_prepare<8>(resident, resident_pairs);
    default: return batch_prepare<4>(resident, resident_pairs);
  }
}

template <int K>
cudaError_t batch_launch(const BatchWaves& w, const float* src, float* dst, const Consts<float>& c,
                         const BatchSides& sides, bool per, cudaStream_t st) {
  if (w.count > 0) {
    batch_temporal_periodic<K, 192><<<w.grid, 192, batch_smem<K>(), st>>>(w.units, w.first, src, dst, c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  constexpr PairCfg pc = pair_cfg(K);
  if constexpr (pc.cols > 0)
    if (w.pcount > 0) {
      if (per)
        return launch_pdl(batch_temporal_pairs<K, pc.cols, pc.pf, pc.l0r>, dim3(w.pgrid), dim3(pc.cols / 2),
                          batch_pair_smem<K>(), st, w.punits, w.pfirst, src, dst, c);
      else
        return launch_pdl(batch_temporal_pairs_bounded<K, pc.cols, pc.pf, pc.l0r>, dim3(w.pgrid), dim3(pc.cols / 2),
                          batch_pair_smem<K>(), st, w.punits, w.pfirst, src, dst, c, sides);
    }
  return cudaGetLastError();
}

// Units of the given instances at strip width <= wmax (even widths when `even`), balanced
// longest-first over `grid` CTAs; uploads them and the per-CTA ranges.
cudaError_t build_list(const std::vector<int>& ids, const int* nx, const int* ny, const long long* offset,
                       const long long* pitch, const long long* plane, int k, int wmax, bool even, int grid,
                       WaveUnit** d_units, int** d_first, int* count) {
  // row segments of about a sixth of a CTA's share of the strip rows, no shorter than 4k
  long long strip_rows = 0;
  for (int i : ids) strip_rows += static_cast<long long>((nx[i] + wmax - 1) / wmax) * ny[i];
  const long long target = std::max<long long>(4LL * k, (strip_rows + 6LL * grid - 1) / (6LL * grid));
  std::vector<WaveUnit> units;
  std::vector<long long> cost;
  for (int i : ids) {
    int strips = (nx[i] + wmax - 1) / wmax;
    int w = (nx[i] + strips - 1) / strips;
    if (even) {
      w += w & 1;  // <= wmax, which is even
      strips = (nx[i] + w - 1) / w;
    }
    const int segs = static_cast<int>(std::max<long long>(1, (ny[i] + target - 1) / target));
    const int rows = (ny[i] + segs - 1) / segs;
    for (int sgi = 0; sgi < segs; ++sgi)
      for (int st = 0; st < strips; ++st) {
        WaveUnit u;
        u.offset = offset[i];
        u.plane = plane[i];
        u.pitch = static_cast<int>(pitch[i]);
        u.nx = nx[i];
        u.ny = ny[i];
        u.x0 = st * w;
        u.w = w;
        u.ys = sgi * rows;
        u.ye = std::min(ny[i], u.ys + rows);
        u.pad = 0;
        if (u.ys >= u.ye) continue;
        units.push_back(u);
        cost.push_back(static_cast<long long>(u.ye - u.ys + 2 * k) * (std::min(w, nx[i] - u.x0) + 2 * k));
      }
  }
  // longest-processing-time-first onto the least loaded CTA
  std::vector<int> order(units.size());
  for (size_t u = 0; u < order.size(); ++u) order[u] = static_cast<int>(u);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  using Load = std::pair<long long, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int b = 0; b < grid; ++b) heap.push({0, b});
  std::vector<std::vector<int>> per(grid);
  for (int u : order) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(u);
    heap.push({l.first + cost[u], l.second});
  }
  std::vector<WaveUnit> sorted;
  std::vector<int> first(grid + 1, 0);
  sorted.reserve(units.size());
  for (int b = 0; b < grid; ++b) {
    first[b] = static_cast<int>(sorted.size());
    for (int u : per[b]) sorted.push_back(units[u]);
  }
  first[grid] = static_cast<int>(sorted.size());
  cudaError_t e = cudaMalloc(d_units, std::max<size_t>(1, sorted.size()) * sizeof(WaveUnit));
  if (e == cudaSuccess) e = cudaMalloc(d_first, first.size() * sizeof(int));
  if (e == cudaSuccess && !sorted.empty())
    e = cudaMemcpy(*d_units, sorted.data(), sorted.size() * sizeof(WaveUnit), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(*d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice);
  *count = static_cast<int>(sorted.size());
  return e;
}

}  // namespace

cudaError_t batch_waves_build(int count, const int* nx, const int* ny, const long long* offset, const long long* pitch,
                              const long long* plane, int k, int sm_count, BatchWaves* out) {
  batch_waves_free(out);
  int resident = 1, resident_pairs = 0;
  cudaError_t e = batch_prepare_k(k, &resident, &resident_pairs);
  if (e != cudaSuccess) return e;
  const PairCfg pc = pair_cfg(k);
  std::vector<int> odd, even;
  // at even K every instance takes the paired kernel (periodic sides: any width)
  for (int i = 0; i < count; ++i) (pc.cols > 0 ? even : odd).push_back(i);
  out->grid = std::max(1, resident * std::max(sm_count, 1));
  e = build_list(odd, nx, ny, offset, pitch, plane, k, 192 - 2 * k, false, out->grid, &out->units, &out->first,
                 &out->count);
  if (e == cudaSuccess && !even.empty()) {
    out->pgrid = std::max(1, resident_pairs * std::max(sm_count, 1));
    e = build_list(even, nx, ny, offset, pitch, plane, k, pc.cols - 2 * k, true, out->pgrid, &out->punits,
                   &out->pfirst, &out->pcount);
  }
  if (e != cudaSuccess) batch_waves_free(out);
  return e;
}

void batch_waves_free(BatchWaves* w) {
  if (w->units) cudaFree(w->units);
  if (w->first) cudaFree(w->first);
  if (w->punits) cudaFree(w->punits);
  if (w->pfirst) cudaFree(w->pfirst);
  *w = BatchWaves();
}

cudaError_t launch_batch_temporal(const BatchWaves& w, int k, const float* src, float* dst, const ConstsD& kd,
                                  const int bc[4], const float* inflow_feq, cudaStream_t st) {
  if (w.grid < 1) return cudaErrorInvalidValue;
  bool per = true;
  BatchSides sides;
  for (int s = 0; s < 4; ++s) {
    sides.bc[s] = bc[s];
    per = per && bc[s] == LBM_SW_BC_PERIODIC;
  }
  sides.inflow_feq = inflow_feq;
  if (!per && (k % 2 || w.count > 0)) return cudaErrorNotSupported;  // the bounded form is the paired one
  int resident = 1, resident_pairs = 0;
  cudaError_t e = batch_prepare_k(k, &resident, &resident_pairs);  // the shared-memory attributes, on this device
  if (e != cudaSuccess) return e;
  const Consts<float> c = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  switch (k) {
    case 2: return batch_launch<2>(w, src, dst, c, sides, per, st);
    case 3: return batch_launch<3>(w, src, dst, c, sides, per, st);
    case 5: return batch_launch<5>(w, src, dst, c, sides, per, st);
    case 6: return batch_launch<6>(w, src, dst, c, sides, per, st);
    case 7: return batch_launch<7>(w, src, dst, c, sides, per, st);
    case 8: return batch_launch<8>(w, src, dst, c, sides, per, st);
    default: return batch_launch<4>(w, src, dst, c, sides, per, st);
  }
}

}  // namespace lbm
