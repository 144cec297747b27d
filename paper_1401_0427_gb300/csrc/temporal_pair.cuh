// The temporal-blocking wavefront with two columns per thread (temporal.cu: BGK kernels,
// temporal_mrt.cu: MRT kernels).
#pragma once

#include <cuda_pipeline.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "scheme.cuh"

namespace lbm {
namespace {

// Level-0 plane p -> (group, index): A = {4, 8, 12}, B = {0, 1, 3, 5, 7, 9, 11}, C = {2, 6, 10}.
__host__ __device__ constexpr int plane_group(int p) {
  return (p == 4 || p == 8 || p == 12) ? 0 : ((p == 2 || p == 6 || p == 10) ? 2 : 1);
}
__host__ __device__ constexpr int plane_index(int p) {
  return plane_group(p) == 0 ? (p - 4) / 4 : (plane_group(p) == 2 ? (p - 2) / 4 : (p == 0 ? 0 : (p + 1) / 2));
}

// The wavefront with two columns per thread (tile columns 2c and 2c + 1) and the collision
// on FP32 pairs (collide13x2: the same rounded operations, so the same bits).
// Rows of the shared-memory planes have COLS + 4 floats, tile column i at i + 2, so a
// pair is 8-byte aligned and a read one column beyond either end of the tile stays inside
// the row (the cells that read it lie outside the level's valid range and are never used).
// Input pairs land by 8-byte cp.async; with the left halo rounded up to even (K + 1 columns
// at odd K) and even strip widths every tile starts at an even column, so with an even nx no
// pair straddles the periodic seam (with an odd nx the few that do land in two 4-byte
// copies).
template <int K, int COLS, int PF, bool L0R = false>
struct PairShape {
  static constexpr int RS = COLS + 4;  // floats per plane row
  // Input ring per plane group: the row read now, the rows landed but not yet read by this
  // group, and PF rows in flight.  Groups: the -y movers (read in the landing iteration),
  // f0 and the x movers (one iteration later), the +y movers (two later).  With L0R, f0 and
  // the +y movers go to registers when their row lands, so only the x movers wait in
  // shared memory: groups -y movers [1 + PF][3], x movers [2 + PF][6], f0 and +y movers
  // [1 + PF][4].
  static constexpr int A0 = 1 + PF, B0 = 2 + PF, C0 = L0R ? 1 + PF : 3 + PF;
  static constexpr int BP = L0R ? 6 : 7, CP = L0R ? 4 : 3;  // planes per row of groups B, C
  static constexpr int L0_FLOATS = RS * (3 * A0 + BP * B0 + CP * C0);
  static constexpr int LV_FLOATS = RS * 2 * 6;
  static constexpr size_t floats() { return static_cast<size_t>(L0_FLOATS) + (K - 1) * LV_FLOATS; }
};

// Input plane p -> (group, index) in the L0R layout: 0 = {4, 8, 12}, 1 = x movers
// {1, 3, 5, 7, 9, 11}, 2 = {0, 2, 6, 10}.
__host__ __device__ constexpr int reg_group(int p) {
  return (p == 4 || p == 8 || p == 12) ? 0 : ((p == 0 || p == 2 || p == 6 || p == 10) ? 2 : 1);
}
__host__ __device__ constexpr int reg_index(int p) {
  return reg_group(p) == 0 ? (p - 4) / 4 : (reg_group(p) == 1 ? (p - 1) / 2 : (p == 0 ? 0 : (p - 2) / 4 + 1));
}

// MRT: the MRT collision (collide13x2_mrt) in place of BGK.  ODD: any nx (see below); false
// for kernels launched on even widths only.  U3: the row loop unrolled by three, so the
// register rows of the previous rows are addressed by the iteration mod 3 instead of being
// moved down at every iteration.  Measured at 4096^2: +6 % for the periodic BGK kernels up
// to K = 6 and +4 % for the batch; slower where the tripled code or its registers cost more
// than the moves (K = 8, walls, MRT, the replay that stores the moments), which move them.
// With STORE_W, the moments (h, hu, hv) of every time level t = 1 .. K are also written, for
// the launch's output cells, to the three planes at wout + (t - 1) * wslot (the replay of the
// discrete adjoint keeps the moments of every step).
//
// PER: every side periodic.  Otherwise the sides that are not periodic apply their rule
// (WALL, OUTFLOW, INFLOW) without a branch in the pull.  x sides: the edge lane reads its
// pulled x mover from another place in the same row -- its own opposite mover (WALL, times
// -1 for the hu family, an exact product), its own mover (OUTFLOW), or the column outside
// the domain, which holds the inflow equilibrium from the start (INFLOW).  y sides: when a
// level computes the first row, or reaches the row past the last, the value the rule gives
// is put in the register the next level pulls from (for level 0, in the input ring).  Tile
// columns and rows outside the domain are neither loaded nor computed, except the second lane
// of the pair that holds the last column of an odd nx (loaded from the row's padding,
// computed, never stored, never pulled).
//
// STEADY (periodic): the iterations in which every level's row lies in its range run a
// body without the per-level row and column tests: every lane of a warp with a live column
// computes every level, lanes outside a level's columns produce values that no valid cell
// pulls, and the stores keep their tests.  One branch-free block per iteration lets the
// code generator overlap a level's loads with the previous level's collision (BGK at K = 6
// with 256 columns +1 %, MRT +1.4 %; BGK at K = 4 and with 128 columns measured slower and
// keeps the tests).
template <int K, int COLS, int PF, bool STORE_W, bool L0R, bool PER = true, bool MRT = false, bool ODD = true,
          bool U3 = false, bool STEADY = false>
__device__ __forceinline__ void pair_wave(const StepArgs<float>& A, const Consts<float>& Kc, float* smem, int x0, int w,
                                          int ys, int ye, float* __restrict__ wout, long long wslot) {
  using S = PairShape<K, COLS, PF, L0R>;
  constexpr int RS = S::RS;
  const int c = threadIdx.x;  // pair index: tile columns 2c, 2c + 1
  const int col = 2 * c;
  const int nx = A.nx, ny = A.ny;

  float* const l0a = smem;
  float* const l0b = l0a + S::A0 * 3 * RS;
  float* const l0c = l0b + S::B0 * S::BP * RS;
  auto xm = [&](int t, int slot) { return smem + S::L0_FLOATS + (t - 1) * S::LV_FLOATS + slot * 6 * RS; };
  auto ld2 = [](const float* q) { return *reinterpret_cast<const float2*>(q); };
  auto st2 = [](float* q, float2 v) { *reinterpret_cast<float2*>(q) = v; };
  auto grp = [](int p) { return L0R ? reg_group(p) : plane_group(p); };
  auto idx = [](int p) { return L0R ? reg_index(p) : plane_index(p); };

  // left halo KL = K rounded up to even, so that tile columns keep the parity of the global
  // columns (8-byte aligned pairs) at odd K too; the tile spans w + K + KL columns
  constexpr int KL = K + (K & 1);
  const int gx_raw = x0 - KL + col;
  const bool px = PER || A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC;
  const bool py = PER || A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  const bool col_live = col < w + K + KL && (px || (gx_raw >= 0 && gx_raw < nx));
  const int gx = px ? ((gx_raw % nx) + nx) % nx : gx_raw;
  // An odd nx puts, with periodic x sides, the pairs of the halo that wraps around at odd
  // columns and one pair across the periodic seam: those land by two 4-byte copies; with
  // either kind of x side the output pair at the last column stores its first lane only.
  // ODD = false: nx is even (no such pairs, and no test for them).
  const int gx2 = px ? (gx + 1 == nx ? 0 : gx + 1) : gx + 1;
  const bool split = ODD && ((gx & 1) || gx2 != gx + 1);
  const bool lane_y_out = ODD && gx_raw + 1 >= nx;
  const bool at_xm = !px && gx_raw == 0;           // lane .x is the domain's first column
  const bool at_xp = !px && gx_raw + 1 == nx - 1;  // lane .y is its last (even nx)
  const bool at_xp_x = !px && gx_raw == nx - 1;    // lane .x is its last (odd nx)
  const int iters = (ye - ys) + 2 * K;
  const bool warp_live = __any_sync(0xffffffffu, col_live);  // STEADY: a warp with no live column skips

  // Level t's values as the input of level t + 1: the -y movers of the row computed now
  // (a_now), and f0 (f0r) and the +y movers (cr) of the rows of the last three iterations,
  // at slot j mod 3 with U3 (the rows of iterations j, j - 1, j - 2 at slots PH, P1, P2),
  // else at slots 0, 1, 2, moved down once the next level has read them.
  constexpr int NF = U3 ? 3 : 2;
  float2 a_now[K][3], f0r[K][NF], cr[K][3][3];
#pragma unroll
  for (int t = 0; t < K; ++t) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      a_now[t][q] = make_float2(0.f, 0.f);
      if (q < NF) f0r[t][q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 3; ++u) cr[t][q][u] = make_float2(0.f, 0.f);
    }
  }

  // x sides: offsets of the edge lane's pulled x movers from the +x (-x) plane pointer at
  // this pair (normally -1 for lane .x of the +x movers, 1 and 2 for the lanes of the -x
  // movers), and the signs of the hu family's.  With an odd nx the last column is lane .x of
  // a pair whose lane .y lies outside the domain (computed, never stored, never pulled).
  int o_p1 = -1, o_p3x = 1, o_p3 = 2;
  float sgn1x = 1.f;
  float2 sgn3 = make_float2(1.f, 1.f);
  if (!PER) {
    const int bm = A.bc[LBM_SW_SIDE_XM], bp = A.bc[LBM_SW_SIDE_XP];
    if (at_xm && bm != LBM_SW_BC_INFLOW) {
      o_p1 = bm == LBM_SW_BC_WALL ? RS : 0;  // own -x mover / own +x mover
      if (bm == LBM_SW_BC_WALL) sgn1x = -1.f;
    }
    if (at_xp && bp != LBM_SW_BC_INFLOW) {
      o_p3 = bp == LBM_SW_BC_WALL ? 1 - RS : 1;  // own +x mover / own -x mover
      if (bp == LBM_SW_BC_WALL) sgn3.y = -1.f;
    }
    if (at_xp_x) {
      o_p3x = bp == LBM_SW_BC_WALL ? -RS : (bp == LBM_SW_BC_OUTFLOW ? 0 : 2);  // own +x, own -x, inflow column
      if (bp == LBM_SW_BC_WALL) sgn3.x = -1.f;
    }
    // INFLOW: the column outside the domain of every x-mover row (for an odd nx the one past
    // the pair at the last column) holds the inflow equilibrium (nothing else writes there)
    const bool in_m = at_xm && bm == LBM_SW_BC_INFLOW, in_p = (at_xp || at_xp_x) && bp == LBM_SW_BC_INFLOW;
    if (in_m || in_p) {
      for (int fam = 0; fam < 3; ++fam) {
        const float vm = A.inflow_feq[LBM_SW_SIDE_XM * 13 + 1 + 4 * fam];
        const float vp = A.inflow_feq[LBM_SW_SIDE_XP * 13 + 3 + 4 * fam];
        for (int q = 0; q < S::B0; ++q) {
          float* rb = l0b + q * S::BP * RS + col + 2;
          if (in_m) rb[idx(1 + 4 * fam) * RS - 1] = vm;
          if (in_p) rb[idx(3 + 4 * fam) * RS + 2] = vp;
        }
        for (int t = 1; t < K; ++t)
          for (int q = 0; q < 2; ++q) {
            float* x = xm(t, q) + col + 2;
            if (in_m) x[(2 * fam) * RS - 1] = vm;
            if (in_p) x[(2 * fam + 1) * RS + 2] = vp;
          }
      }
    }
  }
  // the pulled x movers of family fam from the +x / -x planes at this pair
  auto pull_x = [&](int fam, const float* px, const float* mx, float2* f) {
    if constexpr (PER) {
      f[1 + 4 * fam] = make_float2(px[-1], px[0]);
      f[3 + 4 * fam] = make_float2(mx[1], mx[2]);
    } else {
      f[1 + 4 * fam] = make_float2(px[o_p1], px[0]);
      f[3 + 4 * fam] = make_float2(mx[o_p3x], mx[o_p3]);
      if (fam == 1) {
        f[5].x *= sgn1x;
        f[7].x *= sgn3.x;
        f[7].y *= sgn3.y;
      }
    }
  };
  // y sides: from the edge row's own -y (p4) and +y (p2) movers, the +y movers of row -1 and
  // the -y movers of row ny.
  auto ym_ghost = [&](int fam, float2 p4, float2 p2) {
    const int b = A.bc[LBM_SW_SIDE_YM];
    return b == LBM_SW_BC_WALL      ? (fam == 2 ? make_float2(-p4.x, -p4.y) : p4)
           : b == LBM_SW_BC_OUTFLOW ? p2
                                    : dup2(A.inflow_feq[LBM_SW_SIDE_YM * 13 + 2 + 4 * fam]);
  };
  auto yp_ghost = [&](int fam, float2 p4, float2 p2) {
    const int b = A.bc[LBM_SW_SIDE_YP];
    return b == LBM_SW_BC_WALL      ? (fam == 2 ? make_float2(-p2.x, -p2.y) : p2)
           : b == LBM_SW_BC_OUTFLOW ? p4
                                    : dup2(A.inflow_feq[LBM_SW_SIDE_YP * 13 + 4 + 4 * fam]);
  };

  // rows land in order, one per call of issue_row (j = 0, 1, 2, ...): with periodic y sides
  // the wrapped row advances by one per call instead of being reduced modulo ny every row
  int next_gr = py ? ((ys - K) % ny + ny) % ny : 0;
  // BGK: two commit groups per row: first the planes read in the iteration the row lands (the
  // -y movers, and f0 and the +y movers of the C group), then the B group, first read one
  // iteration later; an iteration waits for its row's first group and the previous row's
  // B group, so the B copies have two iterations to land in the same ring slots (+0.4 %
  // periodic, +1.5 % with walls at K = 6).  MRT keeps one group per row (the split measured
  // 2-3 % slower there).
  constexpr bool SPLIT = !MRT;
  auto issue_row = [&](int j) {
    const int r = ys - K + j;
    const int gr = py ? next_gr : r;
    if (py) next_gr = next_gr + 1 == ny ? 0 : next_gr + 1;
    if constexpr (SPLIT) {
      const bool live = j < iters && col_live && (py || (r >= 0 && r < ny));
      const float* g = A.src + static_cast<long long>(gr) * A.pitch + gx;
      const float* g2 = A.src + static_cast<long long>(gr) * A.pitch + gx2;
      float* sa = l0a + (j % S::A0) * 3 * RS + col + 2;
      float* sb = l0b + (j % S::B0) * S::BP * RS + col + 2;
      float* sc = l0c + (j % S::C0) * S::CP * RS + col + 2;
      auto copies = [&](bool b_group) {
        if (!live) return;
#pragma unroll
        for (int p = 0; p < 13; ++p) {
          if ((grp(p) == 1) != b_group) continue;
          float* d = grp(p) == 0 ? sa : (grp(p) == 1 ? sb : sc);
          if (!split) {
            __pipeline_memcpy_async(d + idx(p) * RS, g + p * A.plane, 2 * sizeof(float));
          } else {
            __pipeline_memcpy_async(d + idx(p) * RS, g + p * A.plane, sizeof(float));
            __pipeline_memcpy_async(d + idx(p) * RS + 1, g2 + p * A.plane, sizeof(float));
          }
        }
      };
      copies(false);
      __pipeline_commit();
      copies(true);
      __pipeline_commit();
    } else {
      if (j < iters && col_live && (py || (r >= 0 && r < ny))) {
        const float* g = A.src + static_cast<long long>(gr) * A.pitch + gx;
        float* sa = l0a + (j % S::A0) * 3 * RS + col + 2;
        float* sb = l0b + (j % S::B0) * S::BP * RS + col + 2;
        float* sc = l0c + (j % S::C0) * S::CP * RS + col + 2;
        if (!split) {
#pragma unroll
          for (int p = 0; p < 13; ++p) {
            float* d = grp(p) == 0 ? sa : (grp(p) == 1 ? sb : sc);
            __pipeline_memcpy_async(d + idx(p) * RS, g + p * A.plane, 2 * sizeof(float));
          }
        } else {
          const float* g2 = A.src + static_cast<long long>(gr) * A.pitch + gx2;
#pragma unroll
          for (int p = 0; p < 13; ++p) {
            float* d = grp(p) == 0 ? sa : (grp(p) == 1 ? sb : sc);
            __pipeline_memcpy_async(d + idx(p) * RS, g + p * A.plane, sizeof(float));
            __pipeline_memcpy_async(d + idx(p) * RS + 1, g2 + p * A.plane, sizeof(float));
          }
        }
      }
      __pipeline_commit();
    }
  };

#pragma unroll
  for (int q = 0; q < PF; ++q) issue_row(q);
  auto iter = [&](int j, auto phc, auto fullc) {
    constexpr bool FULL = decltype(fullc)::value;  // every level's row valid, every lane computes
    // slots of the rows of iterations j, j - 1, j - 2
    constexpr int PH = decltype(phc)::value, P1 = U3 ? (PH + 2) % 3 : 1, P2 = U3 ? (PH + 1) % 3 : 2;
    // row j's first group and row j - 1's B group (SPLIT), or all of row j, have landed
    __pipeline_wait_prior(SPLIT ? 2 * PF - 1 : PF - 1);
    __syncthreads();                // ... and every thread's; iteration j - 1 is over everywhere
    if (L0R) {
      // f0 and the +y movers of the row just landed, into registers (read by level 1 one
      // and two iterations later)
      const float* rf = l0c + (j % S::C0) * S::CP * RS + col + 2;
      f0r[0][PH] = ld2(rf);
#pragma unroll
      for (int fam = 0; fam < 3; ++fam) cr[0][PH][fam] = ld2(rf + (1 + fam) * RS);
    }
    if constexpr (!PER) {
      // level 0 y sides, from the landed rows (this thread's own columns, which only this
      // thread reads before the next barrier)
      const int r = ys - K + j;
      float* ra = l0a + (j % S::A0) * 3 * RS + col + 2;
      if (col_live && !py && r == 0) {
        // the +y movers of row -1, read by level 1 as the row two back
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          if constexpr (L0R) {
            cr[0][P1][fam] = ym_ghost(fam, ld2(ra + fam * RS), cr[0][PH][fam]);
          } else {
            const float* rc = l0c + (j % S::C0) * 3 * RS + col + 2;
            st2(l0c + ((j + S::C0 - 1) % S::C0) * 3 * RS + col + 2 + fam * RS,
                ym_ghost(fam, ld2(ra + fam * RS), ld2(rc + fam * RS)));
          }
        }
      }
      if (col_live && !py && r == ny) {
        // the -y movers of row ny, read by level 1 in this iteration from the landed slot
        // (row ny is not loaded; row ny - 1's slots are not reused while no row is loaded)
        const float* ra1 = l0a + ((j + S::A0 - 1) % S::A0) * 3 * RS + col + 2;
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          const float2 p2 = L0R ? cr[0][P1][fam] : ld2(l0c + ((j + S::C0 - 1) % S::C0) * 3 * RS + col + 2 + fam * RS);
          st2(ra + fam * RS, yp_ghost(fam, ld2(ra1 + fam * RS), p2));
        }
      }
    }
    issue_row(j + PF);
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int R = ys - K + j - t;
      const bool row_ok = R >= ys - K + t && R < ye + K - t;
      const bool row_live = py || (R >= 0 && R < ny);
      if (FULL ? warp_live : (row_ok && row_live && col_live && col + 1 >= t && col < w + K + KL - t)) {
        float2 f[13];
        if (t == 1 && L0R) {
          const float* ra = l0a + (j % S::A0) * 3 * RS + col + 2;                 // row R + 1
          const float* rb = l0b + ((j + S::B0 - 1) % S::B0) * 6 * RS + col + 2;  // row R
          f[0] = f0r[0][P1];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            const float* px = rb + (2 * fam) * RS;      // +x movers from columns 2c - 1, 2c
            const float* mx = rb + (2 * fam + 1) * RS;  // -x movers from columns 2c + 1, 2c + 2
            f[2 + 4 * fam] = cr[0][P2][fam];
            f[4 + 4 * fam] = ld2(ra + fam * RS);
            pull_x(fam, px, mx, f);
          }
        } else if (t == 1) {
          const float* ra = l0a + (j % S::A0) * 3 * RS + col + 2;
          const float* rb = l0b + ((j + S::B0 - 1) % S::B0) * 7 * RS + col + 2;
          const float* rc = l0c + ((j + S::C0 - 2) % S::C0) * 3 * RS + col + 2;
          f[0] = ld2(rb);
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            const float* px = rb + (1 + 2 * fam) * RS;  // +x movers from columns 2c - 1, 2c
            const float* mx = rb + (2 + 2 * fam) * RS;  // -x movers from columns 2c + 1, 2c + 2
            f[2 + 4 * fam] = ld2(rc + fam * RS);
            f[4 + 4 * fam] = ld2(ra + fam * RS);
            pull_x(fam, px, mx, f);
          }
        } else {
          const float* x = xm(t - 1, (j + 1) & 1) + col + 2;
          f[0] = f0r[t - 1][P1];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            const float* px = x + (2 * fam) * RS;
            const float* mx = x + (2 * fam + 1) * RS;
            f[2 + 4 * fam] = cr[t - 1][P2][fam];
            f[4 + 4 * fam] = a_now[t - 1][fam];
            pull_x(fam, px, mx, f);
          }
        }
        float2 wh, wx, wy;
        collide13x2_any<MRT>(f, Kc, wh, wx, wy);
        if (STORE_W && R >= ys && R < ye && col >= KL && col < KL + w && gx_raw < nx) {
          float* wp = wout + (t - 1) * wslot + static_cast<long long>(R) * A.pitch + gx_raw;
          if (!lane_y_out) {
            st2(wp, wh);
            st2(wp + A.plane, wx);
            st2(wp + 2 * A.plane, wy);
          } else {
            wp[0] = wh.x;
            wp[A.plane] = wx.x;
            wp[2 * A.plane] = wy.x;
          }
        }
        if (t < K) {
          float* x = xm(t, j & 1) + col + 2;
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            st2(x + (2 * fam) * RS, f[1 + 4 * fam]);
            st2(x + (2 * fam + 1) * RS, f[3 + 4 * fam]);
            a_now[t][fam] = f[4 + 4 * fam];
            cr[t][PH][fam] = f[2 + 4 * fam];
          }
          f0r[t][PH] = f[0];
          if constexpr (!PER) {
            if (!py && R == 0) {
              // row -1's +y movers: aged into the row two back by the time level t + 1 pulls row 0
#pragma unroll
              for (int fam = 0; fam < 3; ++fam) cr[t][P1][fam] = ym_ghost(fam, f[4 + 4 * fam], f[2 + 4 * fam]);
            }
          }
        } else if (col >= KL && col < KL + w && gx_raw < nx) {
          float* g = A.dst + static_cast<long long>(R) * A.pitch + gx_raw;
          if (!lane_y_out) {
#pragma unroll
            for (int p = 0; p < 13; ++p) st2(g + p * A.plane, f[p]);
          } else {
#pragma unroll
            for (int p = 0; p < 13; ++p) g[p * A.plane] = f[p].x;
          }
        }
      } else if (!PER && t < K && !py && R == ny) {
        // row ny's -y movers, pulled by level t + 1 in this iteration; a_now / c_now still hold
        // row ny - 1
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) a_now[t][fam] = yp_ghost(fam, a_now[t][fam], cr[t][P1][fam]);
      }
      if constexpr (!U3) {
        // level t - 1's rows move down a slot once level t has read them
        if (t > 1 || L0R) {
          f0r[t - 1][1] = f0r[t - 1][0];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            cr[t - 1][2][fam] = cr[t - 1][1][fam];
            cr[t - 1][1][fam] = cr[t - 1][0][fam];
          }
        }
      }
    }
  };
  if constexpr (U3) {
    // extra iterations past iters compute and load nothing (their rows are out of range)
    const int iters3 = (iters + 2) / 3 * 3;
    using F0 = std::integral_constant<bool, false>;
    using F1 = std::integral_constant<bool, true>;
    int j = 0;
    if constexpr (STEADY && PER) {
      for (; j < 2 * K; j += 3) {  // fill: a level whose first row is not reached yet
        iter(j, std::integral_constant<int, 0>{}, F0{});
        iter(j + 1, std::integral_constant<int, 1>{}, F0{});
        iter(j + 2, std::integral_constant<int, 2>{}, F0{});
      }
      for (; j + 2 < iters; j += 3) {  // steady state: j in [2K, iters)
        iter(j, std::integral_constant<int, 0>{}, F1{});
        iter(j + 1, std::integral_constant<int, 1>{}, F1{});
        iter(j + 2, std::integral_constant<int, 2>{}, F1{});
      }
    }
    for (; j < iters3; j += 3) {
      iter(j, std::integral_constant<int, 0>{}, F0{});
      iter(j + 1, std::integral_constant<int, 1>{}, F0{});
      iter(j + 2, std::integral_constant<int, 2>{}, F0{});
    }
  } else {
    int j = 0;
    if constexpr (STEADY && PER) {
      for (; j < 2 * K; ++j) iter(j, std::integral_constant<int, 0>{}, std::integral_constant<bool, false>{});
      for (; j < iters; ++j) iter(j, std::integral_constant<int, 0>{}, std::integral_constant<bool, true>{});
    }
    for (; j < iters; ++j) iter(j, std::integral_constant<int, 0>{}, std::integral_constant<bool, false>{});
  }
  __pipeline_wait_prior(0);
}

}  // namespace
}  // namespace lbm
