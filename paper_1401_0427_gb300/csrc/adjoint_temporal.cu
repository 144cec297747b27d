// K reverse steps of the discrete adjoint per launch (temporal blocking of the adjoint
// recurrence of adjoint.cu), FP32: all-periodic domains, and any sides with an even nx.
#include <cuda_pipeline.h>
#include <type_traits>
#include <cuda_runtime.h>

#include "internal.h"
#include "scheme.cuh"
#include "temporal.cuh"

namespace lbm {

// K reverse steps of the discrete adjoint per launch on an all-periodic domain:
// Phi^{n-1} = J_C(W^{n-1})^T S^T Phi^n, where the transposed pull S^T reads population q
// of the cell the forward step sent it to (+x movers from column c + 1, -x movers from
// c - 1, +y movers from row R + 1, -y movers from row R - 1) and J_C^T psi =
// (1 - s) psi + s M^T D(W)^T psi.  Level 0 is Phi^{n0} (A.src), level t is Phi^{n0 - t},
// level K goes to A.dst; level t reads the moments W^{n0 - t} at w0 - (t - 1) * wslot.
// The wavefront is the forward one with the roles of the y movers swapped: the +y movers
// are read from the newest row (registers), the -y movers two rows later.  The rows of
// moments each level needs land by cp.async with the input row, two iterations ahead.
__host__ __device__ constexpr int adj_group(int p) {
  return (p == 2 || p == 6 || p == 10) ? 0 : ((p == 4 || p == 8 || p == 12) ? 2 : 1);
}
__host__ __device__ constexpr int adj_index(int p) {
  return adj_group(p) == 0 ? (p - 2) / 4 : (adj_group(p) == 2 ? (p - 4) / 4 : (p == 0 ? 0 : (p + 1) / 2));
}

template <int K, int COLS>
__device__ __forceinline__ void adjoint_wave(const StepArgs<float>& A, const float* __restrict__ w0, long long wslot,
                                             const Consts<float>& Kc, float* smem, int x0, int w, int ys, int ye) {
  using S = PeriodicShape<K, COLS>;
  const int c = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  float* const l0a = smem;
  float* const l0b = l0a + S::A0 * 3 * COLS;
  float* const l0c = l0b + S::B0 * 7 * COLS;
  auto xm = [&](int t, int slot) { return smem + S::L0_FLOATS + (t - 1) * S::LV_FLOATS + slot * 6 * COLS; };
  // moments of every level, prefetched like the input rows: [K][3 rows][3 planes][COLS]
  auto wr = [&](int t, int slot) { return smem + S::floats() + ((t - 1) * 3 + slot) * 3 * COLS; };
  const int gx_raw = x0 - K + c;
  const bool in_tile = c < w + 2 * K;
  const int gx = ((gx_raw % nx) + nx) % nx;
  const int iters = (ye - ys) + 2 * K;
  const float oms = 1.0f - Kc.s;

  // level t as the input of level t + 1: the +y movers of the row computed now, f0 of the
  // previous row, the -y movers of the previous two rows (stale where not computed)
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
        float* d = adj_group(p) == 0 ? sa : (adj_group(p) == 1 ? sb : sc);
        __pipeline_memcpy_async(d + adj_index(p) * COLS, g + p * A.plane, sizeof(float));
      }
      // the moments level t will read at iteration j (row r - t)
#pragma unroll
      for (int t = 1; t <= K; ++t) {
        const int rt = ((r - t) % ny + ny) % ny;
        const float* gw = w0 - (t - 1) * wslot + static_cast<long long>(rt) * A.pitch + gx;
        float* d = wr(t, j % 3) + c;
#pragma unroll
        for (int q = 0; q < 3; ++q) __pipeline_memcpy_async(d + q * COLS, gw + q * A.plane, sizeof(float));
      }
    }
    __pipeline_commit();
  };

  issue_row(0);
  issue_row(1);
  for (int j = 0; j < iters; ++j) {
    __pipeline_wait_prior(1);
    __syncthreads();
    issue_row(j + 2);
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int R = ys - K + j - t;
      const bool row_ok = R >= ys - K + t && R < ye + K - t;
      if (row_ok && c >= t && c < w + 2 * K - t) {
        const float* wp = wr(t, j % 3) + c;
        const float wh = wp[0], wx = wp[COLS], wy = wp[2 * COLS];
        float psi[13];
        if (t == 1) {
          const float* ra = l0a + (j % S::A0) * 3 * COLS + c;                 // row R + 1
          const float* rb = l0b + ((j + S::B0 - 1) % S::B0) * 7 * COLS + c;  // row R
          const float* rc = l0c + ((j + S::C0 - 2) % S::C0) * 3 * COLS + c;  // row R - 1
          psi[0] = rb[0];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            psi[1 + 4 * fam] = rb[(1 + 2 * fam) * COLS + 1];
            psi[2 + 4 * fam] = ra[fam * COLS];
            psi[3 + 4 * fam] = rb[(2 + 2 * fam) * COLS - 1];
            psi[4 + 4 * fam] = rc[fam * COLS];
          }
        } else {
          const float* x = xm(t - 1, (j + 1) & 1) + c;
          psi[0] = f0_prev[t - 1];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            psi[1 + 4 * fam] = x[(2 * fam) * COLS + 1];
            psi[2 + 4 * fam] = a_now[t - 1][fam];
            psi[3 + 4 * fam] = x[(2 * fam + 1) * COLS - 1];
            psi[4 + 4 * fam] = c_prev2[t - 1][fam];
          }
        }
        float zh, zx, zy;
        equilibrium_vjp(wh, wx, wy, psi, Kc, zh, zx, zy);
        float out[13];
#pragma unroll
        for (int q = 0; q < 13; ++q) out[q] = oms * psi[q] + Kc.s * (q < 5 ? zh : (q < 9 ? zx : zy));
        if (t < K) {
          float* x = xm(t, j & 1) + c;
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            x[(2 * fam) * COLS] = out[1 + 4 * fam];
            x[(2 * fam + 1) * COLS] = out[3 + 4 * fam];
            a_now[t][fam] = out[2 + 4 * fam];
            c_now[t][fam] = out[4 + 4 * fam];
          }
          f0_now[t] = out[0];
        } else if (c >= K && c < K + w && gx_raw < nx) {
          float* g = A.dst + static_cast<long long>(R) * A.pitch + gx_raw;
#pragma unroll
          for (int p = 0; p < 13; ++p) g[p * A.plane] = out[p];
        }
      }
      if (t > 1) {
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
__global__ void __launch_bounds__(COLS, 2)
    adjoint_temporal_periodic(const StepArgs<float> A, const float* __restrict__ w0, long long wslot,
                              const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    adjoint_wave<K, COLS>(A, w0, wslot, Kc, smem, strip * P.w, P.w, ys, ye);
  });
}

// ---- Two columns per thread ----
// The same reverse wavefront with tile columns 2c and 2c + 1 in one thread and the local
// product J_C^T on FP32 pairs.  Shared memory per CTA: the input ring (the +y movers read
// in the landing iteration, f0 and the x movers one iteration later, the -y movers two
// later, each with PF rows in flight), two rows of x movers per intermediate level, and
// the moment rows of every level (1 + PF rows each).  Rows carry two pad floats each side,
// so the x-shifted reads of the edge pairs stay in bounds.
template <int K, int COLS, int PF>
struct AdjPairShape {
  static constexpr int RS = COLS + 4;
  static constexpr int A0 = 1 + PF, B0 = 2 + PF, C0 = 3 + PF, W0 = 1 + PF;
  static constexpr int L0_FLOATS = RS * (3 * A0 + 7 * B0 + 3 * C0);
  static constexpr int LV_FLOATS = RS * 2 * 6;
  static constexpr int W_FLOATS = RS * 3 * W0;  // per level
  static constexpr size_t floats() {
    return static_cast<size_t>(L0_FLOATS) + (K - 1) * LV_FLOATS + static_cast<size_t>(K) * W_FLOATS;
  }
};

// z = D(W)^T psi on a pair of cells (the products of equilibrium_vjp, contracted freely).
__device__ __forceinline__ void equilibrium_vjp_x2(float2 h, float2 qx, float2 qy, const float2 psi[13],
                                                   const Consts<float>& K, float2& zh, float2& zx, float2& zy) {
  const float2 nz = dup2(K.nz);
  auto mul = [&](float2 a, float2 b) { return fma2(a, b, nz); };
  const float2 rh = make_float2(recip(h.x), recip(h.y));
  const float2 u = mul(qx, rh), v = mul(qy, rh);
  const float2 gh = mul(dup2(2.0f * K.half_g), h);
  const float2 inv2gh = mul(dup2(2.0f * K.inv4g), rh);
  const float2 uu = mul(u, u), vv = mul(v, v);
  const float2 kh = fma2(add2(uu, vv), inv2gh, dup2(0.5f));
  const float2 kx = mul(make_float2(-u.x, -u.y), inv2gh);
  const float2 ky = mul(make_float2(-v.x, -v.y), inv2gh);
  const float2 Sf = add2(add2(psi[1], psi[3]), add2(psi[2], psi[4]));
  const float2 Af = fma2(dup2(-0.25f), Sf, psi[0]);
  const float2 Df13 = sub2(psi[1], psi[3]), Df24 = sub2(psi[2], psi[4]);
  const float2 Sx = add2(add2(psi[5], psi[7]), add2(psi[6], psi[8]));
  const float2 Dx13 = sub2(psi[5], psi[7]), Dx24 = sub2(psi[6], psi[8]);
  const float2 Sy = add2(add2(psi[9], psi[11]), add2(psi[10], psi[12]));
  const float2 Dy13 = sub2(psi[9], psi[11]), Dy24 = sub2(psi[10], psi[12]);
  const float2 X = add2(Dx24, Dy13);
  const float2 c = dup2(K.c), a = dup2(K.a), q = dup2(0.25f);
  // zh = a kh Af + Sf / 4 + c (Dx13 (gh - u u) - X u v + Dy24 (gh - v v))
  float2 t = mul(Dx13, sub2(gh, uu));
  t = fma2(make_float2(-X.x, -X.y), mul(u, v), t);
  t = fma2(Dy24, sub2(gh, vv), t);
  zh = fma2(c, t, fma2(mul(a, kh), Af, mul(q, Sf)));
  // zx = a kx Af + c Df13 + Sx / 4 + c (2 Dx13 u + X v)
  t = fma2(add2(Dx13, Dx13), u, mul(X, v));
  zx = fma2(c, add2(Df13, t), fma2(mul(a, kx), Af, mul(q, Sx)));
  // zy = a ky Af + c Df24 + Sy / 4 + c (X u + 2 Dy24 v)
  t = fma2(X, u, mul(add2(Dy24, Dy24), v));
  zy = fma2(c, add2(Df24, t), fma2(mul(a, ky), Af, mul(q, Sy)));
}

// PER: every side periodic.  Otherwise (even nx) the sides that are not periodic apply the
// transposed rules of the one-step adjoint (adjoint.cu reverse_pull): a population whose
// forward destination lies beyond a WALL takes the cell's own mirror partner (times -1 for
// the family normal to the wall), beyond OUTFLOW or INFLOW nothing; and where the side
// behind a cell is OUTFLOW, the cell's own value of the population is added (the forward
// ghost copied it).  x sides: the edge lane reads the mirror partner through a per-lane
// offset (with the sign as an exact product) or the zero-filled column outside the domain,
// and adds its own value where the side behind is OUTFLOW.  y sides: the register (or input
// ring) rows that the next level pulls for the first and last rows get the rule's values.
template <int K, int COLS, int PF, bool PER = true>
__device__ __forceinline__ void adjoint_pair_wave(const StepArgs<float>& A, const float* __restrict__ w0,
                                                  long long wslot, const Consts<float>& Kc, float* smem, int x0,
                                                  int w, int ys, int ye) {
  using S = AdjPairShape<K, COLS, PF>;
  constexpr int RS = S::RS;
  const int c = threadIdx.x;  // pair index: tile columns 2c, 2c + 1
  const int col = 2 * c;
  const int nx = A.nx, ny = A.ny;
  float* const l0a = smem;
  float* const l0b = l0a + S::A0 * 3 * RS;
  float* const l0c = l0b + S::B0 * 7 * RS;
  auto xm = [&](int t, int slot) { return smem + S::L0_FLOATS + (t - 1) * S::LV_FLOATS + slot * 6 * RS; };
  auto wr = [&](int t, int slot) {
    return smem + S::L0_FLOATS + (K - 1) * S::LV_FLOATS + (t - 1) * S::W_FLOATS + slot * 3 * RS;
  };
  auto ld2 = [](const float* q) { return *reinterpret_cast<const float2*>(q); };
  auto st2 = [](float* q, float2 v) { *reinterpret_cast<float2*>(q) = v; };
  const int gx_raw = x0 - K + col;
  const bool px_ = PER || A.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC;
  const bool py = PER || A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  const bool col_live = col < w + 2 * K && (px_ || (gx_raw >= 0 && gx_raw < nx));
  const int gx = px_ ? ((gx_raw % nx) + nx) % nx : gx_raw;
  const bool at_xm = !px_ && gx_raw == 0;           // lane .x is the domain's first column
  const bool at_xp = !px_ && gx_raw + 1 == nx - 1;  // lane .y is its last
  const int iters = (ye - ys) + 2 * K;
  const float2 oms = dup2(1.0f - Kc.s), sv = dup2(Kc.s);
  const float2 zero = make_float2(0.f, 0.f);

  // level t as the input of level t + 1 (as adjoint_wave, on pairs)
  float2 a_now[K][3], f0_now[K], c_now[K][3], f0_prev[K], c_prev1[K][3], c_prev2[K][3];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    f0_now[t] = f0_prev[t] = zero;
#pragma unroll
    for (int q = 0; q < 3; ++q) a_now[t][q] = c_now[t][q] = c_prev1[t][q] = c_prev2[t][q] = zero;
  }

  // x sides: offsets of the pulled +x movers' lane .y (normally 2) and the -x movers' lane
  // .x (normally -1) from the plane pointers at this pair, their signs, and the additions
  int o_a = 2, o_b = -1;
  float sgn_a = 1.f, sgn_b = 1.f;
  bool add_xm = false, add_xp = false;
  if constexpr (!PER) {
    const int bm = A.bc[LBM_SW_SIDE_XM], bp = A.bc[LBM_SW_SIDE_XP];
    if (at_xp && bp == LBM_SW_BC_WALL) {
      o_a = RS + 1;  // own -x mover of the last column
      sgn_a = -1.f;  // (applied to the hu family only)
    }
    if (at_xm && bm == LBM_SW_BC_WALL) {
      o_b = -RS;  // own +x mover of the first column
      sgn_b = -1.f;
    }
    add_xm = at_xm && bm == LBM_SW_BC_OUTFLOW;
    add_xp = at_xp && bp == LBM_SW_BC_OUTFLOW;
    // the columns just outside the domain read as zero (nothing else writes there)
    if (at_xm || at_xp) {
      for (int fam = 0; fam < 3; ++fam) {
        for (int q = 0; q < S::B0; ++q) {
          float* rb = l0b + q * 7 * RS + col + 2;
          if (at_xm) rb[(2 + 2 * fam) * RS - 1] = 0.f;
          if (at_xp) rb[(1 + 2 * fam) * RS + 2] = 0.f;
        }
        for (int t = 1; t < K; ++t)
          for (int q = 0; q < 2; ++q) {
            float* x = xm(t, q) + col + 2;
            if (at_xm) x[(2 * fam + 1) * RS - 1] = 0.f;
            if (at_xp) x[(2 * fam) * RS + 2] = 0.f;
          }
      }
    }
  }
  // the transposed pull of the x movers of family fam from the +x / -x planes at this pair
  auto pull_x = [&](int fam, const float* px, const float* mx, float2* psi) {
    if constexpr (PER) {
      psi[1 + 4 * fam] = make_float2(px[1], px[2]);  // from columns 2c + 1, 2c + 2
      psi[3 + 4 * fam] = make_float2(mx[-1], mx[0]);  // from columns 2c - 1, 2c
    } else {
      psi[1 + 4 * fam] = make_float2(px[1], px[o_a]);
      psi[3 + 4 * fam] = make_float2(mx[o_b], mx[0]);
      if (fam == 1) {
        psi[5].y *= sgn_a;
        psi[7].x *= sgn_b;
      }
      if (add_xm) psi[1 + 4 * fam].x += px[0];
      if (add_xp) psi[3 + 4 * fam].y += mx[1];
    }
  };
  // y sides: the -y movers of row -1 (from row 0's +y movers p2) and the +y movers of row ny
  // (from row ny - 1's -y movers p4) that the pulls of rows 0 and ny - 1 read
  auto ym_ghost = [&](int fam, float2 p2) {
    return A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_WALL ? (fam == 2 ? make_float2(-p2.x, -p2.y) : p2) : zero;
  };
  auto yp_ghost = [&](int fam, float2 p4) {
    return A.bc[LBM_SW_SIDE_YP] == LBM_SW_BC_WALL ? (fam == 2 ? make_float2(-p4.x, -p4.y) : p4) : zero;
  };
  const bool out_ym = !py && A.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_OUTFLOW;
  const bool out_yp = !py && A.bc[LBM_SW_SIDE_YP] == LBM_SW_BC_OUTFLOW;

  // rows land in order, one per call of issue_row: with periodic y sides the wrapped row
  // advances by one per call, and the rows of the moments read by each level follow it
  int next_gr = py ? ((ys - K) % ny + ny) % ny : 0;
  auto issue_row = [&](int j) {
    const int r = ys - K + j;
    const int gr = py ? next_gr : r;
    if (py) next_gr = next_gr + 1 == ny ? 0 : next_gr + 1;
    if (j < iters && col_live && (py || (r >= 0 && r < ny))) {
      const float* g = A.src + static_cast<long long>(gr) * A.pitch + gx;
      float* sa = l0a + (j % S::A0) * 3 * RS + col + 2;
      float* sb = l0b + (j % S::B0) * 7 * RS + col + 2;
      float* sc = l0c + (j % S::C0) * 3 * RS + col + 2;
#pragma unroll
      for (int p = 0; p < 13; ++p) {
        float* d = adj_group(p) == 0 ? sa : (adj_group(p) == 1 ? sb : sc);
        __pipeline_memcpy_async(d + adj_index(p) * RS, g + p * A.plane, 2 * sizeof(float));
      }
    }
    if (j < iters && col_live) {
      // the moments level t reads at iteration j (row r - t)
#pragma unroll
      for (int t = 1; t <= K; ++t) {
        const int rt0 = r - t;
        if (py || (rt0 >= 0 && rt0 < ny)) {
          const int rt = !py ? rt0 : (ny > K ? (gr >= t ? gr - t : gr - t + ny) : (rt0 % ny + ny) % ny);
          const float* gw = w0 - (t - 1) * wslot + static_cast<long long>(rt) * A.pitch + gx;
          float* d = wr(t, j % S::W0) + col + 2;
#pragma unroll
          for (int q = 0; q < 3; ++q) __pipeline_memcpy_async(d + q * RS, gw + q * A.plane, 2 * sizeof(float));
        }
      }
    }
    __pipeline_commit();
  };

#pragma unroll
  for (int q = 0; q < PF; ++q) issue_row(q);
  const bool warp_live = __any_sync(0xffffffffu, col_live);
  auto iter = [&](int j, auto fullc) {
    constexpr bool FULL = decltype(fullc)::value;  // every level's row valid, every lane computes
    __pipeline_wait_prior(PF - 1);
    __syncthreads();
    if constexpr (!PER) {
      // level 0's y sides in the landed rows (this thread's own columns, which only this
      // thread reads before the next barrier; the slots of the previous row are still
      // intact because the next copy is issued below)
      const int r = ys - K + j;
      if (col_live && !py) {
        float* ra = l0a + (j % S::A0) * 3 * RS + col + 2;                    // +y movers of row r
        float* ra1 = l0a + ((j + S::A0 - 1) % S::A0) * 3 * RS + col + 2;     // of row r - 1
        float* rc = l0c + (j % S::C0) * 3 * RS + col + 2;                    // -y movers of row r
        float* rc1 = l0c + ((j + S::C0 - 1) % S::C0) * 3 * RS + col + 2;     // of row r - 1
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          if (r == 0) st2(rc1 + fam * RS, ym_ghost(fam, ld2(ra + fam * RS)));
          if (r == ny) st2(ra + fam * RS, yp_ghost(fam, ld2(rc1 + fam * RS)));
          if (out_ym && r == 1) st2(ra + fam * RS, add2(ld2(ra + fam * RS), ld2(ra1 + fam * RS)));
          if (out_yp && r == ny - 1) st2(rc1 + fam * RS, add2(ld2(rc1 + fam * RS), ld2(rc + fam * RS)));
        }
      }
    }
    issue_row(j + PF);
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int R = ys - K + j - t;
      const bool row_ok = R >= ys - K + t && R < ye + K - t;
      const bool row_live = py || (R >= 0 && R < ny);
      if (FULL ? warp_live : (row_ok && row_live && col_live && col + 1 >= t && col < w + 2 * K - t)) {
        const float* wp = wr(t, j % S::W0) + col + 2;
        const float2 wh = ld2(wp), wx = ld2(wp + RS), wy = ld2(wp + 2 * RS);
        float2 psi[13];
        if (t == 1) {
          const float* ra = l0a + (j % S::A0) * 3 * RS + col + 2;                 // row R + 1
          const float* rb = l0b + ((j + S::B0 - 1) % S::B0) * 7 * RS + col + 2;  // row R
          const float* rc = l0c + ((j + S::C0 - 2) % S::C0) * 3 * RS + col + 2;  // row R - 1
          psi[0] = ld2(rb);
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            psi[2 + 4 * fam] = ld2(ra + fam * RS);
            psi[4 + 4 * fam] = ld2(rc + fam * RS);
            pull_x(fam, rb + (1 + 2 * fam) * RS, rb + (2 + 2 * fam) * RS, psi);
          }
        } else {
          const float* x = xm(t - 1, (j + 1) & 1) + col + 2;
          psi[0] = f0_prev[t - 1];
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            psi[2 + 4 * fam] = a_now[t - 1][fam];
            psi[4 + 4 * fam] = c_prev2[t - 1][fam];
            pull_x(fam, x + (2 * fam) * RS, x + (2 * fam + 1) * RS, psi);
          }
        }
        float2 zh, zx, zy;
        equilibrium_vjp_x2(wh, wx, wy, psi, Kc, zh, zx, zy);
        const float2 szh = fma2(sv, zh, dup2(Kc.nz)), szx = fma2(sv, zx, dup2(Kc.nz)),
                     szy = fma2(sv, zy, dup2(Kc.nz));
        float2 out[13];
#pragma unroll
        for (int q = 0; q < 13; ++q) out[q] = fma2(oms, psi[q], q < 5 ? szh : (q < 9 ? szx : szy));
        if (t < K) {
          float* x = xm(t, j & 1) + col + 2;
#pragma unroll
          for (int fam = 0; fam < 3; ++fam) {
            st2(x + (2 * fam) * RS, out[1 + 4 * fam]);
            st2(x + (2 * fam + 1) * RS, out[3 + 4 * fam]);
            const float2 prev = a_now[t][fam];  // row R - 1's +y movers
            a_now[t][fam] = out[2 + 4 * fam];
            c_now[t][fam] = out[4 + 4 * fam];
            if constexpr (!PER) {
              if (!py && R == 0) c_prev1[t][fam] = ym_ghost(fam, out[2 + 4 * fam]);
              if (out_yp && R == ny - 1) c_prev1[t][fam] = add2(c_prev1[t][fam], out[4 + 4 * fam]);
              if (out_ym && R == 1) a_now[t][fam] = add2(a_now[t][fam], prev);
            }
          }
          f0_now[t] = out[0];
        } else if (col >= K && col < K + w && gx_raw < nx) {
          float* g = A.dst + static_cast<long long>(R) * A.pitch + gx_raw;
#pragma unroll
          for (int p = 0; p < 13; ++p) st2(g + p * A.plane, out[p]);
        }
      } else if (!PER && t < K && !py && R == ny) {
        // row ny's +y movers, pulled by level t + 1 in this iteration (c_now still holds row
        // ny - 1's -y movers; with ny = 1 the OUTFLOW addition of row 0 too)
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          const float2 prev = a_now[t][fam];
          a_now[t][fam] = yp_ghost(fam, c_now[t][fam]);
          if (out_ym && ny == 1) a_now[t][fam] = add2(a_now[t][fam], prev);
        }
      }
      if (t > 1) {
        f0_prev[t - 1] = f0_now[t - 1];
#pragma unroll
        for (int fam = 0; fam < 3; ++fam) {
          c_prev2[t - 1][fam] = c_prev1[t - 1][fam];
          c_prev1[t - 1][fam] = c_now[t - 1][fam];
        }
      }
    }
  };
  int j = 0;
  if constexpr (PER) {
    // the iterations in which every level's row lies in its range run without the per-level
    // tests (lanes outside a level's columns compute values nothing pulls; stores keep theirs)
    for (; j < 2 * K; ++j) iter(j, std::integral_constant<bool, false>{});
    for (; j < iters; ++j) iter(j, std::integral_constant<bool, true>{});
  }
  for (; j < iters; ++j) iter(j, std::integral_constant<bool, false>{});
  __pipeline_wait_prior(0);
}

template <int K, int COLS, int PF>
__global__ void __launch_bounds__(COLS / 2, 2)
    adjoint_temporal_periodic_x2(const StepArgs<float> A, const float* __restrict__ w0, long long wslot,
                                 const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    adjoint_pair_wave<K, COLS, PF>(A, w0, wslot, Kc, smem, strip * P.w, P.w, ys, ye);
  });
  pdl_done();
}

// The same with the transposed rules of sides that are not periodic (even nx).
template <int K, int COLS, int PF>
__global__ void __launch_bounds__(COLS / 2, 2)
    adjoint_temporal_x2(const StepArgs<float> A, const float* __restrict__ w0, long long wslot,
                        const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    adjoint_pair_wave<K, COLS, PF, false>(A, w0, wslot, Kc, smem, strip * P.w, P.w, ys, ye);
  });
  pdl_done();
}

namespace {

template <int K>
cudaError_t launch_adjoint_k(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                             cudaStream_t st, int sm_count) {
  constexpr int COLS = 192;
  const size_t smem = (PeriodicShape<K, COLS>::floats() + static_cast<size_t>(K) * 3 * 3 * COLS) * sizeof(float);
  const void* fn = reinterpret_cast<const void*>(adjoint_temporal_periodic<K, COLS>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS, smem);
  const Partition P = partition(a.nx, a.ny, COLS - 2 * K, K, resident * std::max(sm_count, 1), 1);
  const Consts<float> K_ = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  adjoint_temporal_periodic<K, COLS><<<P.strips * P.segments, COLS, smem, st>>>(a, w0, wslot, K_, P);
  return cudaGetLastError();
}

template <int K, int COLS, int PF, bool PER>
cudaError_t launch_adjoint_pairs(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                                 cudaStream_t st, int sm_count) {
  const size_t smem = AdjPairShape<K, COLS, PF>::floats() * sizeof(float);
  const void* fn = PER ? reinterpret_cast<const void*>(adjoint_temporal_periodic_x2<K, COLS, PF>)
                       : reinterpret_cast<const void*>(adjoint_temporal_x2<K, COLS, PF>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS / 2, smem);
  Partition P = partition(a.nx, a.ny, COLS - 2 * K, K, resident * std::max(sm_count, 1), 1);
  P.w += P.w & 1;  // even strip width
  P.strips = (a.nx + P.w - 1) / P.w;
  const Partition Q = partition_rows(P, a.ny, K, resident * std::max(sm_count, 1), 1);
  const Consts<float> K_ = make_consts<float>(kd.g, kd.lambda, kd.s, kd.a);
  const dim3 grid(Q.strips * Q.segments), block(COLS / 2);
  if constexpr (PER)
    return launch_pdl(adjoint_temporal_periodic_x2<K, COLS, PF>, grid, block, smem, st, a, w0, wslot, K_, Q);
  else
    return launch_pdl(adjoint_temporal_x2<K, COLS, PF>, grid, block, smem, st, a, w0, wslot, K_, Q);
}

// Even widths at K <= 4 (the library's adjoint launches): two columns per thread, 192-column
// strips, two rows of prefetch (97 KB of shared memory at K = 4, two CTAs per SM; measured
// on the 1024^2 and 2048^2 inverse problems against 256 columns with one row of prefetch
// and 128 columns with two: 9-16 % and 0.5-1.5 % faster), any sides.  Otherwise one column
// per thread (every side periodic).
template <int K>
cudaError_t launch_adjoint_any(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                               cudaStream_t st, int sm_count) {
  bool per = true;
  for (int s = 0; s < 4; ++s) per = per && a.bc[s] == LBM_SW_BC_PERIODIC;
  if constexpr (K <= 4)
    if (a.nx % 2 == 0)
      return per ? launch_adjoint_pairs<K, 192, 2, true>(a, w0, wslot, kd, st, sm_count)
                 : launch_adjoint_pairs<K, 192, 2, false>(a, w0, wslot, kd, st, sm_count);
  return launch_adjoint_k<K>(a, w0, wslot, kd, st, sm_count);
}

}  // namespace

bool adjoint_temporal_supported(const StepArgs<float>& a, int k) {
  bool per = true;
  for (int s = 0; s < 4; ++s) per = per && a.bc[s] == LBM_SW_BC_PERIODIC;
  if (per) return k == 2 || k == 4 || k == 6 || k == 8;
  return a.nx % 2 == 0 && (k == 2 || k == 4);  // the two-column kernel
}

cudaError_t launch_adjoint_temporal(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                                    int k, cudaStream_t st, int sm_count) {
  if (!adjoint_temporal_supported(a, k)) return cudaErrorNotSupported;
  switch (k) {
    case 2: return launch_adjoint_any<2>(a, w0, wslot, kd, st, sm_count);
    case 6: return launch_adjoint_any<6>(a, w0, wslot, kd, st, sm_count);
    case 8: return launch_adjoint_any<8>(a, w0, wslot, kd, st, sm_count);
    default: return launch_adjoint_any<4>(a, w0, wslot, kd, st, sm_count);
  }
}

}  // namespace lbm
