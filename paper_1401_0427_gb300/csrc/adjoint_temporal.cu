// K reverse steps of the discrete adjoint per launch (temporal blocking of the adjoint
// recurrence of adjoint.cu), FP32, all-periodic domains.
#include <cuda_pipeline.h>
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

}  // namespace

bool adjoint_temporal_supported(const StepArgs<float>& a, int k) {
  bool per = true;
  for (int s = 0; s < 4; ++s) per = per && a.bc[s] == LBM_SW_BC_PERIODIC;
  return per && (k == 2 || k == 4 || k == 6 || k == 8);
}

cudaError_t launch_adjoint_temporal(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                                    int k, cudaStream_t st, int sm_count) {
  if (!adjoint_temporal_supported(a, k)) return cudaErrorNotSupported;
  switch (k) {
    case 2: return launch_adjoint_k<2>(a, w0, wslot, kd, st, sm_count);
    case 6: return launch_adjoint_k<6>(a, w0, wslot, kd, st, sm_count);
    case 8: return launch_adjoint_k<8>(a, w0, wslot, kd, st, sm_count);
    default: return launch_adjoint_k<4>(a, w0, wslot, kd, st, sm_count);
  }
}

}  // namespace lbm
