// K fused D2Q5Q4Q4 steps per launch with the MRT collision (Eq. 2-relaxation with one rate
// per non-conserved moment), FP32: the two-column wavefront of temporal_pair.cuh with
// collide13x2_mrt, for even K.  Every cell update is the pull + collide13_mrt of the
// one-step kernels on the same values, in the same rounded operations, so K steps of this
// kernel equal K single steps bit for bit.
#include <cuda_pipeline.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "scheme.cuh"
#include "temporal.cuh"
#include "temporal_pair.cuh"

namespace lbm {
namespace {

template <int K, int COLS, int PF, bool L0R, bool PER>
__global__ void __launch_bounds__(COLS / 2, 2)
    step2d_temporal_x2_mrt(const StepArgs<float> A, const Consts<float> Kc, const Partition P) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  run_segment(P, A.ny, [&](int strip, int ys, int ye) {
    pair_wave<K, COLS, PF, false, L0R, PER, true, true, false, PER>(A, Kc, smem, strip * P.w, P.w, ys, ye, nullptr, 0);
  });
  pdl_done();
}

template <int K, int COLS, int PF, bool L0R, bool PER>
cudaError_t launch_pairs_mrt(const StepArgs<float>& a, const ConstsD& kd, cudaStream_t st, int sm_count) {
  const size_t smem = PairShape<K, COLS, PF, L0R>::floats() * sizeof(float);
  const void* fn = reinterpret_cast<const void*>(step2d_temporal_x2_mrt<K, COLS, PF, L0R, PER>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int resident = cached_resident(fn, COLS / 2, smem);
  const Partition Q = pair_partition(a.nx, a.ny, K, COLS, resident * std::max(sm_count, 1));
  const Consts<float> K_ = make_consts_mrt<float>(kd.g, kd.lambda, kd.s, kd.a, kd.rates, 10);
  return launch_pdl(step2d_temporal_x2_mrt<K, COLS, PF, L0R, PER>, dim3(Q.strips * Q.segments), dim3(COLS / 2), smem,
                    st, a, K_, Q);
}

// The shapes of the BGK kernel at each K.
template <int K>
cudaError_t launch_mrt_k(const StepArgs<float>& a, const ConstsD& kd, cudaStream_t st, int sm_count) {
  const bool per = a.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC && a.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  if constexpr (K <= 4) {
    // 128-column strips below 2^21 cells at K = 4, as the BGK kernel
    if (K == 4 && static_cast<long long>(a.nx) * a.ny < (1LL << 21))
      return per ? launch_pairs_mrt<K, 128, 2, false, true>(a, kd, st, sm_count)
                 : launch_pairs_mrt<K, 128, 2, false, false>(a, kd, st, sm_count);
    return per ? launch_pairs_mrt<K, 256, 2, false, true>(a, kd, st, sm_count)
               : launch_pairs_mrt<K, 256, 2, false, false>(a, kd, st, sm_count);
  }
  else if constexpr (K == 6) {
    // 128-column strips below 2^23 cells, as the BGK kernel (measured with MRT: +7 % at
    // 1024^2, +2 % at 2048^2, -3.5 % at 4096^2)
    if (static_cast<long long>(a.nx) * a.ny < (1LL << 23))
      return per ? launch_pairs_mrt<K, 128, 1, true, true>(a, kd, st, sm_count)
                 : launch_pairs_mrt<K, 128, 1, true, false>(a, kd, st, sm_count);
    return per ? launch_pairs_mrt<K, 256, 1, true, true>(a, kd, st, sm_count)
               : launch_pairs_mrt<K, 256, 1, true, false>(a, kd, st, sm_count);
  }
  else
    return per ? launch_pairs_mrt<K, 192, 1, false, true>(a, kd, st, sm_count)
               : launch_pairs_mrt<K, 192, 1, false, false>(a, kd, st, sm_count);
}

}  // namespace

bool temporal_mrt_supported(const int*, int, int k) { return k == 2 || k == 4 || k == 6 || k == 8; }

cudaError_t launch_step2d_temporal_mrt(const StepArgs<float>& a, const ConstsD& kd, int k, cudaStream_t st,
                                       int sm_count) {
  if (!kd.mrt || !temporal_mrt_supported(a.bc, a.nx, k)) return cudaErrorNotSupported;
  switch (k) {
    case 2: return launch_mrt_k<2>(a, kd, st, sm_count);
    case 6: return launch_mrt_k<6>(a, kd, st, sm_count);
    case 8: return launch_mrt_k<8>(a, kd, st, sm_count);
    default: return launch_mrt_k<4>(a, kd, st, sm_count);
  }
}

}  // namespace lbm
