// Allocation-free diagnostics: the FP64 totals / health check of lbm_sw_diagnostics
// for callers that may not allocate device memory when they need the check.
//
// The pass-1 partials live in a file-scope device array instead of memory the caller
// or the library allocates.  In host code `g_noalloc_partials` names a host-side
// stand-in, not a device address, so every call looks up its device address in the
// current context (cudaGetSymbolAddress) and hands that to the kernels.  The lookup is not
// cached: after a device reset, or in another context of the same device, the runtime loads
// the module again at another address, and a cached pointer would go stale.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int kMaxRows = LBM_SW_NOALLOC_MAX_ROWS;  // one pass-1 partial per row

// 5 doubles (sum h, sum hu, sum hv, min h, bad cells) per row: 8192 * 5 * 8 = 327,680
// bytes.  Every device that loads the library holds this array until the process
// exits.  Pass 1 of a call writes the partial of every row it reduces before the
// final pass of that call reads it, so nothing has to start at zero; calls that
// overlap on the GPU share the array and race.
static __device__ __align__(256) double g_noalloc_partials[kMaxRows * 5];

// Device address of g_noalloc_partials in the current context (the first call in a
// context loads the module there).
cudaError_t partials_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

template <class T>
int run(const void* populations, int q, int nx, int ny, size_t row_pitch, size_t plane_pitch, double* out,
        cudaStream_t st) {
  double* partials = nullptr;
  if (partials_on_current_device(&partials) != cudaSuccess) return LBM_SW_E_CUDA;
  lbm::StepArgs<T> a;
  a.src = static_cast<const T*>(populations);
  a.dst = nullptr;
  a.inflow_feq = nullptr;
  a.nx = nx;
  a.ny = ny;
  a.pitch = static_cast<long long>(row_pitch);
  a.plane = static_cast<long long>(plane_pitch);
  for (int s = 0; s < 4; ++s) a.bc[s] = LBM_SW_BC_PERIODIC;
  return lbm::launch_diagnostics_blocks<T>(a, q, ny, partials, out, st) == cudaSuccess ? LBM_SW_OK
                                                                                        : LBM_SW_E_CUDA;
}

}  // namespace

extern "C" int lbm_sw_diagnostics_noalloc(const void* populations, int dim, int precision, int nx, int ny,
                                          size_t row_pitch, size_t plane_pitch, double* out, void* stream) {
  if (!populations || !out) return LBM_SW_E_ARG;
  if (dim != 1 && dim != 2) return LBM_SW_E_ARG;
  if (precision != LBM_SW_FP32 && precision != LBM_SW_FP64) return LBM_SW_E_ARG;
  if (nx < 1 || ny < 1 || (dim == 1 && ny != 1)) return LBM_SW_E_ARG;
  if (ny > kMaxRows) return LBM_SW_E_ARG;  // more rows than the static scratch holds
  if (row_pitch < static_cast<size_t>(nx) || plane_pitch < row_pitch * static_cast<size_t>(ny))
    return LBM_SW_E_ARG;
  const int q = dim == 1 ? 5 : 13;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == LBM_SW_FP64 ? run<double>(populations, q, nx, ny, row_pitch, plane_pitch, out, st)
                                  : run<float>(populations, q, nx, ny, row_pitch, plane_pitch, out, st);
}
