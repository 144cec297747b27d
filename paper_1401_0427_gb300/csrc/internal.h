// Internal declarations shared by the library's translation units (host side).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm_sw.h"

namespace lbm {

// Direction of each 2D population: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y (Eq. 3-stencil-d2q5).
// Plane p of family k (f: 0..4, gx: 5..8, gy: 9..12) with direction d has index
// p = d for f and p = 4 + d (gx), 8 + d (gy).

// Kernel arguments of one fused step (and of the helpers that read/write states).
template <class T>
struct StepArgs {
  const T* __restrict__ src;  // post-collision populations at time n (pitched planes)
  T* __restrict__ dst;        // post-collision populations at time n + 1
  const T* inflow_feq;        // [4][q] equilibrium of each INFLOW side (device)
  int nx, ny;
  long long pitch;            // elements per row
  long long plane;            // elements per plane (pitch * ny)
  int bc[4];
};

struct ConstsD {  // scheme constants before conversion to T
  double g, lambda, s, a;
  bool mrt = false;        // relax each non-conserved moment at its own rate
  double rates[10] = {};   // MRT rates (Consts::r order); unused when mrt is false
};

// ---- 2D launchers (kernels_2d.cu) ----
template <class T>
cudaError_t launch_step2d(const StepArgs<T>& a, const ConstsD& k, int variant, cudaStream_t st);
template <class T>
cudaError_t launch_init2d(const StepArgs<T>& a, const ConstsD& k, const double* h, const double* hu,
                          const double* hv, cudaStream_t st);
template <class T>
cudaError_t launch_collide2d_dense(const StepArgs<T>& a, const ConstsD& k, const T* dense,
                                  const unsigned char* solid, cudaStream_t st);
// one step with obstacles (solid: [ny][nx] device mask, nonzero = solid); variant SIMPLE:
// one thread per cell, otherwise the vectorised row kernel
template <class T>
cudaError_t launch_step2d_obstacle(const StepArgs<T>& a, const ConstsD& k, const unsigned char* solid, int variant,
                                   cudaStream_t st);
template <class T>
cudaError_t launch_moments2d(const StepArgs<T>& a, double* h, double* hu, double* hv, cudaStream_t st);
template <class T>
cudaError_t launch_inflow_feq2d(T* out, const int bc[4], const double inflow[4][3], const ConstsD& k,
                                cudaStream_t st);

// Fused step that also writes the moments of the new state into w_out (3 planes of the
// population pitch), moments of a state into such planes, and element-wise conversion.
template <class T>
cudaError_t launch_step2d_store_w(const StepArgs<T>& a, const ConstsD& k, T* w_out, cudaStream_t st);
template <class T>
cudaError_t launch_moments2d_planes(const StepArgs<T>& a, T* w_out, cudaStream_t st);
// An FP64 checkpoint (pitched planes of a.dst's layout) restored into a.dst, with its moments
// in the three planes at w_out (as launch_moments2d_planes of the restored state).
template <class T>
cudaError_t launch_restore_moments2d(const double* ck, const StepArgs<T>& a, T* w_out, cudaStream_t st);
template <class Tin, class Tout>
cudaError_t launch_convert(const Tin* in, Tout* out, long long n, cudaStream_t st);

// K reverse steps of the discrete adjoint per launch (adjoint_temporal.cu; FP32; every side
// periodic with k in {2, 4, 6, 8}, or any sides with an even nx and k in {2, 4}): Phi^{n0}
// in a.src -> Phi^{n0 - k} in a.dst; reverse step t reads the moments W^{n0 - t} at
// w0 - (t - 1) * wslot.
bool adjoint_temporal_supported(const StepArgs<float>& a, int k);
cudaError_t launch_adjoint_temporal(const StepArgs<float>& a, const float* w0, long long wslot, const ConstsD& kd,
                                    int k, cudaStream_t st, int sm_count);

// Batched temporal blocking (temporal.cu): one wavefront unit covers rows [ys, ye) of the
// output columns [x0, x0 + w) of one instance (clipped at nx) of a batch whose sides are
// all periodic; a work list holds the units of every instance, grouped by CTA.
struct WaveUnit {
  long long offset;  // element offset of the instance's first plane in each buffer
  long long plane;   // elements per plane
  int pitch;         // elements per row
  int nx, ny;
  int x0, w;
  int ys, ye;
  int pad;
};
struct BatchWaves {
  // units of odd-width instances (one column per thread) and, for even K, of even-width
  // instances (two columns per thread); each list balanced over its own wave of CTAs
  WaveUnit* units = nullptr;  // device
  int* first = nullptr;       // device, grid + 1 entries: CTA b runs units [first[b], first[b + 1])
  int count = 0;
  int grid = 0;
  WaveUnit* punits = nullptr;
  int* pfirst = nullptr;
  int pcount = 0;
  int pgrid = 0;
};
// Build the work list of k-step wavefronts for the given instances (host arrays of count
// entries) on the current device; free with batch_waves_free.
cudaError_t batch_waves_build(int count, const int* nx, const int* ny, const long long* offset, const long long* pitch,
                              const long long* plane, int k, int sm_count, BatchWaves* out);
void batch_waves_free(BatchWaves* w);
// k fused steps of every instance: src -> dst (the batch's two buffers), under the batch's
// sides bc (sides that are not periodic need an even k; inflow_feq: [4][13] device floats).
cudaError_t launch_batch_temporal(const BatchWaves& w, int k, const float* src, float* dst, const ConstsD& kd,
                                  const int bc[4], const float* inflow_feq, cudaStream_t st);

// k fused steps per launch (temporal.cu; FP32, BGK; k in 2 .. 8): src -> dst.
bool temporal_steps_supported(int k);
// k fused steps that also write the moments of every level t = 1 .. k, for every cell, to
// the three planes at wout + (t - 1) * wslot (even k).
bool temporal_store_w_supported(const StepArgs<float>& a, int k);
cudaError_t launch_step2d_temporal_store_w(const StepArgs<float>& a, const ConstsD& kd, int k, float* wout,
                                           long long wslot, cudaStream_t st, int sm_count);
cudaError_t launch_step2d_temporal(const StepArgs<float>& a, const ConstsD& kd, int k, cudaStream_t st,
                                   int sm_count);
// The same with the MRT collision (temporal_mrt.cu; kd.mrt set; even k).
bool temporal_mrt_supported(const int bc[4], int nx, int k);
cudaError_t launch_step2d_temporal_mrt(const StepArgs<float>& a, const ConstsD& kd, int k, cudaStream_t st,
                                       int sm_count);

// ---- 1D launchers (kernels_1d.cu) ----
template <class T>
cudaError_t launch_step1d(const StepArgs<T>& a, const ConstsD& k, cudaStream_t st);
// All nsteps steps of a line in one thread-block-cluster launch (src -> dst); lines of up to
// cluster1d_max_cells<T>() cells.
template <class T>
int cluster1d_max_cells();
template <class T>
cudaError_t launch_step1d_cluster(const StepArgs<T>& a, const ConstsD& k, int nsteps, cudaStream_t st);
template <class T>
cudaError_t launch_init1d(const StepArgs<T>& a, const ConstsD& k, const double* h, const double* hu,
                          cudaStream_t st);
template <class T>
cudaError_t launch_collide1d_dense(const StepArgs<T>& a, const ConstsD& k, const T* dense, cudaStream_t st);
template <class T>
cudaError_t launch_moments1d(const StepArgs<T>& a, double* h, double* hu, cudaStream_t st);
template <class T>
cudaError_t launch_inflow_feq1d(T* out, const int bc[4], const double inflow[4][3], const ConstsD& k,
                                cudaStream_t st);

// Message returned by lbm_sw_create_error() on the calling thread (api.cu).
void set_create_error(const char* msg);

// ---- reductions (reduce.cu) ----
// Block partials (5 doubles each: sum h, sum hu, sum hv, min h, bad-cell count) then a
// fixed-order final pass into out[5].  partials must hold diag_max_blocks() * 5 doubles.
int diag_max_blocks();
template <class T>
cudaError_t launch_diagnostics(const StepArgs<T>& a, int q, double* partials, double* out, cudaStream_t st);
// Same reduction with an explicit number of pass-1 blocks (partials must hold nblocks * 5).
template <class T>
cudaError_t launch_diagnostics_blocks(const StepArgs<T>& a, int q, int nblocks, double* partials, double* out,
                                      cudaStream_t st);

}  // namespace lbm

struct lbm_sw {
  lbm_sw_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int q = 13;
  size_t elem = 4;          // sizeof(T)
  long long pitch = 0;      // elements per row
  long long plane = 0;      // elements per plane
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;              // buffer holding the current state
  void* inflow_feq = nullptr;
  double* moments_staging = nullptr;  // 3 * nx * ny doubles, for host transfers
  void* pop_staging = nullptr;        // dense populations, for host transfers / collide
  double* diag_partials = nullptr;
  double* diag_out = nullptr;         // device, 8 doubles
  double* diag_host = nullptr;        // pinned host, 8 doubles
  int kernel = LBM_SW_KERNEL_VEC;
  int temporal_k = 4;
  bool auto_kernel = false;  // the kernel was the library's choice (LBM_SW_KERNEL_AUTO)
  int sm_count = 152;
  bool mrt = false;          // set by lbm_sw_set_relaxation
  double mrt_rates[10] = {};
  unsigned char* solid = nullptr;  // obstacle mask [ny][nx] on the device (lbm_sw_set_obstacle)
  bool has_obstacles = false;
  int graph_chunk = 64;
  bool has_state = false;
  long long steps_done = 0;
  long long launches = 0;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // CUDA graph of graph_chunk steps from buffer 0 / 1
  std::string err;
};

namespace lbm {

// Kernel arguments of a step of handle h reading buffer src_buf (writing the other).
template <class T>
inline StepArgs<T> handle_args(const lbm_sw* h, int src_buf) {
  StepArgs<T> a;
  a.src = static_cast<const T*>(h->buf[src_buf]);
  a.dst = static_cast<T*>(h->buf[1 - src_buf]);
  a.inflow_feq = static_cast<const T*>(h->inflow_feq);
  a.nx = h->p.nx;
  a.ny = h->p.ny;
  a.pitch = h->pitch;
  a.plane = h->plane;
  for (int s = 0; s < 4; ++s) a.bc[s] = h->p.bc[s];
  return a;
}

inline ConstsD handle_consts(const lbm_sw* h) {
  ConstsD k{h->p.g, h->p.lambda, h->p.s, h->p.a};
  k.mrt = h->mrt;
  for (int i = 0; i < 10; ++i) k.rates[i] = h->mrt_rates[i];
  return k;
}

}  // namespace lbm
