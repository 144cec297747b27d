// C ABI of the library (declarations and contracts in include/lbm_sw.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"
#include "launch_plan.h"

namespace {

// Smallest 2D FP32 grid (cells) that AUTO steps with temporal blocking: 640^2 ran 10 .. 37 %
// faster fused (K = 4) than one step per launch, 512^2 with a wall and an inflow side 19 %
// slower.
constexpr long long kAutoTemporalCells = 3LL << 17;

int fail(lbm_sw* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

int cuda_fail(lbm_sw* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? LBM_SW_E_NOMEM : LBM_SW_E_CUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

#define LBM_CUDA(h, call, what)                       \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

size_t state_bytes(const lbm_sw* h) { return static_cast<size_t>(h->q) * h->plane * h->elem; }

template <class T>
lbm::StepArgs<T> args(const lbm_sw* h, int src_buf) {
  return lbm::handle_args<T>(h, src_buf);
}

lbm::ConstsD consts(const lbm_sw* h) { return lbm::handle_consts(h); }

// Whether lbm_sw_step fuses temporal_k steps per launch: FP32 2D TEMPORAL handles without
// obstacles, with the BGK collision or with MRT where the two-column kernel applies.
bool temporal_active(const lbm_sw* h) {
  if (h->p.dim != 2 || h->kernel != LBM_SW_KERNEL_TEMPORAL || h->p.precision != LBM_SW_FP32 || h->has_obstacles)
    return false;
  if (!h->mrt) return true;
  // MRT: the two-column kernel's K; under AUTO from 2^19 cells (868^2 with walls and inflow:
  // +14 % fused at K = 4; 724^2 even, 628^2 -12 %)
  const bool large = static_cast<long long>(h->p.nx) * h->p.ny >= (1LL << 19);
  return lbm::temporal_mrt_supported(h->p.bc, h->p.nx, h->temporal_k) && (large || !h->auto_kernel);
}

// Launch plan of a fused handle (launch_plan.h): K, and whether odd sizes above one may run
// (BGK with every side periodic: the paired kernel with an even left halo at K = 3 and 5 on
// large grids, else the one-column kernel).
int plan_fused_launches(const lbm_sw* h, int n, int* plan, int max_plan) {
  const bool odd_ok = !h->mrt && h->p.bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC &&
                      h->p.bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  return lbm::plan_launches(h->temporal_k, odd_ok, n, plan, max_plan);
}
static_assert(64 > lbm::kMaxTail, "plan buffers of lbm_sw_step and lbm_sw_step_plan hold a whole tail");

// One step from buffer `from` into the other buffer, on stream st (the TEMPORAL choice
// takes single steps with the VEC kernel).
cudaError_t launch_one_step(lbm_sw* h, int from, cudaStream_t st) {
  const int variant = h->kernel == LBM_SW_KERNEL_TEMPORAL ? LBM_SW_KERNEL_VEC : h->kernel;
  if (h->has_obstacles)
    return h->p.precision == LBM_SW_FP64
               ? lbm::launch_step2d_obstacle<double>(args<double>(h, from), consts(h), h->solid, variant, st)
               : lbm::launch_step2d_obstacle<float>(args<float>(h, from), consts(h), h->solid, variant, st);
  if (h->p.precision == LBM_SW_FP64) {
    auto a = args<double>(h, from);
    return h->p.dim == 1 ? lbm::launch_step1d<double>(a, consts(h), st)
                         : lbm::launch_step2d<double>(a, consts(h), variant, st);
  }
  auto a = args<float>(h, from);
  return h->p.dim == 1 ? lbm::launch_step1d<float>(a, consts(h), st)
                       : lbm::launch_step2d<float>(a, consts(h), variant, st);
}

// Capture graph_chunk steps starting from buffer `from` (graph_chunk is even, so the
// chunk ends in the buffer it started from).
int build_graph(lbm_sw* h, int from) {
  if (!h->capture_stream)
    LBM_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  LBM_CUDA(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cudaError_t le = cudaSuccess;
  int b = from;
  for (int i = 0; i < h->graph_chunk && le == cudaSuccess; ++i, b ^= 1) le = launch_one_step(h, b, h->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, le, "step launch during graph capture");
  }
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&h->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return cuda_fail(h, ie, "cudaGraphInstantiate");
  return LBM_SW_OK;
}

int validate(const lbm_sw_params* p, lbm_sw* h) {
  if (p->dim != 1 && p->dim != 2) return fail(h, LBM_SW_E_ARG, "dim must be 1 or 2 (got %d)", p->dim);
  if (p->nx < 1 || p->ny < 1) return fail(h, LBM_SW_E_ARG, "nx and ny must be >= 1 (got %d, %d)", p->nx, p->ny);
  if (p->dim == 1 && p->ny != 1) return fail(h, LBM_SW_E_ARG, "ny must be 1 when dim == 1");
  if (p->nx > (1 << 30) || p->ny > (1 << 30)) return fail(h, LBM_SW_E_ARG, "nx, ny must be <= 2^30");
  if (p->precision != LBM_SW_FP32 && p->precision != LBM_SW_FP64)
    return fail(h, LBM_SW_E_ARG, "precision must be LBM_SW_FP32 or LBM_SW_FP64");
  if (!(p->g > 0) || !std::isfinite(p->g)) return fail(h, LBM_SW_E_ARG, "g must be finite and > 0");
  if (!(p->lambda > 0) || !std::isfinite(p->lambda)) return fail(h, LBM_SW_E_ARG, "lambda must be finite and > 0");
  if (!(p->s >= 0 && p->s < 2)) return fail(h, LBM_SW_E_ARG, "s must be in [0, 2)");
  if (!(p->a >= 0) || !std::isfinite(p->a)) return fail(h, LBM_SW_E_ARG, "a must be finite and >= 0");
  const int nsides = p->dim == 1 ? 2 : 4;
  for (int s = 0; s < nsides; ++s) {
    if (p->bc[s] < LBM_SW_BC_PERIODIC || p->bc[s] > LBM_SW_BC_INFLOW)
      return fail(h, LBM_SW_E_ARG, "bc[%d] = %d is not a LBM_SW_BC_* value", s, p->bc[s]);
    if (p->bc[s] == LBM_SW_BC_INFLOW) {
      if (!(p->inflow[s][0] > 0) || !std::isfinite(p->inflow[s][0]) || !std::isfinite(p->inflow[s][1]) ||
          !std::isfinite(p->inflow[s][2]))
        return fail(h, LBM_SW_E_ARG, "inflow[%d] must be finite with depth > 0", s);
    }
  }
  for (int pair = 0; pair < nsides; pair += 2)
    if ((p->bc[pair] == LBM_SW_BC_PERIODIC) != (p->bc[pair + 1] == LBM_SW_BC_PERIODIC))
      return fail(h, LBM_SW_E_ARG, "periodic sides come in pairs (bc[%d], bc[%d])", pair, pair + 1);
  if (p->kernel < LBM_SW_KERNEL_AUTO || p->kernel > LBM_SW_KERNEL_TEMPORAL)
    return fail(h, LBM_SW_E_ARG, "kernel must be a LBM_SW_KERNEL_* value");
  if ((p->dim == 2 && p->kernel == LBM_SW_KERNEL_CLUSTER) ||
      (p->dim == 1 && (p->kernel == LBM_SW_KERNEL_VEC || p->kernel == LBM_SW_KERNEL_TEMPORAL)))
    return fail(h, LBM_SW_E_ARG, "kernel: CLUSTER is for 1D handles, VEC and TEMPORAL for 2D handles");
  if (p->temporal_steps != 0 && !lbm::temporal_steps_supported(p->temporal_steps))
    return fail(h, LBM_SW_E_ARG, "temporal_steps must be 0 or 2 .. 8");
  for (int r = 0; r < 5; ++r)
    if (p->reserved[r] != 0) return fail(h, LBM_SW_E_ARG, "reserved fields must be zero");
  return LBM_SW_OK;
}

thread_local std::string g_create_error;

}  // namespace

namespace lbm {
void set_create_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace lbm

extern "C" {

int lbm_sw_abi_version(void) { return LBM_SW_ABI_VERSION; }

const char* lbm_sw_status_string(int status) {
  switch (status) {
    case LBM_SW_OK: return "ok";
    case LBM_SW_E_ARG: return "invalid argument";
    case LBM_SW_E_CUDA: return "CUDA error";
    case LBM_SW_E_UNSTABLE: return "unstable state (NaN/Inf or depth <= 0)";
    case LBM_SW_E_STATE: return "call not valid in the current state";
    case LBM_SW_E_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

int lbm_sw_params_init(lbm_sw_params* p) {
  if (!p) return LBM_SW_E_ARG;
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->precision = LBM_SW_FP32;
  p->g = 1.0;
  p->lambda = 8.0;
  p->s = 1.8;
  p->a = 0.05;
  for (int s = 0; s < 4; ++s) {
    p->bc[s] = LBM_SW_BC_PERIODIC;
    p->inflow[s][0] = 1.0;
  }
  p->kernel = LBM_SW_KERNEL_AUTO;
  return LBM_SW_OK;
}

const char* lbm_sw_last_error(const lbm_sw* h) { return h ? h->err.c_str() : "null handle"; }

const char* lbm_sw_create_error(void) { return g_create_error.c_str(); }

void lbm_sw_destroy(lbm_sw* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int i = 0; i < 2; ++i) {
    if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
    if (h->buf[i]) cudaFree(h->buf[i]);
  }
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->inflow_feq) cudaFree(h->inflow_feq);
  if (h->moments_staging) cudaFree(h->moments_staging);
  if (h->pop_staging) cudaFree(h->pop_staging);
  if (h->diag_partials) cudaFree(h->diag_partials);
  if (h->diag_out) cudaFree(h->diag_out);
  if (h->diag_host) cudaFreeHost(h->diag_host);
  if (h->solid) cudaFree(h->solid);
  delete h;
}

int lbm_sw_create(const lbm_sw_params* p, lbm_sw** out) {
  if (!out) return LBM_SW_E_ARG;
  *out = nullptr;
  if (!p) return LBM_SW_E_ARG;
  lbm_sw* h = new (std::nothrow) lbm_sw;
  if (!h) return LBM_SW_E_NOMEM;
  g_create_error.clear();
  int rc = validate(p, h);
  if (rc != LBM_SW_OK) {
    g_create_error = h->err;  // the handle is not returned: keep the message per thread
    delete h;
    return rc;
  }
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(p->stream);
  h->q = p->dim == 1 ? 5 : 13;
  h->elem = p->precision == LBM_SW_FP64 ? 8 : 4;
  h->pitch = round_up(p->nx, 32);
  h->plane = round_up(h->pitch * p->ny, 64);  // 256-byte aligned planes in FP32 and FP64
  const bool all_periodic = p->bc[LBM_SW_SIDE_XM] == LBM_SW_BC_PERIODIC && p->bc[LBM_SW_SIDE_YM] == LBM_SW_BC_PERIODIC;
  // default steps per fused launch: 4 below 2^20 cells (shorter wavefront fill), else 6
  const long long cells = static_cast<long long>(p->nx) * p->ny;
  h->temporal_k = p->temporal_steps ? p->temporal_steps : (cells < (1LL << 20) ? 4 : 6);
  h->auto_kernel = p->kernel == LBM_SW_KERNEL_AUTO;
  if (p->dim == 2) {
    // AUTO: temporal blocking where it was measured faster (FP32, at least 3 * 2^17 cells,
    // all sides periodic or the two-column kernel: even K), otherwise one vectorised step
    // per launch
    const int k = h->temporal_k;
    const bool temporal = p->precision == LBM_SW_FP32 && (all_periodic || k % 2 == 0) && cells >= kAutoTemporalCells;
    h->kernel = p->kernel == LBM_SW_KERNEL_AUTO ? (temporal ? LBM_SW_KERNEL_TEMPORAL : LBM_SW_KERNEL_VEC) : p->kernel;
  } else {
    h->kernel = p->kernel == LBM_SW_KERNEL_AUTO ? LBM_SW_KERNEL_CLUSTER : p->kernel;
  }
  h->graph_chunk = p->graph_chunk == 0 ? 64 : (p->graph_chunk < 0 ? 0 : p->graph_chunk + (p->graph_chunk & 1));

  auto bail = [&](int code) {
    g_create_error = std::string("create: ") + lbm_sw_status_string(code) + ": " +
                     cudaGetErrorString(cudaGetLastError());
    lbm_sw_destroy(h);
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return bail(LBM_SW_E_CUDA);
  if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    return bail(LBM_SW_E_CUDA);
  const size_t bytes = state_bytes(h);
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&h->buf[i], bytes) != cudaSuccess) return bail(LBM_SW_E_NOMEM);
    if (cudaMemsetAsync(h->buf[i], 0, bytes, h->stream) != cudaSuccess) return bail(LBM_SW_E_CUDA);
  }
  if (cudaMalloc(&h->inflow_feq, 4 * h->q * h->elem) != cudaSuccess) return bail(LBM_SW_E_NOMEM);
  if (cudaMalloc(&h->diag_partials, 5 * sizeof(double) * lbm::diag_max_blocks()) != cudaSuccess)
    return bail(LBM_SW_E_NOMEM);
  if (cudaMalloc(&h->diag_out, 8 * sizeof(double)) != cudaSuccess) return bail(LBM_SW_E_NOMEM);
  if (cudaMallocHost(&h->diag_host, 8 * sizeof(double)) != cudaSuccess) return bail(LBM_SW_E_NOMEM);
  cudaError_t e;
  if (p->precision == LBM_SW_FP64)
    e = p->dim == 1 ? lbm::launch_inflow_feq1d<double>(static_cast<double*>(h->inflow_feq), p->bc, p->inflow, consts(h), h->stream)
                    : lbm::launch_inflow_feq2d<double>(static_cast<double*>(h->inflow_feq), p->bc, p->inflow, consts(h), h->stream);
  else
    e = p->dim == 1 ? lbm::launch_inflow_feq1d<float>(static_cast<float*>(h->inflow_feq), p->bc, p->inflow, consts(h), h->stream)
                    : lbm::launch_inflow_feq2d<float>(static_cast<float*>(h->inflow_feq), p->bc, p->inflow, consts(h), h->stream);
  if (e != cudaSuccess) return bail(LBM_SW_E_CUDA);
  h->launches += 1;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(LBM_SW_E_CUDA);
  *out = h;
  return LBM_SW_OK;
}

int lbm_sw_set_state(lbm_sw* h, const double* depth, const double* hu, const double* hv, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (!depth || !hu || (h->p.dim == 2 && !hv && on_device))
    return fail(h, LBM_SW_E_ARG, "set_state: depth and hu are required (and hv for device input in 2D)");
  const size_t n = static_cast<size_t>(h->p.nx) * h->p.ny;
  const double *d = depth, *u = hu, *v = (h->p.dim == 2) ? hv : nullptr;
  if (!on_device) {
    if (!h->moments_staging)
      LBM_CUDA(h, cudaMalloc(&h->moments_staging, 3 * n * sizeof(double)), "cudaMalloc(moments staging)");
    double* s = h->moments_staging;
    LBM_CUDA(h, cudaMemcpyAsync(s, depth, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy h");
    LBM_CUDA(h, cudaMemcpyAsync(s + n, hu, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy hu");
    if (h->p.dim == 2) {
      if (hv)
        LBM_CUDA(h, cudaMemcpyAsync(s + 2 * n, hv, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy hv");
      else
        LBM_CUDA(h, cudaMemsetAsync(s + 2 * n, 0, n * sizeof(double), h->stream), "zero hv");
    }
    d = s;
    u = s + n;
    v = h->p.dim == 2 ? s + 2 * n : nullptr;
  }
  cudaError_t e;
  // the equilibrium is written into the current buffer (as the destination of "args")
  const int from = 1 - h->cur;
  if (h->p.precision == LBM_SW_FP64)
    e = h->p.dim == 1 ? lbm::launch_init1d<double>(args<double>(h, from), consts(h), d, u, h->stream)
                      : lbm::launch_init2d<double>(args<double>(h, from), consts(h), d, u, v, h->stream);
  else
    e = h->p.dim == 1 ? lbm::launch_init1d<float>(args<float>(h, from), consts(h), d, u, h->stream)
                      : lbm::launch_init2d<float>(args<float>(h, from), consts(h), d, u, v, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state kernel launch");
  h->launches += 1;
  if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_state synchronize");
  h->has_state = true;
  h->steps_done = 0;
  return LBM_SW_OK;
}

int lbm_sw_step(lbm_sw* h, int n) {
  if (!h) return LBM_SW_E_ARG;
  if (n < 0) return fail(h, LBM_SW_E_ARG, "step: n must be >= 0 (got %d)", n);
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "step: no state set (call set_state or set_populations)");
  if (h->p.dim == 1 && h->kernel == LBM_SW_KERNEL_CLUSTER && n > 0) {
    const bool fp64 = h->p.precision == LBM_SW_FP64;
    const int max_cells = fp64 ? lbm::cluster1d_max_cells<double>() : lbm::cluster1d_max_cells<float>();
    if (h->p.nx <= max_cells) {
      cudaError_t e = fp64 ? lbm::launch_step1d_cluster<double>(args<double>(h, h->cur), consts(h), n, h->stream)
                           : lbm::launch_step1d_cluster<float>(args<float>(h, h->cur), consts(h), n, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "cluster step launch");
      h->cur ^= 1;
      h->steps_done += n;
      h->launches += 1;
      return LBM_SW_OK;
    }
  }
  if (temporal_active(h)) {
    int plan[64];
    while (n > 0) {
      const int count = plan_fused_launches(h, n, plan, 64);
      for (int i = 0; i < count; ++i) {
        const int k = plan[i];
        cudaError_t e;
        if (k == 1) {  // one step per launch (the vectorised kernel; FP32 here)
          e = lbm::launch_step2d<float>(args<float>(h, h->cur), consts(h), LBM_SW_KERNEL_VEC, h->stream);
        } else {
          e = h->mrt ? lbm::launch_step2d_temporal_mrt(args<float>(h, h->cur), consts(h), k, h->stream, h->sm_count)
                     : lbm::launch_step2d_temporal(args<float>(h, h->cur), consts(h), k, h->stream, h->sm_count);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, k == 1 ? "step kernel launch" : "temporal step launch");
        h->cur ^= 1;
        n -= k;
        h->steps_done += k;
        h->launches += 1;
      }
    }
    return LBM_SW_OK;
  }
  while (n > 0) {
    if (h->graph_chunk > 0 && n >= h->graph_chunk) {
      if (!h->graph[h->cur]) {
        int rc = build_graph(h, h->cur);
        if (rc != LBM_SW_OK) return rc;
      }
      LBM_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->stream), "cudaGraphLaunch");
      n -= h->graph_chunk;
      h->steps_done += h->graph_chunk;
      h->launches += h->graph_chunk;
    } else {
      cudaError_t e = launch_one_step(h, h->cur, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
      h->cur ^= 1;
      n -= 1;
      h->steps_done += 1;
      h->launches += 1;
    }
  }
  return LBM_SW_OK;
}

int lbm_sw_step_plan(const lbm_sw* h, int n, int* sizes, int max_sizes) {
  if (!h || n < 0 || max_sizes < 0 || (max_sizes > 0 && !sizes)) return LBM_SW_E_ARG;
  int count = 0;
  auto put = [&](int k) {
    if (count < max_sizes) sizes[count] = k;
    ++count;
  };
  if (n == 0) return 0;
  if (h->p.dim == 1 && h->kernel == LBM_SW_KERNEL_CLUSTER) {
    const int max_cells = h->p.precision == LBM_SW_FP64 ? lbm::cluster1d_max_cells<double>()
                                                        : lbm::cluster1d_max_cells<float>();
    if (h->p.nx <= max_cells) {
      put(n);
      return count;
    }
  }
  if (temporal_active(h)) {
    int plan[64];
    while (n > 0) {
      const int c = plan_fused_launches(h, n, plan, 64);
      for (int i = 0; i < c; ++i) {
        put(plan[i]);
        n -= plan[i];
      }
    }
    return count;
  }
  for (int i = 0; i < n; ++i) put(1);
  return count;
}

int lbm_sw_get_moments(lbm_sw* h, double* depth, double* hu, double* hv, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (!depth || !hu) return fail(h, LBM_SW_E_ARG, "get_moments: depth and hu are required");
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "get_moments: no state set");
  const size_t n = static_cast<size_t>(h->p.nx) * h->p.ny;
  double *d = depth, *u = hu, *v = (h->p.dim == 2) ? hv : nullptr;
  if (!on_device) {
    if (!h->moments_staging)
      LBM_CUDA(h, cudaMalloc(&h->moments_staging, 3 * n * sizeof(double)), "cudaMalloc(moments staging)");
    d = h->moments_staging;
    u = d + n;
    v = (h->p.dim == 2 && hv) ? d + 2 * n : nullptr;
  }
  cudaError_t e;
  const int from = h->cur;
  if (h->p.precision == LBM_SW_FP64)
    e = h->p.dim == 1 ? lbm::launch_moments1d<double>(args<double>(h, from), d, u, h->stream)
                      : lbm::launch_moments2d<double>(args<double>(h, from), d, u, v, h->stream);
  else
    e = h->p.dim == 1 ? lbm::launch_moments1d<float>(args<float>(h, from), d, u, h->stream)
                      : lbm::launch_moments2d<float>(args<float>(h, from), d, u, v, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel launch");
  h->launches += 1;
  if (!on_device) {
    LBM_CUDA(h, cudaMemcpyAsync(depth, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy h");
    LBM_CUDA(h, cudaMemcpyAsync(hu, u, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy hu");
    if (v) LBM_CUDA(h, cudaMemcpyAsync(hv, v, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy hv");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_moments synchronize");
  }
  return LBM_SW_OK;
}

int lbm_sw_diagnostics(lbm_sw* h, double out[4]) {
  if (!h || !out) return h ? fail(h, LBM_SW_E_ARG, "diagnostics: out is NULL") : LBM_SW_E_ARG;
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "diagnostics: no state set");
  cudaError_t e = h->p.precision == LBM_SW_FP64
                      ? lbm::launch_diagnostics<double>(args<double>(h, h->cur), h->q, h->diag_partials, h->diag_out, h->stream)
                      : lbm::launch_diagnostics<float>(args<float>(h, h->cur), h->q, h->diag_partials, h->diag_out, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics kernel launch");
  h->launches += 2;
  LBM_CUDA(h, cudaMemcpyAsync(h->diag_host, h->diag_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "copy diagnostics");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "diagnostics synchronize");
  for (int k = 0; k < 4; ++k) out[k] = h->diag_host[k];
  if (h->diag_host[4] > 0)
    return fail(h, LBM_SW_E_UNSTABLE, "diagnostics: %.0f cells with NaN/Inf or depth <= 0", h->diag_host[4]);
  return LBM_SW_OK;
}

int lbm_sw_get_populations(lbm_sw* h, void* dst, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (!dst) return fail(h, LBM_SW_E_ARG, "get_populations: dst is NULL");
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "get_populations: no state set");
  const size_t row = static_cast<size_t>(h->p.nx) * h->elem;
  const size_t dplane = row * h->p.ny;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const char* src = static_cast<const char*>(h->buf[h->cur]);
  for (int p = 0; p < h->q; ++p)
    LBM_CUDA(h, cudaMemcpy2DAsync(static_cast<char*>(dst) + p * dplane, row, src + p * h->plane * h->elem,
                                  h->pitch * h->elem, row, h->p.ny, kind, h->stream),
             "copy populations out");
  if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_populations synchronize");
  return LBM_SW_OK;
}

int lbm_sw_set_populations(lbm_sw* h, const void* src, int on_device, int form) {
  if (!h) return LBM_SW_E_ARG;
  if (!src) return fail(h, LBM_SW_E_ARG, "set_populations: src is NULL");
  if (form != LBM_SW_POST_COLLISION && form != LBM_SW_PRE_COLLISION)
    return fail(h, LBM_SW_E_ARG, "set_populations: form must be LBM_SW_POST_COLLISION or LBM_SW_PRE_COLLISION");
  const size_t row = static_cast<size_t>(h->p.nx) * h->elem;
  const size_t dplane = row * h->p.ny;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (form == LBM_SW_POST_COLLISION) {
    char* dst = static_cast<char*>(h->buf[h->cur]);
    for (int p = 0; p < h->q; ++p)
      LBM_CUDA(h, cudaMemcpy2DAsync(dst + p * h->plane * h->elem, h->pitch * h->elem,
                                    static_cast<const char*>(src) + p * dplane, row, row, h->p.ny, kind, h->stream),
               "copy populations in");
  } else {
    const void* dense = src;
    if (!on_device) {
      if (!h->pop_staging)
        LBM_CUDA(h, cudaMalloc(&h->pop_staging, h->q * dplane), "cudaMalloc(population staging)");
      LBM_CUDA(h, cudaMemcpyAsync(h->pop_staging, src, h->q * dplane, cudaMemcpyHostToDevice, h->stream),
               "copy populations in");
      dense = h->pop_staging;
    }
    const int from = 1 - h->cur;  // write into the current buffer
    cudaError_t e;
    if (h->p.precision == LBM_SW_FP64)
      e = h->p.dim == 1 ? lbm::launch_collide1d_dense<double>(args<double>(h, from), consts(h), static_cast<const double*>(dense), h->stream)
                        : lbm::launch_collide2d_dense<double>(args<double>(h, from), consts(h), static_cast<const double*>(dense),
                                                              h->has_obstacles ? h->solid : nullptr, h->stream);
    else
      e = h->p.dim == 1 ? lbm::launch_collide1d_dense<float>(args<float>(h, from), consts(h), static_cast<const float*>(dense), h->stream)
                        : lbm::launch_collide2d_dense<float>(args<float>(h, from), consts(h), static_cast<const float*>(dense),
                                                             h->has_obstacles ? h->solid : nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide kernel launch");
    h->launches += 1;
  }
  if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_populations synchronize");
  h->has_state = true;
  h->steps_done = 0;
  return LBM_SW_OK;
}

int lbm_sw_get_rows(lbm_sw* h, int y0, int nrows, void* dst, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (!dst) return fail(h, LBM_SW_E_ARG, "get_rows: dst is NULL");
  if (h->p.dim != 2) return fail(h, LBM_SW_E_ARG, "get_rows: rows are for 2D handles");
  if (y0 < 0 || nrows < 0 || y0 > h->p.ny - nrows)
    return fail(h, LBM_SW_E_ARG, "get_rows: rows [%d, %d) outside [0, %d)", y0, y0 + nrows, h->p.ny);
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "get_rows: no state set");
  if (nrows == 0) return LBM_SW_OK;
  const size_t row = static_cast<size_t>(h->p.nx) * h->elem;
  const size_t dplane = row * nrows;
  const char* src = static_cast<const char*>(h->buf[h->cur]) + static_cast<size_t>(y0) * h->pitch * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int p = 0; p < h->q; ++p)
    LBM_CUDA(h, cudaMemcpy2DAsync(static_cast<char*>(dst) + p * dplane, row, src + p * h->plane * h->elem,
                                  h->pitch * h->elem, row, nrows, kind, h->stream),
             "copy rows out");
  if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_rows synchronize");
  return LBM_SW_OK;
}

int lbm_sw_set_rows(lbm_sw* h, int y0, int nrows, const void* src, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (!src) return fail(h, LBM_SW_E_ARG, "set_rows: src is NULL");
  if (h->p.dim != 2) return fail(h, LBM_SW_E_ARG, "set_rows: rows are for 2D handles");
  if (y0 < 0 || nrows < 0 || y0 > h->p.ny - nrows)
    return fail(h, LBM_SW_E_ARG, "set_rows: rows [%d, %d) outside [0, %d)", y0, y0 + nrows, h->p.ny);
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "set_rows: no state set");
  if (nrows == 0) return LBM_SW_OK;
  const size_t row = static_cast<size_t>(h->p.nx) * h->elem;
  const size_t dplane = row * nrows;
  char* dst = static_cast<char*>(h->buf[h->cur]) + static_cast<size_t>(y0) * h->pitch * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int p = 0; p < h->q; ++p)
    LBM_CUDA(h, cudaMemcpy2DAsync(dst + p * h->plane * h->elem, h->pitch * h->elem,
                                  static_cast<const char*>(src) + p * dplane, row, row, nrows, kind, h->stream),
             "copy rows in");
  if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_rows synchronize");
  return LBM_SW_OK;
}

int lbm_sw_diagnostics_rows(lbm_sw* h, int y0, int nrows, double out[4]) {
  if (!h || !out) return h ? fail(h, LBM_SW_E_ARG, "diagnostics_rows: out is NULL") : LBM_SW_E_ARG;
  if (y0 < 0 || nrows < 1 || y0 > h->p.ny - nrows)
    return fail(h, LBM_SW_E_ARG, "diagnostics_rows: rows [%d, %d) outside [0, %d)", y0, y0 + nrows, h->p.ny);
  if (!h->has_state) return fail(h, LBM_SW_E_STATE, "diagnostics_rows: no state set");
  cudaError_t e;
  if (h->p.precision == LBM_SW_FP64) {
    auto a = args<double>(h, h->cur);
    a.src += static_cast<long long>(y0) * h->pitch;
    a.ny = nrows;
    e = lbm::launch_diagnostics<double>(a, h->q, h->diag_partials, h->diag_out, h->stream);
  } else {
    auto a = args<float>(h, h->cur);
    a.src += static_cast<long long>(y0) * h->pitch;
    a.ny = nrows;
    e = lbm::launch_diagnostics<float>(a, h->q, h->diag_partials, h->diag_out, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics kernel launch");
  h->launches += 2;
  LBM_CUDA(h, cudaMemcpyAsync(h->diag_host, h->diag_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "copy diagnostics");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "diagnostics synchronize");
  for (int k = 0; k < 4; ++k) out[k] = h->diag_host[k];
  if (h->diag_host[4] > 0)
    return fail(h, LBM_SW_E_UNSTABLE, "diagnostics: %.0f cells with NaN/Inf or depth <= 0", h->diag_host[4]);
  return LBM_SW_OK;
}

int lbm_sw_set_relaxation(lbm_sw* h, const double* rates, int count) {
  if (!h) return LBM_SW_E_ARG;
  if (!rates) {
    h->mrt = false;
  } else {
    const int want = h->p.dim == 1 ? 5 : 13;
    if (count != want) return fail(h, LBM_SW_E_ARG, "set_relaxation: %d rates expected (got %d)", want, count);
    static const int map2[10] = {1, 2, 3, 4, 6, 7, 8, 10, 11, 12};
    static const int map1[3] = {1, 2, 4};
    const int n = h->p.dim == 1 ? 3 : 10;
    const int* map = h->p.dim == 1 ? map1 : map2;
    for (int i = 0; i < n; ++i) {
      const double r = rates[map[i]];
      if (!(r >= 0.0 && r < 2.0)) return fail(h, LBM_SW_E_ARG, "set_relaxation: rate %d = %g is not in [0, 2)", map[i], r);
    }
    for (int i = 0; i < 10; ++i) h->mrt_rates[i] = i < n ? rates[map[i]] : 0.0;
    h->mrt = true;
  }
  // the captured graphs hold the old constants
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
  return LBM_SW_OK;
}

int lbm_sw_set_obstacle(lbm_sw* h, const unsigned char* solid, int on_device) {
  if (!h) return LBM_SW_E_ARG;
  if (h->p.dim != 2) return fail(h, LBM_SW_E_ARG, "set_obstacle: obstacles are for 2D handles");
  if (!solid) {
    h->has_obstacles = false;
  } else {
    const size_t n = static_cast<size_t>(h->p.nx) * h->p.ny;
    if (!h->solid) LBM_CUDA(h, cudaMalloc(&h->solid, n), "cudaMalloc (obstacle mask)");
    LBM_CUDA(h, cudaMemcpyAsync(h->solid, solid, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                h->stream), "obstacle mask copy");
    // the caller may reuse its buffer when this returns
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_obstacle synchronize");
    h->has_obstacles = true;
  }
  // the captured graphs hold the previous step kernel
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
  return LBM_SW_OK;
}

int lbm_sw_synchronize(lbm_sw* h) {
  if (!h) return LBM_SW_E_ARG;
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_SW_OK;
}

int lbm_sw_get_info(const lbm_sw* h, lbm_sw_info* out) {
  if (!h || !out) return LBM_SW_E_ARG;
  out->q = h->q;
  out->kernel = h->kernel;
  if (h->p.dim == 1 && h->kernel == LBM_SW_KERNEL_CLUSTER) {
    const int max_cells = h->p.precision == LBM_SW_FP64 ? lbm::cluster1d_max_cells<double>()
                                                        : lbm::cluster1d_max_cells<float>();
    if (h->p.nx > max_cells) out->kernel = LBM_SW_KERNEL_SIMPLE;
  }
  out->pitch = static_cast<size_t>(h->pitch);
  out->population_bytes = static_cast<size_t>(h->q) * h->p.nx * h->p.ny * h->elem;
  out->bytes_per_update = 2.0 * h->q * static_cast<double>(h->elem);
  out->steps_done = h->steps_done;
  out->kernel_launches = h->launches;
  out->steps_per_launch = 1;
  if (out->kernel == LBM_SW_KERNEL_CLUSTER) out->steps_per_launch = 0;
  if (temporal_active(h)) out->steps_per_launch = h->temporal_k;
  return LBM_SW_OK;
}

}  // extern "C"
