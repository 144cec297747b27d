// Batched D2Q5Q4Q4 instances: one launch per step over a tile list that covers many
// independent grids of uneven sizes, CUDA-graph replay of long runs, and an autotuner
// for the tile shape (rows per CTA) and the schedule (one CTA per tile, or a persistent
// grid of a few CTAs per SM).  The per-row device code is the one of the single-grid kernel (step2d_vec.cuh),
// so every instance evolves bit for bit as it would in its own handle.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "launch_plan.h"
#include "scheme.cuh"
#include "step2d_vec.cuh"

namespace lbm {
namespace {

struct BatchInst {
  long long offset;  // element offset of the instance's first plane in each buffer
  long long pitch;   // elements per row
  long long plane;   // elements per plane
  int nx, ny;
  int tiles_x;       // 32-vector segments per row
  int pad;
};

struct BcSet {
  int bc[4];
};

// Work item of one CTA: BY rows of one 32-vector segment of one instance, with
// everything the CTA needs in one record (a single broadcast load per tile).
struct TileRec {
  long long offset;  // element offset of the instance's first plane
  long long plane;   // elements per plane
  int pitch;         // elements per row
  int nx, ny;
  int x0;            // first cell of the segment
  int y0;            // first row of the tile
  int pad;
};

// Persistent form: gridDim.x CTAs walk the tile list; one CTA per tile when the
// grid has as many CTAs as there are tiles.
template <class T, int BY>
__global__ void __launch_bounds__(32 * BY)
    batch_step(const TileRec* __restrict__ tiles, long long total_tiles, const T* __restrict__ src,
               T* __restrict__ dst, const T* __restrict__ inflow_feq, const BcSet bc, const Consts<T> K) {
  constexpr int V = V16<T>::n;
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    const TileRec r = tiles[t];
    const int y = r.y0 + threadIdx.y;
    if (y >= r.ny) continue;  // warp-uniform
    StepArgs<T> A;
    A.src = src + r.offset;
    A.dst = dst + r.offset;
    A.inflow_feq = inflow_feq;
    A.nx = r.nx;
    A.ny = r.ny;
    A.pitch = r.pitch;
    A.plane = r.plane;
#pragma unroll
    for (int s = 0; s < 4; ++s) A.bc[s] = bc.bc[s];
    vec_row<T, false>(A, K, y, r.x0 + threadIdx.x * V, threadIdx.x, nullptr);
  }
}

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace
}  // namespace lbm

struct lbm_sw_batch {
  lbm_sw_batch_params p{};
  std::vector<int> nx, ny;
  std::vector<lbm::BatchInst> inst;
  std::vector<char> has_state;
  int states_set = 0;
  cudaStream_t stream = nullptr;
  size_t elem = 4;
  long long total_elems = 0;  // elements per buffer
  long long cells = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  // tile lists for every tile_rows in {1, 2, 4, 8}
  lbm::TileRec* d_tiles[4] = {nullptr, nullptr, nullptr, nullptr};
  long long tiles[4] = {0, 0, 0, 0};
  void* inflow_feq = nullptr;
  double* moments_staging = nullptr;
  size_t moments_staging_cells = 0;
  double* diag_partials = nullptr;
  double* diag_out = nullptr;
  double* diag_host = nullptr;
  int sm_count = 152;
  int tile_rows = 4;
  int ctas_per_sm = 4;
  int candidates = 0;
  double tuned_ms = 0.0;
  int graph_chunk = 50;
  bool temporal_allowed = false;  // FP32
  bool temporal_auto = false;     // temporal_steps left to the library (autotune may choose)
  int temporal_k = 0;             // steps per temporal launch; 0 = one step per launch
  lbm::BatchWaves waves[9];       // work lists by K (built on first use)
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::string err;
};

namespace {

int bfail(lbm_sw_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return code;
}

int bcuda(lbm_sw_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? LBM_SW_E_NOMEM : LBM_SW_E_CUDA, "%s: %s (%s)", what,
               cudaGetErrorString(e), cudaGetErrorName(e));
}

#define BATCH_CUDA(b, call, what)                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return bcuda(b, e_, what);     \
  } while (0)

int rows_index(int rows) { return rows == 1 ? 0 : rows == 2 ? 1 : rows == 4 ? 2 : 3; }

template <class T>
lbm::StepArgs<T> inst_args(const lbm_sw_batch* b, int i, int src_buf) {
  lbm::StepArgs<T> a;
  const lbm::BatchInst& I = b->inst[i];
  a.src = static_cast<const T*>(b->buf[src_buf]) + I.offset;
  a.dst = static_cast<T*>(b->buf[1 - src_buf]) + I.offset;
  a.inflow_feq = static_cast<const T*>(b->inflow_feq);
  a.nx = I.nx;
  a.ny = I.ny;
  a.pitch = I.pitch;
  a.plane = I.plane;
  for (int s = 0; s < 4; ++s) a.bc[s] = b->p.bc[s];
  return a;
}

lbm::ConstsD bconsts(const lbm_sw_batch* b) { return lbm::ConstsD{b->p.g, b->p.lambda, b->p.s, b->p.a}; }

template <class T>
cudaError_t launch_batch_t(const lbm_sw_batch* b, int from, int rows, int ctas, cudaStream_t st) {
  const int ri = rows_index(rows);
  const long long tiles = b->tiles[ri];
  const long long want = ctas > 0 ? static_cast<long long>(b->sm_count) * ctas : tiles;  // 0: one CTA per tile
  const unsigned grid = static_cast<unsigned>(tiles < want ? tiles : want);
  lbm::BcSet bc;
  for (int s = 0; s < 4; ++s) bc.bc[s] = b->p.bc[s];
  const lbm::Consts<T> K = lbm::make_consts<T>(b->p.g, b->p.lambda, b->p.s, b->p.a);
  const T* src = static_cast<const T*>(b->buf[from]);
  T* dst = static_cast<T*>(b->buf[1 - from]);
  const T* fe = static_cast<const T*>(b->inflow_feq);
  switch (rows) {
    case 1:
      lbm::batch_step<T, 1><<<grid, dim3(32, 1), 0, st>>>(b->d_tiles[ri], tiles, src, dst, fe, bc, K);
      break;
    case 2:
      lbm::batch_step<T, 2><<<grid, dim3(32, 2), 0, st>>>(b->d_tiles[ri], tiles, src, dst, fe, bc, K);
      break;
    case 4:
      lbm::batch_step<T, 4><<<grid, dim3(32, 4), 0, st>>>(b->d_tiles[ri], tiles, src, dst, fe, bc, K);
      break;
    default:
      lbm::batch_step<T, 8><<<grid, dim3(32, 8), 0, st>>>(b->d_tiles[ri], tiles, src, dst, fe, bc, K);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch(const lbm_sw_batch* b, int from, int rows, int ctas, cudaStream_t st) {
  return b->p.precision == LBM_SW_FP64 ? launch_batch_t<double>(b, from, rows, ctas, st)
                                       : launch_batch_t<float>(b, from, rows, ctas, st);
}

int ensure_waves(lbm_sw_batch* b, int k) {
  if (b->waves[k].grid > 0) return LBM_SW_OK;
  std::vector<long long> off(b->p.count), pitch(b->p.count), plane(b->p.count);
  for (int i = 0; i < b->p.count; ++i) {
    off[i] = b->inst[i].offset;
    pitch[i] = b->inst[i].pitch;
    plane[i] = b->inst[i].plane;
  }
  BATCH_CUDA(b, lbm::batch_waves_build(b->p.count, b->nx.data(), b->ny.data(), off.data(), pitch.data(), plane.data(),
                                       k, b->sm_count, &b->waves[k]),
             "temporal work list");
  return LBM_SW_OK;
}

cudaError_t launch_temporal(const lbm_sw_batch* b, int from, int k, cudaStream_t st) {
  return lbm::launch_batch_temporal(b->waves[k], k, static_cast<const float*>(b->buf[from]),
                                    static_cast<float*>(b->buf[1 - from]), bconsts(b), b->p.bc,
                                    static_cast<const float*>(b->inflow_feq), st);
}

void drop_graphs(lbm_sw_batch* b) {
  for (int i = 0; i < 2; ++i)
    if (b->graph[i]) {
      cudaGraphExecDestroy(b->graph[i]);
      b->graph[i] = nullptr;
    }
}

int build_graph(lbm_sw_batch* b, int from) {
  if (!b->capture_stream)
    BATCH_CUDA(b, cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  BATCH_CUDA(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cudaError_t le = cudaSuccess;
  int f = from;
  for (int i = 0; i < b->graph_chunk && le == cudaSuccess; ++i, f ^= 1)
    le = launch_batch(b, f, b->tile_rows, b->ctas_per_sm, b->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(b, le, "batch step launch during graph capture");
  }
  if (ce != cudaSuccess) return bcuda(b, ce, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&b->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return bcuda(b, ie, "cudaGraphInstantiate");
  return LBM_SW_OK;
}

int check_instance(lbm_sw_batch* b, int i) {
  if (i < 0 || i >= b->p.count) return bfail(b, LBM_SW_E_ARG, "instance %d out of range [0, %d)", i, b->p.count);
  return LBM_SW_OK;
}

int ensure_staging(lbm_sw_batch* b, size_t cells) {
  if (b->moments_staging_cells >= cells) return LBM_SW_OK;
  if (b->moments_staging) cudaFree(b->moments_staging);
  b->moments_staging = nullptr;
  b->moments_staging_cells = 0;
  BATCH_CUDA(b, cudaMalloc(&b->moments_staging, 3 * cells * sizeof(double)), "cudaMalloc(moments staging)");
  b->moments_staging_cells = cells;
  return LBM_SW_OK;
}

int validate_batch(const lbm_sw_batch_params* p, lbm_sw_batch* b) {
  if (p->count < 1 || p->count > 65536) return bfail(b, LBM_SW_E_ARG, "count must be in [1, 65536] (got %d)", p->count);
  if (!p->nx || !p->ny) return bfail(b, LBM_SW_E_ARG, "nx and ny arrays are required");
  for (int i = 0; i < p->count; ++i)
    if (p->nx[i] < 1 || p->ny[i] < 1 || p->nx[i] > (1 << 20) || p->ny[i] > (1 << 20))
      return bfail(b, LBM_SW_E_ARG, "instance %d: nx, ny must be in [1, 2^20] (got %d, %d)", i, p->nx[i], p->ny[i]);
  if (p->precision != LBM_SW_FP32 && p->precision != LBM_SW_FP64)
    return bfail(b, LBM_SW_E_ARG, "precision must be LBM_SW_FP32 or LBM_SW_FP64");
  if (!(p->g > 0) || !std::isfinite(p->g)) return bfail(b, LBM_SW_E_ARG, "g must be finite and > 0");
  if (!(p->lambda > 0) || !std::isfinite(p->lambda)) return bfail(b, LBM_SW_E_ARG, "lambda must be finite and > 0");
  if (!(p->s >= 0 && p->s < 2)) return bfail(b, LBM_SW_E_ARG, "s must be in [0, 2)");
  if (!(p->a >= 0) || !std::isfinite(p->a)) return bfail(b, LBM_SW_E_ARG, "a must be finite and >= 0");
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < LBM_SW_BC_PERIODIC || p->bc[s] > LBM_SW_BC_INFLOW)
      return bfail(b, LBM_SW_E_ARG, "bc[%d] = %d is not a LBM_SW_BC_* value", s, p->bc[s]);
    if (p->bc[s] == LBM_SW_BC_INFLOW && (!(p->inflow[s][0] > 0) || !std::isfinite(p->inflow[s][0]) ||
                                          !std::isfinite(p->inflow[s][1]) || !std::isfinite(p->inflow[s][2])))
      return bfail(b, LBM_SW_E_ARG, "inflow[%d] must be finite with depth > 0", s);
  }
  for (int pair = 0; pair < 4; pair += 2)
    if ((p->bc[pair] == LBM_SW_BC_PERIODIC) != (p->bc[pair + 1] == LBM_SW_BC_PERIODIC))
      return bfail(b, LBM_SW_E_ARG, "periodic sides come in pairs (bc[%d], bc[%d])", pair, pair + 1);
  if (p->tile_rows != 0 && p->tile_rows != 1 && p->tile_rows != 2 && p->tile_rows != 4 && p->tile_rows != 8)
    return bfail(b, LBM_SW_E_ARG, "tile_rows must be 0, 1, 2, 4 or 8");
  if (p->ctas_per_sm < 0 || p->ctas_per_sm > 32) return bfail(b, LBM_SW_E_ARG, "ctas_per_sm must be in [0, 32]");
  if (p->temporal_steps < 0 || p->temporal_steps > 8)
    return bfail(b, LBM_SW_E_ARG, "temporal_steps must be in [0, 8] (got %d)", p->temporal_steps);
  if (p->temporal_steps >= 2) {
    bool per = true;
    for (int s = 0; s < 4; ++s) per = per && p->bc[s] == LBM_SW_BC_PERIODIC;
    if (p->precision != LBM_SW_FP32 || (!per && p->temporal_steps % 2))
      return bfail(b, LBM_SW_E_ARG, "temporal_steps >= 2 needs FP32, and an even value unless every side is periodic");
  }
  for (int r = 0; r < 4; ++r)
    if (p->reserved[r] != 0) return bfail(b, LBM_SW_E_ARG, "reserved fields must be zero");
  return LBM_SW_OK;
}

}  // namespace

extern "C" {

int lbm_sw_batch_params_init(lbm_sw_batch_params* p) {
  if (!p) return LBM_SW_E_ARG;
  std::memset(p, 0, sizeof(*p));
  p->precision = LBM_SW_FP32;
  p->g = 1.0;
  p->lambda = 8.0;
  p->s = 1.8;
  p->a = 0.05;
  for (int s = 0; s < 4; ++s) {
    p->bc[s] = LBM_SW_BC_PERIODIC;
    p->inflow[s][0] = 1.0;
  }
  return LBM_SW_OK;
}

const char* lbm_sw_batch_last_error(const lbm_sw_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lbm_sw_batch_destroy(lbm_sw_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (int i = 0; i < 2; ++i)
    if (b->buf[i]) cudaFree(b->buf[i]);
  for (int r = 0; r < 4; ++r)
    if (b->d_tiles[r]) cudaFree(b->d_tiles[r]);
  if (b->inflow_feq) cudaFree(b->inflow_feq);
  if (b->moments_staging) cudaFree(b->moments_staging);
  if (b->diag_partials) cudaFree(b->diag_partials);
  if (b->diag_out) cudaFree(b->diag_out);
  if (b->diag_host) cudaFreeHost(b->diag_host);
  for (int k = 0; k < 9; ++k) lbm::batch_waves_free(&b->waves[k]);
  delete b;
}

int lbm_sw_batch_create(const lbm_sw_batch_params* p, lbm_sw_batch** out) {
  if (!out) return LBM_SW_E_ARG;
  *out = nullptr;
  if (!p) return LBM_SW_E_ARG;
  lbm_sw_batch* b = new (std::nothrow) lbm_sw_batch;
  if (!b) return LBM_SW_E_NOMEM;
  lbm::set_create_error("");
  int rc = validate_batch(p, b);
  if (rc != LBM_SW_OK) {
    lbm::set_create_error(b->err.c_str());
    delete b;
    return rc;
  }
  b->p = *p;
  b->p.nx = nullptr;
  b->p.ny = nullptr;
  b->nx.assign(p->nx, p->nx + p->count);
  b->ny.assign(p->ny, p->ny + p->count);
  b->stream = static_cast<cudaStream_t>(p->stream);
  b->elem = p->precision == LBM_SW_FP64 ? 8 : 4;
  b->tile_rows = p->tile_rows ? p->tile_rows : 4;
  b->ctas_per_sm = p->ctas_per_sm;  // 0: one CTA per tile
  b->graph_chunk = p->graph_chunk == 0 ? 50 : (p->graph_chunk < 0 ? 0 : p->graph_chunk + (p->graph_chunk & 1));
  b->temporal_allowed = p->precision == LBM_SW_FP32;  // any sides (even K where not periodic)
  b->temporal_auto = p->temporal_steps == 0 && b->temporal_allowed;
  b->temporal_k = p->temporal_steps >= 2 ? p->temporal_steps : (b->temporal_auto ? 6 : 0);
  b->has_state.assign(p->count, 0);
  const int V = p->precision == LBM_SW_FP64 ? 2 : 4;

  auto bail = [&](int code, const char* what) {
    lbm::set_create_error((std::string("batch create: ") + what + ": " + cudaGetErrorString(cudaGetLastError())).c_str());
    lbm_sw_batch_destroy(b);
    return code;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(LBM_SW_E_CUDA, "cudaGetDevice");
  if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bail(LBM_SW_E_CUDA, "cudaDeviceGetAttribute");

  long long off = 0;
  b->inst.resize(p->count);
  for (int i = 0; i < p->count; ++i) {
    lbm::BatchInst& I = b->inst[i];
    I.nx = b->nx[i];
    I.ny = b->ny[i];
    I.pitch = lbm::round_up(I.nx, 32);
    I.plane = lbm::round_up(I.pitch * I.ny, 64);
    I.offset = off;
    I.tiles_x = static_cast<int>((I.nx + 32 * V - 1) / (32 * V));
    I.pad = 0;
    off += 13 * I.plane;
    b->cells += static_cast<long long>(I.nx) * I.ny;
  }
  b->total_elems = off;
  const size_t bytes = static_cast<size_t>(off) * b->elem;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&b->buf[i], bytes) != cudaSuccess) return bail(LBM_SW_E_NOMEM, "cudaMalloc(populations)");
    if (cudaMemsetAsync(b->buf[i], 0, bytes, b->stream) != cudaSuccess) return bail(LBM_SW_E_CUDA, "cudaMemset");
  }
  const int rows_list[4] = {1, 2, 4, 8};
  for (int r = 0; r < 4; ++r) {
    std::vector<lbm::TileRec> tl;
    for (int i = 0; i < p->count; ++i) {
      const lbm::BatchInst& I = b->inst[i];
      for (int y0 = 0; y0 < I.ny; y0 += rows_list[r])
        for (int bx = 0; bx < I.tiles_x; ++bx) {
          lbm::TileRec t;
          t.offset = I.offset;
          t.plane = I.plane;
          t.pitch = static_cast<int>(I.pitch);
          t.nx = I.nx;
          t.ny = I.ny;
          t.x0 = bx * 32 * V;
          t.y0 = y0;
          t.pad = 0;
          tl.push_back(t);
        }
    }
    b->tiles[r] = static_cast<long long>(tl.size());
    if (cudaMalloc(&b->d_tiles[r], sizeof(lbm::TileRec) * tl.size()) != cudaSuccess)
      return bail(LBM_SW_E_NOMEM, "cudaMalloc(tile list)");
    if (cudaMemcpy(b->d_tiles[r], tl.data(), sizeof(lbm::TileRec) * tl.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(LBM_SW_E_CUDA, "copy tile list");
  }
  if (cudaMalloc(&b->inflow_feq, 4 * 13 * b->elem) != cudaSuccess) return bail(LBM_SW_E_NOMEM, "cudaMalloc");
  if (cudaMalloc(&b->diag_partials, 5 * sizeof(double) * lbm::diag_max_blocks()) != cudaSuccess ||
      cudaMalloc(&b->diag_out, 8 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&b->diag_host, 8 * sizeof(double)) != cudaSuccess)
    return bail(LBM_SW_E_NOMEM, "cudaMalloc(diagnostics)");
  cudaError_t e = p->precision == LBM_SW_FP64
                      ? lbm::launch_inflow_feq2d<double>(static_cast<double*>(b->inflow_feq), p->bc, p->inflow, bconsts(b), b->stream)
                      : lbm::launch_inflow_feq2d<float>(static_cast<float*>(b->inflow_feq), p->bc, p->inflow, bconsts(b), b->stream);
  if (e != cudaSuccess) return bail(LBM_SW_E_CUDA, "inflow equilibria");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(LBM_SW_E_CUDA, "synchronize");
  *out = b;
  return LBM_SW_OK;
}

int lbm_sw_batch_set_state(lbm_sw_batch* b, int i, const double* depth, const double* hu, const double* hv,
                           int on_device) {
  if (!b) return LBM_SW_E_ARG;
  int rc = check_instance(b, i);
  if (rc) return rc;
  if (!depth || !hu || (!hv && on_device)) return bfail(b, LBM_SW_E_ARG, "set_state: depth, hu (and hv on device) are required");
  const size_t n = static_cast<size_t>(b->nx[i]) * b->ny[i];
  const double *d = depth, *u = hu, *v = hv;
  if (!on_device) {
    rc = ensure_staging(b, n);
    if (rc) return rc;
    double* s = b->moments_staging;
    BATCH_CUDA(b, cudaMemcpyAsync(s, depth, n * sizeof(double), cudaMemcpyHostToDevice, b->stream), "copy h");
    BATCH_CUDA(b, cudaMemcpyAsync(s + n, hu, n * sizeof(double), cudaMemcpyHostToDevice, b->stream), "copy hu");
    if (hv)
      BATCH_CUDA(b, cudaMemcpyAsync(s + 2 * n, hv, n * sizeof(double), cudaMemcpyHostToDevice, b->stream), "copy hv");
    else
      BATCH_CUDA(b, cudaMemsetAsync(s + 2 * n, 0, n * sizeof(double), b->stream), "zero hv");
    d = s;
    u = s + n;
    v = s + 2 * n;
  }
  const int from = 1 - b->cur;  // init writes the current buffer
  cudaError_t e = b->p.precision == LBM_SW_FP64
                      ? lbm::launch_init2d<double>(inst_args<double>(b, i, from), bconsts(b), d, u, v, b->stream)
                      : lbm::launch_init2d<float>(inst_args<float>(b, i, from), bconsts(b), d, u, v, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "set_state kernel launch");
  if (!on_device) BATCH_CUDA(b, cudaStreamSynchronize(b->stream), "set_state synchronize");
  if (!b->has_state[i]) {
    b->has_state[i] = 1;
    b->states_set += 1;
  }
  return LBM_SW_OK;
}

int lbm_sw_batch_step(lbm_sw_batch* b, int n) {
  if (!b) return LBM_SW_E_ARG;
  if (n < 0) return bfail(b, LBM_SW_E_ARG, "step: n must be >= 0 (got %d)", n);
  if (b->states_set != b->p.count)
    return bfail(b, LBM_SW_E_STATE, "step: %d of %d instances have no state", b->p.count - b->states_set, b->p.count);
  if (b->temporal_k >= 2) {
    // as lbm_sw_step: launches of K, the tail split into shorter fused launches (each with
    // its own work list, built on first use), odd sizes only where every side is periodic
    bool per = true;
    for (int s = 0; s < 4; ++s) per = per && b->p.bc[s] == LBM_SW_BC_PERIODIC;
    int plan[64];
    while (n > 0) {
      const int count = lbm::plan_launches(b->temporal_k, per, n, plan, 64);
      for (int i = 0; i < count; ++i) {
        const int k = plan[i];
        cudaError_t e;
        if (k == 1) {
          e = launch_batch(b, b->cur, b->tile_rows, b->ctas_per_sm, b->stream);
        } else {
          const int rc = ensure_waves(b, k);
          if (rc) return rc;
          e = launch_temporal(b, b->cur, k, b->stream);
        }
        if (e != cudaSuccess) return bcuda(b, e, k == 1 ? "batch step launch" : "batch temporal launch");
        b->cur ^= 1;
        n -= k;
      }
    }
    return LBM_SW_OK;
  }
  while (n > 0) {
    if (b->graph_chunk > 0 && n >= b->graph_chunk) {
      if (!b->graph[b->cur]) {
        int rc = build_graph(b, b->cur);
        if (rc) return rc;
      }
      BATCH_CUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream), "cudaGraphLaunch");
      n -= b->graph_chunk;
    } else {
      cudaError_t e = launch_batch(b, b->cur, b->tile_rows, b->ctas_per_sm, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
      b->cur ^= 1;
      n -= 1;
    }
  }
  return LBM_SW_OK;
}

int lbm_sw_batch_get_moments(lbm_sw_batch* b, int i, double* depth, double* hu, double* hv, int on_device) {
  if (!b) return LBM_SW_E_ARG;
  int rc = check_instance(b, i);
  if (rc) return rc;
  if (!depth || !hu) return bfail(b, LBM_SW_E_ARG, "get_moments: depth and hu are required");
  if (!b->has_state[i]) return bfail(b, LBM_SW_E_STATE, "get_moments: instance %d has no state", i);
  const size_t n = static_cast<size_t>(b->nx[i]) * b->ny[i];
  double *d = depth, *u = hu, *v = hv;
  if (!on_device) {
    rc = ensure_staging(b, n);
    if (rc) return rc;
    d = b->moments_staging;
    u = d + n;
    v = hv ? d + 2 * n : nullptr;
  }
  const int from = b->cur;
  cudaError_t e = b->p.precision == LBM_SW_FP64
                      ? lbm::launch_moments2d<double>(inst_args<double>(b, i, from), d, u, v, b->stream)
                      : lbm::launch_moments2d<float>(inst_args<float>(b, i, from), d, u, v, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "moments kernel launch");
  if (!on_device) {
    BATCH_CUDA(b, cudaMemcpyAsync(depth, d, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy h");
    BATCH_CUDA(b, cudaMemcpyAsync(hu, u, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy hu");
    if (v) BATCH_CUDA(b, cudaMemcpyAsync(hv, v, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy hv");
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream), "get_moments synchronize");
  }
  return LBM_SW_OK;
}

int lbm_sw_batch_get_populations(lbm_sw_batch* b, int i, void* dst, int on_device) {
  if (!b) return LBM_SW_E_ARG;
  int rc = check_instance(b, i);
  if (rc) return rc;
  if (!dst) return bfail(b, LBM_SW_E_ARG, "get_populations: dst is NULL");
  if (!b->has_state[i]) return bfail(b, LBM_SW_E_STATE, "get_populations: instance %d has no state", i);
  const lbm::BatchInst& I = b->inst[i];
  const size_t row = static_cast<size_t>(I.nx) * b->elem, dplane = row * I.ny;
  const char* src = static_cast<const char*>(b->buf[b->cur]) + I.offset * b->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int p = 0; p < 13; ++p)
    BATCH_CUDA(b, cudaMemcpy2DAsync(static_cast<char*>(dst) + p * dplane, row, src + p * I.plane * b->elem,
                                    I.pitch * b->elem, row, I.ny, kind, b->stream),
               "copy populations out");
  if (!on_device) BATCH_CUDA(b, cudaStreamSynchronize(b->stream), "get_populations synchronize");
  return LBM_SW_OK;
}

int lbm_sw_batch_diagnostics(lbm_sw_batch* b, int i, double out[4]) {
  if (!b || !out) return b ? bfail(b, LBM_SW_E_ARG, "diagnostics: out is NULL") : LBM_SW_E_ARG;
  int rc = check_instance(b, i);
  if (rc) return rc;
  if (!b->has_state[i]) return bfail(b, LBM_SW_E_STATE, "diagnostics: instance %d has no state", i);
  cudaError_t e = b->p.precision == LBM_SW_FP64
                      ? lbm::launch_diagnostics<double>(inst_args<double>(b, i, b->cur), 13, b->diag_partials, b->diag_out, b->stream)
                      : lbm::launch_diagnostics<float>(inst_args<float>(b, i, b->cur), 13, b->diag_partials, b->diag_out, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "diagnostics kernel launch");
  BATCH_CUDA(b, cudaMemcpyAsync(b->diag_host, b->diag_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
             "copy diagnostics");
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream), "diagnostics synchronize");
  for (int k = 0; k < 4; ++k) out[k] = b->diag_host[k];
  if (b->diag_host[4] > 0)
    return bfail(b, LBM_SW_E_UNSTABLE, "diagnostics: %.0f cells with NaN/Inf or depth <= 0", b->diag_host[4]);
  return LBM_SW_OK;
}

int lbm_sw_batch_get_tuning(const lbm_sw_batch* b, lbm_sw_batch_tuning* out) {
  if (!b || !out) return LBM_SW_E_ARG;
  out->tile_rows = b->tile_rows;
  out->ctas_per_sm = b->ctas_per_sm;
  out->candidates = b->candidates;
  out->ms_per_step = b->tuned_ms;
  out->tiles = b->tiles[rows_index(b->tile_rows)];
  out->cells = b->cells;
  out->temporal_steps = b->temporal_k >= 2 ? b->temporal_k : 1;
  return LBM_SW_OK;
}

int lbm_sw_batch_autotune(lbm_sw_batch* b, int trial_steps, lbm_sw_batch_tuning* out) {
  if (!b) return LBM_SW_E_ARG;
  if (trial_steps < 1) return bfail(b, LBM_SW_E_ARG, "autotune: trial_steps must be >= 1");
  if (b->states_set != b->p.count) return bfail(b, LBM_SW_E_STATE, "autotune: every instance needs a state");
  cudaEvent_t e0, e1;
  BATCH_CUDA(b, cudaEventCreate(&e0), "cudaEventCreate");
  BATCH_CUDA(b, cudaEventCreate(&e1), "cudaEventCreate");
  const int rows_c[4] = {1, 2, 4, 8};
  const int ctas_c[4] = {0, 2, 4, 8};  // 0: one CTA per tile
  double best = 1e30;
  int best_rows = b->tile_rows, best_ctas = b->ctas_per_sm, tried = 0;
  int rc = LBM_SW_OK;
  for (int r = 0; r < 4 && rc == LBM_SW_OK; ++r) {
    for (int c = 0; c < 4 && rc == LBM_SW_OK; ++c) {
      cudaError_t e = launch_batch(b, b->cur, rows_c[r], ctas_c[c], b->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_batch(b, b->cur, rows_c[r], ctas_c[c], b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = bcuda(b, e, "autotune trial");
        break;
      }
      ++tried;
      const double per = ms / trial_steps;
      if (per < best) {
        best = per;
        best_rows = rows_c[r];
        best_ctas = ctas_c[c];
      }
    }
  }
  // temporal blocking: K steps per launch, compared per step
  int best_k = b->temporal_auto ? 0 : b->temporal_k;
  if (rc == LBM_SW_OK && b->temporal_auto) {
    const int ks[3] = {4, 6, 8};
    for (int q = 0; q < 3 && rc == LBM_SW_OK; ++q) {
      const int k = ks[q];
      rc = ensure_waves(b, k);
      if (rc != LBM_SW_OK) break;
      const int launches = std::max(1, (trial_steps + k - 1) / k);
      cudaError_t e = launch_temporal(b, b->cur, k, b->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int r = 0; r < launches && e == cudaSuccess; ++r) e = launch_temporal(b, b->cur, k, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = bcuda(b, e, "autotune temporal trial");
        break;
      }
      ++tried;
      const double per = ms / (static_cast<double>(launches) * k);
      if (per < best) {
        best = per;
        best_k = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LBM_SW_OK) return rc;
  if (best_rows != b->tile_rows || best_ctas != b->ctas_per_sm) drop_graphs(b);
  b->tile_rows = best_rows;
  b->ctas_per_sm = best_ctas;
  b->temporal_k = best_k;
  b->candidates = tried;
  b->tuned_ms = best;
  if (out) lbm_sw_batch_get_tuning(b, out);
  return LBM_SW_OK;
}

}  // extern "C"
