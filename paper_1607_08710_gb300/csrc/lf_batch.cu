// Batched mode of the C ABI (include/lagflux.h, lf_batch_*): many independent
// 2D meshes advanced together by the Heun/RK2 Lagrange-flux step of
// arXiv:1607.08710, Sec. 4 -- one persistent launch per stage over all
// problems, the step loop captured once as a CUDA graph, and a tile height
// picked by timing the candidates on the actual problem set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/lagflux.h"
#include "lf_internal.h"

struct lf_batch {
  lf_config common;                 // scheme parameters shared by all problems
  std::vector<lf_config> cfgs;      // per problem (sizes and domains)
  int nprob = 0;
  size_t elem = 8;
  cudaStream_t stream = nullptr;    // caller's stream: all work runs here
  cudaStream_t capture = nullptr;   // private stream used only to record the graph
  void* U = nullptr;                // pool of current states
  void* Ustar = nullptr;            // pool of predictor states
  size_t pool_elems = 0;
  std::vector<lf::ProbDesc> hprobs;
  std::vector<lf::Unit> hunits;
  lf::Unit* units = nullptr;
  size_t units_cap = 0;
  int ty = 64;                      // rows per work unit
  int grid = 0;                     // persistent CTAs
  lf::Scalars* sc = nullptr;        // one per problem
  lf::Scalars* hsc = nullptr;       // pinned mirror
  int* counters = nullptr;          // per-stage work counters
  std::vector<char> has_state;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  char last_error[512] = {0};
};

namespace {

void berr(lf_batch* b, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  if (b) vsnprintf(b->last_error, sizeof(b->last_error), fmt, ap);
  else {
    char buf[512];
    vsnprintf(buf, sizeof(buf), fmt, ap);
    lf::set_init_error("%s", buf);
  }
  va_end(ap);
}

lf_status bcuda(lf_batch* b, cudaError_t e, const char* what) {
  berr(b, "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA;
}

#define LF_BCUDA(b, call)                                \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);   \
  } while (0)

struct Guard {
  int prev = -1;
  bool ok = true;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~Guard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

const char* check_problem(const lf_config* c, const lf_config* c0) {
  if (c->dim != 2) return "batched problems must be 2D";
  if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
  if ((long long)c->nx * c->ny > (1LL << 30)) return "problem larger than 2^30 cells";
  // element offsets inside a problem's planes are 32-bit (rows padded to 128 bytes)
  if ((c->nx + 31LL) / 32 * 32 * c->ny >= (1LL << 31)) return "problem plane (rows padded) of 2^31 or more elements";
  if (c->limiter < 0 || c->limiter > 2 || c->bc < 0 || c->bc > 1 || c->riemann < 0 || c->riemann > 1)
    return "unknown limiter, boundary condition or interface solver";
  if (c->precision != LF_FP64 && c->precision != LF_FP32) return "unknown precision";
  if (!(c->xmax > c->xmin) || !(c->ymax > c->ymin)) return "empty domain";
  if (!(c->gamma > 1.0 && c->gamma <= 3.0) || !(c->cfl > 0.0 && c->cfl <= 1.0)) return "gamma or cfl out of range";
  if (c->limiter == LF_LIMITER_SWEBY && !(c->beta >= 1.0 && c->beta <= 2.0)) return "beta out of range";
  if (c->device < 0) return "device must be >= 0";
  if (c->time_order != 0 && c->time_order != LF_TIME_HEUN) return "batched mode runs the Heun time integrator";
  if (c->nspecies != 0) return "batched mode carries no species";
  if (c0 && (c->limiter != c0->limiter || c->bc != c0->bc || c->precision != c0->precision ||
             c->riemann != c0->riemann || c->gamma != c0->gamma || c->cfl != c0->cfl || c->beta != c0->beta ||
             c->device != c0->device))
    return "scheme parameters (limiter, bc, precision, riemann, gamma, cfl, beta, device) differ between problems";
  return nullptr;
}

lf::MeshDesc problem_mesh(const lf_batch* b, int p) {
  const lf::ProbDesc& d = b->hprobs[p];
  lf::MeshDesc m;
  m.nx = d.nx;
  m.ny = d.ny;
  m.pitch = d.pitch;
  m.plane = d.plane;
  m.dim = 2;
  m.bc = b->common.bc;
  m.limiter = b->common.limiter;
  m.riemann = b->common.riemann;
  m.gamma = b->common.gamma;
  m.beta = b->common.limiter == LF_LIMITER_MINMOD ? 1.0 : b->common.beta;
  m.rdx = d.rdx;
  m.rdy = d.rdy;
  m.vec = 1;
  return m;
}

// Order of the unit list: 1 = mesh order (problem by problem, row tile by row
// tile, strip by strip: neighbouring units share halo rows and columns while
// they are in L2); 0 = the inner-strip units of all problems, then the
// edge-strip units (measured as fast only while the two march bodies were
// unrolled and competed for the instruction cache).  Either way the short
// last row tiles go to the end.
#ifndef LF_BATCH_ORDER
#define LF_BATCH_ORDER 1
#endif

// Work units for a tile height: problem by problem, row tile by row tile,
// strip by strip, so that warps taking consecutive units share halo rows.
lf_status build_units(lf_batch* b, int ty) {
  const int cols = b->elem == 4 ? 64 : 32;  // columns of a warp strip (CPL=2 FP32, CPL=1 FP64)
  const int out_cols = cols - 4;           // its output columns
  // (LF_BATCH_ORDER 0: units of strips that lie inside their rows -- the
  // kernel's inner march -- first, then the edge strips on the mapped march.)
  b->hunits.clear();
  std::vector<lf::Unit> edge;
  for (int p = 0; p < b->nprob; ++p) {
    const lf::ProbDesc& d = b->hprobs[p];
    for (int j0 = 0; j0 < d.ny; j0 += ty)
      for (int i0 = 0; i0 < d.nx; i0 += out_cols) {
        const lf::Unit u{p, i0, j0, std::min(j0 + ty, d.ny), d};
        if (LF_BATCH_ORDER == 1 || (i0 - 2 >= 0 && i0 - 2 + cols <= d.nx)) b->hunits.push_back(u);
        else edge.push_back(u);
      }
  }
  // Within each group, the short last row tiles of the problems go last, so
  // that the end of a stage is made of the smallest units.
  auto taller = [](const lf::Unit& a, const lf::Unit& c) { return a.jend - a.j0 > c.jend - c.j0; };
  std::stable_sort(b->hunits.begin(), b->hunits.end(), taller);
  std::stable_sort(edge.begin(), edge.end(), taller);
  b->hunits.insert(b->hunits.end(), edge.begin(), edge.end());
  if (b->hunits.size() > b->units_cap) {
    cudaFree(b->units);
    b->units = nullptr;
    LF_BCUDA(b, cudaMalloc(&b->units, b->hunits.size() * sizeof(lf::Unit)));
    b->units_cap = b->hunits.size();
  }
  LF_BCUDA(b, cudaMemcpyAsync(b->units, b->hunits.data(), b->hunits.size() * sizeof(lf::Unit),
                              cudaMemcpyHostToDevice, b->stream));
  LF_BCUDA(b, cudaStreamSynchronize(b->stream));
  b->ty = ty;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = -1;
  }
  return LF_OK;
}

lf::BatchDesc batch_desc(const lf_batch* b) {
  lf::BatchDesc d;
  d.common = problem_mesh(b, 0);
  d.units = b->units;
  d.nunits = (int)b->hunits.size();
  d.grid = b->grid;
  return d;
}

template <typename T>
lf_status enqueue_steps_t(lf_batch* b, int nsteps, cudaStream_t s) {
  const lf::BatchDesc d = batch_desc(b);
  T* U = static_cast<T*>(b->U);
  T* Us = static_cast<T*>(b->Ustar);
  for (int k = 0; k < nsteps; ++k) {
    LF_BCUDA(b, lf::launch_batch_begin(b->sc, b->nprob, 0.0, b->counters, s));
    LF_BCUDA(b, lf::launch_batch_stage<T>(0, d, U, U, Us, b->sc, b->counters, s));
    LF_BCUDA(b, lf::launch_batch_stage<T>(1, d, Us, U, U, b->sc, b->counters + 1, s));
    LF_BCUDA(b, lf::launch_batch_end(b->sc, b->nprob, s));
  }
  return LF_OK;
}

lf_status enqueue_steps(lf_batch* b, int nsteps, cudaStream_t s) {
  return b->elem == 8 ? enqueue_steps_t<double>(b, nsteps, s) : enqueue_steps_t<float>(b, nsteps, s);
}

lf_status read_scalars(lf_batch* b) {
  LF_BCUDA(b, cudaMemcpyAsync(b->hsc, b->sc, b->nprob * sizeof(lf::Scalars), cudaMemcpyDeviceToHost, b->stream));
  LF_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LF_OK;
}

lf_status error_status(lf_batch* b) {
  for (int p = 0; p < b->nprob; ++p)
    if (b->hsc[p].err) {
      berr(b, "problem %d: non-positive density or pressure, NaN, or bad dt", p);
      return LF_ERR_NONPHYSICAL;
    }
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_batch_init(const lf_config* cfgs, int32_t nprob, void* stream, lf_batch** out) {
  if (!cfgs || nprob < 1 || !out) {
    berr(nullptr, "lf_batch_init: need cfgs, nprob >= 1 and out");
    return LF_ERR_ARG;
  }
  for (int p = 0; p < nprob; ++p)
    if (const char* why = check_problem(&cfgs[p], p ? &cfgs[0] : nullptr)) {
      berr(nullptr, "lf_batch_init: problem %d: %s", p, why);
      return LF_ERR_ARG;
    }
  lf_batch* b = new lf_batch();
  b->common = cfgs[0];
  b->cfgs.assign(cfgs, cfgs + nprob);
  b->nprob = nprob;
  b->elem = cfgs[0].precision == LF_FP64 ? 8 : 4;
  b->stream = static_cast<cudaStream_t>(stream);
  b->has_state.assign(nprob, 0);
  const int align = 128 / (int)b->elem;
  size_t off = 0;
  for (int p = 0; p < nprob; ++p) {
    const lf_config& c = cfgs[p];
    lf::ProbDesc d;
    d.nx = c.nx;
    d.ny = c.ny;
    d.pitch = (c.nx + align - 1) / align * align;
    d.pad = 0;
    d.plane = (long long)d.pitch * d.ny;
    d.off = (long long)off;
    d.rdx = c.nx / (c.xmax - c.xmin);
    d.rdy = c.ny / (c.ymax - c.ymin);
    b->hprobs.push_back(d);
    off += 4 * (size_t)d.plane;
  }
  b->pool_elems = off;
  Guard g(b->common.device);
  lf_status st = LF_OK;
  auto fail = [&](lf_status s) {
    lf_batch_destroy(b);
    return s;
  };
  if (!g.ok) {
    berr(nullptr, "lf_batch_init: cannot select device %d", b->common.device);
    return fail(LF_ERR_CUDA);
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&b->U, off * b->elem);
  if (e == cudaSuccess) e = cudaMalloc(&b->Ustar, off * b->elem);
  if (e == cudaSuccess) e = cudaMalloc(&b->sc, nprob * sizeof(lf::Scalars));
  if (e == cudaSuccess) e = cudaMalloc(&b->counters, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->hsc, nprob * sizeof(lf::Scalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->U, 0, off * b->elem, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->Ustar, 0, off * b->elem, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counters, 0, 2 * sizeof(int), b->stream);
  for (int p = 0; p < nprob && e == cudaSuccess; ++p) e = lf::launch_reset_scalars(b->sc + p, b->common.cfl, b->stream);
  if (e != cudaSuccess) {
    bcuda(nullptr, e, "lf_batch_init");
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA);
  }
  // persistent grid: every SM filled to the stage kernels' occupancy
  int dev = b->common.device, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int occ = std::max(1, std::min(b->elem == 8 ? lf::batch_blocks_per_sm<double>(1, b->common.limiter)
                                                    : lf::batch_blocks_per_sm<float>(1, b->common.limiter),
                                       b->elem == 8 ? lf::batch_blocks_per_sm<double>(0, b->common.limiter)
                                                    : lf::batch_blocks_per_sm<float>(0, b->common.limiter)));
  b->grid = std::max(1, sms) * occ;
  if ((st = build_units(b, 64)) != LF_OK) {
    lf::set_init_error("%s", b->last_error);
    return fail(st);
  }
  *out = b;
  return LF_OK;
}

void lf_batch_destroy(lf_batch* b) {
  if (!b) return;
  {
    Guard g(b->common.device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->U);
    cudaFree(b->Ustar);
    cudaFree(b->units);
    cudaFree(b->sc);
    cudaFree(b->counters);
    cudaFreeHost(b->hsc);
  }
  delete b;
}

lf_status lf_batch_set_primitive(lf_batch* b, int32_t p, const void* rho, const void* u, const void* v,
                                 const void* pr, int on_device) {
  if (!b) return LF_ERR_ARG;
  if (p < 0 || p >= b->nprob || !rho || !u || !v || !pr) {
    berr(b, "lf_batch_set_primitive: bad problem index or NULL plane");
    return LF_ERR_ARG;
  }
  Guard g(b->common.device);
  const lf::MeshDesc m = problem_mesh(b, p);
  const size_t n = (size_t)m.nx * m.ny;
  const void* src[4] = {rho, u, v, pr};
  void* staging = nullptr;
  if (!on_device) {
    // stage through the problem's own predictor slot, which the next step overwrites anyway
    staging = static_cast<char*>(b->Ustar) + (size_t)b->hprobs[p].off * b->elem;
    for (int l = 0; l < 4; ++l) {
      char* dst = static_cast<char*>(staging) + l * n * b->elem;
      LF_BCUDA(b, cudaMemcpyAsync(dst, src[l], n * b->elem, cudaMemcpyHostToDevice, b->stream));
      src[l] = dst;
    }
  }
  cudaError_t e;
  if (b->elem == 8) {
    double* U = static_cast<double*>(b->U) + b->hprobs[p].off;
    e = lf::launch_prim_to_cons<double>(m, (const double*)src[0], (const double*)src[1], (const double*)src[2],
                                        (const double*)src[3], (long long)n, U, b->stream);
    if (e == cudaSuccess) e = lf::launch_reset_scalars(b->sc + p, b->common.cfl, b->stream);
    if (e == cudaSuccess) e = lf::launch_wave_speed<double>(m, U, b->sc + p, b->stream);
  } else {
    float* U = static_cast<float*>(b->U) + b->hprobs[p].off;
    e = lf::launch_prim_to_cons<float>(m, (const float*)src[0], (const float*)src[1], (const float*)src[2],
                                       (const float*)src[3], (long long)n, U, b->stream);
    if (e == cudaSuccess) e = lf::launch_reset_scalars(b->sc + p, b->common.cfl, b->stream);
    if (e == cudaSuccess) e = lf::launch_wave_speed<float>(m, U, b->sc + p, b->stream);
  }
  if (e != cudaSuccess) return bcuda(b, e, "lf_batch_set_primitive");
  if (!on_device) LF_BCUDA(b, cudaStreamSynchronize(b->stream));
  b->has_state[p] = 1;
  return LF_OK;
}

lf_status lf_batch_get_state(lf_batch* b, int32_t p, void* rho, void* rhou, void* rhov, void* rhoE, int on_device) {
  if (!b) return LF_ERR_ARG;
  if (p < 0 || p >= b->nprob || !rho || !rhou || !rhov || !rhoE) {
    berr(b, "lf_batch_get_state: bad problem index or NULL plane");
    return LF_ERR_ARG;
  }
  Guard g(b->common.device);
  const lf::ProbDesc& d = b->hprobs[p];
  void* dst[4] = {rho, rhou, rhov, rhoE};
  const size_t w = (size_t)d.nx * b->elem;
  for (int l = 0; l < 4; ++l) {
    const char* src = static_cast<const char*>(b->U) + ((size_t)d.off + (size_t)l * d.plane) * b->elem;
    LF_BCUDA(b, cudaMemcpy2DAsync(dst[l], w, src, (size_t)d.pitch * b->elem, w, d.ny,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  }
  if (!on_device) LF_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LF_OK;
}

lf_status lf_batch_run(lf_batch* b, int32_t nsteps, int32_t use_graph) {
  if (!b) return LF_ERR_ARG;
  if (nsteps < 0) {
    berr(b, "lf_batch_run: nsteps must be >= 0");
    return LF_ERR_ARG;
  }
  for (int p = 0; p < b->nprob; ++p)
    if (!b->has_state[p]) {
      berr(b, "lf_batch_run: problem %d has no state", p);
      return LF_ERR_STATE;
    }
  if (nsteps == 0) return LF_OK;
  Guard g(b->common.device);
  if (!use_graph) return enqueue_steps(b, nsteps, b->stream);
  if (b->graph_steps != nsteps) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      b->graph_steps = -1;
    }
    // Record the whole loop once on the private stream; replays run on the
    // caller's stream.  Nothing executes during the recording.
    LF_BCUDA(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeRelaxed));
    lf_status st = enqueue_steps(b, nsteps, b->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
    if (st != LF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
    b->graph_steps = nsteps;
  }
  LF_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  return LF_OK;
}

lf_status lf_batch_autotune(lf_batch* b, int32_t trial_steps, int32_t* chosen_rows) {
  if (!b) return LF_ERR_ARG;
  if (trial_steps < 1) {
    berr(b, "lf_batch_autotune: trial_steps must be >= 1");
    return LF_ERR_ARG;
  }
  for (int p = 0; p < b->nprob; ++p)
    if (!b->has_state[p]) {
      berr(b, "lf_batch_autotune: problem %d has no state", p);
      return LF_ERR_STATE;
    }
  Guard g(b->common.device);
  // Trials advance the state; keep a copy of the states and scalars and put it back afterwards.
  void* save = nullptr;
  lf::Scalars* save_sc = nullptr;
  LF_BCUDA(b, cudaMalloc(&save, b->pool_elems * b->elem));
  cudaError_t e = cudaMalloc(&save_sc, b->nprob * sizeof(lf::Scalars));
  if (e != cudaSuccess) {
    cudaFree(save);
    return bcuda(b, e, "lf_batch_autotune: cudaMalloc");
  }
  cudaMemcpyAsync(save, b->U, b->pool_elems * b->elem, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(save_sc, b->sc, b->nprob * sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, b->stream);
  const int candidates[] = {16, 24, 32, 48, 64, 96, 128};
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best_ms = 1e30f;
  int best = b->ty;
  lf_status st = LF_OK;
  for (int ty : candidates) {
    if ((st = build_units(b, ty)) != LF_OK) break;
    if ((st = enqueue_steps(b, 1, b->stream)) != LF_OK) break;  // warm-up
    cudaEventRecord(t0, b->stream);
    if ((st = enqueue_steps(b, trial_steps, b->stream)) != LF_OK) break;
    cudaEventRecord(t1, b->stream);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best_ms) {
      best_ms = ms;
      best = ty;
    }
    cudaMemcpyAsync(b->U, save, b->pool_elems * b->elem, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->sc, save_sc, b->nprob * sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, b->stream);
  }
  cudaMemcpyAsync(b->U, save, b->pool_elems * b->elem, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(b->sc, save_sc, b->nprob * sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(save);
  cudaFree(save_sc);
  if (st != LF_OK) return st;
  if ((st = build_units(b, best)) != LF_OK) return st;
  if (chosen_rows) *chosen_rows = best;
  return LF_OK;
}

lf_status lf_batch_set_rows(lf_batch* b, int32_t rows) {
  if (!b) return LF_ERR_ARG;
  if (rows < 1 || rows > 4096) {
    berr(b, "lf_batch_set_rows: rows must be in [1, 4096]");
    return LF_ERR_ARG;
  }
  Guard g(b->common.device);
  return build_units(b, rows);
}

lf_status lf_batch_get_times(lf_batch* b, double* t, int64_t* steps) {
  if (!b) return LF_ERR_ARG;
  Guard g(b->common.device);
  if (lf_status st = read_scalars(b)) return st;
  for (int p = 0; p < b->nprob; ++p) {
    if (t) t[p] = b->hsc[p].t;
    if (steps) steps[p] = b->hsc[p].steps;
  }
  return error_status(b);
}

lf_status lf_batch_profile(lf_batch* b, int32_t nsteps, double ms[2]) {
  if (!b || !ms) return LF_ERR_ARG;
  if (nsteps < 1) {
    berr(b, "lf_batch_profile: nsteps must be >= 1");
    return LF_ERR_ARG;
  }
  for (int p = 0; p < b->nprob; ++p)
    if (!b->has_state[p]) {
      berr(b, "lf_batch_profile: problem %d has no state", p);
      return LF_ERR_STATE;
    }
  Guard g(b->common.device);
  const lf::BatchDesc d = batch_desc(b);
  cudaEvent_t ev[4];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < 4 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) made--;
  float acc[2] = {0.f, 0.f};
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    e = lf::launch_batch_begin(b->sc, b->nprob, 0.0, b->counters, b->stream);
    for (int stage = 0; stage < 2 && e == cudaSuccess; ++stage) {
      e = cudaEventRecord(ev[2 * stage], b->stream);
      if (e != cudaSuccess) break;
      if (b->elem == 8) {
        double* U = static_cast<double*>(b->U);
        double* Us = static_cast<double*>(b->Ustar);
        e = stage == 0 ? lf::launch_batch_stage<double>(0, d, U, U, Us, b->sc, b->counters, b->stream)
                       : lf::launch_batch_stage<double>(1, d, Us, U, U, b->sc, b->counters + 1, b->stream);
      } else {
        float* U = static_cast<float*>(b->U);
        float* Us = static_cast<float*>(b->Ustar);
        e = stage == 0 ? lf::launch_batch_stage<float>(0, d, U, U, Us, b->sc, b->counters, b->stream)
                       : lf::launch_batch_stage<float>(1, d, Us, U, U, b->sc, b->counters + 1, b->stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[2 * stage + 1], b->stream);
    }
    if (e == cudaSuccess) e = lf::launch_batch_end(b->sc, b->nprob, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    for (int stage = 0; stage < 2 && e == cudaSuccess; ++stage) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[2 * stage], ev[2 * stage + 1]);
      acc[stage] += t;
    }
  }
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return bcuda(b, e, "lf_batch_profile");
  ms[0] = acc[0];
  ms[1] = acc[1];
  return LF_OK;
}

const char* lf_batch_last_error(const lf_batch* b) { return b ? b->last_error : lf_last_error(nullptr); }

}  // extern "C"
