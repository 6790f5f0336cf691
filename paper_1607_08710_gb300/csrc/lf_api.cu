// C ABI of liblagflux (declared in include/lagflux.h): context management,
// state transfer, and the Heun time loop of arXiv:1607.08710, Sec. 4, driven
// entirely by device-side scalars.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/lagflux.h"
#include "lf_host.h"

namespace {
char g_init_error[512] = "";
}  // namespace

void lf::set_err(lf_ctx* c, const char* fmt, ...) {
  char* dst = c ? c->last_error : g_init_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

lf_status lf::cuda_fail(lf_ctx* c, cudaError_t e, const char* what) {
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA;
}

using lf::cuda_fail;
using lf::DeviceGuard;
using lf::set_err;

namespace {

const char* validate(const lf_config* c) {
  if (!c) return "config is NULL";
  if (c->dim < 1 || c->dim > 3) return "dim must be 1, 2 or 3";
  if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
  if (c->dim == 1 && c->ny != 1) return "ny must be 1 when dim == 1";
  if (c->dim < 3 && c->nz > 1) return "nz must be 0 or 1 below 3D";
  if (c->dim == 3 && c->nz < 1) return "nz must be >= 1 in 3D";
  if (c->nz < 0) return "nz must be >= 0";
  const long long nz = c->dim == 3 ? c->nz : 1;
  // Rows are padded to 128 bytes and element offsets inside a field plane are
  // 32-bit in the kernels, so the padded plane must stay below 2^31 elements.
  const long long align = c->precision == LF_FP32 ? 32 : 16;
  if ((c->nx + align - 1) / align * align * c->ny * nz >= (1LL << 31))
    return "mesh too large: a field plane (rows padded to 128 bytes) must have fewer than 2^31 elements";
  if (c->dim == 3 && (!(c->zmax > c->zmin) || !std::isfinite(c->zmax - c->zmin))) return "need zmin < zmax";
  if (c->tile_rows < 0 || c->tile_rows > 4096) return "tile_rows must be in 0 .. 4096";
  if (c->limiter < 0 || c->limiter > 2) return "unknown limiter";
  if (c->bc < 0 || c->bc > 1) return "unknown boundary condition";
  if (c->precision != LF_FP64 && c->precision != LF_FP32) return "unknown precision";
  if (c->riemann < 0 || c->riemann > 1) return "unknown interface solver";
  if (c->device < 0) return "device must be >= 0";
  if (!(c->xmax > c->xmin) || !std::isfinite(c->xmax - c->xmin)) return "need xmin < xmax";
  if (c->dim >= 2 && (!(c->ymax > c->ymin) || !std::isfinite(c->ymax - c->ymin))) return "need ymin < ymax";
  if (!(c->gamma > 1.0 && c->gamma <= 3.0)) return "gamma must be in (1, 3]";
  if (!(c->cfl > 0.0 && c->cfl <= 1.0)) return "cfl must be in (0, 1]";
  if (c->limiter == LF_LIMITER_SWEBY && !(c->beta >= 1.0 && c->beta <= 2.0)) return "beta must be in [1, 2]";
  if (c->time_order != 0 && c->time_order != LF_TIME_HEUN && c->time_order != LF_TIME_SSPRK3)
    return "time_order must be 0, 2 (Heun) or 3 (SSP-RK3)";
  if (c->nspecies < 0 || c->nspecies > LF_MAX_SPECIES) return "nspecies must be in [0, LF_MAX_SPECIES]";
  return nullptr;
}

// Event pair for the next traced launch (pool grows in chunks outside the
// launch path as far as possible).
lf_status trace_begin(lf_ctx* c, int stage, cudaEvent_t* stop) {
  if (c->ev_used * 2 + 2 > c->ev_pool.size()) {
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      LF_CUDA(c, cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
  }
  cudaEvent_t start = c->ev_pool[c->ev_used * 2];
  *stop = c->ev_pool[c->ev_used * 2 + 1];
  c->ev_stage.resize(c->ev_used + 1);
  c->ev_stage[c->ev_used] = stage;
  ++c->ev_used;
  LF_CUDA(c, cudaEventRecord(start, c->stream));
  return LF_OK;
}

// Stage `stage` of the step (see launch_stage): Heun 0 (U -> U*), 1 (U*, U -> U);
// SSP-RK3 0 (U -> U1 in Ustar), 2 (U1, U -> U2), 3 (U2, U -> U).  Traced
// launches are filed as the first stage (0) or a later stage (1).
template <typename T>
lf_status dispatch_stage(lf_ctx* c, int stage) {
  T* U = static_cast<T*>(c->U);
  T* Us = static_cast<T*>(c->Ustar);
  T* U2 = static_cast<T*>(c->U2);
  cudaEvent_t stop = nullptr;
  if (c->profiling)
    if (lf_status st = trace_begin(c, stage == 0 ? 0 : 1, &stop)) return st;
  const T* in[4] = {U, Us, Us, U2};
  T* out[4] = {Us, U, U2, U};
  const cudaError_t e = c->cfg.dim == 3
                            ? lf::launch_stage3d(stage, c->mesh3, in[stage], U, out[stage], c->sc, c->stream)
                            : lf::launch_stage<T>(stage, c->mesh, in[stage], U, out[stage], c->sc, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage launch");
  if (stop) LF_CUDA(c, cudaEventRecord(stop, c->stream));
  return LF_OK;
}

}  // namespace

// begin (dt) -> predictor -> corrector -> end (t, steps, parity)
lf_status lf::enqueue_step(lf_ctx* c, double dt_fixed) {
  LF_CUDA(c, lf::launch_begin_step(c->sc, dt_fixed, c->stream));
  static const int heun[] = {0, 1}, rk3[] = {0, 2, 3};
  const bool third = c->cfg.time_order == LF_TIME_SSPRK3;
  const int* stages = third ? rk3 : heun;
  for (int k = 0; k < (third ? 3 : 2); ++k) {
    lf_status st = c->elem == 8 ? dispatch_stage<double>(c, stages[k]) : dispatch_stage<float>(c, stages[k]);
    if (st != LF_OK) return st;
  }
  LF_CUDA(c, lf::launch_end_step(c->sc, c->stream));
  return LF_OK;
}

lf_status lf::read_scalars(lf_ctx* c) {
  LF_CUDA(c, cudaMemcpyAsync(c->hsc, c->sc, sizeof(lf::Scalars), cudaMemcpyDeviceToHost, c->stream));
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf::device_error_status(lf_ctx* c) {
  if (c->hsc->err & lf::ERR_NONPHYSICAL) {
    set_err(c, "non-positive density or pressure (or NaN) in the state");
    return LF_ERR_NONPHYSICAL;
  }
  if (c->hsc->err & lf::ERR_BAD_DT) {
    set_err(c, "non-finite or non-positive CFL time step");
    return LF_ERR_NONPHYSICAL;
  }
  return LF_OK;
}

using lf::device_error_status;
using lf::enqueue_step;
using lf::read_scalars;

namespace {

// Fresh time loop on the state just written into c->U.
lf_status restart_clock(lf_ctx* c) {
  LF_CUDA(c, lf::launch_reset_scalars(c->sc, c->cfg.cfl, c->stream));
  cudaError_t e;
  if (c->cfg.dim == 3)
    e = c->elem == 8 ? lf::launch_wave_speed3d(c->mesh3, static_cast<double*>(c->U), c->sc, c->stream)
                     : lf::launch_wave_speed3d(c->mesh3, static_cast<float*>(c->U), c->sc, c->stream);
  else
    e = c->elem == 8 ? lf::launch_wave_speed<double>(c->mesh, static_cast<double*>(c->U), c->sc, c->stream)
                     : lf::launch_wave_speed<float>(c->mesh, static_cast<float*>(c->U), c->sc, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "wave speed launch");
  c->has_state = true;
  return LF_OK;
}

char* plane_ptr(lf_ctx* c, void* base, int l) {
  return static_cast<char*>(base) + (size_t)l * c->mesh.plane * c->elem;
}

// Dense caller planes <-> pitched state planes.  When the rows carry no
// padding (nx a multiple of the row alignment) a plane is one contiguous
// block and moves as a single copy.
lf_status copy_plane_in(lf_ctx* c, int l, const void* src, cudaMemcpyKind kind) {
  const size_t w = (size_t)c->mesh.nx * c->elem;
  char* dst = plane_ptr(c, c->U, l);
  if (!src) {
    LF_CUDA(c, cudaMemset2DAsync(dst, (size_t)c->mesh.pitch * c->elem, 0, w, c->mesh.ny, c->stream));
    return LF_OK;
  }
  if (c->mesh.pitch == c->mesh.nx)
    LF_CUDA(c, cudaMemcpyAsync(dst, src, w * c->mesh.ny, kind, c->stream));
  else
    LF_CUDA(c, cudaMemcpy2DAsync(dst, (size_t)c->mesh.pitch * c->elem, src, w, w, c->mesh.ny, kind, c->stream));
  return LF_OK;
}

lf_status copy_plane_out(lf_ctx* c, int l, void* dst, cudaMemcpyKind kind) {
  if (!dst) return LF_OK;
  const size_t w = (size_t)c->mesh.nx * c->elem;
  if (c->mesh.pitch == c->mesh.nx)
    LF_CUDA(c, cudaMemcpyAsync(dst, plane_ptr(c, c->U, l), w * c->mesh.ny, kind, c->stream));
  else
    LF_CUDA(c, cudaMemcpy2DAsync(dst, w, plane_ptr(c, c->U, l), (size_t)c->mesh.pitch * c->elem, w, c->mesh.ny,
                                 kind, c->stream));
  return LF_OK;
}

lf_status ensure_staging(lf_ctx* c) {
  if (c->staging) return LF_OK;
  const int planes = c->nf > 4 ? c->nf : 4;
  LF_CUDA(c, cudaMalloc(&c->staging, planes * (size_t)c->mesh.nx * c->mesh.ny * c->elem));
  return LF_OK;
}

// The four-plane calls describe 1D/2D states only.
lf_status reject_3d(lf_ctx* c, const char* who) {
  if (c->cfg.dim != 3) return LF_OK;
  set_err(c, "%s: 3D contexts transfer the whole state (lf_set_conservative / lf_set_primitives)", who);
  return LF_ERR_ARG;
}

}  // namespace

void lf::set_init_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_init_error, sizeof(g_init_error), fmt, ap);
  va_end(ap);
}

extern "C" {

const char* lf_status_string(lf_status s) {
  switch (s) {
    case LF_OK: return "LF_OK";
    case LF_ERR_ARG: return "LF_ERR_ARG";
    case LF_ERR_CUDA: return "LF_ERR_CUDA";
    case LF_ERR_OOM: return "LF_ERR_OOM";
    case LF_ERR_NONPHYSICAL: return "LF_ERR_NONPHYSICAL";
    case LF_ERR_TIMEOUT: return "LF_ERR_TIMEOUT";
    case LF_ERR_STATE: return "LF_ERR_STATE";
  }
  return "LF_ERR_UNKNOWN";
}

const char* lf_last_error(const lf_ctx* ctx) { return ctx ? ctx->last_error : g_init_error; }

void lf_destroy(lf_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->cfg.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->U);
    cudaFree(c->Ustar);
    cudaFree(c->U2);
    cudaFree(c->staging);
    cudaFree(c->sc);
    cudaFree(c->partials);
    cudaFree(c->dsums);
    cudaFreeHost(c->hsc);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->run_graph) cudaGraphExecDestroy(c->run_graph);
    if (c->capture) cudaStreamDestroy(c->capture);
    lf::free_adjoint(c);
  }
  delete c;
}

lf_status lf_init(const lf_config* cfg, void* stream, lf_ctx** out) {
  if (!out) {
    set_err(nullptr, "out is NULL");
    return LF_ERR_ARG;
  }
  if (const char* why = validate(cfg)) {
    set_err(nullptr, "invalid configuration: %s", why);
    return LF_ERR_ARG;
  }
  // Test hook: simulate a failed device allocation without touching the GPU.
  if (const char* f = std::getenv("LF_TEST_FAIL_ALLOC")) {
    if (f[0] && f[0] != '0') {
      set_err(nullptr, "device allocation failed (simulated by LF_TEST_FAIL_ALLOC)");
      return LF_ERR_OOM;
    }
  }
  lf_ctx* c = new lf_ctx();
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(stream);
  c->elem = cfg->precision == LF_FP64 ? 8 : 4;
  lf::MeshDesc& m = c->mesh;
  m.nx = cfg->nx;
  m.ny = cfg->ny;
  const int align = 128 / (int)c->elem;  // rows start on 128-byte boundaries
  m.pitch = (cfg->nx + align - 1) / align * align;
  m.plane = (long long)m.pitch * m.ny;
  m.dim = cfg->dim;
  m.bc = cfg->bc;
  m.limiter = cfg->limiter;
  m.riemann = cfg->riemann;
  m.gamma = cfg->gamma;
  m.beta = cfg->limiter == LF_LIMITER_MINMOD ? 1.0 : cfg->beta;
  m.rdx = cfg->nx / (cfg->xmax - cfg->xmin);
  m.rdy = cfg->dim == 2 ? cfg->ny / (cfg->ymax - cfg->ymin) : 0.0;
  m.vec = 1;  // pitch is a multiple of 128 bytes and the planes come from cudaMalloc
  m.nspecies = cfg->nspecies;
  static_assert(LF_MAX_SPECIES == lf::MAX_SPECIES, "public and kernel species limits agree");
  c->nf = 4 + cfg->nspecies;
  c->nspecies = cfg->nspecies;
  c->sp0 = 4;
  if (cfg->dim == 3) {
    lf::Mesh3Desc& m3 = c->mesh3;
    m3.nx = cfg->nx;
    m3.ny = cfg->ny;
    m3.nz = cfg->nz;
    m3.pitch = m.pitch;
    m3.plane = (long long)m.pitch * cfg->ny * cfg->nz;
    m3.bc = cfg->bc;
    m3.limiter = cfg->limiter;
    m3.riemann = cfg->riemann;
    m3.nspecies = cfg->nspecies;
    m3.gamma = m.gamma;
    m3.beta = m.beta;
    m3.rdx = m.rdx;
    m3.rdy = cfg->ny / (cfg->ymax - cfg->ymin);
    m3.rdz = cfg->nz / (cfg->zmax - cfg->zmin);
    m = lf::mesh_view(m3, 0);  // the row view: copies and sums walk ny*nz rows
    c->nf = 5 + cfg->nspecies;
    c->sp0 = 5;
  }
  const int nf = c->nf;

  DeviceGuard g(cfg->device);
  if (!g.ok) {
    set_err(nullptr, "cannot select CUDA device %d", cfg->device);
    delete c;
    return LF_ERR_CUDA;
  }
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess) sms = 0;
    const int cpl = c->elem == 4 ? 2 : 1;
    if (cfg->dim == 2) m.ty = cfg->tile_rows > 0 ? cfg->tile_rows : lf::auto_tile_rows(m, cpl, sms);
    if (cfg->dim == 3)
      c->mesh3.tz = cfg->tile_rows > 0 ? cfg->tile_rows
                                       : lf::auto_tile_planes(c->mesh3, cpl, lf::stage3d_rows_per_cta(), sms);
  }
  const size_t state_bytes = nf * (size_t)m.plane * c->elem;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&c->U, state_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->Ustar, state_bytes);
  if (e == cudaSuccess && cfg->time_order == LF_TIME_SSPRK3) e = cudaMalloc(&c->U2, state_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->sc, sizeof(lf::Scalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->partials, (size_t)lf::sums_blocks() * nf * 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->dsums, nf * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c->hsc, sizeof(lf::Scalars));
  if (e == cudaSuccess) e = lf::launch_reset_scalars(c->sc, cfg->cfl, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->U, 0, state_bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->Ustar, 0, state_bytes, c->stream);
  if (e != cudaSuccess) {
    lf_status st = cuda_fail(nullptr, e, "lf_init");
    cudaGetLastError();
    lf_destroy(c);
    return st;
  }
  *out = c;
  return LF_OK;
}

lf_status lf_set_state(lf_ctx* c, const void* rho, const void* rhou, const void* rhov, const void* rhoE,
                       int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = reject_3d(c, "lf_set_state")) return st;
  if (!rho || !rhou || !rhoE || (c->cfg.dim == 2 && !rhov)) {
    set_err(c, "lf_set_state: NULL plane");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const void* src[4] = {rho, rhou, rhov, rhoE};
  for (int l = 0; l < 4; ++l)
    if (lf_status st = copy_plane_in(c, l, src[l], kind)) return st;
  if (lf_status st = restart_clock(c)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_set_primitive(lf_ctx* c, const void* rho, const void* u, const void* v, const void* p,
                           int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = reject_3d(c, "lf_set_primitive")) return st;
  if (!rho || !u || !p || (c->cfg.dim == 2 && !v)) {
    set_err(c, "lf_set_primitive: NULL plane");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  const void* src[4] = {rho, u, v, p};
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;
    for (int l = 0; l < 4; ++l) {
      char* dst = static_cast<char*>(c->staging) + l * n * c->elem;
      if (src[l]) LF_CUDA(c, cudaMemcpyAsync(dst, src[l], n * c->elem, cudaMemcpyHostToDevice, c->stream));
      else LF_CUDA(c, cudaMemsetAsync(dst, 0, n * c->elem, c->stream));
      src[l] = dst;
    }
  }
  cudaError_t e;
  if (c->elem == 8)
    e = lf::launch_prim_to_cons<double>(c->mesh, (const double*)src[0], (const double*)src[1],
                                        (const double*)src[2], (const double*)src[3], (long long)n,
                                        static_cast<double*>(c->U), c->stream);
  else
    e = lf::launch_prim_to_cons<float>(c->mesh, (const float*)src[0], (const float*)src[1], (const float*)src[2],
                                       (const float*)src[3], (long long)n, static_cast<float*>(c->U), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "prim_to_cons launch");
  if (lf_status st = restart_clock(c)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_state(lf_ctx* c, void* rho, void* rhou, void* rhov, void* rhoE, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = reject_3d(c, "lf_get_state")) return st;
  if (!rho || !rhou || !rhoE || (c->cfg.dim == 2 && !rhov)) {
    set_err(c, "lf_get_state: NULL plane");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  void* dst[4] = {rho, rhou, rhov, rhoE};
  for (int l = 0; l < 4; ++l)
    if (lf_status st = copy_plane_out(c, l, dst[l], kind)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_primitive(lf_ctx* c, void* rho, void* u, void* v, void* p, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = reject_3d(c, "lf_get_primitive")) return st;
  if (!rho || !u || !p || (c->cfg.dim == 2 && !v)) {
    set_err(c, "lf_get_primitive: NULL plane");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  void* dst[4] = {rho, u, v, p};
  void* kdst[4];
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;
    for (int l = 0; l < 4; ++l) kdst[l] = static_cast<char*>(c->staging) + l * n * c->elem;
  } else {
    for (int l = 0; l < 4; ++l) kdst[l] = dst[l];
  }
  cudaError_t e;
  if (c->elem == 8)
    e = lf::launch_cons_to_prim<double>(c->mesh, static_cast<double*>(c->U), (double*)kdst[0], (double*)kdst[1],
                                        (double*)kdst[2], (double*)kdst[3], c->stream);
  else
    e = lf::launch_cons_to_prim<float>(c->mesh, static_cast<float*>(c->U), (float*)kdst[0], (float*)kdst[1],
                                       (float*)kdst[2], (float*)kdst[3], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cons_to_prim launch");
  if (!on_device) {
    for (int l = 0; l < 4; ++l)
      if (dst[l]) LF_CUDA(c, cudaMemcpyAsync(dst[l], kdst[l], n * c->elem, cudaMemcpyDeviceToHost, c->stream));
    LF_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LF_OK;
}

}  // extern "C"

namespace {

lf_status species_args(lf_ctx* c, const void* p, const char* who) {
  if (c->nspecies == 0) {
    set_err(c, "%s: the context carries no species (nspecies == 0)", who);
    return LF_ERR_ARG;
  }
  if (!p) {
    set_err(c, "%s: NULL buffer", who);
    return LF_ERR_ARG;
  }
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_set_partial_densities(lf_ctx* c, const void* rho_y, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = species_args(c, rho_y, "lf_set_partial_densities")) return st;
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  for (int k = 0; k < c->nspecies; ++k)
    if (lf_status st = copy_plane_in(c, c->sp0 + k, static_cast<const char*>(rho_y) + k * n * c->elem, kind))
      return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_partial_densities(lf_ctx* c, void* rho_y, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = species_args(c, rho_y, "lf_get_partial_densities")) return st;
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  for (int k = 0; k < c->nspecies; ++k)
    if (lf_status st = copy_plane_out(c, c->sp0 + k, static_cast<char*>(rho_y) + k * n * c->elem, kind)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_set_mass_fractions(lf_ctx* c, const void* y, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = species_args(c, y, "lf_set_mass_fractions")) return st;
  DeviceGuard g(c->cfg.device);
  const size_t bytes = (size_t)c->nspecies * c->mesh.nx * c->mesh.ny * c->elem;
  const void* src = y;
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;  // 4 planes >= LF_MAX_SPECIES planes
    LF_CUDA(c, cudaMemcpyAsync(c->staging, y, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->staging;
  }
  cudaError_t e;
  if (c->cfg.dim == 3)
    e = c->elem == 8 ? lf::launch_species_to_cons3d(c->mesh3, static_cast<const double*>(src),
                                                    static_cast<double*>(c->U), c->stream)
                     : lf::launch_species_to_cons3d(c->mesh3, static_cast<const float*>(src),
                                                    static_cast<float*>(c->U), c->stream);
  else
    e = c->elem == 8 ? lf::launch_species_to_cons<double>(c->mesh, static_cast<const double*>(src),
                                                         static_cast<double*>(c->U), c->stream)
                     : lf::launch_species_to_cons<float>(c->mesh, static_cast<const float*>(src),
                                                        static_cast<float*>(c->U), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "species_to_cons launch");
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_mass_fractions(lf_ctx* c, void* y, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (lf_status st = species_args(c, y, "lf_get_mass_fractions")) return st;
  DeviceGuard g(c->cfg.device);
  const size_t bytes = (size_t)c->nspecies * c->mesh.nx * c->mesh.ny * c->elem;
  void* dst = y;
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;
    dst = c->staging;
  }
  cudaError_t e;
  if (c->cfg.dim == 3)
    e = c->elem == 8 ? lf::launch_cons_to_species3d(c->mesh3, static_cast<const double*>(c->U),
                                                    static_cast<double*>(dst), c->stream)
                     : lf::launch_cons_to_species3d(c->mesh3, static_cast<const float*>(c->U),
                                                    static_cast<float*>(dst), c->stream);
  else
    e = c->elem == 8 ? lf::launch_cons_to_species<double>(c->mesh, static_cast<const double*>(c->U),
                                                         static_cast<double*>(dst), c->stream)
                     : lf::launch_cons_to_species<float>(c->mesh, static_cast<const float*>(c->U),
                                                        static_cast<float*>(dst), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cons_to_species launch");
  if (!on_device) {
    LF_CUDA(c, cudaMemcpyAsync(y, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    LF_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LF_OK;
}

lf_status lf_set_conservative(lf_ctx* c, const void* U, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!U) {
    set_err(c, "lf_set_conservative: NULL buffer");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  for (int l = 0; l < c->nf; ++l)
    if (lf_status st = copy_plane_in(c, l, static_cast<const char*>(U) + l * n * c->elem, kind)) return st;
  if (lf_status st = restart_clock(c)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_conservative(lf_ctx* c, void* U, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!U) {
    set_err(c, "lf_get_conservative: NULL buffer");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  for (int l = 0; l < c->nf; ++l)
    if (lf_status st = copy_plane_out(c, l, static_cast<char*>(U) + l * n * c->elem, kind)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_set_primitives(lf_ctx* c, const void* q, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!q) {
    set_err(c, "lf_set_primitives: NULL buffer");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  const char* src = static_cast<const char*>(q);
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;
    LF_CUDA(c, cudaMemcpyAsync(c->staging, q, c->nf * n * c->elem, cudaMemcpyHostToDevice, c->stream));
    src = static_cast<const char*>(c->staging);
  }
  cudaError_t e;
  if (c->cfg.dim == 3) {
    e = c->elem == 8 ? lf::launch_prim_to_cons3d(c->mesh3, (const double*)src, static_cast<double*>(c->U), c->stream)
                     : lf::launch_prim_to_cons3d(c->mesh3, (const float*)src, static_cast<float*>(c->U), c->stream);
  } else {
    const size_t pb = n * c->elem;
    if (c->elem == 8)
      e = lf::launch_prim_to_cons<double>(c->mesh, (const double*)src, (const double*)(src + pb),
                                          (const double*)(src + 2 * pb), (const double*)(src + 3 * pb), (long long)n,
                                          static_cast<double*>(c->U), c->stream);
    else
      e = lf::launch_prim_to_cons<float>(c->mesh, (const float*)src, (const float*)(src + pb),
                                         (const float*)(src + 2 * pb), (const float*)(src + 3 * pb), (long long)n,
                                         static_cast<float*>(c->U), c->stream);
    if (e == cudaSuccess && c->mesh.nspecies > 0)
      e = c->elem == 8 ? lf::launch_species_to_cons<double>(c->mesh, (const double*)(src + 4 * pb),
                                                           static_cast<double*>(c->U), c->stream)
                       : lf::launch_species_to_cons<float>(c->mesh, (const float*)(src + 4 * pb),
                                                          static_cast<float*>(c->U), c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "primitive conversion launch");
  if (lf_status st = restart_clock(c)) return st;
  if (!on_device) LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_get_primitives(lf_ctx* c, void* q, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!q) {
    set_err(c, "lf_get_primitives: NULL buffer");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  const size_t n = (size_t)c->mesh.nx * c->mesh.ny;
  char* dst = static_cast<char*>(q);
  if (!on_device) {
    if (lf_status st = ensure_staging(c)) return st;
    dst = static_cast<char*>(c->staging);
  }
  cudaError_t e;
  if (c->cfg.dim == 3) {
    e = c->elem == 8 ? lf::launch_cons_to_prim3d(c->mesh3, static_cast<const double*>(c->U), (double*)dst, c->stream)
                     : lf::launch_cons_to_prim3d(c->mesh3, static_cast<const float*>(c->U), (float*)dst, c->stream);
  } else {
    const size_t pb = n * c->elem;
    if (c->elem == 8)
      e = lf::launch_cons_to_prim<double>(c->mesh, static_cast<double*>(c->U), (double*)dst, (double*)(dst + pb),
                                          (double*)(dst + 2 * pb), (double*)(dst + 3 * pb), c->stream);
    else
      e = lf::launch_cons_to_prim<float>(c->mesh, static_cast<float*>(c->U), (float*)dst, (float*)(dst + pb),
                                         (float*)(dst + 2 * pb), (float*)(dst + 3 * pb), c->stream);
    if (e == cudaSuccess && c->mesh.nspecies > 0)
      e = c->elem == 8 ? lf::launch_cons_to_species<double>(c->mesh, static_cast<const double*>(c->U),
                                                           (double*)(dst + 4 * pb), c->stream)
                       : lf::launch_cons_to_species<float>(c->mesh, static_cast<const float*>(c->U),
                                                          (float*)(dst + 4 * pb), c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "primitive conversion launch");
  if (!on_device) {
    LF_CUDA(c, cudaMemcpyAsync(q, dst, c->nf * n * c->elem, cudaMemcpyDeviceToHost, c->stream));
    LF_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LF_OK;
}

lf_status lf_step(lf_ctx* c, double* dt_out) {
  if (!c) return LF_ERR_ARG;
  if (!c->has_state) {
    set_err(c, "lf_step: no state set");
    return LF_ERR_STATE;
  }
  DeviceGuard g(c->cfg.device);
  if (lf_status st = enqueue_step(c, 0.0)) return st;
  if (dt_out) {
    if (lf_status st = read_scalars(c)) return st;
    *dt_out = c->hsc->dt;
    return device_error_status(c);
  }
  return LF_OK;
}

lf_status lf_step_fixed(lf_ctx* c, double dt) {
  if (!c) return LF_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) {
    set_err(c, "lf_step_fixed: dt must be positive and finite");
    return LF_ERR_ARG;
  }
  if (!c->has_state) {
    set_err(c, "lf_step_fixed: no state set");
    return LF_ERR_STATE;
  }
  DeviceGuard g(c->cfg.device);
  return enqueue_step(c, dt);
}

namespace {

constexpr int kRunBatch = 32;  // steps per graph replay in lf_run

// kRunBatch steps as one graph launch (steps past t_end are device-side
// no-ops).  Falls back to direct launches while stage tracing is on, since
// the tracing events are host-side bookkeeping.
lf_status enqueue_batch(lf_ctx* c, int nsteps) {
  if (nsteps != kRunBatch || c->profiling) {
    for (int k = 0; k < nsteps; ++k)
      if (lf_status st = enqueue_step(c, 0.0)) return st;
    return LF_OK;
  }
  if (!c->run_graph) {
    if (!c->capture) LF_CUDA(c, cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    LF_CUDA(c, cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeRelaxed));
    cudaStream_t user = c->stream;
    c->stream = c->capture;
    lf_status st = LF_OK;
    for (int k = 0; k < nsteps && st == LF_OK; ++k) st = enqueue_step(c, 0.0);
    c->stream = user;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
    if (st != LF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->run_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  LF_CUDA(c, cudaGraphLaunch(c->run_graph, c->stream));
  return LF_OK;
}

}  // namespace

lf_status lf_run(lf_ctx* c, double t_end, int32_t max_steps, int32_t* steps_done, double* t_out) {
  if (!c) return LF_ERR_ARG;
  if (max_steps < 0 || !std::isfinite(t_end)) {
    set_err(c, "lf_run: max_steps must be >= 0 and t_end finite");
    return LF_ERR_ARG;
  }
  if (!c->has_state) {
    set_err(c, "lf_run: no state set");
    return LF_ERR_STATE;
  }
  DeviceGuard g(c->cfg.device);
  if (lf_status st = read_scalars(c)) return st;
  const long long steps0 = c->hsc->steps;
  LF_CUDA(c, lf::launch_set_t_end(c->sc, t_end > 0.0 ? t_end : 0.0, c->stream));
  // Steps are enqueued in batches of kRunBatch (one graph replay each); with
  // a final time the host polls t between batches, and steps past t_end are
  // device-side no-ops.
  int launched = 0;
  lf_status st = LF_OK;
  while (launched < max_steps) {
    const int nb = max_steps - launched < kRunBatch ? max_steps - launched : kRunBatch;
    if ((st = enqueue_batch(c, nb)) != LF_OK) break;
    launched += nb;
    if (t_end > 0.0 || launched >= max_steps) {
      if ((st = read_scalars(c)) != LF_OK) break;
      if (c->hsc->err || (t_end > 0.0 && c->hsc->t >= t_end)) break;
    }
  }
  lf_status st2 = LF_OK;
  if (cudaError_t e = lf::launch_set_t_end(c->sc, 0.0, c->stream)) st2 = cuda_fail(c, e, "set_t_end");
  if (st == LF_OK) st = st2;
  if (st == LF_OK) st = read_scalars(c);
  if (st != LF_OK) return st;
  if (steps_done) *steps_done = (int32_t)(c->hsc->steps - steps0);
  if (t_out) *t_out = c->hsc->t;
  return device_error_status(c);
}

lf_status lf_get_time(lf_ctx* c, double* t, int64_t* steps) {
  if (!c) return LF_ERR_ARG;
  DeviceGuard g(c->cfg.device);
  if (lf_status st = read_scalars(c)) return st;
  if (t) *t = c->hsc->t;
  if (steps) *steps = c->hsc->steps;
  return LF_OK;
}

lf_status lf_conservation_sums(lf_ctx* c, double* out) {
  if (!c || !out) return LF_ERR_ARG;
  DeviceGuard g(c->cfg.device);
  // planes past the first four are summed as the view's extra planes
  lf::MeshDesc view = c->mesh;
  view.nspecies = c->nf - 4;
  cudaError_t e = c->elem == 8 ? lf::launch_sums<double>(view, static_cast<double*>(c->U), c->partials,
                                                         lf::sums_blocks(), c->dsums, c->stream)
                               : lf::launch_sums<float>(view, static_cast<float*>(c->U), c->partials,
                                                        lf::sums_blocks(), c->dsums, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "sums launch");
  LF_CUDA(c, cudaMemcpyAsync(out, c->dsums, c->nf * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_profile_enable(lf_ctx* c, int enable) {
  if (!c) return LF_ERR_ARG;
  DeviceGuard g(c->cfg.device);
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  c->profiling = enable != 0;
  c->ev_used = 0;
  c->ev_stage.clear();
  return LF_OK;
}

lf_status lf_profile_read(lf_ctx* c, double ms[2], int64_t launches[2]) {
  if (!c || !ms || !launches) return LF_ERR_ARG;
  DeviceGuard g(c->cfg.device);
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (size_t k = 0; k < c->ev_used; ++k) {
    float t = 0.0f;
    LF_CUDA(c, cudaEventElapsedTime(&t, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]));
    ms[c->ev_stage[k]] += t;
    launches[c->ev_stage[k]] += 1;
  }
  return LF_OK;
}

namespace {

// Rows (2D) or planes (3D) per tile of the march; 0 for 1D meshes.
int tile_of(const lf_ctx* c) { return c->cfg.dim == 3 ? c->mesh3.tz : c->cfg.dim == 2 ? c->mesh.ty : 0; }

void set_tile(lf_ctx* c, int rows) {
  if (c->cfg.dim == 3) c->mesh3.tz = rows;
  else c->mesh.ty = rows;
  if (c->run_graph) {  // the recorded steps carry the old launch shape
    cudaGraphExecDestroy(c->run_graph);
    c->run_graph = nullptr;
  }
}

}  // namespace

lf_status lf_set_tile_rows(lf_ctx* c, int32_t rows) {
  if (!c) return LF_ERR_ARG;
  if (c->cfg.dim == 1 || rows < 1 || rows > 4096) {
    set_err(c, "lf_set_tile_rows: needs a 2D or 3D mesh and 1 <= rows <= 4096");
    return LF_ERR_ARG;
  }
  DeviceGuard g(c->cfg.device);
  LF_CUDA(c, cudaStreamSynchronize(c->stream));  // a replay in flight keeps the old graph
  set_tile(c, rows);
  return LF_OK;
}

lf_status lf_get_tile_rows(lf_ctx* c, int32_t* rows) {
  if (!c || !rows) return LF_ERR_ARG;
  *rows = tile_of(c);
  return LF_OK;
}

lf_status lf_autotune(lf_ctx* c, int32_t trial_steps, int32_t* chosen_rows) {
  if (!c) return LF_ERR_ARG;
  if (c->cfg.dim == 1 || trial_steps < 1) {
    set_err(c, "lf_autotune: needs a 2D or 3D mesh and trial_steps >= 1");
    return LF_ERR_ARG;
  }
  if (!c->has_state) {
    set_err(c, "lf_autotune: no state set");
    return LF_ERR_STATE;
  }
  DeviceGuard g(c->cfg.device);
  const size_t bytes = c->nf * (size_t)c->mesh.plane * c->elem;
  void* save = nullptr;
  lf::Scalars* save_sc = nullptr;
  LF_CUDA(c, cudaMalloc(&save, bytes));
  cudaError_t e = cudaMalloc(&save_sc, sizeof(lf::Scalars));
  if (e != cudaSuccess) {
    cudaFree(save);
    return cuda_fail(c, e, "lf_autotune: cudaMalloc");
  }
  // the trial steps advance the state: copy it (and dt, t, the step count)
  // and put it back after every candidate
  e = cudaMemcpyAsync(save, c->U, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(save_sc, c->sc, sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, c->stream);
  const int cand2[] = {4, 8, 16, 32, 64, 128};
  const int cand3[] = {8, 16, 32, 64};
  const int* cand = c->cfg.dim == 3 ? cand3 : cand2;
  const int ncand = c->cfg.dim == 3 ? 4 : 6;
  const bool profiling = c->profiling;
  c->profiling = false;
  const int before = tile_of(c);
  int best = before;
  float best_ms = 1e30f;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  lf_status st = e == cudaSuccess ? LF_OK : cuda_fail(c, e, "lf_autotune");
  for (int i = 0; i < ncand && st == LF_OK; ++i) {
    set_tile(c, cand[i]);
    if ((st = lf::enqueue_step(c, 0.0)) != LF_OK) break;  // warm-up
    if ((e = cudaEventRecord(t0, c->stream)) != cudaSuccess) break;
    for (int k = 0; k < trial_steps && st == LF_OK; ++k) st = lf::enqueue_step(c, 0.0);
    if (st != LF_OK) break;
    if ((e = cudaEventRecord(t1, c->stream)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(t1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = cand[i];
    }
    if ((e = cudaMemcpyAsync(c->U, save, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(c->sc, save_sc, sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, c->stream)) !=
        cudaSuccess)
      break;
  }
  if (st == LF_OK && e != cudaSuccess) st = cuda_fail(c, e, "lf_autotune");
  cudaMemcpyAsync(c->U, save, bytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->sc, save_sc, sizeof(lf::Scalars), cudaMemcpyDeviceToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(save);
  cudaFree(save_sc);
  c->profiling = profiling;
  set_tile(c, st == LF_OK ? best : before);
  if (st != LF_OK) return st;
  if (chosen_rows) *chosen_rows = best;
  return LF_OK;
}

lf_status lf_sync(lf_ctx* c) {
  if (!c) return LF_ERR_ARG;
  DeviceGuard g(c->cfg.device);
  if (lf_status st = read_scalars(c)) return st;
  return device_error_status(c);
}

}  // extern "C"
