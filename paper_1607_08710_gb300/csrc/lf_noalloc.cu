// lf_step_noalloc: one Heun step that allocates no device memory.
//
// Who needs this.  Some callers cannot call cudaMalloc: code that runs inside
// another framework's memory manager, which owns all of the GPU's memory and
// must not be bypassed; code that must not allocate inside a time-critical
// loop, because cudaMalloc/cudaFree can synchronise the whole device; and
// hosts that reserve the GPU's memory up front so that a later allocation
// would fail.  lf_init allocates a context (two states and scalars), so it is
// closed to them.  This entry point instead keeps its scratch -- the Heun
// predictor state U* and the step's scalars -- in one fixed array compiled
// into this library.
//
// The array is a file-scope static __device__ variable: every GPU that loads
// the library holds it (LF_NOALLOC_SCRATCH_BYTES) until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the first call on each device looks up the
// real address with cudaGetSymbolAddress, with that device current, checks
// the result and caches it; later calls reuse it.  A failed lookup is not
// cached: the next call tries again.  Because the lookup may load the module,
// the first call on a device must come before any stream capture; a first
// call made on a stream that is being captured is refused (LF_ERR_ARG) before
// it touches the device.
//
// Every call shares the one array and the array keeps the previous call's
// contents: each call clears the scalars it needs (dt, wave-speed maximum,
// error flags) before use.  Two calls whose work overlaps on the GPU (e.g. on
// different streams) race on the array and give undefined results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lagflux.h"
#include "lf_internal.h"
#include "lf_stage.cuh"

namespace {

constexpr long long kMaxCells = LF_NOALLOC_MAX_CELLS;
constexpr size_t kScalarBytes = 256;
constexpr size_t kScratchBytes = kScalarBytes + 4 * (size_t)kMaxCells * sizeof(double);
static_assert(sizeof(lf::Scalars) <= kScalarBytes, "scalars do not fit their slot");
static_assert(kScratchBytes == LF_NOALLOC_SCRATCH_BYTES, "header and library disagree on the scratch size");

// The scratch: [0, 256) step scalars, [256, ...) the predictor state U* as
// four dense planes of nx*ny elements (FP64 or FP32).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mutex;
bool g_found[kMaxDevices];
void* g_scratch_addr[kMaxDevices];

// The device address of g_scratch on `dev` (the current device), looked up
// on the first successful call for that device and cached.
lf_status scratch_address(int dev, cudaStream_t s, void** out) {
  std::lock_guard<std::mutex> lock(g_lookup_mutex);
  if (!g_found[dev]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();  // leave no pending error for the caller's next launch check
      lf::set_init_error("lf_step_noalloc: the first call on device %d looks up the scratch address and must not "
                         "be made while its stream is being captured (%s)",
                         dev, e != cudaSuccess ? cudaGetErrorString(e) : "stream is capturing");
      return LF_ERR_ARG;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      lf::set_init_error("lf_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return LF_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
    g_found[dev] = true;
  }
  *out = g_scratch_addr[dev];
  return LF_OK;
}

// The FP32 stage kernels move CPL consecutive cells of a lane with one vector
// copy (CPL * sizeof(T) bytes) when the mesh description allows it (m.vec);
// FP64 kernels (CPL = 1) copy single cells.  Vector copies start at even
// columns of every row of every plane, so dense planes need nx to be a
// multiple of CPL and both state buffers aligned to the vector width.
template <typename T>
bool vector_access_ok(int nx, const void* a, const void* b) {
  constexpr int cpl = lf::StageShape<T>::CPL;
  constexpr uintptr_t bytes = cpl * sizeof(T);
  static_assert(bytes == 8, "stage kernels copy 8-byte lane vectors (FP32 pairs, FP64 cells)");
  return nx % cpl == 0 && (uintptr_t)a % bytes == 0 && (uintptr_t)b % bytes == 0;
}

const char* check_config(const lf_config* c) {
  if (!c) return "config is NULL";
  if (c->dim != 1 && c->dim != 2) return "dim must be 1 or 2";
  if (c->nx < 1 || c->ny < 1 || (c->dim == 1 && c->ny != 1)) return "bad mesh size";
  if ((long long)c->nx * c->ny > kMaxCells) return "mesh larger than LF_NOALLOC_MAX_CELLS";
  if (c->limiter < 0 || c->limiter > 2 || c->bc < 0 || c->bc > 1 || c->riemann < 0 || c->riemann > 1)
    return "unknown limiter, boundary condition or interface solver";
  if (c->precision != LF_FP64 && c->precision != LF_FP32) return "unknown precision";
  if (c->tile_rows < 0 || c->tile_rows > 4096) return "tile_rows must be in 0 .. 4096";
  if (c->device < 0 || c->device >= kMaxDevices) return "device out of range";
  if (!(c->xmax > c->xmin) || (c->dim == 2 && !(c->ymax > c->ymin))) return "empty domain";
  if (!(c->gamma > 1.0 && c->gamma <= 3.0) || !(c->cfl > 0.0 && c->cfl <= 1.0)) return "gamma or cfl out of range";
  if (c->limiter == LF_LIMITER_SWEBY && !(c->beta >= 1.0 && c->beta <= 2.0)) return "beta out of range";
  if (c->time_order != 0 && c->time_order != LF_TIME_HEUN) return "only the Heun time integrator";
  if (c->nspecies != 0) return "no species";
  return nullptr;
}

template <typename T>
cudaError_t enqueue(const lf::MeshDesc& m, const T* Uin, T* Uout, T* Ustar, lf::Scalars* sc, double dt,
                    double cfl, cudaStream_t s) {
  cudaError_t e = lf::launch_reset_scalars(sc, cfl, s);
  if (e == cudaSuccess && !(dt > 0.0)) e = lf::launch_wave_speed<T>(m, Uin, sc, s);
  if (e == cudaSuccess) e = lf::launch_begin_step(sc, dt > 0.0 ? dt : 0.0, s);
  if (e == cudaSuccess) e = lf::launch_stage<T>(0, m, Uin, Uin, Ustar, sc, s);
  if (e == cudaSuccess) e = lf::launch_stage<T>(1, m, Ustar, Uin, Uout, sc, s);
  if (e == cudaSuccess) e = lf::launch_end_step(sc, s);
  return e;
}

}  // namespace

extern "C" lf_status lf_step_noalloc(const lf_config* cfg, const void* U_in, void* U_out, double dt,
                                     double* dt_used, void* stream) {
  if (const char* why = check_config(cfg)) {
    lf::set_init_error("lf_step_noalloc: %s (limit %lld cells)", why, kMaxCells);
    return LF_ERR_ARG;
  }
  if (!U_in || !U_out || !std::isfinite(dt)) {
    lf::set_init_error("lf_step_noalloc: NULL state buffer or non-finite dt");
    return LF_ERR_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != cfg->device && cudaSetDevice(cfg->device) != cudaSuccess) {
    lf::set_init_error("lf_step_noalloc: cannot select device %d", cfg->device);
    return LF_ERR_CUDA;
  }
  void* base = nullptr;
  lf_status st = scratch_address(cfg->device, static_cast<cudaStream_t>(stream), &base);
  if (st == LF_OK) {
    lf::MeshDesc m;
    m.nx = cfg->nx;
    m.ny = cfg->ny;
    m.pitch = cfg->nx;
    m.plane = (long long)cfg->nx * cfg->ny;
    m.dim = cfg->dim;
    m.bc = cfg->bc;
    m.limiter = cfg->limiter;
    m.riemann = cfg->riemann;
    m.gamma = cfg->gamma;
    m.beta = cfg->limiter == LF_LIMITER_MINMOD ? 1.0 : cfg->beta;
    m.rdx = cfg->nx / (cfg->xmax - cfg->xmin);
    m.rdy = cfg->dim == 2 ? cfg->ny / (cfg->ymax - cfg->ymin) : 0.0;
    // dense planes (pitch nx): vector access only when every row and plane start stays aligned
    m.vec = cfg->precision == LF_FP64 ? vector_access_ok<double>(cfg->nx, U_in, U_out)
                                      : vector_access_ok<float>(cfg->nx, U_in, U_out);
    if (cfg->dim == 2) {  // the tile height of lf_init contexts (or the configured one)
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess) sms = 0;
      m.ty = cfg->tile_rows > 0 ? cfg->tile_rows : lf::auto_tile_rows(m, cfg->precision == LF_FP32 ? 2 : 1, sms);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lf::Scalars* sc = static_cast<lf::Scalars*>(base);
    void* ustar = static_cast<unsigned char*>(base) + kScalarBytes;
    cudaError_t e;
    if (cfg->precision == LF_FP64)
      e = enqueue<double>(m, static_cast<const double*>(U_in), static_cast<double*>(U_out),
                          static_cast<double*>(ustar), sc, dt, cfg->cfl, s);
    else
      e = enqueue<float>(m, static_cast<const float*>(U_in), static_cast<float*>(U_out),
                         static_cast<float*>(ustar), sc, dt, cfg->cfl, s);
    if (e != cudaSuccess) {
      lf::set_init_error("lf_step_noalloc: launch failed: %s", cudaGetErrorString(e));
      st = LF_ERR_CUDA;
    } else if (dt_used) {
      lf::Scalars h;
      e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        lf::set_init_error("lf_step_noalloc: %s", cudaGetErrorString(e));
        st = LF_ERR_CUDA;
      } else {
        *dt_used = h.dt;
        if (h.err) {
          lf::set_init_error("lf_step_noalloc: non-positive density or pressure, or bad dt");
          st = LF_ERR_NONPHYSICAL;
        }
      }
    }
  }
  if (prev >= 0 && prev != cfg->device) cudaSetDevice(prev);
  return st;
}
