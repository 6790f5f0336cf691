// Host-side internals shared by the C-ABI translation units: the context
// structure and small helpers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/lagflux.h"
#include "lf_internal.h"
#include "lf_internal3d.h"

struct lf_ctx {
  lf_config cfg;
  lf::MeshDesc mesh;          // 1D/2D mesh; for 3D the row view (ny*nz rows of nx cells)
  lf::Mesh3Desc mesh3{};      // 3D meshes only
  int nf = 4;                 // state planes: 4 (+1 in 3D) + nspecies
  int nspecies = 0;           // transported mass fractions
  int sp0 = 4;                // first species plane (4, or 5 in 3D)
  cudaStream_t stream = nullptr;
  size_t elem = 8;            // bytes per element
  void* U = nullptr;          // current state, nf pitched planes
  void* Ustar = nullptr;      // Heun predictor / first RK3 stage, nf pitched planes
  void* U2 = nullptr;         // second SSP-RK3 stage (time_order 3 only)
  void* staging = nullptr;    // dense max(4, nf) planes for host transfers (lazy)
  lf::Scalars* sc = nullptr;  // device scalars
  lf::Scalars* hsc = nullptr; // pinned host mirror for read-back
  double* partials = nullptr; // conservation-sum partials
  double* dsums = nullptr;    // nf device doubles
  bool has_state = false;
  // lf_run replays a CUDA graph of kRunBatch steps (recorded once, on a
  // private stream; replayed on `stream`)
  cudaStream_t capture = nullptr;
  cudaGraphExec_t run_graph = nullptr;
  // stage tracing: event pairs recorded around each stage launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_stage;   // stage of each recorded pair
  size_t ev_used = 0;          // pairs recorded
  // discrete adjoint (lf_adjoint_*): checkpoints of the forward run and work buffers
  struct Adjoint {
    int nsteps = 0;            // steps of the recorded forward run (0: none)
    int seg = 0;               // checkpoint interval
    std::vector<double> dts;   // frozen dt sequence
    size_t state_elems = 0;    // elements of one state (4 planes)
    size_t ck_cap = 0, seg_cap = 0, face_cap = 0, dts_cap = 0, prep_cap = 0;
    void* ck = nullptr;        // checkpoints: ceil(nsteps / seg) states
    void* segbuf = nullptr;    // recomputed states of one segment
    void* lam = nullptr;       // cotangent of the state
    void* lamstar = nullptr;   // cotangent of the predictor state
    void* fx = nullptr;        // face-state cotangents, x-faces
    void* fy = nullptr;        // face-state cotangents, y-faces
    void* prep = nullptr;      // primitives (4 dense planes) and the x and y slope tables of one state
    double* dts_dev = nullptr; // dt of each forward step, recorded on the device
    lf::Scalars* sc = nullptr; // scalars of the recomputation
  } adj;
  int adj_passes = LF_ADJOINT_PASSES_AUTO;  // lf_adjoint_set_passes
  char last_error[512] = {0};
};

namespace lf {

void set_err(lf_ctx* c, const char* fmt, ...);
lf_status cuda_fail(lf_ctx* c, cudaError_t e, const char* what);
// One Heun step on the context (dt_fixed > 0: that dt; else the CFL dt).
lf_status enqueue_step(lf_ctx* c, double dt_fixed);
lf_status read_scalars(lf_ctx* c);
lf_status device_error_status(lf_ctx* c);
void free_adjoint(lf_ctx* c);

// Makes the context's device current for the duration of a call and puts
// the caller's device back afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace lf

#define LF_CUDA(ctx, call)                                      \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return lf::cuda_fail(ctx, e_, #call); \
  } while (0)
