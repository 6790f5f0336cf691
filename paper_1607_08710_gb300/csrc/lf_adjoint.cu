// Discrete adjoint of the Heun/RK2 Lagrange-flux step (arXiv:1607.08710,
// Sec. 4) with sqrt(N) checkpointing of the time loop (C ABI lf_adjoint_*).
//
// lf_adjoint_forward runs N CFL steps from the context's state, keeping a
// checkpoint every S = ceil(sqrt(N)) steps and the dt of every step (the dt
// sequence is frozen for the derivative).  lf_adjoint_backward sweeps the
// segments backwards: it recomputes a segment's states from its checkpoint,
// then reverses its steps one by one with the face/cell adjoint kernels.
// Memory: ceil(N/S) + S states plus a few work states, instead of N, and in
// FP64 the prep tables of one state (28 values per cell).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "lf_host.h"

namespace {

using lf::cuda_fail;
using lf::set_err;

lf_status grow(lf_ctx* c, void** buf, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return LF_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  LF_CUDA(c, cudaMalloc(buf, bytes));
  *cap = bytes;
  return LF_OK;
}

char* state_ptr(lf_ctx* c, void* base, size_t k) {
  return static_cast<char*>(base) + k * c->adj.state_elems * c->elem;
}

const char* adjoint_unsupported(const lf_ctx* c) {
  if (c->cfg.dim != 2) return "the adjoint is implemented for 2D meshes";
  if (c->cfg.riemann != LF_RIEMANN_MAXC) return "the adjoint is implemented for the eqs. 13-14 solver (max c)";
  if (c->cfg.time_order == LF_TIME_SSPRK3) return "the adjoint is implemented for the Heun time integrator";
  if (c->cfg.nspecies != 0) return "the adjoint is implemented for the gas dynamics without species";
  return nullptr;
}

bool uses_tables(const lf_ctx* c) {
  if (c->adj_passes == LF_ADJOINT_PASSES_TABLES) return true;
  if (c->adj_passes == LF_ADJOINT_PASSES_DIRECT) return false;
  return c->elem == 8;
}

template <typename T>
lf_status backward_t(lf_ctx* c) {
  auto& A = c->adj;
  const lf::MeshDesc& m = c->mesh;
  cudaStream_t s = c->stream;
  T* lam = static_cast<T*>(A.lam);
  T* lamstar = static_cast<T*>(A.lamstar);
  T* fx = static_cast<T*>(A.fx);
  T* fy = static_cast<T*>(A.fy);
  const bool tables = uses_tables(c);
  if (tables) {
    const size_t prep_elems =
        4 * (size_t)m.nx * m.ny + 12 * ((size_t)(m.nx + 2) * m.ny + (size_t)(m.ny + 2) * m.nx);
    if (lf_status st = grow(c, &A.prep, &A.prep_cap, prep_elems * c->elem)) return st;
  }
  T* Q = static_cast<T*>(A.prep);
  T* tabx = tables ? Q + 4 * (size_t)m.nx * m.ny : nullptr;
  T* taby = tables ? tabx + 12 * (size_t)(m.nx + 2) * m.ny : nullptr;
  T* Us = static_cast<T*>(c->Ustar);
  LF_CUDA(c, lf::launch_reset_scalars(A.sc, c->cfg.cfl, s));
  const int nseg = (A.nsteps + A.seg - 1) / A.seg;
  for (int g = nseg - 1; g >= 0; --g) {
    const int n0 = g * A.seg;
    const int len = A.nsteps - n0 < A.seg ? A.nsteps - n0 : A.seg;
    // states of the segment: X[0] is the checkpoint, X[k] the recomputed step k
    auto X = [&](int k) -> T* {
      return reinterpret_cast<T*>(k == 0 ? state_ptr(c, A.ck, g) : state_ptr(c, A.segbuf, k - 1));
    };
    for (int k = 0; k + 1 < len; ++k) {
      LF_CUDA(c, lf::launch_begin_step(A.sc, A.dts[n0 + k], s));
      LF_CUDA(c, lf::launch_stage<T>(0, m, X(k), X(k), Us, A.sc, s));
      LF_CUDA(c, lf::launch_stage<T>(1, m, Us, X(k), X(k + 1), A.sc, s));
      LF_CUDA(c, lf::launch_end_step(A.sc, s));
    }
    for (int k = len - 1; k >= 0; --k) {
      const double dt = A.dts[n0 + k];
      T* Un = X(k);
      // predictor state of this step
      LF_CUDA(c, lf::launch_begin_step(A.sc, dt, s));
      LF_CUDA(c, lf::launch_stage<T>(0, m, Un, Un, Us, A.sc, s));
      LF_CUDA(c, lf::launch_end_step(A.sc, s));
      // lambda* = lambda/2 - dt/2 (dD/dU)(U*)^T lambda, then
      // lambda <- lambda/2 + lambda* - dt (dD/dU)(U^n)^T lambda*.  The table
      // passes read the forward quantities from prep tables (FP64 default:
      // its divisions dominate); the direct passes recompute them (FP32
      // default: measured faster there).
      if (tables) {
        LF_CUDA(c, lf::launch_adjoint_prep<T>(m, Us, Q, tabx, taby, s));
        LF_CUDA(c, lf::launch_face_vjp<T>(m, 0, Q, tabx, lam, fx, s));
        LF_CUDA(c, lf::launch_face_vjp<T>(m, 1, Q, taby, lam, fy, s));
        LF_CUDA(c, lf::launch_cell_vjp<T>(m, Q, fx, fy, tabx, taby, lam, 0.5, nullptr, 0.0, -0.5 * dt, lamstar, s));
        LF_CUDA(c, lf::launch_adjoint_prep<T>(m, Un, Q, tabx, taby, s));
        LF_CUDA(c, lf::launch_face_vjp<T>(m, 0, Q, tabx, lamstar, fx, s));
        LF_CUDA(c, lf::launch_face_vjp<T>(m, 1, Q, taby, lamstar, fy, s));
        LF_CUDA(c, lf::launch_cell_vjp<T>(m, Q, fx, fy, tabx, taby, lam, 0.5, lamstar, 1.0, -dt, lam, s));
      } else {
        LF_CUDA(c, lf::launch_face_vjp_direct<T>(m, 0, Us, lam, fx, s));
        LF_CUDA(c, lf::launch_face_vjp_direct<T>(m, 1, Us, lam, fy, s));
        LF_CUDA(c, lf::launch_cell_vjp_direct<T>(m, Us, fx, fy, lam, 0.5, nullptr, 0.0, -0.5 * dt, lamstar, s));
        LF_CUDA(c, lf::launch_face_vjp_direct<T>(m, 0, Un, lamstar, fx, s));
        LF_CUDA(c, lf::launch_face_vjp_direct<T>(m, 1, Un, lamstar, fy, s));
        LF_CUDA(c, lf::launch_cell_vjp_direct<T>(m, Un, fx, fy, lam, 0.5, lamstar, 1.0, -dt, lam, s));
      }
    }
  }
  return LF_OK;
}

}  // namespace

void lf::free_adjoint(lf_ctx* c) {
  auto& A = c->adj;
  cudaFree(A.ck);
  cudaFree(A.segbuf);
  cudaFree(A.lam);
  cudaFree(A.lamstar);
  cudaFree(A.fx);
  cudaFree(A.fy);
  cudaFree(A.prep);
  cudaFree(A.dts_dev);
  cudaFree(A.sc);
  A = lf_ctx::Adjoint();
}

extern "C" {

lf_status lf_adjoint_forward(lf_ctx* c, int32_t nsteps, double* dts_out) {
  if (!c) return LF_ERR_ARG;
  if (const char* why = adjoint_unsupported(c)) {
    set_err(c, "lf_adjoint_forward: %s", why);
    return LF_ERR_ARG;
  }
  if (nsteps < 1) {
    set_err(c, "lf_adjoint_forward: nsteps must be >= 1");
    return LF_ERR_ARG;
  }
  if (!c->has_state) {
    set_err(c, "lf_adjoint_forward: no state set");
    return LF_ERR_STATE;
  }
  lf::DeviceGuard guard(c->cfg.device);
  auto& A = c->adj;
  A.nsteps = 0;
  const int seg = (int)std::ceil(std::sqrt((double)nsteps));
  const int nck = (nsteps + seg - 1) / seg;
  const lf::MeshDesc& m = c->mesh;
  A.state_elems = 4 * (size_t)m.plane;
  const size_t sb = A.state_elems * c->elem;
  const size_t faces = (size_t)(m.nx + 1) * m.ny > (size_t)(m.ny + 1) * m.nx ? (size_t)(m.nx + 1) * m.ny
                                                                               : (size_t)(m.ny + 1) * m.nx;
  size_t lam_cap = A.lam ? sb : 0, lams_cap = A.lamstar ? sb : 0, fy_cap = A.fy ? A.face_cap : 0;
  size_t sc_cap = A.sc ? sizeof(lf::Scalars) : 0;
  if (lf_status st = grow(c, &A.ck, &A.ck_cap, (size_t)nck * sb)) return st;
  if (lf_status st = grow(c, &A.segbuf, &A.seg_cap, (size_t)(seg > 1 ? seg - 1 : 1) * sb)) return st;
  if (lf_status st = grow(c, &A.lam, &lam_cap, sb)) return st;
  if (lf_status st = grow(c, &A.lamstar, &lams_cap, sb)) return st;
  size_t fx_cap = A.face_cap;
  if (lf_status st = grow(c, &A.fx, &fx_cap, faces * 8 * c->elem)) return st;
  if (lf_status st = grow(c, &A.fy, &fy_cap, faces * 8 * c->elem)) return st;
  A.face_cap = fx_cap < fy_cap ? fx_cap : fy_cap;
  if (lf_status st = grow(c, reinterpret_cast<void**>(&A.dts_dev), &A.dts_cap, nsteps * sizeof(double))) return st;
  if (lf_status st = grow(c, reinterpret_cast<void**>(&A.sc), &sc_cap, sizeof(lf::Scalars))) return st;
  for (int n = 0; n < nsteps; ++n) {
    if (n % seg == 0)
      LF_CUDA(c, cudaMemcpyAsync(state_ptr(c, A.ck, n / seg), c->U, sb, cudaMemcpyDeviceToDevice, c->stream));
    if (lf_status st = lf::enqueue_step(c, 0.0)) return st;
    LF_CUDA(c, cudaMemcpyAsync(A.dts_dev + n, &c->sc->dt, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  A.dts.assign(nsteps, 0.0);
  LF_CUDA(c, cudaMemcpyAsync(A.dts.data(), A.dts_dev, nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (lf_status st = lf::read_scalars(c)) return st;
  if (lf_status st = lf::device_error_status(c)) return st;
  for (int n = 0; n < nsteps; ++n)
    if (!(A.dts[n] > 0.0)) {
      set_err(c, "lf_adjoint_forward: step %d did not advance (dt = %g)", n, A.dts[n]);
      return LF_ERR_STATE;
    }
  A.nsteps = nsteps;
  A.seg = seg;
  if (dts_out) std::memcpy(dts_out, A.dts.data(), nsteps * sizeof(double));
  return LF_OK;
}

lf_status lf_adjoint_backward(lf_ctx* c, const void* lambda_T, void* grad_U0, void* grad_q0, int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!lambda_T) {
    set_err(c, "lf_adjoint_backward: lambda_T is NULL");
    return LF_ERR_ARG;
  }
  if (c->adj.nsteps < 1) {
    set_err(c, "lf_adjoint_backward: no recorded forward run (call lf_adjoint_forward first)");
    return LF_ERR_STATE;
  }
  lf::DeviceGuard guard(c->cfg.device);
  auto& A = c->adj;
  const lf::MeshDesc& m = c->mesh;
  const size_t w = (size_t)m.nx * c->elem, dp = (size_t)m.pitch * c->elem;
  const size_t dense_plane = (size_t)m.nx * m.ny * c->elem;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int l = 0; l < 4; ++l)
    LF_CUDA(c, cudaMemcpy2DAsync(static_cast<char*>(A.lam) + (size_t)l * m.plane * c->elem, dp,
                                 static_cast<const char*>(lambda_T) + l * dense_plane, w, w, m.ny, kin, c->stream));
  lf_status st = c->elem == 8 ? backward_t<double>(c) : backward_t<float>(c);
  if (st != LF_OK) return st;
  if (grad_U0)
    for (int l = 0; l < 4; ++l)
      LF_CUDA(c, cudaMemcpy2DAsync(static_cast<char*>(grad_U0) + l * dense_plane, w,
                                   static_cast<const char*>(A.lam) + (size_t)l * m.plane * c->elem, dp, w, m.ny,
                                   kout, c->stream));
  if (grad_q0) {
    // host output: the dense planes are formed in the x-face buffer (at least
    // 8 (nx+1) ny values, more than the 4 nx ny needed) and copied out
    void* gq = on_device ? grad_q0 : A.fx;
    cudaError_t e = c->elem == 8
        ? lf::launch_grad_prim<double>(m, static_cast<const double*>(A.ck), static_cast<const double*>(A.lam),
                                       static_cast<double*>(gq), c->stream)
        : lf::launch_grad_prim<float>(m, static_cast<const float*>(A.ck), static_cast<const float*>(A.lam),
                                      static_cast<float*>(gq), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "grad_prim launch");
    if (!on_device) LF_CUDA(c, cudaMemcpyAsync(grad_q0, gq, 4 * dense_plane, kout, c->stream));
  }
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  return LF_OK;
}

lf_status lf_adjoint(lf_ctx* c, int32_t nsteps, const void* lambda_T, void* grad_U0, void* grad_q0, double* dts_out,
                     int on_device) {
  if (!c) return LF_ERR_ARG;
  if (!lambda_T) {
    set_err(c, "lf_adjoint: lambda_T is NULL");
    return LF_ERR_ARG;
  }
  if (lf_status st = lf_adjoint_forward(c, nsteps, dts_out)) return st;
  return lf_adjoint_backward(c, lambda_T, grad_U0, grad_q0, on_device);
}

lf_status lf_adjoint_set_passes(lf_ctx* c, int32_t passes) {
  if (!c) return LF_ERR_ARG;
  if (passes != LF_ADJOINT_PASSES_AUTO && passes != LF_ADJOINT_PASSES_TABLES && passes != LF_ADJOINT_PASSES_DIRECT) {
    set_err(c, "lf_adjoint_set_passes: passes must be LF_ADJOINT_PASSES_AUTO, _TABLES or _DIRECT (got %d)", passes);
    return LF_ERR_ARG;
  }
  c->adj_passes = passes;
  return LF_OK;
}

}  // extern "C"
