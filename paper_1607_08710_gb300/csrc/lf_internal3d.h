// Internal declarations of the three-dimensional path (not part of the
// public ABI; include/lagflux.h is).
#pragma once

#include <cuda_runtime.h>

#include "lf_internal.h"

namespace lf {

// Geometry and physics of one 3D mesh.  Planes of nz x ny rows of `pitch`
// elements (x fastest, then y, then z); fields (rho, rho u, rho v, rho w,
// rho E, rho y_k) plane after plane.
struct Mesh3Desc {
  int nx, ny, nz;
  int pitch;          // elements between rows (>= nx, rows start 128-byte aligned)
  long long plane;    // elements between field planes (= pitch * ny * nz)
  int bc, limiter, riemann, nspecies;
  double gamma, beta;
  double rdx, rdy, rdz;
};

// The 2D descriptor whose fields the shared device helpers read (Phys: gamma,
// beta, riemann, 1/dx, 1/dy), and the row view of the mesh used by the
// element-wise kernels (ny * nz rows of nx cells).
__host__ __device__ inline MeshDesc mesh_view(const Mesh3Desc& m, int extra_planes) {
  MeshDesc d{};
  d.nx = m.nx;
  d.ny = m.ny * m.nz;
  d.pitch = m.pitch;
  d.plane = m.plane;
  d.dim = 2;
  d.bc = m.bc;
  d.limiter = m.limiter;
  d.riemann = m.riemann;
  d.gamma = m.gamma;
  d.beta = m.beta;
  d.rdx = m.rdx;
  d.rdy = m.rdy;
  d.vec = 1;
  d.nspecies = extra_planes;
  return d;
}

// One Runge-Kutta stage over a 3D mesh (stages as launch_stage).
cudaError_t launch_stage3d(int stage, const Mesh3Desc& m, const float* Uin, const float* Un, float* out, Scalars* sc,
                           cudaStream_t s);
cudaError_t launch_stage3d(int stage, const Mesh3Desc& m, const double* Uin, const double* Un, double* out,
                           Scalars* sc, cudaStream_t s);
// CFL wave-speed maximum of a freshly set state.
cudaError_t launch_wave_speed3d(const Mesh3Desc& m, const float* U, Scalars* sc, cudaStream_t s);
cudaError_t launch_wave_speed3d(const Mesh3Desc& m, const double* U, Scalars* sc, cudaStream_t s);
// Primitive (rho, u, v, w, p, y_k) <-> conservative; q is dense (5 + nspecies
// planes of nx*ny*nz).
cudaError_t launch_prim_to_cons3d(const Mesh3Desc& m, const float* q, float* U, cudaStream_t s);
cudaError_t launch_prim_to_cons3d(const Mesh3Desc& m, const double* q, double* U, cudaStream_t s);
cudaError_t launch_cons_to_prim3d(const Mesh3Desc& m, const float* U, float* q, cudaStream_t s);
cudaError_t launch_cons_to_prim3d(const Mesh3Desc& m, const double* U, double* q, cudaStream_t s);
// Species planes from dense mass fractions (rho y_k = rho * y_k) and back.
cudaError_t launch_species_to_cons3d(const Mesh3Desc& m, const float* y, float* U, cudaStream_t s);
cudaError_t launch_species_to_cons3d(const Mesh3Desc& m, const double* y, double* U, cudaStream_t s);
cudaError_t launch_cons_to_species3d(const Mesh3Desc& m, const float* U, float* y, cudaStream_t s);
cudaError_t launch_cons_to_species3d(const Mesh3Desc& m, const double* U, double* y, cudaStream_t s);

}  // namespace lf
