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
  int tz = 0;         // planes per z-tile of the 3D stage kernels (0: the compiled default)
};

// Planes per z-tile for a 3D mesh: 64, halved down to 8 while the grid of
// (strips x row blocks x z-tiles) CTAs of rows_per_cta warps gives fewer
// than 6 CTAs per SM (two waves of the three resident CTAs).  cpl: cells per
// lane; sms <= 0: keep 64.
inline int auto_tile_planes(const Mesh3Desc& m, int cpl, int rows_per_cta, int sms) {
  const int out_cols = 32 * cpl - 4;
  const long long cols = (long long)((m.nx + out_cols - 1) / out_cols) * ((m.ny + rows_per_cta - 1) / rows_per_cta);
  int tz = 64;
  while (tz > 8 && cols * ((m.nz + tz - 1) / tz) < 6LL * sms) tz /= 2;
  return tz;
}

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
// Warps (= rows) per CTA of the 3D stage kernels.
int stage3d_rows_per_cta();

}  // namespace lf
