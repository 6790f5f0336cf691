// Internal declarations shared by the CUDA translation units of liblagflux.
// Not part of the public ABI (include/lagflux.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lf {

// Device-resident scalars of one time loop.  dt never leaves the device
// during a run; the host reads t and steps only between batches of steps.
struct Scalars {
  double t;                     // current time
  double t_end;                 // final time (<= 0: none)
  double dt;                    // dt of the step in progress (0: no-op step)
  double cfl;                   // CFL number
  unsigned long long smax[2];   // max wave speed, FP64 bits, double-buffered
  long long steps;              // completed steps
  int err;                      // sticky error bits (ERR_*)
  int parity;                   // smax[parity] holds the max of the current state
};

enum : int { ERR_NONPHYSICAL = 1, ERR_BAD_DT = 2 };
enum : int { LIM_MINMOD = 0, LIM_SWEBY = 1, LIM_VANLEER = 2 };
enum : int { BC_TRANSMISSIVE = 0, BC_PERIODIC = 1 };
enum : int { RIEMANN_MAXC = 0, RIEMANN_PER_SIDE = 1 };

// Geometry and physics of one mesh, passed by value to every kernel.
struct MeshDesc {
  int nx, ny;        // cells
  int pitch;         // elements between rows (>= nx)
  long long plane;   // elements between field planes (>= pitch * ny)
  int dim;           // 1 or 2
  int bc;            // BC_*
  int limiter;       // LIM_*
  int riemann;       // RIEMANN_*
  double gamma, beta;
  double rdx, rdy;   // 1 / dx, 1 / dy
  int vec;           // 1: pitch and plane even and every state buffer aligned to
                     // 8 bytes, so two adjacent FP32 cells may be moved as one vector
  int nspecies = 0;  // transported mass fractions: planes 4 .. 3 + nspecies hold rho y_k
  int ty = 0;        // rows per tile of the 2D stage kernels (0: the compiled default)
};

// Rows per tile for a 2D mesh.  A tile pays for its two halo rows below and
// above and for filling its copy pipeline, so tiles are 64 rows unless the
// grid of (strips x tiles) one-warp CTAs is too small for the GPU: halved
// down to 16 rows while there are fewer than 32 CTAs per SM (about two
// resident waves), then down to 4 rows while fewer than 8.  (Fitted to
// GB300 timings of square meshes from 256^2 to 8192^2; lf_autotune times the
// candidates on the actual mesh instead.)  cpl: cells per lane (2 for FP32,
// 1 for FP64); sms <= 0: keep 64.
inline int auto_tile_rows(const MeshDesc& m, int cpl, int sms) {
  const int out_cols = 32 * cpl - 4;
  const long long strips = (m.nx + out_cols - 1) / out_cols;
  auto ctas = [&](int ty) { return strips * ((m.ny + ty - 1) / ty); };
  int ty = 64;
  while (ty > 16 && ctas(ty) < 32LL * sms) ty /= 2;
  while (ty > 4 && ctas(ty) < 8LL * sms) ty /= 2;
  return ty;
}

// Largest nspecies the stage kernels are built for.
constexpr int MAX_SPECIES = 2;

// Batched mode: many independent 2D meshes share one pool per state.  Each
// problem has its own descriptor and its own Scalars (dt, t, wave-speed max).
struct ProbDesc {
  int nx, ny, pitch, pad;
  long long off;    // element offset of the problem's first plane in the pool
  long long plane;  // elements between its planes
  double rdx, rdy;
};
// A unit of work: one warp strip of one problem over rows [j0, jend), with
// a copy of the problem's descriptor, so that a warp starting a unit waits
// for one load of the unit instead of two dependent ones.
struct alignas(16) Unit {
  int p, i0, j0, jend;
  ProbDesc d;
};
struct BatchDesc {
  MeshDesc common;        // bc, limiter, riemann, gamma, beta, vec (per-problem sizes unused)
  const Unit* units;      // device
  int nunits;
  int grid;               // persistent CTAs
};

// Per-stage launch of the fused stage kernel (one Runge-Kutta stage over the
// mesh), out = alpha Un + beta (Uin - dt D(Uin)):
// stage 0: alpha 0, beta 1       (Heun predictor, step 6; first SSP-RK3 stage)
// stage 1: alpha 1/2, beta 1/2   (Heun corrector, step 11), also accumulates
//          the new state's max wave speed for the next dt
// stage 2: alpha 3/4, beta 1/4   (second SSP-RK3 stage)
// stage 3: alpha 1/3, beta 2/3   (third SSP-RK3 stage, with the wave speed)
// `out` may alias `Un` (stage 1 updates in place); Uin must not alias out.
template <typename T>
cudaError_t launch_stage(int stage, const MeshDesc& m, const T* Uin, const T* Un, T* out,
                         Scalars* sc, cudaStream_t s);

// The same for m.nspecies in 1 .. MAX_SPECIES (4 + nspecies planes per state);
// built in their own translation units.
cudaError_t launch_stage_species(int stage, const MeshDesc& m, const float* Uin, const float* Un, float* out,
                                 Scalars* sc, cudaStream_t s);
cudaError_t launch_stage_species(int stage, const MeshDesc& m, const double* Uin, const double* Un, double* out,
                                 Scalars* sc, cudaStream_t s);

template <typename T>
cudaError_t launch_wave_speed(const MeshDesc& m, const T* U, Scalars* sc, cudaStream_t s);

template <typename T>
cudaError_t launch_prim_to_cons(const MeshDesc& m, const T* rho, const T* u, const T* v, const T* p,
                                long long src_plane_stride, T* U, cudaStream_t s);

template <typename T>
cudaError_t launch_cons_to_prim(const MeshDesc& m, const T* U, T* rho, T* u, T* v, T* p, cudaStream_t s);

// Species planes of U from dense mass-fraction planes y (nspecies planes of
// nx*ny): rho y_k = rho * y_k with the density already in U; and back.
template <typename T>
cudaError_t launch_species_to_cons(const MeshDesc& m, const T* y, T* U, cudaStream_t s);
template <typename T>
cudaError_t launch_cons_to_species(const MeshDesc& m, const T* U, T* y, cudaStream_t s);

// Compensated sums of the 4 + m.nspecies conserved fields (partials: blocks x
// fields x 2 doubles; out: 4 + m.nspecies doubles).
template <typename T>
cudaError_t launch_sums(const MeshDesc& m, const T* U, double* partials, int nblocks, double* out,
                        cudaStream_t s);

// One persistent launch per stage over all problems of a batch; counter is
// the stage's work counter (reset by launch_batch_begin).
template <typename T>
cudaError_t launch_batch_stage(int stage, const BatchDesc& b, const T* Uin, const T* Un, T* out, Scalars* sc,
                               int* counter, cudaStream_t s);
// Resident CTAs per SM of the batch stage kernel (for sizing the persistent grid).
template <typename T>
int batch_blocks_per_sm(int stage, int limiter);
cudaError_t launch_batch_begin(Scalars* sc, int nprob, double dt_fixed, int* counters, cudaStream_t s);
cudaError_t launch_batch_end(Scalars* sc, int nprob, cudaStream_t s);

// Discrete adjoint (lf_adjoint.cuh).  Prep: primitives Q (4 dense planes) of
// the state U and the slope tables of x (tabx: (nx+2)*ny slots) and y (taby:
// (ny+2)*nx slots), 12 values per slot.
template <typename T>
cudaError_t launch_adjoint_prep(const MeshDesc& m, const T* U, T* Q, T* tabx, T* taby, cudaStream_t s);
// Face pass: cotangents of the face states of every x-face (dir 0) or y-face
// (dir 1) for the cell cotangent mu.
template <typename T>
cudaError_t launch_face_vjp(const MeshDesc& m, int dir, const T* Q, const T* tab, const T* mu, T* Fq,
                            cudaStream_t s);
// Cell pass: out = alpha X + beta Y + c (dD/dU)^T mu (X, Y nullable).
template <typename T>
cudaError_t launch_cell_vjp(const MeshDesc& m, const T* Q, const T* Fx, const T* Fy, const T* tabx, const T* taby,
                            const T* X, double alpha, const T* Y, double beta, double c, T* out, cudaStream_t s);
// The same two passes recomputing the primitives and slopes from U (FP32).
template <typename T>
cudaError_t launch_face_vjp_direct(const MeshDesc& m, int dir, const T* U, const T* mu, T* Fq, cudaStream_t s);
template <typename T>
cudaError_t launch_cell_vjp_direct(const MeshDesc& m, const T* U, const T* Fx, const T* Fy, const T* X, double alpha,
                                   const T* Y, double beta, double c, T* out, cudaStream_t s);
// Gradient with respect to the primitive initial fields (dense planes).
template <typename T>
cudaError_t launch_grad_prim(const MeshDesc& m, const T* U0, const T* lam, T* gq, cudaStream_t s);

cudaError_t launch_begin_step(Scalars* sc, double dt_fixed, cudaStream_t s);
cudaError_t launch_end_step(Scalars* sc, cudaStream_t s);
cudaError_t launch_reset_scalars(Scalars* sc, double cfl, cudaStream_t s);
cudaError_t launch_set_t_end(Scalars* sc, double t_end, cudaStream_t s);

int sums_blocks();

// Sets the message returned by lf_last_error(NULL) (printf-style).
void set_init_error(const char* fmt, ...);

}  // namespace lf
