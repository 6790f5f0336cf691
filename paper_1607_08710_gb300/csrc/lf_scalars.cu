// Single-thread kernels that keep the time loop's scalars on the device, so
// that a run needs no host round trip per step (Sec. 4, Heun step 1: the
// CFL time step), and the final pass of the deterministic conservation sums.
#include "lf_aux.cuh"
#include "lf_internal.h"

namespace lf {

// dt for the step about to run: CFL / (max wave speed of the current state)
// or dt_fixed > 0, clipped to t_end - t; 0 once t_end is reached or after a
// device error (the stage kernels then return at once).  Also clears the
// wave-speed slot the coming corrector will fill.
__device__ __forceinline__ void begin_step_one(Scalars* sc, double dt_fixed) {
  double dt = 0.0;
  if (sc->err == 0) {
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      const double s = __longlong_as_double((long long)sc->smax[sc->parity]);
      dt = sc->cfl / s;
      if (!(dt > 0.0) || !isfinite(dt)) {
        sc->err |= ERR_BAD_DT;
        dt = 0.0;
      }
    }
    if (dt > 0.0 && sc->t_end > 0.0) {
      const double rem = sc->t_end - sc->t;
      dt = rem <= 0.0 ? 0.0 : fmin(dt, rem);
    }
  }
  sc->dt = dt;
  sc->smax[sc->parity ^ 1] = 0ull;
}

__device__ __forceinline__ void end_step_one(Scalars* sc) {
  if (sc->dt > 0.0) {
    sc->t += sc->dt;
    sc->steps += 1;
    sc->parity ^= 1;
  }
}

__global__ void begin_step_kernel(Scalars* sc, double dt_fixed) { begin_step_one(sc, dt_fixed); }
__global__ void end_step_kernel(Scalars* sc) { end_step_one(sc); }

// Batched mode: one thread per problem; thread 0 also resets the two stage
// work counters of the coming step.
__global__ void batch_begin_kernel(Scalars* sc, int n, double dt_fixed, int* counters) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    counters[0] = 0;
    counters[1] = 0;
  }
  if (p < n) begin_step_one(sc + p, dt_fixed);
}

__global__ void batch_end_kernel(Scalars* sc, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) end_step_one(sc + p);
}

__global__ void reset_scalars_kernel(Scalars* sc, double cfl) {
  sc->t = 0.0;
  sc->t_end = 0.0;
  sc->dt = 0.0;
  sc->cfl = cfl;
  sc->smax[0] = 0ull;
  sc->smax[1] = 0ull;
  sc->steps = 0;
  sc->err = 0;
  sc->parity = 0;
}

__global__ void set_t_end_kernel(Scalars* sc, double t_end) { sc->t_end = t_end; }

__global__ void sums_final_kernel(const double* partials, int nblocks, int nfields, double* out) {
  if (threadIdx.x < nfields) {
    const int l = threadIdx.x;
    KahanNeumaier tot;
    for (int b = 0; b < nblocks; ++b) {
      tot.add(partials[(l * nblocks + b) * 2]);
      tot.add(partials[(l * nblocks + b) * 2 + 1]);
    }
    out[l] = tot.s + tot.c;
  }
}

cudaError_t launch_begin_step(Scalars* sc, double dt_fixed, cudaStream_t s) {
  begin_step_kernel<<<1, 1, 0, s>>>(sc, dt_fixed);
  return cudaGetLastError();
}
cudaError_t launch_end_step(Scalars* sc, cudaStream_t s) {
  end_step_kernel<<<1, 1, 0, s>>>(sc);
  return cudaGetLastError();
}
cudaError_t launch_batch_begin(Scalars* sc, int nprob, double dt_fixed, int* counters, cudaStream_t s) {
  batch_begin_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(sc, nprob, dt_fixed, counters);
  return cudaGetLastError();
}
cudaError_t launch_batch_end(Scalars* sc, int nprob, cudaStream_t s) {
  batch_end_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(sc, nprob);
  return cudaGetLastError();
}
cudaError_t launch_reset_scalars(Scalars* sc, double cfl, cudaStream_t s) {
  reset_scalars_kernel<<<1, 1, 0, s>>>(sc, cfl);
  return cudaGetLastError();
}
cudaError_t launch_set_t_end(Scalars* sc, double t_end, cudaStream_t s) {
  set_t_end_kernel<<<1, 1, 0, s>>>(sc, t_end);
  return cudaGetLastError();
}

int sums_blocks() { return SUMS_BLOCKS; }

}  // namespace lf
