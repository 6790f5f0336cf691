// Arithmetic peaks of the GPU this library runs on, measured rather than
// derived from data-sheet rates: the denominators of the ALU rooflines that
// the benchmark reports for the FP64 step (bound by the FP64 pipe) and, for
// context, the FP32 step.  The paper has no counterpart (its roofline is for
// multicore CPUs); this is a measurement helper of the library.
//
// Each thread runs eight independent fused multiply-add chains
// a <- a * b + c (|b| < 1, so every chain converges to c / (1 - b) and never
// overflows or goes subnormal), enough independent work per warp to keep the
// FMA pipes busy at full occupancy.  The chains' sum is stored only if it
// equals a value it cannot reach, which the compiler cannot prove, so no
// chain is removed.  Flops per launch = 2 (multiply and add) x 8 chains x
// iterations x threads, x 2 for the paired FP32 form (two lanes per
// instruction).
#include <cuda_runtime.h>

#include "../../include/lagflux.h"
#include "lf_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(T* sink, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1)) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) ffma2_chains_kernel(float* sink, int iters, float b, float c) {
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x + 2 * k) * 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.f) sink[blockIdx.x] = s;
}

cudaError_t launch(int kind, int blocks, int iters, void* sink, cudaStream_t s) {
  if (kind == LF_PEAK_FP64)
    fma_chains_kernel<double><<<blocks, kThreads, 0, s>>>(static_cast<double*>(sink), iters, 0.999999, 1e-3);
  else if (kind == LF_PEAK_FP32)
    fma_chains_kernel<float><<<blocks, kThreads, 0, s>>>(static_cast<float*>(sink), iters, 0.999f, 1e-3f);
  else
    ffma2_chains_kernel<<<blocks, kThreads, 0, s>>>(static_cast<float*>(sink), iters, 0.999f, 1e-3f);
  return cudaGetLastError();
}

}  // namespace

extern "C" lf_status lf_measure_peak(int32_t device, int32_t kind, double target_ms, double* tflops) {
  if (!tflops || (kind != LF_PEAK_FP64 && kind != LF_PEAK_FP32 && kind != LF_PEAK_FP32_PAIRED) ||
      !(target_ms > 0.0 && target_ms <= 1000.0)) {
    lf::set_init_error("lf_measure_peak: bad kind, target_ms (0, 1000] or NULL result");
    return LF_ERR_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    lf::set_init_error("lf_measure_peak: cannot select device %d", device);
    return LF_ERR_CUDA;
  }
  lf_status st = LF_OK;
  int sms = 0;
  void* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * kBlocksPerSM;
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double lanes = kind == LF_PEAK_FP32_PAIRED ? 2.0 : 1.0;
  double best = 0.0;
  int iters = 256;
  // calibrate the iteration count to about target_ms per launch, then keep the best of three
  for (int rep = 0; e == cudaSuccess && rep < 5; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch(kind, blocks, iters, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const double flops = 2.0 * kChains * lanes * (double)iters * blocks * kThreads;
    if (rep >= 2 && ms > 0.f) {
      const double tf = flops / (ms * 1e-3) / 1e12;
      if (tf > best) best = tf;
    } else if (ms > 0.f) {
      const double scale = target_ms / ms;
      const double next = iters * (scale > 64.0 ? 64.0 : scale);
      iters = next < 1.0 ? 1 : (next > 2e9 ? 2000000000 : (int)next);
    }
  }
  if (e != cudaSuccess) {
    lf::set_init_error("lf_measure_peak: %s", cudaGetErrorString(e));
    st = LF_ERR_CUDA;
  } else {
    *tflops = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
