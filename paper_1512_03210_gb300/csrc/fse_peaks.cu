// fse_peaks.cu -- arithmetic-throughput probes for the roofline of the split
// step (built as its own library, libfse_peaks.so; not part of the solver).
//
// The FP64 path of the split step runs the same passes as the FP32 path in
// double arithmetic, and GB300 issues double-precision fma at a small fraction
// of the float rate, so that path is bounded by DFMA throughput rather than by
// HBM. The float passes are bounded by instruction issue. These kernels measure
// the two ceilings on the device itself: long chains of independent fma on
// registers (8 chains per thread, so that the pipe never waits on a result),
// timed with CUDA events by the caller's stream. Each fma counts 2 flops; a
// packed float2 fma counts 4.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;  // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(float* out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x - c) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 12345.678f) out[0] = s;
}

}  // namespace

extern "C" {

// Runs `kind` (0: DFMA, 1: FFMA, 2: packed FFMA2) over blocks x 256 threads,
// iters x 8 fma per thread, on the given stream, bracketed by two events;
// writes the elapsed milliseconds and the flops executed. `scratch` is a
// device buffer of at least 8 bytes (never written for these inputs).
// Returns 0 on success, else the CUDA error code.
int fse_peak_run(int kind, int blocks, int iters, void* scratch, void* stream, double* ms, double* flops) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    if (kind == 0) k_dfma<<<blocks, 256, 0, st>>>(static_cast<double*>(scratch), iters, 0.999999, 1e-7);
    else if (kind == 1) k_ffma<<<blocks, 256, 0, st>>>(static_cast<float*>(scratch), iters, 0.999f, 1e-4f);
    else k_ffma2<<<blocks, 256, 0, st>>>(static_cast<float*>(scratch), iters, 0.999f, 1e-4f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *ms = t;
  *flops = (double)blocks * 256.0 * iters * kChains * (kind == 2 ? 4.0 : 2.0);
  return (int)e;
}

}  // extern "C"
