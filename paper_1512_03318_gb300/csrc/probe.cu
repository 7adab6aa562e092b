// Measured issue rates of the CUDA-core pipes that bound the float-float and FP64 kernels
// (mrd_measure_peaks): a grid of independent fused multiply-add chains per pipe, timed with
// CUDA events on the context stream. Roofline fractions of those kernels are quoted against
// these rates rather than against unit counts and a nominal clock.
#include <chrono>

#include "heff_internal.h"

namespace {

constexpr int kChains = 8;      // independent accumulators per thread (hide the pipe latency)
constexpr int kIters = 4096;    // multiply-adds per chain

template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;   // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

template <class T>
int fma_rate(mrd_ctx* ctx, int n_sm, double* instr_per_s) {
  cudaStream_t s = ctx->stream;
  T* out = nullptr;
  const int blocks = n_sm * 8;
  MRD_CUDA(ctx, mrd::cache_alloc((void**)&out, sizeof(T) * blocks, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 6 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    k_fma_rate<T><<<blocks, 256, 0, s>>>(out, (T)0.999999, (T)1e-7);
    mrd::count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;   // the first run warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  mrd::cache_free(out, s);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_measure_peaks");
  *instr_per_s = (double)blocks * 256.0 * kChains * kIters / (best * 1e-3);
  return MRD_OK;
}

}  // namespace

extern "C" int mrd_measure_peaks(mrd_ctx* ctx, double* out4) try {
  if (!ctx || !out4) return MRD_E_ARG;
  Guard g(ctx->device);
  int n_sm = 0;
  MRD_CUDA(ctx, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device);
  double f32 = 0.0, f64 = 0.0;
  int rc = fma_rate<float>(ctx, n_sm, &f32);
  if (rc == MRD_OK) rc = fma_rate<double>(ctx, n_sm, &f64);
  if (rc != MRD_OK) return rc;
  out4[0] = f32;                  // FP32 FMA instructions per second (one per lane)
  out4[1] = f64;                  // FP64 FMA instructions per second
  out4[2] = (double)n_sm;
  out4[3] = (double)clk_khz * 1e3;   // the device's reported maximum SM clock (Hz)
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}
