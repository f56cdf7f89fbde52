// Arithmetic-rate probe of the GPU (sb_measure_rates): the ceilings that bound the
// solver's kernels, measured rather than taken from a data sheet.
//
// Each rate kernel runs kChains independent dependency chains per thread, so the
// pipe (not the latency of one chain) is the limit, on a persistent grid of
// kWarpsPerSM warps per SM; the operands are launch arguments, and every chain's
// result is stored, so nothing folds away.  The time of the middle launch of three
// (after a warm-up) is taken with CUDA events.
//   FP64 FMA: fma(x, a, b) in double (2 flop each).
//   FP32 FMA: the same in float.
//   FP64 <-> FP32 conversion: x = (double)(float)(x) pairs (two conversions each),
//   the operation a mixed-precision kernel spends on rounding and widening.
#include <algorithm>
#include <cuda_runtime.h>

#include "sb_internal.h"

namespace sb {
namespace {

constexpr int kChains = 8;
constexpr int kWarpsPerSM = 32;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) cvt_rate_kernel(double* out, int iters, double a) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = a + threadIdx.x + k;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)__double2float_rn(x[k]);
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Seconds of the middle of three timed launches of `launch` (after one warm-up).
template <typename F>
int time_launch(F launch, double* seconds) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SB_CUDA(cudaEventCreate(&e0));
  int rc = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  float ms[3] = {0.f, 0.f, 0.f};
  if (rc == SB_OK) {
    launch();
    rc = cuda_check(cudaGetLastError(), "rate kernel launch");
    for (int r = 0; r < 3 && rc == SB_OK; ++r) {
      rc = cuda_check(cudaEventRecord(e0), "cudaEventRecord");
      if (rc == SB_OK) launch();
      if (rc == SB_OK) rc = cuda_check(cudaGetLastError(), "rate kernel launch");
      if (rc == SB_OK) rc = cuda_check(cudaEventRecord(e1), "cudaEventRecord");
      if (rc == SB_OK) rc = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
      if (rc == SB_OK) rc = cuda_check(cudaEventElapsedTime(&ms[r], e0, e1), "cudaEventElapsedTime");
    }
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  SB_TRY(rc);
  std::sort(ms, ms + 3);
  *seconds = ms[1] * 1e-3;
  return SB_OK;
}

}  // namespace
}  // namespace sb

using namespace sb;

extern "C" int sb_measure_rates(int device, sb_rates* out) {
  clear_error();
  if (!out) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(device);
  SB_TRY(g.rc);
  const int sms = sm_count(device);
  const int grid = sms * kWarpsPerSM * 32 / kThreads;
  const double threads = (double)grid * kThreads;
  void* buf = nullptr;
  SB_CUDA(cudaMalloc(&buf, (size_t)grid * kThreads * sizeof(double)));
  double* d = static_cast<double*>(buf);
  const int it64 = 4096, it32 = 32768, itc = 4096;
  double t64 = 0, t32 = 0, tc = 0;
  int rc = time_launch([&] { fma_rate_kernel<double><<<grid, kThreads>>>(d, it64, 0.999999, 1e-7); }, &t64);
  if (rc == SB_OK)
    rc = time_launch(
        [&] { fma_rate_kernel<float><<<grid, kThreads>>>(reinterpret_cast<float*>(d), it32, 0.9999f, 1e-5f); },
        &t32);
  if (rc == SB_OK) rc = time_launch([&] { cvt_rate_kernel<<<grid, kThreads>>>(d, itc, 0.25); }, &tc);
  cudaFree(buf);
  SB_TRY(rc);
  out->fp64_fma_per_s = threads * kChains * it64 / t64;
  out->fp32_fma_per_s = threads * kChains * it32 / t32;
  out->f64_f32_conversions_per_s = 2.0 * threads * kChains * itc / tc;
  out->sm_count = sms;
  return SB_OK;
}
