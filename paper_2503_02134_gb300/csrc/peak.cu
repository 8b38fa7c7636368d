// sem_fma_peak: the FMA throughput of the CUDA cores, measured.  The FP64
// operator is bound by the FP64 FMA pipe, not by memory, so its roofline is
// a fraction of this rate; the FP32 figure bounds the CUDA-core contractions
// at high order.  Every thread runs kChains independent FMA chains
// (a <- a * m + b) with register operands, enough to cover the pipe's
// latency with the 64 resident warps per SM; flops = 2 * chains *
// iterations * threads.  The result feeds a sink that a comparison nothing
// satisfies guards, so the chains stay live.
#include "sem_internal.cuh"

namespace sem {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

static __device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, T m0, T b0) {
  // the coefficients in registers (a value the compiler cannot fold), so
  // every FMA is register-only
  const T m = m0 + (T)threadIdx.x * (T)1e-30, b = b0 + (T)blockIdx.x * (T)1e-30;
  T a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = fma(a[c], m, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += a[c];
  if (s == (T)-12345.0) g_peak_sink = (double)s;
}

template <typename T>
static int run_peak(int iters, double* tflops) {
  int dev = 0, sms = 0;
  SEM_CUDA(cudaGetDevice(&dev));
  SEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * kPeakBlocksPerSm;
  const T m = (T)0.999999, b = (T)1e-6;
  ScopedEvents ev;
  SEM_CUDA(ev.create());
  fma_peak_kernel<T><<<grid, kPeakThreads>>>(iters / 8 > 4 ? iters / 8 : 4, m, b);   // warm-up
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaEventRecord(ev.a, 0));
  fma_peak_kernel<T><<<grid, kPeakThreads>>>(iters, m, b);
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaEventRecord(ev.b, 0));
  SEM_CUDA(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  SEM_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
  const double flops = 2.0 * kPeakChains * (double)((iters + 3) / 4 * 4) * grid * kPeakThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" int sem_fma_peak(int fp64, int iters, double* tflops) {
  if (!tflops || iters < 4) {
    set_error("sem_fma_peak: null result or fewer than 4 iterations");
    return SEM_EINVAL;
  }
  return fp64 ? run_peak<double>(iters, tflops) : run_peak<float>(iters, tflops);
}
