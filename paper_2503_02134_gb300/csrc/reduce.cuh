// Dot-product accumulators and deterministic grid reductions.
//
// The paper keeps every global reduction of the CG loop (rtz, pap, rtr and
// the residual norm) in FP64 while the vectors are FP32 (Sec. 3.3; Sec. 4.3,
// "Extended precision for global communication").  On this GPU the FP64
// pipe is narrow, so the per-thread part of an FP32 dot uses the compensated
// Dot2 scheme the paper also evaluates (Ogita, Rump & Oishi 2005: an
// error-free product by FMA plus an error-free TwoSum, carried as a float
// pair), and the pair is promoted to FP64 for the block and grid tree.
// The grid tree is fixed (block partials summed in index order by the last
// block to finish), so results are deterministic run to run.
#pragma once

#include "sem_internal.cuh"

namespace sem {

enum DotMode { kDotFP64 = 0, kDotDot2 = 1, kDotFP32 = 2 };

template <typename T, int DM>
struct DotAcc;

template <>
struct DotAcc<double, kDotFP64> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// FP32 data reduced in FP64: each product of two floats is exact in double.
template <>
struct DotAcc<float, kDotFP64> {
  double s = 0.0;
  __device__ __forceinline__ void add(float a, float b) { s = fma((double)a, (double)b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// Dot2 (Ogita-Rump-Oishi): running sum p with compensation c, both float.
template <>
struct DotAcc<float, kDotDot2> {
  float p = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float h = __fmul_rn(a, b);
    const float r = fmaf(a, b, -h);            // exact error of the product
    const float t = __fadd_rn(p, h);           // TwoSum(p, h) -> (t, q)
    const float z = __fsub_rn(t, p);
    const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));
    p = t;
    c = __fadd_rn(c, __fadd_rn(q, r));
  }
  __device__ __forceinline__ double value() const { return (double)p + (double)c; }
};

template <>
struct DotAcc<float, kDotFP32> {
  float s = 0.f;
  __device__ __forceinline__ void add(float a, float b) { s = fmaf(a, b, s); }
  __device__ __forceinline__ double value() const { return (double)s; }
};

// Block-wide sum of one double per thread (result valid in thread 0).
// `sh` must hold blockDim.x/32 doubles.  FP32 mode rounds every partial to
// float so the all-FP32 variant really reduces in single precision.
template <int DM>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (DM == kDotFP32) {
    float f = (float)v;
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if (lane == 0) sh[wid] = (double)f;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += (float)sh[q];
    __syncthreads();
    return (double)t;
  } else {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    __syncthreads();
    return t;
  }
}

// Publish `nval` block partials and elect the last block to finish.  Returns
// true in every thread of the last block, which may then read all partials.
__device__ __forceinline__ bool publish_and_elect(const double* vals, int nval, double* partials,
                                                  unsigned int* counter) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nval; ++q) partials[(size_t)q * gridDim.x + blockIdx.x] = vals[q];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Sum partials[q*gridDim.x + 0 .. gridDim.x) in a fixed order (all threads
// of the last block take part; result in thread 0).
template <int DM>
__device__ __forceinline__ double reduce_partials(const double* partials, int q, double* sh) {
  if (DM == kDotFP32) {
    float s = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s += (float)__ldcg(partials + (size_t)q * gridDim.x + b);
    return block_sum<DM>((double)s, sh);
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    s += __ldcg(partials + (size_t)q * gridDim.x + b);
  return block_sum<DM>(s, sh);
}

}  // namespace sem
