// Direct-stiffness summation Sigma' = Q Q^T (arXiv 2503.02134, Sec. 3.3).
//
// The set-up builds a map of the global nodes that have more than one local
// copy: seg_off (CSR offsets, one segment per such node, in ascending
// global id) and perm (the local indices of the copies, ascending inside a
// segment).  Nodes with a single copy (element interiors, domain-boundary
// faces) are left untouched.  The kernel is atomic-free: one thread owns a
// segment, sums its copies in the accumulation type (FP64 for the FP64 and
// mixed paths -- the paper's finding that the gather-scatter sum must be
// FP64 for convergence, Tables "Mixed-precision strategy evaluation" -- and
// FP32 only for the all-FP32 variant), and writes the rounded sum back to
// every copy, so all copies stay bit-identical.
#include "sem_internal.cuh"

namespace sem {

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) gs_segments_kernel(T* __restrict__ v,
                                                          const int* __restrict__ seg_off,
                                                          const int* __restrict__ perm,
                                                          int64_t nseg) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int a = __ldg(seg_off + s), b = __ldg(seg_off + s + 1);
    Acc sum = Acc(0);
    for (int q = a; q < b; ++q) sum += (Acc)v[__ldg(perm + q)];
    const T out = (T)sum;
    for (int q = a; q < b; ++q) v[__ldg(perm + q)] = out;
  }
}

int launch_gs(Handle& h, sem_precision p, void* v) {
  if (h.n_segments == 0) return 0;
  int threads = 256;
  int64_t g = (h.n_segments + threads - 1) / threads;
  int64_t cap = (int64_t)h.num_sms * 32;
  int grid = (int)(g < cap ? g : cap);
  if (p == SEM_FP64) {
    gs_segments_kernel<double, double><<<grid, threads, 0, h.stream>>>(
        (double*)v, h.seg_off, h.perm, h.n_segments);
  } else if (p == SEM_FP32_ALL) {
    gs_segments_kernel<float, float><<<grid, threads, 0, h.stream>>>((float*)v, h.seg_off, h.perm,
                                                                      h.n_segments);
  } else {
    gs_segments_kernel<float, double><<<grid, threads, 0, h.stream>>>((float*)v, h.seg_off, h.perm,
                                                                       h.n_segments);
  }
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace sem
