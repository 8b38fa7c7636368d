// Direct-stiffness summation Sigma' = Q Q^T (arXiv 2503.02134, Sec. 3.3).
//
// Set-up (setup_kernels.cu) sorts the local copies of every shared global
// node into a segment (CSR: seg_off, perm; ascending global id, ascending
// local index inside a segment).  Here the segments are regrouped into
// buckets of equal length m, 32 segments per warp-sized chunk, and the local
// indices of a chunk are stored transposed (slot[q][lane] = q-th copy of the
// lane's segment), so that a warp reads its index table with coalesced
// 128-byte loads and no lane diverges on the loop count.  A lane sums the m
// copies of its node and writes the sum back to each copy: atomic-free,
// deterministic, and every copy receives the same bits.  Nodes with a single
// copy (element interiors, domain-boundary faces) are never touched.
//
// Accumulation (the paper: the gather-scatter sum must be FP64 for the mixed
// solver to converge, Tables "Mixed-precision strategy evaluation"):
//   FP64 data            -> FP64 sums;
//   mixed (FP32 data)    -> error-free FP32 TwoSum (Knuth), i.e. the exact
//                           sum carried as a float pair and rounded once --
//                           the FP64-then-round result without the narrow
//                           FP64 pipe; FP64 conversion sums on request;
//   all-FP32 variant     -> plain FP32 sums.
#include <algorithm>

#include "gs_sum.cuh"
#include "sem_internal.cuh"

namespace sem {

constexpr int kGsThreads = 256;
constexpr int kGsRegCopies = 8;   // copies kept in registers; longer segments reload indices

template <typename T, int ACC>
__device__ __forceinline__ void gs_chunk_generic(T* __restrict__ v, const int* sl, int m) {
  GsSum<T, ACC> acc;
  for (int q = 0; q < m; ++q) {
    const int i = __ldg(sl + 32 * q);
    if (i >= 0) acc.add(v[i]);
  }
  const T out = acc.result();
  for (int q = 0; q < m; ++q) {
    const int i = __ldg(sl + 32 * q);
    if (i >= 0) v[i] = out;
  }
}

// One warp per chunk of 32 segments: coalesced index loads, value gathers,
// error-free sums, scatter of the sum to every copy.  (Working on several
// chunks at once, or prefetching the next chunk's indices, measured slower:
// the extra registers cost more occupancy than the added loads in flight.)
template <typename T, int ACC>
__global__ void __launch_bounds__(kGsThreads)
    gs_bucket_kernel(T* __restrict__ v, const int2* __restrict__ chunks, int64_t nchunks,
                     const int* __restrict__ slots) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
       c += nwarps) {
    const int2 d = __ldg(chunks + c);
    const int m = d.x;
    const int* sl = slots + d.y + lane;
    if (m > kGsRegCopies) {
      gs_chunk_generic<T, ACC>(v, sl, m);
      continue;
    }
    int id[kGsRegCopies];
#pragma unroll
    for (int q = 0; q < kGsRegCopies; ++q) id[q] = q < m ? __ldg(sl + 32 * q) : -1;
    GsSum<T, ACC> acc;
#pragma unroll
    for (int q = 0; q < kGsRegCopies; ++q)
      if (id[q] >= 0) acc.add(v[id[q]]);
    const T out = acc.result();
#pragma unroll
    for (int q = 0; q < kGsRegCopies; ++q)
      if (id[q] >= 0) v[id[q]] = out;
  }
}

int launch_gs_acc(Handle& h, sem_precision p, void* v, int acc) {
  if (h.n_chunks == 0) return 0;
  const int64_t chunks_per_block = kGsThreads / 32;
  int64_t g = (h.n_chunks + chunks_per_block - 1) / chunks_per_block;
  int64_t cap = (int64_t)h.num_sms * 8;
  const int grid = (int)(g < cap ? g : cap);
  if (p == SEM_FP64) {
    gs_bucket_kernel<double, kGsFP64><<<grid, kGsThreads, 0, h.stream>>>(
        (double*)v, h.gs_chunks, h.n_chunks, h.gs_slots);
  } else if (p == SEM_FP32_ALL || acc == kGsFP32) {
    gs_bucket_kernel<float, kGsFP32><<<grid, kGsThreads, 0, h.stream>>>(
        (float*)v, h.gs_chunks, h.n_chunks, h.gs_slots);
  } else if (acc == kGsFP64) {
    gs_bucket_kernel<float, kGsFP64><<<grid, kGsThreads, 0, h.stream>>>(
        (float*)v, h.gs_chunks, h.n_chunks, h.gs_slots);
  } else {
    gs_bucket_kernel<float, kGsTwoSum><<<grid, kGsThreads, 0, h.stream>>>(
        (float*)v, h.gs_chunks, h.n_chunks, h.gs_slots);
  }
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_gs(Handle& h, sem_precision p, void* v) { return launch_gs_acc(h, p, v, h.gs_acc); }

// ------------------------------------------------------------------ bucket set-up
__global__ void seg_lengths(const int* seg_off, int64_t nseg, int* len, int* hist, int hist_max) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int m = seg_off[s + 1] - seg_off[s];
    len[s] = m;
    atomicAdd(&hist[m < hist_max ? m : hist_max], 1);
  }
}

__global__ void bucket_flags(const int* len, int64_t nseg, int m, uint64_t* flags) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x)
    flags[s] = len[s] == m ? 1ull : 0ull;
}

__global__ void bucket_fill(const int* len, const uint64_t* rank, const int* seg_off,
                            const int* perm, int64_t nseg, int m, int64_t base, int* slots) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (len[s] != m) continue;
    const int64_t r = (int64_t)rank[s];
    const int64_t chunk = r >> 5, lane = r & 31;
    int* dst = slots + base + chunk * 32 * m + lane;
    const int a = seg_off[s];
    for (int q = 0; q < m; ++q) dst[32 * q] = perm[a + q];
  }
}

__global__ void bucket_chunks(int2* chunks, int64_t first, int64_t count, int m, int64_t base) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
       c += (int64_t)gridDim.x * blockDim.x)
    chunks[first + c] = make_int2(m, (int)(base + c * 32 * m));
}

int exclusive_scan_u64(Handle& h, const uint64_t* in, uint64_t* out, int64_t n,
                       uint64_t* grand_total);

int build_gs_buckets(Handle& h) {
  h.n_chunks = 0;
  if (h.n_segments == 0) return 0;
  constexpr int kHistMax = 256;
  const int64_t ns = h.n_segments;
  int* len = nullptr;
  int* hist = nullptr;
  uint64_t* flags = nullptr;
  uint64_t* tot = nullptr;
  SEM_CUDA(cudaMalloc((void**)&len, sizeof(int) * ns));
  SEM_CUDA(cudaMalloc((void**)&hist, sizeof(int) * (kHistMax + 1)));
  SEM_CUDA(cudaMalloc((void**)&flags, sizeof(uint64_t) * ns));
  SEM_CUDA(cudaMalloc((void**)&tot, sizeof(uint64_t)));
  SEM_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * (kHistMax + 1), h.stream));
  const int grid = (int)std::min<int64_t>((ns + 255) / 256, (int64_t)h.num_sms * 16);
  seg_lengths<<<grid, 256, 0, h.stream>>>(h.seg_off, ns, len, hist, kHistMax);
  SEM_CUDA(cudaGetLastError());
  int hist_h[kHistMax + 1];
  SEM_CUDA(cudaMemcpyAsync(hist_h, hist, sizeof(hist_h), cudaMemcpyDeviceToHost, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  int rc = 0;
  if (hist_h[kHistMax] != 0) {
    set_error("sem_setup: a global node is shared by 256 or more local copies");
    rc = SEM_EINVAL;
  }
  int64_t slots_total = 0, chunks_total = 0;
  for (int m = 2; m < kHistMax && !rc; ++m) {
    const int64_t ch = (hist_h[m] + 31) / 32;
    slots_total += ch * 32 * m;
    chunks_total += ch;
  }
  if (!rc) rc = alloc_t(h, &h.gs_slots, (size_t)std::max<int64_t>(slots_total, 1));
  if (!rc) rc = alloc_t(h, &h.gs_chunks, (size_t)std::max<int64_t>(chunks_total, 1));
  if (!rc) {
    SEM_CUDA(cudaMemsetAsync(h.gs_slots, 0xff, sizeof(int) * std::max<int64_t>(slots_total, 1),
                             h.stream));
    int64_t base = 0, first = 0;
    for (int m = 2; m < kHistMax && !rc; ++m) {
      if (hist_h[m] == 0) continue;
      const int64_t ch = (hist_h[m] + 31) / 32;
      bucket_flags<<<grid, 256, 0, h.stream>>>(len, ns, m, flags);
      rc = exclusive_scan_u64(h, flags, flags, ns, tot);
      if (rc) break;
      bucket_fill<<<grid, 256, 0, h.stream>>>(len, flags, h.seg_off, h.perm, ns, m, base,
                                              h.gs_slots);
      bucket_chunks<<<(int)std::min<int64_t>((ch + 255) / 256, 1024), 256, 0, h.stream>>>(
          h.gs_chunks, first, ch, m, base);
      SEM_CUDA(cudaGetLastError());
      base += ch * 32 * m;
      first += ch;
    }
    h.n_chunks = chunks_total;
    h.n_slots = slots_total;
  }
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  cudaFree(len);
  cudaFree(hist);
  cudaFree(flags);
  cudaFree(tot);
  return rc;
}

}  // namespace sem
