// sem_glsc3_noalloc: the weighted dot product sum_i a_i c_i b_i without any
// device allocation, for callers that cannot call cudaMalloc (code running
// where the allocator is unavailable or forbidden, e.g. inside another
// library's allocation-free hot path or a memory-capped sandbox).  The
// per-block partial sums live in a file-scope __device__ array instead of
// handle-owned memory.
#include <mutex>

#include "reduce.cuh"

namespace sem {

// Scratch shared by every call on a device: one partial sum per tile plus the
// last-block election counter.  Held by every GPU that loads the library
// until the process exits.
constexpr int kNoAllocTileThreads = 256;
constexpr int kNoAllocTileItems = 32;
constexpr int64_t kNoAllocTile = (int64_t)kNoAllocTileThreads * kNoAllocTileItems;  // 8192 values
constexpr int kNoAllocMaxTiles = 4096;                                             // 32 KiB of partials
constexpr int64_t kNoAllocMaxN = kNoAllocMaxTiles * kNoAllocTile;                  // 33,554,432 values

struct NoAllocScratch {
  double partials[kNoAllocMaxTiles];
  unsigned int counter;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(kNoAllocTileThreads)
    glsc3_noalloc_kernel(const double* __restrict__ a, const double* __restrict__ b,
                         const double* __restrict__ c, int64_t n, NoAllocScratch* scratch,
                         double* __restrict__ out) {
  __shared__ double sh[kNoAllocTileThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kNoAllocTile;
  double s = 0.0;
  for (int q = 0; q < kNoAllocTileItems; ++q) {
    const int64_t i = base + (int64_t)q * kNoAllocTileThreads + threadIdx.x;
    if (i < n) s = fma(c[i] * a[i], b[i], s);
  }
  const double part = block_sum<kDotFP64>(s, sh);
  const double vals[1] = {part};
  if (publish_and_elect(vals, 1, scratch->partials, &scratch->counter)) {
    const double t = reduce_partials<kDotFP64>(scratch->partials, 0, sh);
    if (threadIdx.x == 0) {
      *out = t;
      scratch->counter = 0u;
    }
  }
}

// Device address of the scratch array, looked up once per device and kept
// for the life of the process (valid for the context current at the lookup:
// a cudaDeviceReset afterwards invalidates it, which the header states).
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {};

static int noalloc_scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("sem_glsc3_noalloc: device index out of range");
    return SEM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    SEM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<NoAllocScratch*>(g_noalloc_ptr[dev]);
  return 0;
}

}  // namespace sem

using namespace sem;

extern "C" int sem_glsc3_noalloc(const double* a, const double* b, const double* c, int64_t n,
                                 double* result, void* stream) {
  if (!a || !b || !c || !result || n < 0) {
    set_error("sem_glsc3_noalloc: null pointer or negative length");
    return SEM_EINVAL;
  }
  if (n > kNoAllocMaxN) {
    set_error("sem_glsc3_noalloc: n exceeds the static scratch capacity of 33554432 values");
    return SEM_EINVAL;
  }
  NoAllocScratch* scratch = nullptr;
  int rc = noalloc_scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // the election counter must start at zero whatever the previous call left
  SEM_CUDA(cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), st));
  if (n == 0) {
    SEM_CUDA(cudaMemsetAsync(result, 0, sizeof(double), st));
    return SEM_OK;
  }
  const int tiles = (int)((n + kNoAllocTile - 1) / kNoAllocTile);
  glsc3_noalloc_kernel<<<tiles, kNoAllocTileThreads, 0, st>>>(a, b, c, n, scratch, result);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}
