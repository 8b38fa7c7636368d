// Set-up kernels: GLL rule and derivative matrix, box numbering, geometric
// factors, gather-scatter segment map, Jacobi diagonal and right-hand sides.
// Everything here runs once per handle, in FP64 (the paper keeps the
// initialisation in double precision and casts once to FP32, Sec. 4.3).
#include <math.h>

#include <vector>

#include "sem_internal.cuh"

namespace sem {

// ------------------------------------------------------------------ GLL rule
// P_N(x) by the three-term recurrence (k+1)P_{k+1} = (2k+1) x P_k - k P_{k-1}.
__host__ __device__ inline double legendre_p(int N, double x) {
  double p0 = 1.0, p1 = x;
  if (N == 0) return p0;
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Number of eigenvalues below x of the symmetric tridiagonal Jacobi matrix of
// the Jacobi polynomial P^{(1,1)}_m (zero diagonal, off-diagonal entries
// sqrt(k(k+2)/((2k+1)(2k+3))), k = 1..m-1), by Sturm's sequence of pivots.
// The zeros of P^{(1,1)}_{N-1} are the zeros of P_N', i.e. the interior GLL
// nodes, so bisection on this count locates them (Golub-Welsch matrix).
__host__ __device__ inline int sturm_count_jacobi11(int m, double x) {
  int count = 0;
  double q = -x;
  if (q < 0.0) ++count;
  for (int k = 1; k < m; ++k) {
    double b2 = (double)k * (k + 2) / ((2.0 * k + 1.0) * (2.0 * k + 3.0));
    if (q == 0.0) q = 1e-300;
    q = -x - b2 / q;
    if (q < 0.0) ++count;
  }
  return count;
}

__host__ __device__ inline double gll_node(int N, int t) {
  if (t == 0) return -1.0;
  if (t == N) return 1.0;
  double lo = -1.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count_jacobi11(N - 1, mid) > t - 1)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

__global__ void gll_kernel(int N, double* xi, double* wq, double* D64, float* D32) {
  const int n = N + 1;
  __shared__ double sx[kMaxn], sp[kMaxn];
  int t = threadIdx.x;
  if (t < n) {
    double x = gll_node(N, t);
    // symmetric rule: average the two mirrored bisections
    double xm = -gll_node(N, N - t);
    if (t != 0 && t != N) x = 0.5 * (x + xm);
    if (2 * t == N) x = 0.0;
    sx[t] = x;
    sp[t] = legendre_p(N, x);
    xi[t] = x;
    wq[t] = 2.0 / ((double)N * (N + 1) * sp[t] * sp[t]);
  }
  __syncthreads();
  for (int q = t; q < n * n; q += blockDim.x) {
    int i = q / n, j = q % n;
    double d;
    if (i != j)
      d = sp[i] / (sp[j] * (sx[i] - sx[j]));
    else if (i == 0)
      d = -0.25 * N * (N + 1);
    else if (i == N)
      d = 0.25 * N * (N + 1);
    else
      d = 0.0;
    D64[q] = d;
    D32[q] = (float)d;
  }
}

int launch_gll(Handle& h) {
  gll_kernel<<<1, 32, 0, h.stream>>>(h.N, h.xi, h.wq, h.D64, h.D32);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ numbering
__global__ void box_numbering_kernel(int N, int kx, int ky, int kz, int64_t L, int* gid,
                                     uint8_t* faces, double* mask) {
  const int n = N + 1, n3 = n * n * n;
  const int64_t gx = (int64_t)kx * N + 1, gy = (int64_t)ky * N + 1;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = l / n3;
    int rem = (int)(l - e * n3);
    int i = rem % n, j = (rem / n) % n, k = rem / (n * n);
    int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
    int64_t I = (int64_t)ex * N + i, J = (int64_t)ey * N + j, K = (int64_t)ez * N + k;
    gid[l] = (int)(I + gx * (J + gy * K));
    uint8_t f = (ex == 0 ? 1 : 0) | (ex == kx - 1 ? 2 : 0) | (ey == 0 ? 4 : 0) |
                (ey == ky - 1 ? 8 : 0) | (ez == 0 ? 16 : 0) | (ez == kz - 1 ? 32 : 0);
    if (rem == 0) faces[e] = f;
    bool on = (i == 0 && (f & 1)) || (i == N && (f & 2)) || (j == 0 && (f & 4)) ||
              (j == N && (f & 8)) || (k == 0 && (f & 16)) || (k == N && (f & 32));
    mask[l] = on ? 0.0 : 1.0;
  }
}

__global__ void mask_from_faces_kernel(int N, int64_t L, const uint8_t* faces, double* mask) {
  const int n = N + 1, n3 = n * n * n;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = l / n3;
    int rem = (int)(l - e * n3);
    int i = rem % n, j = (rem / n) % n, k = rem / (n * n);
    uint8_t f = faces[e];
    bool on = (i == 0 && (f & 1)) || (i == N && (f & 2)) || (j == 0 && (f & 4)) ||
              (j == N && (f & 8)) || (k == 0 && (f & 16)) || (k == N && (f & 32));
    mask[l] = on ? 0.0 : 1.0;
  }
}

static int grid_for(const Handle& h, int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)h.num_sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int launch_box_connectivity(Handle& h) {
  h.U = ((int64_t)h.kx * h.N + 1) * ((int64_t)h.ky * h.N + 1) * ((int64_t)h.kz * h.N + 1);
  box_numbering_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(
      h.N, h.kx, h.ky, h.kz, h.L, h.gid, h.bfaces, h.mask64);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_user_connectivity(Handle& h, const int64_t* gid_host, const uint8_t* faces_host) {
  // Validate and narrow the ids on the host (they arrive in host memory).
  std::vector<int> g32((size_t)h.L);
  int64_t gmax = -1;
  for (int64_t l = 0; l < h.L; ++l) {
    int64_t g = gid_host[l];
    if (g < 0 || g >= (int64_t)1 << 31) {
      set_error("sem_setup: gid out of [0, 2^31)");
      return SEM_EINVAL;
    }
    if (g > gmax) gmax = g;
    g32[(size_t)l] = (int)g;
  }
  if (gmax + 1 > 8 * h.L + 8) {
    set_error("sem_setup: gid values must be dense (max gid + 1 <= 8 L)");
    return SEM_EINVAL;
  }
  h.U = gmax + 1;
  SEM_CUDA(cudaMemcpyAsync(h.gid, g32.data(), sizeof(int) * h.L, cudaMemcpyHostToDevice, h.stream));
  if (faces_host) {
    SEM_CUDA(cudaMemcpyAsync(h.bfaces, faces_host, (size_t)h.E, cudaMemcpyHostToDevice, h.stream));
  } else {
    SEM_CUDA(cudaMemsetAsync(h.bfaces, 0, (size_t)h.E, h.stream));
  }
  mask_from_faces_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.N, h.L, h.bfaces, h.mask64);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  // the host vector must outlive the copy
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  return 0;
}

// ------------------------------------------------------------------ geometry
// One block per element.  Coordinates of the element's nodes go to shared
// memory, the Jacobian J_{m a} = dx_m/dr_a comes from applying D along each
// reference direction, and G_ab = w_i w_j w_k det(J) sum_m (dr_a/dx_m)(dr_b/dx_m).
__global__ void geometry_kernel(int N, int kx, int ky, int kz, double lo0, double lo1, double lo2,
                                double h0, double h1, double h2, double amp, int deform,
                                const double* __restrict__ user_coords, const double* __restrict__ xi,
                                const double* __restrict__ wq, const double* __restrict__ D, int64_t E,
                                double* coords, double* G64, float* G32, double* B, double* detJ,
                                int* bad) {
  extern __shared__ double sm[];
  const int n = N + 1, n3 = n * n * n;
  const int64_t L = E * n3;
  double* sx = sm;           // 3 * n3
  double* sD = sm + 3 * n3;  // n * n
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) sD[q] = D[q];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      int i = q % n, j = (q / n) % n, k = q / (n * n);
      double X, Y, Z;
      if (user_coords) {
        X = user_coords[e * n3 + q];
        Y = user_coords[L + e * n3 + q];
        Z = user_coords[2 * L + e * n3 + q];
      } else {
        X = lo0 + (ex + 0.5 * (1.0 + xi[i])) * h0;
        Y = lo1 + (ey + 0.5 * (1.0 + xi[j])) * h1;
        Z = lo2 + (ez + 0.5 * (1.0 + xi[k])) * h2;
        if (deform == 1) {
          const double tp = 2.0 * M_PI;
          double sx_ = sin(tp * X), sy_ = sin(tp * Y), sz_ = sin(tp * Z);
          double Xn = X + amp * sy_ * sz_;
          double Yn = Y + amp * sz_ * sx_;
          double Zn = Z + amp * sx_ * sy_;
          X = Xn;
          Y = Yn;
          Z = Zn;
        }
      }
      sx[q] = X;
      sx[n3 + q] = Y;
      sx[2 * n3 + q] = Z;
      coords[e * n3 + q] = X;
      coords[L + e * n3 + q] = Y;
      coords[2 * L + e * n3 + q] = Z;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      int i = q % n, j = (q / n) % n, k = q / (n * n);
      double J[3][3];
      for (int m = 0; m < 3; ++m) {
        const double* c = sx + m * n3;
        double dr = 0.0, ds = 0.0, dt = 0.0;
        for (int l = 0; l < n; ++l) {
          dr += sD[i * n + l] * c[l + n * j + n * n * k];
          ds += sD[j * n + l] * c[i + n * l + n * n * k];
          dt += sD[k * n + l] * c[i + n * j + n * n * l];
        }
        J[m][0] = dr;
        J[m][1] = ds;
        J[m][2] = dt;
      }
      // inverse via the adjugate: Jinv[a][m] = dr_a/dx_m
      double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      if (!(det > 0.0)) atomicExch(bad, 1);
      double inv = 1.0 / det;
      double Ji[3][3];
      Ji[0][0] = c00 * inv;
      Ji[1][0] = c01 * inv;
      Ji[2][0] = c02 * inv;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
      double bq = wq[i] * wq[j] * wq[k] * det;
      const int pa[6] = {0, 1, 2, 0, 0, 1};
      const int pb[6] = {0, 1, 2, 1, 2, 2};
      for (int a = 0; a < 6; ++a) {
        double g = 0.0;
        for (int m = 0; m < 3; ++m) g += Ji[pa[a]][m] * Ji[pb[a]][m];
        g *= bq;
        int64_t off = (e * 6 + a) * n3 + q;
        G64[off] = g;
        G32[off] = (float)g;
      }
      B[e * n3 + q] = bq;
      detJ[e * n3 + q] = det;
    }
    __syncthreads();
  }
}

int launch_geometry(Handle& h, const double* user_coords_dev, double amp, int deform_kind,
                    const double lo[3], const double hi[3]) {
  const int n = h.n, n3 = n * n * n;
  size_t smem = sizeof(double) * (3 * n3 + n * n);
  SEM_CUDA(cudaFuncSetAttribute(geometry_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int* bad = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&bad, sizeof(int), h.stream));
  SEM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), h.stream));
  int threads = n3 >= 256 ? 256 : ((n3 + 31) / 32) * 32;
  int64_t grid = h.E < (int64_t)h.num_sms * 8 ? h.E : (int64_t)h.num_sms * 8;
  geometry_kernel<<<(int)grid, threads, smem, h.stream>>>(
      h.N, h.kx, h.ky, h.kz, lo[0], lo[1], lo[2], (hi[0] - lo[0]) / h.kx, (hi[1] - lo[1]) / h.ky,
      (hi[2] - lo[2]) / h.kz, amp, deform_kind, user_coords_dev, h.xi, h.wq, h.D64, h.E, h.coords,
      h.G64, h.G32, h.B64, h.detJ, bad);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  int bad_h = 0;
  SEM_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  SEM_CUDA(cudaFreeAsync(bad, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  if (bad_h) {
    set_error("sem_setup: non-positive Jacobian determinant (tangled mesh)");
    return SEM_EINVAL;
  }
  return 0;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of uint64 values: per-tile totals, a scan of the
// totals by one block, and a rescan of every tile with its offset.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline uint64_t block_exclusive_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  uint64_t before = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void scan_tile_sums(const uint64_t* in, int64_t n, uint64_t* sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + (int64_t)q * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  uint64_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums_single(uint64_t* sums, int64_t m, uint64_t* grand_total) {
  uint64_t carry = 0;
  for (int64_t base = 0; base < m; base += kScanThreads) {
    int64_t idx = base + threadIdx.x;
    uint64_t v = idx < m ? sums[idx] : 0;
    uint64_t total;
    uint64_t ex = block_exclusive_scan(v, &total);
    if (idx < m) sums[idx] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void scan_tiles(const uint64_t* in, uint64_t* out, int64_t n, const uint64_t* sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint64_t vals[kScanItems];
  uint64_t s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + q;
    vals[q] = idx < n ? in[idx] : 0;
    s += vals[q];
  }
  uint64_t total;
  uint64_t ex = block_exclusive_scan(s, &total) + sums[blockIdx.x];
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + q;
    if (idx < n) out[idx] = ex;
    ex += vals[q];
  }
}

// in/out may alias.  grand_total is a device pointer.
int exclusive_scan_u64(Handle& h, const uint64_t* in, uint64_t* out, int64_t n,
                              uint64_t* grand_total) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  uint64_t* sums = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&sums, sizeof(uint64_t) * tiles, h.stream));
  scan_tile_sums<<<(int)tiles, kScanThreads, 0, h.stream>>>(in, n, sums);
  scan_sums_single<<<1, kScanThreads, 0, h.stream>>>(sums, tiles, grand_total);
  scan_tiles<<<(int)tiles, kScanThreads, 0, h.stream>>>(in, out, n, sums);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaFreeAsync(sums, h.stream));
  return 0;
}

// ------------------------------------------------------------------ gather-scatter map
__global__ void count_copies(const int* gid, int64_t L, int* cnt) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[gid[l]], 1);
}

// packed = (segments << 32) | entries, counting only global nodes with >1 copy
__global__ void pack_counts(const int* cnt, int64_t U, uint64_t* packed) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < U;
       g += (int64_t)gridDim.x * blockDim.x) {
    int c = cnt[g];
    packed[g] = c > 1 ? ((1ull << 32) | (uint64_t)c) : 0ull;
  }
}

__global__ void write_seg_off(const int* cnt, const uint64_t* packed_ex, int64_t U, int* seg_off) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < U;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (cnt[g] > 1) {
      uint64_t p = packed_ex[g];
      seg_off[p >> 32] = (int)(p & 0xffffffffu);
    }
  }
}

__global__ void fill_perm(const int* gid, int64_t L, const int* cnt, const uint64_t* packed_ex,
                          int* cursor, int* perm) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    int g = gid[l];
    if (cnt[g] > 1) {
      int base = (int)(packed_ex[g] & 0xffffffffu);
      int slot = atomicAdd(&cursor[g], 1);
      perm[base + slot] = (int)l;
    }
  }
}

// Stable order inside every segment: ascending local index (insertion sort).
__global__ void sort_segments(const int* seg_off, int64_t nseg, int* perm) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    int a = seg_off[s], b = seg_off[s + 1];
    for (int q = a + 1; q < b; ++q) {
      int v = perm[q];
      int r = q - 1;
      while (r >= a && perm[r] > v) {
        perm[r + 1] = perm[r];
        --r;
      }
      perm[r + 1] = v;
    }
  }
}

__global__ void mult_and_weights(const int* gid, const int* cnt, const double* mask, int64_t L,
                                 double* mult, double* c64, float* c32, uint8_t* cw8) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int mi = cnt[gid[l]];
    double m = (double)mi;
    mult[l] = m;
    double c = mask[l] / m;
    c64[l] = c;
    c32[l] = (float)c;
    cw8[l] = mask[l] != 0.0 ? (uint8_t)(mi < 255 ? mi : 255) : (uint8_t)0;
  }
}

int launch_gs_map(Handle& h) {
  int* cnt = nullptr;
  uint64_t* packed = nullptr;
  uint64_t* tot_d = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int) * h.U, h.stream));
  SEM_CUDA(cudaMallocAsync((void**)&packed, sizeof(uint64_t) * h.U, h.stream));
  SEM_CUDA(cudaMallocAsync((void**)&tot_d, sizeof(uint64_t), h.stream));
  SEM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * h.U, h.stream));
  count_copies<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.gid, h.L, cnt);
  pack_counts<<<grid_for(h, h.U, 256), 256, 0, h.stream>>>(cnt, h.U, packed);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  int rc = exclusive_scan_u64(h, packed, packed, h.U, tot_d);
  if (rc) return rc;
  uint64_t tot = 0;
  SEM_CUDA(cudaMemcpyAsync(&tot, tot_d, sizeof(uint64_t), cudaMemcpyDeviceToHost, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  h.n_segments = (int64_t)(tot >> 32);
  h.n_shared = (int64_t)(tot & 0xffffffffu);
  if ((rc = alloc_t(h, &h.seg_off, (size_t)h.n_segments + 1))) return rc;
  if ((rc = alloc_t(h, &h.perm, (size_t)(h.n_shared > 0 ? h.n_shared : 1)))) return rc;
  int last = (int)h.n_shared;
  SEM_CUDA(cudaMemcpyAsync(h.seg_off + h.n_segments, &last, sizeof(int), cudaMemcpyHostToDevice,
                           h.stream));
  write_seg_off<<<grid_for(h, h.U, 256), 256, 0, h.stream>>>(cnt, packed, h.U, h.seg_off);
  int* cursor = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&cursor, sizeof(int) * h.U, h.stream));
  SEM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * h.U, h.stream));
  fill_perm<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.gid, h.L, cnt, packed, cursor, h.perm);
  sort_segments<<<grid_for(h, h.n_segments, 256), 256, 0, h.stream>>>(h.seg_off, h.n_segments,
                                                                        h.perm);
  mult_and_weights<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.gid, cnt, h.mask64, h.L,
                                                                 h.mult64, h.c64, h.c32, h.cw8);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaFreeAsync(cursor, h.stream));
  SEM_CUDA(cudaFreeAsync(cnt, h.stream));
  SEM_CUDA(cudaFreeAsync(packed, h.stream));
  SEM_CUDA(cudaFreeAsync(tot_d, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  return build_gs_buckets(h);
}

// ------------------------------------------------------------------ Jacobi
// diag of the element operator at node (i,j,k):
//   sum_l D_li^2 G_rr(l,j,k) + sum_l D_lj^2 G_ss(i,l,k) + sum_l D_lk^2 G_tt(i,j,l)
//   + 2 (D_ii D_jj G_rs + D_ii D_kk G_rt + D_jj D_kk G_st)(i,j,k)
__global__ void diag_local_kernel(int N, int64_t E, const double* __restrict__ G,
                                  const double* __restrict__ D, const double* __restrict__ mask,
                                  double* diag) {
  const int n = N + 1, n3 = n * n * n;
  const int64_t L = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = l / n3;
    int q = (int)(l - e * n3);
    int i = q % n, j = (q / n) % n, k = q / (n * n);
    const double* g = G + e * 6 * n3;
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
      double a = D[m * n + i], b = D[m * n + j], c = D[m * n + k];
      s += a * a * g[0 * n3 + m + n * j + n * n * k];
      s += b * b * g[1 * n3 + i + n * m + n * n * k];
      s += c * c * g[2 * n3 + i + n * j + n * n * m];
    }
    double di = D[i * n + i], dj = D[j * n + j], dk = D[k * n + k];
    s += 2.0 * (di * dj * g[3 * n3 + q] + di * dk * g[4 * n3 + q] + dj * dk * g[5 * n3 + q]);
    diag[l] = s * mask[l];
  }
}

__global__ void invert_diag(const double* diag, const double* mask, int64_t L, double* m64,
                            float* m32) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    double v = mask[l] != 0.0 ? 1.0 / diag[l] : 0.0;
    m64[l] = v;
    m32[l] = (float)v;
  }
}

int launch_jacobi(Handle& h) {
  double* diag = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&diag, sizeof(double) * h.L, h.stream));
  diag_local_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.N, h.E, h.G64, h.D64,
                                                                  h.mask64, diag);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  int rc = launch_gs(h, SEM_FP64, diag);
  if (rc) return rc;
  invert_diag<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(diag, h.mask64, h.L, h.minv64,
                                                            h.minv32);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaFreeAsync(diag, h.stream));
  return 0;
}

// ------------------------------------------------------------------ right-hand sides
__device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  // output number counter+1 of SplitMix64 started from state `seed`
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void rhs_uniform_kernel(const int* gid, const double* mask, int64_t L, uint64_t seed,
                                   double* b) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = splitmix64_at(seed, (uint64_t)gid[l]);
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    b[l] = mask[l] * (2.0 * u - 1.0);
  }
}

__global__ void rhs_sine_kernel(const double* coords, const double* B, int64_t L, double* b) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    double x = coords[l], y = coords[L + l], z = coords[2 * L + l];
    b[l] = B[l] * 3.0 * M_PI * M_PI * sin(M_PI * x) * sin(M_PI * y) * sin(M_PI * z);
  }
}

__global__ void mask_inplace(double* v, const double* mask, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    v[l] *= mask[l];
}

// Random Fourier series f = sum_{k in {1..K}^3} a_k sin(pi k1 x) sin(pi k2 y)
// sin(pi k3 z), a_k = xi_k / |k|^2, xi_k uniform in [-1, 1) from SplitMix64
// output number (sample K^3 + index(k)) + 1 of state `seed`,
// index(k) = (k1-1) + K (k2-1) + K^2 (k3-1).
constexpr int kFourierK = 8;

__global__ void fourier_coeff_kernel(uint64_t seed, uint64_t sample, double* a) {
  const int K = kFourierK;
  for (int q = threadIdx.x; q < K * K * K; q += blockDim.x) {
    const int k1 = q % K + 1, k2 = (q / K) % K + 1, k3 = q / (K * K) + 1;
    const uint64_t z = splitmix64_at(seed, sample * (uint64_t)(K * K * K) + (uint64_t)q);
    const double xi = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    a[q] = xi / (double)(k1 * k1 + k2 * k2 + k3 * k3);
  }
}

__global__ void fourier_rhs_kernel(const double* coords, const double* B, const double* a,
                                   int64_t L, double* b) {
  const int K = kFourierK;
  __shared__ double sa[kFourierK * kFourierK * kFourierK];
  for (int q = threadIdx.x; q < K * K * K; q += blockDim.x) sa[q] = a[q];
  __syncthreads();
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    double sx[kFourierK], sy[kFourierK], sz[kFourierK];
    const double x = coords[l], y = coords[L + l], z = coords[2 * L + l];
    for (int k = 0; k < K; ++k) {
      sx[k] = sin(M_PI * (k + 1) * x);
      sy[k] = sin(M_PI * (k + 1) * y);
      sz[k] = sin(M_PI * (k + 1) * z);
    }
    double f = 0.0;
    for (int k3 = 0; k3 < K; ++k3)
      for (int k2 = 0; k2 < K; ++k2) {
        double t = 0.0;
        for (int k1 = 0; k1 < K; ++k1) t += sa[k1 + K * (k2 + K * k3)] * sx[k1];
        f += t * sy[k2] * sz[k3];
      }
    b[l] = B[l] * f;
  }
}

int launch_rhs_fourier(Handle& h, uint64_t seed, uint64_t sample, double* b) {
  double* a = nullptr;
  SEM_CUDA(cudaMallocAsync((void**)&a, sizeof(double) * kFourierK * kFourierK * kFourierK, h.stream));
  fourier_coeff_kernel<<<1, 512, 0, h.stream>>>(seed, sample, a);
  fourier_rhs_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.coords, h.B64, a, h.L, b);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaFreeAsync(a, h.stream));
  int rc = launch_gs(h, SEM_FP64, b);
  if (rc) return rc;
  mask_inplace<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(b, h.mask64, h.L);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_rhs(Handle& h, int kind, uint64_t seed, double* b) {
  if (kind == 1) {
    rhs_uniform_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.gid, h.mask64, h.L, seed, b);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
    return 0;
  }
  if (kind == 0) {
    rhs_sine_kernel<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(h.coords, h.B64, h.L, b);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
    int rc = launch_gs(h, SEM_FP64, b);
    if (rc) return rc;
    mask_inplace<<<grid_for(h, h.L, 256), 256, 0, h.stream>>>(b, h.mask64, h.L);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
    return 0;
  }
  set_error("sem_rhs: unknown kind");
  return SEM_EINVAL;
}

}  // namespace sem
