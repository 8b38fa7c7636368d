// Learned initial guess: an element-local network trained on (right-hand
// side, solution) pairs produced by the solver itself, and used to start
// PCG from x0 = c * QQ^T(s_e * y_e) (the continuity projection with the
// glsc3 weight c of the paper's CG loop, Sec. 3.1).  The paper has no
// learned component; this is the extension the hot path carries.
//
// Network: 544 (530 features, zero padded) -> H -> H -> n^3, ReLU, FP32
// master weights with BF16 copies; products in BF16 with FP32 accumulation
// (GEMM kernel below), Adam (Kingma & Ba 2015) on the master weights.
// Features of element e: b_L / s_e (n^3 values), the element mean and
// standard deviation of each geometric factor G1..G6, and the mean of b_L
// over each face neighbour / s_e (0 on the domain boundary);
// s_e = sqrt(mean_e b_L^2) + 1e-30.  Targets: x_L / s_e, learned divided by
// their training-set RMS t (prediction s_e * t * y).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <random>
#include <vector>

#include "pcg.cuh"

namespace sem {

using bf16 = __nv_bfloat16;

constexpr int kFeat = 530;
constexpr int kFeatPad = 544;

// ------------------------------------------------------------------ GEMM
// C[M][N] = sum_k A(m,k) B(k,n) (+ bias[n]) (ReLU), FP32 accumulation.
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// 64x64 output tile per 256-thread block, 16-deep k slices staged in shared
// memory (converted to FP32), 4x4 outputs per thread; bounds checked.
constexpr int kGT = 64, kGK = 16;

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<bf16>(bf16 v) { return __bfloat162float(v); }

template <typename TAe, typename TBe, bool TA, bool TB>
__global__ void __launch_bounds__(256)
    gemm_kernel(int M, int N, int K, const TAe* __restrict__ A, int lda, const TBe* __restrict__ B,
                int ldb, const float* __restrict__ bias, int relu, float* __restrict__ C32,
                bf16* __restrict__ C16, int ldc) {
  __shared__ float As[kGK][kGT + 4];
  __shared__ float Bs[kGK][kGT + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int q = threadIdx.x; q < kGT * kGK; q += 256) {
      // A tile: rows m0..m0+63, cols k0..k0+15
      int mm, kk;
      if (TA) { mm = q % kGT; kk = q / kGT; } else { kk = q % kGK; mm = q / kGK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = to_f(TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]);
      As[kk][mm] = va;
      int nn, kb;
      if (TB) { kb = q % kGK; nn = q / kGK; } else { nn = q % kGT; kb = q / kGT; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float vb = 0.f;
      if (gn < N && gkb < K) vb = to_f(TB ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn]);
      Bs[kb][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gm = m0 + ty * 4 + r;
    if (gm >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gn = n0 + tx * 4 + c;
      if (gn >= N) continue;
      float v = acc[r][c] + (bias ? bias[gn] : 0.f);
      if (relu) v = v > 0.f ? v : 0.f;
      if (C32) C32[(size_t)gm * ldc + gn] = v;
      if (C16) C16[(size_t)gm * ldc + gn] = __float2bfloat16_rn(v);
    }
  }
}

template <typename TAe, typename TBe, bool TA, bool TB>
static int gemm(cudaStream_t st, int M, int N, int K, const TAe* A, int lda, const TBe* B, int ldb,
                const float* bias, int relu, float* C32, bf16* C16, int ldc) {
  dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
  gemm_kernel<TAe, TBe, TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, bias, relu, C32,
                                                      C16, ldc);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ features
// Per element: sum of b_L, sum of b_L^2 (block reductions, FP64).
__global__ void elem_moments(const double* __restrict__ b, int n3, int64_t E,
                             double* __restrict__ emean, double* __restrict__ escale) {
  __shared__ double sh[8];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    double s = 0.0, s2 = 0.0;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      const double v = b[e * n3 + q];
      s += v;
      s2 += v * v;
    }
    const double t = block_sum<kDotFP64>(s, sh);
    const double t2 = block_sum<kDotFP64>(s2, sh);
    if (threadIdx.x == 0) {
      emean[e] = t / n3;
      escale[e] = sqrt(t2 / n3) + 1e-30;
    }
  }
}

template <typename TO>
__global__ void elem_features(const double* __restrict__ b, const double* __restrict__ G, int n3,
                              int64_t E, int kx, int ky, int kz, const double* __restrict__ emean,
                              const double* __restrict__ escale, TO* __restrict__ X) {
  __shared__ double sh[8];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const double inv = 1.0 / escale[e];
    TO* row = X + e * kFeatPad;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) row[q] = (TO)(b[e * n3 + q] * inv);
    for (int a = 0; a < 6; ++a) {
      const double* g = G + (e * 6 + a) * n3;
      double s = 0.0;
      for (int q = threadIdx.x; q < n3; q += blockDim.x) s += g[q];
      const double mean = block_sum<kDotFP64>(s, sh) / n3;
      __shared__ double s_mean;
      if (threadIdx.x == 0) s_mean = mean;
      __syncthreads();
      double d2 = 0.0;
      for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        const double d = g[q] - s_mean;
        d2 += d * d;
      }
      const double var = block_sum<kDotFP64>(d2, sh) / n3;
      if (threadIdx.x == 0) {
        row[n3 + a] = (TO)s_mean;
        row[n3 + 6 + a] = (TO)sqrt(var);
      }
      __syncthreads();
    }
    if (threadIdx.x < 6) {
      const int f = threadIdx.x;
      const int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
      int64_t nb = -1;
      if (f == 0 && ex > 0) nb = e - 1;
      if (f == 1 && ex < kx - 1) nb = e + 1;
      if (f == 2 && ey > 0) nb = e - kx;
      if (f == 3 && ey < ky - 1) nb = e + kx;
      if (f == 4 && ez > 0) nb = e - (int64_t)kx * ky;
      if (f == 5 && ez < kz - 1) nb = e + (int64_t)kx * ky;
      row[n3 + 12 + f] = (TO)(nb >= 0 ? emean[nb] * inv : 0.0);
    }
    for (int q = n3 + 18 + threadIdx.x; q < kFeatPad; q += blockDim.x) row[q] = (TO)0.0;
  }
}

__global__ void elem_targets(const double* __restrict__ x, int n3, int64_t E,
                             const double* __restrict__ escale, bf16* __restrict__ T) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E * n3;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / n3;
    T[q] = __float2bfloat16_rn((float)(x[q] / escale[e]));
  }
}

// u_L = s_e * t * y (FP64 local vector; t the training-set target scale)
__global__ void scale_prediction(const float* __restrict__ Y, int n3, int64_t E,
                                 const double* __restrict__ escale, double tscale,
                                 double* __restrict__ u) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E * n3;
       q += (int64_t)gridDim.x * blockDim.x)
    u[q] = (double)Y[q] * tscale * escale[q / n3];
}

// sum of squares of BF16 values (per-block partials)
__global__ void sumsq_bf16(const bf16* __restrict__ T, int64_t count, double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)__bfloat162float(T[q]);
    s += v * v;
  }
  const double t = block_sum<kDotFP64>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void mul_weight(double* __restrict__ v, const double* __restrict__ c, int64_t L,
                           double alpha) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L;
       q += (int64_t)gridDim.x * blockDim.x)
    v[q] *= alpha * (c ? c[q] : 1.0);
}

// ------------------------------------------------------------------ training kernels
// dY = 2 (Y - T) / count, and per-block partial sums of (Y - T)^2.
template <typename TT>
__global__ void loss_grad(const float* __restrict__ Y, const TT* __restrict__ T, int64_t count,
                          float scale, float tinv, float* __restrict__ dY,
                          double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[q] - tinv * to_f(T[q]);
    dY[q] = scale * d;
    s += (double)d * d;
  }
  const double t = block_sum<kDotFP64>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// dH *= (H > 0)
__global__ void relu_back(float* __restrict__ dH, const float* __restrict__ H, int64_t count) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    if (!(H[q] > 0.f)) dH[q] = 0.f;
}

// db[n] = sum_m D[m][n]
__global__ void col_sums(const float* __restrict__ D, int M, int N, float* __restrict__ db) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(size_t)m * N + n];
    db[n] = s;
  }
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, bf16* __restrict__ w16,
                            int64_t count, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    w[q] = wq;
    w16[q] = __float2bfloat16_rn(wq);
  }
}

__global__ void to_bf16(const float* __restrict__ a, bf16* __restrict__ b, int64_t count) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    b[q] = __float2bfloat16_rn(a[q]);
}

template <typename TE>
__global__ void gather_rows(const TE* __restrict__ src, const int* __restrict__ rows, int nrows,
                            int width, TE* __restrict__ dst) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)nrows * width;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / width), c = (int)(q % width);
    dst[q] = src[(size_t)rows[r] * width + c];
  }
}

}  // namespace sem

// ------------------------------------------------------------------ model object
struct sem_x0_model_s {
  sem_handle_s* h = nullptr;
  int H = 256, in = sem::kFeatPad, out = 0;
  // parameter layout in one flat buffer: W1 [in x H], b1 [H], W2 [H x H], b2, W3 [H x out], b3
  int64_t off[6] = {}, size[6] = {}, nparam = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  sem::bf16* w16 = nullptr;
  int adam_t = 0;
  double tscale = 1.0;   // RMS of the training targets: the network learns targets / tscale
  // training set
  sem::bf16 *Xtr = nullptr, *Ttr = nullptr;
  int64_t rows = 0, cap = 0;
  // scratch (batch rows)
  int bcap = 0;
  sem::bf16 *Xb = nullptr, *Tb = nullptr, *H1b = nullptr, *H2b = nullptr;
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH = nullptr, *dH2 = nullptr;
  int* rowidx = nullptr;
  double* part = nullptr;
  double *emean = nullptr, *escale = nullptr, *u = nullptr;
  float* Xf = nullptr;   // FP32 features for gradient checks
};

namespace sem {

static int x0_alloc(sem_x0_model_s& M, int64_t bytes, void** p) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  return 0;
}

static int x0_ensure_batch(sem_x0_model_s& M, int rows) {
  if (rows <= M.bcap) return 0;
  void* ptrs[] = {M.Xb, M.Tb, M.H1b, M.H2b, M.H1, M.H2, M.Y, M.dY, M.dH, M.dH2, M.rowidx, M.part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  int rc;
  const int64_t r = rows;
  if ((rc = x0_alloc(M, r * M.in * 2, (void**)&M.Xb)) || (rc = x0_alloc(M, r * M.out * 2, (void**)&M.Tb)) ||
      (rc = x0_alloc(M, r * M.H * 2, (void**)&M.H1b)) || (rc = x0_alloc(M, r * M.H * 2, (void**)&M.H2b)) ||
      (rc = x0_alloc(M, r * M.H * 4, (void**)&M.H1)) || (rc = x0_alloc(M, r * M.H * 4, (void**)&M.H2)) ||
      (rc = x0_alloc(M, r * M.out * 4, (void**)&M.Y)) || (rc = x0_alloc(M, r * M.out * 4, (void**)&M.dY)) ||
      (rc = x0_alloc(M, r * std::max(M.H, M.in) * 4, (void**)&M.dH)) ||
      (rc = x0_alloc(M, r * M.H * 4, (void**)&M.dH2)) || (rc = x0_alloc(M, r * 4, (void**)&M.rowidx)) ||
      (rc = x0_alloc(M, 4096 * 8, (void**)&M.part)))
    return rc;
  M.bcap = rows;
  return 0;
}

// Forward pass over `rows` rows of X (BF16, or FP32 when Xf32), ending in
// M.Y (FP32).  fp32 = true keeps every operand in FP32 (debug precision).
static int x0_forward(sem_x0_model_s& M, cudaStream_t st, int rows, const bf16* X, const float* Xf32,
                      bool fp32) {
  int rc;
  const float* wf = M.w;
  const bf16* wb = M.w16;
  if (fp32) {
    if ((rc = gemm<float, float, false, false>(st, rows, M.H, M.in, Xf32, M.in, wf + M.off[0], M.H,
                                               wf + M.off[1], 1, M.H1, nullptr, M.H)))
      return rc;
    if ((rc = gemm<float, float, false, false>(st, rows, M.H, M.H, M.H1, M.H, wf + M.off[2], M.H,
                                               wf + M.off[3], 1, M.H2, nullptr, M.H)))
      return rc;
    return gemm<float, float, false, false>(st, rows, M.out, M.H, M.H2, M.H, wf + M.off[4], M.out,
                                            wf + M.off[5], 0, M.Y, nullptr, M.out);
  }
  if ((rc = gemm<bf16, bf16, false, false>(st, rows, M.H, M.in, X, M.in, wb + M.off[0], M.H,
                                           wf + M.off[1], 1, M.H1, M.H1b, M.H)))
    return rc;
  if ((rc = gemm<bf16, bf16, false, false>(st, rows, M.H, M.H, M.H1b, M.H, wb + M.off[2], M.H,
                                           wf + M.off[3], 1, M.H2, M.H2b, M.H)))
    return rc;
  return gemm<bf16, bf16, false, false>(st, rows, M.out, M.H, M.H2b, M.H, wb + M.off[4], M.out,
                                        wf + M.off[5], 0, M.Y, nullptr, M.out);
}

// Backward pass from M.dY: gradients into M.g (same layout as M.w).
static int x0_backward(sem_x0_model_s& M, cudaStream_t st, int rows, const bf16* X, const float* Xf32,
                       bool fp32) {
  int rc;
  const int64_t ro = rows;
  const int vg = 256;
  const int grid = (int)std::min<int64_t>((ro * M.H + vg - 1) / vg, 4096);
  // layer 3: dW3 = H2^T dY, db3 = colsum(dY), dH2 = dY W3^T * (H2 > 0)
  if (fp32) {
    if ((rc = gemm<float, float, true, false>(st, M.H, M.out, rows, M.H2, M.H, M.dY, M.out, nullptr, 0,
                                              M.g + M.off[4], nullptr, M.out)))
      return rc;
  } else {
    if ((rc = gemm<bf16, float, true, false>(st, M.H, M.out, rows, M.H2b, M.H, M.dY, M.out, nullptr, 0,
                                             M.g + M.off[4], nullptr, M.out)))
      return rc;
  }
  col_sums<<<(M.out + 255) / 256, 256, 0, st>>>(M.dY, rows, M.out, M.g + M.off[5]);
  if (fp32) {
    if ((rc = gemm<float, float, false, true>(st, rows, M.H, M.out, M.dY, M.out, M.w + M.off[4], M.out,
                                              nullptr, 0, M.dH2, nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm<float, bf16, false, true>(st, rows, M.H, M.out, M.dY, M.out, M.w16 + M.off[4], M.out,
                                             nullptr, 0, M.dH2, nullptr, M.H)))
      return rc;
  }
  relu_back<<<grid, vg, 0, st>>>(M.dH2, M.H2, ro * M.H);
  // layer 2
  if (fp32) {
    if ((rc = gemm<float, float, true, false>(st, M.H, M.H, rows, M.H1, M.H, M.dH2, M.H, nullptr, 0,
                                              M.g + M.off[2], nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm<bf16, float, true, false>(st, M.H, M.H, rows, M.H1b, M.H, M.dH2, M.H, nullptr, 0,
                                             M.g + M.off[2], nullptr, M.H)))
      return rc;
  }
  col_sums<<<(M.H + 255) / 256, 256, 0, st>>>(M.dH2, rows, M.H, M.g + M.off[3]);
  if (fp32) {
    if ((rc = gemm<float, float, false, true>(st, rows, M.H, M.H, M.dH2, M.H, M.w + M.off[2], M.H,
                                              nullptr, 0, M.dH, nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm<float, bf16, false, true>(st, rows, M.H, M.H, M.dH2, M.H, M.w16 + M.off[2], M.H,
                                             nullptr, 0, M.dH, nullptr, M.H)))
      return rc;
  }
  relu_back<<<grid, vg, 0, st>>>(M.dH, M.H1, ro * M.H);
  // layer 1
  if (fp32) {
    if ((rc = gemm<float, float, true, false>(st, M.in, M.H, rows, Xf32, M.in, M.dH, M.H, nullptr, 0,
                                              M.g + M.off[0], nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm<bf16, float, true, false>(st, M.in, M.H, rows, X, M.in, M.dH, M.H, nullptr, 0,
                                             M.g + M.off[0], nullptr, M.H)))
      return rc;
  }
  col_sums<<<(M.H + 255) / 256, 256, 0, st>>>(M.dH, rows, M.H, M.g + M.off[1]);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// loss (mean of squares) and dY for `rows` rows against targets T
template <typename TT>
static int x0_loss(sem_x0_model_s& M, cudaStream_t st, int rows, const TT* T, double* loss,
                   float tinv = 1.f) {
  const int64_t count = (int64_t)rows * M.out;
  const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
  loss_grad<TT><<<grid, 256, 0, st>>>(M.Y, T, count, 2.f / (float)count, tinv, M.dY, M.part);
  SEM_CUDA(cudaGetLastError());
  if (loss) {
    std::vector<double> h(grid);
    SEM_CUDA(cudaMemcpyAsync(h.data(), M.part, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    *loss = s / (double)count;
  }
  return 0;
}

static int x0_features(sem_x0_model_s& M, const double* b, bf16* X16, float* X32) {
  Handle& h = *M.h;
  const int n3 = h.n * h.n * h.n;
  const int grid = (int)std::min<int64_t>(h.E, (int64_t)h.num_sms * 8);
  elem_moments<<<grid, 256, 0, h.stream>>>(b, n3, h.E, M.emean, M.escale);
  if (X16)
    elem_features<bf16><<<grid, 256, 0, h.stream>>>(b, h.G64, n3, h.E, h.kx, h.ky, h.kz, M.emean,
                                                    M.escale, X16);
  if (X32)
    elem_features<float><<<grid, 256, 0, h.stream>>>(b, h.G64, n3, h.E, h.kx, h.ky, h.kz, M.emean,
                                                     M.escale, X32);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

static void x0_free(sem_x0_model_s* M) {
  if (!M) return;
  if (M->h && M->h->stream) cudaStreamSynchronize(M->h->stream);
  void* ptrs[] = {M->w, M->g, M->m, M->v, M->w16, M->Xtr, M->Ttr, M->Xb, M->Tb, M->H1b, M->H2b,
                  M->H1, M->H2, M->Y, M->dY, M->dH, M->dH2, M->rowidx, M->part, M->emean,
                  M->escale, M->u, M->Xf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete M;
}

}  // namespace sem

using namespace sem;

extern "C" int sem_x0_create(sem_handle h, int hidden, uint64_t seed, sem_x0_model* out) {
  if (!h || !out || hidden < 8 || hidden > 4096) {
    set_error("sem_x0_create: invalid argument");
    return SEM_EINVAL;
  }
  if (h->gid_user) {
    set_error("sem_x0_create: the learned guess needs a box mesh (face neighbours)");
    return SEM_EINVAL;
  }
  if (h->n * h->n * h->n + 18 > kFeatPad) {
    set_error("sem_x0_create: the network's 544 inputs hold n^3 + 18 features (N <= 7)");
    return SEM_EINVAL;
  }
  *out = nullptr;
  sem_x0_model_s* M = new sem_x0_model_s();
  M->h = h;
  M->H = hidden;
  M->out = h->n * h->n * h->n;
  const int64_t sz[6] = {(int64_t)M->in * hidden, hidden, (int64_t)hidden * hidden, hidden,
                         (int64_t)hidden * M->out, M->out};
  int64_t o = 0;
  for (int q = 0; q < 6; ++q) {
    M->off[q] = o;
    M->size[q] = sz[q];
    o += (sz[q] + 31) / 32 * 32;
  }
  M->nparam = o;
  int rc;
  if ((rc = x0_alloc(*M, o * 4, (void**)&M->w)) || (rc = x0_alloc(*M, o * 4, (void**)&M->g)) ||
      (rc = x0_alloc(*M, o * 4, (void**)&M->m)) || (rc = x0_alloc(*M, o * 4, (void**)&M->v)) ||
      (rc = x0_alloc(*M, o * 2, (void**)&M->w16)) || (rc = x0_alloc(*M, h->E * 8, (void**)&M->emean)) ||
      (rc = x0_alloc(*M, h->E * 8, (void**)&M->escale)) ||
      (rc = x0_alloc(*M, h->L * 8, (void**)&M->u))) {
    x0_free(M);
    return rc;
  }
  // He-normal initial weights (host PRNG, seeded), zero biases; padded input rows zero
  std::vector<float> w(o, 0.f);
  std::mt19937_64 gen(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  const int fan_in[3] = {kFeat, hidden, hidden};
  for (int l = 0; l < 3; ++l) {
    const int64_t rowsz = (l == 2) ? M->out : hidden;
    const int64_t nrows = (l == 0) ? kFeat : hidden;
    const float sd = sqrtf(2.f / fan_in[l]);
    for (int64_t r = 0; r < nrows; ++r)
      for (int64_t c = 0; c < rowsz; ++c) w[M->off[2 * l] + r * rowsz + c] = sd * nd(gen);
  }
  cudaError_t ce;
  if ((ce = cudaMemcpy(M->w, w.data(), o * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemset(M->m, 0, o * 4)) != cudaSuccess || (ce = cudaMemset(M->v, 0, o * 4)) != cudaSuccess) {
    x0_free(M);
    return cuda_fail(ce, "sem_x0_create");
  }
  to_bf16<<<256, 256, 0, h->stream>>>(M->w, M->w16, o);
  if ((ce = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    x0_free(M);
    return cuda_fail(ce, "sem_x0_create");
  }
  *out = M;
  return SEM_OK;
}

extern "C" void sem_x0_destroy(sem_x0_model m) { x0_free(m); }

extern "C" int sem_x0_param_count(sem_x0_model m, int64_t* sizes6, int64_t* offsets6) {
  if (!m) {
    set_error("sem_x0_param_count: null model");
    return SEM_EINVAL;
  }
  for (int q = 0; q < 6; ++q) {
    if (sizes6) sizes6[q] = m->size[q];
    if (offsets6) offsets6[q] = m->off[q];
  }
  return SEM_OK;
}

extern "C" int sem_x0_params(sem_x0_model m, float* host, int set) {
  if (!m || !host) {
    set_error("sem_x0_params: null argument");
    return SEM_EINVAL;
  }
  cudaStream_t st = m->h->stream;
  if (set) {
    SEM_CUDA(cudaMemcpyAsync(m->w, host, m->nparam * 4, cudaMemcpyHostToDevice, st));
    to_bf16<<<256, 256, 0, st>>>(m->w, m->w16, m->nparam);
    SEM_CUDA(cudaGetLastError());
    m->adam_t = 0;
    SEM_CUDA(cudaMemsetAsync(m->m, 0, m->nparam * 4, st));
    SEM_CUDA(cudaMemsetAsync(m->v, 0, m->nparam * 4, st));
  } else {
    SEM_CUDA(cudaMemcpyAsync(host, m->w, m->nparam * 4, cudaMemcpyDeviceToHost, st));
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  return SEM_OK;
}

extern "C" int sem_x0_gradients(sem_x0_model m, const float* X, const float* T, int rows, int bf16_mode,
                                float* grads, double* loss) {
  if (!m || !X || !T || !grads || rows < 1) {
    set_error("sem_x0_gradients: invalid argument");
    return SEM_EINVAL;
  }
  cudaStream_t st = m->h->stream;
  int rc;
  if ((rc = x0_ensure_batch(*m, rows))) return rc;
  float *Xd = nullptr, *Td = nullptr;
  SEM_CUDA(cudaMalloc((void**)&Xd, (size_t)rows * m->in * 4));
  SEM_CUDA(cudaMalloc((void**)&Td, (size_t)rows * m->out * 4));
  SEM_CUDA(cudaMemcpyAsync(Xd, X, (size_t)rows * m->in * 4, cudaMemcpyHostToDevice, st));
  SEM_CUDA(cudaMemcpyAsync(Td, T, (size_t)rows * m->out * 4, cudaMemcpyHostToDevice, st));
  const bool fp32 = !bf16_mode;
  if (!fp32) {
    to_bf16<<<256, 256, 0, st>>>(Xd, m->Xb, (int64_t)rows * m->in);
    to_bf16<<<256, 256, 0, st>>>(Td, m->Tb, (int64_t)rows * m->out);
  }
  rc = x0_forward(*m, st, rows, m->Xb, Xd, fp32);
  if (!rc) rc = fp32 ? x0_loss<float>(*m, st, rows, Td, loss) : x0_loss<bf16>(*m, st, rows, m->Tb, loss);
  if (!rc) rc = x0_backward(*m, st, rows, m->Xb, Xd, fp32);
  if (!rc) {
    cudaError_t ce = cudaMemcpyAsync(grads, m->g, m->nparam * 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "sem_x0_gradients");
  }
  cudaFree(Xd);
  cudaFree(Td);
  return rc;
}

extern "C" int sem_x0_features(sem_x0_model m, const double* b, float* X, double* scale) {
  if (!m || !b || !X) {
    set_error("sem_x0_features: invalid argument");
    return SEM_EINVAL;
  }
  Handle& h = *m->h;
  int rc;
  if (!m->Xf) {
    SEM_CUDA(cudaMalloc((void**)&m->Xf, (size_t)h.E * kFeatPad * 4));
  }
  if ((rc = x0_features(*m, b, nullptr, m->Xf))) return rc;
  SEM_CUDA(cudaMemcpyAsync(X, m->Xf, (size_t)h.E * kFeatPad * 4, cudaMemcpyDefault, h.stream));
  if (scale)
    SEM_CUDA(cudaMemcpyAsync(scale, m->escale, (size_t)h.E * 8, cudaMemcpyDefault, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  return SEM_OK;
}

extern "C" int sem_x0_add_pair(sem_x0_model m, const double* b, const double* x) {
  if (!m || !b || !x || !is_device_ptr(b) || !is_device_ptr(x)) {
    set_error("sem_x0_add_pair: b and x must be device pointers");
    return SEM_EINVAL;
  }
  Handle& h = *m->h;
  const int64_t E = h.E, n3 = m->out;
  if (m->rows + E > m->cap) {
    const int64_t ncap = std::max<int64_t>(2 * m->cap, m->rows + E);
    bf16 *X2 = nullptr, *T2 = nullptr;
    SEM_CUDA(cudaMalloc((void**)&X2, (size_t)ncap * m->in * 2));
    SEM_CUDA(cudaMalloc((void**)&T2, (size_t)ncap * n3 * 2));
    if (m->rows) {
      SEM_CUDA(cudaMemcpyAsync(X2, m->Xtr, (size_t)m->rows * m->in * 2, cudaMemcpyDeviceToDevice, h.stream));
      SEM_CUDA(cudaMemcpyAsync(T2, m->Ttr, (size_t)m->rows * n3 * 2, cudaMemcpyDeviceToDevice, h.stream));
    }
    SEM_CUDA(cudaStreamSynchronize(h.stream));
    if (m->Xtr) cudaFree(m->Xtr);
    if (m->Ttr) cudaFree(m->Ttr);
    m->Xtr = X2;
    m->Ttr = T2;
    m->cap = ncap;
  }
  int rc;
  if ((rc = x0_features(*m, b, m->Xtr + m->rows * m->in, nullptr))) return rc;
  elem_targets<<<(int)std::min<int64_t>((E * n3 + 255) / 256, 4096), 256, 0, h.stream>>>(
      x, (int)n3, E, m->escale, m->Ttr + m->rows * n3);
  SEM_CUDA(cudaGetLastError());
  m->rows += E;
  return SEM_OK;
}

extern "C" int sem_x0_train(sem_x0_model m, int epochs, int batch, float lr, uint64_t seed,
                            double* final_loss) {
  if (!m || epochs < 0 || batch < 1 || !(lr > 0.f)) {
    set_error("sem_x0_train: invalid argument");
    return SEM_EINVAL;
  }
  if (m->rows == 0) {
    set_error("sem_x0_train: no training pairs (sem_x0_add_pair)");
    return SEM_EINVAL;
  }
  Handle& h = *m->h;
  cudaStream_t st = h.stream;
  int rc;
  const int bs = (int)std::min<int64_t>(batch, m->rows);
  if ((rc = x0_ensure_batch(*m, bs))) return rc;
  // global target scale: the RMS of every stored target value
  {
    const int64_t count = m->rows * m->out;
    const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
    sumsq_bf16<<<grid, 256, 0, st>>>(m->Ttr, count, m->part);
    std::vector<double> hp(grid);
    SEM_CUDA(cudaMemcpyAsync(hp.data(), m->part, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    double ss = 0.0;
    for (double v : hp) ss += v;
    m->tscale = ss > 0.0 ? sqrt(ss / (double)count) : 1.0;
  }
  const float tinv = (float)(1.0 / m->tscale);
  std::vector<int> perm((size_t)m->rows);
  for (int64_t q = 0; q < m->rows; ++q) perm[(size_t)q] = (int)q;
  std::mt19937_64 gen(seed);
  int* idx_dev = nullptr;
  SEM_CUDA(cudaMalloc((void**)&idx_dev, sizeof(int) * m->rows));
  double loss = 0.0;
  for (int ep = 0; ep < epochs && !rc; ++ep) {
    std::shuffle(perm.begin(), perm.end(), gen);
    SEM_CUDA(cudaMemcpyAsync(idx_dev, perm.data(), sizeof(int) * m->rows, cudaMemcpyHostToDevice, st));
    double ep_loss = 0.0;
    int nb = 0;
    for (int64_t r0 = 0; r0 + bs <= m->rows && !rc; r0 += bs) {
      gather_rows<bf16><<<1024, 256, 0, st>>>(m->Xtr, idx_dev + r0, bs, m->in, m->Xb);
      gather_rows<bf16><<<1024, 256, 0, st>>>(m->Ttr, idx_dev + r0, bs, m->out, m->Tb);
      rc = x0_forward(*m, st, bs, m->Xb, nullptr, false);
      const bool last = (ep == epochs - 1);
      double bl = 0.0;
      if (!rc) rc = x0_loss<bf16>(*m, st, bs, m->Tb, last ? &bl : nullptr, tinv);
      if (!rc) rc = x0_backward(*m, st, bs, m->Xb, nullptr, false);
      if (!rc) {
        m->adam_t += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        adam_kernel<<<1024, 256, 0, st>>>(m->w, m->g, m->m, m->v, m->w16, m->nparam, lr, b1, b2,
                                          1e-8f, c1, c2);
        if (cudaGetLastError() != cudaSuccess) rc = SEM_ECUDA;
      }
      ep_loss += bl;
      ++nb;
    }
    if (epochs - 1 == ep && nb) loss = ep_loss / nb;
  }
  cudaStreamSynchronize(st);
  cudaFree(idx_dev);
  if (rc) return rc;
  if (final_loss) *final_loss = loss;
  return SEM_OK;
}

extern "C" int sem_x0_predict(sem_x0_model m, const double* b, double* x0, int energy_scale) {
  if (!m || !b || !x0 || !is_device_ptr(b) || !is_device_ptr(x0)) {
    set_error("sem_x0_predict: b and x0 must be device pointers");
    return SEM_EINVAL;
  }
  Handle& h = *m->h;
  cudaStream_t st = h.stream;
  int rc;
  const int rows = (int)h.E;
  if ((rc = x0_ensure_batch(*m, rows))) return rc;
  if ((rc = x0_features(*m, b, m->Xb, nullptr))) return rc;
  if ((rc = x0_forward(*m, st, rows, m->Xb, nullptr, false))) return rc;
  const int grid = (int)std::min<int64_t>((h.L + 255) / 256, (int64_t)h.num_sms * 8);
  scale_prediction<<<grid, 256, 0, st>>>(m->Y, m->out, h.E, m->escale, m->tscale, x0);
  SEM_CUDA(cudaGetLastError());
  // continuity projection x0 = c * QQ^T(u_pred)
  if ((rc = launch_gs(h, SEM_FP64, x0))) return rc;
  mul_weight<<<grid, 256, 0, st>>>(x0, h.c64, h.L, 1.0);
  SEM_CUDA(cudaGetLastError());
  if (energy_scale) {
    // alpha = <b, c, x0> / <x0, c, A x0>: the energy-optimal multiple of x0,
    // never worse than x0 = 0 in the A-norm
    if ((rc = launch_ax_local(h, SEM_FP64, x0, m->u, nullptr))) return rc;
    if ((rc = launch_gs(h, SEM_FP64, m->u))) return rc;
    double num = 0.0, den = 0.0;
    if ((rc = launch_glsc3(h, SEM_FP64, b, x0, h.dot_out))) return rc;
    SEM_CUDA(cudaMemcpyAsync(&num, h.dot_out, 8, cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    if ((rc = launch_glsc3(h, SEM_FP64, x0, m->u, h.dot_out))) return rc;
    SEM_CUDA(cudaMemcpyAsync(&den, h.dot_out, 8, cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    const double alpha = den > 0.0 ? num / den : 0.0;
    mul_weight<<<grid, 256, 0, st>>>(x0, nullptr, h.L, alpha);
    SEM_CUDA(cudaGetLastError());
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  return SEM_OK;
}
