// Learned initial guess: an element-local network trained on (right-hand
// side, solution) pairs produced by the solver itself, and used to start
// PCG from x0 = c * QQ^T(s_e * y_e) (the continuity projection with the
// glsc3 weight c of the paper's CG loop, Sec. 3.1).  The paper has no
// learned component; this is the extension the hot path carries.
//
// Network: 544 (530 features, or 539 with the coarse features, zero
// padded) -> H -> H -> n^3, ReLU, FP32 master weights with BF16 copies;
// products on the tensor cores in BF16 with FP32 accumulation (gemm_tc
// below: tcgen05 with the accumulator in tensor memory, or warp-level
// mma.sync; the FP32 gradient-check mode uses the CUDA-core GEMM), Adam
// (Kingma & Ba 2015) on the master weights.
// Features of element e: b_L / s_e (n^3 values), the element mean and
// standard deviation of each geometric factor G1..G6, and the mean of b_L
// over each face neighbour / s_e (0 on the domain boundary);
// s_e = sqrt(mean_e b_L^2) + 1e-30.  Targets: x_L / s_e, learned divided by
// their training-set RMS t (prediction s_e * t * y).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "pcg.cuh"
#include "umma.cuh"

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

// ------------------------------------------------------------------ tensor-core GEMM
// The BF16 products of training and inference on the tensor cores: warp-level
// mma.sync m16n8k16 (BF16 operands, FP32 accumulation).  A block computes a
// 64x64 tile of C with 4 warps (2 x 2, 32x32 each); 32-deep k slices of A
// and B are converted to BF16 (FP32 operands, e.g. dY, are rounded once
// here) and stored k-contiguous in shared memory with rows padded to 40
// elements, so each fragment register is one conflict-free 32-bit load.
// splits > 1 divides K (the batch rows of the weight gradients) over
// gridDim.z blocks writing FP32 partial tiles to `part`; reduce_splits adds
// them in split order (deterministic), then bias / ReLU are applied.
constexpr int kTM = 64, kTN = 64, kTK = 32, kTKP = kTK + 8;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
template <typename T>
__device__ __forceinline__ bf16 to_bf(T v);
template <>
__device__ __forceinline__ bf16 to_bf<float>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ bf16 to_bf<bf16>(bf16 v) { return v; }

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TAe, typename TBe, bool TA, bool TB>
__global__ void __launch_bounds__(128)
    gemm_tc_kernel(int M, int N, int K, int kchunk, const TAe* __restrict__ A, int lda,
                   const TBe* __restrict__ B, int ldb, const float* __restrict__ bias, int relu,
                   float* __restrict__ C32, bf16* __restrict__ C16, int ldc,
                   float* __restrict__ part) {
  __shared__ __align__(16) bf16 As[kTM][kTKP];   // As[m][k]
  __shared__ __align__(16) bf16 Bs[kTN][kTKP];   // Bs[n][k]
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int wm = (warp / 2) * 32, wn = (warp % 2) * 32;
  const int gid = lane / 4, tig = lane % 4;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[2][4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += kTK) {
    // stage: 64 x 32 of A and of B, 16 elements per thread each, read along
    // the operand's contiguous index
    for (int q = threadIdx.x; q < kTM * kTK; q += 128) {
      int mm, kk;
      if (TA) { mm = q % kTM; kk = q / kTM; } else { kk = q % kTK; mm = q / kTK; }
      const int gm = m0 + mm, gk = k0 + kk;
      bf16 va = __float2bfloat16_rn(0.f);
      if (gm < M && gk < ke) va = to_bf(TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]);
      As[mm][kk] = va;
      int nn, kq;
      if (TB) { kq = q % kTK; nn = q / kTK; } else { nn = q % kTN; kq = q / kTN; }
      const int gn = n0 + nn, gkb = k0 + kq;
      bf16 vb = __float2bfloat16_rn(0.f);
      if (gn < N && gkb < ke) vb = to_bf(TB ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn]);
      Bs[nn][kq] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + gid;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tig]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tig]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tig + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + gid;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tig]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + 16 * i + gid + 8 * h;
        if (gm >= M) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int gn = n0 + wn + 8 * j + 2 * tig + c;
          if (gn >= N) continue;
          const float v0 = acc[i][j][2 * h + c];
          if (part) {
            part[((size_t)blockIdx.z * M + gm) * N + gn] = v0;
            continue;
          }
          float v = v0 + (bias ? bias[gn] : 0.f);
          if (relu) v = v > 0.f ? v : 0.f;
          if (C32) C32[(size_t)gm * ldc + gn] = v;
          if (C16) C16[(size_t)gm * ldc + gn] = __float2bfloat16_rn(v);
        }
      }
}

// C = sum over splits of the partial tiles (in split order), bias, ReLU.
__global__ void reduce_splits(const float* __restrict__ part, int splits, int M, int N,
                              const float* __restrict__ bias, int relu, float* __restrict__ C32,
                              bf16* __restrict__ C16, int ldc) {
  const int64_t MN = (int64_t)M * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < MN;
       q += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += part[z * MN + q];
    const int gm = (int)(q / N), gn = (int)(q % N);
    v += bias ? bias[gn] : 0.f;
    if (relu) v = v > 0.f ? v : 0.f;
    if (C32) C32[(size_t)gm * ldc + gn] = v;
    if (C16) C16[(size_t)gm * ldc + gn] = __float2bfloat16_rn(v);
  }
}

// Operand preparation for the tcgen05 GEMM: dst[r][k] = src(r, k) in BF16
// for r < R, k < Kp (zero for k >= K), src(r, k) = TR ? src[k ld + r] :
// src[r ld + k]; 32 x 32 tiles through shared memory, so that both the
// reads and the writes run along contiguous addresses.
template <typename T, bool TR>
__global__ void __launch_bounds__(256)
    to_kmajor_bf16(const T* __restrict__ src, int ld, int R, int K, int Kp, bf16* __restrict__ dst) {
  __shared__ float tile[32][33];   // tile[k - k0][r - r0]
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int i = ty; i < 32; i += 8) {
    if (TR) {
      const int k = k0 + i, r = r0 + tx;
      tile[i][tx] = (k < K && r < R) ? to_f(src[(size_t)k * ld + r]) : 0.f;
    } else {
      const int r = r0 + i, k = k0 + tx;
      tile[tx][i] = (r < R && k < K) ? to_f(src[(size_t)r * ld + k]) : 0.f;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r < R && k < Kp) dst[(size_t)r * Kp + k] = __float2bfloat16_rn(tile[tx][i]);
  }
}

// The same product on the tcgen05 tensor cores (umma.cuh), for K-major
// BF16 operands A [M][K] (row stride lda) and B [N][K] (ldb), K and the
// strides multiples of 8, 16-byte aligned: a 128 x 128 output tile per
// 128-thread block, K in chunks of 64 through four shared-memory stages
// filled by 16-byte cp.async copies (three chunks in flight while the MMAs
// of the fourth run) in the 128-byte-swizzled layout (each 8-thread phase
// fills one 128-byte row: no bank conflicts), the FP32 accumulator in 128
// TMEM columns.  Epilogue in four passes of 32 columns: each warp reads its
// TMEM lane quarter into a padded shared tile, then every warp writes whole
// 32-column row segments.  Splits, bias, ReLU and outputs as
// gemm_tc_kernel.  A bounded wait that gives up sets *err, waits (bounded)
// for the MMAs in flight and for its copies, frees the TMEM and leaves the
// tile unwritten.
__global__ void __launch_bounds__(128)
    gemm_umma_kernel(int M, int N, int K, int kchunk, const bf16* __restrict__ A, int lda,
                     const bf16* __restrict__ B, int ldb, const float* __restrict__ bias, int relu,
                     float* __restrict__ C32, bf16* __restrict__ C16, int ldc,
                     float* __restrict__ part, int* __restrict__ err) {
  constexpr int S = kUStages;
  extern __shared__ uint8_t usm_raw[];
  uint8_t* const usm = reinterpret_cast<uint8_t*>(((uintptr_t)usm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* const sA = usm;
  uint8_t* const sB = usm + S * kUTileA;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(usm + S * (kUTileA + kUTileB));
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(bar + S);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int m0 = blockIdx.y * kUM, n0 = blockIdx.x * kUN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int nch = ke > kb ? (ke - kb + kUK - 1) / kUK : 0;
  if (warp == 0) {
    tmem_alloc(tslot, kUCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = umma_idesc(kUM, kUN);
  // chunk c into stage c % S: 128 rows x 8 chunks of 16 bytes per operand,
  // 8 per thread, eight consecutive threads on the eight chunks of one row
  auto load_chunk = [&](int c) {
    const int st = c % S, k0 = kb + c * kUK;
    uint8_t* const a_st = sA + st * kUTileA;
    uint8_t* const b_st = sB + st * kUTileB;
#pragma unroll
    for (int i = 0; i < kUM * (kUK / 8) / 128; ++i) {
      const int q = tid + 128 * i;
      const int row = q >> 3, ch = q & 7;
      const int gk = k0 + 8 * ch;
      const int gm = m0 + row, gn = n0 + row;
      const bool ia = gk < ke && gm < M, ib = gk < ke && gn < N;
      cp_async16(a_st + umma_chunk_off(row, ch), ia ? A + (size_t)gm * lda + gk : A, ia ? 16u : 0u);
      cp_async16(b_st + umma_chunk_off(row, ch), ib ? B + (size_t)gn * ldb + gk : B, ib ? 16u : 0u);
    }
  };
#pragma unroll
  for (int c = 0; c < S - 1; ++c) {
    if (c < nch) load_chunk(c);
    cp_async_commit();
  }
  bool ok = true;
  int issued = 0;   // chunks whose MMAs thread 0 issued and committed
  for (int c = 0; c < nch; ++c) {
    const int s = c % S;
    // groups committed so far: S - 1 + c; chunk c's is complete once at
    // most S - 2 are pending
    cp_async_wait<S - 2>();
    // the tensor core reads shared memory through the async proxy
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_addr(sA + s * kUTileA), b0 = smem_addr(sB + s * kUTileB);
#pragma unroll
      for (int ks = 0; ks < kUK / 16; ++ks)
        umma_bf16(tmem, umma_desc(a0 + ks * 32), umma_desc(b0 + ks * 32), idesc,
                  (c > 0 || ks > 0) ? 1u : 0u);
      umma_commit(&bar[s]);
    }
    issued = c + 1;
    // chunk c + S - 1 refills the stage of chunk c - 1 once its MMAs are done
    const int cn = c + S - 1;
    if (cn < nch) {
      if (c >= 1) {
        const bool w = mbar_wait_bounded(&bar[(c - 1) % S], (uint32_t)(((c - 1) / S) & 1));
        if (__syncthreads_or(!w)) {
          ok = false;
          break;
        }
      }
      load_chunk(cn);
    }
    cp_async_commit();
  }
  if (ok && nch > 0) {
    // the last commit completes after every MMA issued before it
    const int c = nch - 1;
    const bool w = mbar_wait_bounded(&bar[c % S], (uint32_t)((c / S) & 1));
    if (__syncthreads_or(!w)) ok = false;
  }
  cp_async_wait<0>();   // no copy into this block's shared memory outlives it
  if (!ok) {
    if (tid == 0) {
      atomicExch(err, 1);
      const int c = issued - 1;
      if (c >= 0) mbar_wait_bounded(&bar[c % S], (uint32_t)((c / S) & 1));
    }
  } else {
    tc_fence_after();
    // the operand stages are free: a [128][33] float tile for one pass
    float (*tileC)[33] = reinterpret_cast<float (*)[33]>(usm);
#pragma unroll 1
    for (int cc = 0; cc < kUN / 32; ++cc) {
      float v[32];
      if (nch > 0) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) tileC[warp * 32 + lane][j] = v[j];
      __syncthreads();
      const int gn = n0 + cc * 32 + lane;
#pragma unroll 4
      for (int rr = warp; rr < kUM; rr += 4) {
        const int gm = m0 + rr;
        if (gm < M && gn < N) {
          const float a = tileC[rr][lane];
          if (part) {
            part[((size_t)blockIdx.z * M + gm) * N + gn] = a;
          } else {
            float o = a + (bias ? bias[gn] : 0.f);
            if (relu) o = o > 0.f ? o : 0.f;
            if (C32) C32[(size_t)gm * ldc + gn] = o;
            if (C16) C16[(size_t)gm * ldc + gn] = __float2bfloat16_rn(o);
          }
        }
      }
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kUCols);
}

// Partial tiles of the split-K products: up to kMaxSplits x M x N floats.
constexpr int kMaxSplits = 32;

// Which tensor-core GEMM runs the BF16 products, and the error word of its
// bounded waits.
struct TcCfg {
  bool umma = true;      // tcgen05 (gemm_umma_kernel); false: mma.sync (gemm_tc_kernel)
  int* err = nullptr;
  bf16 *ua = nullptr, *ub = nullptr;   // K-major BF16 copies of the operands (grown on demand)
  int64_t ua_cap = 0, ub_cap = 0;
};

// Grows one operand scratch buffer to hold `need` values.
static int tc_scratch(bf16** buf, int64_t* cap, int64_t need) {
  if (need <= *cap) return 0;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  SEM_CUDA(cudaMalloc((void**)buf, (size_t)need * sizeof(bf16)));
  *cap = need;
  return 0;
}

template <typename TAe, typename TBe, bool TA, bool TB>
static int gemm_tc(TcCfg& cfg, cudaStream_t st, int num_sms, float* scratch,
                   int64_t scratch_floats, int M, int N, int K, const TAe* A, int lda, const TBe* B,
                   int ldb, const float* bias, int relu, float* C32, bf16* C16, int ldc,
                   double* ms_acc = nullptr) {
  const int tm = cfg.umma ? kUM : kTM, tn = cfg.umma ? kUN : kTN, tk = cfg.umma ? kUK : kTK;
  const int gx = (N + tn - 1) / tn, gy = (M + tm - 1) / tm;
  // split K until the grid covers the SMs about twice (weight gradients:
  // K = the batch rows, M x N = one weight matrix)
  int splits = 1;
  while (splits < kMaxSplits && (int64_t)gx * gy * splits < 2LL * num_sms &&
         K / (2 * splits) >= 4 * tk && (int64_t)(2 * splits) * M * N <= scratch_floats)
    splits *= 2;
  const int kchunk = ((K + splits - 1) / splits + tk - 1) / tk * tk;
  dim3 grid(gx, gy, splits);
  if (cfg.umma) {
    // K-major BF16 operands: used in place where they already are, else
    // converted (and transposed) into the model's scratch, K padded to a
    // multiple of 8 with zeros
    const int Kp = (K + 7) / 8 * 8;
    const int kch = ((Kp + splits - 1) / splits + kUK - 1) / kUK * kUK;
    const bf16* Ak = nullptr;
    const bf16* Bk = nullptr;
    int ldak = Kp, ldbk = Kp;
    if (std::is_same<TAe, bf16>::value && !TA && lda % 8 == 0 && K % 8 == 0 &&
        ((uintptr_t)A & 15) == 0) {
      Ak = reinterpret_cast<const bf16*>(A);
      ldak = lda;
    } else {
      int rc = tc_scratch(&cfg.ua, &cfg.ua_cap, (int64_t)M * Kp);
      if (rc) return rc;
      to_kmajor_bf16<TAe, TA><<<dim3((Kp + 31) / 32, (M + 31) / 32), 256, 0, st>>>(A, lda, M, K, Kp, cfg.ua);
      Ak = cfg.ua;
    }
    if (std::is_same<TBe, bf16>::value && TB && ldb % 8 == 0 && K % 8 == 0 &&
        ((uintptr_t)B & 15) == 0) {
      Bk = reinterpret_cast<const bf16*>(B);
      ldbk = ldb;
    } else {
      int rc = tc_scratch(&cfg.ub, &cfg.ub_cap, (int64_t)N * Kp);
      if (rc) return rc;
      to_kmajor_bf16<TBe, !TB><<<dim3((Kp + 31) / 32, (N + 31) / 32), 256, 0, st>>>(B, ldb, N, K, Kp, cfg.ub);
      Bk = cfg.ub;
    }
    SEM_CUDA(cudaGetLastError());
    SEM_CUDA(cudaFuncSetAttribute(gemm_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kUSmem));
    gemm_umma_kernel<<<grid, 128, kUSmem, st>>>(M, N, Kp, kch, Ak, ldak, Bk, ldbk, bias, relu, C32,
                                                C16, ldc, splits > 1 ? scratch : nullptr, cfg.err);
  } else {
    gemm_tc_kernel<TAe, TBe, TA, TB><<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, bias,
                                                           relu, C32, C16, ldc,
                                                           splits > 1 ? scratch : nullptr);
  }
  SEM_CUDA(cudaGetLastError());
  if (splits > 1) {
    const int64_t MN = (int64_t)M * N;
    reduce_splits<<<(int)std::min<int64_t>((MN + 255) / 256, 4096), 256, 0, st>>>(
        scratch, splits, M, N, bias, relu, C32, C16, ldc);
    SEM_CUDA(cudaGetLastError());
  }
  (void)ms_acc;
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
                              const double* __restrict__ escale, const float* __restrict__ zc,
                              double zmul, TO* __restrict__ X) {
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
    if (zc) {
      // coarse information: a multigrid approximation z of the solution at
      // the element's 8 vertices and its element mean, / s_e
      __syncthreads();
      int n = 1;
      while (n * n * n < n3) ++n;
      if (threadIdx.x < 8) {
        const int c = threadIdx.x;
        const int vi = (c & 1) ? n - 1 : 0, vj = (c & 2) ? n - 1 : 0, vk = (c & 4) ? n - 1 : 0;
        row[n3 + 18 + c] = (TO)((double)zc[e * n3 + vi + n * (vj + n * vk)] * inv * zmul);
      }
      double s = 0.0;
      for (int q = threadIdx.x; q < n3; q += blockDim.x) s += zc[e * n3 + q];
      const double zm = block_sum<kDotFP64>(s, sh) / n3;
      if (threadIdx.x == 0) row[n3 + 26] = (TO)(zm * inv * zmul);
    }
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

// db[n] = sum_m D[m][n] in two deterministic passes: block (x, y) sums
// rows y, y + gridDim.y, ... of 32 columns (a warp reads 32 consecutive
// floats of a row; the 8 warps' sums are added in warp order) into
// part[y][n]; col_sums_finish adds the gridDim.y partials in order.
constexpr int kColChunks = 32;
__global__ void __launch_bounds__(256)
    col_sums(const float* __restrict__ D, int M, int N, float* __restrict__ part) {
  __shared__ float sh[8][33];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int n = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (n < N)
    for (int m = blockIdx.y + gridDim.y * warp; m < M; m += gridDim.y * 8) s += D[(size_t)m * N + n];
  sh[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && n < N) {
    float t = 0.f;
    for (int q = 0; q < 8; ++q) t += sh[q][lane];
    part[(size_t)blockIdx.y * N + n] = t;
  }
}
__global__ void col_sums_finish(const float* __restrict__ part, int chunks, int N,
                                float* __restrict__ db) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int y = 0; y < chunks; ++y) s += part[(size_t)y * N + n];
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
  float* gs = nullptr;          // split-K partial tiles of the tensor-core products
  int64_t gs_floats = 0;
  double *emean = nullptr, *escale = nullptr, *u = nullptr;
  float* Xf = nullptr;   // FP32 features for gradient checks
  // options (sem_x0_set_option)
  int64_t pair_rows = 0;    // element rows kept per training pair (0: all E)
  int coarse_cycles = 0;    // FP32 multigrid cycles behind the coarse features (0: off)
  int post_cycles = 0;      // multigrid-Richardson steps applied to the prediction
  int64_t pairs = 0;        // training pairs added so far
  double zmul = 1.0;        // coarse features' factor: 1 / RMS of the first pair's x_L / s_e
  float *zc = nullptr, *rc32 = nullptr, *dz32 = nullptr;   // coarse / smoothing work (L each)
  double* r64 = nullptr;    // residual (L)
  double* ratio = nullptr;  // device scalars of the energy scaling: {<b,c,x0>, <x0,c,A x0>}
  sem::bf16* Xall = nullptr;   // features of every element of one pair (E rows)
  sem::bf16* Tall = nullptr;
  int* sel = nullptr;       // selected element rows of one pair
  sem::TcCfg tc;            // BF16 GEMM kind ("umma" option) and its device error word
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
  if ((rc = gemm_tc<bf16, bf16, false, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, rows, M.H, M.in, X, M.in, wb + M.off[0], M.H,
                                           wf + M.off[1], 1, M.H1, M.H1b, M.H)))
    return rc;
  if ((rc = gemm_tc<bf16, bf16, false, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, rows, M.H, M.H, M.H1b, M.H, wb + M.off[2], M.H,
                                           wf + M.off[3], 1, M.H2, M.H2b, M.H)))
    return rc;
  return gemm_tc<bf16, bf16, false, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, rows, M.out, M.H, M.H2b, M.H, wb + M.off[4], M.out,
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
    if ((rc = gemm_tc<bf16, float, true, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, M.H, M.out, rows, M.H2b, M.H, M.dY, M.out, nullptr, 0,
                                             M.g + M.off[4], nullptr, M.out)))
      return rc;
  }
  col_sums<<<dim3((M.out + 31) / 32, kColChunks), 256, 0, st>>>(M.dY, rows, M.out, M.gs);
  col_sums_finish<<<(M.out + 255) / 256, 256, 0, st>>>(M.gs, kColChunks, M.out, M.g + M.off[5]);
  if (fp32) {
    if ((rc = gemm<float, float, false, true>(st, rows, M.H, M.out, M.dY, M.out, M.w + M.off[4], M.out,
                                              nullptr, 0, M.dH2, nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm_tc<float, bf16, false, true>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, rows, M.H, M.out, M.dY, M.out, M.w16 + M.off[4], M.out,
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
    if ((rc = gemm_tc<bf16, float, true, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, M.H, M.H, rows, M.H1b, M.H, M.dH2, M.H, nullptr, 0,
                                             M.g + M.off[2], nullptr, M.H)))
      return rc;
  }
  col_sums<<<dim3((M.H + 31) / 32, kColChunks), 256, 0, st>>>(M.dH2, rows, M.H, M.gs);
  col_sums_finish<<<(M.H + 255) / 256, 256, 0, st>>>(M.gs, kColChunks, M.H, M.g + M.off[3]);
  if (fp32) {
    if ((rc = gemm<float, float, false, true>(st, rows, M.H, M.H, M.dH2, M.H, M.w + M.off[2], M.H,
                                              nullptr, 0, M.dH, nullptr, M.H)))
      return rc;
  } else {
    if ((rc = gemm_tc<float, bf16, false, true>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, rows, M.H, M.H, M.dH2, M.H, M.w16 + M.off[2], M.H,
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
    if ((rc = gemm_tc<bf16, float, true, false>(M.tc, st, M.h->num_sms, M.gs, M.gs_floats, M.in, M.H, rows, X, M.in, M.dH, M.H, nullptr, 0,
                                             M.g + M.off[0], nullptr, M.H)))
      return rc;
  }
  col_sums<<<dim3((M.H + 31) / 32, kColChunks), 256, 0, st>>>(M.dH, rows, M.H, M.gs);
  col_sums_finish<<<(M.H + 255) / 256, 256, 0, st>>>(M.gs, kColChunks, M.H, M.g + M.off[1]);
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

__global__ void to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t L) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L;
       q += (int64_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}
// y += x (FP32 into FP32 or FP64), r = b - w (FP32 or FP64)
template <typename TY, typename TX>
__global__ void add_to(TY* __restrict__ y, const TX* __restrict__ x, int64_t L) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] += (TY)x[q];
}
template <typename T>
__global__ void sub_from(const T* __restrict__ b, const T* __restrict__ w, T* __restrict__ r,
                         int64_t L) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L;
       q += (int64_t)gridDim.x * blockDim.x)
    r[q] = b[q] - w[q];
}

int mg_apply(Handle& h, sem_precision p, const void* r, void* z);

// Coarse approximation of the solution for the features: `cycles` FP32
// multigrid-Richardson steps from z = 0 (z += M^{-1}(b - A z)), into M.zc.
static int x0_coarse(sem_x0_model_s& M, const double* b) {
  Handle& h = *M.h;
  const int grid = (int)std::min<int64_t>((h.L + 255) / 256, (int64_t)h.num_sms * 8);
  int rc;
  to_f32<<<grid, 256, 0, h.stream>>>(b, M.rc32, h.L);   // r = b (z = 0)
  SEM_CUDA(cudaMemsetAsync(M.zc, 0, sizeof(float) * h.L, h.stream));
  for (int c = 0; c < M.coarse_cycles; ++c) {
    if (c > 0) {
      // r = b - A z (FP32 operator, summed, masked)
      if ((rc = launch_ax_local(h, SEM_MIXED_FP32, M.zc, M.dz32, nullptr))) return rc;
      if ((rc = launch_gs(h, SEM_MIXED_FP32, M.dz32))) return rc;
      to_f32<<<grid, 256, 0, h.stream>>>(b, M.rc32, h.L);
      sub_from<float><<<grid, 256, 0, h.stream>>>(M.rc32, M.dz32, M.rc32, h.L);
    }
    if ((rc = mg_apply(h, SEM_MIXED_FP32, M.rc32, M.dz32))) return rc;
    add_to<float, float><<<grid, 256, 0, h.stream>>>(M.zc, M.dz32, h.L);
  }
  SEM_CUDA(cudaGetLastError());
  return 0;
}

static int x0_features(sem_x0_model_s& M, const double* b, bf16* X16, float* X32) {
  Handle& h = *M.h;
  const int n3 = h.n * h.n * h.n;
  const int grid = (int)std::min<int64_t>(h.E, (int64_t)h.num_sms * 8);
  int rc;
  if (M.coarse_cycles > 0 && (rc = x0_coarse(M, b))) return rc;
  const float* zc = M.coarse_cycles > 0 ? M.zc : nullptr;
  elem_moments<<<grid, 256, 0, h.stream>>>(b, n3, h.E, M.emean, M.escale);
  if (X16)
    elem_features<bf16><<<grid, 256, 0, h.stream>>>(b, h.G64, n3, h.E, h.kx, h.ky, h.kz, M.emean,
                                                    M.escale, zc, M.zmul, X16);
  if (X32)
    elem_features<float><<<grid, 256, 0, h.stream>>>(b, h.G64, n3, h.E, h.kx, h.ky, h.kz, M.emean,
                                                     M.escale, zc, M.zmul, X32);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// After a stream synchronisation: whether a tensor-core GEMM's bounded wait
// gave up since the last check (its tile was then left unwritten).
static int x0_check_err(sem_x0_model_s& M) {
  int e = 0;
  SEM_CUDA(cudaMemcpy(&e, M.tc.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!e) return 0;
  SEM_CUDA(cudaMemset(M.tc.err, 0, sizeof(int)));
  set_error("learned guess: a tensor-core GEMM's bounded wait gave up (MMA did not complete)");
  return SEM_ETIMEOUT;
}

static void x0_free(sem_x0_model_s* M) {
  if (!M) return;
  if (M->h && M->h->stream) cudaStreamSynchronize(M->h->stream);
  void* ptrs[] = {M->w, M->g, M->m, M->v, M->w16, M->Xtr, M->Ttr, M->Xb, M->Tb, M->H1b, M->H2b,
                  M->H1, M->H2, M->Y, M->dY, M->dH, M->dH2, M->rowidx, M->part, M->emean,
                  M->escale, M->u, M->Xf, M->gs, M->zc, M->rc32, M->dz32, M->r64,
                  M->ratio, M->Xall, M->Tall, M->sel, M->tc.err, M->tc.ua, M->tc.ub};
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
      (rc = x0_alloc(*M, h->L * 8, (void**)&M->u)) || (rc = x0_alloc(*M, 4, (void**)&M->tc.err)) ||
      (rc = x0_alloc(*M, (M->gs_floats = (int64_t)kMaxSplits *
                                         std::max<int64_t>({sz[0], sz[2], sz[4], 1 << 20})) * 4,
                     (void**)&M->gs))) {
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
      (ce = cudaMemset(M->m, 0, o * 4)) != cudaSuccess || (ce = cudaMemset(M->v, 0, o * 4)) != cudaSuccess ||
      (ce = cudaMemset(M->tc.err, 0, 4)) != cudaSuccess) {
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
  if (!rc) rc = x0_check_err(*m);
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

// Grow the training set to hold `rows` rows (one allocation, old rows copied).
static int x0_reserve(sem_x0_model_s& m, int64_t rows) {
  if (rows <= m.cap) return 0;
  Handle& h = *m.h;
  bf16 *X2 = nullptr, *T2 = nullptr;
  SEM_CUDA(cudaMalloc((void**)&X2, (size_t)rows * m.in * 2));
  cudaError_t ce = cudaMalloc((void**)&T2, (size_t)rows * m.out * 2);
  if (ce != cudaSuccess) {
    cudaFree(X2);
    return cuda_fail(ce, "cudaMalloc");
  }
  if (m.rows) {
    SEM_CUDA(cudaMemcpyAsync(X2, m.Xtr, (size_t)m.rows * m.in * 2, cudaMemcpyDeviceToDevice, h.stream));
    SEM_CUDA(cudaMemcpyAsync(T2, m.Ttr, (size_t)m.rows * m.out * 2, cudaMemcpyDeviceToDevice, h.stream));
  }
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  if (m.Xtr) cudaFree(m.Xtr);
  if (m.Ttr) cudaFree(m.Ttr);
  m.Xtr = X2;
  m.Ttr = T2;
  m.cap = rows;
  return 0;
}

extern "C" int sem_x0_add_pair(sem_x0_model m, const double* b, const double* x) {
  if (!m || !b || !x || !is_device_ptr(b) || !is_device_ptr(x)) {
    set_error("sem_x0_add_pair: b and x must be device pointers");
    return SEM_EINVAL;
  }
  Handle& h = *m->h;
  const int64_t E = h.E, n3 = m->out;
  const int64_t keep = (m->pair_rows > 0 && m->pair_rows < E) ? m->pair_rows : E;
  int rc;
  if (m->rows + keep > m->cap &&
      (rc = x0_reserve(*m, std::max<int64_t>(2 * m->cap, m->rows + keep))))
    return rc;
  const int tg = (int)std::min<int64_t>((E * n3 + 255) / 256, 4096);
  if (m->coarse_cycles > 0 && m->pairs == 0) {
    // the coarse values z / s_e approximate the targets x_L / s_e, whose
    // size is set by the problem (b carries the mass matrix): scale them by
    // the first pair's target RMS so the features are O(1) like the others
    if (!m->Tall) SEM_CUDA(cudaMalloc((void**)&m->Tall, (size_t)E * n3 * 2));
    if (!m->part && (rc = x0_ensure_batch(*m, 1))) return rc;
    const int grid = (int)std::min<int64_t>(E, (int64_t)h.num_sms * 8);
    elem_moments<<<grid, 256, 0, h.stream>>>(b, (int)n3, E, m->emean, m->escale);
    elem_targets<<<tg, 256, 0, h.stream>>>(x, (int)n3, E, m->escale, m->Tall);
    sumsq_bf16<<<tg, 256, 0, h.stream>>>(m->Tall, E * n3, m->part);
    std::vector<double> hp(tg);
    SEM_CUDA(cudaMemcpyAsync(hp.data(), m->part, sizeof(double) * tg, cudaMemcpyDeviceToHost, h.stream));
    SEM_CUDA(cudaStreamSynchronize(h.stream));
    double ss = 0.0;
    for (double v : hp) ss += v;
    m->zmul = ss > 0.0 ? 1.0 / sqrt(ss / (double)(E * n3)) : 1.0;
  }
  if (keep == E) {
    if ((rc = x0_features(*m, b, m->Xtr + m->rows * m->in, nullptr))) return rc;
    elem_targets<<<tg, 256, 0, h.stream>>>(x, (int)n3, E, m->escale, m->Ttr + m->rows * n3);
  } else {
    // a seeded random subset of `keep` elements of this pair (seed: the pair's index)
    if (!m->Xall) {
      SEM_CUDA(cudaMalloc((void**)&m->Xall, (size_t)E * m->in * 2));
      SEM_CUDA(cudaMalloc((void**)&m->Tall, (size_t)E * n3 * 2));
      SEM_CUDA(cudaMalloc((void**)&m->sel, (size_t)E * sizeof(int)));
    }
    if ((rc = x0_features(*m, b, m->Xall, nullptr))) return rc;
    elem_targets<<<tg, 256, 0, h.stream>>>(x, (int)n3, E, m->escale, m->Tall);
    std::vector<int> idx((size_t)E);
    for (int64_t q = 0; q < E; ++q) idx[(size_t)q] = (int)q;
    std::mt19937_64 gen(0x9e3779b97f4a7c15ull ^ (uint64_t)m->pairs);
    std::shuffle(idx.begin(), idx.end(), gen);
    SEM_CUDA(cudaMemcpyAsync(m->sel, idx.data(), sizeof(int) * keep, cudaMemcpyHostToDevice, h.stream));
    gather_rows<bf16><<<1024, 256, 0, h.stream>>>(m->Xall, m->sel, (int)keep, m->in,
                                                  m->Xtr + m->rows * m->in);
    gather_rows<bf16><<<1024, 256, 0, h.stream>>>(m->Tall, m->sel, (int)keep, (int)n3,
                                                  m->Ttr + m->rows * n3);
    // the host index array is reused by the next call: wait for its copy
    SEM_CUDA(cudaStreamSynchronize(h.stream));
  }
  SEM_CUDA(cudaGetLastError());
  m->rows += keep;
  m->pairs += 1;
  return SEM_OK;
}

extern "C" int sem_x0_set_option(sem_x0_model m, const char* key, int64_t value) {
  if (!m || !key) {
    set_error("sem_x0_set_option: null argument");
    return SEM_EINVAL;
  }
  const std::string k(key);
  Handle& h = *m->h;
  if (k == "pair_rows" && value >= 0) {
    m->pair_rows = value;
  } else if (k == "umma" && (value == 0 || value == 1)) {
    m->tc.umma = value != 0;
  } else if (k == "reserve_rows" && value >= 0) {
    return x0_reserve(*m, value);
  } else if ((k == "coarse_cycles" || k == "post_cycles") && value >= 0 && value <= 16) {
    if (k == "coarse_cycles") {
      if (value > 0 && h.n * h.n * h.n + 27 > kFeatPad) {
        set_error("sem_x0_set_option: no room for the coarse features at this order");
        return SEM_EINVAL;
      }
      if (m->rows > 0 && (value > 0) != (m->coarse_cycles > 0)) {
        set_error("sem_x0_set_option: the feature set cannot change once pairs are stored");
        return SEM_EINVAL;
      }
      m->coarse_cycles = (int)value;
    } else {
      m->post_cycles = (int)value;
    }
    if (value > 0 && !m->zc) {
      SEM_CUDA(cudaMalloc((void**)&m->zc, sizeof(float) * h.L));
      SEM_CUDA(cudaMalloc((void**)&m->rc32, sizeof(float) * h.L));
      SEM_CUDA(cudaMalloc((void**)&m->dz32, sizeof(float) * h.L));
      SEM_CUDA(cudaMalloc((void**)&m->r64, sizeof(double) * h.L));
    }
  } else {
    set_error("sem_x0_set_option: unknown key or value out of range: " + k);
    return SEM_EINVAL;
  }
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
  if ((rc = x0_check_err(*m))) return rc;
  if (final_loss) *final_loss = loss;
  return SEM_OK;
}

// x0 *= <b, c, x0> / <x0, c, A x0> (0 if the denominator is not positive),
// from the two device scalars, without a host round trip
__global__ void scale_by_ratio(double* __restrict__ x0, const double* __restrict__ nd, int64_t L) {
  const double den = nd[1];
  const double alpha = den > 0.0 ? nd[0] / den : 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L;
       q += (int64_t)gridDim.x * blockDim.x)
    x0[q] *= alpha;
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
  if (!m->ratio) SEM_CUDA(cudaMalloc((void**)&m->ratio, 2 * sizeof(double)));
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
    if ((rc = launch_glsc3(h, SEM_FP64, b, x0, m->ratio))) return rc;
    if ((rc = launch_glsc3(h, SEM_FP64, x0, m->u, m->ratio + 1))) return rc;
    scale_by_ratio<<<grid, 256, 0, st>>>(x0, m->ratio, h.L);
    SEM_CUDA(cudaGetLastError());
  }
  // post-smoothing: x0 += M^{-1}(b - A x0), the residual in FP64, the cycle
  // in FP32 (its rough error is what the guess carries)
  for (int c = 0; c < m->post_cycles; ++c) {
    if ((rc = launch_ax_local(h, SEM_FP64, x0, m->r64, nullptr))) return rc;
    if ((rc = launch_gs(h, SEM_FP64, m->r64))) return rc;
    sub_from<double><<<grid, 256, 0, st>>>(b, m->r64, m->r64, h.L);
    to_f32<<<grid, 256, 0, st>>>(m->r64, m->rc32, h.L);
    if ((rc = mg_apply(h, SEM_MIXED_FP32, m->rc32, m->dz32))) return rc;
    add_to<double, float><<<grid, 256, 0, st>>>(x0, m->dz32, h.L);
    SEM_CUDA(cudaGetLastError());
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  return x0_check_err(*m);
}
