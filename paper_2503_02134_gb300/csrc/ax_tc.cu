// Element operator with the D-contractions on tensor cores.
//
// The six contractions of the paper's `ax` (Sec. 3.1: local_grad3 and
// local_grad3_t, i.e. mxm with the n x n derivative matrix) are, for one
// element, products of an (n^2 x n) matrix of nodal values with D^T or D:
//   r: Ur[(k,j), i] = sum_l u[k][j][l] D[i][l]     s: Us[(k,i), j] = sum_l u[k][l][i] D[j][l]
//   t: Ut[(j,i), k] = sum_l u[l][j][i] D[k][l]     and the same with D for D^T v.
// Each warp computes 16-row x 8-column tiles with warp-level MMAs
// (m16n8k8 TF32, or m16n8k16 BF16 with the error-compensating split
// a = a_hi + a_lo and a*b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32
// accumulation; n is padded to a multiple of 8 (16) with zero rows of D.
// The geometric factor step between the contractions and the Dirichlet mask
// run on CUDA cores from shared memory.  One element per block.
#include <cuda_bf16.h>

#include "ax_kernel.cuh"

namespace sem {

enum TcMode { kTcTF32 = 0, kTcBF16x3 = 1 };

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_col, float hi_col) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);   // .x = first (lower) element
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void split_bf16(float a, float& hi, float& lo) {
  hi = __bfloat162float(__float2bfloat16_rn(a));
  lo = a - hi;
}

// One contraction of an element: out[(p,q), o] (+)= sum_l in(p,q,l) * M[o][l]
// where in(p,q,l) = src[p*sp + q*sq + l*sl] (element local, floats) and
// M[o][l] = Dm[o*n + l] (transposeD: Dm[l*n + o]).  Rows r = p*n + q of the
// n^2 x n product; the result goes to dst[p*dp + q*dq + o*do_] (ACC: +=).
template <int n, int NP, int MODE, bool transposeD, bool ACC>
__device__ void tc_contract(const float* __restrict__ src, int sp, int sq, int sl,
                            const float* __restrict__ Dm, float* __restrict__ dst, int dp, int dq,
                            int do_) {
  constexpr int rows = n * n;
  constexpr int mtiles = (rows + 15) / 16;
  constexpr int ntiles = NP / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  auto A = [&](int r, int l) -> float {   // zero outside the n^2 x n matrix
    if (r >= rows || l >= n) return 0.f;
    const int p = r / n, q = r % n;
    return src[p * sp + q * sq + l * sl];
  };
  auto B = [&](int l, int o) -> float {   // B[l][o] = M[o][l]
    if (l >= n || o >= n) return 0.f;
    return transposeD ? Dm[l * n + o] : Dm[o * n + l];
  };
  for (int tile = warp; tile < mtiles * ntiles; tile += nwarps) {
    const int mt = tile / ntiles, nt = tile % ntiles;
    const int r0 = mt * 16, o0 = nt * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    if (MODE == kTcTF32) {
      for (int k0 = 0; k0 < NP; k0 += 8) {
        uint32_t a[4], b[2];
        a[0] = to_tf32(A(r0 + g, k0 + t));
        a[1] = to_tf32(A(r0 + g + 8, k0 + t));
        a[2] = to_tf32(A(r0 + g, k0 + t + 4));
        a[3] = to_tf32(A(r0 + g + 8, k0 + t + 4));
        b[0] = to_tf32(B(k0 + t, o0 + g));
        b[1] = to_tf32(B(k0 + t + 4, o0 + g));
        mma_tf32(c, a, b);
      }
    } else {
      for (int k0 = 0; k0 < NP; k0 += 16) {
        float av[8], bv[4];
        av[0] = A(r0 + g, k0 + 2 * t);
        av[1] = A(r0 + g, k0 + 2 * t + 1);
        av[2] = A(r0 + g + 8, k0 + 2 * t);
        av[3] = A(r0 + g + 8, k0 + 2 * t + 1);
        av[4] = A(r0 + g, k0 + 2 * t + 8);
        av[5] = A(r0 + g, k0 + 2 * t + 9);
        av[6] = A(r0 + g + 8, k0 + 2 * t + 8);
        av[7] = A(r0 + g + 8, k0 + 2 * t + 9);
        bv[0] = B(k0 + 2 * t, o0 + g);
        bv[1] = B(k0 + 2 * t + 1, o0 + g);
        bv[2] = B(k0 + 2 * t + 8, o0 + g);
        bv[3] = B(k0 + 2 * t + 9, o0 + g);
        float ah[8], al[8], bh[4], bl[4];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16(av[q], ah[q], al[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) split_bf16(bv[q], bh[q], bl[q]);
        uint32_t aH[4], aL[4], bH[2], bL[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          aH[q] = pack_bf16(ah[2 * q], ah[2 * q + 1]);
          aL[q] = pack_bf16(al[2 * q], al[2 * q + 1]);
        }
        bH[0] = pack_bf16(bh[0], bh[1]);
        bH[1] = pack_bf16(bh[2], bh[3]);
        bL[0] = pack_bf16(bl[0], bl[1]);
        bL[1] = pack_bf16(bl[2], bl[3]);
        mma_bf16(c, aL, bH);   // small terms first
        mma_bf16(c, aH, bL);
        mma_bf16(c, aH, bH);
      }
    }
    // C fragment: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + g + (q >= 2 ? 8 : 0);
      const int o = o0 + 2 * t + (q & 1);
      if (r < rows && o < n) {
        const int p = r / n, qq = r % n;
        float* d = dst + p * dp + qq * dq + o * do_;
        if (ACC) *d += c[q]; else *d = c[q];
      }
    }
  }
}

template <int n, int MODE>
__global__ void __launch_bounds__(256)
    ax_tc_kernel(const float* __restrict__ uin, float* __restrict__ wout,
                 const float* __restrict__ G, const float* __restrict__ Dg,
                 const uint8_t* __restrict__ faces, int64_t E) {
  constexpr int n2 = n * n, n3 = n * n * n;
  constexpr int NP = MODE == kTcTF32 ? ((n + 7) / 8) * 8 : ((n + 15) / 16) * 16;
  extern __shared__ __align__(16) float sm[];
  float* su = sm;            // u, later w
  float* sr = su + n3;       // u_r, later v_r
  float* ss = sr + n3;       // u_s, later v_s
  float* st = ss + n3;       // u_t, later v_t
  float* sD = st + n3;       // D (n*n)
  for (int q = threadIdx.x; q < n2; q += blockDim.x) sD[q] = Dg[q];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    for (int q = threadIdx.x; q < n3; q += blockDim.x) su[q] = uin[e * n3 + q];
    __syncthreads();
    // u_r[k][j][i] (rows (k,j)), u_s[k][j][i] (rows (k,i)), u_t[k][j][i] (rows (j,i))
    tc_contract<n, NP, MODE, false, false>(su, n2, n, 1, sD, sr, n2, n, 1);
    tc_contract<n, NP, MODE, false, false>(su, n2, 1, n, sD, ss, n2, 1, n);
    tc_contract<n, NP, MODE, false, false>(su, n, 1, n2, sD, st, n, 1, n2);
    __syncthreads();
    const float* Ge = G + e * 6 * n3;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      const float ur = sr[q], us = ss[q], ut = st[q];
      const float g0 = Ge[q], g1 = Ge[n3 + q], g2 = Ge[2 * n3 + q];
      const float g3 = Ge[3 * n3 + q], g4 = Ge[4 * n3 + q], g5 = Ge[5 * n3 + q];
      sr[q] = g0 * ur + g3 * us + g4 * ut;
      ss[q] = g3 * ur + g1 * us + g5 * ut;
      st[q] = g4 * ur + g5 * us + g2 * ut;
    }
    __syncthreads();
    // w = D_r^T v_r + D_s^T v_s + D_t^T v_t, accumulated in su in three passes
    tc_contract<n, NP, MODE, true, false>(sr, n2, n, 1, sD, su, n2, n, 1);
    __syncthreads();
    tc_contract<n, NP, MODE, true, true>(ss, n2, 1, n, sD, su, n2, 1, n);
    __syncthreads();
    tc_contract<n, NP, MODE, true, true>(st, n, 1, n2, sD, su, n, 1, n2);
    __syncthreads();
    const uint8_t f = faces[e];
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      const int i = q % n, j = (q / n) % n, k = q / n2;
      wout[e * n3 + q] = on_dirichlet(f, i, j, k, n - 1) ? 0.f : su[q];
    }
  }
}

template <int n, int MODE>
static int tc_launch(Handle& h, const float* u, float* w) {
  auto kern = ax_tc_kernel<n, MODE>;
  const size_t smem = sizeof(float) * (4 * n * n * n + n * n);
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
  const int64_t cap = (int64_t)h.num_sms * (per_sm > 0 ? per_sm : 1);
  const int grid = (int)(h.E < cap ? h.E : cap);
  kern<<<grid, 256, smem, h.stream>>>(u, w, h.G32, h.D32, h.bfaces, h.E);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

template <int MODE>
static int tc_dispatch(Handle& h, const float* u, float* w) {
  switch (h.n) {
    case 2: return tc_launch<2, MODE>(h, u, w);
    case 3: return tc_launch<3, MODE>(h, u, w);
    case 4: return tc_launch<4, MODE>(h, u, w);
    case 5: return tc_launch<5, MODE>(h, u, w);
    case 6: return tc_launch<6, MODE>(h, u, w);
    case 7: return tc_launch<7, MODE>(h, u, w);
    case 8: return tc_launch<8, MODE>(h, u, w);
    case 9: return tc_launch<9, MODE>(h, u, w);
    case 10: return tc_launch<10, MODE>(h, u, w);
    case 11: return tc_launch<11, MODE>(h, u, w);
    case 12: return tc_launch<12, MODE>(h, u, w);
    case 13: return tc_launch<13, MODE>(h, u, w);
    case 14: return tc_launch<14, MODE>(h, u, w);
    case 15: return tc_launch<15, MODE>(h, u, w);
    case 16: return tc_launch<16, MODE>(h, u, w);
    default: set_error("ax: unsupported order"); return SEM_EINVAL;
  }
}

int ax_dispatch_tc(Handle& h, const float* u, float* w, sem_precision p) {
  if (p == SEM_MIXED_TF32) return tc_dispatch<kTcTF32>(h, u, w);
  return tc_dispatch<kTcBF16x3>(h, u, w);
}

}  // namespace sem
