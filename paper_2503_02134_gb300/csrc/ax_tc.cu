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
// run on CUDA cores from shared memory.  Small orders put several elements
// in one block so every warp has row tiles to work on.
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

// Tensor-core shape of a block: EPB elements share the block, so one
// contraction is an (EPB n^2 x n) by (n x n) product; every element uses the
// same D, whose B fragments a warp loads once per kernel.
template <int n, int MODE>
struct TcShape {
  static constexpr int n2 = n * n, n3 = n * n * n;
  static constexpr int KSTEP = MODE == kTcTF32 ? 8 : 16;
  static constexpr int NP = ((n + KSTEP - 1) / KSTEP) * KSTEP;   // padded contraction length
  static constexpr int NT = (n + 7) / 8;                          // 8-wide output tiles
  static constexpr int EPB = n2 >= 128 ? 1 : (n2 >= 64 ? 2 : (n2 >= 32 ? 4 : 8));
  static constexpr int ROWS = EPB * n2;
  static constexpr int MT = (ROWS + 15) / 16;
};

// B fragments of M^T (M = D, or D^T when transposeD) for every (output tile,
// k-step): TF32 2 registers, BF16 split 2 (hi) + 2 (lo) registers each.
template <int n, int MODE, bool transposeD>
struct TcB {
  using S = TcShape<n, MODE>;
  static constexpr int KS = S::NP / S::KSTEP;
  uint32_t hi[S::NT][KS][2];
  uint32_t lo[S::NT][KS][2];
  __device__ void load(const float* __restrict__ Dm) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    auto B = [&](int l, int o) -> float {   // B[l][o] = M[o][l]
      if (l >= n || o >= n) return 0.f;
      return transposeD ? Dm[l * n + o] : Dm[o * n + l];
    };
#pragma unroll
    for (int nt = 0; nt < S::NT; ++nt)
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int k0 = ks * S::KSTEP, o = nt * 8 + g;
        if (MODE == kTcTF32) {
          hi[nt][ks][0] = to_tf32(B(k0 + t, o));
          hi[nt][ks][1] = to_tf32(B(k0 + t + 4, o));
        } else {
          float bv[4] = {B(k0 + 2 * t, o), B(k0 + 2 * t + 1, o), B(k0 + 2 * t + 8, o),
                         B(k0 + 2 * t + 9, o)};
          float bh[4], bl[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) split_bf16(bv[q], bh[q], bl[q]);
          hi[nt][ks][0] = pack_bf16(bh[0], bh[1]);
          hi[nt][ks][1] = pack_bf16(bh[2], bh[3]);
          lo[nt][ks][0] = pack_bf16(bl[0], bl[1]);
          lo[nt][ks][1] = pack_bf16(bl[2], bl[3]);
        }
      }
  }
};

// One contraction for the block's EPB elements:
//   out(e, p, q, o) (+)= sum_l src[e*n3 + p*sp + q*sq + l*sl] * M[o][l]
// rows r = e*n^2 + p*n + q of the (EPB n^2 x n) product; the result goes to
// dst[e*n3 + p*dp + q*dq + o*do_] (ACC: +=, each entry written by one lane).
template <int n, int MODE, bool transposeD, bool ACC>
__device__ __forceinline__ void tc_contract(const float* __restrict__ src, int sp, int sq, int sl,
                                            const TcB<n, MODE, transposeD>& Bf,
                                            float* __restrict__ dst, int dp, int dq, int do_) {
  using S = TcShape<n, MODE>;
  constexpr int KS = S::NP / S::KSTEP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int mt = warp; mt < S::MT; mt += nwarps) {
    // the two rows this lane touches in A and C: r0 + g and r0 + g + 8
    int abase[2], cbase[2];
    bool rok[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = mt * 16 + g + 8 * h;
      rok[h] = r < S::ROWS;
      const int rr = rok[h] ? r : 0;
      const int e = rr / S::n2, pq = rr % S::n2, p = pq / n, q = pq % n;
      abase[h] = e * S::n3 + p * sp + q * sq;
      cbase[h] = e * S::n3 + p * dp + q * dq;
    }
    auto A = [&](int h, int l) -> float {
      return (rok[h] && l < n) ? src[abase[h] + l * sl] : 0.f;
    };
    float c[S::NT][4];
#pragma unroll
    for (int nt = 0; nt < S::NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * S::KSTEP;
      if (MODE == kTcTF32) {
        uint32_t a[4];
        a[0] = to_tf32(A(0, k0 + t));
        a[1] = to_tf32(A(1, k0 + t));
        a[2] = to_tf32(A(0, k0 + t + 4));
        a[3] = to_tf32(A(1, k0 + t + 4));
#pragma unroll
        for (int nt = 0; nt < S::NT; ++nt) mma_tf32(c[nt], a, Bf.hi[nt][ks]);
      } else {
        const float av[8] = {A(0, k0 + 2 * t), A(0, k0 + 2 * t + 1), A(1, k0 + 2 * t),
                             A(1, k0 + 2 * t + 1), A(0, k0 + 2 * t + 8), A(0, k0 + 2 * t + 9),
                             A(1, k0 + 2 * t + 8), A(1, k0 + 2 * t + 9)};
        float ah[8], al[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16(av[q], ah[q], al[q]);
        uint32_t aH[4], aL[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          aH[q] = pack_bf16(ah[2 * q], ah[2 * q + 1]);
          aL[q] = pack_bf16(al[2 * q], al[2 * q + 1]);
        }
#pragma unroll
        for (int nt = 0; nt < S::NT; ++nt) {
          mma_bf16(c[nt], aL, Bf.hi[nt][ks]);   // small terms first
          mma_bf16(c[nt], aH, Bf.lo[nt][ks]);
          mma_bf16(c[nt], aH, Bf.hi[nt][ks]);
        }
      }
    }
    // C fragment: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
#pragma unroll
    for (int nt = 0; nt < S::NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int h = q >> 1;
        const int o = nt * 8 + 2 * t + (q & 1);
        if (rok[h] && o < n) {
          float* d = dst + cbase[h] + o * do_;
          if (ACC) *d += c[nt][q]; else *d = c[nt][q];
        }
      }
  }
}

template <int n, int MODE>
__global__ void __launch_bounds__(256)
    ax_tc_kernel(const float* __restrict__ uin, float* __restrict__ wout,
                 const float* __restrict__ G, const float* __restrict__ Dg,
                 const uint8_t* __restrict__ faces, int64_t E) {
  using S = TcShape<n, MODE>;
  constexpr int n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) float sm[];
  float* su = sm;                // u, later w        (EPB n^3 each)
  float* sr = su + EPB * n3;     // u_r, later v_r
  float* ss = sr + EPB * n3;     // u_s, later v_s
  float* st = ss + EPB * n3;     // u_t, later v_t
  TcB<n, MODE, false> Bd;        // fragments of D^T (forward) and D (transposed)
  TcB<n, MODE, true> BdT;
  Bd.load(Dg);
  BdT.load(Dg);
  for (int64_t e0 = (int64_t)blockIdx.x * EPB; e0 < E; e0 += (int64_t)gridDim.x * EPB) {
    const int cnt = (int)(E - e0 < EPB ? E - e0 : EPB);
    __syncthreads();
    for (int q = threadIdx.x; q < EPB * n3; q += blockDim.x)
      su[q] = q < cnt * n3 ? uin[e0 * n3 + q] : 0.f;
    __syncthreads();
    tc_contract<n, MODE, false, false>(su, n2, n, 1, Bd, sr, n2, n, 1);
    tc_contract<n, MODE, false, false>(su, n2, 1, n, Bd, ss, n2, 1, n);
    tc_contract<n, MODE, false, false>(su, n, 1, n2, Bd, st, n, 1, n2);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * n3; q += blockDim.x) {
      const int le = q / n3, node = q - le * n3;
      const float* Ge = G + (e0 + le) * 6 * n3 + node;
      const float ur = sr[q], us = ss[q], ut = st[q];
      const float g0 = Ge[0], g1 = Ge[n3], g2 = Ge[2 * n3];
      const float g3 = Ge[3 * n3], g4 = Ge[4 * n3], g5 = Ge[5 * n3];
      sr[q] = g0 * ur + g3 * us + g4 * ut;
      ss[q] = g3 * ur + g1 * us + g5 * ut;
      st[q] = g4 * ur + g5 * us + g2 * ut;
    }
    __syncthreads();
    // w = D_r^T v_r + D_s^T v_s + D_t^T v_t, accumulated in su in three passes
    tc_contract<n, MODE, true, false>(sr, n2, n, 1, BdT, su, n2, n, 1);
    __syncthreads();
    tc_contract<n, MODE, true, true>(ss, n2, 1, n, BdT, su, n2, 1, n);
    __syncthreads();
    tc_contract<n, MODE, true, true>(st, n, 1, n2, BdT, su, n, 1, n2);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * n3; q += blockDim.x) {
      const int le = q / n3, node = q - le * n3;
      const int i = node % n, j = (node / n) % n, k = node / n2;
      wout[e0 * n3 + q] = on_dirichlet(faces[e0 + le], i, j, k, n - 1) ? 0.f : su[q];
    }
  }
}

template <int n, int MODE>
static int tc_launch(Handle& h, const float* u, float* w) {
  auto kern = ax_tc_kernel<n, MODE>;
  const size_t smem = sizeof(float) * 4 * TcShape<n, MODE>::EPB * n * n * n;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
  const int64_t cap = (int64_t)h.num_sms * (per_sm > 0 ? per_sm : 1);
  const int64_t groups = (h.E + TcShape<n, MODE>::EPB - 1) / TcShape<n, MODE>::EPB;
  const int grid = (int)(groups < cap ? groups : cap);
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
