// The matrix-free SEM element operator (arXiv 2503.02134, Sec. 3.1: `ax`,
// i.e. local_grad3 -> geometric factors -> local_grad3_t, with the mxm
// contractions of the derivative matrix D):
//
//   u_r = (I x I x D) u,  u_s = (I x D x I) u,  u_t = (D x I x I) u
//   v_a = sum_b G_ab u_b                    (G symmetric, 6 factors per node)
//   w   = D_r^T v_r + D_s^T v_s + D_t^T v_t, then the Dirichlet mask.
//
// Thread layout: a block holds EPB elements; inside an element a thread owns
// the column (i, j) and keeps the n values along t in registers, so the
// t-contractions need no shared memory; u, v_r and v_s go through shared
// memory for the r and s contractions.  The kernel is persistent: blocks
// stride over elements.  G streams through registers with coalesced loads
// (per k-plane the n*n threads of an element read n*n consecutive values).
//
// PCG mode fuses the preconditioner and add2s1 into the prologue
// (p = J^{-1} r + beta p, written back) and the pap dot product into the
// epilogue: for a continuous, masked p, sum_l p_l (A_L p)_l over the
// unassembled result equals <p, c, QQ^T A_L p>, so pap needs no extra pass.
#pragma once

#include "reduce.cuh"

namespace sem {

// D by value (row-major D[i][l] at d[i * n + l]).  As a kernel parameter it
// lives in the constant bank; indexed only by unrolled loop counters, its
// entries are immediate operands of the FMAs (no shared-memory load).
template <int n, typename T = float>
struct DMat {
  T d[n * n];
};

template <int n>
struct AxShape {
  static constexpr int n2 = n * n;
  static constexpr int n3 = n * n * n;
  static constexpr int EPB = (256 / n2) > 0 ? (256 / n2) : 1;
  static constexpr int NT = ((n2 * EPB + 31) / 32) * 32;
};

__device__ __forceinline__ bool on_dirichlet(uint8_t f, int i, int j, int k, int N) {
  return (i == 0 && (f & 1)) || (i == N && (f & 2)) || (j == 0 && (f & 4)) ||
         (j == N && (f & 8)) || (k == 0 && (f & 16)) || (k == N && (f & 32));
}

template <int n, typename T, bool PCG, int DM>
__global__ void __launch_bounds__(AxShape<n>::NT)
    ax_kernel(const T* __restrict__ uin, T* __restrict__ wout, const T* __restrict__ G,
              const T* __restrict__ Dg, const __grid_constant__ DMat<n, T> Dc,
              const uint8_t* __restrict__ faces, int64_t E,
              const T* __restrict__ rr, const T* __restrict__ minv, T* __restrict__ pp,
              PcgScalars* __restrict__ scal, double* __restrict__ partials) {
  using S = AxShape<n>;
  constexpr int n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  // rows/columns of D live in registers while they fit (FP32, or FP64 up to n = 8)
  constexpr bool kRegD = sizeof(T) * n <= 64;
  __shared__ T sD[n][n + 1];
  __shared__ double sh_red[S::NT / 32];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* const su = reinterpret_cast<T*>(dyn_smem);
  T* const sr = su + EPB * n3;
  T* const ss = sr + EPB * n3;

  if (PCG && scal->done) return;
  const T beta = PCG ? (T)scal->beta : T(0);

  const int tid = threadIdx.x;
  const int le = tid / n2;
  const int ij = tid - le * n2;
  const int i = ij % n, j = ij / n;
  const bool lane_ok = le < EPB;   // threads past EPB*n2 (warp rounding) only idle

  for (int q = tid; q < n2; q += blockDim.x) sD[q / n][q % n] = Dg[q];
  __syncthreads();
  T Di[kRegD ? n : 1], Dj[kRegD ? n : 1], DiT[kRegD ? n : 1], DjT[kRegD ? n : 1];
  if constexpr (kRegD) {
#pragma unroll
    for (int l = 0; l < n; ++l) {
      Di[l] = lane_ok ? sD[i][l] : T(0);
      Dj[l] = lane_ok ? sD[j][l] : T(0);
      DiT[l] = lane_ok ? sD[l][i] : T(0);
      DjT[l] = lane_ok ? sD[l][j] : T(0);
    }
  }
  const int ir = lane_ok ? i : 0, jr = lane_ok ? j : 0;
  auto d_i = [&](int l) -> T { if constexpr (kRegD) return Di[l]; else return sD[ir][l]; };
  auto d_j = [&](int l) -> T { if constexpr (kRegD) return Dj[l]; else return sD[jr][l]; };
  auto dT_i = [&](int l) -> T { if constexpr (kRegD) return DiT[l]; else return sD[l][ir]; };
  auto dT_j = [&](int l) -> T { if constexpr (kRegD) return DjT[l]; else return sD[l][jr]; };

  DotAcc<T, DM> acc;
  T* const su_e = su + (lane_ok ? le : 0) * n3;
  T* const sr_e = sr + (lane_ok ? le : 0) * n3;
  T* const ss_e = ss + (lane_ok ? le : 0) * n3;

  for (int64_t e0 = (int64_t)blockIdx.x * EPB; e0 < E; e0 += (int64_t)gridDim.x * EPB) {
    const int64_t e = e0 + le;
    const bool act = lane_ok && e < E;
    const int64_t base = e * n3 + ij;
    T ureg[n];
#pragma unroll
    for (int k = 0; k < n; ++k) {
      T v = T(0);
      if (act) {
        const int64_t idx = base + k * n2;
        if (PCG) {
          v = minv[idx] * rr[idx] + beta * pp[idx];
          pp[idx] = v;
        } else {
          v = uin[idx];
        }
      }
      ureg[k] = v;
      if (lane_ok) su_e[k * n2 + ij] = v;
    }
    __syncthreads();

    T wreg[n];
#pragma unroll
    for (int k = 0; k < n; ++k) wreg[k] = T(0);
    const T* Ge = G + (act ? e : 0) * 6 * n3 + ij;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        ur += d_i(l) * su_e[k * n2 + jr * n + l];
        us += d_j(l) * su_e[k * n2 + l * n + ir];
        // FP32: D from the constant bank; FP64 (DFMA-bound) measured faster from shared memory
        if constexpr (sizeof(T) == 4) ut += Dc.d[k * n + l] * ureg[l];
        else ut += sD[k][l] * ureg[l];
      }
      T g0 = T(0), g1 = T(0), g2 = T(0), g3 = T(0), g4 = T(0), g5 = T(0);
      if (act) {
        g0 = Ge[0 * n3 + k * n2];
        g1 = Ge[1 * n3 + k * n2];
        g2 = Ge[2 * n3 + k * n2];
        g3 = Ge[3 * n3 + k * n2];
        g4 = Ge[4 * n3 + k * n2];
        g5 = Ge[5 * n3 + k * n2];
      }
      const T vr = g0 * ur + g3 * us + g4 * ut;
      const T vs = g3 * ur + g1 * us + g5 * ut;
      const T vt = g4 * ur + g5 * us + g2 * ut;
      if (lane_ok) {
        sr_e[k * n2 + ij] = vr;
        ss_e[k * n2 + ij] = vs;
      }
#pragma unroll
      for (int kk = 0; kk < n; ++kk) {
        if constexpr (sizeof(T) == 4) wreg[kk] += Dc.d[k * n + kk] * vt;
        else wreg[kk] += sD[k][kk] * vt;
      }
    }
    __syncthreads();

    const uint8_t f = act ? faces[e] : uint8_t(0);
#pragma unroll
    for (int k = 0; k < n; ++k) {
      T wv = wreg[k];
#pragma unroll
      for (int l = 0; l < n; ++l) {
        wv += dT_i(l) * sr_e[k * n2 + jr * n + l];
        wv += dT_j(l) * ss_e[k * n2 + l * n + ir];
      }
      if (on_dirichlet(f, i, j, k, n - 1)) wv = T(0);
      if (act) {
        wout[base + k * n2] = wv;
        if (PCG) acc.add(ureg[k], wv);
      }
    }
    __syncthreads();
  }

  if (PCG) {
    const double part = block_sum<DM>(acc.value(), sh_red);
    const double vals[1] = {part};
    if (publish_and_elect(vals, 1, partials, &scal->counter[0])) {
      const double pap = reduce_partials<DM>(partials, 0, sh_red);
      if (threadIdx.x == 0) {
        scal->pap = pap;
        if (!(pap > 0.0) || !isfinite(pap)) {
          scal->status = SEM_BREAKDOWN;
          scal->done = 1;
          scal->alpha = 0.0;
        } else {
          scal->alpha = scal->rtz / pap;
        }
        scal->counter[0] = 0u;
      }
    }
  }
}

// Host-side dispatch helpers (defined in ax_fp64.cu / ax_fp32.cu).
int ax_dispatch_fp64(Handle& h, const double* u, double* w, const AxPrologue* pro);
int ax_dispatch_fp32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm);

template <int n, typename T, bool PCG, int DM>
int ax_launch(Handle& h, const T* u, T* w, const T* G, const T* D, const AxPrologue* pro) {
  using S = AxShape<n>;
  auto kern = ax_kernel<n, T, PCG, DM>;
  const size_t smem = sizeof(T) * 3 * S::EPB * S::n3;
  // opt in above the 48 KB default (static shared memory comes on top of this)
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::NT, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t blocks_needed = (h.E + S::EPB - 1) / S::EPB;
  int64_t cap = (int64_t)h.num_sms * per_sm;
  int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
  if (grid > h.max_blocks) grid = h.max_blocks;
  if (grid < 1) grid = 1;
  const T* r = PCG ? (const T*)pro->r : nullptr;
  const T* minv = PCG ? (const T*)pro->minv : nullptr;
  PcgScalars* scal = PCG ? const_cast<PcgScalars*>(pro->scal) : nullptr;
  double* partials = PCG ? pro->pap_partials : nullptr;
  T* pp = PCG ? const_cast<T*>(u) : nullptr;
  DMat<n, T> Dc;
  for (int q = 0; q < n * n; ++q)
    Dc.d[q] = sizeof(T) == sizeof(double) ? (T)h.D64_host[q] : (T)h.D32_host[q];
  kern<<<grid, S::NT, smem, h.stream>>>(u, w, G, D, Dc, h.bfaces, h.E, r, minv, pp, scal,
                                        partials);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace sem
