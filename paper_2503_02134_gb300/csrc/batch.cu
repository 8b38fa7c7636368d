// Many independent SEM Poisson problems (uneven E and N) solved together:
// every phase of a PCG iteration is ONE persistent launch over a work list
// that spans all problems, and chunks of iterations are replayed as a CUDA
// graph.  The per-iteration arithmetic is that of the single-problem mixed
// path (the paper's CG loop, Sec. 3.1; FP32 operator with FP64-quality
// gather-scatter sums and dots, Sec. 3.3 and 4.3): the batched operator
// kernel runs the same element computation as ax_tma_kernel for whichever
// order the item's problem has, the gather-scatter and update kernels run
// the single-problem code per chunk / per item.  Reductions are per problem
// (one partial per work item, summed in item order by a per-problem
// finaliser launched after each phase), so each problem's result does not
// depend on the batch it is in.
#include <stdlib.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ax_tma.cuh"
#include "gs_sum.cuh"
#include "pcg.cuh"

namespace sem {

int launch_gs(Handle& h, sem_precision p, void* v);

struct BatchProb {
  float* r;
  const float* minv;
  float* p;
  float* w;
  float* x;
  const float* G;
  const float* D;
  const uint8_t* faces;
  const uint8_t* cw;
  const int* slots;
  PcgScalars* scal;
  double* ax_part;   // one partial per element group
  double* up_part;   // two partials per update item
  int64_t E, L;
  int64_t kx, kxky;   // box strides of the element index (fused summation)
  int n, epb, ngroups, nupd;
  int fuse;           // 1: QQ^T folded into the update (box mesh), 0: separate pass
};

constexpr int kUpdItem4 = 1024;           // float4 per update work item (4096 values)
constexpr int kBatchOrders = 5;           // n = 2, 4, 6, 8, 10 (odd N <= 9)
constexpr int kBatchVariants = 4;         // launch variants 0..3 of the staged operator shape
inline int order_slot(int n) { return n / 2 - 1; }

// Batched operator for the problems of one order n: the PCG-mode element
// computation of ax_tma_kernel (same arithmetic, same launch shape TmaShape
// <n, V>), applied to a work list of (problem, element group) items.  Every
// block owns one contiguous range of the list; the bulk copies of the next
// NS items are in flight while the block computes.  Each item stores its
// partial of pap = sum p (A_L p); batch_finalize_pap sums them per problem.
// Orders whose batched operator takes the whole-line contractions: n >= 10
// (at n = 6 and 8 the per-node form measured faster in the batch, 3.54
// against 3.61 s for the 64-problem solve, while the single-problem
// operator gains from the lines there).
template <int n>
constexpr bool batch_sline() {
  return n >= 10;
}

template <int n, int V>
__global__ void __launch_bounds__(TmaShape<n, V>::NT)
    batch_ax_kernel(const BatchProb* __restrict__ probs, const int2* __restrict__ items,
                    const int* __restrict__ seg, int* __restrict__ err,
                    const __grid_constant__ DMatEO<n> Dc) {
  using S = TmaShape<n, V>;
  constexpr int n2 = S::n2, n3 = S::n3, EPB = S::EPB, NS = S::NS;
  constexpr int SV = EPB * n3;       // floats of one vector per stage
  constexpr int STAGE = 9 * SV;      // r | J^{-1} | p_old | G1..G6
  // the whole-line contractions of ax_tma_kernel, with its s-line buffer
  // after the stages
  constexpr bool kSLine = batch_sline<n>();
  constexpr int SSE = n * tma_ps<n>();
  const int off = seg[0], nitems = seg[1];
  extern __shared__ __align__(128) float smem_f[];
  float* const stage0 = smem_f;
  float* const sS = smem_f + NS * STAGE;
  uint64_t* const bar =
      reinterpret_cast<uint64_t*>(smem_f + NS * STAGE + (kSLine ? EPB * SSE : 0));
  __shared__ float sD[n][n + 1];
  __shared__ double sh_red[S::NT / 32];
  __shared__ int2 s_item[NS];   // item staged on each stage ({-1, -1} = none)
  __shared__ int s_phase[NS];   // completed barrier phases per stage
  __shared__ BatchProb sP;      // the problem of the item being computed
  __shared__ float s_beta;
  const int tid = threadIdx.x;
  const int le = tid / n2;
  const int ij = tid - le * n2;
  const int i = ij % n, j = ij / n;
  const bool lane_ok = le < EPB;
  const int ir = lane_ok ? i : 0, jr = lane_ok ? j : 0, ler = lane_ok ? le : 0;

  const int per = (nitems + gridDim.x - 1) / gridDim.x;
  const int it0 = off + blockIdx.x * per;
  const int it1 = off + min(nitems, (int)(blockIdx.x + 1) * per);

  // issuing side (thread 0): descriptor and done flag of the issuing problem
  int ip = -1;
  bool ip_done = true;
  BatchProb IP;
  auto issue = [&](int st, int it) {
    const int2 itm = items[it];
    if (itm.x != ip) {
      ip = itm.x;
      IP = probs[ip];
      ip_done = IP.scal->done != 0;
    }
    if (ip_done) {
      s_item[st] = make_int2(-1, -1);
      return;
    }
    const int64_t e0 = (int64_t)itm.y * EPB;
    const int64_t cnt = IP.E - e0 < EPB ? IP.E - e0 : EPB;
    const uint32_t vb = (uint32_t)(cnt * n3 * 4);
    float* dst = stage0 + st * STAGE;
    s_item[st] = itm;
    mbar_arrive_expect_tx(&bar[st], 9 * vb);
    bulk_load(dst, IP.r + e0 * n3, vb, &bar[st]);
    bulk_load(dst + SV, IP.minv + e0 * n3, vb, &bar[st]);
    bulk_load(dst + 2 * SV, IP.p + e0 * n3, vb, &bar[st]);
    bulk_load(dst + 3 * SV, IP.G + e0 * 6 * n3, 6 * vb, &bar[st]);
  };

  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(&bar[q], 1);
      s_phase[q] = 0;
    }
    fence_mbar_init();
    for (int q = 0; q < NS; ++q) {
      if (it0 + q < it1) issue(q, it0 + q); else s_item[q] = make_int2(-1, -1);
    }
  }
  __syncthreads();

  bool aborted = false;
  int cur_prob = -1;
  float Di[n], Dj[n], DiT[n], DjT[n];
  for (int it = it0, t = 0; it < it1; ++it, ++t) {
    const int st = t % NS;
    const int2 itm = s_item[st];
    bool ok = true;
    if (itm.x >= 0) ok = mbar_wait_bounded(&bar[st], (uint32_t)(s_phase[st] & 1));
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    const int next = it + NS;
    if (itm.x >= 0) {
      if (itm.x != cur_prob) {   // block-uniform: refresh the problem copy, D and beta
        cur_prob = itm.x;
        const int* src = reinterpret_cast<const int*>(probs + itm.x);
        for (int q = tid; q < (int)(sizeof(BatchProb) / sizeof(int)); q += blockDim.x)
          reinterpret_cast<int*>(&sP)[q] = src[q];
        __syncthreads();
        for (int q = tid; q < n2; q += blockDim.x) sD[q / n][q % n] = sP.D[q];
        if (tid == 0) s_beta = (float)sP.scal->beta;
        __syncthreads();
#pragma unroll
        for (int l = 0; l < n; ++l) {
          Di[l] = sD[ir][l];
          Dj[l] = sD[jr][l];
          DiT[l] = sD[l][ir];
          DjT[l] = sD[l][jr];
        }
      }
      const float beta = s_beta;
      float* const sb = stage0 + st * STAGE;
      float* const su_e = sb + 2 * SV + ler * n3;
      const float* const Gs = sb + 3 * SV + ler * 6 * n3 + ij;
      // transposed-contraction inputs over G1, G2 of the stage (each thread
      // reads its own entries there before writing them)
      float* const sr_e = sb + 3 * SV + ler * 6 * n3;
      float* const ss_e = sr_e + n3;
      const int64_t e = (int64_t)itm.y * EPB + le;
      const bool act = lane_ok && e < sP.E;
      const uint8_t f = act ? sP.faces[e] : uint8_t(0);
      float* const pg = sP.p;
      float* const wg = sP.w;
      DotAcc<float, kDotDot2> acc;
      float ureg[n];
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int si = k * n2 + ij;
        const float v = sb[SV + ler * n3 + si] * sb[ler * n3 + si] + beta * su_e[si];
        if (lane_ok) su_e[si] = v;
        if (act) pg[e * n3 + si] = v;
        ureg[k] = v;
      }
      __syncthreads();
      float* const sS_e = sS + ler * SSE;
      if constexpr (kSLine) {
        // s-line (i, k = j) and r-line (j = i, k = j) of this thread: u_s to
        // the s-line buffer, u_r over the row of p once all threads read p
        float a[n], y[n], yr[n];
#pragma unroll
        for (int l = 0; l < n; ++l) a[l] = su_e[jr * n2 + l * n + ir];
        eo_line<n>(Dc.E, Dc.O, a, y);
        if (lane_ok) {
#pragma unroll
          for (int jj = 0; jj < n; ++jj) sS_e[sb_at<n, false>(ir, jj, jr)] = y[jj];
        }
        load_row_lb<n, false>(su_e, ir, jr, a);
        eo_line<n>(Dc.E, Dc.O, a, yr);
        __syncthreads();
        if (lane_ok) store_row_lb<n, false>(su_e, ir, jr, yr);
        __syncthreads();
      }
      float utk[kSLine ? n : 1], vtk[kSLine ? n : 1];
      if constexpr (kSLine) eo_line<n>(Dc.E, Dc.O, ureg, utk);
      float wreg[n];
#pragma unroll
      for (int k = 0; k < n; ++k) wreg[k] = 0.f;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float ur, us, ut = 0.f;
        if constexpr (kSLine) {
          ur = su_e[k * n2 + ij];
          us = sS_e[sb_at<n, false>(i, j, k)];
          ut = utk[k];
        } else {
          ur = row_dot<n>(su_e + k * n2 + jr * n, Di);
          us = 0.f;
#pragma unroll
          for (int l = 0; l < n; ++l) {
            us += Dj[l] * su_e[k * n2 + l * n + ir];
            ut += Dc.d[k * n + l] * ureg[l];
          }
        }
        const float g0 = Gs[0 * n3 + k * n2], g1 = Gs[1 * n3 + k * n2], g2 = Gs[2 * n3 + k * n2];
        const float g3 = Gs[3 * n3 + k * n2], g4 = Gs[4 * n3 + k * n2], g5 = Gs[5 * n3 + k * n2];
        const float vr = g0 * ur + g3 * us + g4 * ut;
        const float vs = g3 * ur + g1 * us + g5 * ut;
        const float vt = g4 * ur + g5 * us + g2 * ut;
        if (lane_ok) {
          sr_e[k * n2 + ij] = vr;
          if constexpr (kSLine) sS_e[sb_at<n, false>(i, j, k)] = vs;
          else ss_e[k * n2 + ij] = vs;
        }
        if constexpr (kSLine) {
          vtk[k] = vt;
        } else {
#pragma unroll
          for (int kk = 0; kk < n; ++kk) wreg[kk] += Dc.d[k * n + kk] * vt;
        }
      }
      if constexpr (kSLine) eo_line<n>(Dc.ET, Dc.OT, vtk, wreg);
      __syncthreads();
      if constexpr (kSLine) {
        // transposed s-line and r-line products, in place
        float b[n], y[n];
#pragma unroll
        for (int l = 0; l < n; ++l) b[l] = sS_e[sb_at<n, false>(ir, l, jr)];
        eo_line<n>(Dc.ET, Dc.OT, b, y);
        if (lane_ok) {
#pragma unroll
          for (int jj = 0; jj < n; ++jj) sS_e[sb_at<n, false>(ir, jj, jr)] = y[jj];
        }
        load_row_lb<n, false>(sr_e, ir, jr, b);
        eo_line<n>(Dc.ET, Dc.OT, b, y);
        if (lane_ok) store_row_lb<n, false>(sr_e, ir, jr, y);
        __syncthreads();
      }
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float wv;
        if constexpr (kSLine) {
          wv = wreg[k] + (sr_e[k * n2 + ij] + sS_e[sb_at<n, false>(i, j, k)]);
        } else {
          wv = wreg[k] + row_dot<n>(sr_e + k * n2 + jr * n, DiT);
#pragma unroll
          for (int l = 0; l < n; ++l) wv += DjT[l] * ss_e[k * n2 + l * n + ir];
        }
        if (on_dirichlet(f, i, j, k, n - 1)) wv = 0.f;
        if (act) {
          wg[e * n3 + k * n2 + ij] = wv;
          acc.add(ureg[k], wv);
        }
      }
      // the reduction's barriers guarantee the stage is no longer read
      const double part = block_sum<kDotDot2>(acc.value(), sh_red);
      if (tid == 0) {
        sP.ax_part[itm.y] = part;
        ++s_phase[st];
        if (next < it1) {
          fence_proxy_async_smem();
          issue(st, next);
        } else {
          s_item[st] = make_int2(-1, -1);
        }
      }
      __syncthreads();
    } else {
      if (tid == 0) {
        if (next < it1) issue(st, next); else s_item[st] = make_int2(-1, -1);
      }
      __syncthreads();
    }
  }
  if (aborted && tid == 0) {
    atomicExch(err, 1);
    for (int q = 0; q < NS; ++q)
      if (s_item[q].x >= 0) mbar_wait_bounded(&bar[q], (uint32_t)(s_phase[q] & 1));
  }
}

template <int n, int V>
constexpr size_t batch_smem_bytes() {
  using S = TmaShape<n, V>;
  return sizeof(float) * (size_t)S::NS * 9 * S::EPB * S::n3 +
         (batch_sline<n>() ? sizeof(float) * (size_t)S::EPB * n * tma_ps<n>() : 0) +
         S::NS * sizeof(uint64_t);
}

// D of order n as the kernel parameter (the full matrix and its even-odd
// halves), from the host copy of any problem of that order (D depends on N
// only).
template <int n>
static DMatEO<n> batch_dmat(const float* D32h, const double* D64h) {
  DMatEO<n> Dc;
  for (int q = 0; q < n * n; ++q) Dc.d[q] = D32h[q];
  constexpr int hh = n / 2;
  for (int a = 0; a < hh; ++a)
    for (int l = 0; l < hh; ++l) {
      const double* D = D64h;
      Dc.E[a * hh + l] = (float)(0.5 * (D[a * n + l] + D[a * n + (n - 1 - l)]));
      Dc.O[a * hh + l] = (float)(0.5 * (D[a * n + l] - D[a * n + (n - 1 - l)]));
      Dc.ET[a * hh + l] = (float)(0.5 * (D[l * n + a] + D[(n - 1 - l) * n + a]));
      Dc.OT[a * hh + l] = (float)(0.5 * (D[l * n + a] - D[(n - 1 - l) * n + a]));
    }
  return Dc;
}

template <int n, int V>
int batch_ax_launch(cudaStream_t st, int grid, const BatchProb* probs, const int2* items,
                    const int* seg, int* err, const float* D32h, const double* D64h) {
  auto kern = batch_ax_kernel<n, V>;
  constexpr size_t smem = batch_smem_bytes<n, V>();
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, TmaShape<n, V>::NT, smem, st>>>(probs, items, seg, err,
                                               batch_dmat<n>(D32h, D64h));
  SEM_CUDA(cudaGetLastError());
  return 0;
}

template <int n, int V>
int batch_ax_occupancy(int* per_sm) {
  auto kern = batch_ax_kernel<n, V>;
  constexpr size_t smem = batch_smem_bytes<n, V>();
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, TmaShape<n, V>::NT, smem));
  return 0;
}

template <int n>
int batch_ax_dispatch(int V, cudaStream_t st, int grid, const BatchProb* probs, const int2* items,
                      const int* seg, int* err, const float* D32h, const double* D64h) {
  switch (V) {
    case 1: return batch_ax_launch<n, 1>(st, grid, probs, items, seg, err, D32h, D64h);
    case 2: return batch_ax_launch<n, 2>(st, grid, probs, items, seg, err, D32h, D64h);
    case 3: return batch_ax_launch<n, 3>(st, grid, probs, items, seg, err, D32h, D64h);
    default: return batch_ax_launch<n, 0>(st, grid, probs, items, seg, err, D32h, D64h);
  }
}

int batch_ax_any(int n, int V, cudaStream_t st, int grid, const BatchProb* probs,
                 const int2* items, const int* seg, int* err, const float* D32h,
                 const double* D64h) {
  switch (n) {
    case 2: return batch_ax_dispatch<2>(V, st, grid, probs, items, seg, err, D32h, D64h);
    case 4: return batch_ax_dispatch<4>(V, st, grid, probs, items, seg, err, D32h, D64h);
    case 6: return batch_ax_dispatch<6>(V, st, grid, probs, items, seg, err, D32h, D64h);
    case 8: return batch_ax_dispatch<8>(V, st, grid, probs, items, seg, err, D32h, D64h);
    default: return batch_ax_dispatch<10>(V, st, grid, probs, items, seg, err, D32h, D64h);
  }
}

int batch_ax_occupancy_any(int n, int V, int* per_sm) {
#define SEM_OCC(NN)                                              \
  if (n == NN) {                                                 \
    if (V == 1) return batch_ax_occupancy<NN, 1>(per_sm);        \
    if (V == 2) return batch_ax_occupancy<NN, 2>(per_sm);        \
    if (V == 3) return batch_ax_occupancy<NN, 3>(per_sm);        \
    return batch_ax_occupancy<NN, 0>(per_sm);                    \
  }
  SEM_OCC(2) SEM_OCC(4) SEM_OCC(6) SEM_OCC(8) SEM_OCC(10)
#undef SEM_OCC
  return SEM_EINVAL;
}

int batch_epb_of(int n, int V) {
  switch (n) {
    case 2: return V == 0 ? TmaShape<2, 0>::EPB : TmaShape<2, 1>::EPB;
    case 4: return V == 0 ? TmaShape<4, 0>::EPB : TmaShape<4, 1>::EPB;
    case 6: return V == 0 ? TmaShape<6, 0>::EPB : TmaShape<6, 1>::EPB;
    case 8: return V == 0 ? TmaShape<8, 0>::EPB : TmaShape<8, 1>::EPB;
    default: return V == 0 ? TmaShape<10, 0>::EPB : TmaShape<10, 1>::EPB;
  }
}

// Gather-scatter of every problem's chunks (same arithmetic as
// gs_bucket_kernel with error-free TwoSum accumulation).
__global__ void __launch_bounds__(256)
    batch_gs_kernel(const BatchProb* __restrict__ probs, const int* __restrict__ chunk_prob,
                    const int2* __restrict__ chunk_desc, const int* __restrict__ nchunks_dev) {
  const int64_t nchunks = *nchunks_dev;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
       c += nwarps) {
    const BatchProb& P = probs[__ldg(chunk_prob + c)];
    if (P.scal->done) continue;
    const int2 d = __ldg(chunk_desc + c);
    const int m = d.x;
    const int* sl = P.slots + d.y + lane;
    float* v = P.w;
    float s = 0.f, cc = 0.f;
    for (int q = 0; q < m; ++q) {
      const int id = __ldg(sl + 32 * q);
      if (id >= 0) {
        const float x = v[id];
        const float t = __fadd_rn(s, x);
        const float z = __fsub_rn(t, s);
        cc = __fadd_rn(cc, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
        s = t;
      }
    }
    const float out = __fadd_rn(s, cc);
    for (int q = 0; q < m; ++q) {
      const int id = __ldg(sl + 32 * q);
      if (id >= 0) v[id] = out;
    }
  }
}

__device__ __forceinline__ float batch_weight(uint8_t m) { return m ? __frcp_rn((float)m) : 0.f; }

// QQ^T w at float4 group q of a box-mesh problem with n = 8, gathered from
// the copies' positions (the separate pass's order and TwoSum accumulation).
__device__ __forceinline__ float4 batch_gather(const BatchProb& P, int64_t q) {
  return gs_gather_row4<8, kGsTwoSum>(P.w, q, P.faces, P.kx, P.kxky);
}

// add2s2 x 2 + glsc3(r,c,r) + glsc3(r,c,z) for one range of every problem
// (for box-mesh problems with the summation QQ^T folded in).
template <bool FUSED>
__global__ void __launch_bounds__(256, 4)
    batch_update_kernel(const BatchProb* __restrict__ probs, const int2* __restrict__ uitems,
                        const int* __restrict__ nuitems_dev) {
  const int nuitems = *nuitems_dev;
  __shared__ double sh[8];
  for (int ui = blockIdx.x; ui < nuitems; ui += gridDim.x) {
    const int2 itm = uitems[ui];
    const BatchProb& P = probs[itm.x];
    // uniform for the block: finished problems, and problems the other
    // instantiation handles (the fused gather needs twice the registers)
    if (P.scal->done || (P.fuse != 0) != FUSED) continue;
    const float alpha = (float)P.scal->alpha;
    const int64_t n4 = P.L >> 2;
    const int64_t q0 = (int64_t)itm.y * kUpdItem4;
    const int64_t q1 = q0 + kUpdItem4 < n4 ? q0 + kUpdItem4 : n4;
    DotAcc<float, kDotDot2> a_rr, a_rz;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      float4 xv = reinterpret_cast<float4*>(P.x)[q];
      float4 rv = reinterpret_cast<float4*>(P.r)[q];
      const float4 pv = reinterpret_cast<const float4*>(P.p)[q];
      const float4 wv = FUSED ? batch_gather(P, q) : reinterpret_cast<const float4*>(P.w)[q];
      const float4 mv = __ldg(reinterpret_cast<const float4*>(P.minv) + q);
      const uchar4 cv = __ldg(reinterpret_cast<const uchar4*>(P.cw) + q);
      xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
      rv.x -= alpha * wv.x; rv.y -= alpha * wv.y; rv.z -= alpha * wv.z; rv.w -= alpha * wv.w;
      reinterpret_cast<float4*>(P.x)[q] = xv;
      reinterpret_cast<float4*>(P.r)[q] = rv;
      float c;
      c = batch_weight(cv.x) * rv.x; a_rr.add(c, rv.x); a_rz.add(c, mv.x * rv.x);
      c = batch_weight(cv.y) * rv.y; a_rr.add(c, rv.y); a_rz.add(c, mv.y * rv.y);
      c = batch_weight(cv.z) * rv.z; a_rr.add(c, rv.z); a_rz.add(c, mv.z * rv.z);
      c = batch_weight(cv.w) * rv.w; a_rr.add(c, rv.w); a_rz.add(c, mv.w * rv.w);
    }
    const double v0 = block_sum<kDotDot2>(a_rr.value(), sh);
    const double v1 = block_sum<kDotDot2>(a_rz.value(), sh);
    if (threadIdx.x == 0) {
      P.up_part[2 * itm.y] = v0;
      P.up_part[2 * itm.y + 1] = v1;
    }
  }
}

// One block per problem: pap = sum of the operator's item partials (item
// order), alpha = rtz / pap (or the breakdown flag).  Runs after the
// operator launch, so no partial needs a fence or an election.
__global__ void __launch_bounds__(256)
    batch_finalize_pap(const BatchProb* __restrict__ probs, int count) {
  __shared__ double sh[8];
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const BatchProb& P = probs[p];
    if (P.scal->done) continue;
    double s = 0.0;
    for (int b = threadIdx.x; b < P.ngroups; b += blockDim.x) s += P.ax_part[b];
    const double pap = block_sum<kDotDot2>(s, sh);
    if (threadIdx.x == 0) {
      P.scal->pap = pap;
      if (!(pap > 0.0) || !isfinite(pap)) {
        P.scal->status = SEM_BREAKDOWN;   // the update finaliser ends this problem
        P.scal->alpha = 0.0;
      } else {
        P.scal->alpha = P.scal->rtz / pap;
      }
    }
    __syncthreads();
  }
}

// One block per problem: rtr, rtz from the update's item partials, then the
// convergence test and the scalar recurrences of the iteration.
__global__ void __launch_bounds__(256)
    batch_finalize_update(const BatchProb* __restrict__ probs, int count) {
  __shared__ double sh[8];
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const BatchProb& P = probs[p];
    if (P.scal->done) continue;
    double a = 0.0, c = 0.0;
    for (int q = threadIdx.x; q < P.nupd; q += blockDim.x) {
      a += P.up_part[2 * q];
      c += P.up_part[2 * q + 1];
    }
    const double rtr = block_sum<kDotDot2>(a, sh);
    const double rtz = block_sum<kDotDot2>(c, sh);
    if (threadIdx.x == 0) {
      if (P.scal->status == SEM_BREAKDOWN)
        P.scal->done = 1;
      else
        finish_iteration(P.scal, rtr, rtz, nullptr);
    }
    __syncthreads();
  }
}

__global__ void batch_gather_scalars(const BatchProb* probs, int count, PcgScalars* out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < count; p += gridDim.x * blockDim.x)
    out[p] = *probs[p].scal;
}

}  // namespace sem

// ------------------------------------------------------------------ host side
struct sem_batch_s {
  std::vector<sem_handle_s*> subs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int count = 0;
  sem::BatchProb* d_probs = nullptr;
  int2* d_items = nullptr;
  int nitems = 0;
  int* d_chunk_prob = nullptr;
  int2* d_chunk_desc = nullptr;
  int64_t nchunks = 0;
  int fused = 0;             // problems whose summation is folded into the update
  int2* d_uitems = nullptr;
  int nuitems = 0;
  double* d_part = nullptr;
  int* d_counts = nullptr;   // per order q: {offset, count} at [2q], then gs chunks, update items
  int* h_counts = nullptr;   // pinned staging of the above
  int2* h_items = nullptr;   // pinned staging of the compacted lists
  int2* h_uitems = nullptr;
  int* h_chunk_prob = nullptr;
  int2* h_chunk_desc = nullptr;
  std::vector<std::vector<int2>> items_of, uitems_of, chunks_of;   // per problem
  sem::PcgScalars* d_scal_all = nullptr;
  sem::PcgScalars* h_scal_all = nullptr;
  int* d_err = nullptr;
  // per order slot q (n = 2q + 2): present, autotuned launch variant and grid
  bool present[sem::kBatchOrders] = {};
  int first_of[sem::kBatchOrders] = {};   // a problem of each order (its D is the order's D)
  int variant[sem::kBatchOrders] = {};
  int grid[sem::kBatchOrders] = {};
  float tune_ms[sem::kBatchOrders][sem::kBatchVariants] = {};
  std::vector<sem::BatchProb> probs_host;
  cudaGraphExec_t graph = nullptr;
  int graph_chunk = 0;
  int64_t graph_nodes = 0;
  int64_t launches = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace sem {

static int batch_launch_ax(sem_batch_s& b) {
  for (int q = 0; q < kBatchOrders; ++q) {
    if (!b.present[q]) continue;
    const Handle& hq = *b.subs[b.first_of[q]];
    int rc = batch_ax_any(2 * q + 2, b.variant[q], b.stream, b.grid[q], b.d_probs, b.d_items,
                          b.d_counts + 2 * q, b.d_err, hq.D32_host, hq.D64_host);
    if (rc) return rc;
    ++b.launches;
  }
  return 0;
}

static int batch_enqueue_iteration(sem_batch_s& b) {
  int rc = batch_launch_ax(b);
  if (rc) return rc;
  int num_sms = b.subs[0]->num_sms;
  batch_finalize_pap<<<b.count, 256, 0, b.stream>>>(b.d_probs, b.count);
  ++b.launches;
  SEM_CUDA(cudaGetLastError());
  const int64_t gs_blocks = std::min<int64_t>((b.nchunks + 7) / 8, (int64_t)num_sms * 8);
  if (b.nchunks > 0) {
    batch_gs_kernel<<<(int)std::max<int64_t>(gs_blocks, 1), 256, 0, b.stream>>>(
        b.d_probs, b.d_chunk_prob, b.d_chunk_desc, b.d_counts + 2 * kBatchOrders);
    ++b.launches;
    SEM_CUDA(cudaGetLastError());
  }
  const int up_blocks = std::min(b.nuitems, num_sms * 8);
  if (b.fused < b.count) {
    batch_update_kernel<false><<<std::max(up_blocks, 1), 256, 0, b.stream>>>(
        b.d_probs, b.d_uitems, b.d_counts + 2 * kBatchOrders + 1);
    ++b.launches;
    SEM_CUDA(cudaGetLastError());
  }
  if (b.fused > 0) {
    batch_update_kernel<true><<<std::max(up_blocks, 1), 256, 0, b.stream>>>(
        b.d_probs, b.d_uitems, b.d_counts + 2 * kBatchOrders + 1);
    ++b.launches;
    SEM_CUDA(cudaGetLastError());
  }
  batch_finalize_update<<<b.count, 256, 0, b.stream>>>(b.d_probs, b.count);
  ++b.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

static int batch_run_chunk(sem_batch_s& b, int chunk, bool use_graph) {
  if (!use_graph) {
    for (int q = 0; q < chunk; ++q) {
      int rc = batch_enqueue_iteration(b);
      if (rc) return rc;
    }
    return 0;
  }
  if (!b.graph || b.graph_chunk != chunk) {
    if (b.graph) cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
    cudaGraph_t g = nullptr;
    const int64_t before = b.launches;
    SEM_CUDA(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int q = 0; q < chunk && !rc; ++q) rc = batch_enqueue_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b.stream, &g);
    b.graph_nodes = b.launches - before;
    b.launches = before;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b.graph_chunk = chunk;
  }
  SEM_CUDA(cudaGraphLaunch(b.graph, b.stream));
  b.launches += b.graph_nodes;
  return 0;
}

// Upload the work lists of the problems still being solved (in the same
// interleaved order as at set-up).  Kernels read the counts from device
// memory, so captured graphs stay valid.
static int batch_compact(sem_batch_s& b, const std::vector<int>& active) {
  int ni = 0, nu = 0, nc = 0;
  const int P = b.count;
  std::vector<size_t> gi(P, 0), ui(P, 0);
  // operator items: one segment per order n (each launched by its own
  // kernel), problems in order inside a segment, each block of that kernel
  // taking one contiguous range: a block rarely switches problem
  for (int q = 0; q < kBatchOrders; ++q) {
    const int start = ni;
    for (int p = 0; p < P; ++p) {
      if (!active[p] || order_slot(b.subs[p]->n) != q) continue;
      for (const int2& itm : b.items_of[p]) b.h_items[ni++] = itm;
    }
    b.h_counts[2 * q] = start;
    b.h_counts[2 * q + 1] = ni - start;
  }
  (void)gi;
  bool more = true;
  while (more) {
    more = false;
    for (int p = 0; p < P; ++p) {
      if (!active[p]) continue;
      for (int q = 0; q < 2 && ui[p] < b.uitems_of[p].size(); ++q) b.h_uitems[nu++] = b.uitems_of[p][ui[p]++];
      more = more || ui[p] < b.uitems_of[p].size();
    }
  }
  for (int p = 0; p < P; ++p) {
    if (!active[p]) continue;
    for (const int2& c : b.chunks_of[p]) {
      b.h_chunk_desc[nc] = c;
      b.h_chunk_prob[nc] = p;
      ++nc;
    }
  }
  b.h_counts[2 * kBatchOrders] = nc;
  b.h_counts[2 * kBatchOrders + 1] = nu;
  SEM_CUDA(cudaMemcpyAsync(b.d_items, b.h_items, sizeof(int2) * std::max(ni, 1),
                           cudaMemcpyHostToDevice, b.stream));
  SEM_CUDA(cudaMemcpyAsync(b.d_uitems, b.h_uitems, sizeof(int2) * std::max(nu, 1),
                           cudaMemcpyHostToDevice, b.stream));
  SEM_CUDA(cudaMemcpyAsync(b.d_chunk_desc, b.h_chunk_desc, sizeof(int2) * std::max(nc, 1),
                           cudaMemcpyHostToDevice, b.stream));
  SEM_CUDA(cudaMemcpyAsync(b.d_chunk_prob, b.h_chunk_prob, sizeof(int) * std::max(nc, 1),
                           cudaMemcpyHostToDevice, b.stream));
  SEM_CUDA(cudaMemcpyAsync(b.d_counts, b.h_counts, sizeof(int) * (2 * kBatchOrders + 2),
                           cudaMemcpyHostToDevice, b.stream));
  // the pinned staging buffers are reused: wait for the copies
  SEM_CUDA(cudaStreamSynchronize(b.stream));
  return 0;
}

static int batch_read_scalars(sem_batch_s& b) {
  batch_gather_scalars<<<(b.count + 63) / 64, 64, 0, b.stream>>>(b.d_probs, b.count, b.d_scal_all);
  ++b.launches;
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaMemcpyAsync(b.h_scal_all, b.d_scal_all, sizeof(PcgScalars) * b.count,
                           cudaMemcpyDeviceToHost, b.stream));
  SEM_CUDA(cudaStreamSynchronize(b.stream));
  return 0;
}

// Element groups of problem p at elements-per-group epb.
static void batch_set_groups(sem_batch_s& b, int p, int epb) {
  BatchProb& P = b.probs_host[p];
  P.epb = epb;
  P.ngroups = (int)((P.E + epb - 1) / epb);
  b.items_of[p].clear();
  for (int g = 0; g < P.ngroups; ++g) b.items_of[p].push_back(make_int2(p, g));
}

// Project autotuner of the batched operator: for every order present, each
// launch variant (elements per block x pipeline stages, as the
// single-problem kernel) and 1..4 blocks per SM, timed with CUDA events on
// the batch's own work list; the fastest is kept.
static int batch_autotune(sem_batch_s& b) {
  const int num_sms = b.subs[0]->num_sms;
  ScopedEvents ev;
  SEM_CUDA(ev.create());
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  for (int p = 0; p < b.count; ++p) {
    Handle& h = *b.subs[p];
    SEM_CUDA(cudaMemsetAsync(h.r32, 0x3f, sizeof(float) * h.L, b.stream));
    SEM_CUDA(cudaMemsetAsync(h.p32, 0x3f, sizeof(float) * h.L, b.stream));
    int rc = launch_scal_setup(h, h.scal, 0.0, 1, 0, 0);
    if (rc) return rc;
  }
  std::vector<int> all(b.count, 1);
  int rc = 0;
  for (int q = 0; q < kBatchOrders && !rc; ++q) {
    if (!b.present[q]) continue;
    const int n = 2 * q + 2;
    float best = 1e30f;
    for (int V = 0; V < kBatchVariants && !rc; ++V) {
      for (int p = 0; p < b.count; ++p)
        if (b.subs[p]->n == n) batch_set_groups(b, p, batch_epb_of(n, V));
      SEM_CUDA(cudaMemcpyAsync(b.d_probs, b.probs_host.data(), sizeof(BatchProb) * b.count,
                               cudaMemcpyHostToDevice, b.stream));
      if ((rc = batch_compact(b, all))) break;
      int per_sm = 0;
      if ((rc = batch_ax_occupancy_any(n, V, &per_sm))) break;
      per_sm = std::max(1, std::min(per_sm, 6));
      float best_v = 1e30f;
      for (int bps = 1; bps <= per_sm && !rc; ++bps) {
        const int grid = num_sms * bps;
        const int* seg = b.d_counts + 2 * q;
        const Handle& hq = *b.subs[b.first_of[q]];
        if ((rc = batch_ax_any(n, V, b.stream, grid, b.d_probs, b.d_items, seg, b.d_err,
                               hq.D32_host, hq.D64_host)))
          break;
        SEM_CUDA(cudaEventRecord(e0, b.stream));
        for (int r = 0; r < 2 && !rc; ++r)
          rc = batch_ax_any(n, V, b.stream, grid, b.d_probs, b.d_items, seg, b.d_err,
                            hq.D32_host, hq.D64_host);
        SEM_CUDA(cudaEventRecord(e1, b.stream));
        SEM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        SEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms *= 0.5f;
        best_v = std::min(best_v, ms);
        if (ms < best) {
          best = ms;
          b.variant[q] = V;
          b.grid[q] = grid;
        }
      }
      b.tune_ms[q][V] = best_v;
    }
    // final grouping of this order
    for (int p = 0; p < b.count; ++p)
      if (b.subs[p]->n == n) batch_set_groups(b, p, batch_epb_of(n, b.variant[q]));
  }
  if (rc) return rc;
  SEM_CUDA(cudaMemcpyAsync(b.d_probs, b.probs_host.data(), sizeof(BatchProb) * b.count,
                           cudaMemcpyHostToDevice, b.stream));
  if ((rc = batch_compact(b, all))) return rc;
  for (int p = 0; p < b.count; ++p) {
    int r2 = launch_scal_setup(*b.subs[p], b.subs[p]->scal, 0.0, 1, 0, 0);
    if (r2) return r2;
  }
  return 0;
}

static void batch_free(sem_batch_s* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto* s : b->subs) sem_destroy(s);
  void* ptrs[] = {b->d_probs, b->d_items, b->d_chunk_prob, b->d_chunk_desc, b->d_uitems,
                  b->d_part, b->d_scal_all, b->d_err, b->d_counts};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* hptrs[] = {b->h_scal_all, b->h_counts, b->h_items, b->h_uitems, b->h_chunk_prob,
                   b->h_chunk_desc};
  for (void* p : hptrs)
    if (p) cudaFreeHost(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // namespace sem

using namespace sem;

extern "C" int sem_batch_setup(const sem_mesh* meshes, const int* Ns, int count, void* stream,
                               sem_batch* out) {
  if (!meshes || !Ns || !out || count < 1) {
    set_error("sem_batch_setup: null argument or count < 1");
    return SEM_EINVAL;
  }
  *out = nullptr;
  for (int p = 0; p < count; ++p) {
    if (Ns[p] < 1 || Ns[p] > 9 || Ns[p] % 2 == 0) {
      set_error("sem_batch_setup: the batched solver takes odd N in 1..9 (even n <= 10)");
      return SEM_EINVAL;
    }
  }
  sem_batch_s* b = new sem_batch_s();
  auto fail = [&](int code) {
    batch_free(b);
    return code;
  };
  cudaError_t ce;
  if (stream == nullptr) {
    if ((ce = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(cuda_fail(ce, "cudaStreamCreate"));
    b->own_stream = true;
  } else {
    b->stream = (cudaStream_t)stream;
  }
  b->count = count;
  int rc;
  for (int p = 0; p < count; ++p) {
    sem_handle h = nullptr;
    if ((rc = sem_setup(&meshes[p], Ns[p], 0, b->stream, &h))) return fail(rc);
    b->subs.push_back(h);
  }
  // work lists
  std::vector<BatchProb> probs(count);
  std::vector<int64_t> ax_off(count), up_off(count);
  int64_t part_total = 0;
  for (int p = 0; p < count; ++p) {
    Handle& h = *b->subs[p];
    BatchProb& P = probs[p];
    P.r = h.r32;
    P.minv = h.minv32;
    P.p = h.p32;
    P.w = h.w32;
    P.x = h.x32;
    P.G = h.G32;
    P.D = h.D32;
    P.faces = h.bfaces;
    P.cw = h.cw8;
    P.slots = h.gs_slots;
    P.scal = h.scal;
    P.E = h.E;
    P.L = h.L;
    P.n = h.n;
    P.epb = 1;
    P.ngroups = (int)h.E;   // the most groups any variant makes
    P.nupd = (int)(((h.L >> 2) + kUpdItem4 - 1) / kUpdItem4);
    P.kx = h.kx;
    P.kxky = (int64_t)h.kx * h.ky;
    // folded summation for n = 8 (whole float4 rows; the batch's orders are
    // N = 5, 7, 9 and the per-node gather of other orders measured slower
    // than the separate pass)
    P.fuse = gs_fusable(h) && h.n == 8 ? 1 : 0;
    if (!b->present[order_slot(h.n)]) b->first_of[order_slot(h.n)] = p;
    b->present[order_slot(h.n)] = true;
    ax_off[p] = part_total;
    part_total += h.E;
    up_off[p] = part_total;
    part_total += 2 * (int64_t)P.nupd;
    if (!P.fuse) b->nchunks += h.n_chunks;
    b->fused += P.fuse;
  }
  // per-problem work lists (kept on the host; the active ones are uploaded
  // interleaved, so every launch spreads over all unfinished problems)
  b->items_of.resize(count);
  b->uitems_of.resize(count);
  b->chunks_of.resize(count);
  for (int p = 0; p < count; ++p) {
    Handle& h = *b->subs[p];
    for (int g = 0; g < probs[p].ngroups; ++g) b->items_of[p].push_back(make_int2(p, g));
    for (int q = 0; q < probs[p].nupd; ++q) b->uitems_of[p].push_back(make_int2(p, q));
    if (!probs[p].fuse) {   // fused problems have no separate summation pass
      b->chunks_of[p].resize((size_t)h.n_chunks);
      if (h.n_chunks > 0 &&
          (ce = cudaMemcpy(b->chunks_of[p].data(), h.gs_chunks, sizeof(int2) * h.n_chunks,
                           cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(cuda_fail(ce, "cudaMemcpy"));
    }
    b->nitems += probs[p].ngroups;
    b->nuitems += probs[p].nupd;
  }
  const size_t nit = std::max(b->nitems, 1), nut = std::max(b->nuitems, 1);
  const size_t nch = (size_t)std::max<int64_t>(b->nchunks, 1);
  if ((ce = cudaMalloc((void**)&b->d_part, sizeof(double) * std::max<int64_t>(part_total, 1))) !=
          cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_probs, sizeof(BatchProb) * count)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_items, sizeof(int2) * nit)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_uitems, sizeof(int2) * nut)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_chunk_prob, sizeof(int) * nch)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_chunk_desc, sizeof(int2) * nch)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_counts, sizeof(int) * (2 * kBatchOrders + 2))) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_scal_all, sizeof(PcgScalars) * count)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&b->d_err, sizeof(int))) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_scal_all, sizeof(PcgScalars) * count)) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_counts, sizeof(int) * (2 * kBatchOrders + 2))) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_items, sizeof(int2) * nit)) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_uitems, sizeof(int2) * nut)) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_chunk_prob, sizeof(int) * nch)) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_chunk_desc, sizeof(int2) * nch)) != cudaSuccess ||
      (ce = cudaEventCreate(&b->ev0)) != cudaSuccess || (ce = cudaEventCreate(&b->ev1)) != cudaSuccess)
    return fail(cuda_fail(ce, "sem_batch_setup"));
  for (int p = 0; p < count; ++p) {
    probs[p].ax_part = b->d_part + ax_off[p];
    probs[p].up_part = b->d_part + up_off[p];
  }
  b->probs_host = probs;
  if ((ce = cudaMemcpyAsync(b->d_probs, probs.data(), sizeof(BatchProb) * count,
                            cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (ce = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream)) != cudaSuccess)
    return fail(cuda_fail(ce, "sem_batch_setup"));
  if ((rc = batch_compact(*b, std::vector<int>(count, 1)))) return fail(rc);
  if ((rc = batch_autotune(*b))) return fail(rc);
  *out = b;
  return SEM_OK;
}

extern "C" void sem_batch_destroy(sem_batch b) { batch_free(b); }

extern "C" int sem_batch_problem(sem_batch b, int i, sem_handle* out) {
  if (!b || !out || i < 0 || i >= b->count) {
    set_error("sem_batch_problem: invalid argument");
    return SEM_EINVAL;
  }
  *out = b->subs[i];
  return SEM_OK;
}

extern "C" int sem_batch_get_option(sem_batch b, const char* key, double* value) {
  if (!b || !key || !value) {
    set_error("sem_batch_get_option: null argument");
    return SEM_EINVAL;
  }
  const std::string k(key);
  auto order_of = [&](const std::string& pre, int* q) {
    if (k.rfind(pre, 0) != 0) return false;
    const int n = std::atoi(k.c_str() + pre.size());
    if (n < 2 || n > 10 || n % 2) return false;
    *q = order_slot(n);
    return true;
  };
  int q = 0;
  if (k == "work_items") *value = b->nitems;
  else if (k == "fused_problems") *value = b->fused;
  else if (k == "launches") *value = (double)b->launches;
  else if (order_of("variant_n", &q)) *value = b->present[q] ? b->variant[q] : -1;
  else if (order_of("grid_n", &q)) *value = b->present[q] ? b->grid[q] : 0;
  else if (k.rfind("tune_ms_n", 0) == 0 && k.size() >= 13 && k[k.size() - 2] == 'v' &&
           k[k.size() - 1] >= '0' && k[k.size() - 1] < '0' + kBatchVariants &&
           order_of("tune_ms_n", &q))
    *value = b->tune_ms[q][k[k.size() - 1] - '0'];
  else {
    set_error("sem_batch_get_option: unknown key: " + k);
    return SEM_EINVAL;
  }
  return SEM_OK;
}

extern "C" int sem_batch_pcg_solve(sem_batch b, const double* const* f, double* const* x,
                                   const sem_solve_opts* opts, sem_info* infos) {
  if (!b || !f || !x || !opts) {
    set_error("sem_batch_pcg_solve: null argument");
    return SEM_EINVAL;
  }
  if (opts->precision != SEM_MIXED_FP32) {
    set_error("sem_batch_pcg_solve: the batched solver runs the mixed precision path");
    return SEM_EINVAL;
  }
  for (int p = 0; p < b->count; ++p) {
    if (!f[p] || !x[p] || !is_device_ptr(f[p]) || !is_device_ptr(x[p])) {
      set_error("sem_batch_pcg_solve: f[i] and x[i] must be device pointers");
      return SEM_EINVAL;
    }
  }
  const double tol = opts->tol > 0 ? opts->tol : 1e-8;
  const int maxit = opts->maxit > 0 ? opts->maxit : 1000;
  const int chunk = opts->chunk > 0 ? opts->chunk : 8;
  const bool use_graph = opts->use_graph >= 0;
  const double delta = opts->replace_factor > 0 ? opts->replace_factor : 1e-2;
  const int P = b->count;
  int rc;
  const int64_t launches0 = b->launches;
  std::vector<int> finished(P, 0), status(P, 0), repl(P, 0), slow(P, 0);
  std::vector<double> relres_true(P, 1.0), bnorm(P, 0.0);
  SEM_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  SEM_CUDA(cudaEventRecord(b->ev0, b->stream));
  int64_t sub_launch0 = 0;
  for (int p = 0; p < P; ++p) sub_launch0 += b->subs[p]->launches;
  // start every problem: FP64 residual, FP32 copy, scalars (x0 = 0)
  for (int p = 0; p < P; ++p) {
    Handle& h = *b->subs[p];
    if ((rc = launch_masked_copy64(h, nullptr, h.x64))) return rc;
    if ((rc = fp64_residual(h, f[p], true, &relres_true[p], &bnorm[p]))) return rc;
    SEM_CUDA(cudaMemsetAsync(h.x32, 0, sizeof(float) * h.L, b->stream));
    SEM_CUDA(cudaMemsetAsync(h.p32, 0, sizeof(float) * h.L, b->stream));
    if (bnorm[p] == 0.0 || relres_true[p] <= tol) {
      finished[p] = 1;
      if ((rc = launch_scal_setup(h, h.scal, tol, 0, 0, 0))) return rc;
      if ((rc = launch_set_bnorm(h, h.scal, 1.0, nullptr))) return rc;   // done = 1
      continue;
    }
    if ((rc = launch_cast64to32(h, h.r64, h.b32))) return rc;
    if ((rc = launch_scal_setup(h, h.scal, std::max(tol, delta * relres_true[p]), maxit, 0, 0)))
      return rc;
    if ((rc = launch_cg_init32(h, kDotDot2, h.r32, h.b32, nullptr, h.minv32, h.scal, nullptr)))
      return rc;
    if ((rc = launch_set_bnorm(h, h.scal, bnorm[p], nullptr))) return rc;
  }
  std::vector<int> active(P);
  for (int p = 0; p < P; ++p) active[p] = !finished[p];
  if ((rc = batch_compact(*b, active))) return rc;
  for (;;) {
    int left = 0, newly = 0;
    for (int p = 0; p < P; ++p) {
      left += !finished[p];
      if (finished[p] && active[p]) {
        active[p] = 0;
        ++newly;
      }
    }
    if (!left) break;
    if (newly && (rc = batch_compact(*b, active))) return rc;
    if ((rc = batch_run_chunk(*b, chunk, use_graph))) return rc;
    if ((rc = batch_read_scalars(*b))) return rc;
    int err = 0;
    SEM_CUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      set_error("sem_batch_pcg_solve: a bounded device wait gave up");
      return SEM_ETIMEOUT;
    }
    for (int p = 0; p < P; ++p) {
      if (finished[p] || !b->h_scal_all[p].done) continue;
      Handle& h = *b->subs[p];
      const PcgScalars& s = b->h_scal_all[p];
      // fold the FP32 correction into x64 and replace the residual in FP64
      if ((rc = launch_add32to64(h, h.x64, h.x32))) return rc;
      SEM_CUDA(cudaMemsetAsync(h.x32, 0, sizeof(float) * h.L, b->stream));
      const double prev = relres_true[p];
      if ((rc = fp64_residual(h, f[p], false, &relres_true[p]))) return rc;
      bool stop = false;
      if (relres_true[p] <= tol) {
        stop = true;
      } else if (s.status == SEM_BREAKDOWN) {
        status[p] = SEM_BREAKDOWN;
        stop = true;
      } else if (s.iter >= maxit) {
        status[p] = SEM_MAXIT;
        stop = true;
      } else {
        slow[p] = relres_true[p] > 0.5 * prev ? slow[p] + 1 : 0;
        if (slow[p] >= 3 || repl[p] >= 80) {
          status[p] = SEM_STAGNATED;
          stop = true;
        }
      }
      if (stop) {
        finished[p] = 1;   // its scalars keep done = 1
        continue;
      }
      if ((rc = launch_cg_replace32(h, kDotDot2, h.r64, h.r32, h.minv32,
                                    std::max(tol, delta * relres_true[p]), h.scal)))
        return rc;
      ++repl[p];
    }
  }
  SEM_CUDA(cudaEventRecord(b->ev1, b->stream));
  if ((rc = batch_read_scalars(*b))) return rc;
  float ms = 0.f;
  SEM_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  int64_t sub_launch1 = 0;
  for (int p = 0; p < P; ++p) sub_launch1 += b->subs[p]->launches;
  int worst = 0;
  for (int p = 0; p < P; ++p) {
    Handle& h = *b->subs[p];
    SEM_CUDA(cudaMemcpyAsync(x[p], h.x64, sizeof(double) * h.L, cudaMemcpyDeviceToDevice,
                             b->stream));
    if (infos) {
      sem_info& in = infos[p];
      in.iters = b->h_scal_all[p].iter;
      in.refinements = repl[p];
      in.status = status[p];
      in.relres = b->h_scal_all[p].relres;
      in.relres_true = relres_true[p];
      in.solve_ms = ms;
      in.launches = (b->launches - launches0) + (sub_launch1 - sub_launch0);
    }
    if (status[p] > worst) worst = status[p];
  }
  SEM_CUDA(cudaStreamSynchronize(b->stream));
  return worst;
}
