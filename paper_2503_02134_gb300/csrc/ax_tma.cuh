// FP32 element operator with bulk-copy (TMA) staging.
//
// Same arithmetic as ax_kernel (ax_kernel.cuh: local_grad3, geometric
// factors, local_grad3_t of the paper's `ax`, Sec. 3.1) but the streamed
// inputs of a group of EPB consecutive elements -- u (or r, J^{-1} and p in
// PCG mode) and G1..G6, all contiguous in the element-major layout -- are
// brought into shared memory by 1-D cp.async.bulk copies issued by one
// thread, two stages deep, while the block computes the previous group.
// The copies complete on an mbarrier (transaction bytes), so the math warps
// never issue a global load: the memory pipe is kept busy by the copy engine
// instead of by occupancy.  Requires 16-byte aligned element blocks, i.e. an
// even number of GLL points per direction (n^3 * 4 bytes % 16 == 0).
//
// The t-direction contractions (u_t = D u along k and the accumulation of
// D^T v_t) index D with the two unrolled loop counters only, so D is passed
// by value as a kernel parameter: the entries are constant-bank operands of
// the FMAs and cost no shared-memory access.  Shared-memory wavefronts
// bounded the per-node form of this kernel at n >= 8 (per k-plane and
// warp: n/4 vector row loads for u_r, n loads for u_s, 6 for G, the same
// again for the transposed pass); the whole-line form that even n >= 6 now
// takes (tma_sline) needs about 19 shared-memory accesses per node.
#pragma once

#include "ax_kernel.cuh"
#include "tma.cuh"

namespace sem {

// Launch variants (elements per block, pipeline stages); the set-up
// autotuner times them on the actual mesh and keeps the fastest.  For
// n >= 12 one element already fills 144..256 threads: variants 0..2 are one
// element per stage with two, three and one stage, variant 3 two elements
// per stage (two stages).  A variant whose stages do not fit in shared
// memory (tma_fits) is never launched.  Variant 4 (line orders below 16,
// see tma_split) splits the stage: G alone single-staged and refilled as
// soon as the geometric loop is done with it, u double-staged.
template <int n, int V>
struct TmaShape {
  static constexpr int n2 = n * n;
  static constexpr int n3 = n * n * n;
  static constexpr int EPB_BIG = (128 / n2) > 0 ? (128 / n2) : 1;
  static constexpr int EPB_SMALL = (64 / n2) > 0 ? (64 / n2) : 1;
  static constexpr int EPB = n >= 12 ? (V == 3 ? 2 : 1) : (V == 0 ? EPB_BIG : EPB_SMALL);
  // bulk-copy stages: for n < 12 variant 0 two (two elements each), 1 three,
  // 2 four, 3 two (one element each: more resident blocks, shallower
  // prefetch); for n >= 12 variant 2 has a single stage, so that two blocks
  // (one computing while the other waits for its copy) fit on an SM where
  // two stages of one block would not leave room for a second block
  static constexpr int NS = V == 0 ? 2 : (V == 1 ? 3 : (V == 2 ? (n >= 12 ? 1 : 4) : 2));
  static constexpr int NT = ((n2 * EPB + 31) / 32) * 32;
  static constexpr uint32_t VEC = EPB * n3 * 4;                 // bytes of one vector per stage
};

// Orders whose contractions run as whole lines (the even-odd halves of D,
// the s-lines through a shared-memory buffer of one element; see
// ax_tma_kernel).  Measured against the per-node contractions at n = 6 and
// 8: 0.80 -> 0.92 and 0.92 -> 0.98 of the HBM peak in plain mode.
template <int n>
constexpr bool tma_sline() {
  return n >= 6;
}
// Orders whose stages hold G only: u (PCG mode: r, J^{-1}, p_old) is read
// by the threads themselves, one group ahead into registers, and stored to
// a single shared buffer; at n = 16 two stages of u and G plus the line
// buffer would exceed shared memory, two stages of G plus u and the line
// buffer fit.
template <int n>
constexpr bool tma_gonly() {
  return n == 16;
}

// Plane stride of the s-line buffer: the smallest P >= n^2 with P = n
// (mod 32), so that the n-thread runs of a warp in consecutive planes fall
// on consecutive banks (n = 16 keeps 256 and uses the swizzled layout).
template <int n>
constexpr int tma_ps() {
  if (n == 16) return 256;
  int P = n * n;
  while (P % 32 != n % 32) ++P;
  return P;
}

// Variant 4, the split stage (line orders below 16): one buffer of G with
// its own barrier, two buffers of u (PCG mode: p_old) with theirs, and in
// PCG mode one buffer of r and J^{-1} with a third barrier.  G of the next
// element is copied while the block is still on the transposed lines and
// the epilogue of this one, r and J^{-1} as soon as p is formed, u of the
// element after next while it computes this one.  Plain mode holds 8
// element vectors per block (two blocks still fit on an SM at n = 14), PCG
// mode 10.
template <int n, bool PCG, int V>
constexpr bool tma_split() {
  return V == 4 && tma_sline<n>() && !tma_gonly<n>();
}

template <int n, bool PCG, int V>
constexpr size_t tma_smem_bytes() {
  using S = TmaShape<n, V>;
  constexpr int NV = tma_gonly<n>() ? 0 : (PCG ? 3 : 1);   // vectors in a stage
  constexpr size_t ubuf = tma_gonly<n>() ? S::VEC : 0;      // thread-written u
  constexpr size_t sbuf = tma_sline<n>() ? (size_t)S::EPB * n * tma_ps<n>() * 4 : 0;
  if constexpr (tma_split<n, PCG, V>())
    return (size_t)(6 + (PCG ? 2 : 0) + S::NS) * S::VEC + sbuf +
           (S::NS + (PCG ? 2 : 1)) * sizeof(uint64_t);
  return S::NS * (size_t)(NV + 6) * S::VEC + ubuf + sbuf + S::NS * sizeof(uint64_t);
}

// Shared memory per block on sm_100/sm_103 (227 KB) and the static part of
// ax_tma_kernel (D with a padded row, one double per warp, alignment slack).
constexpr size_t kMaxSmemPerBlock = 232448;
template <int n, bool PCG, int V>
constexpr bool tma_fits() {
  if constexpr (V == 4 && !tma_split<n, PCG, V>()) return false;   // no split stage here
  return tma_smem_bytes<n, PCG, V>() + sizeof(float) * n * (n + 1) +
             sizeof(double) * (TmaShape<n, V>::NT / 32) + 256 <=
         kMaxSmemPerBlock;
}

// Dot product of a row of n contiguous shared-memory floats (16- or 8-byte
// aligned) with n register coefficients, using the widest vector loads the
// alignment allows.
template <int n>
__device__ __forceinline__ float row_dot(const float* __restrict__ row, const float* coef) {
  float s = 0.f;
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int l = 0; l < n; l += 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + l);
      s += coef[l] * v.x;
      s += coef[l + 1] * v.y;
      s += coef[l + 2] * v.z;
      s += coef[l + 3] * v.w;
    }
  } else if constexpr (n % 2 == 0) {
#pragma unroll
    for (int l = 0; l < n; l += 2) {
      const float2 v = *reinterpret_cast<const float2*>(row + l);
      s += coef[l] * v.x;
      s += coef[l + 1] * v.y;
    }
  } else {
#pragma unroll
    for (int l = 0; l < n; ++l) s += coef[l] * row[l];
  }
  return s;
}

// D by value for the staged kernel: the full matrix (row-major) and, for the
// whole-line contractions, its even-odd halves.  GLL D is centro-antisymmetric
// (D[N-i][N-l] = -D[i][l], nodes symmetric about 0), and so is D^T; for such
// an M, with x_e[l] = x[l] + x[N-l] and x_o[l] = x[l] - x[N-l] (l < n/2),
//   (M x)[i] = e_i + o_i,  (M x)[N-i] = o_i - e_i,
//   e_i = sum_l E[i][l] x_e[l],  o_i = sum_l O[i][l] x_o[l],
//   E[i][l] = (M[i][l] + M[i][N-l]) / 2,  O[i][l] = (M[i][l] - M[i][N-l]) / 2,
// i.e. n^2/2 FMAs and 2n additions instead of n^2 FMAs per line.
template <int n>
struct DMatEO {
  float d[n * n];
  float E[(n / 2) * (n / 2)], O[(n / 2) * (n / 2)];     // M = D
  float ET[(n / 2) * (n / 2)], OT[(n / 2) * (n / 2)];   // M = D^T
};

template <int n>
__device__ __forceinline__ void eo_line(const float (&E)[(n / 2) * (n / 2)],
                                        const float (&O)[(n / 2) * (n / 2)], const float (&x)[n],
                                        float (&y)[n]) {
  constexpr int h = n / 2;
  float xe[h], xo[h];
#pragma unroll
  for (int l = 0; l < h; ++l) {
    xe[l] = x[l] + x[n - 1 - l];
    xo[l] = x[l] - x[n - 1 - l];
  }
#pragma unroll
  for (int i = 0; i < h; ++i) {
    float e = 0.f, o = 0.f;
#pragma unroll
    for (int l = 0; l < h; ++l) {
      e += E[i * h + l] * xe[l];
      o += O[i * h + l] * xo[l];
    }
    y[i] = e + o;
    y[n - 1 - i] = o - e;
  }
}

// A row of n contiguous shared-memory floats (16- or 8-byte aligned) to and
// from registers with the widest vector accesses the alignment allows.
template <int n>
__device__ __forceinline__ void load_row(const float* __restrict__ row, float (&x)[n]) {
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int l = 0; l < n; l += 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + l);
      x[l] = v.x;
      x[l + 1] = v.y;
      x[l + 2] = v.z;
      x[l + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int l = 0; l < n; l += 2) {
      const float2 v = *reinterpret_cast<const float2*>(row + l);
      x[l] = v.x;
      x[l + 1] = v.y;
    }
  }
}
template <int n>
__device__ __forceinline__ void store_row(float* __restrict__ row, const float (&x)[n]) {
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int l = 0; l < n; l += 4)
      *reinterpret_cast<float4*>(row + l) = make_float4(x[l], x[l + 1], x[l + 2], x[l + 3]);
  } else {
#pragma unroll
    for (int l = 0; l < n; l += 2)
      *reinterpret_cast<float2*>(row + l) = make_float2(x[l], x[l + 1]);
  }
}

// Layout of the line buffers.  Node (i, j, k) of an element sits at
// k n^2 + j n + i (the bulk-copied layout) except in the thread-written
// buffers at n = 16, where 64-byte rows and 1 KB planes put the accesses of
// the s-lines (the same row in two planes) and of the r-lines (eight rows
// of a plane, 16 bytes each) on the same banks.  There the row index is
// flipped in odd planes and the 16-byte chunks of a row are permuted by the
// row pair: (i, j, k) -> k 256 + r 16 + (i ^ 4 ((r >> 1) & 3)), r = j ^ (k & 1),
// which makes the column, s-line and r-line accesses conflict-free.
template <int n, bool kSwz>
__device__ __forceinline__ int lb_at(int i, int j, int k) {
  if constexpr (kSwz) {
    static_assert(n == 16, "the swizzled layout is for n = 16");
    const int r = j ^ (k & 1);
    return k * 256 + r * 16 + (i ^ (((r >> 1) & 3) << 2));
  } else {
    return (k * n + j) * n + i;
  }
}
// The s-line buffer: swizzled at n = 16, otherwise planes of tma_ps<n>().
template <int n, bool kSwz>
__device__ __forceinline__ int sb_at(int i, int j, int k) {
  if constexpr (kSwz) return lb_at<n, true>(i, j, k);
  else return k * tma_ps<n>() + j * n + i;
}
// Row (j, k) to and from registers in either layout.
template <int n, bool kSwz>
__device__ __forceinline__ void load_row_lb(const float* __restrict__ buf, int j, int k,
                                            float (&x)[n]) {
  if constexpr (kSwz) {
#pragma unroll
    for (int c = 0; c < n / 4; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(buf + lb_at<n, true>(4 * c, j, k));
      x[4 * c] = v.x;
      x[4 * c + 1] = v.y;
      x[4 * c + 2] = v.z;
      x[4 * c + 3] = v.w;
    }
  } else {
    load_row<n>(buf + (k * n + j) * n, x);
  }
}
template <int n, bool kSwz>
__device__ __forceinline__ void store_row_lb(float* __restrict__ buf, int j, int k,
                                             const float (&x)[n]) {
  if constexpr (kSwz) {
#pragma unroll
    for (int c = 0; c < n / 4; ++c)
      *reinterpret_cast<float4*>(buf + lb_at<n, true>(4 * c, j, k)) =
          make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  } else {
    store_row<n>(buf + (k * n + j) * n, x);
  }
}

// Dot products with two independent accumulator chains (even and odd l,
// added at the end): twice the instruction-level parallelism of one FMA
// chain, for the orders where a block holds only a few warps.
template <int n>
__device__ __forceinline__ float row_dot_2acc(const float* __restrict__ row, const float* coef) {
  float s0 = 0.f, s1 = 0.f;
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int l = 0; l < n; l += 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + l);
      s0 += coef[l] * v.x;
      s1 += coef[l + 1] * v.y;
      s0 += coef[l + 2] * v.z;
      s1 += coef[l + 3] * v.w;
    }
  } else {
#pragma unroll
    for (int l = 0; l < n; l += 2) {
      const float2 v = *reinterpret_cast<const float2*>(row + l);
      s0 += coef[l] * v.x;
      s1 += coef[l + 1] * v.y;
    }
  }
  return s0 + s1;
}
template <int n, int stride>
__device__ __forceinline__ float col_dot_2acc(const float* __restrict__ p, const float* coef) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int l = 0; l < n; l += 2) {
    s0 += coef[l] * p[l * stride];
    s1 += coef[l + 1] * p[(l + 1) * stride];
  }
  return s0 + s1;
}

// Copy parts of the split stage (variant 4), a mask.
constexpr int kPartG = 1, kPartU = 2, kPartRM = 4, kPartAll = 7;

template <int n, bool PCG, int DM, int V>
__global__ void __launch_bounds__(TmaShape<n, V>::NT)
    ax_tma_kernel(const float* __restrict__ uin, float* __restrict__ wout,
                  const float* __restrict__ G, const float* __restrict__ Dg,
                  const __grid_constant__ DMatEO<n> Dc,
                  const uint8_t* __restrict__ faces, int64_t E, const float* __restrict__ rr,
                  const float* __restrict__ minv, float* pp, PcgScalars* __restrict__ scal,
                  double* __restrict__ partials, int* __restrict__ err, int l2h) {
  using S = TmaShape<n, V>;
  constexpr int n2 = S::n2, n3 = S::n3, EPB = S::EPB, NS = S::NS;
  constexpr bool kGOnly = tma_gonly<n>();
  constexpr int NV = kGOnly ? 0 : (PCG ? 3 : 1);   // vectors staged with G
  constexpr int SV = EPB * n3;                 // floats of one vector per stage
  // variant 4: G in one buffer (barrier NS), PCG mode r and J^{-1} in one
  // (barrier NS + 1), u or p_old in NS stages (barriers 0..NS-1)
  constexpr bool kSplitSt = tma_split<n, PCG, V>();
  constexpr int SPLIT_FIXED = 6 + (PCG ? 2 : 0);   // split: vectors of the single buffers
  constexpr int STAGE = kSplitSt ? SV : (NV + 6) * SV;   // floats per stage
  constexpr int STAGED = kSplitSt ? (SPLIT_FIXED + NS) * SV : NS * STAGE;   // floats of all stages
  // n >= 10: split accumulator chains (one or two blocks of few warps per SM)
  constexpr bool kSplit = n >= 10;
  constexpr bool kSLine = tma_sline<n>();
  constexpr bool kSwz = kGOnly && n == 16;   // swizzled thread-written line buffers
  // line orders with two or more stages refill a stage's G as soon as the
  // geometric loop is done with it (measured: faster with two stages,
  // slower with a single stage, where the block waits for its own copy)
  constexpr bool kEarly = kSLine && NS >= 2 && !kSplitSt;
  extern __shared__ __align__(128) float smem_f[];
  float* const stage0 = kSplitSt ? smem_f + SPLIT_FIXED * SV : smem_f;
  // kGOnly: u (or p) of the group, then u_r; kSLine: the s-line buffer
  // (u_s, v_s, then w_s)
  constexpr int SSE = n * tma_ps<n>();                 // floats of one element's s-lines
  float* const sU = smem_f + STAGED;
  float* const sS = smem_f + STAGED + (kGOnly ? SV : 0);
  uint64_t* const bar = reinterpret_cast<uint64_t*>(smem_f + STAGED + (kGOnly ? SV : 0) +
                                                    (kSLine ? EPB * SSE : 0));
  constexpr int NBAR = NS + (kSplitSt ? (PCG ? 2 : 1) : 0);
  // split stage: copies of G and of r, J^{-1} issued so far (thread 0), so
  // that an aborted block knows which phase of their barriers is outstanding
  uint32_t n_g = 0, n_rm = 0;
  __shared__ float sD[n][n + 1];
  __shared__ double sh_red[S::NT / 32];

  if (PCG && scal->done) return;
  const float beta = PCG ? (float)scal->beta : 0.f;

  const int tid = threadIdx.x;
  const int le = tid / n2;
  const int ij = tid - le * n2;
  const int i = ij % n, j = ij / n;
  const bool lane_ok = le < EPB;
  const int ir = lane_ok ? i : 0, jr = lane_ok ? j : 0, ler = lane_ok ? le : 0;
  const int64_t ngroups = (E + EPB - 1) / EPB;
  // with l2h: everything streams through L2 evict-first except the output
  // w, which the next kernel reads (and gathers) again
  const uint64_t pol_first = l2h ? l2_policy_evict_first() : 0ull;
  const uint64_t pol_last = l2h ? l2_policy_evict_last() : 0ull;

  // Copies of group g into stage st.  part 0: everything; part 1 (issued as
  // soon as the stage's G is no longer read): the transaction count of the
  // whole stage, G and, in PCG mode, r and J^{-1}; part 2 (once the group
  // is finished): u, or p_old in PCG mode.  The stage's barrier phase
  // completes only when the bytes of both parts have landed.  Split stage:
  // a mask of kPartG (G into its buffer, barrier NS), kPartU (u or p_old
  // into stage st) and kPartRM (r and J^{-1} into theirs, barrier NS + 1),
  // each with its own transaction count.
  auto issue = [&](int st, int64_t g, int part) {
    const int64_t e0 = g * EPB;
    const int64_t cnt = E - e0 < EPB ? E - e0 : EPB;
    const uint32_t vb = (uint32_t)(cnt * n3 * 4);
    float* dst = stage0 + st * STAGE;
    auto copy_on = [&](float* d, const float* src, uint32_t bytes, uint64_t* b) {
      if (l2h) bulk_load_hint(d, src, bytes, b, pol_first);
      else bulk_load(d, src, bytes, b);
    };
    auto copy = [&](float* d, const float* src, uint32_t bytes) { copy_on(d, src, bytes, &bar[st]); };
    if constexpr (kSplitSt) {
      if (part & kPartG) {
        mbar_arrive_expect_tx(&bar[NS], 6 * vb);
        copy_on(smem_f, G + e0 * 6 * n3, 6 * vb, &bar[NS]);
        ++n_g;
      }
      if (PCG && (part & kPartRM)) {
        mbar_arrive_expect_tx(&bar[NS + 1], 2 * vb);
        copy_on(smem_f + 6 * SV, rr + e0 * n3, vb, &bar[NS + 1]);
        copy_on(smem_f + 7 * SV, minv + e0 * n3, vb, &bar[NS + 1]);
        ++n_rm;
      }
      if (part & kPartU) {
        mbar_arrive_expect_tx(&bar[st], vb);
        copy(dst, PCG ? pp + e0 * n3 : uin + e0 * n3, vb);
      }
      return;
    }
    if (part != 2) {
      mbar_arrive_expect_tx(&bar[st], (NV + 6) * vb);
      copy(dst + NV * SV, G + e0 * 6 * n3, 6 * vb);
      if (PCG && !kGOnly) {
        copy(dst, rr + e0 * n3, vb);
        copy(dst + SV, minv + e0 * n3, vb);
      }
    }
    if (part != 1 && !kGOnly) {
      if (PCG) copy(dst + 2 * SV, pp + e0 * n3, vb);
      else copy(dst, uin + e0 * n3, vb);
    }
  };

  if (tid == 0) {
    for (int q = 0; q < NBAR; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  for (int q = tid; q < n2; q += blockDim.x) sD[q / n][q % n] = Dg[q];
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      const int64_t g0 = (int64_t)blockIdx.x + (int64_t)q * gridDim.x;
      if (g0 < ngroups) {
        if constexpr (kSplitSt) issue(q, g0, q == 0 ? kPartAll : kPartU);   // G, r, J^{-1}: first only
        else issue(q, g0, 0);
      }
    }
  }
  float Di[n], Dj[n], DiT[n], DjT[n];
#pragma unroll
  for (int l = 0; l < n; ++l) {
    Di[l] = sD[ir][l];
    Dj[l] = sD[jr][l];
    DiT[l] = sD[l][ir];
    DjT[l] = sD[l][jr];
  }

  // kGOnly: the next group's vectors, read one group ahead (u; PCG mode r,
  // J^{-1}, p_old of this thread's column)
  float pa[kGOnly ? n : 1], pb[kGOnly && PCG ? n : 1], pc[kGOnly && PCG ? n : 1];
  auto prefetch = [&](int64_t gq) {
    if constexpr (kGOnly) {
      const int64_t eq = gq * EPB + le;
      if (lane_ok && gq < ngroups && eq < E) {
        const int64_t b0 = eq * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          if (PCG) {
            pa[k] = __ldg(rr + b0 + k * n2);
            pb[k] = __ldg(minv + b0 + k * n2);
            pc[k] = pp[b0 + k * n2];   // written by this kernel (other elements)
          } else {
            pa[k] = __ldg(uin + b0 + k * n2);
          }
        }
      }
    }
  };
  prefetch(blockIdx.x);

  DotAcc<float, DM> acc;
  bool aborted = false;
  int t = 0;
  // group t of this block lives on stage t % NS and is that stage's
  // (t / NS)-th use, so its barrier phase parity is (t / NS) & 1
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, ++t) {
    const int st = t % NS;
    bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((t / NS) & 1));
    if constexpr (kSplitSt && PCG) ok = ok && mbar_wait_bounded(&bar[NS + 1], (uint32_t)(t & 1));
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    float* const sb = stage0 + st * STAGE;
    // p (formed in place) or u; r and J^{-1} of the group
    float* const su = kGOnly ? sU : (PCG && !kSplitSt ? sb + 2 * SV : sb);
    const float* const sR = kSplitSt ? smem_f + 6 * SV : sb;
    const float* const sM = kSplitSt ? smem_f + 7 * SV : sb + SV;
    float* const sg = kSplitSt ? smem_f : sb + NV * SV;   // G1..G6 of the group
    const float* const Gs = sg + ler * 6 * n3 + ij;
    float* const su_e = su + ler * n3;
    // the two transposed-contraction inputs overwrite G1 and G2 of the
    // stage: each thread reads its own G entries (k, ij) before it writes
    // the same positions, and the stage is refilled only after the last
    // barrier of the group
    float* const sr_e = sg + ler * 6 * n3;
    float* const ss_e = sr_e + n3;
    const int64_t e = g * EPB + le;
    const bool act = lane_ok && e < E;
    const uint8_t f = act ? faces[e] : uint8_t(0);   // issued early, used in the epilogue

    float ureg[n];
    if constexpr (kGOnly) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const float v = PCG ? pb[k] * pa[k] + beta * pc[k] : pa[k];
        ureg[k] = v;
        if (lane_ok) su_e[lb_at<n, kSwz>(i, j, k)] = v;
      }
      prefetch(g + gridDim.x);
    } else {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int si = k * n2 + ij;
        float v;
        if (PCG) {
          v = sM[ler * n3 + si] * sR[ler * n3 + si] + beta * su_e[si];
          if (lane_ok) su_e[si] = v;   // p goes to memory with w in the epilogue
        } else {
          v = su_e[si];
        }
        ureg[k] = v;
      }
    }
    float* const sS_e = sS + ler * SSE;
    if constexpr (kSLine) {
      // line contractions: besides its t-column (i, j) this thread owns the
      // s-line (i, k = j) and the r-line (j = i, k = j) of the element.  u_s
      // and u_r of a whole line are D times the line by the even-odd halves
      // (constant bank); u_s goes to the s-line buffer at once, u_r over the
      // same row of u once every thread has read u
      if (PCG || kGOnly) __syncthreads();   // u or p complete in shared memory
      if constexpr (kSplitSt && PCG) {
        // r and J^{-1} are no longer read: copy the block's next group's
        if (tid == 0) {
          const int64_t gn = g + (int64_t)gridDim.x;
          if (gn < ngroups) {
            fence_proxy_async_smem();
            issue(st, gn, kPartRM);
          }
        }
      }
      float a[n], y[n], yr[n];
#pragma unroll
      for (int l = 0; l < n; ++l) a[l] = su_e[lb_at<n, kSwz>(ir, l, jr)];
      eo_line<n>(Dc.E, Dc.O, a, y);
      if (lane_ok) {
#pragma unroll
        for (int jj = 0; jj < n; ++jj) sS_e[sb_at<n, kSwz>(ir, jj, jr)] = y[jj];
      }
      load_row_lb<n, kSwz>(su_e, ir, jr, a);
      eo_line<n>(Dc.E, Dc.O, a, yr);
      __syncthreads();
      if (lane_ok) store_row_lb<n, kSwz>(su_e, ir, jr, yr);
      __syncthreads();
    } else {
      if (PCG) __syncthreads();
    }

    // line orders: u_t of the whole t-column by the even-odd halves, and the
    // t-column of v_t kept for the transposed product after the plane loop
    float utk[kSLine ? n : 1], vtk[kSLine ? n : 1];
    if constexpr (kSLine) eo_line<n>(Dc.E, Dc.O, ureg, utk);
    if constexpr (kSplitSt) {
      // G of this group: its copy has run since the geometric loop of the
      // block's previous group
      const bool okg = mbar_wait_bounded(&bar[NS], (uint32_t)(t & 1));
      if (__syncthreads_or(!okg)) {
        aborted = true;
        break;
      }
    }
    float wreg[n];
#pragma unroll
    for (int k = 0; k < n; ++k) wreg[k] = 0.f;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      float ur, us, ut = 0.f;
      if constexpr (kSLine) {
        ur = su_e[lb_at<n, kSwz>(i, j, k)];
        us = sS_e[sb_at<n, kSwz>(i, j, k)];
        ut = utk[k];
      } else if constexpr (kSplit) {
        ur = row_dot_2acc<n>(su_e + k * n2 + jr * n, Di);
        us = col_dot_2acc<n, n>(su_e + k * n2 + ir, Dj);
      } else {
        ur = row_dot<n>(su_e + k * n2 + jr * n, Di);
        us = 0.f;
#pragma unroll
        for (int l = 0; l < n; ++l) us += Dj[l] * su_e[k * n2 + l * n + ir];
      }
      if constexpr (!kSLine) {
#pragma unroll
        for (int l = 0; l < n; ++l) ut += Dc.d[k * n + l] * ureg[l];
      }
      const float g0 = Gs[0 * n3 + k * n2], g1 = Gs[1 * n3 + k * n2], g2 = Gs[2 * n3 + k * n2];
      const float g3 = Gs[3 * n3 + k * n2], g4 = Gs[4 * n3 + k * n2], g5 = Gs[5 * n3 + k * n2];
      const float vr = g0 * ur + g3 * us + g4 * ut;
      const float vs = g3 * ur + g1 * us + g5 * ut;
      const float vt = g4 * ur + g5 * us + g2 * ut;
      if (lane_ok) {
        // line orders: v_r over this thread's own u_r and v_s over its own
        // u_s, so that G is dead after this loop; otherwise v_r, v_s over
        // G1, G2 of the stage
        if constexpr (kSLine) su_e[lb_at<n, kSwz>(i, j, k)] = vr;
        else sr_e[k * n2 + ij] = vr;
        if constexpr (kSLine) sS_e[sb_at<n, kSwz>(i, j, k)] = vs;
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
    if constexpr (kSplitSt) {
      // G is no longer read: copy the block's next group's G now
      if (tid == 0) {
        const int64_t gn = g + (int64_t)gridDim.x;
        if (gn < ngroups) {
          fence_proxy_async_smem();
          issue(st, gn, kPartG);
        }
      }
    }
    if constexpr (kEarly) {
      // G (and r, J^{-1}) of this stage are no longer read: start the copies
      // of the next group that uses this stage now, not after the group
      if (tid == 0) {
        const int64_t gn = g + NS * (int64_t)gridDim.x;
        if (gn < ngroups) {
          fence_proxy_async_smem();
          issue(st, gn, 1);
        }
      }
    }
    if constexpr (kSLine) {
      // transposed s-lines: w_s of line (i, k = j) = D^T times the line of
      // v_s, written back over the same line (this thread reads all of it
      // first; no other thread touches it)
      // and w_r of the r-line (j = i, k = j) = D^T times the row of v_r, in
      // place as well
      float b[n], y[n];
#pragma unroll
      for (int l = 0; l < n; ++l) b[l] = sS_e[sb_at<n, kSwz>(ir, l, jr)];
      eo_line<n>(Dc.ET, Dc.OT, b, y);
      if (lane_ok) {
#pragma unroll
        for (int jj = 0; jj < n; ++jj) sS_e[sb_at<n, kSwz>(ir, jj, jr)] = y[jj];
      }
      float* const vr_e = su_e;
      load_row_lb<n, kSwz>(vr_e, ir, jr, b);
      eo_line<n>(Dc.ET, Dc.OT, b, y);
      if (lane_ok) store_row_lb<n, kSwz>(vr_e, ir, jr, y);
      __syncthreads();
    }

#pragma unroll
    for (int k = 0; k < n; ++k) {
      float wv;
      if constexpr (kSLine) {
        const float wr = su_e[lb_at<n, kSwz>(i, j, k)];
        wv = wreg[k] + (wr + sS_e[sb_at<n, kSwz>(i, j, k)]);
      } else if constexpr (kSplit) {
        wv = wreg[k] + (row_dot_2acc<n>(sr_e + k * n2 + jr * n, DiT) +
                        col_dot_2acc<n, n>(ss_e + k * n2 + ir, DjT));
      } else {
        wv = wreg[k] + row_dot<n>(sr_e + k * n2 + jr * n, DiT);
#pragma unroll
        for (int l = 0; l < n; ++l) wv += DjT[l] * ss_e[k * n2 + l * n + ir];
      }
      if (on_dirichlet(f, i, j, k, n - 1)) wv = 0.f;
      if (act) {
        if (l2h) st_hint(wout + e * n3 + k * n2 + ij, wv, pol_last);
        else wout[e * n3 + k * n2 + ij] = wv;
        if (PCG) {
          if (l2h) st_hint(pp + e * n3 + k * n2 + ij, ureg[k], pol_first);
          else pp[e * n3 + k * n2 + ij] = ureg[k];
          acc.add(ureg[k], wv);
        }
      }
    }
    __syncthreads();   // stage st is free again
    if (tid == 0) {
      const int64_t gn = g + NS * (int64_t)gridDim.x;
      if (gn < ngroups) {
        fence_proxy_async_smem();
        issue(st, gn, kSplitSt ? kPartU : (kEarly ? 2 : 0));
      }
    }
  }

  if (aborted) {
    // A bulk copy never completed: report it, give the copies this block
    // still has in flight a bounded time to land (each stage has at most one
    // outstanding phase), and leave without publishing a partial sum.
    if (tid == 0) {
      atomicExch(err, 1);
      const int64_t g_abort = blockIdx.x + (int64_t)t * gridDim.x;
      for (int s2 = 0; s2 < NS; ++s2) {
        // the group outstanding on stage s2 is the next one mapped to it
        const int64_t g_out = g_abort + (int64_t)((s2 - t % NS + NS) % NS) * gridDim.x;
        const int done_uses = t > s2 ? (t - 1 - s2) / NS + 1 : 0;
        if (g_out < ngroups) mbar_wait_bounded(&bar[s2], (uint32_t)(done_uses & 1));
      }
      // split stage: the last copies of G and of r, J^{-1} that were issued
      // (their barrier phases complete in order, so waiting on the last
      // one covers the earlier ones; a completed phase returns at once)
      if (kSplitSt && n_g) mbar_wait_bounded(&bar[NS], (n_g - 1) & 1u);
      if (kSplitSt && PCG && n_rm) mbar_wait_bounded(&bar[NS + 1], (n_rm - 1) & 1u);
    }
    return;
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

template <int n, bool PCG, int DM, int V>
int ax_tma_launch(Handle& h, const float* u, float* w, const AxPrologue* pro) {
  using S = TmaShape<n, V>;
  auto kern = ax_tma_kernel<n, PCG, DM, V>;
  constexpr size_t smem = tma_smem_bytes<n, PCG, V>();
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::NT, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t groups = (h.E + S::EPB - 1) / S::EPB;
  int64_t cap = (int64_t)h.num_sms * per_sm;
  if (cap > h.max_blocks) cap = h.max_blocks;
  if (h.ax_grid_cap > 0 && cap > h.ax_grid_cap) cap = h.ax_grid_cap;
  const int grid = (int)(groups < cap ? groups : cap);
  const float* r = PCG ? (const float*)pro->r : nullptr;
  const float* minv = PCG ? (const float*)pro->minv : nullptr;
  PcgScalars* scal = PCG ? const_cast<PcgScalars*>(pro->scal) : nullptr;
  double* partials = PCG ? pro->pap_partials : nullptr;
  float* pp = PCG ? const_cast<float*>(u) : nullptr;
  const int l2h = PCG && h.l2_hints ? 1 : 0;
  DMatEO<n> Dc;
  for (int q = 0; q < n * n; ++q) Dc.d[q] = h.D32_host[q];
  constexpr int hh = n / 2;
  for (int a = 0; a < hh; ++a)
    for (int l = 0; l < hh; ++l) {
      const double* D = h.D64_host;   // halves formed in FP64, rounded once
      Dc.E[a * hh + l] = (float)(0.5 * (D[a * n + l] + D[a * n + (n - 1 - l)]));
      Dc.O[a * hh + l] = (float)(0.5 * (D[a * n + l] - D[a * n + (n - 1 - l)]));
      Dc.ET[a * hh + l] = (float)(0.5 * (D[l * n + a] + D[(n - 1 - l) * n + a]));
      Dc.OT[a * hh + l] = (float)(0.5 * (D[l * n + a] - D[(n - 1 - l) * n + a]));
    }
  kern<<<grid, S::NT, smem, h.stream>>>(u, w, h.G32, h.D32, Dc, h.bfaces, h.E, r, minv, pp,
                                        scal, partials, h.dev_err, l2h);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace sem
