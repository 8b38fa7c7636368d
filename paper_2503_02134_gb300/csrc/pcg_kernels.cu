// Vector kernels of the PCG loop (arXiv 2503.02134, profiling table of
// Sec. 3.1): add2s2 (x += alpha p, r -= alpha w) fused with the two dot
// products glsc3(r,c,r) and glsc3(r,c,z) (z = J^{-1} r, Sec. 4.3), the
// convergence test, and the scalar recurrences beta = rtz / rtz_old.
// Also: the initial residual, the weighted dot (glsc3) and the FP64
// refinement helpers of the mixed path.
#include <type_traits>

#include "gs_sum.cuh"
#include "pcg.cuh"
#include "tma.cuh"

namespace sem {

constexpr int kVecThreads = 256;

template <typename T, int DM>
__global__ void __launch_bounds__(kVecThreads)
    cg_update_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                     const T* __restrict__ w, const T* __restrict__ c, const T* __restrict__ minv,
                     int64_t L, PcgScalars* __restrict__ s, double* __restrict__ partials,
                     double* __restrict__ hist) {
  __shared__ double sh[kVecThreads / 32];
  if (s->done) return;
  const T alpha = (T)s->alpha;
  DotAcc<T, DM> a_rr, a_rz;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    const T xv = x[l] + alpha * p[l];
    const T rv = r[l] - alpha * w[l];
    x[l] = xv;
    r[l] = rv;
    const T cr = c[l] * rv;
    a_rr.add(cr, rv);
    a_rz.add(cr, minv[l] * rv);
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[1])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      finish_iteration(s, rtr, rtz, hist);
      s->counter[1] = 0u;
    }
  }
}

// FP32 update with 16-byte vector accesses.  The glsc3 weight c = mask /
// multiplicity comes from a 1-byte code (multiplicity, 0 on the Dirichlet
// boundary), which is exact for the power-of-two multiplicities of a box
// mesh and cuts 3 of the 32 bytes this pass moves per DOF.
__device__ __forceinline__ float weight_of(uint8_t m) {
  return m ? __frcp_rn((float)m) : 0.f;
}

template <int DM>
__global__ void __launch_bounds__(kVecThreads)
    cg_update32_v4_kernel(float* __restrict__ x, float* __restrict__ r,
                          const float* __restrict__ p, const float* __restrict__ w,
                          const uint8_t* __restrict__ cw, const float* __restrict__ minv,
                          int64_t L, PcgScalars* __restrict__ s, double* __restrict__ partials,
                          double* __restrict__ hist) {
  __shared__ double sh[kVecThreads / 32];
  if (s->done) return;
  const float alpha = (float)s->alpha;
  DotAcc<float, DM> a_rr, a_rz;
  const int64_t n4 = L >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto step = [&](int64_t q) {
    float4 xv = reinterpret_cast<float4*>(x)[q];
    float4 rv = reinterpret_cast<float4*>(r)[q];
    const float4 pv = __ldg(reinterpret_cast<const float4*>(p) + q);
    const float4 wv = __ldg(reinterpret_cast<const float4*>(w) + q);
    const float4 mv = __ldg(reinterpret_cast<const float4*>(minv) + q);
    const uchar4 cv = __ldg(reinterpret_cast<const uchar4*>(cw) + q);
    xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
    rv.x -= alpha * wv.x; rv.y -= alpha * wv.y; rv.z -= alpha * wv.z; rv.w -= alpha * wv.w;
    reinterpret_cast<float4*>(x)[q] = xv;
    reinterpret_cast<float4*>(r)[q] = rv;
    float c;
    c = weight_of(cv.x) * rv.x; a_rr.add(c, rv.x); a_rz.add(c, mv.x * rv.x);
    c = weight_of(cv.y) * rv.y; a_rr.add(c, rv.y); a_rz.add(c, mv.y * rv.y);
    c = weight_of(cv.z) * rv.z; a_rr.add(c, rv.z); a_rz.add(c, mv.z * rv.z);
    c = weight_of(cv.w) * rv.w; a_rr.add(c, rv.w); a_rz.add(c, mv.w * rv.w);
  };
  // two independent float4 groups per trip keep twice the loads in flight
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; q + stride < n4; q += 2 * stride) {
    step(q);
    step(q + stride);
  }
  if (q < n4) step(q);
  for (int64_t l = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L; l += stride) {
    const float xv = x[l] + alpha * p[l];
    const float rv = r[l] - alpha * w[l];
    x[l] = xv;
    r[l] = rv;
    const float c = weight_of(cw[l]) * rv;
    a_rr.add(c, rv);
    a_rz.add(c, minv[l] * rv);
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[1])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      finish_iteration(s, rtr, rtz, hist);
      s->counter[1] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Update with the direct-stiffness summation folded in (box meshes).
//
// In the CG loop w = QQ^T A_L p is consumed only by r -= alpha w (the p.w
// dot is taken on the unsummed w with the mask as weight, which is the same
// number because p is continuous).  So instead of a separate pass that sums
// the copies of every shared node and writes the sum back to each copy, each
// local entry here gathers the copies of its own node and sums them itself.
// On a box mesh the copies are found from the entry's position: a node on
// face i = 0 of element e is also node i = n-1 of element e-1 (when the face
// is not on the domain boundary), and likewise in j (element e -+ kx) and k
// (element e -+ kx ky); edges and corners take the products of these.  The
// copies are visited in ascending element order -- ascending local index,
// the order of the separate gather-scatter -- with the same accumulator, so
// every copy computes the same bits and the result equals the unfused path
// bit for bit.  Nodes with one copy keep w unchanged, as there.

// Any n: the float4 traversal of cg_update32_v4_kernel (same groups, same
// dot order), each component gathered on its own.
template <int DM, int ACC>
__global__ void __launch_bounds__(kVecThreads)
    cg_update32_gs_kernel(float* __restrict__ x, float* __restrict__ r,
                          const float* __restrict__ p, const float* __restrict__ w,
                          const uint8_t* __restrict__ cw, const float* __restrict__ minv,
                          const uint8_t* __restrict__ faces, BoxNbr b, int64_t L,
                          PcgScalars* __restrict__ s, double* __restrict__ partials,
                          double* __restrict__ hist) {
  __shared__ double sh[kVecThreads / 32];
  if (s->done) return;
  const float alpha = (float)s->alpha;
  DotAcc<float, DM> a_rr, a_rz;
  auto node = [&](int64_t l) -> float {
    const int64_t e = l / b.n3;
    const int rem = (int)(l - e * b.n3);
    return gs_gather_node<ACC>(w, l, rem % b.n, (rem / b.n) % b.n, rem / (b.n * b.n),
                               __ldg(faces + e), b);
  };
  const int64_t n4 = L >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto step = [&](int64_t q) {
    float4 xv = reinterpret_cast<float4*>(x)[q];
    float4 rv = reinterpret_cast<float4*>(r)[q];
    const float4 pv = __ldg(reinterpret_cast<const float4*>(p) + q);
    const float4 mv = __ldg(reinterpret_cast<const float4*>(minv) + q);
    const uchar4 cv = __ldg(reinterpret_cast<const uchar4*>(cw) + q);
    float4 wv;
    wv.x = node(4 * q);
    wv.y = node(4 * q + 1);
    wv.z = node(4 * q + 2);
    wv.w = node(4 * q + 3);
    xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
    rv.x -= alpha * wv.x; rv.y -= alpha * wv.y; rv.z -= alpha * wv.z; rv.w -= alpha * wv.w;
    reinterpret_cast<float4*>(x)[q] = xv;
    reinterpret_cast<float4*>(r)[q] = rv;
    float c;
    c = weight_of(cv.x) * rv.x; a_rr.add(c, rv.x); a_rz.add(c, mv.x * rv.x);
    c = weight_of(cv.y) * rv.y; a_rr.add(c, rv.y); a_rz.add(c, mv.y * rv.y);
    c = weight_of(cv.z) * rv.z; a_rr.add(c, rv.z); a_rz.add(c, mv.z * rv.z);
    c = weight_of(cv.w) * rv.w; a_rr.add(c, rv.w); a_rz.add(c, mv.w * rv.w);
  };
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += stride) step(q);
  for (int64_t l = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L; l += stride) {
    const float xv = x[l] + alpha * p[l];
    const float rv = r[l] - alpha * node(l);
    x[l] = xv;
    r[l] = rv;
    const float c = weight_of(cw[l]) * rv;
    a_rr.add(c, rv);
    a_rz.add(c, minv[l] * rv);
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[1])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      finish_iteration(s, rtr, rtz, hist);
      s->counter[1] = 0u;
    }
  }
}

// Launch shapes of the folded update: the blocks per SM its register budget
// is set for (the kernel is latency-bound on its gathers, so resident warps
// count most; measured: two float4 groups per thread per trip at 2-3 blocks
// were 40-50 % slower than one group at 4 blocks).
template <int VAR>
struct UpdShape {
  static constexpr int MINB = (VAR == 1 || VAR == 5) ? 5 : (VAR == 2 ? 6 : 4);
  static constexpr int GPT = 1;
  // variant 3: four blocks, and an L2 prefetch of the next trip's streams
  static constexpr bool PREFETCH = VAR == 3;
  // variants 0 and 5 (four, five blocks) index in 32 bits -- fewer registers
  // (measured 5.7 % faster at N = 7, 4.5 % at N = 11 than the same kernel
  // with 64-bit indices, variant 4); the launcher takes them only where
  // every value index the kernel forms fits in 31 bits
  static constexpr bool I32 = VAR == 0 || VAR == 5;
  using I = typename std::conditional<I32, int, int64_t>::type;
};

// Box mesh, n a multiple of 4: the glsc3 weights (mask / multiplicity) of
// the four values of float4 group q, from the nodes' positions and the
// element's face bits f -- the values the 1-byte codes hold: a node on s
// faces shared with other elements has 2^s copies (weight 2^-s, exact),
// and the weight is 0 on a Dirichlet face.
template <int n, typename I>
__device__ __forceinline__ float4 box_weights4(I q, uint8_t f) {
  constexpr int g4 = n * n * n / 4, row4 = n / 4;
  const int rem = (int)(q % g4);
  const int i0 = (rem % row4) * 4;
  const int j = (rem / row4) % n;
  const int k = rem / (row4 * n);
  bool dir = false;   // on a Dirichlet face in y or z
  int syz = 0;        // y and z faces the node lies on
  if (j == 0) { dir |= (f & 4) != 0; ++syz; }
  if (j == n - 1) { dir |= (f & 8) != 0; ++syz; }
  if (k == 0) { dir |= (f & 16) != 0; ++syz; }
  if (k == n - 1) { dir |= (f & 32) != 0; ++syz; }
  const bool lo = i0 == 0, hi = i0 + 3 == n - 1;   // first / last value on an x face
  const float wmid = dir ? 0.f : __int_as_float((127 - syz) << 23);
  const float wlo = dir || (lo && (f & 1)) ? 0.f : __int_as_float((127 - syz - (lo ? 1 : 0)) << 23);
  const float whi = dir || (hi && (f & 2)) ? 0.f : __int_as_float((127 - syz - (hi ? 1 : 0)) << 23);
  return make_float4(wlo, wmid, wmid, whi);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int n, int DM, int ACC, int VAR>
__global__ void __launch_bounds__(kVecThreads, UpdShape<VAR>::MINB)
    cg_update32_gs_row4_kernel(float* __restrict__ x, float* __restrict__ r,
                               const float* __restrict__ p, const float* __restrict__ w,
                               const uint8_t* __restrict__ cw, const float* __restrict__ minv,
                               const uint8_t* __restrict__ faces, int64_t kx, int64_t kxky,
                               int64_t L, PcgScalars* __restrict__ s,
                               double* __restrict__ partials, double* __restrict__ hist,
                               int l2h) {
  constexpr int GPT = UpdShape<VAR>::GPT;
  using I = typename UpdShape<VAR>::I;
  // n % 4 == 0: the dot weights from the node positions, not from the 1-byte
  // codes (one load and four reciprocals less per group; measured 1.6 % at
  // N = 7, 3.5 % at N = 11)
  constexpr bool kPos = n % 4 == 0;
  __shared__ double sh[kVecThreads / 32];
  if (s->done) return;
  const float alpha = (float)s->alpha;
  DotAcc<float, DM> a_rr, a_rz;
  const I n4 = (I)(L >> 2);   // L = E n^3 is a multiple of 4 here
  const I stride = (I)gridDim.x * (I)blockDim.x;
  // with l2h the streams go through L2 evict-first, leaving w (written by
  // the operator evict-last) resident for the gathers
  const uint64_t pol = l2h ? l2_policy_evict_first() : 0ull;
  struct Grp {
    float4 x, r, p, m, w, wt;
    uchar4 c;
  };
  auto load = [&](I q) {
    Grp g;
    if (l2h) {
      g.x = ld_hint4_rw(reinterpret_cast<const float4*>(x) + q, pol);
      g.r = ld_hint4_rw(reinterpret_cast<const float4*>(r) + q, pol);
      g.p = ld_hint4(reinterpret_cast<const float4*>(p) + q, pol);
      g.m = ld_hint4(reinterpret_cast<const float4*>(minv) + q, pol);
      if constexpr (!kPos) g.c = ld_hint_u8x4(reinterpret_cast<const uchar4*>(cw) + q, pol);
    } else {
      g.x = reinterpret_cast<float4*>(x)[q];
      g.r = reinterpret_cast<float4*>(r)[q];
      g.p = __ldg(reinterpret_cast<const float4*>(p) + q);
      g.m = __ldg(reinterpret_cast<const float4*>(minv) + q);
      if constexpr (!kPos) g.c = __ldg(reinterpret_cast<const uchar4*>(cw) + q);
    }
    if constexpr (kPos) {
      const uint8_t f = __ldg(faces + q / (n * n * n / 4));
      g.w = gs_gather_row4_own<n, ACC, I>(w, q, f, __ldg(reinterpret_cast<const float4*>(w) + q),
                                          (I)kx, (I)kxky);
      g.wt = box_weights4<n, I>(q, f);
    } else if constexpr (n % 4 == 0) {
      g.w = gs_gather_row4<n, ACC>(w, q, faces, kx, kxky);
    } else {
      g.w = gs_gather_row2x2<n, ACC, I>(w, q, faces, (I)kx, (I)kxky);
    }
    return g;
  };
  auto finish = [&](I q, Grp g) {
    float4 xv = g.x, rv = g.r;
    const float4 pv = g.p, wv = g.w, mv = g.m;
    float4 wt;
    if constexpr (kPos) {
      wt = g.wt;
    } else {
      wt = make_float4(weight_of(g.c.x), weight_of(g.c.y), weight_of(g.c.z), weight_of(g.c.w));
    }
    xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
    rv.x -= alpha * wv.x; rv.y -= alpha * wv.y; rv.z -= alpha * wv.z; rv.w -= alpha * wv.w;
    if (l2h) {
      st_hint4(reinterpret_cast<float4*>(x) + q, xv, pol);
      st_hint4(reinterpret_cast<float4*>(r) + q, rv, pol);
    } else {
      reinterpret_cast<float4*>(x)[q] = xv;
      reinterpret_cast<float4*>(r)[q] = rv;
    }
    float c;
    c = wt.x * rv.x; a_rr.add(c, rv.x); a_rz.add(c, mv.x * rv.x);
    c = wt.y * rv.y; a_rr.add(c, rv.y); a_rz.add(c, mv.y * rv.y);
    c = wt.z * rv.z; a_rr.add(c, rv.z); a_rz.add(c, mv.z * rv.z);
    c = wt.w * rv.w; a_rr.add(c, rv.w); a_rz.add(c, mv.w * rv.w);
  };
  for (I q = (I)blockIdx.x * (I)blockDim.x + (I)threadIdx.x; q < n4; q += GPT * stride) {
    if constexpr (UpdShape<VAR>::PREFETCH) {
      const I qn = q + stride;
      if (qn < n4) {
        prefetch_l2(reinterpret_cast<const float4*>(x) + qn);
        prefetch_l2(reinterpret_cast<const float4*>(r) + qn);
        prefetch_l2(reinterpret_cast<const float4*>(p) + qn);
        prefetch_l2(reinterpret_cast<const float4*>(minv) + qn);
        prefetch_l2(reinterpret_cast<const float4*>(w) + qn);
      }
    }
    if constexpr (GPT == 1) {
      finish(q, load(q));
    } else {
      const I q2 = q + stride;
      const bool two = q2 < n4;
      const Grp g1 = load(q);
      Grp g2 = g1;
      if (two) g2 = load(q2);
      finish(q, g1);
      if (two) finish(q2, g2);
    }
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[1])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      finish_iteration(s, rtr, rtz, hist);
      s->counter[1] = 0u;
    }
  }
}

// r = b - Ax (Ax may be null: r = b); rtr, rtz, ||b||_c; initialises the scalars.
template <typename T, int DM>
__global__ void __launch_bounds__(kVecThreads)
    cg_init_kernel(T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ ax,
                   const T* __restrict__ c, const T* __restrict__ minv, int64_t L,
                   PcgScalars* __restrict__ s, double* __restrict__ partials,
                   double* __restrict__ hist) {
  __shared__ double sh[kVecThreads / 32];
  DotAcc<T, DM> a_rr, a_rz, a_bb;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    const T bv = b[l];
    const T rv = ax ? bv - ax[l] : bv;
    r[l] = rv;
    const T cr = c[l] * rv;
    a_rr.add(cr, rv);
    a_rz.add(cr, minv[l] * rv);
    a_bb.add(c[l] * bv, bv);
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double v2 = block_sum<DM>(a_bb.value(), sh);
  const double vals[3] = {v0, v1, v2};
  if (publish_and_elect(vals, 3, partials, &s->counter[2])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    const double bb = reduce_partials<DM>(partials, 2, sh);
    if (threadIdx.x == 0) {
      s->rtr = rtr;
      s->rtz = rtz;
      s->rtz_old = 0.0;
      s->beta = 0.0;
      s->alpha = 0.0;
      s->pap = 0.0;
      s->iter = 0;
      s->status = 0;
      s->best_rtr = rtr;
      s->best_it = 0;
      const double bnorm = sqrt(bb);
      s->bnorm = bnorm;
      s->relres = bnorm > 0.0 ? sqrt(rtr) / bnorm : 0.0;
      if (hist) hist[0] = s->relres;
      s->done = (bnorm == 0.0) || (!s->fixed && s->relres <= s->tol) || s->maxit <= 0;
      s->counter[2] = 0u;
    }
  }
}

// Residual replacement (reliable update) of the FP32 recursion: r32 takes
// the FP64 true residual r64 rounded once, rtz/rtr are recomputed from it,
// beta is recomputed from the new rtz, and the search direction p is kept,
// so CG continues instead of restarting.
template <int DM>
__global__ void __launch_bounds__(kVecThreads)
    cg_replace_kernel(const double* __restrict__ r64, float* __restrict__ r32,
                      const float* __restrict__ c, const float* __restrict__ minv, int64_t L,
                      double tol, PcgScalars* __restrict__ s, double* __restrict__ partials) {
  __shared__ double sh[kVecThreads / 32];
  DotAcc<float, DM> a_rr, a_rz;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    const float rv = (float)r64[l];
    r32[l] = rv;
    const float cr = c[l] * rv;
    a_rr.add(cr, rv);
    a_rz.add(cr, minv[l] * rv);
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[2])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      s->rtr = rtr;
      s->relres = sqrt(rtr) / s->bnorm;
      s->beta = s->iter > 0 ? rtz / s->rtz_old : 0.0;
      s->rtz = rtz;
      s->tol = tol;
      s->best_rtr = rtr;
      s->best_it = s->iter;
      s->status = 0;
      s->done = s->iter >= s->maxit ? 1 : 0;
      s->counter[2] = 0u;
    }
  }
}

__global__ void set_bnorm_kernel(PcgScalars* s, double bnorm, double* hist) {
  s->bnorm = bnorm;
  s->relres = bnorm > 0.0 ? sqrt(s->rtr) / bnorm : 0.0;
  if (hist) hist[s->iter] = s->relres;
  s->done = (bnorm == 0.0) || (!s->fixed && s->relres <= s->tol) || s->maxit <= 0;
}

template <typename T, int DM>
__global__ void __launch_bounds__(kVecThreads)
    glsc3_kernel(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c,
                 int64_t L, double* __restrict__ partials, unsigned int* counter,
                 double* __restrict__ out) {
  __shared__ double sh[kVecThreads / 32];
  DotAcc<T, DM> acc;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    acc.add(c[l] * a[l], b[l]);
  const double v = block_sum<DM>(acc.value(), sh);
  const double vals[1] = {v};
  if (publish_and_elect(vals, 1, partials, counter)) {
    const double t = reduce_partials<DM>(partials, 0, sh);
    if (threadIdx.x == 0) {
      *out = t;
      *counter = 0u;
    }
  }
}

// ------------------------------------------------------------------ refinement helpers
__global__ void cast_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    b[l] = (float)a[l];
}

__global__ void add_f32_to_f64(double* __restrict__ x, const float* __restrict__ d, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    x[l] += (double)d[l];
}

__global__ void masked_copy_f64(const double* __restrict__ src, const double* __restrict__ mask,
                                double* __restrict__ dst, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    dst[l] = src ? src[l] * mask[l] : 0.0;
}

__global__ void masked_copy_f32(const double* __restrict__ src, const double* __restrict__ mask,
                                float* __restrict__ dst, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    dst[l] = src ? (float)(src[l] * mask[l]) : 0.f;
}

__global__ void f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t L) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    b[l] = (double)a[l];
}

__global__ void scal_setup_kernel(PcgScalars* s, double tol, int maxit, int fixed, int stag) {
  // s->err is left alone: it reports a bounded wait that gave up
  s->tol = tol;
  s->maxit = maxit;
  s->fixed = fixed;
  s->stag_window = stag;
  s->done = 0;
  s->status = 0;
  s->iter = 0;
  for (int q = 0; q < 4; ++q) s->counter[q] = 0u;
}

// ------------------------------------------------------------------ launchers
int launch_scal_setup(Handle& h, PcgScalars* s, double tol, int maxit, int fixed, int stag_window) {
  scal_setup_kernel<<<1, 1, 0, h.stream>>>(s, tol, maxit, fixed, stag_window);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int vec_grid(const Handle& h, int64_t L) {
  int64_t g = (L + kVecThreads - 1) / kVecThreads;
  int64_t cap = (int64_t)h.num_sms * 8;   // 8 resident blocks of 256 threads per SM
  if (cap > h.max_blocks) cap = h.max_blocks;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
static int update_t(Handle& h, int dm, T* x, T* r, const T* p, const T* w, const T* c,
                    const T* minv, PcgScalars* s, double* hist) {
  const int grid = vec_grid(h, h.L);
  const bool vec_ok = ((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)w |
                       (uintptr_t)minv) % 16 == 0;
  if (dm == kDotFP32) {
    if constexpr (sizeof(T) == 4) {
      if (vec_ok)
        cg_update32_v4_kernel<kDotFP32><<<grid, kVecThreads, 0, h.stream>>>(
            x, r, p, w, h.cw8, minv, h.L, s, h.partials, hist);
      else
        cg_update_kernel<float, kDotFP32><<<grid, kVecThreads, 0, h.stream>>>(
            x, r, p, w, c, minv, h.L, s, h.partials, hist);
    }
  } else if (sizeof(T) == 4) {
    if constexpr (sizeof(T) == 4) {
      if (vec_ok)
        cg_update32_v4_kernel<kDotDot2><<<grid, kVecThreads, 0, h.stream>>>(
            x, r, p, w, h.cw8, minv, h.L, s, h.partials, hist);
      else
        cg_update_kernel<float, kDotDot2><<<grid, kVecThreads, 0, h.stream>>>(
            x, r, p, w, c, minv, h.L, s, h.partials, hist);
    }
  } else {
    if constexpr (sizeof(T) == 8)
      cg_update_kernel<double, kDotFP64><<<grid, kVecThreads, 0, h.stream>>>(
          x, r, p, w, c, minv, h.L, s, h.partials, hist);
  }
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_cg_update64(Handle& h, double* x, double* r, const double* p, const double* w,
                       PcgScalars* s, double* hist) {
  return update_t<double>(h, kDotFP64, x, r, p, w, h.c64, h.minv64, s, hist);
}
int launch_cg_update32(Handle& h, int dm, float* x, float* r, const float* p, const float* w,
                       const float* minv, PcgScalars* s, double* hist) {
  return update_t<float>(h, dm, x, r, p, w, h.c32, minv, s, hist);
}

// Fold QQ^T into the update on box meshes; by default for even n, where
// whole float4 rows (n a multiple of 4) or float2 pairs (n = 2, 6, 10, 14)
// can be gathered: the per-node gather of odd orders measured slower than
// the separate pass.
// ---------------------------------------------------------------------------
// Staged folded update (n = 8): the streams x, r, p, J^{-1}, w and the
// multiplicity code of a group of EPB elements are brought into shared
// memory by 1-D bulk copies, two stages deep, while the block works on the
// previous group (the operator's pipeline: mbarrier completion, bounded
// waits); only the other copies of shared nodes are read directly.  Same
// arithmetic per value as cg_update32_gs_row4_kernel; the dot partial sums
// follow the element groups instead of the grid-stride order.
template <int n>
struct UpdTmaShape {
  static constexpr int n3 = n * n * n, G4 = n3 / 4;
  static constexpr int EPB = 256 / G4 >= 1 ? 256 / G4 : 1;
  static constexpr int NT = EPB * G4;
  static constexpr int NS = 2;
  static constexpr int SV = EPB * n3;                 // floats of one vector per stage
  static constexpr size_t STAGE_BYTES = 5 * 4 * (size_t)SV + SV;   // x, r, p, J^-1, w + code
  static constexpr size_t SMEM = NS * STAGE_BYTES + NS * 8 + 16;
};

template <int n, int DM, int ACC>
__global__ void __launch_bounds__(UpdTmaShape<n>::NT, 4)
    cg_update32_tma_kernel(float* __restrict__ x, float* __restrict__ r,
                           const float* __restrict__ p, const float* __restrict__ w,
                           const uint8_t* __restrict__ cw, const float* __restrict__ minv,
                           const uint8_t* __restrict__ faces, int64_t E, int64_t kx,
                           int64_t kxky, PcgScalars* __restrict__ s,
                           double* __restrict__ partials, double* __restrict__ hist,
                           int* __restrict__ err) {
  using Sh = UpdTmaShape<n>;
  constexpr int n3 = Sh::n3, G4 = Sh::G4, EPB = Sh::EPB, NS = Sh::NS, SV = Sh::SV;
  extern __shared__ __align__(128) unsigned char upd_smem[];
  float* const fbuf = reinterpret_cast<float*>(upd_smem);                 // [NS][5][SV]
  uint8_t* const cbuf = upd_smem + (size_t)NS * 5 * SV * 4;               // [NS][SV]
  uint64_t* const bar = reinterpret_cast<uint64_t*>(cbuf + (size_t)NS * SV);
  __shared__ double sh[Sh::NT / 32];
  if (s->done) return;
  const float alpha = (float)s->alpha;
  DotAcc<float, DM> a_rr, a_rz;
  const int tid = threadIdx.x;
  const int64_t ngroups = (E + EPB - 1) / EPB;

  auto issue = [&](int st, int64_t g) {
    const int64_t e0 = g * EPB;
    const int64_t cnt = E - e0 < EPB ? E - e0 : EPB;
    const uint32_t vb = (uint32_t)(cnt * n3 * 4), cb = (uint32_t)(cnt * n3);
    float* dst = fbuf + (size_t)st * 5 * SV;
    mbar_arrive_expect_tx(&bar[st], 5 * vb + cb);
    bulk_load(dst, x + e0 * n3, vb, &bar[st]);
    bulk_load(dst + SV, r + e0 * n3, vb, &bar[st]);
    bulk_load(dst + 2 * SV, p + e0 * n3, vb, &bar[st]);
    bulk_load(dst + 3 * SV, minv + e0 * n3, vb, &bar[st]);
    bulk_load(dst + 4 * SV, w + e0 * n3, vb, &bar[st]);
    bulk_load(cbuf + (size_t)st * SV, cw + e0 * n3, cb, &bar[st]);
  };

  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      const int64_t g0 = (int64_t)blockIdx.x + (int64_t)q * gridDim.x;
      if (g0 < ngroups) issue(q, g0);
    }
  }
  const int le = tid / G4, gq = tid - le * G4;
  bool aborted = false;
  int t = 0;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, ++t) {
    const int st = t % NS;
    const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((t / NS) & 1));
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    const int64_t e = g * EPB + le;
    if (e < E) {
      const float* sb = fbuf + (size_t)st * 5 * SV + le * n3 + 4 * gq;
      float4 xv = *reinterpret_cast<const float4*>(sb);
      float4 rv = *reinterpret_cast<const float4*>(sb + SV);
      const float4 pv = *reinterpret_cast<const float4*>(sb + 2 * SV);
      const float4 mv = *reinterpret_cast<const float4*>(sb + 3 * SV);
      const float4 own = *reinterpret_cast<const float4*>(sb + 4 * SV);
      const uchar4 cv =
          *reinterpret_cast<const uchar4*>(cbuf + (size_t)st * SV + le * n3 + 4 * gq);
      const int64_t q = e * G4 + gq;
      const float4 wv = gs_gather_row4_own<n, ACC>(w, q, __ldg(faces + e), own, kx, kxky);
      xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
      rv.x -= alpha * wv.x; rv.y -= alpha * wv.y; rv.z -= alpha * wv.z; rv.w -= alpha * wv.w;
      reinterpret_cast<float4*>(x)[q] = xv;
      reinterpret_cast<float4*>(r)[q] = rv;
      float c;
      c = weight_of(cv.x) * rv.x; a_rr.add(c, rv.x); a_rz.add(c, mv.x * rv.x);
      c = weight_of(cv.y) * rv.y; a_rr.add(c, rv.y); a_rz.add(c, mv.y * rv.y);
      c = weight_of(cv.z) * rv.z; a_rr.add(c, rv.z); a_rz.add(c, mv.z * rv.z);
      c = weight_of(cv.w) * rv.w; a_rr.add(c, rv.w); a_rz.add(c, mv.w * rv.w);
    }
    __syncthreads();   // stage st is free again
    if (tid == 0) {
      const int64_t gn = g + NS * (int64_t)gridDim.x;
      if (gn < ngroups) {
        fence_proxy_async_smem();
        issue(st, gn);
      }
    }
  }

  if (aborted) {
    // A bulk copy never completed: report it, give the copies this block
    // still has in flight a bounded time to land, and leave without
    // publishing a partial sum.
    if (tid == 0) {
      atomicExch(err, 1);
      const int64_t g_abort = blockIdx.x + (int64_t)t * gridDim.x;
      for (int s2 = 0; s2 < NS; ++s2) {
        const int64_t g_out = g_abort + (int64_t)((s2 - t % NS + NS) % NS) * gridDim.x;
        const int done_uses = t > s2 ? (t - 1 - s2) / NS + 1 : 0;
        if (g_out < ngroups) mbar_wait_bounded(&bar[s2], (uint32_t)(done_uses & 1));
      }
    }
    return;
  }
  const double v0 = block_sum<DM>(a_rr.value(), sh);
  const double v1 = block_sum<DM>(a_rz.value(), sh);
  const double vals[2] = {v0, v1};
  if (publish_and_elect(vals, 2, partials, &s->counter[1])) {
    const double rtr = reduce_partials<DM>(partials, 0, sh);
    const double rtz = reduce_partials<DM>(partials, 1, sh);
    if (threadIdx.x == 0) {
      finish_iteration(s, rtr, rtz, hist);
      s->counter[1] = 0u;
    }
  }
}

template <int DM, int ACC>
static int update_tma_launch(Handle& h, float* x, float* r, const float* p, const float* w,
                             const float* minv, PcgScalars* s, double* hist) {
  using Sh = UpdTmaShape<8>;
  auto kern = cg_update32_tma_kernel<8, DM, ACC>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::NT, Sh::SMEM));
  const int64_t groups = (h.E + Sh::EPB - 1) / Sh::EPB;
  int64_t cap = (int64_t)h.num_sms * std::max(per_sm, 1);
  if (cap > h.max_blocks) cap = h.max_blocks;
  const int grid = (int)std::max<int64_t>(1, std::min(groups, cap));
  kern<<<grid, Sh::NT, Sh::SMEM, h.stream>>>(x, r, p, w, h.cw8, minv, h.bfaces, h.E, h.kx,
                                             (int64_t)h.kx * h.ky, s, h.partials, hist,
                                             h.dev_err);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

bool gs_fusable(const Handle& h) {
  if (h.gid_user || h.n < 2 || h.fuse_gs == 0) return false;
  return h.fuse_gs == 2 || h.n % 2 == 0;
}

// Grid of a fused update kernel: the v4 update's grid (one thread per DOF,
// capped) with the cap set by the kernel's own occupancy.  Where the cap
// does not bind -- small problems -- the two kernels traverse the vectors
// identically, so their dot products agree bit for bit.
template <typename K>
static int fused_grid(Handle& h, K kernel, int slot) {
  if (h.upd_gs_occ[slot] == 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kVecThreads, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    h.upd_gs_occ[slot] = occ;
  }
  int64_t g = (h.L + kVecThreads - 1) / kVecThreads;
  int64_t cap = (int64_t)h.num_sms * h.upd_gs_occ[slot];
  if (cap > h.max_blocks) cap = h.max_blocks;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <int DM, int ACC>
static void update_gs_dispatch(Handle& h, float* x, float* r, const float* p, const float* w,
                               const float* minv, PcgScalars* s, double* hist, int slot) {
  const int64_t kx = h.kx, kxky = (int64_t)h.kx * h.ky;
  // 32-bit indices: every value index the kernel forms (float4, float2
  // and float indices of the vectors, past the end by at most one grid
  // stride of float4 groups; neighbour offsets are below L / 4) below 2^31
  const bool i32_ok = h.L + 4 * (int64_t)h.max_blocks * kVecThreads < ((int64_t)1 << 31);
  int uv = h.upd_variant;
  if (!i32_ok && (uv == 0 || uv == 5)) uv = uv == 0 ? 4 : 1;   // the 64-bit form
  if (h.upd_tma && h.n == 8) {
    // bulk-copy staged variant (its launch errors surface at the next check)
    update_tma_launch<DM, ACC>(h, x, r, p, w, minv, s, hist);
    return;
  }
#define SEM_UPD_ROW4(NN)                                                                  \
  case NN: {                                                                              \
    auto kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 0>;                               \
    if (uv == 1) kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 1>;                       \
    if (uv == 2) kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 2>;                       \
    if (uv == 3) kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 3>;                       \
    if (uv == 4) kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 4>;                       \
    if (uv == 5) kern = cg_update32_gs_row4_kernel<NN, DM, ACC, 5>;                       \
    const int grid = fused_grid(h, kern, slot + 4 * uv);                                  \
    kern<<<grid, kVecThreads, 0, h.stream>>>(x, r, p, w, h.cw8, minv, h.bfaces, kx, kxky, \
                                             h.L, s, h.partials, hist, h.l2_hints ? 1 : 0); \
    return;                                                                               \
  }
  switch (h.n) {
    SEM_UPD_ROW4(2)
    SEM_UPD_ROW4(4)
    SEM_UPD_ROW4(6)
    SEM_UPD_ROW4(8)
    SEM_UPD_ROW4(10)
    SEM_UPD_ROW4(12)
    SEM_UPD_ROW4(14)
    SEM_UPD_ROW4(16)
    default: break;
  }
#undef SEM_UPD_ROW4
  BoxNbr b{h.n, h.n * h.n * h.n, kx, kxky};
  auto kern = cg_update32_gs_kernel<DM, ACC>;
  const int grid = fused_grid(h, kern, slot);
  kern<<<grid, kVecThreads, 0, h.stream>>>(x, r, p, w, h.cw8, minv, h.bfaces, b, h.L, s,
                                           h.partials, hist);
}

// x += alpha p, r -= alpha QQ^T w with the summation folded in (box meshes,
// FP32 data; `acc` as for the separate gather-scatter).
int launch_cg_update32_gs(Handle& h, int dm, int acc, float* x, float* r, const float* p,
                          const float* w, const float* minv, PcgScalars* s, double* hist) {
  if (((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)w | (uintptr_t)minv) % 16 != 0) {
    set_error("update: vectors must be 16-byte aligned");
    return SEM_EINVAL;
  }
  if (dm == kDotFP32)
    update_gs_dispatch<kDotFP32, kGsFP32>(h, x, r, p, w, minv, s, hist, 0);
  else if (acc == kGsFP64)
    update_gs_dispatch<kDotDot2, kGsFP64>(h, x, r, p, w, minv, s, hist, 1);
  else if (acc == kGsFP32)
    update_gs_dispatch<kDotDot2, kGsFP32>(h, x, r, p, w, minv, s, hist, 2);
  else
    update_gs_dispatch<kDotDot2, kGsTwoSum>(h, x, r, p, w, minv, s, hist, 3);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_cg_init64(Handle& h, double* r, const double* b, const double* ax, const double* minv,
                     PcgScalars* s, double* hist) {
  cg_init_kernel<double, kDotFP64><<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(
      r, b, ax, h.c64, minv, h.L, s, h.partials, hist);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}
int launch_cg_init32(Handle& h, int dm, float* r, const float* b, const float* ax,
                     const float* minv, PcgScalars* s, double* hist) {
  if (dm == kDotFP32)
    cg_init_kernel<float, kDotFP32><<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(
        r, b, ax, h.c32, minv, h.L, s, h.partials, hist);
  else
    cg_init_kernel<float, kDotDot2><<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(
        r, b, ax, h.c32, minv, h.L, s, h.partials, hist);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_glsc3(Handle& h, sem_precision p, const void* a, const void* b, double* out_dev) {
  const int grid = vec_grid(h, h.L);
  unsigned int* counter = &h.scal_aux->counter[3];
  if (p == SEM_FP64)
    glsc3_kernel<double, kDotFP64><<<grid, kVecThreads, 0, h.stream>>>(
        (const double*)a, (const double*)b, h.c64, h.L, h.partials_aux, counter, out_dev);
  else if (p == SEM_FP32_ALL)
    glsc3_kernel<float, kDotFP32><<<grid, kVecThreads, 0, h.stream>>>(
        (const float*)a, (const float*)b, h.c32, h.L, h.partials_aux, counter, out_dev);
  else
    glsc3_kernel<float, kDotDot2><<<grid, kVecThreads, 0, h.stream>>>(
        (const float*)a, (const float*)b, h.c32, h.L, h.partials_aux, counter, out_dev);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_cg_replace32(Handle& h, int dm, const double* r64, float* r32, const float* minv,
                        double tol, PcgScalars* s) {
  if (dm == kDotFP32)
    cg_replace_kernel<kDotFP32><<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(
        r64, r32, h.c32, minv, h.L, tol, s, h.partials);
  else
    cg_replace_kernel<kDotDot2><<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(
        r64, r32, h.c32, minv, h.L, tol, s, h.partials);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_set_bnorm(Handle& h, PcgScalars* s, double bnorm, double* hist) {
  set_bnorm_kernel<<<1, 1, 0, h.stream>>>(s, bnorm, hist);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

int launch_cast64to32(Handle& h, const double* a, float* b) {
  cast_f64_to_f32<<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(a, b, h.L);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}
int launch_cast32to64(Handle& h, const float* a, double* b) {
  f32_to_f64<<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(a, b, h.L);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}
int launch_add32to64(Handle& h, double* x, const float* d) {
  add_f32_to_f64<<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(x, d, h.L);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}
int launch_masked_copy64(Handle& h, const double* src, double* dst) {
  masked_copy_f64<<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(src, h.mask64, dst, h.L);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}
int launch_masked_copy32(Handle& h, const double* src, float* dst) {
  masked_copy_f32<<<vec_grid(h, h.L), kVecThreads, 0, h.stream>>>(src, h.mask64, dst, h.L);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace sem
