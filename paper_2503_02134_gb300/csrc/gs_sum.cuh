// Accumulators of the direct-stiffness summation QQ^T (arXiv 2503.02134,
// Sec. 3.3): the sum of the local copies of a shared global node, taken in
// ascending local index.  The paper's finding is that this sum needs FP64
// for the mixed solver to converge; on FP32 data it is formed here either in
// FP64 or as an error-free FP32 TwoSum (Knuth) pair rounded once.
//
// Also the copy gathers of a box mesh, used where the summation is folded
// into the vector update (pcg_kernels.cu, batch.cu): a local entry finds the
// other copies of its node from its position -- across face i = 0 of
// element e lies node i = n-1 of element e-1 (when the face is not on the
// domain boundary), and likewise in j (element e -+ kx) and k (element
// e -+ kx ky); edges and corners take the products -- and sums them in
// ascending element order, i.e. ascending local index, the order of the
// separate gather-scatter pass.  Face bits f: set where the face of the
// element lies on the domain boundary (bit 0 r-, 1 r+, 2 s-, 3 s+, 4 t-, 5 t+).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sem {

enum GsAcc { kGsFP64 = 0, kGsFP32 = 1, kGsTwoSum = 2 };

template <typename T, int ACC>
struct GsSum;

template <typename T>
struct GsSum<T, kGsFP64> {
  double s = 0.0;
  __device__ __forceinline__ void add(T x) { s += (double)x; }
  __device__ __forceinline__ T result() const { return (T)s; }
};

template <>
struct GsSum<float, kGsFP32> {
  float s = 0.f;
  __device__ __forceinline__ void add(float x) { s = __fadd_rn(s, x); }
  __device__ __forceinline__ float result() const { return s; }
};

template <>
struct GsSum<float, kGsTwoSum> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ float result() const { return __fadd_rn(s, c); }
};

struct BoxNbr {
  int n, n3;
  int64_t kx, kxky;   // element index strides in y and z
};

// Sum of the copies of local node l (coordinates i, j, k in element e,
// face bits f: set where the face lies on the domain boundary).
template <int ACC>
__device__ __forceinline__ float gs_gather_node(const float* __restrict__ w, int64_t l, int i,
                                                int j, int k, uint8_t f, const BoxNbr& b) {
  const int n1 = b.n - 1;
  const int dx = (i == 0 && !(f & 1)) ? -1 : (i == n1 && !(f & 2)) ? 1 : 0;
  const int dy = (j == 0 && !(f & 4)) ? -1 : (j == n1 && !(f & 8)) ? 1 : 0;
  const int dz = (k == 0 && !(f & 16)) ? -1 : (k == n1 && !(f & 32)) ? 1 : 0;
  if (!(dx | dy | dz)) return __ldg(w + l);
  const int64_t ox = (int64_t)dx * (b.n3 - n1);
  const int64_t oy = (int64_t)dy * (b.kx * b.n3 - (int64_t)n1 * b.n);
  const int64_t oz = (int64_t)dz * (b.kxky * b.n3 - (int64_t)n1 * b.n * b.n);
  // each dimension contributes {0} or the ascending pair {min(0,d), max(0,d)}
  const int64_t xs[2] = {dx < 0 ? ox : 0, dx > 0 ? ox : 0};
  const int64_t ys[2] = {dy < 0 ? oy : 0, dy > 0 ? oy : 0};
  const int64_t zs[2] = {dz < 0 ? oz : 0, dz > 0 ? oz : 0};
  GsSum<float, ACC> acc;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (a == 1 && !dz) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 1 && !dy) break;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        if (d == 1 && !dx) break;
        acc.add(__ldg(w + l + zs[a] + ys[c] + xs[d]));
      }
    }
  }
  return acc.result();
}

// Sum of two copies a, b in that order with the accumulator's arithmetic:
// the value GsSum<float, ACC> gives after add(a), add(b).  (For TwoSum the
// error term of a two-term sum is the exact rounding error of fl(a' + b),
// a' = fl(0 + a), so the final rounding returns fl(a' + b) itself.)
template <int ACC>
__device__ __forceinline__ float gs_sum2(float a, float b) {
  if constexpr (ACC == kGsFP64) return (float)((0.0 + (double)a) + (double)b);
  return __fadd_rn(__fadd_rn(0.f, a), b);
}

// Copies of a float4 group lying on NC = 2 (one j or k face) or 4 (a j-k
// edge) rows: rows at float4 offsets ro[0] < ... < ro[NC-1] (one of them 0,
// the group itself), plus, where the group's first (last) value lies on an
// i face, the single values across it in each of those rows.
template <int NC, int n, int ACC, typename I = int64_t>
__device__ __forceinline__ float4 gs_gather_rows(const float* __restrict__ w, I q, const I* ro,
                                                 float4 own, bool xm, bool xp) {
  constexpr int n3 = n * n * n;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  float4 R[NC];
  float XM[NC], XP[NC];
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    R[t] = ro[t] == 0 ? own : __ldg(w4 + (q + ro[t]));
    const I l0 = 4 * (q + ro[t]);
    XM[t] = xm ? __ldg(w + l0 - n3 + (n - 1)) : 0.f;
    XP[t] = xp ? __ldg(w + l0 + 3 + n3 - (n - 1)) : 0.f;
  }
  GsSum<float, ACC> s0, s1, s2, s3;
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    if (xm) s0.add(XM[t]);
    s0.add(R[t].x);
    s1.add(R[t].y);
    s2.add(R[t].z);
    s3.add(R[t].w);
    if (xp) s3.add(XP[t]);
  }
  return make_float4(s0.result(), s1.result(), s2.result(), s3.result());
}

// n a multiple of 4: a float4 group lies inside one row of one element, so
// the copies across j and k faces are whole float4 rows of the neighbouring
// elements; only the copies across i faces (components 0 and 3) are single
// values.  Interior rows (no j or k face) take a short path.
// As gs_gather_row4 below, with the group's own values supplied by the
// caller (from shared memory in the staged update) and the element's face
// bits f.  I: the index type (32-bit where the caller has checked that
// every index of the vectors fits).
template <int n, int ACC, typename I = int64_t>
__device__ __forceinline__ float4 gs_gather_row4_own(const float* __restrict__ w, I q, uint8_t f,
                                                     float4 own, I kx, I kxky) {
  constexpr int n3 = n * n * n, g4 = n3 / 4, row4 = n / 4;
  const I e = q / g4;
  const int rem = (int)(q - e * g4);
  const int i0 = (rem % row4) * 4;
  const int j = (rem / row4) % n;
  const int k = rem / (row4 * n);
  const int dy = (j == 0 && !(f & 4)) ? -1 : (j == n - 1 && !(f & 8)) ? 1 : 0;
  const int dz = (k == 0 && !(f & 16)) ? -1 : (k == n - 1 && !(f & 32)) ? 1 : 0;
  const bool xm = i0 == 0 && !(f & 1);
  const bool xp = i0 + 3 == n - 1 && !(f & 2);
  if (!(dy | dz)) {
    float4 out = own;
    if (xm) out.x = gs_sum2<ACC>(__ldg(w + (4 * q - n3 + (n - 1))), own.x);
    if (xp) out.w = gs_sum2<ACC>(own.w, __ldg(w + (4 * q + 3 + n3 - (n - 1))));
    return out;
  }
  const I oy = (I)dy * (kx * g4 - (I)(n - 1) * row4);
  const I oz = (I)dz * (kxky * g4 - (I)(n - 1) * n * row4);
  if (dy && dz) {
    const I ylo = dy < 0 ? oy : 0, yhi = dy > 0 ? oy : 0;
    const I zlo = dz < 0 ? oz : 0, zhi = dz > 0 ? oz : 0;
    const I ro[4] = {zlo + ylo, zlo + yhi, zhi + ylo, zhi + yhi};
    return gs_gather_rows<4, n, ACC, I>(w, q, ro, own, xm, xp);
  }
  const I o = dy ? oy : oz;
  const I ro[2] = {o < 0 ? o : 0, o > 0 ? o : 0};
  return gs_gather_rows<2, n, ACC, I>(w, q, ro, own, xm, xp);
}

template <int n, int ACC>
__device__ __forceinline__ float4 gs_gather_row4(const float* __restrict__ w, int64_t q,
                                                 const uint8_t* __restrict__ faces,
                                                 int64_t kx, int64_t kxky) {
  constexpr int n3 = n * n * n, g4 = n3 / 4, row4 = n / 4;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  const int64_t e = q / g4;
  const int rem = (int)(q - e * g4);
  const int i0 = (rem % row4) * 4;
  const int j = (rem / row4) % n;
  const int k = rem / (row4 * n);
  const uint8_t f = __ldg(faces + e);
  const int dy = (j == 0 && !(f & 4)) ? -1 : (j == n - 1 && !(f & 8)) ? 1 : 0;
  const int dz = (k == 0 && !(f & 16)) ? -1 : (k == n - 1 && !(f & 32)) ? 1 : 0;
  const bool xm = i0 == 0 && !(f & 1);
  const bool xp = i0 + 3 == n - 1 && !(f & 2);
  const float4 own = __ldg(w4 + q);
  if (!(dy | dz)) {
    float4 out = own;
    if (xm) out.x = gs_sum2<ACC>(__ldg(w + 4 * q - n3 + (n - 1)), own.x);
    if (xp) out.w = gs_sum2<ACC>(own.w, __ldg(w + 4 * q + 3 + n3 - (n - 1)));
    return out;
  }
  // row offsets (float4 units) of the copies across j / k faces
  const int64_t oy = (int64_t)dy * (kx * g4 - (int64_t)(n - 1) * row4);
  const int64_t oz = (int64_t)dz * (kxky * g4 - (int64_t)(n - 1) * n * row4);
  if (dy && dz) {
    const int64_t ylo = dy < 0 ? oy : 0, yhi = dy > 0 ? oy : 0;
    const int64_t zlo = dz < 0 ? oz : 0, zhi = dz > 0 ? oz : 0;
    const int64_t ro[4] = {zlo + ylo, zlo + yhi, zhi + ylo, zhi + yhi};
    return gs_gather_rows<4, n, ACC>(w, q, ro, own, xm, xp);
  }
  const int64_t o = dy ? oy : oz;
  const int64_t ro[2] = {o < 0 ? o : 0, o > 0 ? o : 0};
  return gs_gather_rows<2, n, ACC>(w, q, ro, own, xm, xp);
}

// n even but not a multiple of 4 (6, 10, 14): a float4 group may straddle
// two rows, but its two float2 halves each lie inside one row (rows have an
// even length).  The copies of a float2 pair, as gs_gather_rows for float4:
// rows at float2 offsets ro[t], and single values across the i faces.
template <int NC, int n, int ACC, typename I = int64_t>
__device__ __forceinline__ float2 gs_gather_rows2(const float* __restrict__ w, I q2, const I* ro,
                                                  float2 own, bool xm, bool xp) {
  constexpr int n3 = n * n * n;
  const float2* w2 = reinterpret_cast<const float2*>(w);
  float2 R[NC];
  float XM[NC], XP[NC];
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    R[t] = ro[t] == 0 ? own : __ldg(w2 + (q2 + ro[t]));
    const I l0 = 2 * (q2 + ro[t]);
    XM[t] = xm ? __ldg(w + (l0 - n3 + (n - 1))) : 0.f;
    XP[t] = xp ? __ldg(w + (l0 + 1 + n3 - (n - 1))) : 0.f;
  }
  GsSum<float, ACC> s0, s1;
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    if (xm) s0.add(XM[t]);
    s0.add(R[t].x);
    s1.add(R[t].y);
    if (xp) s1.add(XP[t]);
  }
  return make_float2(s0.result(), s1.result());
}

// The summed copies of float2 pair q2 (element face bits f).
template <int n, int ACC, typename I = int64_t>
__device__ __forceinline__ float2 gs_gather_pair(const float* __restrict__ w, I q2, uint8_t f,
                                                 I kx, I kxky) {
  static_assert(n % 2 == 0, "float2 pairs need an even n");
  constexpr int n3 = n * n * n, g2 = n3 / 2, row2 = n / 2;
  const I e = q2 / g2;
  const int rem = (int)(q2 - e * g2);
  const int i0 = (rem % row2) * 2;
  const int j = (rem / row2) % n;
  const int k = rem / (row2 * n);
  const int dy = (j == 0 && !(f & 4)) ? -1 : (j == n - 1 && !(f & 8)) ? 1 : 0;
  const int dz = (k == 0 && !(f & 16)) ? -1 : (k == n - 1 && !(f & 32)) ? 1 : 0;
  const bool xm = i0 == 0 && !(f & 1);
  const bool xp = i0 + 1 == n - 1 && !(f & 2);
  const float2 own = __ldg(reinterpret_cast<const float2*>(w) + q2);
  if (!(dy | dz)) {
    float2 out = own;
    if (xm) out.x = gs_sum2<ACC>(__ldg(w + (2 * q2 - n3 + (n - 1))), own.x);
    if (xp) out.y = gs_sum2<ACC>(own.y, __ldg(w + (2 * q2 + 1 + n3 - (n - 1))));
    return out;
  }
  const I oy = (I)dy * (kx * g2 - (I)(n - 1) * row2);
  const I oz = (I)dz * (kxky * g2 - (I)(n - 1) * n * row2);
  if (dy && dz) {
    const I ylo = dy < 0 ? oy : 0, yhi = dy > 0 ? oy : 0;
    const I zlo = dz < 0 ? oz : 0, zhi = dz > 0 ? oz : 0;
    const I ro[4] = {zlo + ylo, zlo + yhi, zhi + ylo, zhi + yhi};
    return gs_gather_rows2<4, n, ACC, I>(w, q2, ro, own, xm, xp);
  }
  const I o = dy ? oy : oz;
  const I ro[2] = {o < 0 ? o : 0, o > 0 ? o : 0};
  return gs_gather_rows2<2, n, ACC, I>(w, q2, ro, own, xm, xp);
}

// The summed copies of float4 group q for n = 6, 10, 14: its two float2
// halves (both in element q / (n^3 / 4), since n^3 / 2 is even).
template <int n, int ACC, typename I = int64_t>
__device__ __forceinline__ float4 gs_gather_row2x2(const float* __restrict__ w, I q,
                                                   const uint8_t* __restrict__ faces, I kx,
                                                   I kxky) {
  constexpr int g4 = n * n * n / 4;
  const uint8_t f = __ldg(faces + q / g4);
  const float2 a = gs_gather_pair<n, ACC, I>(w, 2 * q, f, kx, kxky);
  const float2 b = gs_gather_pair<n, ACC, I>(w, 2 * q + 1, f, kx, kxky);
  return make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace sem
