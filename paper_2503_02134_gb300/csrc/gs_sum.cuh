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

// n a multiple of 4: a float4 group lies inside one row of one element, so
// the copies across j and k faces are whole float4 rows of the neighbouring
// elements; only the copies across i faces (components 0 and 3) are single
// values.
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
  if (!(dy | dz) && !xm && !xp) return own;
  // row offsets (float4 units) of the copies across j / k faces
  const int64_t oy = (int64_t)dy * (kx * g4 - (int64_t)(n - 1) * row4);
  const int64_t oz = (int64_t)dz * (kxky * g4 - (int64_t)(n - 1) * n * row4);
  const int64_t ys[2] = {dy < 0 ? oy : 0, dy > 0 ? oy : 0};
  const int64_t zs[2] = {dz < 0 ? oz : 0, dz > 0 ? oz : 0};
  const int ny = dy ? 2 : 1, nz = dz ? 2 : 1;
  float4 R[4];
  float XM[4], XP[4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int t = 2 * a + c;
      if (a < nz && c < ny) {
        const int64_t ro = zs[a] + ys[c];
        R[t] = ro == 0 ? own : __ldg(w4 + q + ro);
        const int64_t l0 = 4 * (q + ro);
        XM[t] = xm ? __ldg(w + l0 - n3 + (n - 1)) : 0.f;
        XP[t] = xp ? __ldg(w + l0 + 3 + n3 - (n - 1)) : 0.f;
      }
    }
  GsSum<float, ACC> s0, s1, s2, s3;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int t = 2 * a + c;
      if (a < nz && c < ny) {
        if (xm) s0.add(XM[t]);
        s0.add(R[t].x);
        s1.add(R[t].y);
        s2.add(R[t].z);
        s3.add(R[t].w);
        if (xp) s3.add(XP[t]);
      }
    }
  float4 out;
  if (dy | dz) {
    out.y = s1.result();
    out.z = s2.result();
  } else {
    out.y = own.y;
    out.z = own.z;
  }
  out.x = (dy | dz) || xm ? s0.result() : own.x;
  out.w = (dy | dz) || xp ? s3.result() : own.w;
  return out;
}

}  // namespace sem
