// p-multigrid preconditioner with overlapping Schwarz smoothing.
//
// The paper runs Nekbone with and without its multigrid preconditioner
// (Sec. 3.1: `solveM` is 70 % of the time when enabled; Sec. 4: the square
// roots of the Schwarz weights must stay FP64 in the mixed version) but
// prints no algorithm.  Built here, for box meshes:
//
//  * levels: the same mesh at orders N, floor(N/2), ..., 1, each a handle of
//    its own (operator, gather-scatter, mask);
//  * transfer: prolongation = per-element tensor-product interpolation J
//    (coarse GLL basis at fine GLL nodes); restriction = its adjoint on
//    unique nodes, r_c = mask_c QQ^T_c (J^T x J^T x J^T)(r_f / mult_f);
//  * smoother: additive Schwarz over the elements extended by one node
//    layer (the (n+2)^3 block of the global node grid), each block solved by
//    fast diagonalisation of the separable operator A x B x B + B x A x B +
//    B x B x A built from 1-D GLL stiffness/mass on the extended 1-D grids
//    (element and neighbour lengths; at N = 1 the overlap node is held at
//    zero); block solutions summed with weights 1/sqrt(c), c = blocks
//    holding the node (computed in FP64, also for the FP32 smoother), and
//    damped by omega = 1/lambda_max(S A) from a power iteration;
//  * h-levels: below the N = 1 level, while kx, ky, kz are all even and their
//    halves at least 2, the N = 1 discretisation of the box with half as many
//    elements per direction (each coarse element holds 2 x 2 x 2 fine ones);
//    prolongation = trilinear interpolation of the coarse element's eight
//    vertex values, restriction its adjoint on unique nodes; same smoother;
//  * cycle: symmetric V-cycle; the coarsest level applies the smoother.
//
// The block sum is a gather over the blocks that hold a node, found from its
// grid position and summed in ascending element order, so every local copy
// of a node gets the same bits (no scatter, no atomics).  The mixed variant
// runs the cycle on FP32 data with the gather-scatter and block sums
// accumulated error-free (TwoSum) and the CG dots in Dot2.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gs_sum.cuh"
#include "pcg.cuh"

namespace sem {

int ax_dispatch_fp64(Handle& h, const double* u, double* w, const AxPrologue* pro);
int ax_dispatch_fp32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm);
int fp64_residual(Handle& h, const double* f, bool x_is_zero, double* relres, double* bnorm);

constexpr int kMgMaxM = kMaxn + 2;   // extended points per direction (n + 2)

struct MgLevel {
  Handle* h = nullptr;     // level 0: the solver's handle (not owned)
  bool owned = false;
  int N = 0, n = 0, m = 0;
  double* S64 = nullptr;   // [3][E][m*m], S_d(a, b) at a*m + b (column b = eigenvector b)
  float* S32 = nullptr;
  double* lam64 = nullptr;  // [3][E][m]
  float* lam32 = nullptr;
  uint8_t* act = nullptr;   // [3][E][m]: 1 where the extended index is an unknown
  double* wsq64 = nullptr;  // [L] 1/sqrt(blocks holding the node)
  float* wsq32 = nullptr;
  double omega = 1.0;
  bool h_to_next = false;   // the next coarser level is this mesh halved (both N = 1)
  double* J64 = nullptr;    // interpolation from the next coarser level: [n][nc]
  float* J32 = nullptr;
  // work vectors of this level (both precisions)
  double *r64 = nullptr, *z64 = nullptr, *t64 = nullptr, *w64 = nullptr, *ext64 = nullptr;
  float *r32 = nullptr, *z32 = nullptr, *t32 = nullptr, *w32 = nullptr, *ext32 = nullptr;
};

struct MgData {
  std::vector<MgLevel> lv;
  // outer-solve vectors
  double *p64 = nullptr, *zz64 = nullptr, *w64 = nullptr, *r64 = nullptr, *x64 = nullptr;
  float *p32 = nullptr, *zz32 = nullptr, *w32 = nullptr, *r32 = nullptr, *x32 = nullptr;
  double* dot = nullptr;    // device scalar of the dots
  double* dot_host = nullptr;
};

// ---------------------------------------------------------------- set-up

// Element lengths along r, s, t: distance between the centroids of the two
// opposite faces.  coords: x block, y block, z block of L values each.
__global__ void mg_lengths_kernel(const double* __restrict__ X, int64_t L, int64_t E, int n,
                                  double* __restrict__ len) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * E;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / E);
    const int64_t e = t - d * E;
    const int64_t n3 = (int64_t)n * n * n;
    double c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        int i0, j0, k0, i1, j1, k1;
        if (d == 0) { i0 = 0; i1 = n - 1; j0 = j1 = a; k0 = k1 = b; }
        else if (d == 1) { j0 = 0; j1 = n - 1; i0 = i1 = a; k0 = k1 = b; }
        else { k0 = 0; k1 = n - 1; i0 = i1 = a; j0 = j1 = b; }
        const int64_t l0 = e * n3 + i0 + n * (j0 + n * k0);
        const int64_t l1 = e * n3 + i1 + n * (j1 + n * k1);
        for (int q = 0; q < 3; ++q) {
          c0[q] += X[q * L + l0];
          c1[q] += X[q * L + l1];
        }
      }
    double s = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double dq = (c1[q] - c0[q]) / (n * n);
      s += dq * dq;
    }
    len[d * E + e] = sqrt(s);
  }
}

// Extended 1-D operators and their generalised eigenpairs, one thread per
// (direction, element).  Extended index 0 = the left neighbour's node N-1,
// 1..n = own nodes, n+1 = the right neighbour's node 1; assembled from the
// three 1-D elements with all other nodes at zero; indices that are not
// unknowns get identity rows.  B is diagonal, so A S = B S L with S^T B S = I
// reduces to the symmetric eigenproblem of B^{-1/2} A B^{-1/2}, solved by
// cyclic Jacobi rotations (Golub & Van Loan, Sec. 8.5).
__global__ void mg_fdm_kernel(int N, int kx, int ky, int kz, int64_t E,
                              const double* __restrict__ D, const double* __restrict__ wq,
                              const double* __restrict__ len, double* __restrict__ S64,
                              float* __restrict__ S32, double* __restrict__ lam64,
                              float* __restrict__ lam32, uint8_t* __restrict__ act) {
  const int n = N + 1, m = n + 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * E;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / E);
    const int64_t e = t - d * E;
    const int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
    const int c = d == 0 ? ex : d == 1 ? ey : ez;
    const int kd = d == 0 ? kx : d == 1 ? ky : kz;
    const int64_t stride = d == 0 ? 1 : d == 1 ? kx : (int64_t)kx * ky;
    const bool hl_ok = c > 0, hr_ok = c < kd - 1;
    const double h = len[d * E + e];
    const double hl = hl_ok ? len[d * E + e - stride] : h;
    const double hr = hr_ok ? len[d * E + e + stride] : h;
    double A[kMgMaxM][kMgMaxM];
    double V[kMgMaxM][kMgMaxM];
    double B[kMgMaxM];
    for (int a = 0; a < m; ++a) {
      B[a] = 0.0;
      for (int b = 0; b < m; ++b) A[a][b] = 0.0;
    }
    // Ahat(a, b) = sum_q D(q, a) w_q D(q, b)
    auto ahat = [&](int a, int b) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += D[q * n + a] * wq[q] * D[q * n + b];
      return s;
    };
    for (int a = 0; a < n; ++a) {
      for (int b = 0; b < n; ++b) A[1 + a][1 + b] += (2.0 / h) * ahat(a, b);
      B[1 + a] += 0.5 * h * wq[a];
    }
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 2; ++b) {
        A[a][b] += (2.0 / hl) * ahat(N - 1 + a, N - 1 + b);
        A[n + a][n + b] += (2.0 / hr) * ahat(a, b);
      }
      B[a] += 0.5 * hl * wq[N - 1 + a];
      B[n + a] += 0.5 * hr * wq[a];
    }
    bool on[kMgMaxM];
    for (int a = 0; a < m; ++a) on[a] = true;
    on[0] = hl_ok && N >= 2;
    on[1] = hl_ok;
    on[n] = hr_ok;
    on[n + 1] = hr_ok && N >= 2;
    for (int a = 0; a < m; ++a) {
      if (on[a]) continue;
      for (int b = 0; b < m; ++b) A[a][b] = A[b][a] = 0.0;
      A[a][a] = 1.0;
      B[a] = 1.0;
    }
    double bi[kMgMaxM];
    for (int a = 0; a < m; ++a) bi[a] = 1.0 / sqrt(B[a]);
    double nrm = 0.0;
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        A[a][b] *= bi[a] * bi[b];
        V[a][b] = a == b ? 1.0 : 0.0;
        nrm += A[a][b] * A[a][b];
      }
    for (int sweep = 0; sweep < 60; ++sweep) {
      double off = 0.0;
      for (int p = 0; p < m; ++p)
        for (int q = p + 1; q < m; ++q) off += A[p][q] * A[p][q];
      if (off <= 1e-32 * nrm) break;
      for (int p = 0; p < m; ++p)
        for (int q = p + 1; q < m; ++q) {
          const double apq = A[p][q];
          if (apq == 0.0) continue;
          const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
          const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
          for (int k = 0; k < m; ++k) {   // columns p, q
            const double akp = A[k][p], akq = A[k][q];
            A[k][p] = cs * akp - sn * akq;
            A[k][q] = sn * akp + cs * akq;
          }
          for (int k = 0; k < m; ++k) {   // rows p, q
            const double apk = A[p][k], aqk = A[q][k];
            A[p][k] = cs * apk - sn * aqk;
            A[q][k] = sn * apk + cs * aqk;
          }
          for (int k = 0; k < m; ++k) {
            const double vkp = V[k][p], vkq = V[k][q];
            V[k][p] = cs * vkp - sn * vkq;
            V[k][q] = sn * vkp + cs * vkq;
          }
        }
    }
    const int64_t so = (d * E + e) * (int64_t)m * m, lo = (d * E + e) * (int64_t)m;
    for (int a = 0; a < m; ++a) {
      lam64[lo + a] = A[a][a];
      lam32[lo + a] = (float)A[a][a];
      act[lo + a] = on[a] ? 1 : 0;
      for (int b = 0; b < m; ++b) {
        const double v = bi[a] * V[a][b];
        S64[so + a * m + b] = v;
        S32[so + a * m + b] = (float)v;
      }
    }
  }
}

// Blocks holding the grid point at local index g (0..n-1) of element
// coordinate c along one direction: up to three candidates c' = c-1, c, c+1
// with extended index a' = c*N + g - c'*N + 1 in [0, n+1] and active.
struct MgCand {
  int cnt;
  int elem[3];   // element coordinate along the direction, ascending
  int ext[3];    // extended index in that element's block
};

__device__ __forceinline__ MgCand mg_candidates(int c, int g, int N, int kd, int64_t E,
                                                int64_t e_of_c0, int64_t stride,
                                                const uint8_t* __restrict__ actd) {
  // actd: act of this direction, [E][m]; e_of_c0: element index with this
  // direction's coordinate set to 0 (other coordinates as the node's element)
  MgCand r;
  r.cnt = 0;
  const int m = N + 3;
  for (int cc = c - 1; cc <= c + 1; ++cc) {
    if (cc < 0 || cc >= kd) continue;
    const int a = (c - cc) * N + g + 1;
    if (a < 0 || a >= m) continue;
    if (!actd[(e_of_c0 + (int64_t)cc * stride) * m + a]) continue;
    r.elem[r.cnt] = cc;
    r.ext[r.cnt] = a;
    ++r.cnt;
  }
  return r;
}

// 1/sqrt(number of blocks holding each local node), in FP64.
__global__ void mg_weights_kernel(int N, int kx, int ky, int kz, int64_t L,
                                  const uint8_t* __restrict__ act, double* __restrict__ w64,
                                  float* __restrict__ w32) {
  const int n = N + 1, n3 = n * n * n;
  const int64_t E = (int64_t)kx * ky * kz;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int rem = (int)(l - e * n3);
    const int i = rem % n, j = (rem / n) % n, k = rem / (n * n);
    const int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
    const int64_t m = N + 3;
    const MgCand cx = mg_candidates(ex, i, N, kx, E, e - ex, 1, act);
    const MgCand cy = mg_candidates(ey, j, N, ky, E, e - (int64_t)ey * kx, kx, act + E * m);
    const MgCand cz = mg_candidates(ez, k, N, kz, E, e - (int64_t)ez * kx * ky, (int64_t)kx * ky,
                                    act + 2 * E * m);
    const double c = (double)(cx.cnt * cy.cnt * cz.cnt);
    const double w = 1.0 / sqrt(c > 1.0 ? c : 1.0);
    w64[l] = w;
    w32[l] = (float)w;
  }
}

// ---------------------------------------------------------------- cycle kernels

// Block solve: gather the weighted residual on every element's extended
// block, apply S^T along each direction, divide by lam_x + lam_y + lam_z,
// apply S, write the block (inactive points zero).
// The same block solve with the order fixed at compile time: rows held in
// registers, contractions unrolled, EPB elements per CTA at low order.
template <int N>
struct MgShape {
  static constexpr int n = N + 1, m = n + 2, m2 = m * m, m3 = m2 * m, n3 = n * n * n;
  static constexpr int NT = 256;
  // rows per thread in the contraction passes: two when a block has an even
  // number of rows (each matrix entry read from shared memory feeds two FMAs)
  static constexpr int RPT = m2 % 2 == 0 ? 2 : 1;
  static constexpr int EPB = (RPT * NT / m2) > 0 ? (RPT * NT / m2) : 1;
  // shared-memory layout of a block: index a + P1 b + P2 c with an odd row
  // stride P1, so that threads on consecutive rows of any direction hit
  // distinct banks
  static constexpr int P1 = m % 2 == 0 ? m + 1 : m;
  static constexpr int P2 = P1 * m;
  static constexpr int BUF = P2 * m;
};

template <typename T, int N>
constexpr size_t mg_block_smem() {
  using Sh = MgShape<N>;
  return sizeof(T) * ((size_t)Sh::EPB * (Sh::BUF + 6 * Sh::m2 + 3 * Sh::m)) + 3 * Sh::EPB * Sh::m + 16;
}

// One contraction pass of the block solve along direction D: every row
// along D of every block in shared memory is replaced by (S^T row) when FWD
// or (S row); a thread holds RPT rows (r and r + m2/2 of one element).
template <typename T, int N, int D, bool FWD>
__device__ __forceinline__ void mg_pass(T* buf, const T* sT, const T* sS) {
  using Sh = MgShape<N>;
  constexpr int m = Sh::m, m2 = Sh::m2, EPB = Sh::EPB, P1 = Sh::P1, P2 = Sh::P2, BUF = Sh::BUF;
  constexpr int RPT = Sh::RPT, H = m2 / RPT;
  constexpr int step = D == 0 ? 1 : (D == 1 ? P1 : P2);
  for (int pr = threadIdx.x; pr < EPB * H; pr += blockDim.x) {
    const int le = pr / H, r0 = pr - le * H;
    T* bl[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int rr = r0 + q * H;
      const int u = rr % m, v2 = rr / m;
      const int base = D == 0 ? P1 * u + P2 * v2 : (D == 1 ? u + P2 * v2 : u + P1 * v2);
      bl[q] = buf + le * BUF + base;
    }
    // row o of S^T (forward) or of S (backward): contiguous in shared memory
    const T* Md = (FWD ? sT : sS) + le * 3 * m2 + D * m2;
    T in[RPT][m];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int t = 0; t < m; ++t) in[q][t] = bl[q][t * step];
#pragma unroll
    for (int o = 0; o < m; ++o) {
      T acc[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[q] = T(0);
#pragma unroll
      for (int t = 0; t < m; ++t) {
        const T mv = Md[o * m + t];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] += mv * in[q][t];
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) bl[q][o * step] = acc[q];
    }
  }
}

// The middle of the block solve in one pass over the rows along z: S_z^T,
// the division by lam_x + lam_y + lam_z (FP32: times the correctly rounded
// reciprocal), S_z -- the row stays in registers throughout.
template <typename T, int N>
__device__ __forceinline__ void mg_pass_z(T* buf, const T* sT, const T* sS, const T* sl) {
  using Sh = MgShape<N>;
  constexpr int m = Sh::m, m2 = Sh::m2, EPB = Sh::EPB, P1 = Sh::P1, P2 = Sh::P2, BUF = Sh::BUF;
  constexpr int RPT = Sh::RPT, H = m2 / RPT;
  for (int pr = threadIdx.x; pr < EPB * H; pr += blockDim.x) {
    const int le = pr / H, r0 = pr - le * H;
    T* bl[RPT];
    T lab[RPT];
    const T* L = sl + le * 3 * m;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int rr = r0 + q * H;
      const int a = rr % m, b = rr / m;
      bl[q] = buf + le * BUF + a + P1 * b;
      lab[q] = L[a] + L[m + b];
    }
    const T* Mf = sT + le * 3 * m2 + 2 * m2;   // rows of S_z^T
    const T* Mb = sS + le * 3 * m2 + 2 * m2;   // rows of S_z
    T v[RPT][m];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int t = 0; t < m; ++t) v[q][t] = bl[q][t * P2];
    T w[RPT][m];
#pragma unroll
    for (int o = 0; o < m; ++o) {
      T acc[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[q] = T(0);
#pragma unroll
      for (int t = 0; t < m; ++t) {
        const T mv = Mf[o * m + t];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] += mv * v[q][t];
      }
      const T lc = L[2 * m + o];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        if constexpr (sizeof(T) == 4) w[q][o] = acc[q] * __frcp_rn(lab[q] + lc);
        else w[q][o] = acc[q] / (lab[q] + lc);
      }
    }
#pragma unroll
    for (int o = 0; o < m; ++o) {
      T acc[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[q] = T(0);
#pragma unroll
      for (int t = 0; t < m; ++t) {
        const T mv = Mb[o * m + t];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] += mv * w[q][t];
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) bl[q][o * P2] = acc[q];
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(MgShape<N>::NT)
    mg_block_solve_t(int kx, int ky, int64_t E, const T* __restrict__ r, const T* __restrict__ wsq,
                     const T* __restrict__ S, const T* __restrict__ lam,
                     const uint8_t* __restrict__ act, T* __restrict__ ext) {
  using Sh = MgShape<N>;
  constexpr int n = Sh::n, m = Sh::m, m2 = Sh::m2, m3 = Sh::m3, n3 = Sh::n3, EPB = Sh::EPB;
  constexpr int P1 = Sh::P1, P2 = Sh::P2, BUF = Sh::BUF;
  extern __shared__ __align__(16) unsigned char mg_smem[];
  T* buf = reinterpret_cast<T*>(mg_smem);   // [EPB][BUF], point (a, b, c) at a + P1 b + P2 c
  T* sS = buf + EPB * BUF;                    // [EPB][3][m2]: S_d(a, b) at a*m + b
  T* sT = sS + EPB * 3 * m2;                  // [EPB][3][m2]: S_d(b, a) at a*m + b
  T* sl = sT + EPB * 3 * m2;                  // [EPB][3][m]
  uint8_t* sa = reinterpret_cast<uint8_t*>(sl + EPB * 3 * m);   // [EPB][3][m]
  const int64_t kxky = (int64_t)kx * ky;
  const int64_t ngroups = (E + EPB - 1) / EPB;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t e0 = g * EPB;
    for (int q = threadIdx.x; q < EPB * 3 * m2; q += blockDim.x) {
      const int le = q / (3 * m2), o = q - le * 3 * m2, d = o / m2, oo = o - d * m2;
      const int64_t e = e0 + le;
      const T v = e < E ? S[(d * E + e) * m2 + oo] : T(0);
      sS[q] = v;
      sT[le * 3 * m2 + d * m2 + (oo % m) * m + oo / m] = v;
    }
    for (int q = threadIdx.x; q < EPB * 3 * m; q += blockDim.x) {
      const int le = q / (3 * m), o = q - le * 3 * m, d = o / m, oo = o - d * m;
      const int64_t e = e0 + le;
      sl[q] = e < E ? lam[(d * E + e) * m + oo] : T(1);
      sa[q] = e < E ? act[(d * E + e) * m + oo] : 0;
    }
    __syncthreads();
    // gather by rows along x: extended row (b, c) is the neighbour's node
    // N-1, the n nodes of the element row (j, k) -- contiguous in memory --
    // and the next neighbour's node 1
    for (int row = threadIdx.x; row < EPB * m2; row += blockDim.x) {
      const int le = row / m2, rr = row - le * m2;
      const int b = rr % m, c = rr / m;
      const uint8_t* A = sa + le * 3 * m;
      T* out = buf + le * BUF + P1 * b + P2 * c;
      if (!(A[m + b] && A[2 * m + c]) || e0 + le >= E) {
#pragma unroll
        for (int a = 0; a < m; ++a) out[a] = T(0);
        continue;
      }
      const int dy = b == 0 ? -1 : (b == m - 1 ? 1 : 0);
      const int dz = c == 0 ? -1 : (c == m - 1 ? 1 : 0);
      const int j = b == 0 ? N - 1 : (b == m - 1 ? 1 : b - 1);
      const int k = c == 0 ? N - 1 : (c == m - 1 ? 1 : c - 1);
      const int64_t ee = e0 + le + (int64_t)dy * kx + (int64_t)dz * kxky;
      const int64_t l0 = ee * n3 + n * (j + n * k);     // node (0, j, k) of element ee
      const T* rp = r + l0;
      const T* wp = wsq + l0;
#pragma unroll
      for (int a = 1; a <= n; ++a)
        out[a] = A[a] ? rp[a - 1] * wp[a - 1] : T(0);
      // the x neighbours exist only where their extended index is active
      T lo = T(0), hi = T(0);
      if (A[0]) lo = rp[N - 1 - n3] * wp[N - 1 - n3];   // element ee-1, i = N-1
      if (A[m - 1]) hi = rp[1 + n3] * wp[1 + n3];       // element ee+1, i = 1
      out[0] = lo;
      out[m - 1] = hi;
    }
    __syncthreads();
    // contraction passes: S^T along x, y; then along z S^T, the eigenvalue
    // scaling and S in one pass; then S along y, x (the backward
    // contractions commute)
    mg_pass<T, N, 0, true>(buf, sT, sS);
    __syncthreads();
    mg_pass<T, N, 1, true>(buf, sT, sS);
    __syncthreads();
    mg_pass_z<T, N>(buf, sT, sS, sl);
    __syncthreads();
    mg_pass<T, N, 1, false>(buf, sT, sS);
    __syncthreads();
    mg_pass<T, N, 0, false>(buf, sT, sS);
    __syncthreads();
    // write the blocks (inactive points zero), by rows along x
    for (int row = threadIdx.x; row < EPB * m2; row += blockDim.x) {
      const int le = row / m2, rr = row - le * m2;
      const int b = rr % m, c = rr / m;
      const int64_t e = e0 + le;
      if (e >= E) continue;
      const uint8_t* A = sa + le * 3 * m;
      const bool on = A[m + b] && A[2 * m + c];
      const T* v = buf + le * BUF + P1 * b + P2 * c;
      T* out = ext + e * m3 + m * b + m2 * c;
#pragma unroll
      for (int a = 0; a < m; ++a) out[a] = (on && A[a]) ? v[a] : T(0);
    }
    __syncthreads();
  }
}

template <typename T, int N>
static int mg_block_solve_launch(Handle& h, const T* r, const T* wsq, const T* S, const T* lam,
                                 const uint8_t* act, T* ext) {
  using Sh = MgShape<N>;
  auto k = mg_block_solve_t<T, N>;
  constexpr size_t smem = mg_block_smem<T, N>();
  SEM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Sh::NT, smem));
  const int64_t groups = (h.E + Sh::EPB - 1) / Sh::EPB;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)h.num_sms * std::max(per_sm, 1)));
  k<<<grid, Sh::NT, smem, h.stream>>>(h.kx, h.ky, h.E, r, wsq, S, lam, act, ext);
  SEM_CUDA(cudaGetLastError());
  return 0;
}

template <typename T>
static int mg_block_solve_dispatch(Handle& h, const T* r, const T* wsq, const T* S, const T* lam,
                                   const uint8_t* act, T* ext) {
  switch (h.N) {
#define SEM_MG_N(NN) \
  case NN: return mg_block_solve_launch<T, NN>(h, r, wsq, S, lam, act, ext);
    SEM_MG_N(1) SEM_MG_N(2) SEM_MG_N(3) SEM_MG_N(4) SEM_MG_N(5) SEM_MG_N(6) SEM_MG_N(7)
    SEM_MG_N(8) SEM_MG_N(9) SEM_MG_N(10) SEM_MG_N(11) SEM_MG_N(12) SEM_MG_N(13) SEM_MG_N(14)
    SEM_MG_N(15)
#undef SEM_MG_N
    default:
      set_error("multigrid: order out of range");
      return SEM_EINVAL;
  }
}

// Blocks holding node g (0..N) of an element along one direction, from the
// element's face bits (lo/hi: the face on that side lies on the domain
// boundary): the lower neighbour's block at extended index n (g = 0) or n+1
// (g = 1, N >= 2), the element's own at g+1 (unless g is a boundary-face
// node), the upper neighbour's at 0 (g = N-1, N >= 2) or 1 (g = N); listed
// in ascending element order (offsets -1, 0, +1).
template <int N>
struct MgCand1 {
  int cnt;
  int off[3];
  int ext[3];
};

template <int N>
__device__ __forceinline__ MgCand1<N> mg_cand1(int g, bool lo_bnd, bool hi_bnd) {
  constexpr int n = N + 1;
  MgCand1<N> c;
  c.cnt = 0;
  if (!lo_bnd && g == 0) { c.off[c.cnt] = -1; c.ext[c.cnt++] = n; }
  if (!lo_bnd && N >= 2 && g == 1) { c.off[c.cnt] = -1; c.ext[c.cnt++] = n + 1; }
  if (!((g == 0 && lo_bnd) || (g == N && hi_bnd))) { c.off[c.cnt] = 0; c.ext[c.cnt++] = g + 1; }
  if (!hi_bnd && N >= 2 && g == N - 1) { c.off[c.cnt] = 1; c.ext[c.cnt++] = 0; }
  if (!hi_bnd && g == N) { c.off[c.cnt] = 1; c.ext[c.cnt++] = 1; }
  return c;
}

// Block sum with the order fixed at compile time.  The node's element
// coordinates give its boundary flags (a box mesh is Dirichlet on all six
// faces), so no load precedes the block loads; each thread sums four nodes
// per trip, whose loads are independent.
// Blocks holding node g along one direction, in three fixed slots (the
// lower neighbour's, the element's own, the upper neighbour's -- ascending
// element order): offsets into the block array (element stride es,
// extended-index stride xs) and whether the lower / upper slots are used.
template <int N>
struct MgSlots {
  int64_t lo, own, hi;
  bool has_lo, has_hi;
};

template <int N>
__device__ __forceinline__ MgSlots<N> mg_slots(int g, bool lo_bnd, bool hi_bnd, int64_t es,
                                               int xs) {
  constexpr int n = N + 1;
  MgSlots<N> r;
  r.own = (int64_t)(g + 1) * xs;                     // g is not a boundary node here
  r.has_lo = !lo_bnd && (g == 0 || (N >= 2 && g == 1));
  r.lo = -es + (int64_t)(g == 0 ? n : n + 1) * xs;
  r.has_hi = !hi_bnd && (g == N || (N >= 2 && g == N - 1));
  r.hi = es + (int64_t)(g == N ? 1 : 0) * xs;
  return r;
}

// Block sum by element rows: one thread per row (e, j, k), all n nodes of
// the row.  The y/z candidate blocks are the same for the whole row (no
// divergence between the nodes of a row), the x candidates are fixed per
// node index; each (z, y) combination contributes a contiguous row of the
// block array plus the two x-neighbour values.  Every copy of a node sums
// the same blocks in the same order (ascending element: lower, own, upper
// in z, then y, then x), so all copies get the same bits.
template <typename T, int ACC, int N>
__global__ void __launch_bounds__(256)
    mg_block_sum_rows(int kx, int ky, int64_t E, const uint8_t* __restrict__ faces,
                      const T* __restrict__ ext, const T* __restrict__ wsq, T omega,
                      int accumulate, T* __restrict__ z) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, m = n + 2, m2 = m * m, m3 = m2 * m;
  const int64_t rows = E * n2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / n2;
    const int jk = (int)(t - e * n2), j = jk % n, k = jk / n;
    const uint8_t f = __ldg(faces + e);
    const bool xl = f & 1, xh = f & 2, yl = f & 4, yh = f & 8, zl = f & 16, zh = f & 32;
    T* zr = z + e * n3 + n * jk;
    const T* wr = wsq + e * n3 + n * jk;
    const bool row_dirichlet = (j == 0 && yl) || (j == N && yh) || (k == 0 && zl) || (k == N && zh);
    T out[n];
    if (row_dirichlet) {
#pragma unroll
      for (int i = 0; i < n; ++i) out[i] = T(0);
    } else {
      const MgSlots<N> sy = mg_slots<N>(j, yl, yh, (int64_t)kx * m3, m);
      const MgSlots<N> sz = mg_slots<N>(k, zl, zh, (int64_t)kx * ky * m3, m2);
      const int64_t yo[3] = {sy.lo, sy.own, sy.hi}, zo[3] = {sz.lo, sz.own, sz.hi};
      const bool yu[3] = {sy.has_lo, true, sy.has_hi}, zu[3] = {sz.has_lo, true, sz.has_hi};
      GsSum<T, ACC> acc[n];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (!zu[c]) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (!yu[b]) continue;
          const T* rp = ext + e * m3 + zo[c] + yo[b];   // block row, extended index a = 0
#pragma unroll
          for (int i = 0; i < n; ++i) {
            if (i == 0 && !xl) acc[i].add(__ldg(rp - m3 + n));
            if (N >= 2 && i == 1 && !xl) acc[i].add(__ldg(rp - m3 + n + 1));
            acc[i].add(__ldg(rp + i + 1));
            if (N >= 2 && i == N - 1 && !xh) acc[i].add(__ldg(rp + m3));
            if (i == N && !xh) acc[i].add(__ldg(rp + m3 + 1));
          }
        }
      }
#pragma unroll
      for (int i = 0; i < n; ++i)
        out[i] = ((i == 0 && xl) || (i == N && xh)) ? T(0) : omega * (wr[i] * acc[i].result());
    }
#pragma unroll
    for (int i = 0; i < n; ++i) zr[i] = accumulate ? zr[i] + out[i] : out[i];
  }
}

// Transfers with the orders fixed at compile time: fine order NF, coarse
// order max(1, NF/2).  RESTRICT: out(coarse) = (J^T)^{x3}(in(fine) / m_f)
// with 1/m_f from the multiplicity code (exact: powers of two; 0 on the
// Dirichlet boundary, where in is zero); otherwise out(fine) += J^{x3} in(coarse).
template <int NF>
struct MgTransferShape {
  static constexpr int NC = NF / 2 > 1 ? NF / 2 : 1;
  static constexpr int nf = NF + 1, nc = NC + 1, nf3 = nf * nf * nf;
  // elements per CTA iteration: about 1024 fine values, so the loads and
  // the three contraction stages of several elements overlap
  static constexpr int EPB = 1024 / nf3 > 1 ? 1024 / nf3 : 1;
};

template <typename T, int NF, bool RESTRICT>
__global__ void __launch_bounds__(256)
    mg_transfer_t(int64_t E, const T* __restrict__ J, const T* __restrict__ in,
                  const uint8_t* __restrict__ cw, T* __restrict__ out) {
  using Sh = MgTransferShape<NF>;
  constexpr int nf = Sh::nf, nc = Sh::nc, EPB = Sh::EPB;
  constexpr int ni = RESTRICT ? nf : nc, no = RESTRICT ? nc : nf;
  constexpr int ni3 = ni * ni * ni, no3 = no * no * no;
  constexpr int S1 = ni * ni * no, S2 = ni * no * no;   // stage sizes per element
  constexpr int BUF = nf * nf * nf;                      // >= every stage
  extern __shared__ __align__(16) unsigned char mg_smem[];
  T* b0 = reinterpret_cast<T*>(mg_smem);   // [EPB][BUF]
  T* b1 = b0 + EPB * BUF;                  // [EPB][BUF]
  T* sM = b1 + EPB * BUF;                  // ni * no
  for (int q = threadIdx.x; q < ni * no; q += blockDim.x) {
    const int o = q / ni, t = q - o * ni;   // sM[o][t] = M(o, t)
    sM[q] = RESTRICT ? J[t * nc + o] : J[o * nc + t];
  }
  const int64_t ngroups = (E + EPB - 1) / EPB;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t e0 = g * EPB;
    const int ne = (int)(E - e0 < EPB ? E - e0 : EPB);
    __syncthreads();
    for (int q = threadIdx.x; q < ne * ni3; q += blockDim.x) {
      const int le = q / ni3, p = q - le * ni3;
      T v = in[e0 * ni3 + q];
      if (RESTRICT) {
        const uint8_t m = cw[e0 * ni3 + q];
        v = m ? v * (T(1) / T(m)) : T(0);
      }
      b0[le * BUF + p] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ne * S1; q += blockDim.x) {
      const int le = q / S1, p = q - le * S1;
      const int o = p % no, jk = p / no;
      const T* src = b0 + le * BUF + jk * ni;
      T s = T(0);
#pragma unroll
      for (int t = 0; t < ni; ++t) s += sM[o * ni + t] * src[t];
      b1[le * BUF + p] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ne * S2; q += blockDim.x) {
      const int le = q / S2, p = q - le * S2;
      const int i = p % no, o = (p / no) % no, k = p / (no * no);
      const T* src = b1 + le * BUF + k * ni * no + i;
      T s = T(0);
#pragma unroll
      for (int t = 0; t < ni; ++t) s += sM[o * ni + t] * src[t * no];
      b0[le * BUF + p] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ne * no3; q += blockDim.x) {
      const int le = q / no3, p = q - le * no3;
      const int ij = p % (no * no), o = p / (no * no);
      const T* src = b0 + le * BUF + ij;
      T s = T(0);
#pragma unroll
      for (int t = 0; t < ni; ++t) s += sM[o * ni + t] * src[t * no * no];
      if (RESTRICT) out[e0 * no3 + q] = s;
      else out[e0 * no3 + q] += s;
    }
  }
}

template <typename T, bool RESTRICT>
static int mg_transfer_t_launch(Handle& h, int NF, const T* J, const T* in, const uint8_t* cw,
                                T* out) {
  switch (NF) {
#define SEM_MG_TR(NN)                                                                      \
  case NN: {                                                                               \
    using TS = MgTransferShape<NN>;                                                        \
    constexpr size_t smem =                                                                \
        sizeof(T) * (2 * (size_t)TS::EPB * TS::nf3 + (size_t)TS::nf * TS::nc);             \
    auto k = mg_transfer_t<T, NN, RESTRICT>;                                               \
    SEM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    int per_sm = 0;                                                                        \
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));        \
    const int64_t groups = (h.E + TS::EPB - 1) / TS::EPB;                                  \
    const int gg = (int)std::max<int64_t>(                                                 \
        1, std::min<int64_t>(groups, (int64_t)h.num_sms * std::max(per_sm, 1)));           \
    k<<<gg, 256, smem, h.stream>>>(h.E, J, in, cw, out);                                   \
    break;                                                                                 \
  }
    SEM_MG_TR(2) SEM_MG_TR(3) SEM_MG_TR(4) SEM_MG_TR(5) SEM_MG_TR(6) SEM_MG_TR(7) SEM_MG_TR(8)
    SEM_MG_TR(9) SEM_MG_TR(10) SEM_MG_TR(11) SEM_MG_TR(12) SEM_MG_TR(13) SEM_MG_TR(14)
    SEM_MG_TR(15)
#undef SEM_MG_TR
    default:
      set_error("multigrid: order out of range");
      return SEM_EINVAL;
  }
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// h-transfers between two N = 1 levels: fine mesh kx x ky x kz, coarse mesh
// halved.  Fine element e lies in coarse element (ex/2, ey/2, ez/2), in half
// (ex%2, ey%2, ez%2); its node i (0, 1) sits at t = (s + i)/2 in the coarse
// element, where the coarse vertex a has weight 1 - t (a = 0) or t (a = 1):
// weights 1, 1/2 or 0, exact in either precision.
__device__ __forceinline__ int mg_hw2(int s, int i, int a) {   // 2 x weight
  const int t2 = s + i;
  return a == 0 ? 2 - t2 : t2;
}

// zf += P zc, one thread per fine local node
template <typename T>
__global__ void mg_hprolong_kernel(int kx, int ky, int64_t Ef, const T* __restrict__ zc,
                                   T* __restrict__ zf) {
  const int kxc = kx / 2, kyc = ky / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 8 * Ef;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t >> 3;
    const int node = (int)(t & 7);
    const int i = node & 1, j = (node >> 1) & 1, k = node >> 2;
    const int64_t ex = e % kx, ey = (e / kx) % ky, ez = e / ((int64_t)kx * ky);
    const int sx = (int)(ex & 1), sy = (int)(ey & 1), sz = (int)(ez & 1);
    const T* u = zc + (ex / 2 + kxc * (ey / 2 + (int64_t)kyc * (ez / 2))) * 8;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int w8 = mg_hw2(sx, i, a) * mg_hw2(sy, j, b) * mg_hw2(sz, k, c);
          if (w8) s += (T)(w8 * 0.125) * u[a + 2 * b + 4 * c];
        }
    zf[t] += s;
  }
}

// rc = P^T (rf / m_f) element by element (before the coarse summation), one
// thread per coarse local node gathering from the eight children
template <typename T>
__global__ void mg_hrestrict_kernel(int kxc, int kyc, int64_t Ec, const T* __restrict__ rf,
                                    const uint8_t* __restrict__ cwf, T* __restrict__ rc) {
  const int64_t kx = 2 * (int64_t)kxc, ky = 2 * (int64_t)kyc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 8 * Ec;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ce = t >> 3;
    const int node = (int)(t & 7);
    const int a = node & 1, b = (node >> 1) & 1, c = node >> 2;
    const int64_t cx = ce % kxc, cy = (ce / kxc) % kyc, cz = ce / ((int64_t)kxc * kyc);
    T s = T(0);
#pragma unroll
    for (int sz = 0; sz < 2; ++sz)
#pragma unroll
      for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const int64_t ef = (2 * cx + sx) + kx * ((2 * cy + sy) + ky * (2 * cz + sz));
#pragma unroll
          for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
              for (int i = 0; i < 2; ++i) {
                const int w8 = mg_hw2(sx, i, a) * mg_hw2(sy, j, b) * mg_hw2(sz, k, c);
                if (!w8) continue;
                const int64_t l = ef * 8 + i + 2 * j + 4 * k;
                const uint8_t m = cwf[l];
                const T v = m ? rf[l] * (T(1) / T(m)) : T(0);
                s += (T)(w8 * 0.125) * v;
              }
        }
    rc[t] = s;
  }
}

// t = r - w (r and w masked)
template <typename T>
__global__ void mg_residual_kernel(int64_t L, const T* __restrict__ r, const T* __restrict__ w,
                                   T* __restrict__ t) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    t[l] = r[l] - w[l];
}

template <typename T>
__global__ void mg_mask_kernel(int64_t L, const double* __restrict__ mask, T* __restrict__ v) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    v[l] = (T)mask[l] * v[l];
}

// y = a x + b y
template <typename T>
__global__ void mg_axpby_kernel(int64_t L, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += (int64_t)gridDim.x * blockDim.x)
    y[l] = a * x[l] + b * y[l];
}

static int grid_of(const Handle& h, int64_t work) {
  int64_t g = (work + 255) / 256;
  const int64_t cap = (int64_t)h.num_sms * 8;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

// ---------------------------------------------------------------- level ops

template <typename T>
struct MgPrec;
template <>
struct MgPrec<double> {
  static constexpr sem_precision p = SEM_FP64;
  static double* r(MgLevel& v) { return v.r64; }
  static double* z(MgLevel& v) { return v.z64; }
  static double* t(MgLevel& v) { return v.t64; }
  static double* w(MgLevel& v) { return v.w64; }
  static double* ext(MgLevel& v) { return v.ext64; }
  static const double* S(MgLevel& v) { return v.S64; }
  static const double* lam(MgLevel& v) { return v.lam64; }
  static const double* wsq(MgLevel& v) { return v.wsq64; }
  static const double* J(MgLevel& v) { return v.J64; }
};
template <>
struct MgPrec<float> {
  static constexpr sem_precision p = SEM_MIXED_FP32;
  static float* r(MgLevel& v) { return v.r32; }
  static float* z(MgLevel& v) { return v.z32; }
  static float* t(MgLevel& v) { return v.t32; }
  static float* w(MgLevel& v) { return v.w32; }
  static float* ext(MgLevel& v) { return v.ext32; }
  static const float* S(MgLevel& v) { return v.S32; }
  static const float* lam(MgLevel& v) { return v.lam32; }
  static const float* wsq(MgLevel& v) { return v.wsq32; }
  static const float* J(MgLevel& v) { return v.J32; }
};

// z = (acc ? z : 0) + omega * Schwarz(r) on level lv
template <typename T>
static int mg_schwarz(MgLevel& lv, const T* r, T* z, bool accumulate) {
  Handle& h = *lv.h;
  using P = MgPrec<T>;
  int rc;
  if ((rc = mg_block_solve_dispatch<T>(h, r, P::wsq(lv), P::S(lv), P::lam(lv), lv.act, P::ext(lv))))
    return rc;
  const int acc = accumulate ? 1 : 0;
  const int gr = grid_of(h, h.E * (int64_t)h.n * h.n);
  switch (h.N) {
#define SEM_MG_SUM(NN)                                                                            \
  case NN:                                                                                        \
    if (sizeof(T) == 8)                                                                           \
      mg_block_sum_rows<double, kGsFP64, NN><<<gr, 256, 0, h.stream>>>(                           \
          h.kx, h.ky, h.E, h.bfaces, (const double*)P::ext(lv), (const double*)P::wsq(lv),        \
          lv.omega, acc, (double*)z);                                                             \
    else                                                                                          \
      mg_block_sum_rows<float, kGsTwoSum, NN><<<gr, 256, 0, h.stream>>>(                          \
          h.kx, h.ky, h.E, h.bfaces, (const float*)P::ext(lv), (const float*)P::wsq(lv),          \
          (float)lv.omega, acc, (float*)z);                                                       \
    break;
    SEM_MG_SUM(1) SEM_MG_SUM(2) SEM_MG_SUM(3) SEM_MG_SUM(4) SEM_MG_SUM(5) SEM_MG_SUM(6)
    SEM_MG_SUM(7) SEM_MG_SUM(8) SEM_MG_SUM(9) SEM_MG_SUM(10) SEM_MG_SUM(11) SEM_MG_SUM(12)
    SEM_MG_SUM(13) SEM_MG_SUM(14) SEM_MG_SUM(15)
#undef SEM_MG_SUM
    default:
      set_error("multigrid: order out of range");
      return SEM_EINVAL;
  }
  h.launches += 2;
  SEM_CUDA(cudaGetLastError());
  return 0;
}

// w = mask QQ^T A_L u on level lv
template <typename T>
static int mg_apply_a(MgLevel& lv, const T* u, T* w) {
  Handle& h = *lv.h;
  int rc;
  if (sizeof(T) == 8) {
    if ((rc = ax_dispatch_fp64(h, (const double*)u, (double*)w, nullptr))) return rc;
  } else {
    if ((rc = ax_dispatch_fp32(h, (const float*)u, (float*)w, nullptr, kDotDot2))) return rc;
  }
  // the operator kernels zero w on the Dirichlet boundary and the summation
  // keeps those zeros: w is masked
  return launch_gs(h, MgPrec<T>::p, w);
}

// z_l = V-cycle(r_l)
template <typename T>
static int mg_vcycle(MgData& mg, int l, const T* r, T* z) {
  MgLevel& lv = mg.lv[l];
  Handle& h = *lv.h;
  using P = MgPrec<T>;
  int rc;
  if ((rc = mg_schwarz<T>(lv, r, z, false))) return rc;
  if (l + 1 == (int)mg.lv.size()) return 0;
  MgLevel& cv = mg.lv[l + 1];
  Handle& hc = *cv.h;
  T* t = P::t(lv);
  if ((rc = mg_apply_a<T>(lv, z, P::w(lv)))) return rc;
  mg_residual_kernel<T><<<grid_of(h, h.L), 256, 0, h.stream>>>(h.L, r, P::w(lv), t);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  // restriction: (J^T)^{x3} (t / mult) -- or its trilinear h-counterpart --,
  // then QQ^T and mask on the coarse level
  if (lv.h_to_next) {
    mg_hrestrict_kernel<T><<<grid_of(hc, 8 * hc.E), 256, 0, h.stream>>>(hc.kx, hc.ky, hc.E, t,
                                                                        h.cw8, P::r(cv));
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
  } else if ((rc = mg_transfer_t_launch<T, true>(h, lv.N, P::J(lv), t, h.cw8, P::r(cv)))) {
    return rc;
  }
  if ((rc = launch_gs(hc, P::p, P::r(cv)))) return rc;
  mg_mask_kernel<T><<<grid_of(hc, hc.L), 256, 0, h.stream>>>(hc.L, hc.mask64, P::r(cv));
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  if ((rc = mg_vcycle<T>(mg, l + 1, P::r(cv), P::z(cv)))) return rc;
  if (lv.h_to_next) {
    mg_hprolong_kernel<T><<<grid_of(h, 8 * h.E), 256, 0, h.stream>>>(h.kx, h.ky, h.E, P::z(cv), z);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
  } else if ((rc = mg_transfer_t_launch<T, false>(h, lv.N, P::J(lv), P::z(cv), nullptr, z))) {
    return rc;
  }
  if ((rc = mg_apply_a<T>(lv, z, P::w(lv)))) return rc;
  mg_residual_kernel<T><<<grid_of(h, h.L), 256, 0, h.stream>>>(h.L, r, P::w(lv), t);
  ++h.launches;
  SEM_CUDA(cudaGetLastError());
  return mg_schwarz<T>(lv, t, z, true);
}

// ---------------------------------------------------------------- set-up

static double read_dot(Handle& h, MgData& mg) {
  cudaMemcpyAsync(mg.dot_host, mg.dot, sizeof(double), cudaMemcpyDeviceToHost, h.stream);
  cudaStreamSynchronize(h.stream);
  return *mg.dot_host;
}

template <typename T>
static int mg_alloc(Handle& h, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (multigrid)");
  return 0;
}

static void level_free(MgLevel& v) {
  void* ptrs[] = {v.S64, v.S32, v.lam64, v.lam32, v.act, v.wsq64, v.wsq32, v.J64, v.J32,
                  v.r64, v.z64, v.t64, v.w64, v.ext64, v.r32, v.z32, v.t32, v.w32, v.ext32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (v.owned && v.h) sem_destroy(static_cast<sem_handle>(static_cast<sem_handle_s*>(v.h)));
  v = MgLevel();
}

void mg_free(Handle& h) {
  if (!h.mg) return;
  for (auto& v : h.mg->lv) level_free(v);
  void* ptrs[] = {h.mg->p64, h.mg->zz64, h.mg->w64, h.mg->r64, h.mg->x64, h.mg->p32,
                  h.mg->zz32, h.mg->w32, h.mg->r32, h.mg->x32, h.mg->dot};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h.mg->dot_host) cudaFreeHost(h.mg->dot_host);
  delete h.mg;
  h.mg = nullptr;
}

// Interpolation matrix J[p][a] = l_a(x_p) from coarse nodes xc to fine nodes xf.
static std::vector<double> interp(const std::vector<double>& xc, const std::vector<double>& xf) {
  const int nc = (int)xc.size(), nf = (int)xf.size();
  std::vector<double> J((size_t)nf * nc, 1.0);
  for (int p = 0; p < nf; ++p)
    for (int a = 0; a < nc; ++a)
      for (int q = 0; q < nc; ++q)
        if (q != a) J[(size_t)p * nc + a] *= (xf[p] - xc[q]) / (xc[a] - xc[q]);
  return J;
}

static int level_setup(MgLevel& v) {
  Handle& h = *v.h;
  int rc;
  v.N = h.N;
  v.n = h.n;
  v.m = h.n + 2;
  const size_t E = (size_t)h.E, L = (size_t)h.L, m = (size_t)v.m;
  if ((rc = mg_alloc(h, &v.S64, 3 * E * m * m)) || (rc = mg_alloc(h, &v.S32, 3 * E * m * m)) ||
      (rc = mg_alloc(h, &v.lam64, 3 * E * m)) || (rc = mg_alloc(h, &v.lam32, 3 * E * m)) ||
      (rc = mg_alloc(h, &v.act, 3 * E * m)) || (rc = mg_alloc(h, &v.wsq64, L)) ||
      (rc = mg_alloc(h, &v.wsq32, L)) || (rc = mg_alloc(h, &v.r64, L)) ||
      (rc = mg_alloc(h, &v.z64, L)) || (rc = mg_alloc(h, &v.t64, L)) ||
      (rc = mg_alloc(h, &v.w64, L)) || (rc = mg_alloc(h, &v.ext64, E * m * m * m)) ||
      (rc = mg_alloc(h, &v.r32, L)) || (rc = mg_alloc(h, &v.z32, L)) ||
      (rc = mg_alloc(h, &v.t32, L)) || (rc = mg_alloc(h, &v.w32, L)) ||
      (rc = mg_alloc(h, &v.ext32, E * m * m * m)))
    return rc;
  double* len = nullptr;
  if ((rc = mg_alloc(h, &len, 3 * E))) return rc;
  const int g = grid_of(h, 3 * h.E);
  mg_lengths_kernel<<<g, 256, 0, h.stream>>>(h.coords, h.L, h.E, h.n, len);
  mg_fdm_kernel<<<g, 64, 0, h.stream>>>(h.N, h.kx, h.ky, h.kz, h.E, h.D64, h.wq, len, v.S64,
                                        v.S32, v.lam64, v.lam32, v.act);
  mg_weights_kernel<<<grid_of(h, h.L), 256, 0, h.stream>>>(h.N, h.kx, h.ky, h.kz, h.L, v.act,
                                                           v.wsq64, v.wsq32);
  h.launches += 3;
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h.stream);
  cudaFree(len);
  if (ce != cudaSuccess) return cuda_fail(ce, "multigrid set-up");
  return 0;
}

// lambda_max(S A) by power iteration from the SplitMix64 vector of `seed`,
// Rayleigh quotient in the A inner product (FP64); omega = 1 / lambda.
static int level_omega(MgData& mg, MgLevel& v, int iters, uint64_t seed) {
  Handle& h = *v.h;
  int rc;
  double* x = v.r64;
  double* ax = v.t64;
  double* y = v.z64;
  double* ay = v.w64;
  if ((rc = launch_rhs(h, 1, seed, x))) return rc;
  v.omega = 1.0;
  if ((rc = launch_glsc3(h, SEM_FP64, x, x, mg.dot))) return rc;
  if (read_dot(h, mg) == 0.0) return 0;   // a level without interior nodes: nothing to damp
  double lam = 1.0;
  for (int it = 0; it < iters; ++it) {
    if ((rc = mg_apply_a<double>(v, x, ax))) return rc;
    if ((rc = mg_schwarz<double>(v, ax, y, false))) return rc;   // omega = 1 here
    if ((rc = mg_apply_a<double>(v, y, ay))) return rc;
    if ((rc = launch_glsc3(h, SEM_FP64, y, ay, mg.dot))) return rc;
    const double yay = read_dot(h, mg);
    if ((rc = launch_glsc3(h, SEM_FP64, y, ax, mg.dot))) return rc;
    const double yax = read_dot(h, mg);
    if ((rc = launch_glsc3(h, SEM_FP64, y, y, mg.dot))) return rc;
    const double yy = read_dot(h, mg);
    if (!(yax > 0.0) || !(yy > 0.0)) {
      set_error("multigrid set-up: power iteration broke down");
      return SEM_EINVAL;
    }
    lam = yay / yax;
    mg_axpby_kernel<double><<<grid_of(h, h.L), 256, 0, h.stream>>>(h.L, 1.0 / sqrt(yy), y, 0.0, x);
    SEM_CUDA(cudaGetLastError());
  }
  v.omega = 1.0 / lam;
  return 0;
}

int mg_ensure(Handle& h) {
  if (h.mg) return 0;
  if (h.gid_user) {
    set_error("multigrid: needs a box mesh (sem_setup without gid)");
    return SEM_EINVAL;
  }
  MgData* mg = new MgData();
  h.mg = mg;
  auto fail = [&](int rc) {
    mg_free(h);
    return rc;
  };
  // levels: orders N, N/2, ..., 1 on the mesh, then (h-levels) N = 1 on the
  // mesh halved while every dimension is even and its half at least 2
  struct Spec {
    int N, kx, ky, kz;
  };
  std::vector<Spec> specs{{h.N, h.kx, h.ky, h.kz}};
  while (specs.back().N > 1) specs.push_back({std::max(1, specs.back().N / 2), h.kx, h.ky, h.kz});
  const size_t n_p = specs.size();
  if (h.mg_hcoarsen) {
    int kx = h.kx, ky = h.ky, kz = h.kz;
    while (kx % 2 == 0 && ky % 2 == 0 && kz % 2 == 0 && std::min(kx, std::min(ky, kz)) >= 4) {
      kx /= 2;
      ky /= 2;
      kz /= 2;
      specs.push_back({1, kx, ky, kz});
    }
  }
  mg->lv.resize(specs.size());
  int rc;
  for (size_t l = 0; l < specs.size(); ++l) {
    MgLevel& v = mg->lv[l];
    v.h_to_next = l + 1 < specs.size() && l + 1 >= n_p;
    if (l == 0) {
      v.h = &h;
    } else {
      sem_mesh mesh;
      memset(&mesh, 0, sizeof(mesh));
      mesh.kx = specs[l].kx;
      mesh.ky = specs[l].ky;
      mesh.kz = specs[l].kz;
      for (int d = 0; d < 3; ++d) {
        mesh.lo[d] = h.mesh_lo[d];
        mesh.hi[d] = h.mesh_hi[d];
      }
      mesh.deform_amp = h.deform_amp;
      mesh.deform_kind = h.deform_kind;
      sem_handle sub = nullptr;
      if ((rc = sem_setup(&mesh, specs[l].N, 0, h.stream, &sub))) return fail(rc);
      v.h = sub;
      v.owned = true;
    }
    if ((rc = level_setup(v))) return fail(rc);
  }
  // interpolation matrices of the p-pairs (host FP64 from each level's GLL nodes)
  for (size_t l = 0; l + 1 < n_p; ++l) {
    MgLevel& f = mg->lv[l];
    MgLevel& c = mg->lv[l + 1];
    std::vector<double> xf(f.n), xc(c.n);
    SEM_CUDA(cudaMemcpy(xf.data(), f.h->xi, sizeof(double) * f.n, cudaMemcpyDeviceToHost));
    SEM_CUDA(cudaMemcpy(xc.data(), c.h->xi, sizeof(double) * c.n, cudaMemcpyDeviceToHost));
    const std::vector<double> J = interp(xc, xf);
    std::vector<float> J32(J.begin(), J.end());
    if ((rc = mg_alloc(h, &f.J64, J.size())) || (rc = mg_alloc(h, &f.J32, J.size()))) return fail(rc);
    SEM_CUDA(cudaMemcpy(f.J64, J.data(), sizeof(double) * J.size(), cudaMemcpyHostToDevice));
    SEM_CUDA(cudaMemcpy(f.J32, J32.data(), sizeof(float) * J.size(), cudaMemcpyHostToDevice));
  }
  const size_t L = (size_t)h.L;
  if ((rc = mg_alloc(h, &mg->p64, L)) || (rc = mg_alloc(h, &mg->zz64, L)) ||
      (rc = mg_alloc(h, &mg->w64, L)) || (rc = mg_alloc(h, &mg->r64, L)) ||
      (rc = mg_alloc(h, &mg->x64, L)) || (rc = mg_alloc(h, &mg->p32, L)) ||
      (rc = mg_alloc(h, &mg->zz32, L)) || (rc = mg_alloc(h, &mg->w32, L)) ||
      (rc = mg_alloc(h, &mg->r32, L)) || (rc = mg_alloc(h, &mg->x32, L)) ||
      (rc = mg_alloc(h, &mg->dot, 1)))
    return fail(rc);
  if (cudaMallocHost((void**)&mg->dot_host, sizeof(double)) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation, "cudaMallocHost"));
  for (auto& v : mg->lv)
    if ((rc = level_omega(*mg, v, 20, 12345))) return fail(rc);
  return 0;
}

// ---------------------------------------------------------------- solves

// Apply the preconditioner: z = V(r) (device vectors of the precision's type).
int mg_apply(Handle& h, sem_precision p, const void* r, void* z) {
  int rc;
  if ((rc = mg_ensure(h))) return rc;
  if (p == SEM_FP64) return mg_vcycle<double>(*h.mg, 0, (const double*)r, (double*)z);
  return mg_vcycle<float>(*h.mg, 0, (const float*)r, (float*)z);
}

// CG preconditioned by one V-cycle per iteration (T data; dots in FP64 or
// Dot2) on A d = r0 from d = 0, until ||r||_c <= stop (absolute) or maxit.
// Returns the iterations done through *iters and the last ||r||_c.
template <typename T>
static int mg_cg(Handle& h, MgData& mg, const T* r0, T* d, double stop, int maxit, int* iters,
                 double* rnorm) {
  using P = MgPrec<T>;
  MgLevel& f = mg.lv[0];
  const sem_precision p = P::p;
  T* r = sizeof(T) == 8 ? (T*)mg.r64 : (T*)mg.r32;
  T* z = sizeof(T) == 8 ? (T*)mg.zz64 : (T*)mg.zz32;
  T* pp = sizeof(T) == 8 ? (T*)mg.p64 : (T*)mg.p32;
  T* w = sizeof(T) == 8 ? (T*)mg.w64 : (T*)mg.w32;
  int rc;
  const int g = grid_of(h, h.L);
  SEM_CUDA(cudaMemcpyAsync(r, r0, sizeof(T) * h.L, cudaMemcpyDeviceToDevice, h.stream));
  SEM_CUDA(cudaMemsetAsync(d, 0, sizeof(T) * h.L, h.stream));
  if ((rc = launch_glsc3(h, p, r, r, mg.dot))) return rc;
  double rtr = read_dot(h, mg);
  *iters = 0;
  *rnorm = sqrt(rtr);
  if (*rnorm <= stop) return 0;
  if ((rc = mg_vcycle<T>(mg, 0, r, z))) return rc;
  if ((rc = launch_glsc3(h, p, r, z, mg.dot))) return rc;
  double rtz = read_dot(h, mg);
  SEM_CUDA(cudaMemcpyAsync(pp, z, sizeof(T) * h.L, cudaMemcpyDeviceToDevice, h.stream));
  for (int it = 1; it <= maxit; ++it) {
    if ((rc = mg_apply_a<T>(f, pp, w))) return rc;
    if ((rc = launch_glsc3(h, p, w, pp, mg.dot))) return rc;
    const double pap = read_dot(h, mg);
    if (!(pap > 0.0) || !(rtz > 0.0)) {
      set_error("multigrid CG: breakdown (p.Ap or r.z not positive)");
      return SEM_BREAKDOWN;
    }
    const double alpha = rtz / pap;
    mg_axpby_kernel<T><<<g, 256, 0, h.stream>>>(h.L, (T)alpha, pp, (T)1, d);
    mg_axpby_kernel<T><<<g, 256, 0, h.stream>>>(h.L, (T)(-alpha), w, (T)1, r);
    h.launches += 2;
    SEM_CUDA(cudaGetLastError());
    if ((rc = launch_glsc3(h, p, r, r, mg.dot))) return rc;
    rtr = read_dot(h, mg);
    *iters = it;
    *rnorm = sqrt(rtr);
    if (*rnorm <= stop) return 0;
    if ((rc = mg_vcycle<T>(mg, 0, r, z))) return rc;
    if ((rc = launch_glsc3(h, p, r, z, mg.dot))) return rc;
    const double rtz_new = read_dot(h, mg);
    const double beta = rtz_new / rtz;
    rtz = rtz_new;
    mg_axpby_kernel<T><<<g, 256, 0, h.stream>>>(h.L, (T)1, z, (T)beta, pp);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
  }
  return SEM_MAXIT;
}

// Multigrid-preconditioned solve of A x = f (x0 optional), FP64 or mixed.
// Mixed: FP64 outer residual r64 = f - A64 x64; inner FP32 multigrid CG on
// A d = r64 reducing ||r|| by max(inner_floor, 0.5 tol / relres); x64 += d.
// Mixed multigrid CG with reliable updates (as the Jacobi solver's default):
// one FP32 recursion on d with A d = r64; each time its residual has fallen
// by `delta` (or reached the tolerance) d is folded into x64, the FP64 true
// residual recomputed and copied into r32, and CG continues with the same
// search direction.  Returns the iterations through *iters, replacements
// through *repl; *relres is the final FP64 relative residual.
static int mg_cg_reliable(Handle& h, MgData& mg, const double* f, double tol, double bnorm,
                          int maxit, double delta, int max_repl, int* iters, int* repl,
                          double* relres, double* rec) {
  MgLevel& lv0 = mg.lv[0];
  float* r = mg.r32;
  float* z = mg.zz32;
  float* p = mg.p32;
  float* w = mg.w32;
  float* d = mg.x32;
  int rc;
  const int g = grid_of(h, h.L);
  *iters = 0;
  *repl = 0;
  if ((rc = launch_cast64to32(h, h.r64, r))) return rc;
  SEM_CUDA(cudaMemsetAsync(d, 0, sizeof(float) * h.L, h.stream));
  if ((rc = launch_glsc3(h, SEM_MIXED_FP32, r, r, mg.dot))) return rc;
  double seg_ref = sqrt(read_dot(h, mg));
  if ((rc = mg_vcycle<float>(mg, 0, r, z))) return rc;
  if ((rc = launch_glsc3(h, SEM_MIXED_FP32, r, z, mg.dot))) return rc;
  double rtz = read_dot(h, mg);
  SEM_CUDA(cudaMemcpyAsync(p, z, sizeof(float) * h.L, cudaMemcpyDeviceToDevice, h.stream));
  for (int it = 1; it <= maxit; ++it) {
    if ((rc = mg_apply_a<float>(lv0, p, w))) return rc;
    if ((rc = launch_glsc3(h, SEM_MIXED_FP32, w, p, mg.dot))) return rc;
    const double pap = read_dot(h, mg);
    if (!(pap > 0.0) || !(rtz > 0.0)) {
      set_error("multigrid CG: breakdown (p.Ap or r.z not positive)");
      return SEM_BREAKDOWN;
    }
    const double alpha = rtz / pap;
    mg_axpby_kernel<float><<<g, 256, 0, h.stream>>>(h.L, (float)alpha, p, 1.f, d);
    mg_axpby_kernel<float><<<g, 256, 0, h.stream>>>(h.L, (float)(-alpha), w, 1.f, r);
    h.launches += 2;
    SEM_CUDA(cudaGetLastError());
    if ((rc = launch_glsc3(h, SEM_MIXED_FP32, r, r, mg.dot))) return rc;
    const double rn = sqrt(read_dot(h, mg));
    *iters = it;
    *rec = rn / bnorm;
    if (rn <= delta * seg_ref || rn <= tol * bnorm) {
      // reliable update: fold d into x64, FP64 true residual replaces r32
      if ((rc = launch_add32to64(h, h.x64, d))) return rc;
      SEM_CUDA(cudaMemsetAsync(d, 0, sizeof(float) * h.L, h.stream));
      if ((rc = fp64_residual(h, f, false, relres, nullptr))) return rc;
      if (*relres <= tol) return 0;
      if (++*repl > max_repl) return SEM_STAGNATED;
      if ((rc = launch_cast64to32(h, h.r64, r))) return rc;
      if ((rc = launch_glsc3(h, SEM_MIXED_FP32, r, r, mg.dot))) return rc;
      seg_ref = sqrt(read_dot(h, mg));
    }
    if ((rc = mg_vcycle<float>(mg, 0, r, z))) return rc;
    if ((rc = launch_glsc3(h, SEM_MIXED_FP32, r, z, mg.dot))) return rc;
    const double rtz_new = read_dot(h, mg);
    const double beta = rtz_new / rtz;
    rtz = rtz_new;
    mg_axpby_kernel<float><<<g, 256, 0, h.stream>>>(h.L, 1.f, z, (float)beta, p);
    ++h.launches;
    SEM_CUDA(cudaGetLastError());
  }
  if ((rc = launch_add32to64(h, h.x64, d))) return rc;
  if ((rc = fp64_residual(h, f, false, relres, nullptr))) return rc;
  return SEM_MAXIT;
}

int pcg_mg_solve(Handle& h, const double* f, const double* x0, double* x, double tol, int maxit,
                 sem_precision prec, double inner_floor, int max_cycles, int refine_mode,
                 double replace_factor, sem_info* info) {
  int rc;
  if ((rc = mg_ensure(h))) return rc;
  MgData& mg = *h.mg;
  sem_info res{};
  const int64_t launches0 = h.launches;
  SEM_CUDA(cudaEventRecord(h.ev0, h.stream));
  if ((rc = launch_masked_copy64(h, x0, h.x64))) return rc;
  double relres = 1.0, bnorm = 0.0;
  if ((rc = fp64_residual(h, f, x0 == nullptr, &relres, &bnorm))) return rc;
  int total = 0, cycles = 0;
  res.status = 0;
  if (bnorm > 0.0 && relres > tol) {
    if (prec == SEM_FP64) {
      int its = 0;
      double rn = 0.0;
      const int cg_rc = mg_cg<double>(h, mg, h.r64, mg.x64, tol * bnorm, maxit, &its, &rn);
      if (cg_rc < 0) return cg_rc;
      total = its;
      const int g = grid_of(h, h.L);
      mg_axpby_kernel<double><<<g, 256, 0, h.stream>>>(h.L, 1.0, mg.x64, 1.0, h.x64);
      SEM_CUDA(cudaGetLastError());
      if ((rc = fp64_residual(h, f, false, &relres, nullptr))) return rc;
      res.status = cg_rc == SEM_MAXIT ? SEM_MAXIT : 0;
      res.relres = rn / bnorm;
    } else if (refine_mode == 0) {
      int its = 0, repl = 0;
      double rec = 0.0;
      const double delta = replace_factor > 0 ? replace_factor : 1e-2;
      const int st = mg_cg_reliable(h, mg, f, tol, bnorm, maxit, delta, 4 * max_cycles, &its,
                                    &repl, &relres, &rec);
      if (st < 0) return st;
      total = its;
      cycles = repl;
      res.relres = rec;
      res.status = st == SEM_MAXIT ? SEM_MAXIT : (st == SEM_STAGNATED ? SEM_STAGNATED : 0);
    } else {
      for (;;) {
        if (relres <= tol) break;
        if (cycles >= max_cycles) { res.status = SEM_STAGNATED; break; }
        if (total >= maxit) { res.status = SEM_MAXIT; break; }
        const double red = std::max(inner_floor, 0.5 * tol / relres);
        if ((rc = launch_cast64to32(h, h.r64, mg.lv[0].t32))) return rc;
        // the inner stop is relative to the FP32 copy of r64
        if ((rc = launch_glsc3(h, SEM_MIXED_FP32, mg.lv[0].t32, mg.lv[0].t32, mg.dot))) return rc;
        const double r0n = sqrt(read_dot(h, mg));
        int its = 0;
        double rn = 0.0;
        rc = mg_cg<float>(h, mg, mg.lv[0].t32, mg.x32, red * r0n, maxit - total, &its, &rn);
        if (rc < 0) return rc;
        total += its;
        ++cycles;
        if ((rc = launch_add32to64(h, h.x64, mg.x32))) return rc;
        const double prev = relres;
        if ((rc = fp64_residual(h, f, false, &relres, nullptr))) return rc;
        res.relres = rn / bnorm;
        if (relres > 0.9 * prev && relres > tol) { res.status = SEM_STAGNATED; break; }
      }
    }
  }
  SEM_CUDA(cudaMemcpyAsync(x, h.x64, sizeof(double) * h.L, cudaMemcpyDeviceToDevice, h.stream));
  SEM_CUDA(cudaEventRecord(h.ev1, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h.ev0, h.ev1);
  res.iters = total;
  res.refinements = cycles;
  res.relres_true = relres;
  res.solve_ms = ms;
  res.launches = h.launches - launches0;
  if (res.status == 0 && relres > tol) res.status = SEM_MAXIT;
  if (info) *info = res;
  return res.status;
}

double mg_omega(Handle& h, int level) {
  if (!h.mg || level < 0 || level >= (int)h.mg->lv.size()) return -1.0;
  return h.mg->lv[level].omega;
}
int mg_levels(Handle& h) { return h.mg ? (int)h.mg->lv.size() : 0; }

}  // namespace sem
