"""CPU oracle for the spectral-element Poisson hot path (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  The CUDA library never calls it and
shares no code with it.

What it computes (arXiv 2503.02134, Sec. 3 "Nekbone case study"):
  * the matrix-free element operator ``ax`` (Sec. 3.1, Table "Profiling of the
    CG kernels within Nekbone", line ``ax``; call graph local_grad3 ->
    geometric factors -> local_grad3_t),
  * the direct-stiffness summation Sigma' = Q Q^T over shared GLL nodes
    (Sec. 3.3 "Global communication and gather-scatter modes"),
  * the Jacobi preconditioner z = J^{-1} r with J^{-1} = 1/diag(A) (Sec. 4.3,
    Jacobi paragraph), and
  * the preconditioned CG loop of the profiling table (solveM, glsc3, add2s1,
    ax, glsc3, add2s2, add2s2, glsc3).
The SEM building blocks the paper takes from its textbook reference
(Deville, Fischer & Mund 2002: GLL quadrature, the derivative matrix,
isoparametric geometric factors) are written out from their definitions.

Readings of places where the paper is silent or garbled (each is also listed
with the design notes):
  * the profiling table prints "beta = glsc3(r,c,z)" and "add2s2(x,p,pap)";
    the dot is rtz, beta = rtz/rtz_old and the add2s2 scale is
    alpha = rtz/pap (and -alpha for r);
  * the weight c of glsc3 is mask/multiplicity, so c-weighted local sums are
    sums over unique global nodes;
  * the stopping test is ||r||_c / ||b||_c <= tol;
  * Dirichlet conditions are homogeneous and imposed by masking every node on
    the six faces of the box (by index).

Layout: a local ("L") vector holds E*n^3 values, element-major; inside an
element node (i, j, k) sits at i + n*j + n*n*k (i along r fastest).  Numpy
views reshape it to [e, k, j, i].  The six geometric factors are stored as
G[a, e, k, j, i] with a = (rr, ss, tt, rs, rt, st).
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# 1. GLL nodes, weights and the derivative matrix (textbook definitions).
# --------------------------------------------------------------------------


def legendre(N: int, x):
    """P_N(x) and P_N'(x) by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P'_{k+1} = P'_{k-1} + (2k+1) P_k."""
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    dp_prev, dp = np.zeros_like(x), np.ones_like(x)
    if N == 0:
        return p_prev, dp_prev
    for k in range(1, N):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gll(N: int):
    """Gauss-Lobatto-Legendre nodes (ascending, xi_0 = -1, xi_N = 1) and weights.

    Interior nodes are the roots of P_N', found by Newton's method from the
    Chebyshev-Gauss-Lobatto points, with P_N'' taken from Legendre's equation
    (1 - x^2) P'' = 2 x P' - N(N+1) P.  Weights w_j = 2 / (N(N+1) P_N(xi_j)^2).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    interior = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(N, interior)
        d2p = (2.0 * interior * dp - N * (N + 1) * p) / (1.0 - interior ** 2)
        step = dp / d2p
        interior -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[1:-1] = interior
    x[0], x[-1] = -1.0, 1.0
    p, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * p ** 2)
    return x, w


def deriv_matrix(N: int, x):
    """D_ij = l_j'(xi_i) for the Lagrange basis on the GLL nodes:
    P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j)) off the diagonal,
    D_00 = -N(N+1)/4, D_NN = N(N+1)/4, and 0 on the rest of the diagonal."""
    n = N + 1
    p, _ = legendre(N, x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = p[i] / (p[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


# --------------------------------------------------------------------------
# 2. Box mesh, deformation and geometric factors.
# --------------------------------------------------------------------------


def box_coords(kx, ky, kz, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Node coordinates X[m, e, k, j, i] of an undeformed kx*ky*kz box mesh.

    Element e = ex + kx*(ey + ky*ez) spans [lo + ex*h, lo + (ex+1)*h] along x
    (same for y, z); its node (i, j, k) sits at lo + (ex + (1+xi_i)/2) * h."""
    xi, _ = gll(N)
    n = N + 1
    E = kx * ky * kz
    X = np.zeros((3, E, n, n, n))
    h = [(hi[d] - lo[d]) / k for d, k in enumerate((kx, ky, kz))]
    for ez in range(kz):
        for ey in range(ky):
            for ex in range(kx):
                e = ex + kx * (ey + ky * ez)
                px = lo[0] + (ex + (1.0 + xi) / 2.0) * h[0]
                py = lo[1] + (ey + (1.0 + xi) / 2.0) * h[1]
                pz = lo[2] + (ez + (1.0 + xi) / 2.0) * h[2]
                X[0, e] = px[None, None, :]
                X[1, e] = py[None, :, None]
                X[2, e] = pz[:, None, None]
    return X


def box_coords_elements(kx, ky, kz, N, elems, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Node coordinates X[m, q, k, j, i] of the listed elements of the same
    box mesh (elems[q] = ex + kx*(ey + ky*ez)), for meshes too large to build
    whole; the same formula as box_coords."""
    xi, _ = gll(N)
    n = N + 1
    elems = np.asarray(elems, dtype=np.int64)
    X = np.zeros((3, len(elems), n, n, n))
    h = [(hi[d] - lo[d]) / k for d, k in enumerate((kx, ky, kz))]
    for q, e in enumerate(elems):
        ex, ey, ez = e % kx, (e // kx) % ky, e // (kx * ky)
        X[0, q] = (lo[0] + (ex + (1.0 + xi) / 2.0) * h[0])[None, None, :]
        X[1, q] = (lo[1] + (ey + (1.0 + xi) / 2.0) * h[1])[None, :, None]
        X[2, q] = (lo[2] + (ez + (1.0 + xi) / 2.0) * h[2])[:, None, None]
    return X


def deform_cyclic(X, amp=0.05):
    """x += amp sin(2 pi y) sin(2 pi z), and its cyclic permutations, all
    evaluated from the undeformed coordinates at every GLL node."""
    x, y, z = X
    s = lambda a: np.sin(2.0 * np.pi * a)
    return np.stack([x + amp * s(y) * s(z),
                     y + amp * s(z) * s(x),
                     z + amp * s(x) * s(y)])


def apply_r(D, u):
    """(I x I x D) u : derivative along r (index i) of u[e, k, j, i]."""
    return np.einsum('il,ekjl->ekji', D, u)


def apply_s(D, u):
    """(I x D x I) u : derivative along s (index j)."""
    return np.einsum('jl,ekli->ekji', D, u)


def apply_t(D, u):
    """(D x I x I) u : derivative along t (index k)."""
    return np.einsum('kl,elji->ekji', D, u)


def geometry(X, N):
    """Geometric factors and mass for the coordinates X[m, e, k, j, i].

    J_{m a} = dx_m/dr_a by spectral differentiation of the coordinates,
    G_ab = w_i w_j w_k det(J) sum_m (dr_a/dx_m)(dr_b/dx_m), in the order
    (rr, ss, tt, rs, rt, st); B = w_i w_j w_k det(J).
    Returns G[6, e, k, j, i], B[e, k, j, i], detJ[e, k, j, i]."""
    xi, w = gll(N)
    D = deriv_matrix(N, xi)
    E = X.shape[1]
    n = N + 1
    Jac = np.zeros((E, n, n, n, 3, 3))
    for m in range(3):
        Jac[..., m, 0] = apply_r(D, X[m])
        Jac[..., m, 1] = apply_s(D, X[m])
        Jac[..., m, 2] = apply_t(D, X[m])
    detJ = np.linalg.det(Jac)
    if np.any(detJ <= 0.0):
        raise ValueError("non-positive Jacobian")
    Jinv = np.linalg.inv(Jac)              # Jinv[..., a, m] = dr_a/dx_m
    wq = w[:, None, None] * w[None, :, None] * w[None, None, :]   # [k, j, i]
    B = wq[None] * detJ
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    G = np.zeros((6, E, n, n, n))
    for q, (a, b) in enumerate(pairs):
        G[q] = B * np.sum(Jinv[..., a, :] * Jinv[..., b, :], axis=-1)
    return G, B, detJ


# --------------------------------------------------------------------------
# 3. Connectivity: global numbering, multiplicity, Dirichlet mask.
# --------------------------------------------------------------------------


def box_global_index(kx, ky, kz, N):
    """Integer grid position (I, J, K) of every local node, shape [3, e, k, j, i]."""
    n = N + 1
    E = kx * ky * kz
    P = np.zeros((3, E, n, n, n), dtype=np.int64)
    r = np.arange(n)
    for ez in range(kz):
        for ey in range(ky):
            for ex in range(kx):
                e = ex + kx * (ey + ky * ez)
                P[0, e] = (ex * N + r)[None, None, :]
                P[1, e] = (ey * N + r)[None, :, None]
                P[2, e] = (ez * N + r)[:, None, None]
    return P


def box_gid(kx, ky, kz, N):
    """Global id of every local node: I + (kx N + 1)(J + (ky N + 1) K)."""
    I, J, K = box_global_index(kx, ky, kz, N)
    gx, gy = kx * N + 1, ky * N + 1
    return (I + gx * (J + gy * K)).reshape(-1)


def box_mask(kx, ky, kz, N):
    """1 at interior nodes, 0 at every node on the six faces of the box."""
    I, J, K = box_global_index(kx, ky, kz, N)
    on_face = ((I == 0) | (I == kx * N) | (J == 0) | (J == ky * N)
               | (K == 0) | (K == kz * N))
    return np.where(on_face, 0.0, 1.0).reshape(-1)


def multiplicity(gid):
    """Number of local copies of each local node's global node."""
    return np.bincount(gid)[gid].astype(np.float64)


def dssum(v, gid):
    """Direct-stiffness summation Sigma' = Q Q^T: every local copy of a global
    node receives the sum over all copies of that node."""
    return np.bincount(gid, weights=v)[gid]


# --------------------------------------------------------------------------
# 4. The operator.
# --------------------------------------------------------------------------


def ax_local(u, G, D):
    """Unassembled element operator w_L = sum_a D_a^T (sum_b G_ab D_b u_L).

    u is a flat local vector; G is [6, e, k, j, i]; returns a flat vector."""
    E = G.shape[1]
    n = D.shape[0]
    U = u.reshape(E, n, n, n)
    ur, us, ut = apply_r(D, U), apply_s(D, U), apply_t(D, U)
    grr, gss, gtt, grs, grt, gst = G
    vr = grr * ur + grs * us + grt * ut
    vs = grs * ur + gss * us + gst * ut
    vt = grt * ur + gst * us + gtt * ut
    w = apply_r(D.T, vr) + apply_s(D.T, vs) + apply_t(D.T, vt)
    return w.reshape(-1)


class Problem:
    """One SEM Poisson problem on a box mesh, with everything the hot path reads."""

    def __init__(self, kx, ky, kz, N, deform=False, amp=0.05,
                 lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        self.kx, self.ky, self.kz, self.N = kx, ky, kz, N
        self.n = N + 1
        self.E = kx * ky * kz
        self.L = self.E * self.n ** 3
        self.xi, self.w = gll(N)
        self.D = deriv_matrix(N, self.xi)
        X = box_coords(kx, ky, kz, N, lo, hi)
        if deform:
            X = deform_cyclic(X, amp)
        self.X = X
        self.G, self.B, self.detJ = geometry(X, N)
        self.gid = box_gid(kx, ky, kz, N)
        self.U = int(self.gid.max()) + 1
        self.mask = box_mask(kx, ky, kz, N)
        self.mult = multiplicity(self.gid)
        self.c = self.mask / self.mult
        self.minv = self.jacobi_inverse()

    # -- operator pieces ---------------------------------------------------
    def ax_local(self, u):
        return ax_local(u, self.G, self.D)

    def dssum(self, v):
        return dssum(v, self.gid)

    def ax(self, u):
        """Full operator A_L u = mask * QQ^T (w_L)."""
        return self.mask * self.dssum(self.ax_local(u))

    def ax_unmasked(self, u):
        return self.dssum(self.ax_local(u))

    def diag_local(self):
        """diag of the unassembled element operator at node (i, j, k):
        sum_l D_li^2 G_rr(l,j,k) + sum_l D_lj^2 G_ss(i,l,k) + sum_l D_lk^2 G_tt(i,j,l)
        + 2 (D_ii D_jj G_rs + D_ii D_kk G_rt + D_jj D_kk G_st)(i,j,k)."""
        D = self.D
        D2 = D ** 2
        grr, gss, gtt, grs, grt, gst = self.G
        d = np.einsum('li,ekjl->ekji', D2, grr)
        d = d + np.einsum('lj,ekli->ekji', D2, gss)
        d = d + np.einsum('lk,elji->ekji', D2, gtt)
        dd = np.diag(D)
        di = dd[None, None, None, :]
        dj = dd[None, None, :, None]
        dk = dd[None, :, None, None]
        d = d + 2.0 * (di * dj * grs + di * dk * grt + dj * dk * gst)
        return d.reshape(-1)

    def jacobi_inverse(self):
        """J^{-1} = mask / QQ^T(diag_L): the Jacobi preconditioner, FP64."""
        dg = self.dssum(self.diag_local())
        out = np.zeros_like(dg)
        m = self.mask > 0
        out[m] = 1.0 / dg[m]
        return out

    # -- reductions ----------------------------------------------------------
    def glsc3(self, a, b):
        """Weighted inner product sum_i a_i c_i b_i (glsc3 of the profiling table)."""
        return float(np.sum(a * self.c * b))

    def norm_c(self, v):
        return math.sqrt(self.glsc3(v, v))

    # -- right-hand sides ----------------------------------------------------
    def rhs_sine(self):
        """b = mask * QQ^T(B_L * 3 pi^2 sin(pi x) sin(pi y) sin(pi z)) at the nodes."""
        x, y, z = (self.X[m].reshape(-1) for m in range(3))
        f = 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        return self.mask * self.dssum(self.B.reshape(-1) * f)

    def exact_sine(self):
        x, y, z = (self.X[m].reshape(-1) for m in range(3))
        return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)

    def rhs_uniform(self, seed):
        """b_g ~ U[-1, 1) per global node from SplitMix64(seed, g), masked."""
        return self.mask * splitmix_uniform(seed, self.gid)

    # -- solver --------------------------------------------------------------
    def pcg(self, b, x0=None, tol=1e-10, maxit=500, precond=True, fixed_iters=None):
        """Jacobi-preconditioned CG in the order of the paper's profiling table.

        Returns (x, iterations, history) where history[k] is ||r_k||_c/||b||_c
        after iteration k (history[0] is the initial residual)."""
        minv = self.minv if precond else self.mask.copy()
        x = np.zeros(self.L) if x0 is None else self.mask * x0
        r = b - self.ax(x)
        bnorm = self.norm_c(b)
        if bnorm == 0.0:
            return x, 0, [0.0]
        hist = [self.norm_c(r) / bnorm]
        if fixed_iters is None and hist[0] <= tol:
            return x, 0, hist
        z = minv * r
        rtz = self.glsc3(r, z)
        p = np.zeros(self.L)
        rtz_old = None
        it = 0
        nmax = fixed_iters if fixed_iters is not None else maxit
        while it < nmax:
            it += 1
            beta = 0.0 if rtz_old is None else rtz / rtz_old
            p = z + beta * p                       # add2s1
            w = self.ax(p)                         # ax
            pap = self.glsc3(w, p)                 # glsc3(w, c, p)
            alpha = rtz / pap
            x = x + alpha * p                      # add2s2(x, p, alpha)
            r = r - alpha * w                      # add2s2(r, w, -alpha)
            rtr = self.glsc3(r, r)                 # glsc3(r, c, r)
            hist.append(math.sqrt(rtr) / bnorm)
            if fixed_iters is None and hist[-1] <= tol:
                break
            z = minv * r                           # solveM (Jacobi)
            rtz_old = rtz
            rtz = self.glsc3(r, z)                 # glsc3(r, c, z)
        return x, it, hist

    def true_relres(self, b, x):
        return self.norm_c(b - self.ax(x)) / self.norm_c(b)


# --------------------------------------------------------------------------
# 5. Counter-based random numbers (SplitMix64, Steele, Lea & Flood 2014).
# --------------------------------------------------------------------------

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counter):
    """Output number counter+1 of SplitMix64 started from state `seed`:
    z = seed + (counter + 1) * gamma (mod 2^64), then the finaliser
    z ^= z >> 30; z *= M1; z ^= z >> 27; z *= M2; z ^= z >> 31."""
    with np.errstate(over='ignore'):
        c = np.asarray(counter, dtype=np.uint64)
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix_uniform(seed, counter):
    """2 * (top 53 bits of splitmix64 / 2^53) - 1, in [-1, 1)."""
    z = splitmix64(seed, counter)
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)) - 1.0
