"""p-multigrid preconditioner with overlapping Schwarz smoothing (CPU oracle, numpy FP64).

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU legs).

The paper runs Nekbone both without and with its multigrid preconditioner
(Sec. 3.1, profiling table: `solveM` takes 70 % of the time when enabled;
Sec. 4: the Schwarz weights' square roots must stay FP64 in the mixed
version), but prints no algorithm for it.  The reading implemented here, in
the spirit of Nekbone's hybrid Schwarz multigrid, is:

  * levels: the same box mesh and geometry at polynomial orders
    N_0 = N, N_{l+1} = max(1, floor(N_l / 2)), down to 1; each level's
    operator is the SEM Poisson operator rediscretised at its order;
  * transfer: prolongation P = tensor-product Lagrange interpolation from the
    coarse to the fine GLL nodes in every element (continuous in, continuous
    out); restriction = P^T on unique nodes, i.e. in the local layout
    r_c = mask_c QQ^T_c (J^T x J^T x J^T)(r_f / multiplicity_f);
  * smoother: additive overlapping Schwarz, one subdomain per element,
    extended by one node layer into each neighbour (the (n+2)^3 block of the
    global node grid around the element); the local problem is the
    separable operator A_x (x) B_y (x) B_z + B_x (x) A_y (x) B_z +
    B_x (x) B_y (x) A_z built from 1-D GLL stiffness A and mass B on the
    extended 1-D grids (element and neighbour lengths per direction, homogeneous
    Dirichlet beyond the block and on the domain boundary) and solved by fast
    diagonalisation (A_d S_d = B_d S_d L_d, S_d^T B_d S_d = I); the
    subdomain corrections are summed with symmetric weights 1/sqrt(c), c the
    number of blocks holding the node -- the square root the paper moves to
    FP64 -- and damped by omega = 1/lambda_max(S A) (power iteration);
  * h-levels below the N = 1 level: while kx, ky, kz are all even and their
    halves all at least 2, the next level is the N = 1 discretisation of the
    box with kx/2 x ky/2 x kz/2 elements (same domain and deformation, each
    coarse element holding 2 x 2 x 2 fine ones); prolongation = trilinear
    interpolation of the coarse element's eight vertex values at the fine
    nodes (reference positions 0, 1/2, 1), restriction its adjoint on unique
    nodes; the h-levels use the same smoother;
  * cycle: symmetric V-cycle (pre-smooth, coarse correction, post-smooth);
    the coarsest level applies the smoother only (no direct coarse solve),
    so the preconditioner is linear, symmetric and positive definite.

On an undeformed uniform mesh the separable local operator equals the
assembled stiffness matrix restricted to the block, so each local solve is
exact there (pinned against a dense solve).
"""
from __future__ import annotations

import math

import numpy as np

from .sem_oracle import Problem, box_global_index, deriv_matrix, gll, splitmix_uniform


def level_orders(N):
    """Polynomial orders of the V-cycle levels, finest first."""
    out = [N]
    while out[-1] > 1:
        out.append(max(1, out[-1] // 2))
    return out


def h_levels(kx, ky, kz):
    """Mesh sizes of the h-levels below the N = 1 level, finest first."""
    out = []
    while kx % 2 == 0 and ky % 2 == 0 and kz % 2 == 0 and min(kx, ky, kz) >= 4:
        kx, ky, kz = kx // 2, ky // 2, kz // 2
        out.append((kx, ky, kz))
    return out


# trilinear interpolation inside a coarse element: H[s][i][a] = weight of
# coarse vertex a (0, 1) at fine node i (0, 1) of the fine element in half s
_H = np.array([[[1.0, 0.0], [0.5, 0.5]],
               [[0.5, 0.5], [0.0, 1.0]]])


def interp_matrix(Nc, Nf):
    """J[p, a] = l_a(x_p): coarse GLL Lagrange basis a at fine GLL node p."""
    xc, _ = gll(Nc)
    xf, _ = gll(Nf)
    J = np.ones((Nf + 1, Nc + 1))
    for a in range(Nc + 1):
        for m in range(Nc + 1):
            if m != a:
                J[:, a] *= (xf - xc[m]) / (xc[a] - xc[m])
    return J


def _apply3(M, u):
    """(M x M x M) applied to element blocks u[e, k, j, i] (M: rows out, cols in)."""
    u = np.einsum('ia,ekja->ekji', M, u)
    u = np.einsum('jb,ekbi->ekji', M, u)
    return np.einsum('kc,ecji->ekji', M, u)


def element_lengths(P):
    """[E, 3] length of every element along r, s, t: the distance between the
    centroids of its two opposite faces (exact for undeformed boxes)."""
    X = P.X                                              # [3, e, k, j, i]
    L = np.zeros((P.E, 3))
    L[:, 0] = np.linalg.norm(X[:, :, :, :, -1].mean(axis=(2, 3)) - X[:, :, :, :, 0].mean(axis=(2, 3)), axis=0)
    L[:, 1] = np.linalg.norm(X[:, :, :, -1, :].mean(axis=(2, 3)) - X[:, :, :, 0, :].mean(axis=(2, 3)), axis=0)
    L[:, 2] = np.linalg.norm(X[:, :, -1, :, :].mean(axis=(2, 3)) - X[:, :, 0, :, :].mean(axis=(2, 3)), axis=0)
    return L


def extended_active(N, has_left, has_right):
    """Which of the n+2 extended 1-D indices are unknowns: the overlap node
    needs a neighbour and N >= 2 (at N = 1 it would be the neighbour's far
    node, which is held at zero instead); the element's own end node needs a
    neighbour (otherwise it lies on the Dirichlet boundary)."""
    n = N + 1
    act = np.ones(n + 2, dtype=bool)
    act[0] = has_left and N >= 2
    act[1] = has_left
    act[n] = has_right
    act[n + 1] = has_right and N >= 2
    return act


def extended_1d(N, hl, h, hr, has_left, has_right):
    """1-D stiffness A and (diagonal) mass B on the extended grid of one
    element: index 0 = the left neighbour's node N-1, 1..N+1 = the element's
    nodes 0..N, N+2 = the right neighbour's node 1.  Assembled from the three
    1-D elements (lengths hl, h, hr) with every other node held at zero;
    indices that are not unknowns (extended_active) get identity rows and
    columns."""
    x, w = gll(N)
    n = N + 1
    D = deriv_matrix(N, x)
    Ahat = D.T @ np.diag(w) @ D
    m = n + 2
    A = np.zeros((m, m))
    B = np.zeros(m)
    # own element: ext indices 1..n
    A[1:n + 1, 1:n + 1] += (2.0 / h) * Ahat
    B[1:n + 1] += (h / 2.0) * w
    # left neighbour's nodes N-1, N -> ext 0, 1
    sl = [N - 1, N]
    A[np.ix_([0, 1], [0, 1])] += (2.0 / hl) * Ahat[np.ix_(sl, sl)]
    B[[0, 1]] += (hl / 2.0) * w[sl]
    # right neighbour's nodes 0, 1 -> ext n, n+1
    sr = [0, 1]
    A[np.ix_([n, n + 1], [n, n + 1])] += (2.0 / hr) * Ahat[np.ix_(sr, sr)]
    B[[n, n + 1]] += (hr / 2.0) * w[sr]
    act = extended_active(N, has_left, has_right)
    for q in np.nonzero(~act)[0]:
        A[q, :] = 0.0
        A[:, q] = 0.0
        A[q, q] = 1.0
        B[q] = 1.0
    return A, B


def fdm_1d(A, B):
    """Generalised eigenpairs A S = B S diag(lam), S^T B S = I (B diagonal)."""
    bi = 1.0 / np.sqrt(B)
    lam, V = np.linalg.eigh(bi[:, None] * A * bi[None, :])
    return bi[:, None] * V, lam


class Level:
    """One level: the problem at its order plus the Schwarz data."""

    def __init__(self, kx, ky, kz, N, deform):
        self.P = P = Problem(kx, ky, kz, N, deform=deform)
        n = N + 1
        self.N, self.n = N, n
        self.gx, self.gy, self.gz = kx * N + 1, ky * N + 1, kz * N + 1
        lengths = element_lengths(P)
        # per element, per direction: S (n+2 x n+2) and lam (n+2)
        self.S = np.zeros((3, P.E, n + 2, n + 2))
        self.lam = np.zeros((3, P.E, n + 2))
        self.act = np.zeros((3, P.E, n + 2))          # 1 where the extended index is an unknown
        ks = (kx, ky, kz)
        strides = (1, kx, kx * ky)
        for e in range(P.E):
            ec = (e % kx, (e // kx) % ky, e // (kx * ky))
            for d in range(3):
                has_l = ec[d] > 0
                has_r = ec[d] < ks[d] - 1
                h = lengths[e, d]
                hl = lengths[e - strides[d], d] if has_l else h
                hr = lengths[e + strides[d], d] if has_r else h
                A, B = extended_1d(N, hl, h, hr, has_l, has_r)
                self.S[d, e], self.lam[d, e] = fdm_1d(A, B)
                self.act[d, e] = extended_active(N, has_l, has_r)
        # index arrays of every element's extended block in the padded grid
        # (grid index g -> padded g + 1; block = g in [eN - 1, eN + N + 1])
        ex = np.arange(P.E) % kx
        ey = (np.arange(P.E) // kx) % ky
        ez = np.arange(P.E) // (kx * ky)
        r = np.arange(n + 2)
        self.bx = ex[:, None] * N + r[None, :]
        self.by = ey[:, None] * N + r[None, :]
        self.bz = ez[:, None] * N + r[None, :]
        # grid position of every local node, and the block counts c
        I, J, K = box_global_index(kx, ky, kz, N)
        self.I, self.J, self.K = I.reshape(-1), J.reshape(-1), K.reshape(-1)
        cnt = np.zeros((self.gz + 2, self.gy + 2, self.gx + 2))
        np.add.at(cnt, (self.bz[:, :, None, None], self.by[:, None, :, None],
                        self.bx[:, None, None, :]), self.active_blocks())
        self.count = cnt[1:-1, 1:-1, 1:-1]
        # the Schwarz weights (1 where no block holds the node: Dirichlet nodes)
        self.wsqrt = 1.0 / np.sqrt(np.maximum(self.count, 1.0))
        self.omega = 1.0

    # local (continuous) <-> grid
    def to_grid(self, v):
        g = np.zeros((self.gz, self.gy, self.gx))
        g[self.K, self.J, self.I] = v
        return g

    def from_grid(self, g):
        return g[self.K, self.J, self.I]

    def active_blocks(self):
        """[E, n+2, n+2, n+2]: 1 at the unknowns of every extended block."""
        ax, ay, az = self.act
        return az[:, :, None, None] * ay[:, None, :, None] * ax[:, None, None, :]

    def local_solve(self, blocks):
        """Fast-diagonalisation solve of every element's separable extended
        problem: blocks[e, k, j, i] (n+2)^3 right-hand sides -> solutions."""
        Sx, Sy, Sz = self.S
        lx, ly, lz = self.lam
        t = np.einsum('eai,ekja->ekji', Sx, blocks)          # S_x^T along i
        t = np.einsum('ebj,ekbi->ekji', Sy, t)
        t = np.einsum('eck,ecji->ekji', Sz, t)
        t = t / (lz[:, :, None, None] + ly[:, None, :, None] + lx[:, None, None, :])
        t = np.einsum('eia,ekja->ekji', Sx, t)               # S_x along i
        t = np.einsum('ejb,ekbi->ekji', Sy, t)
        return np.einsum('ekc,ecji->ekji', Sz, t)

    def schwarz(self, r):
        """Weighted additive Schwarz: W^(1/2) sum_e R_e^T Atilde_e^{-1} R_e W^(1/2) r,
        masked (r continuous and masked, local layout)."""
        g = np.zeros((self.gz + 2, self.gy + 2, self.gx + 2))
        g[1:-1, 1:-1, 1:-1] = self.to_grid(r) * self.wsqrt
        idx = (self.bz[:, :, None, None], self.by[:, None, :, None], self.bx[:, None, None, :])
        act = self.active_blocks()
        z = act * self.local_solve(act * g[idx])
        acc = np.zeros_like(g)
        np.add.at(acc, idx, z)
        zg = acc[1:-1, 1:-1, 1:-1] * self.wsqrt
        return self.P.mask * self.from_grid(zg)


class PMG:
    """The V-cycle preconditioner over all levels of a box problem."""

    def __init__(self, kx, ky, kz, N, deform=False, power_iters=20, seed=12345, hcoarsen=True):
        self.levels = [Level(kx, ky, kz, Nl, deform) for Nl in level_orders(N)]
        self.J = [interp_matrix(self.levels[l + 1].N, self.levels[l].N)
                  for l in range(len(self.levels) - 1)]
        self.n_p = len(self.levels)          # levels 0 .. n_p-1: orders N .. 1
        if hcoarsen:
            for dims in h_levels(kx, ky, kz):
                self.levels.append(Level(*dims, 1, deform))
        for lev in self.levels:
            lev.omega = 1.0 / self.lambda_max(lev, power_iters, seed)

    @staticmethod
    def lambda_max(lev, iters, seed):
        """Largest eigenvalue of S A (self-adjoint in the A inner product) by
        power iteration from a SplitMix64 vector, Rayleigh quotient in A."""
        P = lev.P
        x = P.mask * splitmix_uniform(seed, P.gid)
        if P.glsc3(x, x) == 0.0:
            return 1.0          # a level without interior nodes: nothing to damp
        lam = 0.0
        for _ in range(iters):
            y = lev.schwarz(P.ax(x))
            Ax = P.ax(x)
            lam = P.glsc3(y, P.ax(y)) / P.glsc3(y, Ax)    # <SAx, A SAx> / <SAx, A x>
            x = y / math.sqrt(P.glsc3(y, y))
        return lam

    def _children(self, l):
        """h-pair (l, l+1): for every fine element its coarse element and
        its half (sx, sy, sz) in each direction."""
        f, c = self.levels[l].P, self.levels[l + 1].P
        e = np.arange(f.E)
        ex, ey, ez = e % f.kx, (e // f.kx) % f.ky, e // (f.kx * f.ky)
        ce = ex // 2 + c.kx * (ey // 2 + c.ky * (ez // 2))
        return ce, ex % 2, ey % 2, ez % 2

    def prolong(self, l, zc):
        """Coarse level l+1 -> fine level l, element by element."""
        f, c = self.levels[l], self.levels[l + 1]
        if l + 1 >= self.n_p:
            # trilinear: fine node (i, j, k) of the child in half (sx, sy, sz)
            ce, sx, sy, sz = self._children(l)
            u = zc.reshape(c.P.E, 2, 2, 2)[ce]                   # [Ef, c, b, a]
            out = np.einsum('eia,ejb,ekc,ecba->ekji', _H[sx], _H[sy], _H[sz], u)
            return out.reshape(-1)
        u = zc.reshape(c.P.E, c.n, c.n, c.n)
        return _apply3(self.J[l], u).reshape(-1)

    def restrict(self, l, r):
        """Fine level l -> coarse level l+1: P^T on unique nodes."""
        f, c = self.levels[l], self.levels[l + 1]
        if l + 1 >= self.n_p:
            ce, sx, sy, sz = self._children(l)
            u = (r / f.P.mult).reshape(f.P.E, 2, 2, 2)           # [Ef, k, j, i]
            t = np.einsum('eia,ejb,ekc,ekji->ecba', _H[sx], _H[sy], _H[sz], u)
            rc = np.zeros((c.P.E, 2, 2, 2))
            np.add.at(rc, ce, t)
            return c.P.mask * c.P.dssum(rc.reshape(-1))
        u = (r / f.P.mult).reshape(f.P.E, f.n, f.n, f.n)
        rc = _apply3(self.J[l].T, u).reshape(-1)
        return c.P.mask * c.P.dssum(rc)

    def vcycle(self, r, l=0):
        lev = self.levels[l]
        if l == len(self.levels) - 1:
            return lev.omega * lev.schwarz(r)
        z = lev.omega * lev.schwarz(r)
        z = z + self.prolong(l, self.vcycle(self.restrict(l, r - lev.P.ax(z)), l + 1))
        return z + lev.omega * lev.schwarz(r - lev.P.ax(z))

    def pcg(self, b, tol=1e-10, maxit=500):
        """CG preconditioned by one V-cycle per iteration (the profiling
        table's loop with solveM = vcycle).  Returns (x, iterations, history)."""
        P = self.levels[0].P
        x = np.zeros(P.L)
        r = b.copy()
        bnorm = P.norm_c(b)
        hist = [P.norm_c(r) / bnorm]
        z = self.vcycle(r)
        rtz = P.glsc3(r, z)
        p = np.zeros(P.L)
        rtz_old = None
        it = 0
        while it < maxit:
            it += 1
            beta = 0.0 if rtz_old is None else rtz / rtz_old
            p = z + beta * p
            w = P.ax(p)
            alpha = rtz / P.glsc3(w, p)
            x = x + alpha * p
            r = r - alpha * w
            hist.append(math.sqrt(P.glsc3(r, r)) / bnorm)
            if hist[-1] <= tol:
                break
            z = self.vcycle(r)
            rtz_old = rtz
            rtz = P.glsc3(r, z)
        return x, it, hist
