"""CPU oracle for the learned initial guess (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).

The paper has no learned component; this is the extension the hot path
carries: an element-local network maps an element's right-hand side,
a summary of its geometric factors and its neighbours' right-hand-side means
to the element's values of u, and the continuity projection
x0 = c * QQ^T(u_pred) (c = mask / multiplicity, the glsc3 weight of the
paper's CG loop) turns the element predictions into a continuous, masked
initial guess for PCG.  Parity of the guess's QUALITY is unpinned (judged by
the iterations it saves); the network arithmetic below is pinned by central
finite differences.

Definitions (all per element e of a box mesh, local node order i + n j + n^2 k):
  * random Fourier right-hand side: f(x,y,z) = sum_{k in {1..K}^3}
    a_k sin(pi k1 x) sin(pi k2 y) sin(pi k3 z), a_k = xi_k / |k|^2 with
    xi_k uniform in [-1, 1) from SplitMix64(seed, sample * K^3 + index(k)),
    index(k) = (k1-1) + K (k2-1) + K^2 (k3-1); b = mask * QQ^T(B f).
  * scale s_e = sqrt(mean_e(b_L^2)) + 1e-30 over the element's n^3 values.
  * features (n^3 + 12 + 6 values): b_L / s_e; for each geometric factor
    G1..G6 its element mean and standard deviation; for each face
    (r-, r+, s-, s+, t-, t+) the mean of b_L over the whole neighbouring
    element divided by s_e (0 where the face is on the domain boundary).
  * targets: x_L / s_e (x the converged solution); the network is trained
    on targets / t with t the RMS of all training targets (prediction s_e t y).
  * network: h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3,
    loss = mean over rows and outputs of (y - t)^2.
  * prediction: u_pred_e = s_e * y_e, x0 = c * QQ^T(u_pred).
  * coarse features (optional, 9 more values): z_c from c steps of
    multigrid-Richardson iteration z <- z + M^{-1}(b - A z) from z = 0 (M^{-1}
    one V-cycle of the multigrid preconditioner, A the assembled masked
    operator); z_c at the element's 8 vertices (i, j, k in {0, N}, vertex
    index v = (i>0) + 2 (j>0) + 4 (k>0)) and the element mean of z_c, all
    divided by s_e.
"""
from __future__ import annotations

import numpy as np

from .sem_oracle import splitmix_uniform


def fourier_coefficients(seed: int, sample: int, K: int = 8):
    """a_k = xi_k / |k|^2 over k in {1..K}^3, as an array [k3-1, k2-1, k1-1]."""
    idx = np.arange(K ** 3)
    xi = splitmix_uniform(seed, sample * K ** 3 + idx)
    k1 = idx % K + 1
    k2 = (idx // K) % K + 1
    k3 = idx // (K * K) + 1
    a = xi / (k1 ** 2 + k2 ** 2 + k3 ** 2)
    return a.reshape(K, K, K)


def fourier_rhs(P, seed: int, sample: int, K: int = 8):
    """b = mask * QQ^T(B * f) for the random Fourier f of (seed, sample)."""
    return fourier_rhs_from(P, fourier_coefficients(seed, sample, K))


def fourier_rhs_from(P, a):
    """b = mask * QQ^T(B * f), f = sum_k a[k3-1, k2-1, k1-1] sin(pi k1 x) sin(pi k2 y) sin(pi k3 z)."""
    K = a.shape[0]
    x, y, z = (P.X[m].reshape(-1) for m in range(3))
    ks = np.arange(1, K + 1)
    sx = np.sin(np.pi * np.outer(x, ks))
    sy = np.sin(np.pi * np.outer(y, ks))
    sz = np.sin(np.pi * np.outer(z, ks))
    f = np.einsum('lc,lb,la,cba->l', sz, sy, sx, a)
    return P.mask * P.dssum(P.B.reshape(-1) * f)


def element_neighbours(kx, ky, kz):
    """[E, 6] neighbour element index across faces r-, r+, s-, s+, t-, t+ (-1 = boundary)."""
    E = kx * ky * kz
    nb = -np.ones((E, 6), dtype=np.int64)
    for ez in range(kz):
        for ey in range(ky):
            for ex in range(kx):
                e = ex + kx * (ey + ky * ez)
                if ex > 0: nb[e, 0] = e - 1
                if ex < kx - 1: nb[e, 1] = e + 1
                if ey > 0: nb[e, 2] = e - kx
                if ey < ky - 1: nb[e, 3] = e + kx
                if ez > 0: nb[e, 4] = e - kx * ky
                if ez < kz - 1: nb[e, 5] = e + kx * ky
    return nb


def features(P, b):
    """Feature matrix [E, n^3 + 18] and scales [E] of right-hand side b."""
    n3 = P.n ** 3
    bl = b.reshape(P.E, n3)
    s = np.sqrt(np.mean(bl ** 2, axis=1)) + 1e-30
    G = P.G.reshape(6, P.E, n3)
    gm = G.mean(axis=2).T                     # [E, 6]
    gs = G.std(axis=2).T                      # [E, 6]
    nb = element_neighbours(P.kx, P.ky, P.kz)
    emean = bl.mean(axis=1)
    face = np.where(nb >= 0, emean[np.maximum(nb, 0)], 0.0) / s[:, None]
    X = np.concatenate([bl / s[:, None], gm, gs, face], axis=1)
    return X, s


def coarse_features(P, vcycle, b, cycles, s):
    """The 9 coarse features [E, 9] (vertex values and mean of the multigrid-
    Richardson approximation z, / s_e); vcycle(r) applies one V-cycle."""
    z = np.zeros(P.L)
    for _ in range(cycles):
        z = z + vcycle(b - P.ax(z))
    n, n3 = P.n, P.n ** 3
    zl = z.reshape(P.E, n3)
    out = np.zeros((P.E, 9))
    for v in range(8):
        i = n - 1 if v & 1 else 0
        j = n - 1 if v & 2 else 0
        k = n - 1 if v & 4 else 0
        out[:, v] = zl[:, i + n * (j + n * k)]
    out[:, 8] = zl.mean(axis=1)
    return out / s[:, None]


def targets(P, x, s):
    return x.reshape(P.E, P.n ** 3) / s[:, None]


def continuity_projection(P, u_pred_local):
    """x0 = c * QQ^T(u_pred): the average of the element predictions per node, masked."""
    return P.c * P.dssum(u_pred_local.reshape(-1))


class MLP:
    """FP64 reference network with explicit forward and backward passes."""

    def __init__(self, sizes, params=None, seed=0):
        self.sizes = list(sizes)
        if params is None:
            g = np.random.default_rng(seed)
            params = []
            for a, b in zip(sizes[:-1], sizes[1:]):
                params.append(g.standard_normal((a, b)) * np.sqrt(2.0 / a))
                params.append(np.zeros(b))
        self.params = [np.asarray(p, dtype=np.float64) for p in params]

    def forward(self, X):
        acts = [X]
        h = X
        nl = len(self.sizes) - 1
        for li in range(nl):
            W, bvec = self.params[2 * li], self.params[2 * li + 1]
            z = h @ W + bvec
            h = np.maximum(z, 0.0) if li < nl - 1 else z
            acts.append(h)
        return h, acts

    def loss(self, X, T):
        y, _ = self.forward(X)
        return float(np.mean((y - T) ** 2))

    def gradients(self, X, T):
        """Gradients of loss = mean((y - T)^2) with respect to every parameter."""
        y, acts = self.forward(X)
        nl = len(self.sizes) - 1
        d = 2.0 * (y - T) / y.size
        grads = [None] * len(self.params)
        for li in reversed(range(nl)):
            h_in = acts[li]
            grads[2 * li] = h_in.T @ d
            grads[2 * li + 1] = d.sum(axis=0)
            if li > 0:
                d = (d @ self.params[2 * li].T) * (acts[li] > 0.0)
        return grads

    def adam_step(self, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        """One Adam update (Kingma & Ba 2015) of every parameter in place."""
        state["t"] = state.get("t", 0) + 1
        t = state["t"]
        if "m" not in state:
            state["m"] = [np.zeros_like(p) for p in self.params]
            state["v"] = [np.zeros_like(p) for p in self.params]
        for q, g in enumerate(grads):
            state["m"][q] = b1 * state["m"][q] + (1 - b1) * g
            state["v"][q] = b2 * state["v"][q] + (1 - b2) * g * g
            mh = state["m"][q] / (1 - b1 ** t)
            vh = state["v"][q] / (1 - b2 ** t)
            self.params[q] = self.params[q] - lr * mh / (np.sqrt(vh) + eps)
