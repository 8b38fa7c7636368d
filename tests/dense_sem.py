"""Independent dense assembly of the SEM Poisson stiffness matrix, for pinning the oracle.

Nothing here is taken from the oracle: the 1-D Lagrange basis and its
derivative come from numpy's polynomial routines (coefficients of
prod_{m != a} (x - x_m)/(x_a - x_m)), the GLL nodes from the roots of the
derivative of the Legendre polynomial (numpy.polynomial.legendre), the
geometry from differentiating the isoparametric map basis function by basis
function, and the global numbering from an explicit dictionary of grid points.
The element matrix is the textbook quadrature of the Galerkin weak form of
-Laplace(u) = f:  A^e_IJ = sum_q w_q |det J_q| (J_q^{-T} grad phi_I)(J_q^{-T} grad phi_J).
"""
from __future__ import annotations

import itertools

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def gll_numpy(N):
    """GLL nodes as -1, the roots of P_N', 1; weights 2/(N(N+1) P_N(x)^2)."""
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(cN)))) if N > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * npleg.legval(x, cN) ** 2)
    return x, w


def lagrange_tables(x):
    """L[a, p] = l_a(x_p) (identity) and dL[a, p] = l_a'(x_p) from explicit polynomials."""
    n = len(x)
    dL = np.zeros((n, n))
    for a in range(n):
        coef = np.array([1.0])
        for m in range(n):
            if m != a:
                coef = nppoly.polymul(coef, np.array([-x[m], 1.0]) / (x[a] - x[m]))
        dL[a] = nppoly.polyval(x, nppoly.polyder(coef))
    return np.eye(n), dL


def dense_box_matrix(kx, ky, kz, N, deform_amp=0.0):
    """Dense unmasked stiffness matrix on the unique nodes of a box mesh of [0,1]^3.

    Returns (A, gid_local) with gid_local the global index of each local node in
    the solver's local ordering (element ex + kx (ey + ky ez), node i + n j + n^2 k)."""
    x, w = gll_numpy(N)
    n = N + 1
    _, dL = lagrange_tables(x)
    # global numbering: a dict of integer grid points in first-seen order
    index = {}
    gid_local = []
    coords = {}
    for ez, ey, ex in itertools.product(range(kz), range(ky), range(kx)):
        for k, j, i in itertools.product(range(n), range(n), range(n)):
            key = (ex * N + i, ey * N + j, ez * N + k)
            if key not in index:
                index[key] = len(index)
                X0 = np.array([(ex + (1 + x[i]) / 2) / kx,
                               (ey + (1 + x[j]) / 2) / ky,
                               (ez + (1 + x[k]) / 2) / kz])
                if deform_amp:
                    s = lambda a: np.sin(2 * np.pi * a)
                    X0 = X0 + deform_amp * np.array([s(X0[1]) * s(X0[2]),
                                                      s(X0[2]) * s(X0[0]),
                                                      s(X0[0]) * s(X0[1])])
                coords[index[key]] = X0
            gid_local.append(index[key])
    gid_local = np.array(gid_local)
    U = len(index)
    A = np.zeros((U, U))
    nodes = list(itertools.product(range(n), range(n), range(n)))  # (k, j, i)
    for e in range(kx * ky * kz):
        g = gid_local[e * n ** 3:(e + 1) * n ** 3]
        Xe = np.array([coords[gg] for gg in g])                   # [n^3, 3]
        Ae = np.zeros((n ** 3, n ** 3))
        for (qk, qj, qi) in nodes:
            # reference gradients of every basis function at quadrature point q
            grads = np.zeros((n ** 3, 3))
            for b, (k, j, i) in enumerate(nodes):
                grads[b, 0] = dL[i, qi] * (j == qj) * (k == qk)
                grads[b, 1] = (i == qi) * dL[j, qj] * (k == qk)
                grads[b, 2] = (i == qi) * (j == qj) * dL[k, qk]
            Jq = Xe.T @ grads                                        # dx_m/dr_a
            detJ = np.linalg.det(Jq)
            phys = grads @ np.linalg.inv(Jq)                         # [n^3, 3]
            Ae += w[qi] * w[qj] * w[qk] * abs(detJ) * (phys @ phys.T)
        A[np.ix_(g, g)] += Ae
    return A, gid_local


def boundary_unique(kx, ky, kz, N, gid_local):
    """Boolean per unique node: True on the box faces."""
    n = N + 1
    U = gid_local.max() + 1
    on = np.zeros(U, dtype=bool)
    for e, (ez, ey, ex) in enumerate(itertools.product(range(kz), range(ky), range(kx))):
        for l, (k, j, i) in enumerate(itertools.product(range(n), range(n), range(n))):
            I, J, K = ex * N + i, ey * N + j, ez * N + k
            if I in (0, kx * N) or J in (0, ky * N) or K in (0, kz * N):
                on[gid_local[e * n ** 3 + l]] = True
    return on
