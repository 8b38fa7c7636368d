"""Pins of the CPU oracle against closed forms, library routines and brute force.

Each test pins one piece of the oracle to something other than the oracle
itself: textbook values of the GLL rule, numpy's Legendre routines, exact
integrals, an independently assembled dense stiffness matrix, a dense linear
solve, and the published SplitMix64 sequence.
"""
import math
import os

import numpy as np
import pytest

from oracle import sem_oracle as so
from tests.dense_sem import boundary_unique, dense_box_matrix, gll_numpy, lagrange_tables

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- GLL rule
def test_gll_closed_forms():
    x, w = so.gll(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-14)
    x, w = so.gll(3)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)
    x, w = so.gll(4)                       # nodes 0, +-sqrt(3/7), +-1
    s = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


@pytest.mark.parametrize("N", list(range(1, 19)))
def test_gll_matches_numpy_legendre(N):
    x, w = so.gll(N)
    xr, wr = gll_numpy(N)
    np.testing.assert_allclose(x, xr, atol=2e-14)
    np.testing.assert_allclose(w, wr, rtol=1e-12)
    assert abs(w.sum() - 2.0) < 1e-13


@pytest.mark.parametrize("N", [2, 5, 7, 9, 15])
def test_gll_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = so.gll(N)
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13
    # degree 2N is not integrated exactly (the Lobatto rule has degree 2N-1)
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-11


@pytest.mark.parametrize("N", [1, 2, 4, 7, 11, 15])
def test_derivative_matrix_exact_on_polynomials(N):
    x, _ = so.gll(N)
    D = so.deriv_matrix(N, x)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0.0, atol=1e-12)
    for m in range(1, N + 1):
        np.testing.assert_allclose(D @ x ** m, m * x ** (m - 1), atol=1e-11 * N * N)


@pytest.mark.parametrize("N", [2, 3, 6, 9])
def test_derivative_matrix_matches_explicit_lagrange(N):
    x, _ = so.gll(N)
    _, dL = lagrange_tables(gll_numpy(N)[0])
    np.testing.assert_allclose(so.deriv_matrix(N, x), dL.T, atol=1e-10)


# ---------------------------------------------------------------- geometry
def test_geometry_undeformed_closed_form():
    k, N = 3, 5
    P = so.Problem(k, k, k, N)
    h = 1.0 / k
    np.testing.assert_allclose(P.detJ, (h / 2) ** 3, rtol=1e-13)
    x, w = so.gll(N)
    wq = (w[:, None, None] * w[None, :, None] * w[None, None, :])[None]
    for q in range(3):
        np.testing.assert_allclose(P.G[q], np.broadcast_to(wq * h / 2, P.G[q].shape), rtol=1e-12)
    for q in range(3, 6):
        assert np.abs(P.G[q]).max() < 1e-14
    assert abs(P.B.sum() - 1.0) < 1e-13


def test_geometry_deformed_volume_is_one():
    # det(I + grad d) - 1 for the cyclic sine deformation integrates to zero,
    # so the exact volume of the deformed box is 1; the isoparametric GLL
    # approximation converges to it spectrally.
    errs = []
    for N in (3, 5, 7, 9):
        P = so.Problem(4, 4, 4, N, deform=True)
        assert P.detJ.min() > 0
        errs.append(abs(P.B.sum() - 1.0))
    assert errs[-1] < 1e-9
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-12


# ---------------------------------------------------------------- numbering
def test_box_numbering_counts():
    kx, ky, kz, N = 3, 2, 4, 4
    P = so.Problem(kx, ky, kz, N)
    assert P.U == (kx * N + 1) * (ky * N + 1) * (kz * N + 1)
    assert len(np.unique(P.gid)) == P.U
    m = P.mult.reshape(P.E, P.n, P.n, P.n)
    # an interior corner node of the box is shared by 8 elements
    assert m.max() == 8
    assert np.all(m[:, 1:-1, 1:-1, 1:-1] == 1)
    assert abs(np.sum(1.0 / P.mult) - P.U) < 1e-9


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("deform", [False, True])
def test_ax_kills_constants_and_is_symmetric(deform):
    P = so.Problem(3, 2, 2, 5, deform=deform)
    one = np.ones(P.L)
    assert np.abs(P.ax_unmasked(one)).max() < 1e-12
    g = np.random.default_rng(1)
    u = P.dssum(g.standard_normal(P.L)) / P.mult * P.mask
    v = P.dssum(g.standard_normal(P.L)) / P.mult * P.mask
    a = P.glsc3(u, P.ax(v))
    b = P.glsc3(v, P.ax(u))
    assert abs(a - b) <= 1e-13 * abs(a)


def test_energy_identity_polynomial():
    # u = x^2 y + z on the unit cube: int |grad u|^2 = 4/9 + 1/5 + 1 exactly,
    # and the GLL rule (exact to degree 2N-1) integrates the x^4 term exactly for N >= 3.
    for N in (3, 4, 7):
        P = so.Problem(3, 2, 2, N)
        x, y, z = (P.X[m].reshape(-1) for m in range(3))
        u = x ** 2 * y + z
        energy = np.sum(u * P.ax_local(u))
        assert abs(energy - (4 / 9 + 1 / 5 + 1)) < 1e-12


@pytest.mark.parametrize("N,deform", [(2, False), (3, False), (2, True), (3, True), (4, True)])
def test_ax_matches_dense_bruteforce(N, deform):
    k = 2
    A, gl = dense_box_matrix(k, k, k, N, deform_amp=0.05 if deform else 0.0)
    P = so.Problem(k, k, k, N, deform=deform)
    # the independent numbering must partition local nodes like the oracle's
    pairs = set(zip(gl.tolist(), P.gid.tolist()))
    assert len(pairs) == P.U
    g = np.random.default_rng(7)
    ug = g.standard_normal(A.shape[0])
    ref = (A @ ug)[gl]
    got = P.ax_unmasked(ug[gl])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # Jacobi diagonal: assembled diag formula equals the dense diagonal
    dg = P.dssum(P.diag_local())
    np.testing.assert_allclose(dg, np.diag(A)[gl], rtol=1e-12)


def test_ax_undeformed_matches_kronecker_form():
    # A^e = (h/2) (K x M x M + M x K x M + M x M x K), K = D^T W D, M = W (1-D)
    N, k = 4, 2
    x, w = gll_numpy(N)
    _, dL = lagrange_tables(x)
    Dn = dL.T
    K1 = Dn.T @ np.diag(w) @ Dn
    M1 = np.diag(w)
    h = 1.0 / k
    Ae = (h / 2) * (np.kron(np.kron(M1, M1), K1) + np.kron(np.kron(M1, K1), M1)
                    + np.kron(np.kron(K1, M1), M1))
    P = so.Problem(k, k, k, N)
    n3 = (N + 1) ** 3
    u = np.random.default_rng(3).standard_normal(P.L)
    ref = np.concatenate([Ae @ u[e * n3:(e + 1) * n3] for e in range(P.E)])
    np.testing.assert_allclose(P.ax_local(u), ref, atol=1e-12 * np.abs(ref).max())


def test_masked_operator_is_positive_definite():
    k, N = 2, 3
    A, gl = dense_box_matrix(k, k, k, N, deform_amp=0.05)
    on = boundary_unique(k, k, k, N, gl)
    Ai = A[np.ix_(~on, ~on)]
    ev = np.linalg.eigvalsh(Ai)
    assert ev.min() > 1e-3
    np.testing.assert_allclose(Ai, Ai.T, atol=1e-13)


# ---------------------------------------------------------------- PCG
@pytest.mark.parametrize("deform", [False, True])
def test_pcg_matches_dense_solve(deform):
    k, N = 2, 3
    A, gl = dense_box_matrix(k, k, k, N, deform_amp=0.05 if deform else 0.0)
    on = boundary_unique(k, k, k, N, gl)
    P = so.Problem(k, k, k, N, deform=deform)
    b = P.rhs_uniform(seed=5)
    # b at unique nodes (copies are equal)
    bg = np.zeros(A.shape[0])
    bg[gl] = b
    xi = np.linalg.solve(A[np.ix_(~on, ~on)], bg[~on])
    xg = np.zeros(A.shape[0])
    xg[~on] = xi
    x, it, hist = P.pcg(b, tol=1e-14, maxit=500)
    assert hist[-1] <= 1e-14
    np.testing.assert_allclose(x, xg[gl], atol=1e-12 * np.abs(xg).max())


def test_pcg_error_decreases_in_energy_norm():
    k, N = 2, 4
    P = so.Problem(k, k, k, N, deform=True)
    b = P.rhs_uniform(seed=2)
    xs, _, _ = P.pcg(b, tol=1e-14, maxit=1000)
    prev = None
    for m in range(1, 25):
        x, _, _ = P.pcg(b, fixed_iters=m)
        e = xs - x
        en = P.glsc3(e, P.ax(e))
        if prev is not None:
            assert en <= prev * (1 + 1e-10)
        prev = en


def test_manufactured_solution_converges_spectrally():
    errs = {}
    for N in (3, 5, 7, 9):
        P = so.Problem(4, 4, 4, N)
        b = P.rhs_sine()
        x, it, hist = P.pcg(b, tol=1e-13, maxit=2000)
        errs[N] = np.abs(x - P.exact_sine() * P.mask).max()
    for a, bN in ((3, 5), (5, 7), (7, 9)):
        assert errs[bN] < errs[a] / 10.0, errs
    assert errs[9] < 1e-8


def test_jacobi_reduces_iterations_on_deformed_mesh():
    P = so.Problem(4, 4, 4, 5, deform=True)
    b = P.rhs_uniform(seed=0)
    _, it_j, _ = P.pcg(b, tol=1e-8, maxit=2000, precond=True)
    _, it_i, _ = P.pcg(b, tol=1e-8, maxit=2000, precond=False)
    assert it_j < it_i


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for c, hexv in rows:
        assert int(so.splitmix64(0, int(c))) == int(hexv, 16)


def test_uniform_rhs_is_per_global_node_and_in_range():
    P = so.Problem(3, 3, 3, 4, deform=True)
    b = P.rhs_uniform(seed=0)
    u = so.splitmix_uniform(0, np.arange(P.U))
    assert u.min() >= -1 and u.max() < 1
    assert abs(u.mean()) < 0.05
    # every copy of a global node carries the same value
    np.testing.assert_allclose(P.dssum(b) / P.mult, b, rtol=1e-15, atol=1e-16)


def test_box_coords_elements_match_whole_mesh():
    X = so.box_coords(3, 2, 4, 5)
    elems = [0, 5, 7, 23, 11]
    np.testing.assert_array_equal(so.box_coords_elements(3, 2, 4, 5, elems), X[:, elems])
