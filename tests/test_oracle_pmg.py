"""Pins of the multigrid-preconditioner oracle (oracle/pmg.py) against what
the mathematics fixes: interpolation exactness, restriction as the adjoint
of prolongation, the fast-diagonalisation local solve against a dense solve
of the independently assembled stiffness matrix (tests/dense_sem.py) on the
extended block, the Schwarz block counts in closed form, symmetry and
positivity of the smoother and of the V-cycle, the damping against the dense
spectrum, and the preconditioned CG solution against numpy.linalg.solve."""
import itertools

import numpy as np
import pytest

from oracle import pmg
from oracle import sem_oracle as so
from tests.dense_sem import boundary_unique, dense_box_matrix


def test_level_orders():
    assert pmg.level_orders(7) == [7, 3, 1]
    assert pmg.level_orders(9) == [9, 4, 2, 1]
    assert pmg.level_orders(1) == [1]


@pytest.mark.parametrize("Nc,Nf", [(1, 3), (3, 7), (2, 5), (4, 9), (5, 5)])
def test_interpolation_exact_on_coarse_polynomials(Nc, Nf):
    J = pmg.interp_matrix(Nc, Nf)
    xc, _ = so.gll(Nc)
    xf, _ = so.gll(Nf)
    for m in range(Nc + 1):
        np.testing.assert_allclose(J @ xc ** m, xf ** m, atol=1e-13)
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-14)
    if Nc == Nf:
        np.testing.assert_allclose(J, np.eye(Nc + 1), atol=1e-14)


def test_restriction_is_adjoint_of_prolongation():
    M = pmg.PMG(3, 2, 2, 5, deform=True, power_iters=2)
    f, c = M.levels[0].P, M.levels[1].P
    g = np.random.default_rng(0)
    r = f.mask * f.dssum(g.standard_normal(f.L)) / f.mult      # continuous, masked
    v = c.mask * c.dssum(g.standard_normal(c.L)) / c.mult
    pv = M.prolong(0, v)
    np.testing.assert_allclose(f.dssum(pv) / f.mult, pv, atol=1e-13)   # continuous
    assert np.all(pv[f.mask == 0] == 0) or np.abs(pv[f.mask == 0]).max() < 1e-13
    lhs = c.glsc3(M.restrict(0, r), v)
    rhs = f.glsc3(r, pv)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_prolongation_reproduces_coarse_polynomials():
    """A global polynomial of degree <= N_c per direction interpolated at the
    coarse nodes and prolongated equals its fine-node interpolant."""
    M = pmg.PMG(2, 2, 3, 6, deform=False, power_iters=2)
    f, c = M.levels[0].P, M.levels[1].P
    poly = lambda X: X[0] ** 2 * X[1] + X[2] ** 3 - X[0] * X[2]
    uc = poly(c.X).reshape(-1)
    np.testing.assert_allclose(M.prolong(0, uc), poly(f.X).reshape(-1), atol=1e-13)


def test_fdm_local_solve_equals_dense_block_solve():
    """Undeformed uniform mesh: the separable extended-block operator is the
    assembled stiffness restricted to the block, so the fast-diagonalisation
    solve equals a dense solve on the block (interior element, no boundary)."""
    kx = ky = kz = 3
    for N in (2, 3, 4):
        lev = pmg.Level(kx, ky, kz, N, deform=False)
        A, gid_local = dense_box_matrix(kx, ky, kz, N)
        # dense index of every grid point (I, J, K)
        I, J, K = so.box_global_index(kx, ky, kz, N)
        key = {}
        for l, (a, b_, c_) in enumerate(zip(I.reshape(-1), J.reshape(-1), K.reshape(-1))):
            key[(a, b_, c_)] = gid_local[l]
        e = 1 + kx * (1 + ky * 1)                     # the centre element
        n = N + 1
        blk = [(N - 1 + a) for a in range(n + 2)]     # grid indices of its block
        ids = [key[(i, j, k)] for k, j, i in itertools.product(blk, blk, blk)]
        rhs = np.random.default_rng(N).standard_normal(len(ids))
        ref = np.linalg.solve(A[np.ix_(ids, ids)], rhs)
        z = lev.local_solve(np.broadcast_to(rhs.reshape(n + 2, n + 2, n + 2),
                                            (lev.P.E, n + 2, n + 2, n + 2)).copy())[e]
        np.testing.assert_allclose(z.reshape(-1), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_schwarz_counts_closed_form():
    """Blocks holding a grid point: per direction 2 at element faces and at
    the first node inside a neighbour, else 1 (N >= 2, away from the
    boundary), and the 3-D count is the product."""
    kx, ky, kz, N = 4, 3, 3, 4
    lev = pmg.Level(kx, ky, kz, N, deform=False)

    def c1(g, k):
        if g <= 0 or g >= k * N:
            return None                               # boundary: Dirichlet
        r = g % N
        return 2 if r in (0, 1, N - 1) else 1
    for K in range(1, kz * N):
        for J in range(1, ky * N):
            for I in range(1, kx * N):
                cx, cy, cz = c1(I, kx), c1(J, ky), c1(K, kz)
                # the first node next to the domain boundary belongs to one block
                cx = 1 if I in (1, kx * N - 1) else cx
                cy = 1 if J in (1, ky * N - 1) else cy
                cz = 1 if K in (1, kz * N - 1) else cz
                assert lev.count[K, J, I] == cx * cy * cz, (I, J, K)


def _sym_pos(op, P, seed):
    g = np.random.default_rng(seed)
    x = P.mask * P.dssum(g.standard_normal(P.L)) / P.mult
    y = P.mask * P.dssum(g.standard_normal(P.L)) / P.mult
    a, b = P.glsc3(op(x), y), P.glsc3(x, op(y))
    assert abs(a - b) <= 1e-12 * max(abs(a), 1e-30) + 1e-14
    assert P.glsc3(op(x), x) > 0


def test_schwarz_and_vcycle_symmetric_positive():
    M = pmg.PMG(3, 3, 2, 5, deform=True, power_iters=10)
    P = M.levels[0].P
    for lev in M.levels:
        _sym_pos(lev.schwarz, lev.P, 1)
    _sym_pos(M.vcycle, P, 2)


def test_damping_against_dense_spectrum():
    """omega = 1 / (power-iteration estimate of lambda_max(S A)): within a few
    per cent of the dense largest eigenvalue, never above it."""
    lev = pmg.Level(2, 2, 2, 3, deform=True)
    P = lev.P
    inner = np.nonzero(P.mask)[0]
    # dense S A on continuous masked vectors, in unique-node coordinates
    uniq = {}
    for l in inner:
        uniq.setdefault(P.gid[l], l)
    cols = []
    for g_, l in uniq.items():
        e = np.zeros(P.L)
        e[P.gid == g_] = 1.0
        cols.append(lev.schwarz(P.ax(e))[[uniq[h] for h in uniq]])
    lam = np.max(np.real(np.linalg.eigvals(np.array(cols).T)))
    est = pmg.PMG.lambda_max(lev, 30, 12345)
    assert 0.95 * lam <= est <= lam * (1 + 1e-10)


def test_level_without_interior_nodes():
    """ky = 1 leaves the N = 1 level without interior nodes: its smoother is
    the zero map, omega is 1, and the cycle still converges."""
    M = pmg.PMG(2, 1, 3, 2, deform=False)
    assert M.levels[-1].P.mask.sum() == 0 and M.levels[-1].omega == 1.0
    P = M.levels[0].P
    b = P.rhs_uniform(1)
    x, it, _ = M.pcg(b, tol=1e-10, maxit=100)
    assert P.true_relres(b, x) <= 1e-9


def test_mg_pcg_solution_equals_dense_solve():
    kx = ky = kz = 2
    N = 3
    M = pmg.PMG(kx, ky, kz, N, deform=True)
    P = M.levels[0].P
    b = P.rhs_uniform(3)
    x, it, _ = M.pcg(b, tol=1e-13, maxit=200)
    A, gid_local = dense_box_matrix(kx, ky, kz, N, deform_amp=0.05)
    on = boundary_unique(kx, ky, kz, N, gid_local)
    inner = np.nonzero(~on)[0]
    bu = np.zeros(A.shape[0])
    bu[gid_local] = b
    xu = np.zeros(A.shape[0])
    xu[inner] = np.linalg.solve(A[np.ix_(inner, inner)], bu[inner])
    np.testing.assert_allclose(x, xu[gid_local], rtol=1e-9, atol=1e-11 * np.abs(xu).max())


def test_mg_needs_far_fewer_iterations_than_jacobi():
    M = pmg.PMG(4, 3, 3, 7, deform=True)
    P = M.levels[0].P
    b = P.rhs_uniform(0)
    x, it, _ = M.pcg(b, tol=1e-10, maxit=300)
    _, itj, _ = P.pcg(b, tol=1e-10, maxit=5000)
    assert P.true_relres(b, x) <= 1e-9
    assert it * 5 <= itj, (it, itj)


def test_h_level_sizes():
    assert pmg.h_levels(32, 32, 32) == [(16, 16, 16), (8, 8, 8), (4, 4, 4), (2, 2, 2)]
    assert pmg.h_levels(8, 4, 4) == [(4, 2, 2)]
    assert pmg.h_levels(4, 3, 3) == [] and pmg.h_levels(2, 2, 2) == []
    M = pmg.PMG(4, 4, 4, 3, deform=False, power_iters=2)
    assert [(lv.P.kx, lv.N) for lv in M.levels] == [(4, 3), (4, 1), (2, 1)] and M.n_p == 2
    assert len(pmg.PMG(4, 4, 4, 3, power_iters=2, hcoarsen=False).levels) == 2


def test_h_prolongation_reproduces_trilinear_functions():
    """Undeformed mesh: a global trilinear function sampled at the coarse
    N = 1 nodes and prolongated equals its values at the fine nodes."""
    M = pmg.PMG(4, 4, 4, 1, deform=False, power_iters=2)
    f, c = M.levels[0].P, M.levels[1].P
    poly = lambda X: (1 + X[0] + 2 * X[1] - X[2] + X[0] * X[1] - X[1] * X[2]
                      + 3 * X[0] * X[2] + X[0] * X[1] * X[2])
    np.testing.assert_allclose(M.prolong(0, poly(c.X).reshape(-1)), poly(f.X).reshape(-1),
                               atol=1e-14)


def test_h_restriction_is_adjoint_of_prolongation():
    M = pmg.PMG(8, 4, 4, 2, deform=True, power_iters=2)
    l = M.n_p - 1                                     # the N = 1 level and its h-level
    f, c = M.levels[l].P, M.levels[l + 1].P
    assert (c.kx, c.ky, c.kz, c.N) == (4, 2, 2, 1)
    g = np.random.default_rng(3)
    r = f.mask * f.dssum(g.standard_normal(f.L)) / f.mult
    v = c.mask * c.dssum(g.standard_normal(c.L)) / c.mult
    pv = M.prolong(l, v)
    np.testing.assert_allclose(f.dssum(pv) / f.mult, pv, atol=1e-13)   # continuous
    assert np.abs(pv[f.mask == 0]).max() == 0.0                        # masked
    lhs, rhs = c.glsc3(M.restrict(l, r), v), f.glsc3(r, pv)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_h_levels_vcycle_symmetric_positive():
    M = pmg.PMG(4, 4, 4, 3, deform=True, power_iters=10)
    assert len(M.levels) == 3
    for lev in M.levels:
        _sym_pos(lev.schwarz, lev.P, 4)
    _sym_pos(M.vcycle, M.levels[0].P, 5)


def test_h_levels_solution_equals_dense_solve():
    kx = ky = kz = 4
    N = 1
    M = pmg.PMG(kx, ky, kz, N, deform=True)
    assert len(M.levels) == 2
    P = M.levels[0].P
    b = P.rhs_uniform(2)
    x, it, _ = M.pcg(b, tol=1e-13, maxit=200)
    A, gid_local = dense_box_matrix(kx, ky, kz, N, deform_amp=0.05)
    on = boundary_unique(kx, ky, kz, N, gid_local)
    inner = np.nonzero(~on)[0]
    bu = np.zeros(A.shape[0])
    bu[gid_local] = b
    xu = np.zeros(A.shape[0])
    xu[inner] = np.linalg.solve(A[np.ix_(inner, inner)], bu[inner])
    np.testing.assert_allclose(x, xu[gid_local], rtol=1e-9, atol=1e-11 * np.abs(xu).max())


def test_h_levels_make_iterations_mesh_independent():
    """With the h-levels the iteration count barely grows from 4^3 to 8^3
    elements; with the p-levels alone it grows by half."""
    its = {}
    for k in (4, 8):
        for h in (True, False):
            M = pmg.PMG(k, k, k, 3, deform=True, hcoarsen=h)
            P = M.levels[0].P
            b = P.rhs_uniform(0)
            x, its[k, h], _ = M.pcg(b, tol=1e-8, maxit=300)
            assert P.true_relres(b, x) <= 1e-8
    assert its[8, True] <= its[4, True] + 2
    assert its[8, False] >= its[4, False] + 4
    assert its[8, True] < its[8, False]
