"""Pins of the learned-initial-guess oracle: finite differences for the
network's gradients, a closed-form single-mode right-hand side, the
definitions of the features, and the first Adam step."""
import numpy as np
import pytest

from oracle import learned_x0 as lx
from oracle import sem_oracle as so


def test_mlp_gradients_match_central_differences():
    g = np.random.default_rng(0)
    net = lx.MLP([7, 6, 5, 4], seed=1)
    X = g.standard_normal((9, 7))
    T = g.standard_normal((9, 4))
    grads = net.gradients(X, T)
    h = 1e-6
    for q, p in enumerate(net.params):
        flat = p.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = net.loss(X, T)
            flat[idx] = old - h
            lm = net.loss(X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[q].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (q, idx, fd, an)


def test_adam_first_step_is_a_signed_lr_step():
    net = lx.MLP([3, 2], seed=0)
    before = [p.copy() for p in net.params]
    grads = [np.full_like(p, 0.5) for p in net.params]
    grads[0][0, 0] = -2.0
    net.adam_step(grads, {}, lr=1e-3)
    for p0, p1, gr in zip(before, net.params, grads):
        np.testing.assert_allclose(p1 - p0, -1e-3 * np.sign(gr), rtol=1e-6)


def test_single_mode_fourier_rhs_is_the_sine_rhs():
    P = so.Problem(3, 3, 2, 5, deform=True)
    a = np.zeros((8, 8, 8))
    a[0, 0, 0] = 1.0
    b = lx.fourier_rhs_from(P, a)
    np.testing.assert_allclose(b, P.rhs_sine() / (3 * np.pi ** 2), rtol=1e-12, atol=1e-16)


def test_fourier_coefficients_decay_and_determinism():
    a = lx.fourier_coefficients(3, 5)
    b = lx.fourier_coefficients(3, 5)
    np.testing.assert_array_equal(a, b)
    k = np.arange(1, 9)
    k2 = k[None, None, :] ** 2 + k[None, :, None] ** 2 + k[:, None, None] ** 2
    assert np.all(np.abs(a) * k2 <= 1.0)
    assert not np.array_equal(a, lx.fourier_coefficients(3, 6))


def test_features_definitions():
    P = so.Problem(3, 2, 2, 3, deform=True)
    b = lx.fourier_rhs(P, 0, 0)
    X, s = lx.features(P, b)
    n3 = P.n ** 3
    assert X.shape == (P.E, n3 + 18)
    X2, s2 = lx.features(P, 2.0 * b)
    np.testing.assert_allclose(X2, X, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(s2, 2 * s, rtol=1e-12)
    # neighbours by brute force over element centres
    nb = lx.element_neighbours(P.kx, P.ky, P.kz)
    for e in range(P.E):
        ex, ey, ez = e % 3, (e // 3) % 2, e // 6
        for f, (dx, dy, dz) in enumerate([(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                                          (0, 0, -1), (0, 0, 1)]):
            x, y, z = ex + dx, ey + dy, ez + dz
            inside = 0 <= x < 3 and 0 <= y < 2 and 0 <= z < 2
            assert nb[e, f] == (x + 3 * (y + 2 * z) if inside else -1)
            if not inside:
                assert X[e, n3 + 12 + f] == 0.0
    bl = b.reshape(P.E, n3)
    np.testing.assert_allclose(X[:, :n3] * s[:, None], bl, rtol=1e-13)
    G = P.G.reshape(6, P.E, n3)
    np.testing.assert_allclose(X[:, n3:n3 + 6], G.mean(axis=2).T, rtol=1e-13)


def test_continuity_projection():
    P = so.Problem(3, 2, 2, 3, deform=True)
    g = np.random.default_rng(2)
    u = g.standard_normal(P.L)
    x0 = lx.continuity_projection(P, u)
    np.testing.assert_allclose(P.dssum(x0) / P.mult, x0, rtol=1e-13, atol=1e-15)
    assert np.all(x0[P.mask == 0] == 0)
    cont = P.mask * P.dssum(u) / P.mult
    np.testing.assert_allclose(lx.continuity_projection(P, cont), cont, rtol=1e-13, atol=1e-15)


def test_coarse_features_converge_to_the_solution():
    """Multigrid-Richardson converges to A^{-1} b, so with many steps the
    coarse features equal the exact solution's values at the element
    vertices and its element means (pins the iteration's sign and the vertex
    order v = (i>0) + 2 (j>0) + 4 (k>0))."""
    from oracle import pmg
    M = pmg.PMG(2, 2, 2, 3, deform=True)
    P = M.levels[0].P
    b = lx.fourier_rhs(P, 4, 2)
    _, s = lx.features(P, b)
    x, _, _ = P.pcg(b, tol=1e-14, maxit=2000)
    C = lx.coarse_features(P, M.vcycle, b, 60, s)
    n = P.n
    xl = x.reshape(P.E, n ** 3)
    want = np.stack([xl[:, (n - 1 if v & 1 else 0) + n * ((n - 1 if v & 2 else 0) +
                                                       n * (n - 1 if v & 4 else 0))]
                     for v in range(8)] + [xl.mean(axis=1)], axis=1) / s[:, None]
    assert np.abs(C - want).max() <= 1e-8 * np.abs(want).max()
    # one step is far from it: the pin is the convergence, not the start
    C1 = lx.coarse_features(P, M.vcycle, b, 1, s)
    assert np.abs(C1 - want).max() > 1e-3 * np.abs(want).max()
