"""Parity at the benchmark's full size: the deformed 32^3 hex mesh at N = 7
(16,777,216 local DOFs), set up and launched as the benchmark does, checked
on sampled outputs the oracle computes element by element (the oracle
builds the coordinates and geometric factors of the sampled elements only):
the element operator in FP64 and FP32, the right-hand side bit for bit, and
the residual of the mixed solve at element-interior nodes, where the
assembled operator is the element operator alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import sem_oracle as so  # noqa: E402
from tests.gpu_util import rel_maxerr  # noqa: E402

K, N = 32, 7
n = N + 1
n3 = n ** 3


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as sem
    S = sem.Solver(K, K, K, N, deform=True)
    g = np.random.default_rng(123)
    E = K ** 3
    # corners, edges, faces of the box and random interior elements
    picks = {0, K - 1, K * K - 1, E - 1, E - K, K * (K - 1), E // 2 + K // 2}
    picks |= set(int(e) for e in g.integers(0, E, 40))
    elems = np.array(sorted(picks))
    X = so.deform_cyclic(so.box_coords_elements(K, K, K, N, elems))
    G, B, _ = so.geometry(X, N)
    xi, _ = so.gll(N)
    D = so.deriv_matrix(N, xi)
    # Dirichlet mask of the sampled elements from their grid positions
    ex, ey, ez = elems % K, (elems // K) % K, elems // (K * K)
    r = np.arange(n)
    I = ex[:, None, None, None] * N + r[None, None, None, :]
    J = ey[:, None, None, None] * N + r[None, None, :, None]
    Kz = ez[:, None, None, None] * N + r[None, :, None, None]
    on = (I == 0) | (I == K * N) | (J == 0) | (J == K * N) | (Kz == 0) | (Kz == K * N)
    mask = np.where(on, 0.0, 1.0)
    gx = K * N + 1
    gid = I + gx * (J + gx * Kz)
    yield sem, S, elems, G, D, mask, gid
    S.close()


def _rows(elems):
    return (elems[:, None] * n3 + np.arange(n3)[None, :]).reshape(-1)


def test_operator_full_size_sampled(setup):
    sem, S, elems, G, D, mask, _ = setup
    rows = _rows(elems)
    gen = torch.Generator(device="cuda").manual_seed(5)
    u = torch.rand(S.L, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
    w = torch.empty_like(u)
    sem.sem_ax_local(S.h, u, w, sem.SEM_FP64)
    us = u.cpu().numpy()[rows]
    ref = mask.reshape(-1) * so.ax_local(us, G, D)
    assert rel_maxerr(w.cpu().numpy()[rows], ref) < 1e-12
    u32 = u.float()
    w32 = torch.empty_like(u32)
    sem.sem_ax_local(S.h, u32, w32, sem.SEM_MIXED_FP32)     # the staged kernel the solver uses
    ref32 = mask.reshape(-1) * so.ax_local(u32.double().cpu().numpy()[rows], G, D)
    assert rel_maxerr(w32.double().cpu().numpy()[rows], ref32) < 1e-6


def test_rhs_full_size_bitwise(setup):
    sem, S, elems, _, _, mask, gid = setup
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    ref = mask.reshape(-1) * so.splitmix_uniform(0, gid.reshape(-1))
    np.testing.assert_array_equal(b.cpu().numpy()[_rows(elems)], ref)


def test_mixed_solve_full_size_residual(setup):
    """The benchmark solve (mixed, 1e-8): its FP64 true residual, and the
    residual b - A_e x_e at element-interior nodes of the sampled elements
    computed by the oracle agrees with the device's b - A x there."""
    sem, S, elems, G, D, mask, _ = setup
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    x, info = S.solve(b, tol=1e-8, maxit=5000, precision=sem.SEM_MIXED_FP32)
    assert info["rc"] == 0 and info["relres_true"] <= 1e-8
    ax = torch.empty_like(b)
    sem.sem_ax(S.h, x, ax, sem.SEM_FP64)
    rows = _rows(elems)
    inner = np.zeros((n, n, n), dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    sel = np.tile(inner.reshape(-1), len(elems))
    r_dev = (b - ax).cpu().numpy()[rows][sel]
    r_ora = (b.cpu().numpy()[rows] - mask.reshape(-1) * so.ax_local(x.cpu().numpy()[rows], G, D))[sel]
    bmax = float(b.abs().max())
    assert np.abs(r_dev - r_ora).max() <= 1e-11 * bmax
    # an element-interior node is a unique node, so |r| there is bounded by
    # ||r||_c <= tol ||b||_c
    bnorm = sem.sem_glsc3(S.h, b, b, sem.SEM_FP64) ** 0.5
    assert np.abs(r_ora).max() <= 1e-8 * bnorm * 1.0001


@pytest.mark.parametrize("Nsw", [5, 9, 11, 13, 15])
def test_order_sweep_full_size_sampled(Nsw):
    """The order sweep's meshes (about 2^24 local DOFs per order, deformed),
    as the benchmark sets them up: the FP32 operator and its two
    tensor-core variants against the oracle on sampled elements (TF32 keeps
    10 mantissa bits, the BF16 split about 16; bounds as in the small-case
    tests)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as sem
    import sem_inputs
    c = sem_inputs.order_sweep_case(Nsw)
    S = sem.Solver(c.kx, c.ky, c.kz, Nsw, deform=True)
    nn = Nsw + 1
    E = c.kx * c.ky * c.kz
    g = np.random.default_rng(Nsw)
    elems = np.array(sorted({0, E - 1, c.kx - 1, E // 2} | set(int(e) for e in g.integers(0, E, 12))))
    X = so.deform_cyclic(so.box_coords_elements(c.kx, c.ky, c.kz, Nsw, elems))
    G, _, _ = so.geometry(X, Nsw)
    xi, _ = so.gll(Nsw)
    D = so.deriv_matrix(Nsw, xi)
    ex, ey, ez = elems % c.kx, (elems // c.kx) % c.ky, elems // (c.kx * c.ky)
    r = np.arange(nn)
    I = ex[:, None, None, None] * Nsw + r[None, None, None, :]
    J = ey[:, None, None, None] * Nsw + r[None, None, :, None]
    Kz = ez[:, None, None, None] * Nsw + r[None, :, None, None]
    on = ((I == 0) | (I == c.kx * Nsw) | (J == 0) | (J == c.ky * Nsw) | (Kz == 0)
          | (Kz == c.kz * Nsw))
    mask = np.where(on, 0.0, 1.0).reshape(-1)
    rows = (elems[:, None] * nn ** 3 + np.arange(nn ** 3)[None, :]).reshape(-1)
    gen = torch.Generator(device="cuda").manual_seed(Nsw)
    u = (torch.rand(S.L, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1).float()
    ref = mask * so.ax_local(u.double().cpu().numpy()[rows], G, D)
    w = torch.empty_like(u)
    for prec, tol in ((sem.SEM_MIXED_FP32, 1e-6), (sem.SEM_MIXED_TF32, 2.0 ** -11 * 8 * nn),
                      (sem.SEM_MIXED_BF16X3, 2.0 ** -16 * 8 * nn)):
        sem.sem_ax_local(S.h, u, w, prec)
        err = rel_maxerr(w.double().cpu().numpy()[rows], ref)
        assert err < tol, (Nsw, prec, err, tol)
    S.close()
