"""GPU parity: every step of the CUDA path against the FP64 CPU oracle.

Sizes span several thread blocks and ragged tails (element counts that are
not multiples of the elements-per-block of any order) while keeping the
oracle within seconds.  Tolerances: FP64 results to 1e-12 relative (max
norm), integer/index results bit-exact, the counter-based RHS bit-exact,
FP32 operator results to a bound derived from FP32 rounding (Sec. "readings"
of the design notes: ~ n * 2^-24 * condition of the contraction).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import sem_oracle as so  # noqa: E402
import sem_inputs  # noqa: E402
from tests.gpu_util import rel_maxerr  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as m
    return m


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda").contiguous()


CASES = [
    (3, 2, 2, 1, False),
    (3, 2, 5, 3, True),
    (3, 2, 3, 4, True),
    (5, 3, 2, 5, True),
    (2, 3, 3, 6, True),
    (4, 4, 4, 7, False),
    (5, 3, 3, 7, True),
    (3, 3, 2, 9, True),
    (2, 3, 2, 11, True),
    (2, 2, 2, 13, True),
    (2, 1, 2, 15, True),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_N{c[3]}_{'def' if c[4] else 'box'}")
def pair(request, sem):
    kx, ky, kz, N, deform = request.param
    P = so.Problem(kx, ky, kz, N, deform=deform)
    S = sem.Solver(kx, ky, kz, N, deform=deform)
    yield P, S
    S.close()


def test_sizes(pair):
    P, S = pair
    assert (S.E, S.L, S.U) == (P.E, P.L, P.U)
    assert S.sizes.n_shared == int(np.sum(P.mult > 1))
    assert S.sizes.n_segments == int(np.sum(np.bincount(P.gid) > 1))


def test_gll_and_derivative_matrix(pair, sem):
    P, S = pair
    assert rel_maxerr(S.field(sem.FIELD_XI).cpu(), P.xi) < 1e-14
    assert rel_maxerr(S.field(sem.FIELD_W).cpu(), P.w) < 1e-13
    D = S.field(sem.FIELD_D).cpu().numpy().reshape(P.n, P.n)
    assert rel_maxerr(D, P.D) < 1e-12


def test_geometry(pair, sem):
    P, S = pair
    n3 = P.n ** 3
    G = S.field(sem.FIELD_G).cpu().numpy().reshape(P.E, 6, n3)
    Gref = P.G.reshape(6, P.E, n3).transpose(1, 0, 2)
    assert rel_maxerr(G, Gref) < 1e-12
    assert rel_maxerr(S.field(sem.FIELD_B).cpu(), P.B.reshape(-1)) < 1e-12
    # det J is a cubic in the Jacobian entries dx/dr = sum_l D_il x_l, whose
    # rounding error grows with the row sums of |D| (~ N^2): two independent
    # FP64 evaluations differ by up to ~ eps N^3 relative.
    tol_det = max(1e-12, 2e-15 * P.N ** 3)
    assert rel_maxerr(S.field(sem.FIELD_DETJ).cpu(), P.detJ.reshape(-1)) < tol_det
    X = S.field(sem.FIELD_COORDS).cpu().numpy().reshape(3, -1)
    assert rel_maxerr(X, P.X.reshape(3, -1)) < 1e-14


def test_connectivity_bit_exact(pair, sem):
    P, S = pair
    np.testing.assert_array_equal(S.field(sem.FIELD_MULT).cpu().numpy(), P.mult)
    np.testing.assert_array_equal(S.field(sem.FIELD_MASK).cpu().numpy(), P.mask)
    np.testing.assert_array_equal(S.field(sem.FIELD_C).cpu().numpy(), P.c)


def test_jacobi_inverse(pair, sem):
    P, S = pair
    assert rel_maxerr(S.field(sem.FIELD_MINV).cpu(), P.minv) < 1e-12


def test_ax_fp64(pair, sem):
    P, S = pair
    u = sem_inputs.uniform_local(P.L, seed=11)
    w = torch.empty(P.L, dtype=torch.float64, device="cuda")
    sem.sem_ax(S.h, cu(u), w, sem.SEM_FP64)
    assert rel_maxerr(w.cpu(), P.ax(u)) < 1e-12
    sem.sem_ax_local(S.h, cu(u), w, sem.SEM_FP64)
    assert rel_maxerr(w.cpu(), P.mask * P.ax_local(u)) < 1e-12


def test_ax_fp32(pair, sem):
    P, S = pair
    u = sem_inputs.uniform_local(P.L, seed=12, dtype=np.float32)
    w = torch.empty(P.L, dtype=torch.float32, device="cuda")
    sem.sem_ax(S.h, cu(u, torch.float32), w, sem.SEM_MIXED_FP32)
    ref = P.ax(u.astype(np.float64))
    # FP32 rounding of G, D and the n-term contractions: every case of this
    # table (N = 1..15, box and deformed) measured at most 0.46 n 2^-24
    # relative (max norm); the bound 2 n 2^-24 keeps about 4x of headroom
    assert rel_maxerr(w.cpu(), ref) < 2.0 * P.n * 2.0 ** -24


def test_gs(pair, sem):
    P, S = pair
    v = sem_inputs.uniform_local(P.L, seed=13)
    t = cu(v)
    sem.sem_gs(S.h, t, sem.SEM_FP64)
    assert rel_maxerr(t.cpu(), P.dssum(v)) < 1e-15
    # mixed: FP32 storage, FP64 accumulation -> the FP32 rounding of the FP64 sum
    v32 = v.astype(np.float32)
    t32 = cu(v32, torch.float32)
    sem.sem_gs(S.h, t32, sem.SEM_MIXED_FP32)
    ref = P.dssum(v32.astype(np.float64)).astype(np.float32)
    got = t32.cpu().numpy()
    # error-free (TwoSum) accumulation rounded once: equal to the FP64 sum
    # rounded to FP32 up to one unit in the last place in rare tie cases
    ulp = np.spacing(np.abs(ref).astype(np.float32))
    assert np.all(np.abs(got - ref) <= ulp)
    assert np.mean(got != ref) < 1e-3
    # copies of one global node stay bit-identical
    g = P.gid
    first = np.full(P.U, np.nan, dtype=np.float32)
    first[g[::-1]] = got[::-1]
    np.testing.assert_array_equal(got, first[g])


def test_glsc3(pair, sem):
    P, S = pair
    a = sem_inputs.uniform_local(P.L, seed=14)
    b = sem_inputs.uniform_local(P.L, seed=15)
    got = sem.sem_glsc3(S.h, cu(a), cu(b), sem.SEM_FP64)
    ref = P.glsc3(a, b)
    assert abs(got - ref) <= 1e-13 * np.sum(np.abs(a * P.c * b))


def test_rhs(pair, sem):
    P, S = pair
    b = torch.empty(P.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    np.testing.assert_array_equal(b.cpu().numpy(), P.rhs_uniform(0))
    sem.sem_rhs(S.h, sem.RHS_SINE, 0, b)
    assert rel_maxerr(b.cpu(), P.rhs_sine()) < 1e-12


# ------------------------------------------------------------------ solver
def test_pcg_fp64_sine_4x4x4_N7(sem):
    """The plain FP64 Jacobi PCG workload: 64 undeformed elements, N = 7, tol 1e-10."""
    P = so.Problem(4, 4, 4, 7)
    b = P.rhs_sine()
    xo, ito, _ = P.pcg(b, tol=1e-10, maxit=500)
    S = sem.Solver(4, 4, 4, 7)
    x, info = S.solve(cu(b), tol=1e-10, maxit=500, precision=sem.SEM_FP64, history=True)
    assert info["rc"] == 0 and info["relres"] <= 1e-10
    assert abs(info["iters"] - ito) <= 1
    assert rel_maxerr(x.cpu(), xo) < 1e-12
    # both solved tightly the discrete solutions agree to 1e-12
    xo2, _, _ = P.pcg(b, tol=1e-14, maxit=2000)
    x2, info2 = S.solve(cu(b), tol=1e-14, maxit=2000, precision=sem.SEM_FP64)
    assert rel_maxerr(x2.cpu(), xo2) < 1e-12
    # the manufactured solution is reproduced to discretisation accuracy
    assert np.abs(x.cpu().numpy() - P.exact_sine() * P.mask).max() < 1e-5
    S.close()


@pytest.mark.parametrize("deform", [False, True])
def test_pcg_fp64_matches_oracle_history(sem, deform):
    P = so.Problem(5, 4, 3, 5, deform=deform)
    b = P.rhs_uniform(seed=3)
    xo, ito, ho = P.pcg(b, tol=1e-12, maxit=1000)
    S = sem.Solver(5, 4, 3, 5, deform=deform)
    x, info = S.solve(cu(b), tol=1e-12, maxit=1000, precision=sem.SEM_FP64, history=True)
    h = info["history"]
    k = min(len(h), len(ho), 30)
    np.testing.assert_allclose(h[:k], ho[:k], rtol=1e-9)
    assert rel_maxerr(x.cpu(), xo) < 1e-10
    S.close()


def test_pcg_mixed_reaches_fp64_accuracy(sem):
    """Mixed FP32/FP64 with refinement reaches 1e-8 and x within 1e-7 of an
    oracle solution solved to 1e-12 (deformed mesh, N = 7)."""
    P = so.Problem(6, 5, 4, 7, deform=True)
    b = P.rhs_uniform(seed=0)
    xo, _, _ = P.pcg(b, tol=1e-12, maxit=3000)
    S = sem.Solver(6, 5, 4, 7, deform=True)
    x, info = S.solve(cu(b), tol=1e-8, maxit=3000, precision=sem.SEM_MIXED_FP32)
    assert info["rc"] == 0, info
    assert info["relres_true"] <= 1e-8
    assert rel_maxerr(x.cpu(), xo) < 1e-7
    assert P.true_relres(b, x.cpu().numpy()) <= 1.05e-8
    S.close()


def test_all_fp32_stagnates_while_mixed_converges(sem):
    """The paper's qualitative finding (Tables 'Mixed-precision strategy
    evaluation'): FP32 gather-scatter and FP32 dots stagnate above the
    target; FP64 gather-scatter sums and FP64 dots (plus FP64 refinement)
    converge."""
    S = sem.Solver(8, 8, 8, 7, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    _, i32 = S.solve(b, tol=1e-10, maxit=1500, precision=sem.SEM_FP32_ALL)
    _, imx = S.solve(b, tol=1e-10, maxit=1500, precision=sem.SEM_MIXED_FP32)
    assert imx["rc"] == 0 and imx["relres_true"] <= 1e-10
    assert i32["relres_true"] > 1e-8, i32
    S.close()


def test_user_numbering_matches_box(sem):
    """A general mesh given as (relabelled gid, coordinates, Dirichlet faces)
    reproduces the box results: the segment map does not depend on the ids."""
    kx, ky, kz, N = 3, 4, 2, 4
    P = so.Problem(kx, ky, kz, N, deform=True)
    rng = np.random.default_rng(0)
    relabel = rng.permutation(P.U)
    gid = relabel[P.gid].astype(np.int64)
    coords = np.ascontiguousarray(P.X.reshape(3, -1))
    faces = np.zeros(P.E, dtype=np.uint8)
    for ez in range(kz):
        for ey in range(ky):
            for ex in range(kx):
                e = ex + kx * (ey + ky * ez)
                faces[e] = ((ex == 0) | (ex == kx - 1) << 1 | (ey == 0) << 2 | (ey == ky - 1) << 3
                            | (ez == 0) << 4 | (ez == kz - 1) << 5)
    mesh = sem.user_mesh(P.E, gid, coords, faces)
    S = sem.Solver(0, 0, 0, N, mesh=mesh)
    u = sem_inputs.uniform_local(P.L, seed=21)
    w = torch.empty(P.L, dtype=torch.float64, device="cuda")
    sem.sem_ax(S.h, cu(u), w, sem.SEM_FP64)
    assert rel_maxerr(w.cpu(), P.ax(u)) < 1e-12
    S.close()


def test_host_pointers_round_trip(sem):
    P = so.Problem(3, 3, 3, 4, deform=True)
    S = sem.Solver(3, 3, 3, 4, deform=True)
    u = sem_inputs.uniform_local(P.L, seed=5)
    w = np.zeros(P.L)
    sem.sem_ax(S.h, u, w, sem.SEM_FP64)
    assert rel_maxerr(w, P.ax(u)) < 1e-12
    b = P.rhs_uniform(seed=1)
    x = np.zeros(P.L)
    rc, info = sem.sem_pcg_solve(S.h, b, None, x, 1e-10, 500, sem.SEM_FP64)
    xo, _, _ = P.pcg(b, tol=1e-10, maxit=500)
    assert rc == 0 and rel_maxerr(x, xo) < 1e-9
    S.close()


# ------------------------------------------------------------------ edge cases
def test_single_element_all_boundary(sem):
    S = sem.Solver(1, 1, 1, 3)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    P = so.Problem(1, 1, 1, 3)
    np.testing.assert_array_equal(b.cpu().numpy(), P.rhs_uniform(0))
    x, info = S.solve(b, tol=1e-10, maxit=10, precision=sem.SEM_FP64)
    # N = 3 on one element has 8 interior nodes: a real (tiny) system
    xo, _, _ = P.pcg(P.rhs_uniform(0), tol=1e-10, maxit=10)
    assert rel_maxerr(x.cpu(), xo) < 1e-10
    S.close()


def test_zero_rhs_returns_zero(sem):
    S = sem.Solver(2, 2, 2, 2)
    b = torch.zeros(S.L, dtype=torch.float64, device="cuda")
    for prec in (sem.SEM_FP64, sem.SEM_MIXED_FP32):
        x, info = S.solve(b, tol=1e-10, maxit=10, precision=prec)
        assert info["iters"] == 0
        assert torch.all(x == 0)
    S.close()


def test_maxit_reported(sem):
    S = sem.Solver(4, 4, 4, 5, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0, b)
    _, info = S.solve(b, tol=1e-12, maxit=5, precision=sem.SEM_FP64)
    assert info["rc"] == sem.SEM_MAXIT and info["iters"] == 5
    _, info = S.solve(b, fixed_iters=7, precision=sem.SEM_FP64)
    assert info["iters"] == 7 and info["rc"] == 0
    S.close()


def test_invalid_arguments(sem):
    with pytest.raises(sem.SemError):
        sem.Solver(2, 2, 2, 16)
    with pytest.raises(sem.SemError):
        sem.Solver(0, 2, 2, 3)
    S = sem.Solver(2, 2, 2, 3)
    u = torch.zeros(S.L, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.sem_ax(S.h, u, u, sem.SEM_FP64)
    with pytest.raises(sem.SemError):
        sem.sem_ax(S.h, u, torch.zeros_like(u), 9)
    S.close()


def test_graph_and_plain_launch_agree(sem):
    S = sem.Solver(4, 3, 5, 6, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 2, b)
    for prec in (sem.SEM_FP64, sem.SEM_MIXED_FP32):
        x1, i1 = S.solve(b, tol=1e-9, maxit=2000, precision=prec, use_graph=True, chunk=7)
        x2, i2 = S.solve(b, tol=1e-9, maxit=2000, precision=prec, use_graph=False, chunk=5)
        assert i1["iters"] == i2["iters"]
        assert torch.equal(x1, x2)   # deterministic reductions: bitwise equal
    S.close()


@pytest.mark.parametrize("dims,N", [((3, 2, 2), 1), ((2, 3, 1), 2), ((3, 3, 2), 3),
                                    ((1, 2, 3), 5), ((4, 3, 3), 7), ((2, 2, 1), 11)])
def test_fused_gather_scatter_is_bitwise(sem, dims, N):
    """The update with the direct-stiffness summation folded in (box meshes)
    gives the separate pass's bits: same iterations, identical solution, for
    every accumulation mode and the all-FP32 variant (small meshes, where the
    two update kernels run the same grid)."""
    S = sem.Solver(*dims, N, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 5, b)
    assert sem.sem_get_option(S.h, "fuse_gs") == 1
    cases = [(sem.SEM_MIXED_FP32, acc, {}) for acc in (2, 0, 1)]
    fused = 2   # fold the summation for every n (default: n a multiple of 4)
    cases.append((sem.SEM_FP32_ALL, 2, {"fixed_iters": 40}))
    for prec, acc, kw in cases:
        sem.sem_set_option(S.h, "gs_acc", acc)
        out = []
        for fuse in (fused, 0):
            sem.sem_set_option(S.h, "fuse_gs", fuse)
            if kw:
                x, info = S.solve(b, precision=prec, **kw)
            else:
                x, info = S.solve(b, tol=1e-9, maxit=3000, precision=prec)
            out.append((x, info))
        (x1, i1), (x0, i0) = out
        assert i1["iters"] == i0["iters"], (prec, acc)
        assert torch.equal(x1, x0), (prec, acc)
        sem.sem_set_option(S.h, "fuse_gs", 1)
    S.close()


def test_fused_gather_scatter_large_mesh(sem):
    """Where the fused update runs its own (occupancy-sized) grid, the dot
    products are summed in another order: the solves agree to rounding, and
    the folded mixed solve to 1e-9 is within 1e-7 of the oracle's x solved
    to 1e-12 (so the two tolerances are not conflated)."""
    P = so.Problem(12, 10, 9, 7, deform=True)
    S = sem.Solver(12, 10, 9, 7, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 6, b)
    x1, i1 = S.solve(b, tol=1e-9, maxit=5000, precision=sem.SEM_MIXED_FP32)
    sem.sem_set_option(S.h, "fuse_gs", 0)
    x0, i0 = S.solve(b, tol=1e-9, maxit=5000, precision=sem.SEM_MIXED_FP32)
    assert i1["rc"] == 0 and i1["relres_true"] <= 1e-9
    assert abs(i1["iters"] - i0["iters"]) <= max(3, i0["iters"] // 50)
    assert rel_maxerr(x1.cpu(), x0.cpu()) < 1e-7
    assert P.true_relres(b.cpu().numpy(), x1.cpu().numpy()) <= 1.0000001e-9
    xo, _, _ = P.pcg(b.cpu().numpy(), tol=1e-12, maxit=5000)
    assert rel_maxerr(x1.cpu(), xo) < 1e-7
    S.close()


@pytest.mark.parametrize("dims,N", [((3, 2, 2), 7), ((5, 4, 3), 3), ((2, 2, 3), 11),
                                    ((2, 1, 2), 15)])
def test_update_variants(sem, dims, N):
    """Launch shapes of the folded update (register budgets for four, five,
    six blocks per SM; an L2 prefetch of the next group) traverse the
    vectors in the same order -- on these small meshes with the same grid --
    so they give the same bits."""
    S = sem.Solver(*dims, N, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 3, b)
    mixed = sem.SEM_MIXED_FP32
    ref, iref = S.solve(b, tol=1e-9, maxit=3000, precision=mixed)
    assert iref["rc"] == 0 and iref["relres_true"] <= 1e-9
    for v in (1, 2, 3, 4, 5):
        sem.sem_set_option(S.h, "upd_variant", v)
        assert sem.sem_get_option(S.h, "upd_variant") == v
        x, info = S.solve(b, tol=1e-9, maxit=3000, precision=mixed)
        assert info["iters"] == iref["iters"] and torch.equal(x, ref), v
    S.close()


@pytest.mark.parametrize("dims", [(3, 2, 2), (7, 5, 3)])
def test_staged_update_matches_folded(sem, dims):
    """The bulk-copy staged update (N = 7) computes every value as the
    folded update does; only the order of the dot partial sums differs, so
    the solves agree to rounding and converge alike (odd element counts
    leave a partial last group)."""
    S = sem.Solver(*dims, 7, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 9, b)
    for prec, kw in ((sem.SEM_MIXED_FP32, dict(tol=1e-9, maxit=3000)),
                     (sem.SEM_FP32_ALL, dict(fixed_iters=30))):
        sem.sem_set_option(S.h, "upd_tma", 0)
        x0, i0 = S.solve(b, precision=prec, **kw)
        sem.sem_set_option(S.h, "upd_tma", 1)
        x1, i1 = S.solve(b, precision=prec, **kw)
        if "tol" in kw:
            assert i1["rc"] == 0 and i1["relres_true"] <= 1e-9
            assert abs(i1["iters"] - i0["iters"]) <= 2
            assert rel_maxerr(x1.cpu(), x0.cpu()) < 1e-7
        else:
            assert rel_maxerr(x1.cpu(), x0.cpu()) < 1e-4
    sem.sem_set_option(S.h, "upd_tma", 0)
    S.close()


def test_l2_options_change_no_bits(sem):
    """L2 residency controls (access-policy window, per-access eviction
    hints) change where data lives, not the arithmetic."""
    S = sem.Solver(4, 4, 4, 7, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 8, b)
    ref, iref = S.solve(b, tol=1e-9, maxit=3000, precision=sem.SEM_MIXED_FP32)
    for persist, hints in ((0, 0), (0, 1), (1, 1)):
        sem.sem_set_option(S.h, "l2_persist", persist)
        sem.sem_set_option(S.h, "l2_hints", hints)
        x, info = S.solve(b, tol=1e-9, maxit=3000, precision=sem.SEM_MIXED_FP32)
        assert info["iters"] == iref["iters"]
        assert torch.equal(x, ref), (persist, hints)
    S.close()


def test_kernel_timing_mode(sem):
    """Per-kernel event timing changes nothing in the result (same kernels,
    events between them), counts every iteration and reports positive
    per-launch device times; turning it off clears the sums."""
    S = sem.Solver(4, 4, 4, 7, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 4, b)
    for prec in (sem.SEM_FP64, sem.SEM_MIXED_FP32):
        x1, i1 = S.solve(b, tol=1e-9, maxit=2000, precision=prec)
        sem.sem_set_option(S.h, "kernel_timing", 1)
        x2, i2 = S.solve(b, tol=1e-9, maxit=2000, precision=prec)
        assert sem.sem_get_option(S.h, "kt_iters") == i2["iters"]
        for k in ("kt_ms_ax", "kt_ms_gs", "kt_ms_update"):
            assert 0 < sem.sem_get_option(S.h, k) < i2["solve_ms"]
        sem.sem_set_option(S.h, "kernel_timing", 0)
        assert sem.sem_get_option(S.h, "kt_iters") == 0
        assert i1["iters"] == i2["iters"]
        assert torch.equal(x1, x2)
    S.close()


@pytest.mark.parametrize("dims,N", [((4, 3, 3), 5), ((5, 4, 3), 7), ((3, 3, 2), 9), ((3, 2, 3), 11),
                                    ((2, 3, 2), 13), ((3, 2, 2), 15)])
def test_launch_variants_agree(sem, dims, N):
    """Every staged-operator launch variant and the unstaged kernel give the
    same FP32 result (identical arithmetic per element); the set-up
    autotuner's choice is readable.  At N = 11, 13, 15 (one element already
    fills a block) some variants' stages exceed shared memory: their tuner
    entry is -1 and selecting them runs the unstaged kernel.  At N = 15 the
    stages hold G only (96 KB), so one or two stages fit in either mode.
    Variant 4 (G in one buffer, u or p_old in two, PCG mode r and J^-1 in
    a third) exists at the line orders below 15 (N = 5 .. 13).  Each variant also runs with the grid capped at two blocks,
    so that every block walks several element groups through the reuse of
    its stages (barrier phases, early and late refills)."""
    P = so.Problem(*dims, N, deform=True)
    S = sem.Solver(*dims, N, deform=True)
    assert sem.sem_get_option(S.h, "ax_variant") in (0, 1, 2, 3, 4)
    assert sem.sem_get_option(S.h, "ax_variant_pcg") in (0, 1, 2, 3, 4)
    assert sem.sem_get_option(S.h, "ax_tune_ms_plain_0") > 0
    tune = {mode: [sem.sem_get_option(S.h, f"ax_tune_ms_{mode}_{v}") for v in range(5)]
            for mode in ("plain", "pcg")}
    for mode in ("plain", "pcg"):
        assert (tune[mode][4] > 0) == (N in (5, 7, 9, 11, 13))
    if N == 15:
        for mode in ("plain", "pcg"):
            t = tune[mode]
            assert t[1] == t[3] == -1.0 and t[0] > 0 and t[2] > 0
    u = cu(sem_inputs.uniform_local(P.L, seed=31, dtype=np.float32), torch.float32)
    outs = []
    for cap in (0, 2):
        sem.sem_set_option(S.h, "ax_grid_cap", cap)
        assert sem.sem_get_option(S.h, "ax_grid_cap") == cap
        for v in range(5):
            sem.sem_set_option(S.h, "ax_variant", v)
            w = torch.empty_like(u)
            sem.sem_ax_local(S.h, u, w, sem.SEM_MIXED_FP32)
            outs.append(w)
    sem.sem_set_option(S.h, "ax_grid_cap", 0)
    sem.sem_set_option(S.h, "use_tma", 0)
    w = torch.empty_like(u)
    sem.sem_ax_local(S.h, u, w, sem.SEM_MIXED_FP32)
    outs.append(w)
    for o in outs[1:]:
        assert rel_maxerr(o.cpu(), outs[0].cpu()) < 1e-6
    ref = P.mask * P.ax_local(u.cpu().numpy().astype(np.float64))
    assert rel_maxerr(outs[0].cpu(), ref) < 1e-5
    # PCG mode through a solve: every variant converges to the same answer
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 4, b)
    sem.sem_set_option(S.h, "use_tma", 1)
    xs = []
    for cap in (0, 2):
        sem.sem_set_option(S.h, "ax_grid_cap", cap)
        for v in range(5):
            sem.sem_set_option(S.h, "ax_variant_pcg", v)
            x, info = S.solve(b, tol=1e-9, maxit=3000, precision=sem.SEM_MIXED_FP32)
            assert info["rc"] == 0 and info["relres_true"] <= 1e-9
            xs.append(x)
    sem.sem_set_option(S.h, "ax_grid_cap", 0)
    for x in xs[1:]:
        assert rel_maxerr(x.cpu(), xs[0].cpu()) < 1e-7
    S.close()


def test_gs_accumulation_modes(sem):
    P = so.Problem(4, 3, 3, 5, deform=True)
    S = sem.Solver(4, 3, 3, 5, deform=True)
    v32 = sem_inputs.uniform_local(P.L, seed=41, dtype=np.float32)
    ref = P.dssum(v32.astype(np.float64)).astype(np.float32)
    ulp = np.spacing(np.abs(ref).astype(np.float32))
    res = {}
    for mode in (0, 1, 2):
        sem.sem_set_option(S.h, "gs_acc", mode)
        t = cu(v32, torch.float32)
        sem.sem_gs(S.h, t, sem.SEM_MIXED_FP32)
        res[mode] = t.cpu().numpy()
    np.testing.assert_array_equal(res[0], ref)          # FP64 sums, rounded once
    assert np.all(np.abs(res[2] - ref) <= ulp)          # error-free TwoSum
    # plain FP32: m-1 roundings, each bounded by eps32 * (sum of |copies|)
    bound = 8 * 2.0 ** -24 * P.dssum(np.abs(v32.astype(np.float64)))
    assert np.all(np.abs(res[1].astype(np.float64) - ref.astype(np.float64)) <= bound)
    with pytest.raises(sem.SemError):
        sem.sem_set_option(S.h, "gs_acc", 7)
    S.close()


def test_reliable_updates_and_restarts_both_converge(sem):
    """Mixed precision with residual replacement (CG keeps its search
    direction) and with restarted refinement both reach the FP64 target and
    the oracle solution; replacement needs no more iterations than restarts."""
    P = so.Problem(8, 6, 5, 7, deform=True)
    b = P.rhs_uniform(seed=9)
    xo, ito, _ = P.pcg(b, tol=1e-12, maxit=4000)
    S = sem.Solver(8, 6, 5, 7, deform=True)
    res = {}
    for mode in (0, 1):
        x, info = S.solve(cu(b), tol=1e-8, maxit=4000, precision=sem.SEM_MIXED_FP32,
                          refine_mode=mode, history=True)
        assert info["rc"] == 0 and info["relres_true"] <= 1e-8, info
        assert rel_maxerr(x.cpu(), xo) < 1e-7
        assert P.true_relres(b, x.cpu().numpy()) <= 1.05e-8
        res[mode] = info
    assert res[0]["iters"] <= res[1]["iters"]
    h = res[0]["history"]
    assert h[0] == pytest.approx(1.0, rel=1e-6) and h[-1] <= 1e-8
    S.close()


@pytest.mark.parametrize("kx,ky,kz,N", [(3, 2, 2, 3), (3, 2, 3, 4), (2, 3, 2, 7), (2, 2, 3, 9),
                                        (2, 2, 1, 11), (2, 1, 2, 15)])
def test_ax_tensor_cores(sem, kx, ky, kz, N):
    """D-contractions on tensor cores: TF32 products and the three-product
    BF16 split, FP32 accumulation.  Error relative to the FP64 oracle: TF32
    keeps 10 mantissa bits (unit roundoff 2^-11; measured 0.6-1.65 x 2^-11
    on these cases), the BF16 split about 16 (measured 0.36-0.8 x 2^-16).
    Bounds of 3 x those units: a single-product BF16 contraction (unit
    roundoff 2^-8, errors of several 2^-9) fails the TF32 bound."""
    P = so.Problem(kx, ky, kz, N, deform=True)
    S = sem.Solver(kx, ky, kz, N, deform=True)
    u = sem_inputs.uniform_local(P.L, seed=61, dtype=np.float32)
    ref = P.mask * P.ax_local(u.astype(np.float64))
    w = torch.empty(P.L, dtype=torch.float32, device="cuda")
    errs = {}
    for name, prec, tol in (("tf32", sem.SEM_MIXED_TF32, 3.0 * 2.0 ** -11),
                            ("bf16x3", sem.SEM_MIXED_BF16X3, 3.0 * 2.0 ** -16)):
        sem.sem_ax_local(S.h, cu(u, torch.float32), w, prec)
        errs[name] = rel_maxerr(w.cpu(), ref)
        assert errs[name] < tol, (name, errs[name], tol)
    sem.sem_ax_local(S.h, cu(u, torch.float32), w, sem.SEM_MIXED_FP32)
    errs["fp32"] = rel_maxerr(w.cpu(), ref)
    assert errs["bf16x3"] < errs["tf32"]
    # assembled operator through the same path
    sem.sem_ax(S.h, cu(u, torch.float32), w, sem.SEM_MIXED_TF32)
    assert rel_maxerr(w.cpu(), P.ax(u.astype(np.float64))) < 3.0 * 2.0 ** -11
    print(N, errs)
    S.close()
