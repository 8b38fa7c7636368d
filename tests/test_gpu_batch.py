"""Batched solves: each problem of a batch of uneven sizes and orders gets
the same answer as its standalone solve and as the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import sem_oracle as so  # noqa: E402
from tests.gpu_util import rel_maxerr  # noqa: E402

CASES = [(4, 4, 3, 5), (3, 3, 3, 7), (2, 3, 2, 9), (5, 2, 2, 3), (3, 2, 2, 1), (3, 3, 2, 7)]


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as m
    return m


def test_batch_matches_standalone_and_oracle(sem):
    meshes = [sem.box_mesh(kx, ky, kz, deform=True) for kx, ky, kz, _ in CASES]
    Ns = [c[3] for c in CASES]
    b = sem.sem_batch_setup(meshes, Ns)
    for N in set(Ns):
        assert sem.sem_batch_get_option(b, f"variant_n{N + 1}") in (0, 1, 2, 3)
        assert sem.sem_batch_get_option(b, f"grid_n{N + 1}") >= 1
    assert sem.sem_batch_get_option(b, "variant_n4") == -1 or 3 in Ns
    # box meshes with n = 8: the gather-scatter is folded into the update
    assert sem.sem_batch_get_option(b, "fused_problems") == sum(N == 7 for N in Ns)
    fs, xs = [], []
    for i, c in enumerate(CASES):
        h = sem.sem_batch_problem(b, i)
        L = sem.sem_get_sizes(h).L
        f = torch.empty(L, dtype=torch.float64, device="cuda")
        sem.sem_rhs(h, sem.RHS_UNIFORM, 1000 + i, f)
        fs.append(f)
        xs.append(torch.zeros_like(f))
    o = sem.sem_solve_opts()
    o.tol, o.maxit, o.precision = 1e-8, 4000, sem.SEM_MIXED_FP32
    rc, infos = sem.sem_batch_pcg_solve(b, fs, xs, o)
    assert rc == 0, infos
    for i, (kx, ky, kz, N) in enumerate(CASES):
        info = infos[i]
        assert info["status"] == 0 and info["relres_true"] <= 1e-8, (i, info)
        P = so.Problem(kx, ky, kz, N, deform=True)
        bo = P.rhs_uniform(1000 + i)
        np.testing.assert_array_equal(fs[i].cpu().numpy(), bo)
        xo, _, _ = P.pcg(bo, tol=1e-12, maxit=5000)
        assert rel_maxerr(xs[i].cpu(), xo) < 1e-7, i
        S = sem.Solver(kx, ky, kz, N, deform=True)
        xs1, i1 = S.solve(fs[i], tol=1e-8, maxit=4000, precision=sem.SEM_MIXED_FP32)
        assert abs(i1["iters"] - info["iters"]) <= 3, (i, i1["iters"], info["iters"])
        assert rel_maxerr(xs[i].cpu(), xs1.cpu()) < 1e-6
        S.close()
    # a second solve on the same batch (graphs replayed) gives the same result
    xs2 = [torch.zeros_like(f) for f in fs]
    rc2, infos2 = sem.sem_batch_pcg_solve(b, fs, xs2, o)
    assert rc2 == 0
    for i in range(len(CASES)):
        assert infos2[i]["iters"] == infos[i]["iters"]
        assert torch.equal(xs2[i], xs[i])
    sem.sem_batch_destroy(b)


def test_batch_rejects_even_orders(sem):
    with pytest.raises(sem.SemError, match="odd N"):
        sem.sem_batch_setup([sem.box_mesh(2, 2, 2)], [4])
