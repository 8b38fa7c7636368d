"""Multigrid preconditioner on the GPU against the oracle (oracle/pmg.py):
the damping of every level, the V-cycle in FP64 and FP32, its symmetry, and
the multigrid-preconditioned solves (FP64 and mixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pmg  # noqa: E402
from oracle import sem_oracle as so  # noqa: E402
from tests.gpu_util import rel_maxerr  # noqa: E402

CASES = [((3, 3, 2), 5, True), ((4, 3, 3), 7, True), ((2, 1, 3), 2, False), ((3, 2, 2), 9, True),
         # with h-levels below N = 1: 4^3 -> 2^3; 8x4x4 -> 4x2x2; 8^3 -> 4^3 -> 2^3
         ((4, 4, 4), 3, True), ((8, 4, 4), 5, True), ((8, 8, 8), 1, False)]


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as m
    return m


def _continuous(P, seed):
    g = np.random.default_rng(seed)
    return P.mask * P.dssum(g.standard_normal(P.L)) / P.mult


@pytest.mark.parametrize("dims,N,deform", CASES)
def test_vcycle_matches_oracle(sem, dims, N, deform):
    M = pmg.PMG(*dims, N, deform=deform)
    P = M.levels[0].P
    S = sem.Solver(*dims, N, deform=deform)
    r = _continuous(P, 7)
    rg = torch.tensor(r, device="cuda")
    z = torch.empty_like(rg)
    sem.sem_mg_apply(S.h, rg, z, sem.SEM_FP64)
    assert sem.sem_get_option(S.h, "mg_levels") == len(M.levels)
    for l, lev in enumerate(M.levels):
        assert abs(sem.sem_get_option(S.h, f"mg_omega_{l}") - lev.omega) <= 1e-9 * lev.omega
    zo = M.vcycle(r)
    assert rel_maxerr(z.cpu(), zo) < 1e-10
    # FP32 cycle: FP32 rounding of the same arithmetic
    z32 = torch.empty(S.L, dtype=torch.float32, device="cuda")
    sem.sem_mg_apply(S.h, rg.float(), z32, sem.SEM_MIXED_FP32)
    assert rel_maxerr(z32.double().cpu(), zo) < 2e-5
    S.close()


@pytest.mark.parametrize("dims,N", [((4, 3, 3), 7), ((8, 4, 4), 5)])
def test_vcycle_symmetric_on_device(sem, dims, N):
    """<M^-1 a, b> = <a, M^-1 b> on the device.  (8, 4, 4) at N = 5 has an
    h-level (N = 1 on 4x2x2), so the trilinear prolongation and its adjoint
    are part of the cycle; (4, 3, 3) has p-levels only.  FP64 to rounding;
    FP32 cycles to a few FP32 ulps of the Cauchy-Schwarz scale
    sqrt(<M^-1 a, a> <M^-1 b, b>)."""
    S = sem.Solver(*dims, N, deform=True)
    P = so.Problem(*dims, N, deform=True)
    a = torch.tensor(_continuous(P, 1), device="cuda")
    b = torch.tensor(_continuous(P, 2), device="cuda")
    za, zb = torch.empty_like(a), torch.empty_like(b)
    sem.sem_mg_apply(S.h, a, za, sem.SEM_FP64)
    sem.sem_mg_apply(S.h, b, zb, sem.SEM_FP64)
    x = sem.sem_glsc3(S.h, za, b, sem.SEM_FP64)
    y = sem.sem_glsc3(S.h, a, zb, sem.SEM_FP64)
    assert abs(x - y) <= 1e-12 * abs(x)
    assert sem.sem_glsc3(S.h, za, a, sem.SEM_FP64) > 0
    if N == 5:
        assert sem.sem_get_option(S.h, "mg_levels") >= 4   # 5 -> 2 -> 1, then N = 1 on 4x2x2
    a32, b32 = a.float(), b.float()
    za32 = torch.empty_like(a32)
    zb32 = torch.empty_like(b32)
    sem.sem_mg_apply(S.h, a32, za32, sem.SEM_MIXED_FP32)
    sem.sem_mg_apply(S.h, b32, zb32, sem.SEM_MIXED_FP32)
    x32 = sem.sem_glsc3(S.h, za32.double(), b32.double(), sem.SEM_FP64)
    y32 = sem.sem_glsc3(S.h, a32.double(), zb32.double(), sem.SEM_FP64)
    scale = np.sqrt(sem.sem_glsc3(S.h, za32.double(), a32.double(), sem.SEM_FP64) *
                    sem.sem_glsc3(S.h, zb32.double(), b32.double(), sem.SEM_FP64))
    assert abs(x32 - y32) <= 1e-5 * scale
    S.close()


@pytest.mark.parametrize("dims,N", [((4, 3, 3), 7), ((3, 3, 2), 5), ((8, 4, 4), 5), ((4, 4, 4), 7)])
def test_mg_pcg_matches_oracle(sem, dims, N):
    M = pmg.PMG(*dims, N, deform=True)
    P = M.levels[0].P
    b = P.rhs_uniform(0)
    xo, ito, _ = M.pcg(b, tol=1e-10, maxit=300)
    S = sem.Solver(*dims, N, deform=True)
    bg = torch.tensor(b, device="cuda")
    x, info = S.solve(bg, tol=1e-10, maxit=300, precision=sem.SEM_FP64, precond="mg")
    assert info["rc"] == 0 and info["relres_true"] <= 1e-10
    assert abs(info["iters"] - ito) <= 1
    assert rel_maxerr(x.cpu(), xo) < 1e-8
    _, ij = S.solve(bg, tol=1e-10, maxit=5000, precision=sem.SEM_FP64)
    assert info["iters"] * 5 <= ij["iters"]
    # mixed: FP32 cycles and CG, FP64 restarts, to the FP64 true residual
    xm, im = S.solve(bg, tol=1e-8, maxit=300, precision=sem.SEM_MIXED_FP32, precond="mg")
    assert im["rc"] == 0 and im["relres_true"] <= 1e-8
    assert P.true_relres(b, xm.cpu().numpy()) <= 1.0000001e-8
    # reliable updates keep the search direction: about as many iterations
    # as FP64; the restarted refinement (refine_mode 1) also converges
    assert im["iters"] <= info["iters"] + max(5, info["iters"] // 5)
    xr, ir = S.solve(bg, tol=1e-8, maxit=300, precision=sem.SEM_MIXED_FP32, precond="mg",
                     refine_mode=1)
    assert ir["rc"] == 0 and P.true_relres(b, xr.cpu().numpy()) <= 1.0000001e-8
    S.close()


def test_h_coarsening_option(sem):
    """Option "mg_hcoarsen" 0 keeps the orders-only hierarchy (the oracle's
    hcoarsen=False), 1 (default) adds the halved N = 1 meshes; switching
    rebuilds the levels."""
    dims, N = (8, 4, 4), 3
    S = sem.Solver(*dims, N, deform=True)
    P = so.Problem(*dims, N, deform=True)
    r = torch.tensor(_continuous(P, 9), device="cuda")
    z = torch.empty_like(r)
    for hc in (0, 1):
        sem.sem_set_option(S.h, "mg_hcoarsen", hc)
        assert sem.sem_get_option(S.h, "mg_hcoarsen") == hc
        M = pmg.PMG(*dims, N, deform=True, hcoarsen=bool(hc))
        sem.sem_mg_apply(S.h, r, z, sem.SEM_FP64)
        assert sem.sem_get_option(S.h, "mg_levels") == len(M.levels) == 2 + hc
        assert rel_maxerr(z.cpu(), M.vcycle(r.cpu().numpy())) < 1e-10
    S.close()


def test_mg_rejects_user_numbering(sem):
    P = so.Problem(2, 2, 2, 3)
    gid = P.gid.astype(np.int64)
    coords = np.ascontiguousarray(P.X.reshape(3, -1))
    faces = np.full(P.E, 63, dtype=np.uint8)
    S = sem.Solver(0, 0, 0, 3, mesh=sem.user_mesh(P.E, gid, coords, faces))
    r = torch.zeros(P.L, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(sem.SemError):
        sem.sem_mg_apply(S.h, r, z, sem.SEM_FP64)
    S.close()
