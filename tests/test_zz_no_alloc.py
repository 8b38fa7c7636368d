"""The allocation-free weighted dot product (sem_glsc3_noalloc) matches the
handle-based sem_glsc3.

Callers that cannot allocate device memory use this entry point: its
scratch is a static device array, so these tests also check that two calls
in a row (sharing that array) both give the right answer, and that sizes
beyond the array's capacity are refused.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as m
    return m


def test_noalloc_dot_matches_handle_dot_twice(sem):
    import sem_inputs
    S = sem.Solver(5, 4, 3, 7, deform=True)
    c = S.field(sem.FIELD_C)
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (51, 52):   # two calls in a row share the static scratch
        a = torch.as_tensor(sem_inputs.uniform_local(S.L, seed=seed), device="cuda")
        b = torch.as_tensor(sem_inputs.uniform_local(S.L, seed=seed + 100), device="cuda")
        ref = sem.sem_glsc3(S.h, a, b, sem.SEM_FP64)
        sem.sem_glsc3_noalloc(a, b, c, S.L, res)
        torch.cuda.synchronize()
        got = float(res.item())
        scale = float(torch.sum(torch.abs(a * c * b)).item())
        assert abs(got - ref) <= 1e-13 * scale, (got, ref)
    S.close()


def test_noalloc_dot_ragged_and_empty(sem):
    g = np.random.default_rng(3)
    for n in (1, 8191, 8193, 100003):
        a = torch.as_tensor(g.standard_normal(n), device="cuda")
        b = torch.as_tensor(g.standard_normal(n), device="cuda")
        c = torch.as_tensor(g.random(n), device="cuda")
        res = torch.zeros(1, dtype=torch.float64, device="cuda")
        sem.sem_glsc3_noalloc(a, b, c, n, res)
        torch.cuda.synchronize()
        ref = float(np.sum(a.cpu().numpy() * c.cpu().numpy() * b.cpu().numpy()))
        scale = float(np.sum(np.abs(a.cpu().numpy() * c.cpu().numpy() * b.cpu().numpy())))
        assert abs(res.item() - ref) <= 1e-13 * scale
    res = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    sem.sem_glsc3_noalloc(a, b, c, 0, res)
    torch.cuda.synchronize()
    assert res.item() == 0.0


def test_noalloc_dot_rejects_oversize(sem):
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError, match="capacity"):
        sem.sem_glsc3_noalloc(a, a, a, 33554433, res)
