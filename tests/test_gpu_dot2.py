"""Compensated dot products (the dot2 the paper evaluates for its FP32 CG,
Sec. 4.3, Fig. "dot2 results"): the mixed path's reductions keep about FP32
unit roundoff up to condition numbers near 1e8, while plain FP32 sums lose
accuracy in proportion to the condition number.

The ill-conditioned vectors come from a generator written from Ogita, Rump &
Oishi's description (2005, "Accurate sum and dot product"): half of the
products get random exponents spread over log2(cond)/2 bits, the other half
is chosen to cancel the running sum, so the exact result is tiny relative to
sum |x_i y_i|.  Exact references: math.fsum of the exact FP64 products of the
FP32 inputs."""
import math

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


def gen_dot(n, cond, rng):
    """FP32 vectors x, y of length n with dot condition near `cond`."""
    half = n // 2
    b = math.log2(cond)
    x = np.zeros(n, dtype=np.float32)
    y = np.zeros(n, dtype=np.float32)
    e = np.rint(rng.random(half) * b / 2).astype(int)
    e[0] = int(round(b / 2)) + 1
    e[-1] = 0
    x[:half] = ((2 * rng.random(half) - 1) * 2.0 ** e).astype(np.float32)
    y[:half] = ((2 * rng.random(half) - 1) * 2.0 ** e).astype(np.float32)
    e2 = np.rint(np.linspace(b / 2, 0, n - half)).astype(int)
    for i in range(half, n):
        xi = np.float32((2 * rng.random() - 1) * 2.0 ** e2[i - half])
        partial = math.fsum(float(x[j]) * float(y[j]) for j in range(i))
        yi = np.float32(((2 * rng.random() - 1) * 2.0 ** e2[i - half] - partial) / float(xi))
        x[i], y[i] = xi, yi
    perm = rng.permutation(n)
    return x[perm], y[perm]


def exact_dot(x, y):
    return math.fsum(float(a) * float(b) for a, b in zip(x, y))


def test_dot2_keeps_fp32_roundoff_until_cond_1e8(sem):
    # one N = 15 element: its 14^3 interior nodes have glsc3 weight c = 1,
    # every face node has c = 0 (Dirichlet), so glsc3 is a plain dot over them
    S = sem.Solver(1, 1, 1, 15)
    n = S.n
    interior = np.zeros((n, n, n), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    idx = np.flatnonzero(interior.reshape(-1))
    rng = np.random.default_rng(5)
    u32 = 2.0 ** -23
    for cond in (1e2, 1e3, 1e4, 1e6, 1e8):
        x, y = gen_dot(idx.size, cond, rng)
        ref = exact_dot(x, y)
        real_cond = 2 * math.fsum(abs(float(a) * float(b)) for a, b in zip(x, y)) / abs(ref)
        a = np.zeros(S.L, dtype=np.float32)
        b = np.zeros(S.L, dtype=np.float32)
        a[idx], b[idx] = x, y
        ta = torch.as_tensor(a, device="cuda")
        tb = torch.as_tensor(b, device="cuda")
        d2 = sem.sem_glsc3(S.h, ta, tb, sem.SEM_MIXED_FP32)
        d32 = sem.sem_glsc3(S.h, ta, tb, sem.SEM_FP32_ALL)
        e2 = abs(d2 - ref) / abs(ref)
        e32 = abs(d32 - ref) / abs(ref)
        print(f"cond {real_cond:.2e}: dot2 {e2:.2e}  fp32 {e32:.2e}")
        # dot2 runs over the few terms of one thread, FP64 across threads:
        # the error stays near FP32 unit roundoff while cond <~ 1e8
        if real_cond <= 1e8:
            assert e2 <= 128 * u32, (real_cond, e2)
        if real_cond >= 1e6:
            assert e32 > 10 * e2, (real_cond, e32, e2)
    S.close()
