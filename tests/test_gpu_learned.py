"""Learned initial guess on the GPU against the FP64 oracle: the Fourier
right-hand side, the element features, the network gradients (FP32 debug
mode and BF16 mode), and what the trained guess gains over x0 = 0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import learned_x0 as lx  # noqa: E402
from oracle import sem_oracle as so  # noqa: E402
from tests.gpu_util import rel_maxerr  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2503_02134_gb300 as m
    return m


def test_fourier_rhs_matches_oracle(sem):
    P = so.Problem(3, 2, 2, 5, deform=True)
    S = sem.Solver(3, 2, 2, 5, deform=True)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    for sample in (0, 3):
        sem.sem_rhs_fourier(S.h, 1, sample, b)
        assert rel_maxerr(b.cpu(), lx.fourier_rhs(P, 1, sample)) < 1e-12
    S.close()


def test_features_match_oracle(sem):
    P = so.Problem(4, 3, 2, 3, deform=True)
    S = sem.Solver(4, 3, 2, 3, deform=True)
    m = sem.sem_x0_create(S.h, 32, 0)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs_fourier(S.h, 2, 1, b)
    X = np.zeros((S.E, 544), dtype=np.float32)
    sc = np.zeros(S.E)
    sem.sem_x0_features(m, b, X, sc)
    Xo, so_ = lx.features(P, b.cpu().numpy())
    nf = P.n ** 3 + 18
    np.testing.assert_allclose(sc, so_, rtol=1e-12)
    assert rel_maxerr(X[:, :nf], Xo) < 1e-6
    assert np.all(X[:, nf:] == 0)
    sem.sem_x0_destroy(m)
    S.close()


def test_coarse_features_match_oracle(sem):
    """The optional coarse features (two multigrid-Richardson steps, at the
    element vertices and the element mean) against the oracle's FP64
    definition; the GPU's steps run in FP32 (V-cycle and residual), so the
    bound is a few FP32 V-cycle roundings (the V-cycle test allows 2e-5)."""
    from oracle import pmg
    dims, N = (4, 4, 2), 3
    M = pmg.PMG(*dims, N, deform=True)
    P = M.levels[0].P
    S = sem.Solver(*dims, N, deform=True)
    m = sem.sem_x0_create(S.h, 32, 0)
    sem.sem_x0_set_option(m, "coarse_cycles", 2)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    sem.sem_rhs_fourier(S.h, 2, 1, b)
    X = np.zeros((S.E, 544), dtype=np.float32)
    sc = np.zeros(S.E)
    sem.sem_x0_features(m, b, X, sc)
    Xo, so_ = lx.features(P, b.cpu().numpy())
    Co = lx.coarse_features(P, M.vcycle, b.cpu().numpy(), 2, so_)
    nf = P.n ** 3 + 18
    assert rel_maxerr(X[:, :nf], Xo) < 1e-6
    assert rel_maxerr(X[:, nf:nf + 9], Co) < 1e-4
    assert np.all(X[:, nf + 9:] == 0)
    with pytest.raises(sem.SemError):
        sem.sem_x0_set_option(m, "coarse_cycles", 99)
    sem.sem_x0_destroy(m)
    S.close()


def _bf16(a):
    """Round float32 values to bfloat16 (round to nearest even), kept as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _flat_params(net, offsets, total):
    flat = np.zeros(total, dtype=np.float32)
    for q, p in enumerate(net.params):
        flat[offsets[q]:offsets[q] + p.size] = p.reshape(-1)
    return flat


def test_gradients_match_oracle(sem):
    S = sem.Solver(2, 2, 2, 3)
    H = 32
    m = sem.sem_x0_create(S.h, H, 0)
    sizes, offs = sem.sem_x0_param_count(m)
    total = offs[5] + ((sizes[5] + 31) // 32) * 32
    n3 = 64
    net = lx.MLP([544, H, H, n3], seed=3)
    for q in range(1, 6, 2):   # non-zero biases exercise the bias gradients
        net.params[q] = np.random.default_rng(q).standard_normal(net.params[q].shape) * 0.1
    sem.sem_x0_params(m, _flat_params(net, offs, total), set_=True)
    g = np.random.default_rng(11)
    rows = 40
    X = g.standard_normal((rows, 544)).astype(np.float32)
    T = g.standard_normal((rows, n3)).astype(np.float32)
    # FP32 mode against the plain FP64 network; BF16 mode against the FP64
    # network evaluated on BF16-rounded inputs, targets and weights (what the
    # BF16 products consume), leaving the rounding of activations and sums
    net16 = lx.MLP([544, H, H, n3], params=[_bf16(p) if q % 2 == 0 else p.astype(np.float32)
                                             for q, p in enumerate(net.params)])
    cases = ((0, 1e-5, net, X, T), (1, 1e-2, net16, _bf16(X), _bf16(T)))
    for mode, tol, ref_net, Xr, Tr in cases:
        ref = ref_net.gradients(np.asarray(Xr, np.float64), np.asarray(Tr, np.float64))
        ref_loss = ref_net.loss(np.asarray(Xr, np.float64), np.asarray(Tr, np.float64))
        grads = np.zeros(total, dtype=np.float32)
        loss = sem.sem_x0_gradients(m, X, T, rows, mode, grads)
        assert abs(loss - ref_loss) <= tol * ref_loss
        for q, r in enumerate(ref):
            got = grads[offs[q]:offs[q] + r.size].reshape(r.shape).astype(np.float64)
            err = np.linalg.norm(got - r) / max(np.linalg.norm(r), 1e-30)
            assert err <= tol, (mode, q, err)
    sem.sem_x0_destroy(m)
    S.close()


@pytest.mark.parametrize("H,rows", [(32, 40), (136, 1500), (256, 4096)])
def test_tcgen05_gemm_matches_mma_sync_and_oracle(sem, H, rows):
    """The BF16 products on the tcgen05 tensor cores (TMEM accumulator, the
    default) against the warp-level mma.sync kernel and the FP64 network on
    BF16-rounded operands: the forward products (rows x 544 by 544 x H,
    ragged in M, N and K at H = 136), the data gradients (transposed B) and
    the weight gradients (transposed A, K = rows: split over several blocks
    at 1500 and 4096 rows).  The two kernels round the same BF16 products
    and accumulate in FP32 in different orders, so they agree to 2e-3.  The
    reference rounds only the inputs, targets and weights to BF16; the GPU
    also rounds the activations and the back-propagated errors at each
    product's input (seven of the eight products), which moves the weight
    gradients by up to about 2 % at these sizes (ReLU masks flip where a
    pre-activation is near zero): the bound against the reference is 5e-2,
    still far below the O(1) error of a wrong operand layout."""
    S = sem.Solver(2, 2, 2, 3)
    n3 = 64
    m = sem.sem_x0_create(S.h, H, 0)
    sizes, offs = sem.sem_x0_param_count(m)
    total = offs[5] + ((sizes[5] + 31) // 32) * 32
    net = lx.MLP([544, H, H, n3], seed=5)
    for q in range(1, 6, 2):
        net.params[q] = np.random.default_rng(q + 7).standard_normal(net.params[q].shape) * 0.1
    sem.sem_x0_params(m, _flat_params(net, offs, total), set_=True)
    g = np.random.default_rng(H + rows)
    X = g.standard_normal((rows, 544)).astype(np.float32)
    T = g.standard_normal((rows, n3)).astype(np.float32)
    out = {}
    for umma in (1, 0):
        sem.sem_x0_set_option(m, "umma", umma)
        grads = np.zeros(total, dtype=np.float32)
        loss = sem.sem_x0_gradients(m, X, T, rows, 1, grads)
        out[umma] = (loss, grads)
    net16 = lx.MLP([544, H, H, n3], params=[_bf16(p) if q % 2 == 0 else p.astype(np.float32)
                                             for q, p in enumerate(net.params)])
    ref = net16.gradients(_bf16(X), _bf16(T))
    ref_loss = net16.loss(_bf16(X), _bf16(T))
    (l1, g1), (l0, g0) = out[1], out[0]
    assert abs(l1 - l0) <= 1e-3 * l0
    assert abs(l1 - ref_loss) <= 1e-2 * ref_loss
    for q, r in enumerate(ref):
        a = g1[offs[q]:offs[q] + r.size].astype(np.float64)
        b = g0[offs[q]:offs[q] + r.size].astype(np.float64)
        nr = max(np.linalg.norm(r), 1e-30)
        assert np.linalg.norm(a - b) / nr <= 2e-3, (q, np.linalg.norm(a - b) / nr)
        assert np.linalg.norm(a - r.reshape(-1)) / nr <= 5e-2, q
    sem.sem_x0_destroy(m)
    S.close()


def test_training_reduces_loss_and_guess_is_safe(sem):
    """Train on solver-made pairs; the energy-scaled guess is continuous and
    masked, never needs more than a handful of extra iterations, and the
    iterations it saves are reported."""
    S = sem.Solver(6, 6, 6, 5, deform=True)
    m = sem.sem_x0_create(S.h, 64, 1)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    for sample in range(24):
        sem.sem_rhs_fourier(S.h, 1, sample, b)
        x, info = S.solve(b, tol=1e-9, maxit=4000, precision=sem.SEM_MIXED_FP32)
        assert info["rc"] == 0
        sem.sem_x0_add_pair(m, b, x)
    first = sem.sem_x0_train(m, 1, 256, 1e-3, seed=0)
    last = sem.sem_x0_train(m, 30, 256, 1e-3, seed=1)
    assert last < first
    P = so.Problem(6, 6, 6, 5, deform=True)
    x0 = torch.empty_like(b)
    saved = []
    for sample in (100, 101):
        sem.sem_rhs_fourier(S.h, 1, sample, b)
        sem.sem_x0_predict(m, b, x0, True)
        xh = x0.cpu().numpy()
        np.testing.assert_allclose(P.dssum(xh) / P.mult, xh, rtol=1e-12, atol=1e-14)
        assert np.all(xh[P.mask == 0] == 0)
        _, i0 = S.solve(b, tol=1e-8, maxit=4000, precision=sem.SEM_FP64)
        _, i1 = S.solve(b, x0=x0, tol=1e-8, maxit=4000, precision=sem.SEM_FP64)
        assert i1["rc"] == 0 and i1["relres"] <= 1e-8
        assert i1["iters"] <= i0["iters"] + 10
        saved.append(i0["iters"] - i1["iters"])
    print("iterations saved by the learned guess:", saved)
    sem.sem_x0_destroy(m)
    S.close()


def test_subsampled_pairs_coarse_features_and_smoothing(sem):
    """A model that keeps a seeded half of each pair's element rows, uses
    the coarse features and ends its prediction with two multigrid
    smoothing steps: it trains, its guess stays continuous and masked, and
    the solve from it converges."""
    S = sem.Solver(6, 6, 6, 5, deform=True)
    P = so.Problem(6, 6, 6, 5, deform=True)
    m = sem.sem_x0_create(S.h, 64, 1)
    sem.sem_x0_set_option(m, "pair_rows", S.E // 2)
    sem.sem_x0_set_option(m, "reserve_rows", 12 * (S.E // 2))
    sem.sem_x0_set_option(m, "coarse_cycles", 2)
    b = torch.empty(S.L, dtype=torch.float64, device="cuda")
    for sample in range(12):
        sem.sem_rhs_fourier(S.h, 1, sample, b)
        x, info = S.solve(b, tol=1e-9, maxit=200, precision=sem.SEM_MIXED_FP32, precond="mg")
        assert info["rc"] == 0
        sem.sem_x0_add_pair(m, b, x)
    first = sem.sem_x0_train(m, 1, 128, 1e-3, seed=0)
    last = sem.sem_x0_train(m, 20, 128, 1e-3, seed=1)
    assert last < first
    sem.sem_x0_set_option(m, "post_cycles", 2)
    x0 = torch.empty_like(b)
    sem.sem_rhs_fourier(S.h, 1, 100, b)
    sem.sem_x0_predict(m, b, x0, True)
    xh = x0.cpu().numpy()
    np.testing.assert_allclose(P.dssum(xh) / P.mult, xh, rtol=1e-6, atol=1e-12)
    assert np.all(xh[P.mask == 0] == 0)
    _, i1 = S.solve(b, x0=x0, tol=1e-8, maxit=4000, precision=sem.SEM_MIXED_FP32)
    assert i1["rc"] == 0
    sem.sem_x0_destroy(m)
    S.close()
