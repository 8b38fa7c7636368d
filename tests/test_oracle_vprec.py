"""Pins of the reduced-precision emulation (VPREC-style, Sec. 2 and 3.2):
t = 23 and t = 10 reproduce numpy's float32 and float16 rounding, t = 52 is
the FP64 oracle, and the CG loop's attainable true residual falls as the
mantissa grows (the paper's residual-versus-precision sweep)."""
import numpy as np

from oracle import sem_oracle as so
from oracle import vprec


def test_rounding_matches_ieee_formats():
    g = np.random.default_rng(0)
    x = g.standard_normal(20000) * 10.0 ** g.uniform(-3, 3, 20000)
    np.testing.assert_array_equal(vprec.round_t(x, 23), x.astype(np.float32).astype(np.float64))
    # float16's normal range only: below 2^-14 IEEE half loses mantissa bits,
    # the emulation keeps FP64's exponent range (as VPREC does)
    y = g.choice([-1.0, 1.0], 20000) * 2.0 ** g.uniform(-13.9, 15.9, 20000)
    np.testing.assert_array_equal(vprec.round_t(y, 10), y.astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(vprec.round_t(x, 52), x)
    # ties go to even
    assert vprec.round_t(np.array([1.0 + 2.0 ** -24]), 23)[0] == 1.0
    assert vprec.round_t(np.array([1.0 + 3 * 2.0 ** -24]), 23)[0] == 1.0 + 2.0 ** -22


def test_t52_is_the_fp64_oracle():
    P = so.Problem(2, 2, 2, 3, deform=True)
    b = P.rhs_uniform(1)
    hist, true = vprec.pcg_t(P, b, 52, tol=1e-12, maxit=100)
    _, it, ho = P.pcg(b, tol=1e-12, maxit=100)
    assert len(hist) == it
    # the dots here sum sequentially, the oracle's pairwise: agreement to
    # rounding order, which the late iterations amplify
    np.testing.assert_allclose(hist, ho[1:], rtol=1e-6)


def test_attainable_residual_improves_with_mantissa_bits():
    P = so.Problem(3, 3, 3, 4, deform=True)
    b = P.rhs_uniform(0)
    floors = {}
    for t in (7, 10, 16, 23, 52):
        _, true = vprec.pcg_t(P, b, t, tol=1e-13, maxit=150)
        floors[t] = true.min()
    assert floors[7] > floors[10] > floors[16] > floors[23] > floors[52]
    assert floors[23] > 1e-9          # FP32 cannot reach the paper's 1e-10 on its own
    assert floors[52] < 1e-10


def test_random_rounding_noise_is_unbiased_and_bounded():
    """MCA random rounding: |inexact(x) - x| <= 2^(e_x - t - 1) with e_x the
    exponent of x, mean noise ~ 0, zero unchanged; the noise relative to x
    spans the t-bit spacing (x = 1: 2^-t wide)."""
    g = np.random.default_rng(1)
    t = 10
    x = g.standard_normal(200000) * 10.0 ** g.uniform(-5, 5, 200000)
    x[:10] = 0.0
    y = vprec.random_rounding(x, t, np.random.default_rng(2))
    assert np.all(y[:10] == 0.0)
    ex = np.floor(np.log2(np.abs(x[10:])))
    d = (y[10:] - x[10:]) / np.exp2(ex - t)
    assert np.all(np.abs(d) <= 0.5 + 1e-9)
    assert abs(d.mean()) < 0.01 and abs(d.std() * np.sqrt(12) - 1.0) < 0.01   # U[-1/2, 1/2)
    ones = vprec.random_rounding(np.ones(100000), t, np.random.default_rng(3))
    assert np.ptp(ones) > 0.99 * 2.0 ** -t and np.ptp(ones) <= 2.0 ** -t
