"""CPU checks of the arithmetic the exact-digit tensor-core Gram relies on.

The GPU kernel splits each FP32 value x of row i, scaled by a power of two
s_i with max |x s_i| in [32, 64), into three integer digits in base 2^7,
x s = d0 + d1 / 2^7 + d2 / 2^14 + r / 2^14, and forms all nine digit
products exactly in FP32 accumulators over windows of 1024 columns.  These
tests restate that split in plain FP64 numpy (no code shared with the
kernel) and check the facts the design and the GPU tolerances assume: the
digits are integers within +-64 and exact in FP16, the split is exact but
for r, |r| <= 1/2, the worst-case window sums stay below 2^24, and the trace
noise of the representation has the standard deviation the GPU tests use.
"""
import numpy as np


def _scales(X):
    """Power-of-two row scales with max |x s| in [32, 64) (zero row: 1)."""
    rmax = np.abs(X).max(axis=1)
    _, ex = np.frexp(rmax)                 # rmax = m 2^ex, m in [0.5, 1)
    return np.where(rmax > 0, np.ldexp(1.0, 6 - ex), 1.0)


def _split(X):
    """Digits d0, d1, d2 and the remainder r of each scaled value (FP64, exact
    for FP32 inputs: every step is a rounding to an integer or a subtraction
    and scaling by a power of two that FP64 represents exactly)."""
    s = _scales(X)[:, None]
    xs = X * s
    d0 = np.rint(xs)
    e = xs - d0
    d1 = np.rint(128.0 * e)
    f = 128.0 * e - d1
    d2 = np.rint(128.0 * f)
    r = 128.0 * f - d2
    return s, xs, d0, d1, d2, r


def _fp32_matrix(rng, I, K):
    rs = 10.0 ** rng.uniform(-3, 3, I)
    return (rng.standard_normal((I, K)) * rs[:, None]).astype(np.float32).astype(np.float64)


def test_digits_are_bounded_integers_exact_in_fp16():
    rng = np.random.default_rng(1)
    X = _fp32_matrix(rng, 64, 4000)
    s, xs, d0, d1, d2, r = _split(X)
    assert np.all(np.abs(xs) < 64.0) and np.all(np.abs(xs).max(axis=1) >= 32.0)
    for d in (d0, d1, d2):
        assert np.all(d == np.round(d)) and np.abs(d).max() <= 64
        assert np.array_equal(d.astype(np.float16).astype(np.float64), d)
    # d2 / 2^7 is the fourth operand plane: exact in FP16 too
    q = d2 / 128.0
    assert np.array_equal(q.astype(np.float16).astype(np.float64), q)
    # the split is exact but for the last rounding
    assert np.all(xs == d0 + d1 / 2**7 + d2 / 2**14 + r / 2**14)
    assert np.abs(r).max() <= 0.5


def test_representation_error_bound():
    """|x - digits / s| <= 2^(floor(log2 max_k |x_ik|) - 20): the bound the GPU
    exact-digit tests use for every Gram entry."""
    rng = np.random.default_rng(2)
    X = _fp32_matrix(rng, 50, 3000)
    s, xs, d0, d1, d2, r = _split(X)
    err = np.abs(X - (d0 + d1 / 2**7 + d2 / 2**14) / s)
    _, ex = np.frexp(np.abs(X).max(axis=1))
    bound = np.ldexp(1.0, ex - 21)[:, None]
    assert np.all(err <= bound)
    # and not loose: the rounding does reach about half of it
    assert (err / bound).max() > 0.45


def test_window_sums_stay_below_2_24():
    """Over 1024 columns the grouped integer products D0, D1, D2 stay below 2^24
    in magnitude even when every digit sits at its bound, so the FP32
    accumulator holds them exactly (D3 is the only rounded accumulator)."""
    W, dmax = 1024, 64
    d0_max = W * dmax * dmax
    d1_max = W * 2 * dmax * dmax
    d2_max = W * 3 * dmax * dmax
    assert max(d0_max, d1_max, d2_max) < 2**24
    # a 2048-column window would overflow D2: the window is as long as it can be
    assert 2 * d2_max >= 2**24


def test_digit_products_reproduce_the_gram_exactly():
    """The nine digit products, grouped by weight, sum (in exact rational
    arithmetic via FP64 integers per window) to the Gram of the represented
    values: nothing is lost between the digits and the accumulators."""
    rng = np.random.default_rng(3)
    X = _fp32_matrix(rng, 6, 1024)
    s, xs, d0, d1, d2, r = _split(X)
    D0 = d0 @ d0.T
    D1 = d0 @ d1.T + d1 @ d0.T
    D2 = d0 @ d2.T + d1 @ d1.T + d2 @ d0.T
    D3 = d1 @ d2.T + d2 @ d1.T + (d2 / 128.0) @ d2.T
    for D in (D0, D1, D2):
        assert np.all(D == np.round(D)) and np.abs(D).max() < 2**24
    rep = d0 + d1 / 2**7 + d2 / 2**14
    want = rep @ rep.T
    got = D0 + D1 / 2**7 + D2 / 2**14 + D3 / 2**21
    assert np.allclose(got, want, rtol=1e-15, atol=0)


def test_trace_noise_sigma_matches_the_spread():
    """The GPU trace tests allow 6 sigma with sigma^2 = sum_i (4/3) h_i^2
    ||x_i||^2, h_i the half step 2^(floor(log2 max_i) - 20), once the mean of
    sum r^2 is removed from the diagonal.  Over many independent tensors the
    observed trace errors have that spread."""
    rng = np.random.default_rng(4)
    z = []
    for _ in range(60):
        X = _fp32_matrix(rng, 16, 2000)
        s, xs, d0, d1, d2, r = _split(X)
        rep = (d0 + d1 / 2**7 + d2 / 2**14) / s
        dtr = np.sum(rep * rep - X * X) - np.sum((r / 2**14 / s) ** 2)
        _, ex = np.frexp(np.abs(X).max(axis=1))
        h = np.ldexp(1.0, ex - 21)
        sigma = np.sqrt(np.sum(4.0 / 3.0 * h**2 * np.sum(X * X, axis=1)))
        z.append(dtr / sigma)
    z = np.array(z)
    # the bound: the remainder is within half a step, so its variance is at
    # most the uniform one (h^2 / 3); the observed spread is at most ~1
    assert np.abs(z).max() < 6.0
    assert 0.2 < z.std() < 1.3
    assert abs(z.mean()) < 3 * z.std() / np.sqrt(len(z)) + 0.1


def _tail(S, R):
    return float(np.sort(np.linalg.eigvalsh(S))[: S.shape[0] - R].sum())


def test_subtracting_squared_remainders_keeps_the_discarded_sum_unbiased():
    """The sign of the diagonal correction.  r is x's own low part, so the
    digit products sum to S - O(rho) S + diag(sum_k r_ik^2): left alone, the
    last term lifts each of the I - R small eigenvalues by ~K E[r^2].  On a
    rank-8 tensor plus 1e-7 noise (the benchmarks' recipe, FP32) the Gram of
    the digits minus sum_k r^2 on the diagonal has the exact Gram's discarded
    sum to a small fraction of that lift; with no correction the sum is one
    lift high, with sum_k r^2 added (the trace-preserving choice) two."""
    from paper_1901_06043_gb300 import synth
    dims, core = (64, 12, 10, 50), (8, 8, 8, 8)
    x, _ = synth.tucker_numpy(dims, core, decay=0.1, eta=1e-7, seed=5)
    X = x.astype(np.float32).astype(np.float64).reshape(-1, dims[0]).T   # I x K
    I, K, R = dims[0], X.shape[1], 8
    s, xs, d0, d1, d2, r = _split(X)
    rep = (d0 + d1 / 2**7 + d2 / 2**14) / s                # exact in FP64
    Xl, Dl = X.astype(np.longdouble), rep.astype(np.longdouble)
    S = np.array(Xl @ Xl.T, dtype=np.float64)
    G = np.array(Dl @ Dl.T, dtype=np.float64)
    r2 = np.sum((r / 2**14 / s) ** 2, axis=1)
    true = _tail(S, R)
    lift = r2.mean() * (I - R)                             # ~ (I - R) K E[r^2]
    err = {c: _tail(G + c * np.diag(r2), R) - true for c in (-1, 0, 1)}
    assert abs(err[-1]) <= 0.02 * lift, (err, lift)
    assert 0.7 * lift <= err[0] <= 1.3 * lift, (err, lift)
    assert 1.7 * lift <= err[1] <= 2.3 * lift, (err, lift)
