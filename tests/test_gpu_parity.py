"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison runs on the same seeded inputs on both sides.  Tolerances
(FP64 path): relative reconstruction-error difference <= 1e-12, eigenvalues
<= 1e-10 relative to the largest, factor subspaces by largest principal
angle <= 1e-8 rad where the eigenvalue gap at the cut is wide, identical
ranks.  FP32 products get the bound derived from single rounding of each
product (documented beside each test).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_06043_gb300 import tucker
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = tucker.Context(timing=True)
    yield c
    c.close()


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().double().cpu().numpy()


def max_angle(U, W):
    """Largest principal angle between span(U) and span(W) (orthonormal)."""
    s = np.linalg.svd(U.T @ W, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def sin_angle(U, W):
    """sin of the largest principal angle (accurate for small angles)."""
    P = W - U @ (U.T @ W)
    return float(np.linalg.norm(P, 2))


# ----------------------------------------------------------------- norm

@pytest.mark.parametrize("n", [1, 255, 256, 1000, 65537])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_norm_sq(ctx, n, dt):
    x = np.random.default_rng(n).standard_normal(n)
    t = dev(x, dt)
    want = oracle.norm_sq(host(t))
    got = ctx.norm_sq(t)
    assert abs(got - want) <= 1e-13 * want


@pytest.mark.parametrize("scale", ["huge", "tiny", "mixed"])
def test_norm_sq_extreme_magnitudes_fp32(ctx, scale):
    """FP32 inputs whose squares overflow (|x| >= 2^64) or underflow FP32:
    the FP64 sum of the exact squares either way."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100003)
    if scale == "huge":
        x *= 1e25
    elif scale == "tiny":
        x *= 1e-25
    else:
        x *= 10.0 ** rng.uniform(-30, 30, x.size)
    t = dev(x, torch.float32)
    xs = host(t)
    want = oracle.norm_sq(xs)
    got = ctx.norm_sq(t)
    assert abs(got - want) <= 1e-13 * want


def test_norm_nonfinite_is_reported(ctx):
    from paper_1901_06043_gb300.tucker import TuckerError
    x = np.ones(1000)
    x[777] = np.nan
    with pytest.raises(TuckerError) as e:
        ctx.norm_sq(dev(x))
    assert e.value.name == "NONFINITE"
    x[777] = np.inf
    with pytest.raises(TuckerError):
        ctx.sthosvd(dev(x), (10, 100), eps=1e-3)


# ----------------------------------------------------------------- Gram

GRAM_SHAPES = [
    (7,), (1, 5), (130, 3), (3, 130), (65, 9, 4), (5, 64, 3), (4, 3, 70), (33, 1, 17, 2),
    (2, 3, 2, 3, 2), (200, 300), (17, 129, 5), (3, 2, 1000),
    (500, 2000), (257, 1000), (1024, 90),
]


@pytest.mark.parametrize("dims", GRAM_SHAPES)
def test_gram_fp64(ctx, dims):
    x = np.random.default_rng(sum(dims)).standard_normal(oracle.linear_size(dims))
    t = dev(x)
    for n in range(len(dims)):
        want = oracle.gram(x, dims, n)
        got = host(ctx.gram(t, dims, n, "fp64"))
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-13 * scale * max(1, math.log2(x.size)), (dims, n)
        assert np.array_equal(got, got.T)


@pytest.mark.parametrize("dims", GRAM_SHAPES)
def test_gram_fp32_products(ctx, dims):
    """FP32 products of FP32 inputs: each product rounds once (rel 2^-24), the
    FP32 chunk sums add <= 64 terms, chunks are summed in FP64: the error
    stays below 1e-6 of max|S| for these sizes."""
    x = np.random.default_rng(sum(dims) + 1).standard_normal(oracle.linear_size(dims))
    t = dev(x, torch.float32)
    xs = host(t)
    for n in range(len(dims)):
        want = oracle.gram(xs, dims, n)
        got = host(ctx.gram(t, dims, n, "fp32"))
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), (dims, n)


@pytest.mark.parametrize("decay", [False, True])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_gram_fp32_trace_unbiased(ctx, mode, decay):
    """trace(S) = ||Y||^2.  The eps cut is decided by the trace of S's error
    on the discarded subspace, so the FP32-product Gram must not round with
    a bias: on 1.3e8 Gaussian entries its trace must match the FP64 sum of
    squares to 3e-10 (random rounding leaves ~1e-10; summing squares one by
    one into long FP32 runs leaves a -2e-9 bias).  With `decay` the entries
    shrink geometrically along mode 0, as the l index of a row-mode view does
    after truncation."""
    dims = (64, 512, 4000)
    g = torch.Generator(device="cuda").manual_seed(21 + mode)
    t = torch.randn(dims[::-1], generator=g, device="cuda", dtype=torch.float32)
    if decay:
        t *= 0.8 ** torch.arange(64, device="cuda", dtype=torch.float32)
    t = t.reshape(-1)
    want = float((t.double() ** 2).sum())
    got = float(torch.trace(ctx.gram(t, dims, mode, "fp32")))
    # with decay, a few rows carry most of the trace, so fewer independent
    # rounding errors average out
    assert abs(got - want) <= (1e-9 if decay else 3e-10) * want, (got - want) / want


@pytest.mark.parametrize("mode", [2, 3])
def test_gram_fp32_trace_unbiased_two_decaying_modes(ctx, mode):
    """Entries decaying geometrically along modes 0 and 1, as after two
    truncated modes: the l index of modes 2 and 3 runs over (l0, l1) with
    energy falling along each, so a K-block that crossed a multiple of J_0
    would add the small tail of one l0 run after the large head of the next.
    Blocks aligned to J_0 and summed smallest-first keep the trace within
    1e-9 of the FP64 sum of squares, the bound of the one-mode decay case
    (few rows carry the trace, so fewer rounding errors average out)."""
    dims = (40, 40, 512, 200)
    g = torch.Generator(device="cuda").manual_seed(5 + mode)
    t = torch.randn(dims[::-1], generator=g, device="cuda", dtype=torch.float32)
    t *= (0.8 ** torch.arange(40, device="cuda", dtype=torch.float32))
    t *= (0.8 ** torch.arange(40, device="cuda", dtype=torch.float32)).view(40, 1)
    t = t.reshape(-1)
    want = float((t.double() ** 2).sum())
    got = float(torch.trace(ctx.gram(t, dims, mode, "fp32")))
    assert abs(got - want) <= 1e-9 * want, (got - want) / want


def test_sharded_gram_sums_to_unsharded(ctx):
    """A tensor split along its last mode over 2 ranks: the CUDA path's Grams
    of the two shards, summed in rank order (the sharded design's only
    exchange), equal the unsharded Gram and the oracle's, for every mode
    n < N-1, with FP64 and with FP32 products."""
    from paper_1901_06043_gb300 import shard
    dims = (130, 40, 9, 6)
    x = np.random.default_rng(11).standard_normal(oracle.linear_size(dims))
    for dtype, prec, tol in [(torch.float64, "fp64", 1e-13), (torch.float32, "fp32", 1e-6)]:
        t = dev(x, dtype)
        xs = host(t)
        for n in range(len(dims) - 1):
            full = host(ctx.gram(t, dims, n, prec))
            acc = None
            for r in range(2):
                a, b = shard.shard_slice(dims, 2, r)
                part = host(ctx.gram(t[a:b], shard.shard_dims(dims, 2, r), n, prec))
                acc = part if acc is None else acc + part
            want = oracle.gram(xs, dims, n)
            scale = np.abs(want).max() * math.log2(x.size)
            assert np.abs(acc - want).max() <= tol * scale, (prec, n)
            assert np.abs(acc - full).max() <= tol * scale, (prec, n)


MIXED_GRAM_SHAPES = [(64, 300), (128, 2000), (500, 700), (256, 33, 7), (132, 100), (1024, 90),
                     (96, 64)]


@pytest.mark.parametrize("dims", MIXED_GRAM_SHAPES)
def test_gram_tensor_mode0_tensor_cores(ctx, dims):
    """Mode-0 Gram on tcgen05 (two-term FP16 split, all four products).  The
    split represents each value to 2^-22 relative and the tensor-core FP32
    accumulator truncates, which scales S by (1 - c) with c ~ 1e-5 at most
    (proportional: harmless to the rank cut); so S matches the oracle to
    3e-5 relative per entry scale sqrt(S_ii S_jj)."""
    rng = np.random.default_rng(dims[0] + dims[1])
    x = rng.standard_normal(oracle.linear_size(dims)) * rng.uniform(0.5, 2.0, dims[0]).repeat(1)[
        np.arange(oracle.linear_size(dims)) % dims[0]]
    t = dev(x, torch.float32)
    xs = host(t)
    want = oracle.gram(xs, dims, 0)
    got = host(ctx.gram(t, dims, 0, "tensor"))
    d = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    assert np.all(np.abs(got - want) <= 3e-5 * d + 1e-30), np.max(np.abs(got - want) / d)
    assert np.array_equal(got, got.T)


def test_gram_tensor_error_on_discarded_subspace(ctx):
    """What the eps cut sees: the Gram's error projected on the discarded
    eigenvectors.  The tensor-core accumulator truncates toward zero; part
    of that bias is a uniform shrink of S (harmless: it scales the tail),
    the rest projects on the discarded subspace.  That remainder must stay
    far below the eps = 1e-2 threshold (the regime TENSOR is meant for); at
    eps = 1e-4 it is of the order of 100 thresholds, which is why MIXED
    keeps the FP32 round-to-nearest Gram."""
    dims = (256, 64, 40, 11)
    x = synth.tucker_torch(dims, (40, 20, 20, 11), decay=0.1, eta=1e-7, seed=3)
    want = oracle.gram(host(x), dims, 0)
    got = host(ctx.gram(x, dims, 0, "tensor"))
    w, V = oracle.eig_desc(want)
    nrm2 = float(np.trace(want))
    thr = 1e-4 * nrm2 / 4                         # eps = 1e-2, N = 4
    R, tail = oracle.rank_cut(w, thr)
    P = V[:, R:]
    E = got - want
    c = -np.trace(E) / nrm2                       # uniform shrink factor
    proj = np.trace(P.T @ (E + c * want) @ P)     # what remains on the tail
    assert 0 <= c < 3e-5, c
    assert abs(proj) <= 0.05 * thr, (proj / thr, c)


MIXED_X3_SHAPES = [(128, 3000), (500, 2000), (256, 33, 70), (132, 700), (1024, 300), (2048, 64),
                   (500, 257), (64, 3000), (100, 650), (2080, 300), (4096, 70),
                   (130, 700), (250, 333), (66, 2000), (2050, 70)]


@pytest.fixture
def digits(ctx, request):
    """Forces the exact-digit Gram's digit count for one test."""
    from paper_1901_06043_gb300 import tucker
    ctx.set_option(tucker.OPT_GRAM_DIGITS, request.param)
    yield request.param
    ctx.set_option(tucker.OPT_GRAM_DIGITS, 0)


def _digit_delta(X, digits):
    """Half the last digit's unit per row: 2^(floor(log2 max_k |x_ik|) - 20)
    with three 7-bit digits, 2^(... - 13) with two."""
    _, ex = np.frexp(X.max(axis=1))
    return np.where(X.max(axis=1) > 0, np.ldexp(1.0, ex - (21 if digits == 3 else 14)), 0.0)


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
@pytest.mark.parametrize("dims", MIXED_X3_SHAPES)
def test_gram_mixed_mode0_exact_digits(ctx, dims, digits):
    """Mode-0 Gram of MIXED precision: tensor cores on exact integer digit
    products (three or two 7-bit digits of each value under a per-row
    power-of-two scale; window sums below 2^24 are exact in the FP32
    accumulator).  Rows of very different magnitude (10^-3 .. 10^3), one
    zero row, a few exact zeros and a ragged K.  The only error is the digit
    representation, |x - digits| <= delta_i = 2^(floor(log2 max_k |x_ik|) -
    20) (three digits) or 2^(... - 13) (two), so every entry lies within
    delta_j |x_i|_1 + delta_i |x_j|_1 + K delta_i delta_j of the oracle's
    FP64 Gram (plus 1e-12 of sum_k |x_ik x_jk| for the compensated sums)."""
    rng = np.random.default_rng(dims[0] * 7 + dims[-1])
    n = oracle.linear_size(dims)
    rows = np.arange(n) % dims[0]
    rs = 10.0 ** rng.uniform(-3, 3, dims[0])
    rs[dims[0] // 3] = 0.0
    x = rng.standard_normal(n) * rs[rows]
    x[rng.integers(0, n, size=n // 50)] = 0.0
    t = dev(x, torch.float32)
    xs = host(t)
    want = oracle.gram(xs, dims, 0)
    got = host(ctx.gram(t, dims, 0, "mixed"))
    X = np.abs(xs.reshape(-1, dims[0]).T)          # I x K, |x|
    K = X.shape[1]
    delta = _digit_delta(X, digits)
    l1 = X.sum(axis=1)
    bound = (np.outer(l1, delta) + np.outer(delta, l1) + K * np.outer(delta, delta)
             + 1e-12 * (X @ X.T))
    err = np.abs(got - want)
    assert np.all(err <= bound + 1e-300), np.nanmax(err / bound)
    # the bound is not loose by orders of magnitude: rounding errors show
    assert np.nanmax(err / np.where(bound > 0, bound, np.inf)) > 1e-4
    assert np.array_equal(got, got.T)


def _digit_err6(X, thr, digits):
    """Six standard deviations of the digit representation's error on the
    discarded subspace of the I x K matrix X (numpy), the bound the library
    chooses its digit count by: sqrt(4 sigma_max^2 thr + 2 K sigma_max^2
    sum_i sigma_i^2) with sigma_i^2 = delta_i^2 / 3."""
    d = _digit_delta(np.abs(X), digits)
    s2max, s2sum = d.max() ** 2 / 3.0, float((d * d).sum()) / 3.0
    return 6.0 * math.sqrt(4.0 * s2max * thr + 2.0 * X.shape[1] * s2max * s2sum)


def _digit_trace_sigma(X, digits=3):
    """Standard deviation of the trace error of the exact-digit Gram for the
    I x K matrix X (torch, any device): the last digit rounds each value to
    the grid 2^(floor(log2 max_k |x_ik|) - 19) (three digits; - 12 with two),
    a remainder r within +-half a step, independent of the digits; with the
    diagonal correction trace(S~) - trace(S) = -2 sum x r, whose mean
    -2 sum E[r^2] is ~1e-3 of this spread at these sizes."""
    rmax = X.abs().amax(dim=1).double().cpu().numpy()
    rn2 = (X.double() ** 2).sum(dim=1).cpu().numpy()
    _, ex = np.frexp(rmax)
    half = np.where(rmax > 0, np.ldexp(1.0, ex - (21 if digits == 3 else 14)), 0.0)
    return float(np.sqrt(np.sum(4.0 * half ** 2 / 3.0 * rn2)))


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
def test_gram_mixed_mode0_trace_unbiased(ctx, digits):
    """trace(S) = ||Y||^2 on 1.3e8 Gaussian entries: the exact-digit
    tensor-core Gram rounds only unbiasedly (the last digit of each value;
    its square is removed from the diagonal), so its trace matches the FP64
    sum of squares within 6 sigma of that rounding noise (3e-10 here; a
    truncating accumulator is off by ~1e-6)."""
    dims = (256, 64, 8000)
    g = torch.Generator(device="cuda").manual_seed(77)
    t = torch.randn(dims[::-1], generator=g, device="cuda", dtype=torch.float32).reshape(-1)
    want = float((t.double() ** 2).sum())
    got = float(torch.trace(ctx.gram(t, dims, 0, "mixed")))
    sigma = _digit_trace_sigma(t.view(-1, dims[0]).T, digits)
    assert sigma < (1e-9 if digits == 3 else 2e-7) * want
    assert abs(got - want) <= 6 * sigma, ((got - want) / want, (got - want) / sigma)


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
def test_gram_mixed_mode0_error_on_discarded_subspace(ctx, digits):
    """What the eps cut sees, at eps = 1e-4 (the regime MIXED is meant for):
    the exact-digit Gram's error projected on the discarded eigenvectors of a
    Tucker tensor's mode-0 Gram stays below 2 % of the threshold.  The trace
    error itself lies in the kept subspace and is the digit rounding noise:
    within 6 sigma of it."""
    dims = (256, 64, 40, 11)
    x = synth.tucker_torch(dims, (40, 20, 20, 11), decay=0.1, eta=1e-7, seed=3)
    want = oracle.gram(host(x), dims, 0)
    got = host(ctx.gram(x, dims, 0, "mixed"))
    w, V = oracle.eig_desc(want)
    nrm2 = float(np.trace(want))
    thr = 1e-8 * nrm2 / 4                         # eps = 1e-4, N = 4
    R, tail = oracle.rank_cut(w, thr)
    P = V[:, R:]
    E = got - want
    proj = np.trace(P.T @ E @ P)
    sigma = _digit_trace_sigma(x.view(-1, dims[0]).T, digits)
    assert abs(np.trace(E)) <= 6 * sigma, np.trace(E) / sigma
    # within 2 % of the threshold with three digits; with two, within the six
    # standard deviations of the bound the library chooses its digits by
    bound = 0.02 * thr if digits == 3 else _digit_err6(host(x).reshape(-1, dims[0]).T, thr, 2)
    assert abs(proj) <= bound, (proj / thr, bound / thr)


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
def test_gram_mixed_discarded_sum_of_a_low_rank_tensor(ctx, digits):
    """Where the small eigenvalues sit far below the digits' resolution (rank
    40 plus 1e-7 noise, 256 x 720896 mode-0 view), the exact-digit Gram's
    error on the oracle's discarded subspace stays within the six standard
    deviations of its representation error (the library's digit bound with
    the tail sum in place of the threshold).  A systematic error on the
    diagonal of 1 % of sum_k r_ik^2 breaks it (measured before each diagonal
    entry's D3 was summed exactly), and so would the squared remainders
    left on the diagonal (100 times that)."""
    dims = (256, 128, 128, 11, 4)
    x = synth.tucker_torch(dims, (40, 40, 40, 11, 4), decay=0.1, eta=1e-7, seed=6)
    X = host(x).reshape(-1, dims[0]).T
    want = oracle.gram(host(x), dims, 0)
    got = host(ctx.gram(x, dims, 0, "mixed"))
    w, V = oracle.eig_desc(want)
    R = 40
    tail = float(w[R:].sum())
    P = V[:, R:]
    proj = float(np.trace(P.T @ (got - want) @ P))
    bound = _digit_err6(X, tail, digits)
    assert abs(proj) <= bound, (proj, bound, tail)


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_mixed_digit_count_follows_its_bound(ctx, eps):
    """An eps-driven MIXED ST-HOSVD takes two digits for the mode-0 view when
    six standard deviations of the two-digit representation error on the
    discarded subspace stay below 1 % of the threshold, else three: checked
    against the bound computed here from the view's row maxima, on a
    256 x 64 x 200 x 11 tensor at three eps.  Ranks and discarded sums as the
    oracle's."""
    dims = (256, 64, 200, 11)
    x = synth.tucker_torch(dims, (40, 20, 30, 11), decay=0.1, eta=1e-7, seed=4)
    res = ctx.sthosvd(x, dims, eps=eps, prec="mixed")
    ref = oracle.sthosvd(host(x), dims, eps=eps)
    two = _digit_err6(host(x).reshape(-1, dims[0]).T, ref["threshold"], 2) <= 0.01 * ref["threshold"]
    assert res.gram_kernel[0] == ("tcgen05-x2" if two else "tcgen05-x3"), res.gram_kernel
    if eps == 1e-2:
        assert two
    assert res.ranks == ref["ranks"]
    for n in range(4):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"]
    res.close()


@pytest.mark.parametrize("eps,kernel", [(1e-4, "tcgen05-x3"), (1e-6, "simt-fp64")])
def test_mixed_digit_gram_kept_while_its_bound_allows(ctx, eps, kernel):
    """MIXED keeps the exact-digit Gram of a view while six standard
    deviations of its representation error on the discarded subspace,
    sqrt(4 sigma^2 thr + 2 K I sigma^4) with sigma^2 = delta_max^2 / 3, stay
    below 1 % of the threshold; this 256 x 28160 mode-0 view passes at
    eps = 1e-4 (~2 % of the allowance) and fails at eps = 1e-6, where the
    Gram is computed in FP64.  The mode-0 cut equals the oracle's either way;
    at eps = 1e-4 every mode's does (at eps = 1e-6 the later modes see the
    mixed TTMs' rounding, ~1e-14 ||X||^2, a few percent of that threshold)."""
    dims = (256, 64, 40, 11)
    x = synth.tucker_torch(dims, (40, 20, 20, 11), decay=0.1, eta=1e-7, seed=3)
    res = ctx.sthosvd(x, dims, eps=eps, prec="mixed")
    ref = oracle.sthosvd(host(x), dims, eps=eps)
    assert res.gram_kernel[0] == kernel, res.gram_kernel
    modes = range(4) if eps >= 1e-4 else range(1)
    for n in modes:
        assert res.ranks[n] == ref["ranks"][n]
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"]
    res.close()


def _tcx_applies(dims, mode):
    """Whether the exact-digit tensor-core Gram serves this slab view (the
    plan's rule: I <= 4096; column mode needs 64 <= I and >= 64 columns;
    row mode 16-l blocks with at most 25 % zero fill)."""
    L = math.prod(dims[:mode])
    I = dims[mode]
    Rt = math.prod(dims[mode + 1:])
    if not (64 if L == 1 else 128) <= I <= 4096:
        return False
    if L == 1:
        return Rt >= 64
    nlb = -(-L // 16)
    return 4 * nlb * 16 <= 5 * L and L * I < 2 ** 31 and Rt * nlb >= 4


def _unfold(x, dims, mode):
    """Mode-n unfolding (I_n x rest) of a flat natural-descending tensor."""
    N = len(dims)
    if isinstance(x, np.ndarray):
        return np.moveaxis(x.reshape(dims[::-1]), N - 1 - mode, 0).reshape(dims[mode], -1)
    return torch.movedim(x.view(dims[::-1]), N - 1 - mode, 0).reshape(dims[mode], -1)


ROW_X3_CASES = [((54, 300, 40), 1), ((60, 129, 11), 1), ((100, 500, 20), 1),
                ((12, 10, 200, 30), 2), ((16, 136, 9), 1)]


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
@pytest.mark.parametrize("dims,mode", ROW_X3_CASES)
def test_gram_mixed_rowmode_exact_digits(ctx, dims, mode, digits):
    """Row-mode slab views (L > 1: row i's values L apart, stages of 16
    consecutive l of one slab, the last block of a slab zero-filled) on the
    exact-digit tensor-core Gram, row maxima from the slab pass: every entry
    within the digit representation bound of the oracle's FP64 Gram, as for
    the mode-0 view.  Rows of magnitudes 10^-3 .. 10^3, one zero row, exact
    zeros, ragged I and L."""
    assert _tcx_applies(dims, mode)
    rng = np.random.default_rng(dims[mode] * 11 + mode)
    n = oracle.linear_size(dims)
    L = math.prod(dims[:mode])
    rows = (np.arange(n) // L) % dims[mode]
    rs = 10.0 ** rng.uniform(-3, 3, dims[mode])
    rs[dims[mode] // 3] = 0.0
    x = rng.standard_normal(n) * rs[rows]
    x[rng.integers(0, n, size=n // 50)] = 0.0
    t = dev(x, torch.float32)
    xs = host(t)
    want = oracle.gram(xs, dims, mode)
    got = host(ctx.gram(t, dims, mode, "mixed"))
    X = np.abs(_unfold(xs, dims, mode))
    K = X.shape[1]
    delta = _digit_delta(X, digits)
    l1 = X.sum(axis=1)
    bound = (np.outer(l1, delta) + np.outer(delta, l1) + K * np.outer(delta, delta)
             + 1e-12 * (X @ X.T))
    err = np.abs(got - want)
    assert np.all(err <= bound + 1e-300), np.nanmax(err / bound)
    assert np.nanmax(err / np.where(bound > 0, bound, np.inf)) > 1e-4
    assert np.array_equal(got, got.T)


@pytest.mark.parametrize("digits", [3, 2], indirect=True)
def test_gram_mixed_rowmode_error_on_discarded_subspace(ctx, digits):
    """Mode 1 (row mode, L = 64) of a Tucker tensor at eps = 1e-4: the
    exact-digit Gram's error on the discarded eigenvectors stays below 2 % of
    the threshold and its trace error within 6 sigma of the digit rounding
    noise."""
    dims = (64, 256, 40, 11)
    assert _tcx_applies(dims, 1)
    x = synth.tucker_torch(dims, (20, 40, 20, 11), decay=0.1, eta=1e-7, seed=5)
    want = oracle.gram(host(x), dims, 1)
    got = host(ctx.gram(x, dims, 1, "mixed"))
    w, V = oracle.eig_desc(want)
    nrm2 = float(np.trace(want))
    thr = 1e-8 * nrm2 / 4
    R, tail = oracle.rank_cut(w, thr)
    P = V[:, R:]
    E = got - want
    proj = np.trace(P.T @ E @ P)
    sigma = _digit_trace_sigma(_unfold(x, dims, 1), digits)
    assert abs(np.trace(E)) <= 6 * sigma, np.trace(E) / sigma
    assert abs(proj) <= 0.02 * thr, proj / thr


# ---------------------------------------------------------------- eigen

def _spd(n, seed, spectrum=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    if spectrum is None:
        spectrum = np.abs(rng.standard_normal(n)) * 10.0 ** -rng.uniform(0, 8, n)
    return (Q * spectrum) @ Q.T


EIG_CASES = [
    ("one", np.array([[3.0]])),
    ("two", np.array([[2.0, 1.0], [1.0, 2.0]])),
    ("diag", np.diag([5.0, 1.0, 3.0, 0.0, 2.0])),
    ("spd65", _spd(65, 1)),
    ("spd64", _spd(64, 2)),
    ("spd200", _spd(200, 3)),
    ("spd257_odd", _spd(257, 4)),
    ("rankdef", _spd(50, 5, np.r_[np.linspace(10, 1, 10), np.zeros(40)])),
    ("repeated", _spd(40, 6, np.r_[np.full(20, 2.0), np.full(20, 1.0)])),
    ("gram", None),
]


@pytest.mark.parametrize("name,S", EIG_CASES, ids=[c[0] for c in EIG_CASES])
def test_eig_fp64(ctx, name, S):
    if S is None:
        x, _ = synth.tucker_numpy((60, 40, 30), (6, 5, 4), decay=0.2, eta=1e-4, seed=7)
        S = oracle.gram(x, (60, 40, 30), 0)
    S = (S + S.T) / 2
    w_ref, V_ref = oracle.eig_desc(S)
    w, V, sweeps = ctx.eig(dev(S))
    w, V = host(w), host(V)
    lmax = max(abs(w_ref).max(), 1e-300)
    assert np.abs(w - w_ref).max() <= 1e-10 * lmax
    assert np.abs(w - w_ref).max() <= 1e-13 * np.linalg.norm(S) * S.shape[0]
    assert np.all(np.diff(w) <= 0)
    n = S.shape[0]
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(S @ V - V * w).max() <= 1e-13 * np.linalg.norm(S) * n
    # individual vectors where the eigenvalue is isolated
    gaps = np.minimum(np.r_[np.inf, -np.diff(w_ref)], np.r_[-np.diff(w_ref), np.inf])
    for k in range(n):
        if gaps[k] > 1e-3 * lmax:
            assert abs(abs(V[:, k] @ V_ref[:, k]) - 1) <= 1e-12


def _graded(n, seed, decay=0.16, noise=1e-14):
    """A Tucker-like Gram: eigenvalues 10^(-decay i) down to a noise floor
    of nearly equal values, random eigenvectors."""
    rng = np.random.default_rng(seed)
    lam = np.maximum(10.0 ** (-decay * np.arange(n)), noise * rng.uniform(0.5, 1.5, n))
    return _spd(n, seed, lam)


TRUNC_CASES = EIG_CASES + [
    ("graded100", _graded(100, 21)),
    ("graded500", _graded(500, 22, decay=0.03)),
    ("graded300_steep", _graded(300, 23, decay=0.3)),
]


@pytest.fixture
def solver(ctx, request):
    from paper_1901_06043_gb300.tucker import EIG_SOLVER, OPT_EIG_SOLVER
    ctx.set_option(OPT_EIG_SOLVER, EIG_SOLVER[request.param])
    yield request.param
    ctx.set_option(OPT_EIG_SOLVER, 0)


@pytest.mark.parametrize("solver", ["tridiag", "jacobi"], indirect=True)
@pytest.mark.parametrize("name,S", TRUNC_CASES, ids=[c[0] for c in TRUNC_CASES])
@pytest.mark.parametrize("cut", ["thr", "fixed"])
def test_eig_trunc_fp64(ctx, solver, name, S, cut):
    """Eigenvalues, rank cut and leading eigenvectors (Section 5.2, Eq. Un)
    of both solvers against the oracle's eigendecomposition."""
    if S is None:
        x, _ = synth.tucker_numpy((60, 40, 30), (6, 5, 4), decay=0.2, eta=1e-4, seed=7)
        S = oracle.gram(x, (60, 40, 30), 0)
    S = (S + S.T) / 2
    n = S.shape[0]
    w_ref, V_ref = oracle.eig_desc(S)
    lmax = max(abs(w_ref).max(), 1e-300)
    if cut == "thr":
        thr = 1e-7 * abs(w_ref).sum()
        R_ref, tail = oracle.rank_cut(w_ref, thr)
        fixed = 0
    else:
        fixed = max(1, n // 3)
        thr, R_ref = 0.0, fixed
    w, U, R, disc = ctx.eig_trunc(dev(S), thr=thr, R=fixed)
    w, U = host(w), host(U)
    assert np.abs(w - w_ref).max() <= 1e-10 * lmax
    assert np.abs(w - w_ref).max() <= 1e-13 * np.linalg.norm(S) * n
    assert np.all(np.diff(w) <= 0)
    if cut == "thr":
        # the computed eigenvalues decide; where the oracle's tail is within
        # rounding of thr either rank is valid
        R_own, tail_own = oracle.rank_cut(w, thr)
        assert R == R_own
        if abs(tail[R_ref] - thr) > 1e-12 * lmax * n and abs(tail[R_ref - 1] - thr) > 1e-12 * lmax * n:
            assert R == R_ref
    else:
        assert R == fixed
    assert U.shape == (n, R)
    assert np.abs(U.T @ U - np.eye(R)).max() <= 1e-13 * n
    assert np.abs(S @ U - U * w[:R]).max() <= 1e-13 * np.linalg.norm(S) * n
    if R < n and (w_ref[R - 1] - w_ref[R]) > 1e-6 * lmax:
        assert sin_angle(V_ref[:, :R], U) <= 1e-8


@pytest.mark.parametrize("n", [1500, 2080])
def test_eig_trunc_jicf_sized(ctx, n):
    """The truncated eigensolve (tridiagonal solver: all eigenvalues, the R
    leading vectors) at the mode sizes of the JICF dataset (1500 and 2080,
    the paper's largest modes, where it notes the eigensolve becomes
    visible) on a graded Tucker-like spectrum, against the oracle; the time
    of one solve is printed."""
    import time
    S = _graded(n, 31 + n, decay=0.02)
    S = (S + S.T) / 2
    w_ref, V_ref = oracle.eig_desc(S)
    lmax = abs(w_ref).max()
    thr = 1e-8 * abs(w_ref).sum()
    R_ref, tail = oracle.rank_cut(w_ref, thr)
    Sd = dev(S)
    ctx.eig_trunc(Sd, thr=thr)                   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w, U, R, disc = ctx.eig_trunc(Sd, thr=thr)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    print(f"eig_trunc n={n}: R={R}, {ms:.1f} ms")
    w, U = host(w), host(U)
    assert np.abs(w - w_ref).max() <= 1e-10 * lmax
    assert R == R_ref
    assert abs(disc - tail[R]) <= 1e-12 * lmax * n
    assert np.abs(U.T @ U - np.eye(R)).max() <= 1e-13 * n
    assert np.abs(S @ U - U * w[:R]).max() <= 1e-13 * np.linalg.norm(S) * n
    if (w_ref[R - 1] - w_ref[R]) > 1e-6 * lmax:
        assert sin_angle(V_ref[:, :R], U) <= 1e-8


@pytest.mark.parametrize("solver", ["tridiag", "jacobi"], indirect=True)
def test_sthosvd_both_eigensolvers(ctx, solver):
    dims = (120, 100, 80)
    x, _ = synth.tucker_numpy(dims, (12, 10, 8), decay=0.12, eta=1e-6, seed=12)
    ref = oracle.sthosvd(x, dims, eps=1e-4)
    res = ctx.sthosvd(dev(x), dims, eps=1e-4, prec="fp64")
    assert res.eig_kernel == ["tridiag" if solver == "tridiag" else "jacobi"] * 3
    _check_against_oracle(x, dims, res, ref)


def _batch_shapes(count, seed):
    """Uneven 3-way cubes and 4-way tensors, the shape mix of the batched
    workload at a size the oracle finishes quickly."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if k % 2 == 0:
            a = int(rng.integers(20, 72))
            dims = (a, a, a)
        else:
            dims = tuple(int(v) for v in rng.integers(12, 40, size=3)) + (int(rng.integers(4, 9)),)
        core = tuple(min(d, int(rng.integers(3, 9))) for d in dims)
        out.append((dims, core))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sthosvd_batched_uneven(ctx, prec):
    """Every tensor of an uneven batch against the oracle's ST-HOSVD of it
    (Algorithm 1), and against the single-tensor entry point."""
    shapes = _batch_shapes(9, 5)
    xs, dims_list = [], []
    for k, (dims, core) in enumerate(shapes):
        x, _ = synth.tucker_numpy(dims, core, decay=0.2, eta=1e-6, seed=40 + k)
        xs.append(dev(x, torch.float64 if prec == "fp64" else torch.float32))
        dims_list.append(dims)
    res = ctx.sthosvd_batched(xs, dims_list, eps=1e-4, prec=prec)
    assert len(res) == len(xs)
    for t, dims, r in zip(xs, dims_list, res):
        xh = host(t)
        ref = oracle.sthosvd(xh, dims, eps=1e-4)
        assert r.eig_kernel == ["tridiag"] * len(dims)
        if prec == "fp64":
            _check_against_oracle(xh, dims, r, ref)
        else:
            assert r.ranks == ref["ranks"]
            e_ours = oracle.relative_errors(xh, dims, {"core": host(r.core), "core_dims": r.ranks,
                                                       "factors": [host(f) for f in r.factors],
                                                       "discarded": r.discarded,
                                                       "norm_sq": r.norm_sq})
            assert e_ours["err_explicit"] <= 1e-4
        one = ctx.sthosvd(t, dims, eps=1e-4, prec=prec)
        assert one.ranks == r.ranks
        one.close()
        r.close()


def test_sthosvd_batched_mixed_digit_grams(ctx):
    """Sides of 128-256 (multiples of 4), where the batched MIXED path runs
    the exact-digit tensor-core Gram with its side-stream row maxima: every
    tensor against the oracle (identical ranks, discarded sums within 2 % of
    the threshold, explicit error within eps)."""
    shapes = [((128, 128, 128), (20, 20, 20)), ((132, 140, 24, 6), (16, 12, 10, 4)),
              ((200, 200, 60), (24, 24, 16)), ((256, 136, 20, 5), (30, 20, 10, 5)),
              ((160, 160, 160), (12, 30, 20))]
    xs, dims_list = [], []
    for k, (dims, core) in enumerate(shapes):
        x, _ = synth.tucker_numpy(dims, core, decay=0.15, eta=1e-6, seed=70 + k)
        xs.append(dev(x, torch.float32))
        dims_list.append(dims)
    res = ctx.sthosvd_batched(xs, dims_list, eps=1e-4, prec="mixed")
    for t, dims, r in zip(xs, dims_list, res):
        xh = host(t)
        ref = oracle.sthosvd(xh, dims, eps=1e-4)
        assert r.gram_kernel[0] == "tcgen05-x3", r.gram_kernel
        assert r.ranks == ref["ranks"], (dims, r.ranks, ref["ranks"])
        for n in range(len(dims)):
            assert abs(r.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"]
        e = oracle.relative_errors(xh, dims, {"core": host(r.core), "core_dims": r.ranks,
                                              "factors": [host(f) for f in r.factors],
                                              "discarded": r.discarded, "norm_sq": r.norm_sq})
        assert e["err_explicit"] <= 1e-4
        r.close()


def test_sthosvd_batched_rejects_bad_input(ctx):
    from paper_1901_06043_gb300.tucker import TuckerError
    x = dev(np.ones(8))
    with pytest.raises(TuckerError):
        ctx.sthosvd_batched([x], [(2, 0, 4)], eps=1e-3)
    with pytest.raises(TuckerError) as e:
        ctx.sthosvd_batched([dev(np.ones(5000))], [(5000,)], eps=1e-3)   # mode above 4096
    assert e.value.name == "INVALID"
    with pytest.raises(TypeError):   # the binding checks the common dtype
        ctx.sthosvd_batched([x, dev(np.ones(8), torch.float32)], [(2, 2, 2), (2, 2, 2)], eps=1e-3)


def test_eig_sweep_cap_zero_reports_noconv(ctx):
    from paper_1901_06043_gb300.tucker import OPT_MAX_SWEEPS, TuckerError
    ctx.set_option(OPT_MAX_SWEEPS, 0)
    try:
        with pytest.raises(TuckerError) as e:
            ctx.eig(dev(_spd(10, 9)))
        assert e.value.name == "EIG_NOCONV"
    finally:
        ctx.set_option(OPT_MAX_SWEEPS, 40)


# ------------------------------------------------------------- rank cut

def test_rank_cut_cases(ctx):
    cases = [([4, 2, 1, 0.5], 1.5), ([4, 2, 1, 0.5], 1.49), ([3, 1, 0, 0], 0.0),
             ([3, 1, -1e-18], 0.0), ([3, 1, 1], 100.0), ([3, 2, 1], 0.0)]
    rng = np.random.default_rng(11)
    for _ in range(20):
        w = np.sort(rng.exponential(size=rng.integers(1, 300)))[::-1] * 10.0 ** rng.uniform(-5, 5)
        cases.append((w, float(rng.uniform(0, 1) * w.sum())))
    for w, thr in cases:
        R, tail = oracle.rank_cut(w, thr)
        gR, gd = ctx.rank_cut(dev(np.asarray(w, float)), thr)
        assert gR == R
        assert gd == tail[R] or abs(gd - tail[R]) <= 1e-15 * abs(tail[0])


# ------------------------------------------------------------------- TTM

TTM_SHAPES = [((7,), 3), ((130, 3), 5), ((3, 130), 70), ((65, 9, 4), 2), ((5, 64, 3), 64),
              ((4, 3, 70), 1), ((33, 1, 17, 2), 9), ((2, 3, 2, 3, 2), 4), ((200, 300), 130)]


@pytest.mark.parametrize("dims,K", TTM_SHAPES)
def test_ttm_fp64(ctx, dims, K):
    rng = np.random.default_rng(K + len(dims))
    x = rng.standard_normal(oracle.linear_size(dims))
    t = dev(x)
    for n in range(len(dims)):
        A = rng.standard_normal((K, dims[n]))
        want = oracle.ttm(x, dims, n, A)
        got = host(ctx.ttm(t, dims, n, dev(A), "fp64"))
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max() * dims[n], (dims, n)
        # column-major A (a transposed view)
        Ac = dev(np.asfortranarray(A)).t().contiguous().t()
        got = host(ctx.ttm(t, dims, n, Ac, "fp64"))
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max() * dims[n], (dims, n)


@pytest.mark.parametrize("dims,K", TTM_SHAPES)
def test_ttm_fp32(ctx, dims, K):
    rng = np.random.default_rng(K + 2 * len(dims))
    x = rng.standard_normal(oracle.linear_size(dims))
    t = dev(x, torch.float32)
    xs = host(t)
    for n in range(len(dims)):
        A = rng.standard_normal((K, dims[n]))
        want = oracle.ttm(xs, dims, n, A)
        got = host(ctx.ttm(t, dims, n, dev(A), "fp32"))
        # FP32 factor and products: ~2^-24 relative per term, dims[n] terms
        assert np.abs(got - want).max() <= 2e-7 * np.abs(A).max() * np.abs(xs).max() * dims[n]


TC_TTM_SHAPES = [((256, 300), 54), ((500, 1000), 128), ((64, 7, 3), 1), ((68, 513), 100),
                 ((200, 160, 9), 30)]


@pytest.mark.parametrize("dims,K", TC_TTM_SHAPES)
def test_ttm_mixed_tensor_cores_mode0(ctx, dims, K):
    """Mode-0 TTM on tcgen05 (two-term FP16 split of Y and A, products
    hh + hl + lh, truncating FP32 accumulator).  Error per output is bounded
    by the split residuals (3 x 2^-22) plus one truncation per accumulation
    step (<= 2^-23 of the running |sum| per MMA, ~100 steps at I = 500), i.e.
    <= 2e-5 of sum_i |a_ki| |y_i|; checked elementwise against that bound.
    Row-major and column-major A, a ragged last slab tile (Rt % 256 != 0) and
    a partial last 64-wide stage of I are covered."""
    rng = np.random.default_rng(K + 5 * len(dims))
    x = rng.standard_normal(oracle.linear_size(dims))
    t = dev(x, torch.float32)
    xs = host(t)
    A = rng.standard_normal((K, dims[0]))
    want = oracle.ttm(xs, dims, 0, A)
    bound = 2e-5 * oracle.ttm(np.abs(xs), dims, 0, np.abs(A))
    got = host(ctx.ttm(t, dims, 0, dev(A), "mixed"))
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)
    Ac = dev(np.asfortranarray(A)).t().contiguous().t()
    got = host(ctx.ttm(t, dims, 0, Ac, "mixed"))
    assert np.all(np.abs(got - want) <= bound)


TC_ROW_TTM_CASES = [((128, 54, 11), 1, 500), ((20, 40, 7), 1, 300), ((252, 13, 5), 1, 70),
                    ((4, 64, 9), 1, 1000), ((132, 7, 3, 5), 2, 40), ((8, 3, 600), 1, 17)]


@pytest.mark.parametrize("dims,n,K", TC_ROW_TTM_CASES)
def test_ttm_mixed_tensor_cores_rowmode(ctx, dims, n, K):
    """Row-mode TTM on tcgen05 (L = prod dims[:n] with L % 4 == 0, I <= 64:
    the reconstruction's expansions), l as the MMA's M, one or more N-tiles
    of 256 outputs, the same two-term FP16 split and three products as the
    mode-0 kernel: every output within 2e-5 of sum_i |a_ki| |y_i| of the
    oracle's TTM.  Ragged L and I, K above 256, both layouts of A."""
    L = math.prod(dims[:n])
    assert L % 4 == 0 and dims[n] <= 64
    rng = np.random.default_rng(K + 7 * n)
    x = rng.standard_normal(oracle.linear_size(dims))
    t = dev(x, torch.float32)
    xs = host(t)
    A = rng.standard_normal((K, dims[n]))
    want = oracle.ttm(xs, dims, n, A)
    bound = 2e-5 * oracle.ttm(np.abs(xs), dims, n, np.abs(A))
    got = host(ctx.ttm(t, dims, n, dev(A), "mixed"))
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)
    Ac = dev(np.asfortranarray(A)).t().contiguous().t()
    got = host(ctx.ttm(t, dims, n, Ac, "mixed"))
    assert np.all(np.abs(got - want) <= bound)


def test_reconstruct_mixed_tensor_cores(ctx):
    """Multi-TTM reconstruction in MIXED precision (tensor-core TTMs for the
    row-mode expansions) against the oracle: within 1e-4 of the same
    multi-TTM applied to absolute values (four chained TTMs, each within
    2e-5 of its absolute sums)."""
    dims = (64, 48, 40, 6)
    x = synth.tucker_torch(dims, (20, 16, 12, 4), decay=0.05, eta=1e-6, seed=4)
    res32 = ctx.sthosvd(x, dims, eps=1e-3, prec="mixed")
    b, e = (0, 0, 0, 0), (64, 48, 40, 5)
    got = host(res32.reconstruct(b, e, prec="mixed"))
    want32, _ = oracle.reconstruct(host(res32.core), res32.ranks,
                                   [host(f) for f in res32.factors], b, e)
    abs32, _ = oracle.reconstruct(np.abs(host(res32.core)), res32.ranks,
                                  [np.abs(host(f)) for f in res32.factors], b, e)
    assert np.all(np.abs(got - want32) <= 1e-4 * abs32), np.max(np.abs(got - want32) / abs32)


# --------------------------------------------------------- whole ST-HOSVD

def _check_against_oracle(x, dims, res, ref, err_tol=1e-12, eig_tol=1e-10, angle_tol=1e-8,
                          est2_tol=None):
    assert res.ranks == ref["ranks"]
    for n in range(len(dims)):
        lam = host(res.eigvals[n])
        lmax = abs(ref["eigvals"][n]).max()
        assert np.abs(lam - ref["eigvals"][n]).max() <= eig_tol * lmax
        U = host(res.factors[n])
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-12
        w = ref["eigvals"][n]
        R = ref["ranks"][n]
        gap = (w[R - 1] - (w[R] if R < len(w) else 0.0)) / lmax
        if gap > 1e-6:
            assert sin_angle(ref["factors"][n], U) <= angle_tol, (n, gap)
    core = host(res.core)
    ours = {"core": core, "core_dims": res.ranks, "factors": [host(f) for f in res.factors],
            "discarded": res.discarded, "norm_sq": res.norm_sq}
    e_ours = oracle.relative_errors(x, dims, ours)
    e_ref = oracle.relative_errors(x, dims, ref)
    assert abs(e_ours["err_explicit"] - e_ref["err_explicit"]) <= err_tol
    # Corollary 1's estimate is sqrt(discarded / ||X||^2): compared squared,
    # since each discarded eigenvalue carries an absolute error ~eps_64 ||S||
    # (<= eps_64 ||X||^2) on each side (backward-stable solvers, Grams summed
    # in different orders) and the sqrt amplifies it by 1 / (2 err) at small
    # errors: the bound is 2 eps_64 per discarded eigenvalue, at least 1e-14.
    if est2_tol is None:
        ndisc = sum(d - r for d, r in zip(dims, ref["ranks"]))
        est2_tol = max(1e-14, 2.2e-16 * ndisc)
    assert abs(e_ours["err_est"] ** 2 - e_ref["err_est"] ** 2) <= est2_tol
    assert abs(res.norm_sq - ref["norm_sq"]) <= 1e-13 * ref["norm_sq"]


def test_sthosvd_40x50x30_fp64(ctx):
    dims = (40, 50, 30)
    x, _ = synth.tucker_numpy(dims, (5, 6, 4), eta=1e-4, seed=0)
    ref = oracle.sthosvd(x, dims, eps=1e-3)
    res = ctx.sthosvd(dev(x), dims, eps=1e-3, prec="fp64")
    assert res.ranks == (5, 6, 4)
    _check_against_oracle(x, dims, res, ref)
    # full reconstruction by the multi-TTM, against the oracle's multi-TTM of
    # the same core and factors
    full = host(res.reconstruct())
    want, _ = oracle.reconstruct(host(res.core), res.ranks, [host(f) for f in res.factors])
    assert np.abs(full - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("case", [
    dict(dims=(12, 10, 8, 6), core=(4, 3, 3, 2), decay=0.1, eta=1e-3, eps=1e-2),
    dict(dims=(9, 8, 7, 6, 5), core=(3, 3, 3, 2, 2), decay=0.2, eta=1e-3, eps=1e-2),
    dict(dims=(30, 20), core=(6, 5), decay=0.3, eta=1e-3, eps=1e-2),
    dict(dims=(257,), core=(1,), decay=0.0, eta=0.0, eps=1e-3),
    dict(dims=(1, 40, 1, 30), core=(1, 5, 1, 4), decay=0.0, eta=1e-4, eps=1e-3),
    dict(dims=(65, 33, 17), core=(10, 8, 6), decay=0.1, eta=1e-5, eps=1e-4),
])
def test_sthosvd_shapes_fp64(ctx, case):
    dims = case["dims"]
    x, _ = synth.tucker_numpy(dims, case["core"], decay=case["decay"], eta=case["eta"], seed=3)
    ref = oracle.sthosvd(x, dims, eps=case["eps"])
    res = ctx.sthosvd(dev(x), dims, eps=case["eps"], prec="fp64")
    _check_against_oracle(x, dims, res, ref)


def test_sthosvd_rank_specified_and_mode_order(ctx):
    dims = (20, 16, 12)
    x, _ = synth.tucker_numpy(dims, (6, 5, 4), decay=0.2, eta=1e-3, seed=4)
    ref = oracle.sthosvd(x, dims, ranks=(4, 3, 2))
    res = ctx.sthosvd(dev(x), dims, ranks=(4, 3, 2), prec="fp64")
    _check_against_oracle(x, dims, res, ref)
    ref = oracle.sthosvd(x, dims, eps=1e-2, mode_order=(2, 0, 1))
    res = ctx.sthosvd(dev(x), dims, eps=1e-2, mode_order=(2, 0, 1), prec="fp64")
    assert res.mode_order == (2, 0, 1)
    _check_against_oracle(x, dims, res, ref)


def test_sthosvd_fp32_input_fp64_path(ctx):
    dims = (48, 40, 36)
    x, _ = synth.tucker_numpy(dims, (8, 7, 6), decay=0.15, eta=1e-4, seed=5)
    t = dev(x, torch.float32)
    xs = host(t)
    ref = oracle.sthosvd(xs, dims, eps=1e-3)
    res = ctx.sthosvd(t, dims, eps=1e-3, prec="fp64")
    _check_against_oracle(xs, dims, res, ref)


def test_sthosvd_fp32_path_ranks_and_error(ctx):
    """FP32 products: identical ranks (the cut margins here are wide) and an
    error within 1e-6 of the oracle's."""
    dims = (48, 40, 36)
    x, _ = synth.tucker_numpy(dims, (8, 7, 6), decay=0.15, eta=1e-4, seed=5)
    t = dev(x, torch.float32)
    xs = host(t)
    ref = oracle.sthosvd(xs, dims, eps=1e-3)
    res = ctx.sthosvd(t, dims, eps=1e-3, prec="fp32")
    assert res.ranks == ref["ranks"]
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e1 = oracle.relative_errors(xs, dims, ours)["err_explicit"]
    e0 = oracle.relative_errors(xs, dims, ref)["err_explicit"]
    assert abs(e1 - e0) <= 1e-6


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_sthosvd_mixed_path_ranks_and_error(ctx, eps):
    """MIXED (Grams with 128 <= I_n <= 4096 on exact-digit tensor-core
    products, others FP32 or FP64; tensor-core mode-0 TTM): ranks identical to the
    FP64 oracle on a decaying-spectrum FP32 tensor; error within 5e-6 of the
    oracle's."""
    dims = (200, 160, 48, 11)
    x = synth.tucker_torch(dims, (30, 30, 24, 11), decay=0.1, eta=1e-7, seed=9)
    xs = host(x)
    ref = oracle.sthosvd(xs, dims, eps=eps)
    res = ctx.sthosvd(x, dims, eps=eps, prec="mixed")
    digit = ("tcgen05-x3", "tcgen05-x2")
    assert res.gram_kernel[0] in digit
    assert res.ttm_kernel[0] == "tcgen05"
    # natural mode order: the working tensor is kept rotated (each TTM writes
    # its new mode last), so mode 1 is a column-mode view (I = 160) and both
    # its Gram and its TTM run on the tensor cores
    assert res.gram_kernel[1] in digit and res.ttm_kernel[1] == "tcgen05"
    assert res.ranks == ref["ranks"]
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e1 = oracle.relative_errors(xs, dims, ours)["err_explicit"]
    e0 = oracle.relative_errors(xs, dims, ref)["err_explicit"]
    # FP32 TTMs round each core entry to ~u32 sqrt(I_n) ~ 1e-6 relative
    assert abs(e1 - e0) <= 5e-6 and e1 <= eps


def test_sthosvd_tensor_path_at_eps_1e2(ctx):
    """TENSOR (tcgen05 mode-0 Gram) at eps = 1e-2: ranks identical to the
    oracle, error within 1e-6 of the oracle's."""
    dims = (200, 160, 48, 11)
    x = synth.tucker_torch(dims, (30, 30, 24, 11), decay=0.1, eta=1e-7, seed=9)
    xs = host(x)
    ref = oracle.sthosvd(xs, dims, eps=1e-2)
    res = ctx.sthosvd(x, dims, eps=1e-2, prec="tensor")
    assert res.gram_kernel[0] == "tcgen05"
    assert res.ranks == ref["ranks"]
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e1 = oracle.relative_errors(xs, dims, ours)["err_explicit"]
    e0 = oracle.relative_errors(xs, dims, ref)["err_explicit"]
    assert abs(e1 - e0) <= 1e-6 and e1 <= 1e-2


def test_bad_arguments_are_rejected(ctx):
    from paper_1901_06043_gb300.tucker import TuckerError
    t = dev(np.ones(24))
    for kw in [dict(eps=-1.0), dict(ranks=(0, 2, 2)), dict(ranks=(3, 5, 2)),
               dict(eps=1e-2, mode_order=(0, 0, 1))]:
        with pytest.raises(TuckerError) as e:
            ctx.sthosvd(t, (2, 3, 4), **kw)
        assert e.value.name == "INVALID"
    for prec in ("mixed", "tensor"):
        with pytest.raises(TuckerError) as e:
            ctx.sthosvd(t, (2, 3, 4), eps=1e-2, prec=prec)
        assert e.value.name == "UNSUPPORTED"


# -------------------------------------------------------- reconstruction

def test_partial_reconstruction_and_order_independence(ctx):
    dims = (20, 18, 16, 6)
    x, _ = synth.tucker_numpy(dims, (5, 4, 4, 3), eta=1e-3, seed=6)
    res = ctx.sthosvd(dev(x), dims, eps=1e-2, prec="fp64")
    core, F = host(res.core), [host(f) for f in res.factors]
    b, e = (3, 0, 15, 2), (17, 18, 16, 3)
    want, wd = oracle.reconstruct(core, res.ranks, F, b, e)
    for order in itertools.permutations(range(4)):
        got = host(res.reconstruct(b, e, order))
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), order
    got = host(res.reconstruct(b, e))   # library-chosen order
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_multi_ttm_general_operators(ctx):
    """Section 7's operators folded into the factors: averaging pairs
    (downsampling), one-hot selection and all-ones summaries."""
    rng = np.random.default_rng(12)
    cd = (4, 5, 3)
    g = rng.standard_normal(oracle.linear_size(cd))
    U = [np.linalg.qr(rng.standard_normal((I, R)))[0] for I, R in zip((10, 12, 7), cd)]
    C0 = np.zeros((10, 5)); C0[np.arange(10), np.arange(10) // 2] = 0.5
    C1 = np.zeros((12, 1)); C1[7, 0] = 1.0
    C2 = np.ones((7, 1))
    mats = [C0.T @ U[0], C1.T @ U[1], C2.T @ U[2]]
    want, od = oracle.multi_ttm(g, cd, mats)
    got = host(ctx.multi_ttm(dev(g), cd, [dev(m) for m in mats], od, prec="fp64"))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sthosvd_at_jicf_mode_sizes(ctx, prec):
    """A whole ST-HOSVD with two modes of the JICF sizes (1500 and 2080, Tab. 7)
    against the oracle: the tridiagonal eigensolver inside Algorithm 1 at
    those sizes, the exact-digit Gram of a 1500-row view (78 tiles) and of a
    2080-row one (153 tiles, more than one wave; MIXED), and the TTMs at
    rank 40.  FP64: the usual tolerances; MIXED: identical ranks, discarded
    sums within 2 % of the threshold, the explicit error below eps and within
    3e-5 of the oracle's (measured 1.7e-5 against 1.0e-6: the TTMs' rounding
    over contractions of 1500 and 2080 terms)."""
    dims = (1500, 2080, 4)
    x, _ = synth.tucker_numpy(dims, (40, 40, 4), decay=0.05, eta=1e-6, seed=21)
    ref = oracle.sthosvd(x, dims, eps=1e-4)
    if prec == "fp64":
        res = ctx.sthosvd(dev(x), dims, eps=1e-4, prec="fp64")
        assert res.eig_kernel[:2] == ["tridiag", "tridiag"]
        _check_against_oracle(x, dims, res, ref)
        return
    x32 = x.astype(np.float32)
    ref = oracle.sthosvd(x32.astype(np.float64), dims, eps=1e-4)
    res = ctx.sthosvd(dev(x32, torch.float32), dims, eps=1e-4, prec="mixed")
    assert all(k in ("tcgen05-x3", "tcgen05-x2") for k in res.gram_kernel[:2]), res.gram_kernel
    assert res.ranks == ref["ranks"], (res.ranks, ref["ranks"])
    for n in range(3):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"], n
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e_ours = oracle.relative_errors(x32.astype(np.float64), dims, ours)["err_explicit"]
    e_ref = oracle.relative_errors(x32.astype(np.float64), dims, ref)["err_explicit"]
    # eps is met; the tensor-core TTMs (FP16 split products, truncating FP32
    # accumulators over contractions of 1500 and 2080) add ~1e-5 relative
    assert e_ours <= 1e-4 and abs(e_ours - e_ref) <= 3e-5, (e_ours, e_ref)


def test_sthosvd_mixed_rows_not_a_multiple_of_four(ctx):
    """MIXED with mode sizes that are not multiples of 4 (130 and 98): the
    exact-digit Gram reads such column views with 4-byte loads and takes its
    row maxima from the same norm pass.  Ranks identical to the oracle's and
    every discarded sum within 2 % of the threshold."""
    dims = (130, 98, 50, 7)
    x, _ = synth.tucker_numpy(dims, (20, 15, 10, 7), decay=0.1, eta=1e-6, seed=31)
    x32 = x.astype(np.float32)
    ref = oracle.sthosvd(x32.astype(np.float64), dims, eps=1e-4)
    res = ctx.sthosvd(dev(x32, torch.float32), dims, eps=1e-4, prec="mixed")
    assert all(k in ("tcgen05-x3", "tcgen05-x2") for k in res.gram_kernel[:2]), res.gram_kernel
    assert res.ranks == ref["ranks"], (res.ranks, ref["ranks"])
    for n in range(4):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"], n
    res.close()
