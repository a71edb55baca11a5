"""Pins of the oracle's chunked ST-HOSVD, HOSVD, ST-HOSVD mode order and
pre-/post-processing against what the paper and the mathematics fix.

- chunked ST-HOSVD: the same result as the in-memory one (Algorithm 2's
  sum over block columns and Algorithm 3's column-wise TTM taken piece by
  piece), including empty pieces;
- HOSVD (Section 3.2): factors span the leading left singular vectors of
  X's own unfoldings (brute-force SVD), Theorem 1's error bound, the
  truncated SVD for N = 2, agreement with ST-HOSVD on a superdiagonal core;
- mode order (Section 6 costs): the flop count equals the paper's closed
  form for the natural order, the exhaustive search agrees with an
  independent exchange-argument rule, and hand cases;
- Section 3.5: statistics of explicit unfolding rows computed with numpy's
  own routines, standardized slices with mean 0 and variance 1,
  max-rescaled slices within [-1, 1] touching 1, inverse after forward is
  the identity, hand values.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth


# ------------------------------------------------------- chunked ST-HOSVD

@pytest.mark.parametrize("dims,nchunks", [((6, 5, 4, 7), 3), ((9, 8, 5), 5), ((7, 6, 3), 4),
                                          ((5, 4), 2), ((8, 6, 2), 1)])
@pytest.mark.parametrize("spec", ["eps", "ranks"])
def test_chunked_sthosvd_equals_in_memory(dims, nchunks, spec):
    x, _ = synth.tucker_numpy(dims, tuple(max(1, d // 2) for d in dims), decay=0.1, eta=1e-3,
                              seed=sum(dims))
    kw = {"eps": 1e-2} if spec == "eps" else {"ranks": tuple(max(1, d // 2) for d in dims)}
    ref = oracle.sthosvd(x, dims, **kw)
    xt = x.reshape(dims[-1], -1)                  # last mode slowest

    def chunk(c):
        a = dims[-1] * c // nchunks
        b = dims[-1] * (c + 1) // nchunks
        return xt[a:b].reshape(-1)

    got = oracle.sthosvd_chunked(chunk, nchunks, dims, **kw)
    assert got["ranks"] == ref["ranks"]
    assert math.isclose(got["norm_sq"], ref["norm_sq"], rel_tol=1e-13)
    for n in range(len(dims)):
        assert np.allclose(got["eigvals"][n], ref["eigvals"][n], rtol=0,
                           atol=1e-12 * abs(ref["eigvals"][n][0]))
        s = np.linalg.svd(got["factors"][n].T @ ref["factors"][n], compute_uv=False)
        assert np.all(s > 1 - 1e-9)
    e1 = oracle.relative_errors(x, dims, got)["err_explicit"]
    e0 = oracle.relative_errors(x, dims, ref)["err_explicit"]
    assert abs(e1 - e0) < 1e-12


def test_chunked_sthosvd_with_more_pieces_than_last_indices():
    dims = (6, 5, 3)
    x, _ = synth.tucker_numpy(dims, (3, 3, 2), eta=1e-3, seed=2)
    xt = x.reshape(dims[-1], -1)
    got = oracle.sthosvd_chunked(lambda c: xt[3 * c // 7:3 * (c + 1) // 7].reshape(-1), 7, dims,
                                 eps=1e-2)
    ref = oracle.sthosvd(x, dims, eps=1e-2)
    assert got["ranks"] == ref["ranks"]
    assert np.allclose(got["core"] ** 2, ref["core"] ** 2, atol=1e-12 * ref["norm_sq"])


# ------------------------------------------------------------------ HOSVD

@pytest.mark.parametrize("dims", [(7, 6, 5), (5, 4, 3, 4), (4, 3, 3, 2, 3)])
def test_hosvd_factors_are_leading_singular_vectors_of_x_unfoldings(dims):
    rng = np.random.default_rng(sum(dims))
    x = rng.standard_normal(oracle.linear_size(dims)) + 3 * synth.tucker_numpy(
        dims, tuple(max(1, d - 2) for d in dims), seed=1)[0]
    res = oracle.hosvd(x, dims, eps=0.3)
    for n in range(len(dims)):
        Xn = oracle.unfold(x, dims, n)
        Ul, s, _ = np.linalg.svd(Xn)
        lam = np.zeros(dims[n]); lam[:s.shape[0]] = s ** 2
        assert np.allclose(res["eigvals"][n], lam, rtol=0, atol=1e-12 * lam[0])
        R = res["ranks"][n]
        assert R == next(r for r in range(1, dims[n] + 1)
                         if lam[r:].sum() <= 0.09 * np.dot(x, x) / len(dims))
        if R < dims[n] and lam[R - 1] - lam[R] > 1e-6 * lam[0]:
            cos = np.linalg.svd(res["factors"][n].T @ Ul[:, :R], compute_uv=False)
            assert np.all(cos > 1 - 1e-10)
    # the core is X x_n U_n^T in every mode, built from explicit unfoldings
    y, cur = x.copy(), list(dims)
    for n in range(len(dims)):
        U = res["factors"][n]
        Yn = oracle.unfold(y, cur, n)
        cur[n] = U.shape[1]
        y = oracle.fold(U.T @ Yn, cur, n)
    assert np.allclose(y, res["core"], atol=1e-12 * math.sqrt(np.dot(x, x)))


@pytest.mark.parametrize("eps", [0.3, 0.1, 1e-2])
def test_hosvd_error_bound_theorem_1(eps):
    dims = (12, 10, 9, 6)
    x, _ = synth.tucker_numpy(dims, (6, 5, 4, 3), decay=0.1, eta=3e-2, seed=6)
    res = oracle.hosvd(x, dims, eps=eps)
    err = oracle.relative_errors(x, dims, res)
    nrm2 = res["norm_sq"]
    # (rounding-level slack for the case with nothing discarded)
    assert err["err_explicit"] ** 2 * nrm2 <= sum(res["discarded"]) * (1 + 1e-12) + 1e-26 * nrm2
    assert sum(res["ranks"]) < sum(dims) or eps == 1e-2
    assert err["err_explicit"] <= eps * (1 + 1e-12)
    # Section 3: ||X - Xhat||^2 = ||X||^2 - ||G||^2 for orthonormal factors
    assert abs(err["err_gram"] - err["err_explicit"]) < 1e-6


def test_hosvd_two_way_is_truncated_svd():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 6)) @ np.diag(2.0 ** -np.arange(6)) @ rng.standard_normal((6, 15))
    A += 1e-3 * rng.standard_normal(A.shape)
    x = A.reshape(-1, order="F")
    res = oracle.hosvd(x, (20, 15), ranks=(4, 4))
    U, s, Vt = np.linalg.svd(A)
    xhat, _ = oracle.reconstruct(res["core"], res["core_dims"], res["factors"])
    assert np.allclose(xhat.reshape(20, 15, order="F"), (U[:, :4] * s[:4]) @ Vt[:4], atol=1e-12)


def test_hosvd_equals_sthosvd_on_a_superdiagonal_core():
    sig = [10.0, 6.0, 3.0, 1.5, 0.7]
    dims = (9, 8, 7)
    x, _ = synth.tucker_numpy(dims, (5, 5, 5), superdiag=sig, seed=4)
    a = oracle.hosvd(x, dims, eps=0.05)
    b = oracle.sthosvd(x, dims, eps=0.05)
    assert a["ranks"] == b["ranks"]
    ea = oracle.relative_errors(x, dims, a)["err_explicit"]
    eb = oracle.relative_errors(x, dims, b)["err_explicit"]
    assert abs(ea - eb) < 1e-12


def test_hosvd_differs_from_sthosvd_on_generic_data():
    # HOSVD takes every factor from X itself; ST-HOSVD's later modes see the
    # partial core, whose eigenvalues are smaller
    dims = (8, 7, 6)
    x = np.random.default_rng(5).standard_normal(oracle.linear_size(dims))
    a = oracle.hosvd(x, dims, ranks=(3, 3, 3))
    b = oracle.sthosvd(x, dims, ranks=(3, 3, 3))
    assert np.allclose(a["eigvals"][0], b["eigvals"][0], atol=1e-12 * a["eigvals"][0][0])
    assert a["eigvals"][2].sum() > 1.5 * b["eigvals"][2].sum()


# -------------------------------------------------------------- mode order

def _paper_natural_order_flops(dims, ranks):
    """Section 6's per-mode counts for the increasing mode order, one
    processor: Gram (prod_{k<n} R_k) I_n^2 (prod_{k>n} I_k), eigensolve
    (10/3) I_n^3, TTM 2 (prod_{k<n} R_k) R_n I_n (prod_{k>n} I_k)."""
    total = 0.0
    for n in range(len(dims)):
        left = math.prod(ranks[:n])
        right = math.prod(dims[n + 1:])
        total += left * dims[n] ** 2 * right + 10.0 / 3.0 * dims[n] ** 3 \
            + 2.0 * left * ranks[n] * dims[n] * right
    return total


@pytest.mark.parametrize("dims,ranks", [((500, 500, 500, 11, 8), (54, 54, 54, 11, 6)),
                                        ((7, 5, 9), (2, 5, 3)), ((10,), (4,))])
def test_sthosvd_flops_match_the_cost_analysis(dims, ranks):
    got = oracle.sthosvd_flops(dims, ranks, range(len(dims)))
    assert math.isclose(got, _paper_natural_order_flops(dims, ranks), rel_tol=1e-12)
    # relabelling the modes gives another order's count
    for perm in itertools.permutations(range(len(dims))):
        d2 = [dims[p] for p in perm]
        r2 = [ranks[p] for p in perm]
        assert math.isclose(oracle.sthosvd_flops(dims, ranks, perm),
                            _paper_natural_order_flops(d2, r2), rel_tol=1e-12)
        if len(dims) > 3:
            break


def test_best_order_agrees_with_the_exchange_rule():
    rng = np.random.default_rng(11)
    for _ in range(200):
        N = int(rng.integers(2, 6))
        dims = [int(v) for v in rng.integers(2, 60, size=N)]
        ranks = [int(rng.integers(1, d + 1)) for d in dims]
        best, cost = oracle.best_sthosvd_order(dims, ranks)
        rule = oracle.sthosvd_order_ratio_rule(dims, ranks)
        assert math.isclose(oracle.sthosvd_flops(dims, ranks, rule), cost, rel_tol=1e-12), (
            dims, ranks, best, rule)
        for perm in itertools.permutations(range(N)):
            assert oracle.sthosvd_flops(dims, ranks, perm) >= cost * (1 - 1e-12)


def test_order_hand_cases():
    # a mode that collapses to rank 1 goes first; modes that do not shrink last
    assert oracle.best_sthosvd_order((100, 100, 100), (100, 1, 100))[0][0] == 1
    assert oracle.best_sthosvd_order((50, 50, 50), (50, 50, 50))[0] == (0, 1, 2)
    # the Large workload's estimated ranks: the species mode (no shrink) last
    order, _ = oracle.best_sthosvd_order((500, 500, 500, 11, 8), (54, 54, 54, 11, 6))
    assert order[-1] == 3


# ------------------------------------------------ pre-/post-processing (3.5)

@pytest.mark.parametrize("dims,n", [((4, 5, 3), 0), ((4, 5, 3), 1), ((4, 5, 3), 2),
                                    ((3, 4, 3, 2), 3), ((6,), 0)])
def test_slice_stats_are_the_row_statistics_of_the_unfolding(dims, n):
    rng = np.random.default_rng(len(dims) * 10 + n)
    x = rng.standard_normal(oracle.linear_size(dims)) * 3 + 1.5
    st = oracle.slice_stats(x, dims, n)
    Xn = oracle.unfold(x, dims, n)
    assert np.allclose(st[:, 0], Xn.mean(axis=1), rtol=0, atol=1e-14)
    assert np.allclose(st[:, 1], Xn.std(axis=1, ddof=0), rtol=1e-13)
    assert np.array_equal(st[:, 2], Xn.max(axis=1))
    assert np.array_equal(st[:, 3], Xn.min(axis=1))
    assert np.allclose(st[:, 4], np.linalg.norm(Xn, ord=1, axis=1), rtol=1e-14)
    assert np.allclose(st[:, 5], np.linalg.norm(Xn, axis=1), rtol=1e-14)


def test_slice_stats_hand_values():
    # 2 x 3 tensor, natural-descending: x(i, j) at i + 2 j
    x = np.array([1.0, -2.0, 3.0, -4.0, 5.0, 6.0])
    st = oracle.slice_stats(x, (2, 3), 0)       # slices i = 0: {1, 3, 5}; i = 1: {-2, -4, 6}
    assert np.allclose(st[0], [3.0, math.sqrt(8 / 3), 5.0, 1.0, 9.0, math.sqrt(35.0)])
    assert np.allclose(st[1], [0.0, math.sqrt(56 / 3), 6.0, -4.0, 12.0, math.sqrt(56.0)])


@pytest.mark.parametrize("n", [0, 1, 2])
def test_standardization_and_its_inverse(n):
    dims = (5, 6, 4)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(oracle.linear_size(dims)) * 10 ** rng.uniform(-2, 2) + 7.0
    sh, sc = oracle.standardize_params(oracle.slice_stats(x, dims, n))
    y = oracle.slice_transform(x, dims, n, sh, sc)
    st = oracle.slice_stats(y, dims, n)
    assert np.allclose(st[:, 0], 0.0, atol=1e-13)
    assert np.allclose(st[:, 1], 1.0, rtol=1e-13)
    back = oracle.slice_transform(y, dims, n, sh, sc, inverse=True)
    assert np.allclose(back, x, rtol=1e-14, atol=1e-13 * np.abs(x).max())


@pytest.mark.parametrize("n", [0, 1, 2])
def test_max_rescaling_and_its_inverse(n):
    dims = (5, 6, 4)
    rng = np.random.default_rng(10 + n)
    x = rng.standard_normal(oracle.linear_size(dims)) * 10 ** rng.uniform(-3, 3, dims[n])[
        oracle.tucker_fp64._all_indices(dims)[:, n]]
    sh, sc = oracle.max_rescale_params(oracle.slice_stats(x, dims, n))
    assert np.all(sh == 0.0)
    y = oracle.slice_transform(x, dims, n, sh, sc)
    st = oracle.slice_stats(y, dims, n)
    assert np.allclose(np.maximum(np.abs(st[:, 2]), np.abs(st[:, 3])), 1.0, rtol=1e-15)
    back = oracle.slice_transform(y, dims, n, sh, sc, inverse=True)
    assert np.allclose(back, x, rtol=1e-14, atol=0)


def test_constant_and_zero_slices_keep_scale_one():
    dims = (3, 4)
    x = np.zeros(12)
    x[1::3] = 2.5                                 # slice 1 constant, slices 0 and 2 zero
    st = oracle.slice_stats(x, dims, 0)
    sh, sc = oracle.standardize_params(st)
    assert np.array_equal(sc, [1.0, 1.0, 1.0]) and np.array_equal(sh, [0.0, 2.5, 0.0])
    sh2, sc2 = oracle.max_rescale_params(st)
    assert np.array_equal(sc2, [1.0, 0.4, 1.0])
