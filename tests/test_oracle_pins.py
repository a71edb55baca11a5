"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
worked layout example printed in Section 4.2, closed forms (superdiagonal
cores), textbook routines (the SVD for N = 2 and for explicit unfoldings),
exact recovery of noiseless low-rank tensors, the error identities of
Section 3 / Corollary 1, and the mode-order facts of Section 8.5.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "unfold_3x4x3x2.txt")


def _read_golden():
    mats, cur, rows = {}, None, []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("mode"):
                if cur is not None:
                    mats[cur] = np.array(rows, dtype=np.int64)
                _, n, _, _ = line.split()
                cur, rows = int(n), []
            else:
                rows.append([int(v) for v in line.split()])
    mats[cur] = np.array(rows, dtype=np.int64)
    return mats


# ------------------------------------------------------------------ layout

def test_worked_example_unfoldings_exact():
    """Section 4.2: the four printed unfoldings of the 3x4x3x2 tensor whose
    entries are their linear indices (Fig. 1)."""
    dims = (3, 4, 3, 2)
    y = np.arange(72, dtype=np.int64)
    gold = _read_golden()
    for n in range(4):
        assert np.array_equal(oracle.unfold(y, dims, n), gold[n]), n
        # the same matrix as J^>_n row-major J_n x J^<_n submatrices side by side
        sl = oracle.slab_view(y, dims, n)
        assert sl.shape == (oracle.right_size(dims, n), dims[n], oracle.left_size(dims, n))
        assert np.array_equal(np.concatenate(list(sl), axis=1), gold[n]), n


def test_linear_index_labels_of_fig1():
    dims = (3, 4, 3, 2)
    assert oracle.idx2lin((1, 0, 0, 0), dims) == 1
    assert oracle.idx2lin((0, 1, 0, 0), dims) == 3
    assert oracle.idx2lin((0, 0, 1, 0), dims) == 12
    assert oracle.idx2lin((0, 0, 0, 1), dims) == 36
    assert oracle.idx2lin((2, 3, 2, 1), dims) == 71
    for j in range(72):
        assert oracle.idx2lin(oracle.lin2idx(j, dims), dims) == j


def test_sizes_and_edge_cases():
    dims = (3, 4, 3, 2)
    assert oracle.linear_size(dims) == 72
    assert [oracle.left_size(dims, n) for n in range(4)] == [1, 3, 12, 36]
    assert [oracle.right_size(dims, n) for n in range(4)] == [24, 6, 2, 1]
    assert [oracle.unfold_size(dims, n) for n in range(4)] == [24, 18, 24, 36]


def test_fold_inverts_unfold():
    dims = (2, 3, 4, 5)
    y = np.random.default_rng(1).standard_normal(120)
    for n in range(4):
        assert np.array_equal(oracle.fold(oracle.unfold(y, dims, n), dims, n), y)


# ------------------------------------------------------------- Gram and TTM

@pytest.mark.parametrize("dims", [(7,), (5, 6), (4, 3, 5), (3, 1, 4, 2), (2, 3, 2, 3, 2)])
def test_gram_equals_explicit_unfolding_product(dims):
    """Algorithm 2's slab loop against S = Y_(n) Y_(n)^T of the explicit
    unfolding (index map of Section 2.2.1); trace(S) = ||Y||^2."""
    y = np.random.default_rng(2).standard_normal(oracle.linear_size(dims))
    for n in range(len(dims)):
        Yn = oracle.unfold(y, dims, n)
        S = oracle.gram(y, dims, n)
        assert np.allclose(S, Yn @ Yn.T, rtol=0, atol=1e-12 * np.abs(Yn).max() ** 2 * Yn.shape[1])
        assert np.array_equal(S, S.T) or np.allclose(S, S.T, atol=1e-13)
        assert math.isclose(np.trace(S), oracle.norm_sq(y), rel_tol=1e-13)


@pytest.mark.parametrize("dims", [(5, 6), (4, 3, 5), (3, 1, 4, 2), (2, 3, 2, 3, 2)])
def test_ttm_definition_and_identities(dims):
    """Section 2.2.3: Y = X x_n U <=> Y_(n) = U X_(n); modes commute; same-mode
    products compose (Eq. same_mode)."""
    rng = np.random.default_rng(3)
    y = rng.standard_normal(oracle.linear_size(dims))
    for n in range(len(dims)):
        U = rng.standard_normal((4, dims[n]))
        z = oracle.ttm(y, dims, n, U)
        zd = list(dims); zd[n] = 4
        assert np.allclose(oracle.unfold(z, zd, n), U @ oracle.unfold(y, dims, n), atol=1e-12)
        V = rng.standard_normal((3, 4))
        zz = oracle.ttm(z, zd, n, V)
        zd2 = list(dims); zd2[n] = 3
        assert np.allclose(zz, oracle.ttm(y, dims, n, V @ U), atol=1e-11)
    if len(dims) >= 2:
        A = rng.standard_normal((2, dims[0]))
        B = rng.standard_normal((3, dims[1]))
        d1 = list(dims); d1[0] = 2
        d2 = list(dims); d2[1] = 3
        ab = oracle.ttm(oracle.ttm(y, dims, 0, A), d1, 1, B)
        ba = oracle.ttm(oracle.ttm(y, dims, 1, B), d2, 0, A)
        assert np.allclose(ab, ba, atol=1e-12)


# ---------------------------------------------------------------- rank cut

def test_rank_cut_hand_cases():
    """Eq. Un with the inclusive '<=' and R in {1..I}."""
    assert oracle.rank_cut([4, 2, 1, 0.5], 1.5)[0] == 2      # tail(2) = 1.5 <= 1.5
    assert oracle.rank_cut([4, 2, 1, 0.5], 1.49)[0] == 3
    assert oracle.rank_cut([3, 1, 0, 0], 0.0)[0] == 2
    assert oracle.rank_cut([3, 1, -1e-18], 0.0)[0] == 2       # signed tail -1e-18 <= 0
    assert oracle.rank_cut([3, 1, 1e-18, -2e-18], 0.0)[0] == 2  # tail(2) = -1e-18
    R, tail = oracle.rank_cut([3, 1, 1e-18, -2e-18], 0.0)
    assert tail[3] == -2e-18
    assert oracle.rank_cut([3, 1, 1], 100.0)[0] == 1          # never 0
    assert oracle.rank_cut([3, 2, 1], 0.0)[0] == 3            # R = I allowed
    R, tail = oracle.rank_cut([4, 2, 1, 0.5], 0.0)
    assert list(tail) == [7.5, 3.5, 1.5, 0.5, 0.0]


# ------------------------------------------------------ closed-form spectra

def _superdiag_expected(sig, dims, eps):
    """Closed form for a superdiagonal core with orthonormal factors: every
    mode-n Gram of the partial core has eigenvalues sigma_k^2 over the
    components still kept (plus zeros); the cut follows Eq. Un."""
    N = len(dims)
    s2 = sorted([float(s) ** 2 for s in sig], reverse=True)
    nrm2 = sum(s2)
    thr = eps ** 2 * nrm2 / N
    active, ranks, disc, eigs = list(s2), [], [], []
    for n in range(N):
        lam = active + [0.0] * (dims[n] - len(active))
        eigs.append(lam)
        R = next(R for R in range(1, dims[n] + 1) if sum(lam[R:]) <= thr)
        ranks.append(R)
        disc.append(sum(lam[R:]))
        active = active[:R]
    return ranks, disc, eigs, nrm2


@pytest.mark.parametrize("eps", [0.3, 0.05, 1e-3])
def test_superdiagonal_core_closed_form(eps):
    sig = [10.0, 6.0, 3.0, 1.5, 0.7, 0.2]
    dims = (9, 8, 7)
    x, _ = synth.tucker_numpy(dims, (6, 6, 6), superdiag=sig, seed=4)
    res = oracle.sthosvd(x, dims, eps=eps)
    ranks, disc, eigs, nrm2 = _superdiag_expected(sig, dims, eps)
    assert res["ranks"] == tuple(ranks)
    assert math.isclose(res["norm_sq"], nrm2, rel_tol=1e-13)
    for n in range(3):
        assert np.allclose(res["eigvals"][n], eigs[n], rtol=0, atol=1e-12 * nrm2)
        assert math.isclose(res["discarded"][n], disc[n], rel_tol=1e-9, abs_tol=1e-12 * nrm2)
    err = oracle.relative_errors(x, dims, res)
    want = math.sqrt(sum(disc) / nrm2)
    # compared squared: sqrt() turns rounding-level discarded mass (~1e-16)
    # into ~1e-8 when nothing is discarded
    assert abs(err["err_explicit"] ** 2 - want ** 2) < 1e-13
    assert abs(err["err_est"] ** 2 - want ** 2) < 1e-13


# ------------------------------------------------------------ whole method

def test_noiseless_low_rank_exact_recovery():
    dims, core = (10, 12, 9, 7), (3, 4, 2, 5)
    x, parts = synth.tucker_numpy(dims, core, seed=5)
    res = oracle.sthosvd(x, dims, eps=1e-6)
    assert res["ranks"] == core
    err = oracle.relative_errors(x, dims, res)
    assert err["err_explicit"] < 1e-13
    for n in range(4):
        U = res["factors"][n]
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
        # same column space as the generating factor
        s = np.linalg.svd(U.T @ parts["factors"][n], compute_uv=False)
        assert np.all(s > 1 - 1e-12)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_error_identities_and_bound(eps):
    """Corollary 1: ||X - Xhat||^2 = sum of discarded eigenvalues; Section 3:
    = ||X||^2 - ||G||^2; Algorithm 1's guarantee ||X - Xhat|| <= eps ||X||."""
    dims = (14, 11, 9, 6)
    x, _ = synth.tucker_numpy(dims, (6, 5, 4, 3), decay=0.1, eta=1e-2, seed=6)
    res = oracle.sthosvd(x, dims, eps=eps)
    err = oracle.relative_errors(x, dims, res)
    assert abs(err["err_est"] - err["err_explicit"]) < 1e-12
    assert abs(err["err_gram"] - err["err_explicit"]) < 1e-6
    assert err["err_explicit"] <= eps * (1 + 1e-12)
    for n, U in enumerate(res["factors"]):
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)


def test_config_40x50x30_expected_ranks():
    """40x50x30 Tucker(5x6x4) + 1e-4 relative noise, seed 0, eps = 1e-3."""
    x, _ = synth.tucker_numpy((40, 50, 30), (5, 6, 4), eta=1e-4, seed=0)
    res = oracle.sthosvd(x, (40, 50, 30), eps=1e-3)
    assert res["ranks"] == (5, 6, 4)
    err = oracle.relative_errors(x, (40, 50, 30), res)
    assert err["err_explicit"] <= 1e-3


def test_two_way_is_truncated_svd():
    """N = 2: ST-HOSVD of a matrix is the truncated SVD (Eckart-Young)."""
    rng = np.random.default_rng(7)
    m, n = 30, 20
    A = rng.standard_normal((m, 8)) @ np.diag(2.0 ** -np.arange(8)) @ rng.standard_normal((8, n))
    A += 1e-3 * rng.standard_normal((m, n))
    x = A.reshape(-1, order="F")
    sv = np.linalg.svd(A, compute_uv=False)
    eps = 0.05
    res = oracle.sthosvd(x, (m, n), eps=eps)
    lam0 = res["eigvals"][0]
    assert np.allclose(lam0[:n], sv ** 2, rtol=0, atol=1e-12 * sv[0] ** 2)
    R = min(res["ranks"])
    xhat, _ = oracle.reconstruct(res["core"], res["core_dims"], res["factors"])
    U, s, Vt = np.linalg.svd(A)
    Ar = (U[:, :R] * s[:R]) @ Vt[:R]
    assert np.allclose(xhat.reshape(m, n, order="F"), Ar, atol=1e-12)
    err = oracle.relative_errors(x, (m, n), res)
    assert abs(err["err_explicit"] - math.sqrt(np.sum(sv[R:] ** 2)) / np.linalg.norm(sv)) < 1e-12


def test_mode0_factor_spans_leading_left_singular_vectors():
    dims = (12, 10, 8)
    x, _ = synth.tucker_numpy(dims, (4, 4, 4), decay=0.2, eta=1e-3, seed=8)
    res = oracle.sthosvd(x, dims, eps=1e-2)
    U0 = res["factors"][0]
    Ul, s, _ = np.linalg.svd(oracle.unfold(x, dims, 0))
    R = U0.shape[1]
    cos = np.linalg.svd(U0.T @ Ul[:, :R], compute_uv=False)
    assert np.all(cos > 1 - 1e-10)


@pytest.mark.parametrize("dims", [(2, 3, 4), (3, 4, 3, 2), (5, 4, 3, 2, 2)])
def test_bruteforce_svd_of_every_partial_core_unfolding(dims):
    """At each step the oracle's eigenvalues are the squared singular values
    of the explicit unfolding of the partial core, built here with
    unfold/fold only (no slab code)."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal(oracle.linear_size(dims))
    res = oracle.sthosvd(x, dims, eps=0.2)
    cur, y = list(dims), x.copy()
    for n in range(len(dims)):
        Yn = oracle.unfold(y, cur, n)
        s = np.linalg.svd(Yn, compute_uv=False)
        lam = np.zeros(cur[n]); lam[:s.shape[0]] = s ** 2
        assert np.allclose(res["eigvals"][n], lam, rtol=0, atol=1e-12 * lam[0])
        U = res["factors"][n]
        cur[n] = U.shape[1]
        y = oracle.fold(U.T @ Yn, cur, n)
    assert np.allclose(y, res["core"], atol=1e-12)


def test_rank_specified_variant():
    dims = (10, 9, 8)
    x, _ = synth.tucker_numpy(dims, (4, 4, 4), eta=1e-2, seed=10)
    res = oracle.sthosvd(x, dims, ranks=(3, 2, 4))
    assert res["core_dims"] == (3, 2, 4)
    err = oracle.relative_errors(x, dims, res)
    assert abs(err["err_est"] - err["err_explicit"]) < 1e-12


def test_mode_order_permutation():
    dims = (8, 9, 10)
    x, _ = synth.tucker_numpy(dims, (3, 4, 5), eta=1e-3, seed=11)
    res = oracle.sthosvd(x, dims, eps=1e-2, mode_order=(2, 0, 1))
    err = oracle.relative_errors(x, dims, res)
    assert err["err_explicit"] <= 1e-2
    assert abs(err["err_est"] - err["err_explicit"]) < 1e-12


# ------------------------------------------------------------- multi-TTM

def test_multittm_any_order_same_result():
    """Section 8.5: any ordering gives the same result up to rounding."""
    rng = np.random.default_rng(12)
    cd = (3, 4, 2, 3)
    g = rng.standard_normal(oracle.linear_size(cd))
    mats = [rng.standard_normal((k, r)) for k, r in zip((5, 2, 6, 1), cd)]
    ref, dims = oracle.multi_ttm(g, cd, mats)
    for perm in itertools.permutations(range(4)):
        z, d = oracle.multi_ttm(g, cd, mats, perm)
        assert d == dims
        assert np.allclose(z, ref, atol=1e-12)


def test_partial_reconstruction_is_a_slice():
    dims = (9, 8, 7)
    x, _ = synth.tucker_numpy(dims, (3, 3, 3), eta=1e-2, seed=13)
    res = oracle.sthosvd(x, dims, eps=1e-2)
    full, _ = oracle.reconstruct(res["core"], res["core_dims"], res["factors"])
    part, pd = oracle.reconstruct(res["core"], res["core_dims"], res["factors"],
                                  begin=(2, 0, 3), end=(7, 8, 4), mode_order=(2, 1, 0))
    F = full.reshape(dims, order="F")[2:7, 0:8, 3:4]
    assert pd == (5, 8, 1)
    assert np.allclose(part, F.reshape(-1, order="F"), atol=1e-12)


def _gb(words):
    return words * 8 / 1e9


def test_partial_reconstruction_intermediate_sizes_table():
    """Section 8.5 table of intermediate sizes (8-byte words), SP core
    30x38x35x6x11 -> 500x500x500x1x1, orders 01234 and 43120."""
    core, out = (30, 38, 35, 6, 11), (500, 500, 500, 1, 1)
    s = [_gb(w) for w in oracle.ttm_chain_sizes(core, out, (0, 1, 2, 3, 4))]
    assert [round(v, 2) for v in s] == [0.02, 0.35, 4.62, 66.0, 11.0, 1.0]
    s = [_gb(w) for w in oracle.ttm_chain_sizes(core, out, (4, 3, 1, 2, 0))]
    assert round(s[0], 2) == 0.02 and all(v < 0.01 for v in s[1:4])
    assert round(s[4], 2) == 0.06 and round(s[5], 2) == 1.0


@pytest.mark.parametrize("core", [(30, 38, 35, 6, 11), (95, 129, 125, 7, 125)])
def test_43120_unique_flop_minimiser(core):
    """Section 8.5: 43120 is the unique flop minimiser of the 500^3x1x1
    partial reconstruction for both compression scenarios; the pairwise
    comparator of Section 7 finds it too."""
    out = (500, 500, 500, 1, 1)
    best, cost = oracle.best_order(core, out, "flops")
    assert best == (4, 3, 1, 2, 0)
    others = [oracle.ttm_chain_flops(core, out, p) for p in itertools.permutations(range(5))
              if p != best]
    assert min(others) > cost
    assert oracle.order_flop_comparator(core, out) == (4, 3, 1, 2, 0)


def test_43120_is_a_memory_minimiser_high_compression():
    core, out = (30, 38, 35, 6, 11), (500, 500, 500, 1, 1)
    _, cost = oracle.best_order(core, out, "memory")
    s = oracle.ttm_chain_sizes(core, out, (4, 3, 1, 2, 0))
    assert max(s[i] + s[i + 1] for i in range(5)) == cost


def test_memory_comparator_matches_the_exhaustive_search():
    """Section 7: the optimal order is the one the exhaustive search over all
    N! permutations finds; the pairwise memory rule must reproduce it.  For
    every serial measure of temporary memory -- the largest input + output of
    one TTM, the largest intermediate, the sum of the intermediates -- the
    oracle's comparator (most-shrinking mode first, K_i/R_i ascending) attains
    the minimum on random cores and outputs, while the inequality as printed
    (R_i/K_i ascending, most-growing first) does not."""
    import random

    def pair(core, out, order):
        s = oracle.ttm_chain_sizes(core, out, order)
        return max(s[i] + s[i + 1] for i in range(len(order)))

    def peak(core, out, order):
        return max(oracle.ttm_chain_sizes(core, out, order))

    def total(core, out, order):
        return sum(oracle.ttm_chain_sizes(core, out, order)[1:])

    rng = random.Random(7)
    printed_optimal = 0
    for _ in range(200):
        N = rng.randint(2, 5)
        core = [rng.randint(2, 40) for _ in range(N)]
        out = [rng.randint(1, 80) for _ in range(N)]
        order = oracle.order_memory_comparator(core, out)
        assert sorted(order) == list(range(N))
        printed = tuple(sorted(range(N), key=lambda i: (core[i] / out[i], i)))
        for f in (pair, peak, total):
            best = min(f(core, out, p) for p in itertools.permutations(range(N)))
            assert f(core, out, order) == best, (core, out, f.__name__)
        printed_optimal += pair(core, out, printed) == min(
            pair(core, out, p) for p in itertools.permutations(range(N)))
    assert printed_optimal == 0
    # the library's memory objective (exhaustive) agrees with the comparator's cost
    core, out = (30, 38, 35, 6, 11), (500, 500, 500, 1, 1)
    _, cost = oracle.best_order(core, out, "memory")
    assert pair(core, out, oracle.order_memory_comparator(core, out)) == cost
