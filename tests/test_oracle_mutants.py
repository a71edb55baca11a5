"""Planted mistakes in the oracle (CPU only): each plausible slip -- a dropped
slab, a wrong index term, an ascending eigenvalue order, a strict '<' in the
cut, eps instead of eps^2 -- must make at least one pin fail.  This is what
gives the pins their meaning: they are sensitive to the errors they guard."""
import math

import numpy as np
import pytest

import oracle
import oracle.tucker_fp64 as O
from paper_1901_06043_gb300 import synth


def _pins_pass():
    """A compact subset of the pins of test_oracle_pins; True if all hold."""
    try:
        # golden worked example (Section 4.2), mode 1 and 2
        dims = (3, 4, 3, 2)
        y = np.arange(72)
        if not np.array_equal(O.unfold(y, dims, 1)[0, :6], [0, 1, 2, 12, 13, 14]):
            return False
        if not np.array_equal(O.unfold(y, dims, 2)[1, :3], [12, 13, 14]):
            return False
        # trace(S) = ||Y||^2 for every mode
        rng = np.random.default_rng(0)
        d4 = (3, 4, 2, 3)
        y = rng.standard_normal(72)
        for n in range(4):
            if not math.isclose(np.trace(O.gram(y, d4, n)), O.norm_sq(y), rel_tol=1e-12):
                return False
        # cut semantics
        if O.rank_cut([4, 2, 1, 0.5], 1.5)[0] != 2:
            return False
        # noiseless exact recovery
        x, _ = synth.tucker_numpy((8, 9, 7), (2, 3, 2), seed=1)
        res = O.sthosvd(x, (8, 9, 7), eps=1e-6)
        if res["ranks"] != (2, 3, 2):
            return False
        if O.relative_errors(x, (8, 9, 7), res)["err_explicit"] > 1e-12:
            return False
        # Algorithm 1's guarantee ||X - Xhat|| <= eps ||X|| on a decaying spectrum
        x, _ = synth.tucker_numpy((14, 11, 9, 6), (8, 8, 6, 5), decay=0.2, eta=1e-3, seed=6)
        res = O.sthosvd(x, (14, 11, 9, 6), eps=0.05)
        if O.relative_errors(x, (14, 11, 9, 6), res)["err_explicit"] > 0.05:
            return False
        # config 40x50x30 ranks
        x, _ = synth.tucker_numpy((40, 50, 30), (5, 6, 4), eta=1e-4, seed=0)
        if O.sthosvd(x, (40, 50, 30), eps=1e-3)["ranks"] != (5, 6, 4):
            return False
        return True
    except Exception:
        return False


def test_unmodified_oracle_passes():
    assert _pins_pass()


def _gram_drop_last_slab(y, dims, n):
    y = np.asarray(y, dtype=np.float64)
    I = int(dims[n])
    if n == 0:
        y0 = y.reshape(-1, I).T[:, :-1]
        return y0 @ y0.T
    sl = O.slab_view(y, dims, n)
    S = np.zeros((I, I))
    for j in range(sl.shape[0] - 1):
        S += sl[j] @ sl[j].T
    return S


def _unfold_column_no_division(idx, dims, n):
    col = np.zeros(idx.shape[0], dtype=np.int64)
    for k in range(len(dims)):
        if k != n:
            col += idx[:, k] * O.left_size(dims, k)
    return col


def _eig_ascending(S):
    return np.linalg.eigh(np.asarray(S, dtype=np.float64))


def _rank_cut_strict(lam, thr):
    lam = np.asarray(lam, dtype=np.float64)
    I = lam.shape[0]
    tail = np.zeros(I + 1)
    for i in range(I - 1, -1, -1):
        tail[i] = tail[i + 1] + lam[i]
    for R in range(1, I + 1):
        if tail[R] < thr:
            return R, tail
    return I, tail


def _ttm_transposed_slabs(y, dims, n, V):
    y = np.asarray(y, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    K, I = V.shape
    if n == 0:
        return (V @ y.reshape(-1, I).T).T.reshape(-1).copy()
    sl = O.slab_view(y, dims, n)
    out = np.empty((sl.shape[0], K, sl.shape[2]))
    for j in range(sl.shape[0]):
        out[sl.shape[0] - 1 - j] = V @ sl[j]        # slabs written in reverse order
    return out.reshape(-1)


@pytest.mark.parametrize("name,target,mutant", [
    ("gram drops a slab", "gram", _gram_drop_last_slab),
    ("unfolding index term not divided by I_n", "_unfold_column", _unfold_column_no_division),
    ("eigenvalues ascending", "eig_desc", _eig_ascending),
    ("strict < in the cut", "rank_cut", _rank_cut_strict),
    ("TTM slabs misplaced", "ttm", _ttm_transposed_slabs),
])
def test_planted_mistake_is_caught(monkeypatch, name, target, mutant):
    monkeypatch.setattr(O, target, mutant)
    assert not _pins_pass(), name


def test_eps_not_squared_is_caught(monkeypatch):
    real = O.sthosvd

    def wrong(x, dims, eps=None, ranks=None, mode_order=None):
        return real(x, dims, eps=None if eps is None else math.sqrt(eps), ranks=ranks,
                    mode_order=mode_order)

    monkeypatch.setattr(O, "sthosvd", wrong)
    assert not _pins_pass()
