"""Plain FP64 CPU oracle for the ST-HOSVD hot path of TuckerMPI.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run it; the library itself never does,
and it shares no code with the CUDA path (neither side imports the other).

Everything follows Ballard, Klinvex and Kolda, "TuckerMPI: A Parallel
C++/MPI Software Package for Large-scale Data Compression via the Tucker
Tensor Decomposition" (arXiv 1901.06043):

* sizes                       -- Section 2.1, Eqs. linear-size, unfold-size,
                                 left-size, right-size
* natural-descending layout   -- Section 4.1, Eq. idxtolin
* mode-n unfolding            -- Section 2.2.1 (index map of the unfolding)
* unfolding as row-major
  submatrices ("slabs")       -- Section 4.2
* tensor norm                 -- Section 2.2.2
* TTM                         -- Section 2.2.3 and Algorithm 3 (Section 5.3)
* Gram                        -- Algorithm 2 (Section 5.1)
* eigendecomposition          -- Section 5.2 (LAPACK symmetric solver)
* rank cut                    -- Eq. Un (Section 3.2) and Algorithm 1
* ST-HOSVD                    -- Algorithm 1 (Section 3.3)
* error identities            -- Section 3 (||X - Xhat||^2 = ||X||^2 - ||G||^2)
                                 and Corollary 1
* multi-TTM reconstruction
  and mode ordering           -- Section 7 ("Optimized reconstruction")
* HOSVD                       -- Section 3.2 (Eq. Un on the Gram of X in every
                                 mode, Theorem 1's error bound)
* ST-HOSVD mode order for
  given ranks                 -- the flop counts of the cost analysis of
                                 Section 6 (Gram, eigensolve, TTM per mode),
                                 minimised over all orders as Section 7 does
                                 for reconstruction
* pre- and post-processing    -- Section 3.5 (hyperslice statistics,
                                 standardization, max rescaling, inverses)

Storage convention: a tensor of dims (J_0, ..., J_{N-1}) is a flat 1-D
float64 array in natural-descending order (first index fastest), exactly
the paper's Eq. idxtolin.

Readings where the paper is silent or inconsistent (each one is listed in
the design notes of the repository):

* Eq. Un searches R over [I_n] = {0..I_n-1} but R = I_n must be allowed
  (it reproduces the tensor exactly); R = 0 gives no core.  The search is
  over R in {1..I_n}; R = I_n always qualifies since its tail is empty.
* The cut uses "<=" (inclusive), as printed.
* The tail sums add the eigenvalues exactly as eig(S) returns them, signs
  included (Algorithm 1 sums the computed lambda_i; lambda >= 0 in Eq.
  Xeigprob describes the exact S).  Clamping negative rounding-level
  eigenvalues to zero would turn symmetric rounding noise into a one-sided
  bias that grows with the number of discarded eigenvalues.
* The threshold is eps^2 ||X||^2 / N with N the number of modes and ||X||
  the norm of the ORIGINAL tensor, for every mode and any mode order.
* Section 3.3 says "for n > 1" the partial core is used; Algorithm 1 uses
  the partial core for every n >= 1, which is what is implemented.

* Section 7's memory comparator is printed as "R_i/K_i < R_j/K_j"; taken
  literally it orders the most-growing TTMs first, which the exhaustive
  search (the section's definition of the optimal order) never does.  The
  oracle reads it as K_i/R_i < K_j/R_j (most-shrinking first), pinned against
  that search.  The memory figures of the partial-reconstruction table come
  from the parallel code and are not reproduced by a serial model.
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np

__all__ = [
    "linear_size", "unfold_size", "left_size", "right_size",
    "idx2lin", "lin2idx", "unfold", "fold", "slab_view",
    "norm_sq", "gram", "eig_desc", "rank_cut", "ttm",
    "sthosvd", "multi_ttm", "reconstruct",
    "ttm_chain_sizes", "ttm_chain_flops", "best_order",
    "order_flop_comparator", "order_memory_comparator",
    "relative_errors", "sthosvd_chunked", "hosvd",
    "sthosvd_flops", "best_sthosvd_order", "sthosvd_order_ratio_rule",
    "slice_stats", "standardize_params", "max_rescale_params", "slice_transform",
]


# ---------------------------------------------------------------- sizes (2.1)

def linear_size(dims) -> int:
    """J^* = prod_n J_n (Section 2.1, Eq. linear-size)."""
    return int(np.prod([int(d) for d in dims], dtype=np.int64)) if len(dims) else 1


def unfold_size(dims, n: int) -> int:
    """Product of all sizes except mode n (Eq. unfold-size)."""
    return linear_size(dims) // int(dims[n])


def left_size(dims, n: int) -> int:
    """Product of the sizes below mode n; 1 for n = 0 (Eq. left-size)."""
    return linear_size(dims[:n])


def right_size(dims, n: int) -> int:
    """Product of the sizes above mode n; 1 for n = N-1 (Eq. right-size)."""
    return linear_size(dims[n + 1:])


# ------------------------------------------------------------ layout (4.1/4.2)

def idx2lin(idx, dims) -> int:
    """Linear index j' = sum_n j_n * (product of sizes below n) (Eq. idxtolin)."""
    return int(sum(int(j) * left_size(dims, n) for n, j in enumerate(idx)))


def lin2idx(j: int, dims):
    """Inverse of :func:`idx2lin` (Section 4.1)."""
    out = []
    for d in dims:
        out.append(int(j) % int(d))
        j = int(j) // int(d)
    return tuple(out)


def _all_indices(dims):
    """Multi-index of every linear position 0..J^*-1, shape (J^*, N)."""
    lin = np.arange(linear_size(dims), dtype=np.int64)
    cols = []
    for d in dims:
        cols.append(lin % int(d))
        lin = lin // int(d)
    return np.stack(cols, axis=1) if cols else np.zeros((1, 0), np.int64)


def _unfold_column(idx, dims, n):
    """Column index of the mode-n unfolding (Section 2.2.1):
    sum_{k<n} i_k * left_k + sum_{k>n} i_k * left_k / I_n."""
    col = np.zeros(idx.shape[0], dtype=np.int64)
    for k in range(len(dims)):
        if k < n:
            col += idx[:, k] * left_size(dims, k)
        elif k > n:
            col += idx[:, k] * (left_size(dims, k) // int(dims[n]))
    return col


def unfold(y, dims, n: int) -> np.ndarray:
    """Explicit mode-n unfolding Y_(n) (I_n x J^/n) built element by element
    from the index map of Section 2.2.1.  Independent of :func:`slab_view`;
    used to pin the slab layout and the Gram/TTM on small tensors."""
    y = np.asarray(y).reshape(-1)
    idx = _all_indices(dims)
    col = _unfold_column(idx, dims, n)
    out = np.zeros((int(dims[n]), unfold_size(dims, n)), dtype=y.dtype)
    out[idx[:, n], col] = y
    return out


def fold(mat, dims, n: int) -> np.ndarray:
    """Inverse of :func:`unfold`: flat natural-descending tensor from Y_(n)."""
    idx = _all_indices(dims)
    col = _unfold_column(idx, dims, n)
    return np.asarray(mat)[idx[:, n], col].copy()


def slab_view(y, dims, n: int) -> np.ndarray:
    """The mode-n unfolding as J^>_n contiguous row-major J_n x J^<_n
    submatrices (Section 4.2): element (l, i, r) sits at l + L*(i + I*r),
    which is the C-order array of shape (Rt, I, L)."""
    L, I, Rt = left_size(dims, n), int(dims[n]), right_size(dims, n)
    return np.asarray(y).reshape(Rt, I, L)


# ------------------------------------------------------------- kernels (5.x)

def norm_sq(y) -> float:
    """||Y||^2, the sum of squares of all entries (Section 2.2.2), in FP64."""
    v = np.asarray(y, dtype=np.float64).reshape(-1)
    return float(np.dot(v, v))


def gram(y, dims, n: int) -> np.ndarray:
    """Local Gram S = Y_(n) Y_(n)^T (Algorithm 2).

    n = 0: one product on the column-major J_0 x J^/0 matrix.
    n > 0: S = sum_j Y_(n)[j] Y_(n)[j]^T over the J^>_n row-major
    J_n x J^<_n block columns.  FP64 throughout.
    """
    y = np.asarray(y, dtype=np.float64)
    I = int(dims[n])
    if n == 0:
        y0 = y.reshape(-1, I).T          # column-major I_0 x J^/0
        return y0 @ y0.T
    slabs = slab_view(y, dims, n)
    S = np.zeros((I, I), dtype=np.float64)
    for j in range(slabs.shape[0]):
        S += slabs[j] @ slabs[j].T
    return S


def eig_desc(S):
    """All eigenpairs of the symmetric S, eigenvalues in descending order
    (Section 5.2; the paper calls LAPACK's symmetric eigensolver)."""
    w, V = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    return w[::-1].copy(), V[:, ::-1].copy()


def rank_cut(lam, thr: float):
    """R_n = min R in {1..I_n} with sum_{i>=R} lambda_i <= thr (Eq. Un,
    0-based: keeping R eigenvectors discards lambda[R:]).  The computed
    eigenvalues are summed as they are (Algorithm 1).  Returns (R, tail)
    with tail[R] the sum of the discarded eigenvalues, tail[I] = 0."""
    lam = np.asarray(lam, dtype=np.float64)
    I = lam.shape[0]
    tail = np.zeros(I + 1, dtype=np.float64)
    for i in range(I - 1, -1, -1):       # smallest eigenvalue first
        tail[i] = tail[i + 1] + lam[i]
    for R in range(1, I + 1):
        if tail[R] <= thr:
            return R, tail
    return I, tail


def ttm(y, dims, n: int, V) -> np.ndarray:
    """Local TTM Z = Y x_n V for V of size K x J_n (Algorithm 3).

    n = 0: Z_(0) = V Y_(0), both column-major.
    n > 0: Z_(n)[j] = V Y_(n)[j] for every row-major block column j.
    Returns the flat natural-descending Z with dims J with J_n -> K.
    """
    y = np.asarray(y, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    K, I = V.shape
    assert I == int(dims[n])
    if n == 0:
        y0 = y.reshape(-1, I).T
        z0 = V @ y0
        return z0.T.reshape(-1).copy()
    slabs = slab_view(y, dims, n)
    out = np.empty((slabs.shape[0], K, slabs.shape[2]), dtype=np.float64)
    for j in range(slabs.shape[0]):
        out[j] = V @ slabs[j]
    return out.reshape(-1)


# ------------------------------------------------------------ ST-HOSVD (Alg 1)

def sthosvd(x, dims, eps=None, ranks=None, mode_order=None):
    """ST-HOSVD (Algorithm 1), FP64.

    Exactly one of ``eps`` (relative accuracy) or ``ranks`` (the core size,
    the rank-specified variant of Section 8.4) is given.  ``mode_order``
    is a permutation of the modes (default 0..N-1).  Returns a dict with
    the core (flat, natural-descending), its dims, the factors U_n
    (I_n x R_n), all eigenvalues per mode (descending), the ranks, the
    discarded eigenvalue sums, ||X||^2 and the threshold eps^2 ||X||^2 / N.
    """
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    order = list(range(N)) if mode_order is None else [int(m) for m in mode_order]
    if sorted(order) != list(range(N)):
        raise ValueError("mode_order is not a permutation")
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    nrm2 = norm_sq(x)
    thr = (float(eps) ** 2) * nrm2 / N if eps is not None else None
    state = _new_state(x, dims)
    for n in order:
        S = gram(state["y"], state["cur"], n)
        _truncate_mode(state, n, S, thr, ranks)
    return _finish(state, nrm2, thr, order)


def _new_state(y, dims):
    N = len(dims)
    return {"y": y, "cur": list(dims), "factors": [None] * N, "eigvals": [None] * N,
            "ranks": [0] * N, "discarded": [0.0] * N}


def _choose_factor(S, cur_n, thr, rank):
    """One mode of Algorithm 1 after the Gram: eigenpairs in descending
    order, R_n by Eq. Un (or the given rank), U_n = the leading R_n
    eigenvectors.  Returns (U, eigenvalues, R, discarded sum)."""
    lam, V = eig_desc(S)
    if rank is not None:
        R = int(rank)
        if not 1 <= R <= cur_n:
            raise ValueError("rank out of range")
        _, tail = rank_cut(lam, 0.0)
    else:
        R, tail = rank_cut(lam, thr)
    return V[:, :R].copy(), lam, R, float(tail[R])


def _truncate_mode(state, n, S, thr, ranks):
    """Algorithm 1's steps after the Gram of mode n: eig, cut, Y <- Y x_n U_n^T."""
    U, lam, R, disc = _choose_factor(S, state["cur"][n], thr,
                                     None if ranks is None else ranks[n])
    state["y"] = ttm(state["y"], state["cur"], n, U.T)
    state["cur"][n] = R
    state["factors"][n], state["eigvals"][n] = U, lam
    state["ranks"][n], state["discarded"][n] = R, disc


def _finish(state, nrm2, thr, order):
    return {
        "core": state["y"], "core_dims": tuple(state["cur"]), "factors": state["factors"],
        "eigvals": state["eigvals"], "ranks": tuple(state["ranks"]),
        "discarded": state["discarded"], "norm_sq": nrm2, "threshold": thr,
        "mode_order": tuple(order),
    }


def sthosvd_chunked(chunk, nchunks, dims, eps=None, ranks=None):
    """ST-HOSVD (Algorithm 1, mode order 0..N-1) of a tensor supplied in
    pieces, for inputs too large to hold in FP64 at once.  ``chunk(c)``
    returns the flat natural-descending sub-tensor whose last-mode indices
    are [J_{N-1} c / nchunks, J_{N-1} (c + 1) / nchunks), c = 0..nchunks-1
    (N >= 2).  Each piece is a contiguous run of the block columns of every
    unfolding of modes n < N-1, so:
      ||X||^2 = sum over pieces of their sums of squares (Section 2.2.2);
      the mode-0 Gram = sum over pieces of their mode-0 Grams (Algorithm 2
        sums over block columns; the column-major mode-0 unfolding of a
        piece is a contiguous range of columns of X's);
      the mode-0 TTM acts on each column independently (Algorithm 3), so
        the partial core is the pieces' TTMs laid end to end.
    Modes 1..N-1 then run on the partial core exactly as in :func:`sthosvd`.
    Same result dict as :func:`sthosvd`."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    if N < 2:
        raise ValueError("sthosvd_chunked needs N >= 2")
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    last = dims[-1]
    bounds = [(last * c // nchunks, last * (c + 1) // nchunks) for c in range(nchunks)]
    nrm2, S0 = 0.0, np.zeros((dims[0], dims[0]), dtype=np.float64)
    for c, (a, b) in enumerate(bounds):
        if b <= a:
            continue
        piece = np.asarray(chunk(c), dtype=np.float64).reshape(-1)
        pdims = dims[:-1] + (b - a,)
        nrm2 += norm_sq(piece)
        S0 += gram(piece, pdims, 0)
    thr = (float(eps) ** 2) * nrm2 / N if eps is not None else None
    U, lam, R, disc = _choose_factor(S0, dims[0], thr, None if ranks is None else ranks[0])
    parts = []
    for c, (a, b) in enumerate(bounds):
        if b <= a:
            continue
        piece = np.asarray(chunk(c), dtype=np.float64).reshape(-1)
        parts.append(ttm(piece, dims[:-1] + (b - a,), 0, U.T))
    state = _new_state(np.concatenate(parts), dims)
    state["cur"][0] = R
    state["factors"][0], state["eigvals"][0] = U, lam
    state["ranks"][0], state["discarded"][0] = R, disc
    for n in range(1, N):
        S = gram(state["y"], state["cur"], n)
        _truncate_mode(state, n, S, thr, ranks)
    return _finish(state, nrm2, thr, list(range(N)))


# ------------------------------------------------------------ HOSVD (3.2)

def hosvd(x, dims, eps=None, ranks=None):
    """HOSVD (Section 3.2): for every mode n the eigendecomposition of the
    Gram of X's own mode-n unfolding (Eq. Xeigprob), R_n by Eq. Un with the
    same threshold eps^2 ||X||^2 / N (or the given ranks), U_n the leading
    R_n eigenvectors; then the core G = X x_0 U_0^T ... x_{N-1} U_{N-1}^T.
    Theorem 1 bounds the error: ||X - Xhat||^2 <= sum_n discarded_n.
    Same result dict as :func:`sthosvd` (mode_order records 0..N-1)."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    nrm2 = norm_sq(x)
    thr = (float(eps) ** 2) * nrm2 / N if eps is not None else None
    state = _new_state(x, dims)
    for n in range(N):
        U, lam, R, disc = _choose_factor(gram(x, dims, n), dims[n], thr,
                                         None if ranks is None else ranks[n])
        state["factors"][n], state["eigvals"][n] = U, lam
        state["ranks"][n], state["discarded"][n] = R, disc
    y, cur = x, list(dims)
    for n in range(N):
        y = ttm(y, cur, n, state["factors"][n].T)
        cur[n] = state["ranks"][n]
    state["y"], state["cur"] = y, cur
    return _finish(state, nrm2, thr, list(range(N)))


# --------------------------------------------------- reconstruction (Sec. 7)

def multi_ttm(core, core_dims, mats, mode_order=None):
    """Z = G x_{p(0)} A_{p(0)} ... x_{p(N-1)} A_{p(N-1)} with A_n of size
    K_n x R_n (Section 7).  Any order gives the same result up to rounding."""
    dims = [int(d) for d in core_dims]
    order = list(range(len(dims))) if mode_order is None else list(mode_order)
    z = np.asarray(core, dtype=np.float64).reshape(-1)
    for n in order:
        z = ttm(z, dims, n, mats[n])
        dims[n] = np.asarray(mats[n]).shape[0]
    return z, tuple(dims)


def reconstruct(core, core_dims, factors, begin=None, end=None, mode_order=None):
    """(Partial) reconstruction of the subtensor [begin_n, end_n) in every
    mode: A_n = rows begin_n..end_n-1 of U_n, i.e. C_n^T U_n with C_n a
    column selection (Section 7)."""
    N = len(core_dims)
    begin = [0] * N if begin is None else list(begin)
    end = [np.asarray(f).shape[0] for f in factors] if end is None else list(end)
    mats = [np.asarray(factors[n])[begin[n]:end[n], :] for n in range(N)]
    return multi_ttm(core, core_dims, mats, mode_order)


def ttm_chain_sizes(core_dims, out_dims, order):
    """Number of entries of the tensor after each TTM of the chain
    (the intermediate sizes of the partial-reconstruction table, Sec. 8.5)."""
    cur = [int(d) for d in core_dims]
    sizes = [linear_size(cur)]
    for n in order:
        cur[n] = int(out_dims[n])
        sizes.append(linear_size(cur))
    return sizes


def ttm_chain_flops(core_dims, out_dims, order) -> int:
    """Multiply-adds of the chain: the mode-n TTM of a tensor of size J^*
    with a K_n x J_n matrix costs J^* K_n (Section 5.3, O(J^* K))."""
    cur = [int(d) for d in core_dims]
    total = 0
    for n in order:
        total += linear_size(cur) * int(out_dims[n])
        cur[n] = int(out_dims[n])
    return total


def best_order(core_dims, out_dims, objective="flops"):
    """Exhaustive search over all N! mode orders (what the paper says
    TuckerMPI does, Section 7).  objective 'flops' minimises
    :func:`ttm_chain_flops`; 'memory' minimises the largest
    input+output pair of one TTM.  Ties go to the lexicographically first
    order.  Returns (order, cost)."""
    N = len(core_dims)
    best, best_cost = None, None
    for perm in itertools.permutations(range(N)):
        if objective == "flops":
            cost = ttm_chain_flops(core_dims, out_dims, perm)
        elif objective == "memory":
            s = ttm_chain_sizes(core_dims, out_dims, perm)
            cost = max(s[i] + s[i + 1] for i in range(N))
        else:
            raise ValueError(objective)
        if best_cost is None or cost < best_cost:
            best, best_cost = perm, cost
    return tuple(best), best_cost


def order_flop_comparator(core_dims, out_dims):
    """O(N log N) order from the pairwise flop rule of Section 7: mode i
    precedes mode j when K_i R_i R_j + K_i R_j K_j < R_i R_j K_j + R_i K_i K_j."""
    R = [int(r) for r in core_dims]
    K = [int(k) for k in out_dims]

    def cmp(i, j):
        a = K[i] * R[i] * R[j] + K[i] * R[j] * K[j]
        b = R[i] * R[j] * K[j] + R[i] * K[i] * K[j]
        return -1 if a < b else (1 if a > b else (i > j) - (i < j))

    return tuple(sorted(range(len(R)), key=functools.cmp_to_key(cmp)))


def order_memory_comparator(core_dims, out_dims):
    """Section 7's memory rule, read with R and K in the order its exchange
    argument needs: a TTM in mode i scales the tensor by K_i / R_i, so the
    temporary memory is smallest when the most-shrinking modes go first --
    mode i precedes mode j if K_i/R_i < K_j/R_j.  (As printed the inequality
    reads R_i/K_i < R_j/K_j, which puts the most-growing modes first; the
    exhaustive search the same section calls optimal never picks that order.)
    Compared division-free: K_i R_j < K_j R_i."""
    R = [int(r) for r in core_dims]
    K = [int(k) for k in out_dims]

    def cmp(i, j):
        a, b = K[i] * R[j], K[j] * R[i]
        return -1 if a < b else (1 if a > b else (i > j) - (i < j))

    return tuple(sorted(range(len(R)), key=functools.cmp_to_key(cmp)))


# ------------------------------------------- ST-HOSVD mode order (Sec. 6, 7)

def sthosvd_flops(dims, ranks, order):
    """Flops of ST-HOSVD in the given mode order with the given ranks, from
    the cost analysis of Section 6: the mode-n Gram of the current tensor
    (L, I_n, Rt) performs L I_n^2 Rt flops (symmetry exploited), the
    eigensolve (10/3) I_n^3, the TTM 2 L R_n I_n Rt; L and Rt are products
    of the ranks of the modes already processed and the sizes of the rest."""
    cur = [int(d) for d in dims]
    total = 0.0
    for n in order:
        numel = float(linear_size(cur))           # L I_n Rt
        I, R = int(dims[n]), int(ranks[n])
        total += numel * I + (10.0 / 3.0) * I ** 3 + 2.0 * numel * R
        cur[n] = R
    return total


def best_sthosvd_order(dims, ranks):
    """The flop-minimal ST-HOSVD mode order for given ranks, by exhaustive
    search over all N! orders of :func:`sthosvd_flops` (the way Section 7
    picks reconstruction orders); ties to the lexicographically first.
    Returns (order, flops)."""
    best, best_cost = None, None
    for perm in itertools.permutations(range(len(dims))):
        cost = sthosvd_flops(dims, ranks, perm)
        if best_cost is None or cost < best_cost:
            best, best_cost = perm, cost
    return tuple(best), best_cost


def sthosvd_order_ratio_rule(dims, ranks):
    """The same order from a pairwise exchange argument.  Step n costs
    c_n = I_n + 2 R_n per entry of the current tensor (plus the eigensolve,
    which no order changes) and multiplies its size by a_n = R_n / I_n.  For
    adjacent modes i, j after a prefix of size P, i first costs
    P (c_i + a_i c_j) and j first P (c_j + a_j c_i): i goes first iff
    c_i (1 - a_j) < c_j (1 - a_i), i.e. by c_n / (1 - a_n) ascending, and
    modes that do not shrink (R_n = I_n) go last.  Compared without
    division: c_i (I_j - R_j) I_i < c_j (I_i - R_i) I_j."""
    I = [int(d) for d in dims]
    R = [int(r) for r in ranks]
    c = [I[n] + 2 * R[n] for n in range(len(I))]

    def cmp(i, j):
        a = c[i] * (I[j] - R[j]) * I[i]
        b = c[j] * (I[i] - R[i]) * I[j]
        return -1 if a < b else (1 if a > b else (i > j) - (i < j))

    return tuple(sorted(range(len(I)), key=functools.cmp_to_key(cmp)))


# ------------------------------------------ pre- and post-processing (3.5)

STAT_NAMES = ("mean", "std", "max", "min", "norm1", "norm2")


def slice_stats(x, dims, n: int) -> np.ndarray:
    """Statistics of every mode-n hyperslice X(:, ..., i, ..., :) (Section
    3.5): an (I_n, 6) array of mean, standard deviation, maximum, minimum,
    1-norm and 2-norm of its J^*/I_n entries.  The standard deviation is the
    population one, sqrt(sum (x - mean)^2 / count) (the paper does not say
    which; this one makes a standardized slice have variance exactly 1).
    The hyperslice is row i of the explicit mode-n unfolding."""
    X = slab_view(np.asarray(x, dtype=np.float64), dims, n)   # (Rt, I, L)
    I = int(dims[n])
    out = np.zeros((I, 6), dtype=np.float64)
    for i in range(I):
        v = X[:, i, :].reshape(-1)
        mean = v.sum() / v.size
        out[i] = (mean, math.sqrt(((v - mean) ** 2).sum() / v.size), v.max(), v.min(),
                  np.abs(v).sum(), math.sqrt((v * v).sum()))
    return out


def standardize_params(stats):
    """Standardization (Section 3.5 (a)): shift by the mean, scale by the
    standard deviation, i.e. y = (x - mean_i) / std_i; returned as
    (shift, scale) with y = (x - shift_i) * scale_i.  A constant slice
    (std 0) keeps scale 1."""
    st = np.asarray(stats, dtype=np.float64)
    shift = st[:, 0].copy()
    scale = np.where(st[:, 1] > 0, 1.0 / np.where(st[:, 1] > 0, st[:, 1], 1.0), 1.0)
    return shift, scale


def max_rescale_params(stats):
    """Max rescaling (Section 3.5 (b)): divide by the largest absolute value
    of the slice, so it ranges within [-1, 1]; (shift, scale) = (0, 1 /
    max |x|).  An all-zero slice keeps scale 1."""
    st = np.asarray(stats, dtype=np.float64)
    m = np.maximum(np.abs(st[:, 2]), np.abs(st[:, 3]))
    return np.zeros(st.shape[0]), np.where(m > 0, 1.0 / np.where(m > 0, m, 1.0), 1.0)


def slice_transform(x, dims, n: int, shift, scale, inverse=False) -> np.ndarray:
    """Applies one linear function per mode-n hyperslice (Section 3.5):
    y = (x - shift_i) * scale_i, or its inverse x = y / scale_i + shift_i
    (post-processing after a reconstruction)."""
    X = slab_view(np.asarray(x, dtype=np.float64), dims, n).copy()
    sh = np.asarray(shift, dtype=np.float64)[None, :, None]
    sc = np.asarray(scale, dtype=np.float64)[None, :, None]
    Y = X / sc + sh if inverse else (X - sh) * sc
    return Y.reshape(-1)


# ------------------------------------------------------------ error metrics

def relative_errors(x, dims, result, explicit=True):
    """Relative errors of an ST-HOSVD result:
    err_est      = sqrt(sum_n discarded_n / ||X||^2)     (Corollary 1)
    err_gram     = sqrt((||X||^2 - ||G||^2) / ||X||^2)   (Section 3)
    err_explicit = ||X - Xhat|| / ||X||                  (definition)."""
    nrm2 = result["norm_sq"]
    out = {
        "err_est": math.sqrt(max(sum(result["discarded"]), 0.0) / nrm2),
        "err_gram": math.sqrt(max(nrm2 - norm_sq(result["core"]), 0.0) / nrm2),
    }
    if explicit:
        xhat, _ = reconstruct(result["core"], result["core_dims"], result["factors"])
        d = np.asarray(x, dtype=np.float64).reshape(-1) - xhat
        out["err_explicit"] = math.sqrt(float(np.dot(d, d)) / nrm2)
    return out
