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
    "relative_errors",
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
    y, cur = x, list(dims)
    factors, eigvals = [None] * N, [None] * N
    out_ranks, discarded = [0] * N, [0.0] * N
    for n in order:
        S = gram(y, cur, n)
        lam, V = eig_desc(S)
        if ranks is not None:
            R = int(ranks[n])
            if not 1 <= R <= cur[n]:
                raise ValueError("rank out of range")
            _, tail = rank_cut(lam, 0.0)
        else:
            R, tail = rank_cut(lam, thr)
        U = V[:, :R].copy()
        y = ttm(y, cur, n, U.T)
        cur[n] = R
        factors[n], eigvals[n] = U, lam
        out_ranks[n], discarded[n] = R, float(tail[R])
    return {
        "core": y, "core_dims": tuple(cur), "factors": factors,
        "eigvals": eigvals, "ranks": tuple(out_ranks),
        "discarded": discarded, "norm_sq": nrm2, "threshold": thr,
        "mode_order": tuple(order),
    }


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
