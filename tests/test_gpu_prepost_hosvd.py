"""Parity of the pre-/post-processing (Section 3.5), the HOSVD (Section 3.2)
and ST-HOSVD in a flop-optimal mode order with the FP64 oracle, through the
C ABI.

Tolerances: statistics are sums of exactly converted inputs (FP64 sums, or
exact FP32 pairs moved into FP64 for FP32 data), so each matches the oracle
to 1e-12 relative (the standard deviation to 1e-12 of max(std, 1e-3 |mean|),
since both sides subtract a mean that carries rounding); max and min are
exact.  Transforms of FP64 data are evaluated in FP64 (a few ulps from the
oracle); of FP32 data in FP32-pair arithmetic rounded once to FP32, within
one FP32 ulp of the oracle's FP64 value.
HOSVD in FP64 follows the FP64 path's tolerances (eigenvalues 1e-10 of the
largest, subspaces by principal angle 1e-8 where the gap is wide, identical
ranks, explicit error within 1e-12).
"""
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


# (dims, mode): the rows regime (L < 256, including L = 1 with I above and
# below a block) and the runs regime (L >= 256, ragged chunks, L not a
# multiple of 4)
STAT_CASES = [((50, 40, 30), 0), ((50, 40, 30), 1), ((50, 40, 30), 2), ((1500, 20, 3), 0),
              ((7, 300, 11), 1), ((300, 11, 5), 1), ((4097, 3, 2), 1), ((16, 16, 3, 11, 2), 3),
              ((1, 9), 1), ((5,), 0), ((257, 33, 4), 2), ((1000, 1000, 50), 0),
              ((1000, 1000, 50), 2), ((3, 7, 100000), 1)]


def _data(dims, mode, seed):
    rng = np.random.default_rng(seed)
    n = oracle.linear_size(dims)
    idx = oracle.tucker_fp64._all_indices(dims)[:, mode]
    off = rng.uniform(-5, 5, dims[mode])[idx]
    sc = (10.0 ** rng.uniform(-2, 2, dims[mode]))[idx]
    return rng.standard_normal(n) * sc + off


@pytest.mark.parametrize("dims,mode", STAT_CASES)
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_slice_stats(ctx, dims, mode, dt):
    t = dev(_data(dims, mode, sum(dims) + mode), dt)
    xs = host(t)
    want = oracle.slice_stats(xs, dims, mode)
    got = host(ctx.slice_stats(t, dims, mode))
    for k in (0, 4, 5):
        assert np.allclose(got[:, k], want[:, k], rtol=1e-12, atol=1e-13 * np.abs(want[:, k]).max())
    sd_tol = 1e-12 * np.maximum(want[:, 1], 1e-3 * np.abs(want[:, 0]))
    assert np.all(np.abs(got[:, 1] - want[:, 1]) <= sd_tol + 1e-300)
    assert np.array_equal(got[:, 2], want[:, 2]) and np.array_equal(got[:, 3], want[:, 3])


def test_slice_stats_nonfinite_is_reported(ctx):
    from paper_1901_06043_gb300 import tucker
    x = np.ones(600)
    x[17] = np.inf
    with pytest.raises(tucker.TuckerError) as e:
        ctx.slice_stats(dev(x, torch.float32), (20, 30), 1)
    assert e.value.name == "NONFINITE"


@pytest.mark.parametrize("dims,mode", STAT_CASES[:8])
@pytest.mark.parametrize("method", ["standardize", "max"])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_preprocess_and_inverse(ctx, dims, mode, method, dt):
    t = dev(_data(dims, mode, 3 * sum(dims) + mode), dt)
    xs = host(t)
    st = oracle.slice_stats(xs, dims, mode)
    sh_w, sc_w = (oracle.standardize_params(st) if method == "standardize"
                  else oracle.max_rescale_params(st))
    y, sh, sc = ctx.preprocess(t, dims, mode, method)
    assert np.allclose(host(sh), sh_w, rtol=1e-12, atol=1e-13 * np.abs(sh_w).max())
    assert np.allclose(host(sc), sc_w, rtol=1e-11)
    # the transform with the library's own parameters, against the oracle's
    want = oracle.slice_transform(xs, dims, mode, host(sh), host(sc))
    got = host(y)
    if dt == torch.float64:
        assert np.allclose(got, want, rtol=4e-16 * 8, atol=1e-15 * np.abs(want).max())
    else:
        assert np.all(np.abs(got - want) <= np.spacing(np.abs(want).astype(np.float32)))
    # post-processing: the inverse in place restores x
    ctx.slice_transform(y, dims, mode, sh, sc, inverse=True, out=y)
    back = host(y)
    want_b = oracle.slice_transform(got, dims, mode, host(sh), host(sc), inverse=True)
    if dt == torch.float64:
        assert np.allclose(back, want_b, rtol=1e-15, atol=1e-15 * np.abs(want_b).max())
        assert np.allclose(back, xs, rtol=1e-13, atol=1e-13 * np.abs(xs).max())
    else:
        assert np.all(np.abs(back - want_b) <= np.spacing(np.abs(want_b).astype(np.float32)))


def test_postprocess_of_a_reconstructed_subtensor(ctx):
    """The paper's use: max-rescale a species mode (Section 8.4), compress,
    reconstruct a subtensor, undo the scaling of its mode-3 range; the same
    pipeline in the oracle, with the library's scaling parameters."""
    dims = (40, 30, 20, 11, 3)
    x = synth.tucker_torch(dims, (10, 10, 8, 11, 3), decay=0.1, eta=1e-6, seed=9,
                           dtype=torch.float64)
    y, sh, sc = ctx.preprocess(x, dims, 3, "max")
    res = ctx.sthosvd(y, dims, eps=1e-4, prec="fp64")
    b, e = (0, 0, 0, 4, 1), (40, 30, 20, 9, 3)
    sub = res.reconstruct(b, e)
    sdims = tuple(e[k] - b[k] for k in range(5))
    got = host(ctx.slice_transform(sub, sdims, 3, sh[4:], sc[4:], inverse=True))
    yo = oracle.slice_transform(host(x), dims, 3, host(sh), host(sc))
    ref = oracle.sthosvd(yo, dims, eps=1e-4)
    assert ref["ranks"] == res.ranks
    so, _ = oracle.reconstruct(ref["core"], ref["core_dims"], ref["factors"], b, e)
    want = oracle.slice_transform(so, sdims, 3, host(sh)[4:9], host(sc)[4:9], inverse=True)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    xsub = host(x).reshape(dims[::-1])[1:3, 4:9].reshape(-1)
    assert np.linalg.norm(got - xsub) <= 1e-3 * np.linalg.norm(xsub)
    res.close()


# ------------------------------------------------------------------ HOSVD

def _compare(x, dims, res, ref, eig_tol=1e-10, angle_tol=1e-8, err_tol=1e-12):
    assert res.ranks == ref["ranks"]
    for n in range(len(dims)):
        lam = host(res.eigvals[n])
        w = ref["eigvals"][n]
        assert np.abs(lam - w).max() <= eig_tol * abs(w).max()
        U = host(res.factors[n])
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-12
        R = res.ranks[n]
        if R < dims[n] and (w[R - 1] - w[R]) > 1e-6 * w[0]:
            W = ref["factors"][n]       # sin of the largest principal angle
            assert np.linalg.norm(W - U @ (U.T @ W), 2) <= angle_tol
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e1 = oracle.relative_errors(x, dims, ours)
    e0 = oracle.relative_errors(x, dims, ref)
    assert abs(e1["err_explicit"] - e0["err_explicit"]) <= err_tol
    return e1


@pytest.mark.parametrize("dims,core,eps", [((40, 50, 30), (5, 6, 4), 1e-3),
                                           ((70, 64, 20, 6), (12, 10, 8, 4), 1e-2),
                                           ((130, 20, 9), (20, 8, 5), 1e-4)])
def test_hosvd_fp64(ctx, dims, core, eps):
    x, _ = synth.tucker_numpy(dims, core, decay=0.1, eta=1e-3, seed=sum(dims))
    ref = oracle.hosvd(x, dims, eps=eps)
    res = ctx.hosvd(dev(x), dims, eps=eps, prec="fp64")
    e = _compare(x, dims, res, ref)
    # Theorem 1's bound and the eps guarantee
    assert e["err_explicit"] ** 2 <= sum(res.discarded) / res.norm_sq * (1 + 1e-9) + 1e-24
    assert e["err_explicit"] <= eps
    res.close()


def test_hosvd_rank_specified_fp64(ctx):
    dims = (30, 25, 20)
    x, _ = synth.tucker_numpy(dims, (6, 6, 6), decay=0.05, eta=1e-2, seed=4)
    ref = oracle.hosvd(x, dims, ranks=(5, 4, 6))
    res = ctx.hosvd(dev(x), dims, ranks=(5, 4, 6), prec="fp64")
    _compare(x, dims, res, ref)
    res.close()


def test_hosvd_mixed_large_modes(ctx):
    """FP32 input, MIXED: exact-digit Grams of X in every mode (mode 0
    column mode, modes 1 and 2 row mode), tensor-core TTM for mode 0;
    identical ranks, error within eps and within the oracle's error."""
    dims = (256, 160, 136, 6)
    x = synth.tucker_torch(dims, (30, 24, 20, 6), decay=0.1, eta=1e-6, seed=12)
    xs = host(x)
    ref = oracle.hosvd(xs, dims, eps=1e-4)
    res = ctx.hosvd(x, dims, eps=1e-4, prec="mixed")
    assert res.ranks == ref["ranks"]
    assert res.gram_kernel[0] == "tcgen05-x3"
    for n in range(4):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"]
    ours = {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}
    e1 = oracle.relative_errors(xs, dims, ours)["err_explicit"]
    e0 = oracle.relative_errors(xs, dims, ref)["err_explicit"]
    # FP32 TTMs round each core entry to ~u32 sqrt(I_n) ~ 1e-6 relative
    assert e1 <= 1e-4 and abs(e1 - e0) <= 5e-6
    res.close()


# ------------------------------------------------------------- mode order

def test_sthosvd_in_the_flop_optimal_order(ctx):
    """The order tucker_sthosvd_order picks for the ranks of a first run,
    passed back as the mode order: the same ranks, Corollary 1's error, and
    fewer Gram + TTM flops than the natural order."""
    from paper_1901_06043_gb300 import tucker
    dims = (60, 12, 50, 4)
    x, _ = synth.tucker_numpy(dims, (8, 12, 30, 1), decay=0.1, eta=1e-5, seed=21)
    r0 = ctx.sthosvd(dev(x), dims, eps=1e-3, prec="fp64")
    order = tucker.sthosvd_order(dims, r0.ranks)
    assert order != (0, 1, 2, 3)
    ref = oracle.sthosvd(x, dims, eps=1e-3, mode_order=order)
    res = ctx.sthosvd(dev(x), dims, eps=1e-3, mode_order=order, prec="fp64")
    assert res.mode_order == order
    _compare(x, dims, res, ref)
    assert oracle.sthosvd_flops(dims, res.ranks, order) < oracle.sthosvd_flops(
        dims, res.ranks, range(4))
    r0.close()
    res.close()
