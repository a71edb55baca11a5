"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration bench.py times (the same library calls at the same shapes).

- 200x200x200x50 FP64 (3.2 GB): the whole FP64 ST-HOSVD against the oracle,
  which finishes in seconds at this size; reconstruction of the
  200x200x200x1 slice by multi-TTM.
- 256x256x256x11x32 FP32 (23 GB) at eps 1e-2, 1e-4, 1e-5: the mixed path
  against the FP64 GPU path (same ranks, errors within the bound), and
  sampled mode-0 Gram entries against the oracle.
- 500x500x500x11x8 FP32 (44 GB), eps 1e-4: sampled mode-0 Gram entries of
  both precisions against the oracle, mixed ranks equal to the FP64 path's,
  Cor. 1 (error estimate from the discarded eigenvalues), and sampled
  entries of the 500x500x500x11x1 reconstruction against the oracle's
  multi-TTM of the same core and factors.

Inputs follow the synthetic recipe of the workloads (synth.tucker_torch).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_06043_gb300 import tucker
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = tucker.Context(timing=True)
    yield c
    c.close()


def host(t):
    return t.detach().cpu().numpy()


def _mode0_gram_samples(x, dims, pairs):
    """Oracle 2x2 Grams of column pairs (i, j) of the mode-0 view (FP64)."""
    I0 = dims[0]
    xv = x.view(-1, I0)
    out = {}
    for i, j in pairs:
        ci = xv[:, i].double().cpu().numpy()
        cj = xv[:, j].double().cpu().numpy()
        y = np.stack([ci, cj], axis=1).reshape(-1)          # dims (2, K)
        out[(i, j)] = oracle.gram(y, (2, ci.size), 0)
    return out


def _check_gram_samples(S, samples, rel):
    for (i, j), G in samples.items():
        scale = math.sqrt(G[0, 0] * G[1, 1])
        assert abs(S[i, j] - G[0, 1]) <= rel * scale, ((i, j), S[i, j], G[0, 1])
        assert abs(S[i, i] - G[0, 0]) <= rel * G[0, 0]
        assert abs(S[j, j] - G[1, 1]) <= rel * G[1, 1]


def _result_dict(res):
    return {"core": host(res.core), "core_dims": res.ranks,
            "factors": [host(f) for f in res.factors], "discarded": res.discarded,
            "norm_sq": res.norm_sq}


def test_c200_fp64_full_parity(ctx):
    dims, core = (200, 200, 200, 50), (30, 30, 30, 12)
    x = synth.tucker_torch(dims, core, decay=0.15, eta=1e-6, seed=0, dtype=torch.float64)
    xs = host(x)
    ref = oracle.sthosvd(xs, dims, eps=1e-4)
    res = ctx.sthosvd(x, dims, eps=1e-4, prec="fp64")
    assert res.ranks == ref["ranks"]
    for n in range(len(dims)):
        lam = host(res.eigvals[n])
        assert np.abs(lam - ref["eigvals"][n]).max() <= 1e-10 * abs(ref["eigvals"][n]).max()
        U = host(res.factors[n])
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-12
        R = res.ranks[n]
        w = ref["eigvals"][n]
        if R < dims[n] and (w[R - 1] - w[R]) > 1e-6 * w[0]:
            # largest principal angle between the kept subspaces
            sv = np.linalg.svd(U.T @ ref["factors"][n], compute_uv=False)
            assert math.acos(min(1.0, sv.min())) <= 1e-8
    ours = _result_dict(res)
    # the explicit error ||X - Xhat|| / ||X||: the estimate from the
    # discarded eigenvalues carries their FP64 rounding (~1e-16 lambda_max
    # each) divided by 2 err, ~1e-11 here, on both sides
    r1 = oracle.relative_errors(xs, dims, ours)
    r0 = oracle.relative_errors(xs, dims, ref)
    assert abs(r1["err_explicit"] - r0["err_explicit"]) <= 1e-12
    assert r1["err_est"] <= 1e-4 and abs(r1["err_est"] - r1["err_explicit"]) <= 1e-9
    # reconstruction of the 200x200x200x1 slice (last index 0)
    b, e = (0, 0, 0, 0), (200, 200, 200, 1)
    want, _ = oracle.reconstruct(ours["core"], res.ranks, ours["factors"], b, e)
    got = host(res.reconstruct(b, e))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_c256_mixed_vs_fp64_ranks_and_errors(ctx):
    dims, core = (256, 256, 256, 11, 32), (40, 40, 40, 11, 16)
    x = synth.tucker_torch(dims, core, decay=0.1, eta=1e-7, seed=0)
    rng = np.random.default_rng(1)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, dims[0], size=(6, 2))]
    _check_gram_samples(host(ctx.gram(x, dims, 0, "fp32")), _mode0_gram_samples(x, dims, pairs),
                        2e-6)
    for eps in (1e-2, 1e-4, 1e-5):
        r64 = ctx.sthosvd(x, dims, eps=eps, prec="fp64")
        rmx = ctx.sthosvd(x, dims, eps=eps, prec="mixed")
        assert rmx.ranks == r64.ranks, (eps, rmx.ranks, r64.ranks)
        d64, dmx = sum(r64.discarded), sum(rmx.discarded)
        assert d64 <= eps ** 2 * r64.norm_sq and dmx <= eps ** 2 * rmx.norm_sq
        # the FP32 Gram rounds without bias: its discarded sum stays within a
        # small fraction of the eps^2 ||X||^2 budget of the FP64 path's
        assert abs(dmx - d64) <= 0.02 * eps ** 2 * r64.norm_sq, (eps, dmx, d64)
        r64.close()
        rmx.close()


def test_large_mixed_path_full_size(ctx):
    dims, core = (500, 500, 500, 11, 8), (60, 60, 60, 11, 6)
    x = synth.tucker_torch(dims, core, decay=0.08, eta=1e-7, seed=0)
    rng = np.random.default_rng(2)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, dims[0], size=(4, 2))]
    samples = _mode0_gram_samples(x, dims, pairs)
    S = host(ctx.gram(x, dims, 0, "fp32"))
    _check_gram_samples(S, samples, 2e-6)
    del S
    S = host(ctx.gram(x, dims, 0, "fp64"))
    _check_gram_samples(S, samples, 1e-12)
    del S
    r64 = ctx.sthosvd(x, dims, eps=1e-4, prec="fp64")
    rmx = ctx.sthosvd(x, dims, eps=1e-4, prec="mixed")
    assert rmx.ranks == r64.ranks
    assert rmx.gram_kernel[0] == "tcgen05-x3" and rmx.ttm_kernel[0] == "tcgen05"
    err = math.sqrt(sum(rmx.discarded) / rmx.norm_sq)
    assert err <= 1e-4
    # Cor. 1: ||X - Xhat||^2 = sum of the discarded eigenvalues (relative to
    # ||X||^2) -- the explicit error of the full reconstruction, computed on
    # the device from the library's own multi-TTM
    full = rmx.reconstruct((0,) * 5, dims)
    diff2 = 0.0
    step = 1 << 28
    for a in range(0, x.numel(), step):
        diff2 += float(((x[a:a + step].double() - full[a:a + step].double()) ** 2).sum())
    del full
    # the estimate sums eigenvalues of FP32-product Grams, whose tails carry
    # up to ~1% of a threshold each (err^2 is ~5 thresholds here): 1%
    assert abs(math.sqrt(diff2 / rmx.norm_sq) - err) <= 1e-2 * err
    # the 500x500x500x11x1 slice at sampled entries against the oracle
    b, e = (0, 0, 0, 0, 0), (500, 500, 500, 11, 1)
    got = rmx.reconstruct(b, e).view(1, 11, 500, 500, 500)
    core_h, F = host(rmx.core), [host(f) for f in rmx.factors]
    idx = rng.integers(0, 500, size=(24, 3))
    for i0, i1, i2 in idx:
        i3 = int(rng.integers(0, 11))
        bb = (int(i0), int(i1), int(i2), i3, 0)
        ee = (int(i0) + 1, int(i1) + 1, int(i2) + 1, i3 + 1, 1)
        want, _ = oracle.reconstruct(core_h.astype(np.float64), rmx.ranks, F, bb, ee)
        g = float(got[0, i3, int(i2), int(i1), int(i0)])
        assert abs(g - float(want[0])) <= 1e-5 * math.sqrt(rmx.norm_sq / x.numel()) * 10
    r64.close()
    rmx.close()
