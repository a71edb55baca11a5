"""ST-HOSVD of a tensor in host memory (tucker_sthosvd_host) against the FP64
oracle and against the device-input path, through the C ABI.

The library copies the input in pieces and runs the norm pass and, when
mode 0 comes first, the mode-0 Gram on each piece as it lands (summed in
FP64).  Small pieces (TUCKER_OPT_HOST_CHUNK) make many of them, with a
ragged last one.  Tolerances are those of the device path against the
oracle: ranks identical; discarded sums within 1e-10 ||X||^2 (FP64), 2e-10
||X||^2 (FP32 products) or 2 % of the threshold eps^2 ||X||^2 / N (MIXED).  Against the device path the FP64 results agree to
rounding (the only difference is the order of the FP64 Gram and norm sums).
"""
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


@pytest.fixture
def chunk(ctx, request):
    from paper_1901_06043_gb300 import tucker
    ctx.set_option(tucker.OPT_HOST_CHUNK, request.param)
    yield request.param
    ctx.set_option(tucker.OPT_HOST_CHUNK, float(1 << 30))


def _host_tensor(dims, core, dtype, seed, pinned):
    x, _ = synth.tucker_numpy(dims, core, decay=0.1, eta=1e-7, seed=seed)
    x = x.astype(dtype)
    if pinned:
        t = torch.empty(x.size, dtype=torch.float32 if dtype == np.float32 else torch.float64,
                        pin_memory=True)
        t.copy_(torch.from_numpy(x))
        return x, t
    return x, x


def _check_oracle(res, ref, prec):
    assert res.ranks == ref["ranks"], (res.ranks, ref["ranks"])
    assert abs(res.norm_sq - ref["norm_sq"]) <= 1e-12 * ref["norm_sq"]
    thr = ref["threshold"]
    # FP32 products: their rounding leaves up to ~1.5e-10 ||X||^2 on the
    # discarded subspace (the reason tucker_sthosvd computes FP32-precision
    # Grams in FP64 below eps^2 / N = 1e-9)
    tol = {"fp64": 1e-10 * ref["norm_sq"], "fp32": 2e-10 * ref["norm_sq"]}.get(prec, 0.02 * thr)
    for n in range(len(ref["ranks"])):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= tol, (n, res.discarded[n],
                                                                     ref["discarded"][n], thr)


@pytest.mark.parametrize("chunk", [1 << 20], indirect=True)
@pytest.mark.parametrize("prec,pinned", [("fp64", True), ("mixed", True), ("mixed", False),
                                         ("fp32", True)])
def test_host_input_against_the_oracle_and_the_device_path(ctx, chunk, prec, pinned):
    dims, core = (256, 64, 40, 11), (40, 20, 20, 11)
    x, xh = _host_tensor(dims, core, np.float32, 11, pinned)
    ref = oracle.sthosvd(x.astype(np.float64), dims, eps=1e-4)
    res = ctx.sthosvd_host(xh, dims, eps=1e-4, prec=prec)
    _check_oracle(res, ref, prec)
    # 28160 mode-0 columns in pieces of 1024 columns (1 MB): 28 pieces
    dref = ctx.sthosvd(torch.from_numpy(x).cuda(), dims, eps=1e-4, prec=prec)
    assert res.ranks == dref.ranks
    if prec == "fp64":
        for n in range(len(dims)):
            w, wd = res.eigvals[n].cpu().numpy(), dref.eigvals[n].cpu().numpy()
            assert np.abs(w - wd).max() <= 1e-12 * abs(wd).max()
    if prec == "mixed":
        assert res.gram_kernel[0] in ("tcgen05-x3", "tcgen05-x2")
    res.close()
    dref.close()


@pytest.mark.parametrize("chunk", [3 << 18], indirect=True)
def test_host_input_fp64_tensor_and_another_mode_order(ctx, chunk):
    """FP64 input, and a first mode other than 0 (the pieces then carry only
    the norm pass; the first Gram runs on the resident copy)."""
    dims, core = (30, 41, 52, 7), (6, 7, 8, 3)
    x, xh = _host_tensor(dims, core, np.float64, 12, True)
    order = [2, 0, 3, 1]
    ref = oracle.sthosvd(x, dims, eps=1e-5, mode_order=order)
    res = ctx.sthosvd_host(xh, dims, eps=1e-5, mode_order=order, prec="fp64")
    _check_oracle(res, ref, "fp64")
    res.close()
    res = ctx.sthosvd_host(xh, dims, eps=1e-5, prec="fp64")
    _check_oracle(res, oracle.sthosvd(x, dims, eps=1e-5), "fp64")
    res.close()


@pytest.mark.parametrize("chunk", [1 << 20], indirect=True)
def test_host_input_falls_back_to_an_fp64_gram_where_the_bound_asks(ctx, chunk):
    """At eps = 1e-6 the digit bound of this 256 x 28160 view fails: the
    pieces' exact-digit Gram sum is replaced by an FP64 Gram of the resident
    copy, and the cut is the oracle's."""
    dims, core = (256, 64, 40, 11), (40, 20, 20, 11)
    x, xh = _host_tensor(dims, core, np.float32, 11, True)
    ref = oracle.sthosvd(x.astype(np.float64), dims, eps=1e-6)
    res = ctx.sthosvd_host(xh, dims, eps=1e-6, prec="mixed")
    assert res.gram_kernel[0] == "simt-fp64", res.gram_kernel
    assert res.ranks[0] == ref["ranks"][0]
    assert abs(res.discarded[0] - ref["discarded"][0]) <= 0.02 * ref["threshold"]
    res.close()


def test_host_input_rank_specified_and_rejections(ctx):
    from paper_1901_06043_gb300 import tucker
    dims = (64, 20, 9)
    x, xh = _host_tensor(dims, (5, 4, 3), np.float32, 13, False)
    res = ctx.sthosvd_host(xh, dims, ranks=(5, 4, 3), prec="mixed")
    assert res.ranks == (5, 4, 3)
    ref = oracle.sthosvd(x.astype(np.float64), dims, ranks=(5, 4, 3))
    for n in range(3):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 1e-6 * ref["norm_sq"]
    res.close()
    with pytest.raises(ValueError):
        ctx.sthosvd_host(xh[:-1], dims, eps=1e-3)
    with pytest.raises(tucker.TuckerError):
        ctx.sthosvd_host(xh, dims, ranks=(65, 4, 3))
    with pytest.raises(ValueError):
        ctx.sthosvd_host(torch.from_numpy(x).cuda(), dims, eps=1e-3)


def test_host_input_concurrent_calls_on_two_contexts():
    """Two host threads, each with its own context and stream, run the call
    on the same pinned input at once (their input copies then run one after
    the other): both results equal the oracle's, and each other's."""
    import threading
    from paper_1901_06043_gb300 import tucker
    dims, core = (96, 40, 30, 7), (12, 10, 8, 5)
    x, xh = _host_tensor(dims, core, np.float64, 17, True)
    ref = oracle.sthosvd(x, dims, eps=1e-5)
    streams = [torch.cuda.Stream() for _ in range(2)]
    ctxs = []
    for s in streams:
        with torch.cuda.stream(s):
            c = tucker.Context(stream=s.cuda_stream)
        c.set_option(tucker.OPT_HOST_CHUNK, float(1 << 16))
        ctxs.append(c)
    out, errors = [[], []], []

    def run(i):
        try:
            with torch.cuda.stream(streams[i]):
                for _ in range(3):
                    r = ctxs[i].sthosvd_host(xh, dims, eps=1e-5, prec="fp64")
                    core_h, _ = r.to_host()
                    out[i].append((r.ranks, list(r.discarded), core_h.copy()))
                    r.close()
        except Exception as e:
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for c in ctxs:
        c.close()
    assert not errors, errors
    first = out[0][0]
    for i in range(2):
        for ranks, disc, core_h in out[i]:
            assert ranks == ref["ranks"], (ranks, ref["ranks"])
            for n in range(len(dims)):
                assert abs(disc[n] - ref["discarded"][n]) <= 1e-10 * ref["norm_sq"]
            assert ranks == first[0] and disc == first[1]
            np.testing.assert_array_equal(core_h, first[2])
