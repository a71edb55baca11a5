"""The Gram entry point that allocates nothing (tucker_gram_noalloc).

Some callers cannot call cudaMalloc: their device memory is all owned by
their own allocator, or they run where an allocation must not happen.  For
them the library offers the Gram step with a fixed 16 MiB device scratch
array.  This checks, through the C ABI, that two calls in a row give what the
allocating tucker_gram gives, within the tolerances of the Gram parity tests.
It is collected last on purpose, and passes alone in a fresh process too
(the first call sets the scratch address up).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,prec,tol", [(torch.float64, "fp64", 1e-13),
                                            (torch.float32, "fp32", 1e-6)])
def test_gram_noalloc_matches_tucker_gram_twice(dtype, prec, tol):
    from paper_1901_06043_gb300 import tucker
    ctx = tucker.Context()
    for dims in [(65, 9, 4), (200, 300), (3, 130, 7)]:
        x = np.random.default_rng(len(dims) + dims[0]).standard_normal(int(np.prod(dims)))
        y = torch.from_numpy(x).to(device="cuda", dtype=dtype)
        for n in range(len(dims)):
            want = ctx.gram(y, dims, n, prec).cpu().numpy()
            scale = np.abs(want).max() * (max(1, math.log2(y.numel())) if prec == "fp64" else 1)
            for _ in range(2):   # two calls in a row share and reuse the scratch
                S = torch.full((dims[n], dims[n]), float("nan"), dtype=torch.float64, device="cuda")
                tucker.gram_noalloc(y, dims, n, S, prec)
                torch.cuda.synchronize()
                got = S.cpu().numpy()
                assert np.abs(got - want).max() <= tol * scale, (dims, n)
    ctx.close()


def test_gram_noalloc_fewer_splits_when_the_scratch_caps_them():
    # I_n = 1000 has 136 lower-triangle tiles of 64 x 64 FP64 (4.46 MB per K
    # split); the allocating planner wants 5 splits for a 4096-column K
    # (22 MB), which the 16 MiB array cannot hold, so this call runs 3.
    from paper_1901_06043_gb300 import tucker
    ctx = tucker.Context()
    dims = (1000, 4096)
    x = np.random.default_rng(7).standard_normal(int(np.prod(dims)))
    for dtype, prec, tol in [(torch.float64, "fp64", 1e-13), (torch.float32, "fp32", 1e-6)]:
        y = torch.from_numpy(x).to(device="cuda", dtype=dtype)
        want = ctx.gram(y, dims, 0, prec).cpu().numpy()
        scale = np.abs(want).max() * (max(1, math.log2(y.numel())) if prec == "fp64" else 1)
        for _ in range(2):
            S = torch.full((1000, 1000), float("nan"), dtype=torch.float64, device="cuda")
            tucker.gram_noalloc(y, dims, 0, S, prec)
            torch.cuda.synchronize()
            assert np.abs(S.cpu().numpy() - want).max() <= tol * scale, prec
    ctx.close()


def test_gram_noalloc_rejects_sizes_beyond_its_scratch():
    # nothing is launched and nothing is written for a size it cannot hold
    from paper_1901_06043_gb300 import tucker
    y = torch.zeros(2000 * 3, dtype=torch.float64, device="cuda")
    S = torch.full((2000, 2000), 7.25, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    n0 = tucker.kernel_launches()
    with pytest.raises(tucker.TuckerError) as e:
        tucker.gram_noalloc(y, (2000, 3), 0, S, "fp64")
    assert e.value.name == "INVALID"
    torch.cuda.synchronize()
    assert tucker.kernel_launches() == n0
    assert bool((S == 7.25).all())
