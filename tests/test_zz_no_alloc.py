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


def test_gram_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1901_06043_gb300 import tucker
    y = torch.zeros(2000 * 3, dtype=torch.float64, device="cuda")
    S = torch.zeros((2000, 2000), dtype=torch.float64, device="cuda")
    with pytest.raises(tucker.TuckerError) as e:
        tucker.gram_noalloc(y, (2000, 3), 0, S, "fp64")
    assert e.value.name == "INVALID"
