"""The split-K autotuner (TUCKER_OPT_AUTOTUNE): results of a tuned run match
the oracle exactly as the untuned ones do (the K split only reorders the
FP64 sums of the split partial tiles), the cache gains one entry per new
(kernel, shape) and none on a repeated call, and the batched path, where
the spec workload uses it, agrees with the untuned batch."""
import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture
def tuned():
    from paper_1901_06043_gb300 import tucker
    c = tucker.Context()
    c.set_option(tucker.OPT_AUTOTUNE, 1)
    yield c
    c.close()


def test_autotuned_sthosvd_matches_oracle_and_caches(tuned):
    from paper_1901_06043_gb300 import tucker
    dims = (256, 96, 40, 11)
    x = synth.tucker_torch(dims, (40, 20, 20, 11), decay=0.1, eta=1e-7, seed=8)
    n0 = tucker.autotune_entries()
    res = tuned.sthosvd(x, dims, eps=1e-4, prec="mixed")
    n1 = tucker.autotune_entries()
    assert n1 > n0
    ref = oracle.sthosvd(host(x), dims, eps=1e-4)
    assert res.ranks == ref["ranks"]
    for n in range(4):
        assert abs(res.discarded[n] - ref["discarded"][n]) <= 0.02 * ref["threshold"]
    again = tuned.sthosvd(x, dims, eps=1e-4, prec="mixed")
    assert tucker.autotune_entries() == n1        # every shape already tuned
    assert again.ranks == res.ranks
    res.close()
    again.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_autotuned_gram_equals_untuned(tuned, prec):
    from paper_1901_06043_gb300 import tucker
    plain = tucker.Context()
    dims = (200, 60, 300) if prec != "mixed" else (256, 60, 300)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(int(np.prod(dims)))).cuda()
    x = x.float() if prec != "fp64" else x
    for mode in range(3):
        a = host(plain.gram(x, dims, mode, prec))
        b = host(tuned.gram(x, dims, mode, prec))
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.abs(a - b).max() <= tol * np.abs(a).max(), (prec, mode)
    plain.close()


def test_autotuned_batch_equals_untuned(tuned):
    from paper_1901_06043_gb300 import tucker
    plain = tucker.Context()
    shapes = [((128, 128, 64), (16, 16, 8)), ((60, 70, 40, 6), (10, 10, 8, 4)),
              ((200, 100, 30), (20, 12, 10))]
    xs, dl = [], []
    for k, (d, c) in enumerate(shapes):
        xs.append(synth.tucker_torch(d, c, decay=0.15, eta=1e-6, seed=50 + k))
        dl.append(d)
    ra = plain.sthosvd_batched(xs, dl, eps=1e-4, prec="mixed")
    rb = tuned.sthosvd_batched(xs, dl, eps=1e-4, prec="mixed")
    for a, b, d in zip(ra, rb, dl):
        assert a.ranks == b.ranks
        thr = a.threshold
        for n in range(len(d)):
            assert abs(a.discarded[n] - b.discarded[n]) <= 0.02 * thr
        a.close()
        b.close()
    plain.close()
