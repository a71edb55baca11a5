"""Error paths of the library on the GPU, made without faulting it.

- The eigensolvers' grid barriers are bounded: under a tiny poll limit
  (TUCKER_OPT_BARRIER_POLLS) the CTAs give up instead of waiting, the call
  returns TUCKER_ERR_CUDA with the barrier message, and the next call with
  the default limit on the same context succeeds.  (The TMA / tensor-core
  kernels are not driven to their limits: an early exit there could leave
  bulk copies in flight.)
- Out of memory is predicted from the workspace formula before anything is
  launched or allocated (TUCKER_OPT_MEM_LIMIT stands in for the free-memory
  figure), both for the first mode and for a later TTM.
- The tridiagonal solver's hand-written FP64 reciprocal (an FP32 seed and
  two Newton-Raphson steps) is within one ulp of the correctly rounded 1/x
  over the exponent range, signs included.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx():
    from paper_1901_06043_gb300 import tucker
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = tucker.Context()
    yield c
    c.close()


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return torch.from_numpy(A @ A.T + n * np.eye(n)).cuda()


@pytest.mark.parametrize("solver", ["tridiag", "jacobi"])
def test_grid_barrier_timeout_returns_an_error_and_the_context_recovers(ctx, solver):
    from paper_1901_06043_gb300 import tucker
    S = _spd(500, 3)                       # tridiagonal: a team of several CTAs
    ctx.set_option(tucker.OPT_EIG_SOLVER, tucker.EIG_SOLVER[solver])
    ctx.set_option(tucker.OPT_BARRIER_POLLS, 1)
    with pytest.raises(tucker.TuckerError) as e:
        if solver == "jacobi":
            ctx.eig(S)
        else:
            ctx.eig_trunc(S, 0.0, 10)
    assert e.value.name == "CUDA" and "barrier gave up" in str(e.value)
    ctx.set_option(tucker.OPT_BARRIER_POLLS, 1 << 24)
    w, U, R, _ = ctx.eig_trunc(S, 0.0, 10)
    want, _ = oracle.eig_desc(S.cpu().numpy())
    assert R == 10
    assert np.abs(w.cpu().numpy() - want).max() <= 1e-10 * want[0]


def test_oom_predicted_before_any_launch(ctx):
    from paper_1901_06043_gb300 import tucker
    dims = (40, 50, 30)
    x, _ = synth.tucker_numpy(dims, (5, 6, 4), eta=1e-4, seed=0)
    xd = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    ctx.set_option(tucker.OPT_MEM_LIMIT, 1000)      # below the 40 KB of Gram matrices
    n0 = tucker.kernel_launches()
    with pytest.raises(tucker.TuckerError) as e:
        ctx.sthosvd(xd, dims, eps=1e-3, prec="fp64")
    assert e.value.name == "OOM" and "predicted" in str(e.value)
    assert tucker.kernel_launches() == n0
    ctx.set_option(tucker.OPT_MEM_LIMIT, 0)
    res = ctx.sthosvd(xd, dims, eps=1e-3, prec="fp64")
    assert res.ranks == (5, 6, 4)
    res.close()


def test_oom_predicted_before_a_ttm(ctx):
    """A figure that holds the first mode's minimum (Gram and eigenvector
    matrices, the Gram's split-K scratch, a rank-1 TTM output) but not the
    TTM output at the rank the cut asks for: the call stops there with a
    predicted OOM.  The boundary is found by bisection on the figure."""
    from paper_1901_06043_gb300 import tucker
    dims = (64, 64, 2000)
    x, _ = synth.tucker_numpy(dims, (40, 10, 10), decay=0.01, eta=1e-4, seed=1)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.sthosvd(x, dims, eps=1e-3)
    assert ref["ranks"][0] >= 30            # a mode-0 output of >= 30 MB in FP64
    res = ctx.sthosvd(xd, dims, eps=1e-3, prec="fp64")
    assert res.ranks == ref["ranks"]
    res.close()

    def outcome(limit):
        ctx.set_option(tucker.OPT_MEM_LIMIT, limit)
        try:
            ctx.sthosvd(xd, dims, eps=1e-3, prec="fp64").close()
            return "ok"
        except tucker.TuckerError as e:
            assert e.name == "OOM" and "predicted" in str(e), str(e)
            return "first" if "first mode" in str(e) else "ttm"

    lo, hi = 1000.0, 4e9
    assert outcome(lo) == "first" and outcome(hi) == "ok"
    while hi - lo > 1.0:
        mid = 0.5 * (lo + hi)
        if outcome(mid) == "first":
            lo = mid
        else:
            hi = mid
    # just above the first mode's minimum, the rank-R output does not fit
    assert outcome(hi) == "ttm"
    ctx.set_option(tucker.OPT_MEM_LIMIT, 0)


def test_rcp64_within_one_ulp():
    from paper_1901_06043_gb300 import tucker
    rng = np.random.default_rng(5)
    e = rng.uniform(-1020, 1020, 200000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(np.int64))
    x *= np.where(rng.random(e.size) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, [1.0, -1.0, 2.0, 0.75, 1.5, np.nextafter(2.0, 1.0), 3.0, 1e-300,
                            1e300, 5e-310, np.finfo(np.float64).max]])
    y = tucker.selftest_rcp64(torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(over="ignore", divide="ignore"):
        want = 1.0 / x
    fin = np.isfinite(want)
    assert np.array_equal(y[~fin], want[~fin])      # reciprocals of subnormals overflow
    ulp = np.spacing(np.abs(want[fin]))
    err = np.abs(y[fin] - want[fin])
    assert np.all(err <= ulp), np.max(err / ulp)
