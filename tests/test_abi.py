"""CPU checks of the C ABI boundary: the in-tree library loads and exports
every function that include/tucker_gb300.h declares (no compute calls, so
no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tucker_gb300.h")
LIB = os.path.join(ROOT, "paper_1901_06043_gb300", "libtucker_gb300.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tucker_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["tucker_sthosvd", "tucker_reconstruct", "tucker_create", "tucker_destroy",
                 "tucker_result_destroy", "tucker_last_error", "tucker_gram", "tucker_eig",
                 "tucker_rank_cut", "tucker_ttm", "tucker_multi_ttm", "tucker_norm_sq"]:
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    if not os.path.exists(LIB):
        pytest.fail("libtucker_gb300.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1901_06043_gb300 import tucker
    assert sorted(tucker.EXPORTS) == declared_functions()


def test_binding_types_every_call_that_takes_arguments():
    """Every entry point the binding calls with arguments has its ctypes
    argument types set (an untyped call cannot pass a double)."""
    from paper_1901_06043_gb300 import tucker
    L = tucker.lib()
    no_args = {"tucker_kernel_launches", "tucker_autotune_entries"}
    untyped = [n for n in tucker.EXPORTS if n not in no_args and getattr(L, n).argtypes is None]
    assert not untyped, untyped


def test_ttm_order_host_call_matches_oracle():
    """tucker_ttm_order is host-only C code: check it against the oracle's
    exhaustive search (Section 8.5's 43120 optimum) without a GPU."""
    import oracle
    from paper_1901_06043_gb300 import tucker
    for core in [(30, 38, 35, 6, 11), (95, 129, 125, 7, 125), (3, 4, 2), (5, 1, 7, 2)]:
        out = (500, 500, 500, 1, 1)[:len(core)] if len(core) == 5 else tuple(c + 3 for c in core)
        assert tucker.ttm_order(core, out, "flops") == oracle.best_order(core, out, "flops")[0]
        assert tucker.ttm_order(core, out, "memory") == oracle.best_order(core, out, "memory")[0]


def test_sthosvd_order_host_call_matches_oracle():
    """tucker_sthosvd_order is host-only C code: its order costs exactly the
    oracle's exhaustive minimum of the Section 6 flop count."""
    import math

    import numpy as np

    import oracle
    from paper_1901_06043_gb300 import tucker
    rng = np.random.default_rng(4)
    cases = [((500, 500, 500, 11, 8), (54, 54, 54, 11, 6)), ((100, 100, 100), (100, 1, 100)),
             ((9,), (3,))]
    for _ in range(60):
        N = int(rng.integers(2, 6))
        dims = tuple(int(v) for v in rng.integers(2, 80, size=N))
        cases.append((dims, tuple(int(rng.integers(1, d + 1)) for d in dims)))
    for dims, ranks in cases:
        got = tucker.sthosvd_order(dims, ranks)
        assert sorted(got) == list(range(len(dims)))
        _, best = oracle.best_sthosvd_order(dims, ranks)
        assert math.isclose(oracle.sthosvd_flops(dims, ranks, got), best, rel_tol=1e-12)
    with pytest.raises(tucker.TuckerError):
        tucker.sthosvd_order((5, 4), (6, 1))
