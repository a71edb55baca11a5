"""Host-side checks of bench.py's roofline arithmetic (no GPU).

The per-step roofline rows the benchmark prints are computed from the
library's per-mode times; these tests feed `step_rooflines` a synthetic
result with known times and check the algorithmic work, the peaks and the
scaled ncu traffic against hand-computed values.
"""
import os
import sys
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PK = {"hbm_gbs": 6800.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1700.0, "src": "test"}


def _result(dims, ranks, gram, ttm, eig, order=None, eig_kernel=None, gms=None, tms=None):
    N = len(dims)
    return types.SimpleNamespace(
        ranks=tuple(ranks),
        mode_order=tuple(range(N)) if order is None else tuple(order),
        gram_kernel=tuple(gram), ttm_kernel=tuple(ttm),
        eig_kernel=tuple(eig_kernel or ["tridiag"] * N),
        sweeps=(0,) * N, core_dtype=0,
        ms={"gram": list(gms or [10.0] * N), "ttm": list(tms or [2.0] * N), "eig": [1.0] * N})


def _row(rows, name):
    return next(r for r in rows if r["kernel"] == name)


def test_digit_gram_row():
    """tcgen05-x3 Gram: rated on its algorithmic work, I(I+1)K flops and
    4 I K bytes, against whichever of the HBM and BF16 peaks binds (HBM for
    a 500-row Gram); executed digit products (9 x 2 x 128^2 per column per
    lower-triangle tile) as a separate MMA diagnostic; traffic scaled from
    the capture by I*K."""
    w = {"dims": (500, 500, 40, 11, 2), "dtype": "f32"}
    res = _result(w["dims"], (54, 54, 40, 11, 2),
                  ["tcgen05-x3", "tcgen05-x3", "small-fp64", "small-fp64", "small-fp64"],
                  ["tcgen05", "tcgen05", "simt-fp32", "simt-fp32", "simt-fp32"],
                  eig=None, gms=[1.25, 1, 1, 1, 1])
    rows = bench.step_rooflines(res, w, PK)
    g = _row(rows, "gram mode 0 (tcgen05-x3)")
    I, K = 500, 500 * 40 * 11 * 2
    t = 1.25e-3
    # HBM floor 4IK / 6800 GB/s = 0.129 ms > flop floor I(I+1)K / 1800 TF/s = 0.061 ms
    assert g["bound"] == "hbm" and g["unit"] == "GB/s"
    assert g["achieved"] == pytest.approx(4 * I * K / t / 1e9)
    assert g["peak"] == 6800.0
    assert g["frac"] == pytest.approx((4 * I * K / 6800e9) / t)
    assert g["mma_tflops"] == pytest.approx(9 * 2 * 128 * 128 * K * 10 / t / 1e12)
    assert g["mma_frac"] == pytest.approx(g["mma_tflops"] / 1800.0)
    cap = bench.CAPTURED_TRAFFIC[("gram", "tcgen05-x3", "col")]
    assert g["traffic"] == pytest.approx(cap["bytes"] * I * K / cap["elems"])
    assert g["algorithmic_bytes"] == 4 * I * K


def test_flop_bound_row():
    """A Gram whose flops outweigh its bytes at the peaks is tensor-bound:
    I = 8192 rows, I(I+1)K / 1800 TF/s > 4 I K / 6800 GB/s."""
    w = {"dims": (8192, 3000), "dtype": "f32"}
    res = _result(w["dims"], (10, 3000), ["simt-fp32", "simt-fp32"], ["simt-fp32", "simt-fp32"],
                  eig=None, gms=[1.0, 1.0])
    g = _row(bench.step_rooflines(res, w, PK), "gram mode 0 (simt-fp32)")
    I, K = 8192, 3000
    assert g["bound"] == "tensor" and g["peak"] == 1800.0
    assert g["frac"] == pytest.approx(I * (I + 1) * K / 1800e12 / 1e-3)


def test_rotated_layout_uses_column_captures_for_later_modes():
    """Natural mode order: every mode runs column-mode kernels, so mode 1's
    tensor-core TTM gets the column-mode capture's traffic; another order
    (row-mode views) gets none."""
    w = {"dims": (500, 500, 40, 11, 2), "dtype": "f32"}
    kern = (["tcgen05-x3", "tcgen05-x3", "small-fp64", "small-fp64", "small-fp64"],
            ["tcgen05", "tcgen05", "simt-fp32", "simt-fp32", "simt-fp32"])
    rows = bench.step_rooflines(_result(w["dims"], (54, 54, 40, 11, 2), *kern, eig=None), w, PK)
    t1 = _row(rows, "ttm mode 1 (tcgen05)")
    # mode 1 input: 54 x 500 x 40 x 11 x 2 -> I = 500, K = 54 * 880
    cap = bench.CAPTURED_TRAFFIC[("ttm", "tcgen05", "col")]
    assert t1["traffic"] == pytest.approx(cap["bytes"] * 500 * 54 * 880 / cap["elems"])
    rows = bench.step_rooflines(_result(w["dims"], (54, 54, 40, 11, 2), *kern, eig=None,
                                        order=(0, 2, 1, 3, 4)), w, PK)
    assert _row(rows, "ttm mode 1 (tcgen05)")["traffic"] is None


def test_hbm_and_alu_rows():
    """TTM rows are rated on read + write bytes and 2RIK flops (HBM-bound
    here); the tridiagonal eigensolve counts (4/3) I^3 FP64 flops."""
    w = {"dims": (256, 300, 9), "dtype": "f32"}
    res = _result(w["dims"], (30, 40, 9), ["tcgen05-x3", "simt-fp32", "small-fp64"],
                  ["tcgen05", "simt-fp32", "simt-fp32"], eig=None, tms=[0.5, 0.25, 0.1])
    rows = bench.step_rooflines(res, w, PK)
    t0 = _row(rows, "ttm mode 0 (tcgen05)")
    I, K, R = 256, 300 * 9, 30
    assert t0["bound"] == "hbm"
    assert t0["achieved"] == pytest.approx((4 * I * K + 4 * R * K) / 0.5e-3 / 1e9)
    assert t0["peak"] == 6800.0
    t1 = _row(rows, "ttm mode 1 (simt-fp32)")
    # mode 1 after mode 0: I = 300, K = 30 * 9 (rank of mode 0 times the rest), R = 40
    nb = 4 * 300 * 270 + 4 * 40 * 270
    assert t1["bound"] == "hbm" and t1["peak"] == 6800.0
    assert t1["achieved"] == pytest.approx(nb / 0.25e-3 / 1e9)
    e0 = _row(rows, "eig mode 0 (fp64-tridiag)")
    assert e0["bound"] == "alu"
    assert e0["achieved"] == pytest.approx((4.0 / 3.0) * 256 ** 3 / 1e-3 / 1e12)


def test_reconstruction_row_is_rated_on_its_output():
    w = {"recon": (500, 500, 500, 11, 1)}
    r = bench.recon_roofline((54, 54, 54, 11, 6), w, 3.0, 4 * 500 ** 3 * 11, "mixed", PK)
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(4 * 500 ** 3 * 11 / 3e-3 / 1e9)
    assert r["frac"] == pytest.approx(4 * 500 ** 3 * 11 / 6800e9 / 3e-3)
