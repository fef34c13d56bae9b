"""Host-side bookkeeping of bench.py (no GPU): the per-kernel algorithmic
bytes add up to the step's, the dominant-kernel roofline arithmetic, the
ncu-traffic lookup that refuses figures taken on other kernel sources, and
the end-to-end block that reports the fastest measured variant."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

STEP_KERNELS = ("rows_r2c_image", "lines_fwd_image", "dec_lines", "rows_c2r_coeffs",
                "rows_r2c_coeffs", "rec_lines", "rows_c2r_image")


@pytest.mark.parametrize("B,K,N,M,s", [(16, 49, 512, 512, 4), (16, 49, 512, 512, 2),
                                       (3, 17, 256, 128, 4), (1, 1, 16, 16, 2)])
def test_kernel_bytes_add_up_to_the_step(B, K, N, M, s):
    dec, rec = bench._algorithmic_bytes(B, K, N, M, s)
    per_kernel = sum(bench.kernel_alg_bytes(k, B, K, N, M, s) for k in STEP_KERNELS)
    assert per_kernel == dec + rec
    # the alternative column pass of the bfloat16 decomposition counts the same bytes
    assert bench.kernel_alg_bytes("dec_lines_tc", B, K, N, M, s) == \
        bench.kernel_alg_bytes("dec_lines", B, K, N, M, s)


def test_roofline_picks_the_dominant_kernel():
    B, K, N, M, steps = 16, 49, 512, 512, 10
    prof = {"rows_r2c_coeffs": {"launches": steps, "ms": 3.0},
            "rows_c2r_coeffs": {"launches": steps, "ms": 2.7},
            "dec_lines": {"launches": steps, "ms": 2.1}}
    r = bench.roofline(prof, steps, B, K, N, M, 4, 6683.5, "measured")
    assert r["kernel"] == "rows_r2c_coeffs"
    alg = B * K * N * M * 4                        # the coefficient read
    assert r["algorithmic_bytes_per_launch"] == alg
    assert r["launch_ms"] == pytest.approx(0.3)
    assert r["achieved"] == pytest.approx(alg / 0.3e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6683.5)
    assert bench.roofline({}, steps, B, K, N, M, 4, 1.0, "x") is None


def test_profiled_traffic_only_for_the_profiled_sources(monkeypatch):
    # the committed summary of the dominant kernel carries the source hash
    # it was captured on; the figure is reported only while it matches
    cur = bench.kernel_source_hash()
    text = open(os.path.join(ROOT, "profiles", "rows_r2c_coeffs_512_k49.md")).read()
    if "source_sha256_16: %s" % cur in text:
        t = bench._profiled_traffic("rows_r2c_coeffs")
        assert t is not None and 1.0e6 < t < 4.0e6     # bytes per subband
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench._profiled_traffic("rows_r2c_coeffs") is None
    assert bench._profiled_traffic("no_such_kernel") is None


def test_e2e_block_reports_the_fastest_variant():
    units = 1000.0
    blk = bench._e2e_block(units, 64, [(2.0e-3, "a", 1e-7), (1.0e-3, "b", 2e-7),
                                       (3.0e-3, "c", None)])
    assert blk["value"] == pytest.approx(units / 1.0e-3)
    assert blk["transfer"] == "b" and blk["max_rel_err"] == 2e-7
    assert blk["h2d_bytes_per_step"] == 64 and blk["d2h_bytes_per_step"] == 64
    assert [v["transfer"] for v in blk["variants"]] == ["a", "b", "c"]
    assert blk["variants"][2]["ms_per_step"] == pytest.approx(3.0)
