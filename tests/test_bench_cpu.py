"""Host logic of bench.py on the CPU: the roofline arithmetic, the stored
traffic figures and the workload definitions it reports against."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads  # noqa: E402


def test_fp64_roofline_counts_algorithmic_flops_against_the_derived_peak():
    pts, ms = 128 ** 3, 0.5
    r = bench.roofline_for("fp64", pts, ms, 6672.5, traffic=1.7e8)
    achieved = bench.FP64_FLOP_PER_POINT * pts / (ms * 1e-3) / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(achieved)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(achieved / r["peak"])
    assert r["traffic"] == 1.7e8
    # the HBM view alongside: 80 algorithmic bytes per point against the measured copy peak
    hv = r["hbm_view"]
    assert hv["bytes_per_point"] == 80
    assert hv["achieved"] == pytest.approx(80 * pts / (ms * 1e-3) / 1e9)
    assert hv["frac"] == pytest.approx(hv["achieved"] / 6672.5)


def test_fp32_roofline_is_hbm_bound_and_names_the_kernel_form():
    pts, ms = 256 ** 3, 0.21
    for form in (3,):
        r = bench.roofline_for("fp32", pts, ms, 6672.5, None, form)
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["achieved"] == pytest.approx(56 * pts / (ms * 1e-3) / 1e9)
        assert r["frac"] == pytest.approx(r["achieved"] / 6672.5)
        assert r["kernel"].startswith(bench.F32_FORMS[form].split(" ")[0])
        assert r["traffic"] is None


def test_flop_count_is_the_sum_of_its_parts():
    # rates 144 (7 + 15 + 18 + 5 + 8 + 2 + 24 + 16 + 17 + 17 + 13 + 2), update 11, sums 10, spectral 25
    rates = 7 + 15 + 18 + 5 + 8 + 2 + 24 + 16 + 17 + 17 + 13 + 2
    assert rates == 144
    assert bench.FP64_FLOP_PER_POINT == rates + 11 + 10 + 25


def test_traffic_entries_are_keyed_by_a_compiled_shape_and_are_near_the_algorithmic_bytes():
    for (prec, wl, blocks, shape), traffic in bench.TRAFFIC.items():
        if wl == "cfg4":  # the batch: halos of many small tiles re-read from DRAM
            pts = sum(a * b * c for a, b, c in (cv["n"] for cv in workloads.batch_cavities()))
            hi = 1.5
        else:
            n = bench.WORKLOADS[wl]["n"]
            pts, hi = n[0] * n[1] * n[2], 1.2
        algorithmic = bench.BYTES_PER_POINT[prec] * pts
        assert 0.95 * algorithmic <= traffic <= hi * algorithmic, (prec, wl, traffic / algorithmic)
        if prec == "fp64":
            assert shape == bench.FP64_SHAPE
        else:
            ty, kc, r, form = (int(x) for x in shape.split(","))
            assert form == 3 and ty in (8, 16) and r in (4, 5) and kc > 0


def test_batch_workload_is_deterministic_and_in_range():
    a = workloads.batch_cavities()
    b = workloads.batch_cavities()
    assert a == b and len(a) == 64
    for c in a:
        assert all(24 <= d <= 96 for d in c["n"])
        assert 1e3 <= c["Ra"] <= 1e6


def test_default_arguments_give_the_headline_workload():
    args = bench.parse([])
    assert (args.gpus, args.precision, args.workload, args.impl) == (1, "fp64", "cfg2", "ours")
    assert args.warmup >= 3 and args.steps > 0
