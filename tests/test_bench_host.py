"""The bench's roofline arithmetic on the host: the dominant kernel, its algorithmic work per launch
(the per-unit figures the design states: K6 8 lane-ops per evaluated pair + 10 per blended pair,
K9+K10 1 416 B per Gaussian + 48 B per instance + 8 B per record, ...), achieved = work / the
kernel's time, frac = achieved / the measured peak."""
import pytest

import bench

STATS = {"pairs": 63_000_000.0, "blended": 6_000_000.0, "instances": 335_000.0, "visible": 96_000}
N = 200_000
PEAKS = {"hbm_gbs": 6793.4, "sm_max_mhz": 2070.0}


def per_kernel_ms(dom_k6=True):
    ms = [0.024, 0.012, 0.016, 0.053, 0.012, 0.118, 0.082, 0.094, 0.084]
    if not dom_k6:
        ms[8] = 0.2
    return ms


def test_blend_forward_is_dominant_and_measured_against_the_fp32_issue_peak():
    steps = 10
    kms = [x * steps for x in per_kernel_ms()]
    rl = bench.roofline(kms, steps, STATS, N, 5, PEAKS, "measured", {"K6 blend fwd": 21.8e6}, n_sms=152)
    assert rl["kernel"] == "K6 blend fwd" and rl["bound"] == "alu"
    work = 8.0 * STATS["pairs"] + 10.0 * STATS["blended"]
    assert rl["work_per_launch"] == pytest.approx(work)
    peak = 152 * 128 * 2070e6 / 1e12
    assert rl["peak"] == pytest.approx(peak)
    assert rl["achieved"] == pytest.approx(work / 0.118e-3 / 1e12)
    assert rl["frac"] == pytest.approx(rl["achieved"] / peak)
    assert rl["traffic"] == 21.8e6
    # the scope table's own count for K6, 16 FP32 instructions per evaluated pair, beside it
    assert rl["survey_count"]["work_per_launch"] == pytest.approx(16.0 * STATS["pairs"])
    assert rl["survey_count"]["frac"] == pytest.approx(16.0 * STATS["pairs"] / 0.118e-3 / 1e12 / peak)
    # the SM count comes from the device (here given): another count scales the peak
    rl2 = bench.roofline(kms, steps, STATS, N, 5, PEAKS, "measured", {}, n_sms=76)
    assert rl2["peak"] == pytest.approx(peak / 2) and rl2["n_sms"] == 76
    # every kernel has its own fraction on its own bound
    assert set(rl["per_kernel_frac"]) == set(bench.KERNELS)
    assert rl["per_kernel_frac"]["K8 blend bwd"]["bound"] == "alu"
    assert rl["per_kernel_frac"]["K4 sort"]["bound"] == "hbm"


def test_an_hbm_bound_dominant_kernel_uses_the_measured_copy_bandwidth():
    steps = 4
    kms = [x * steps for x in per_kernel_ms(dom_k6=False)]
    rl = bench.roofline(kms, steps, STATS, N, 5, PEAKS, "measured", {}, n_sms=152)
    assert rl["kernel"] == "K9+K10 project bwd + Adam" and rl["bound"] == "hbm"
    work = 1416.0 * N + 48.0 * STATS["instances"] + 8.0 * N
    assert rl["work_per_launch"] == pytest.approx(work)
    assert rl["achieved"] == pytest.approx(work / 0.2e-3 / 1e9)
    assert rl["frac"] == pytest.approx(rl["achieved"] / 6793.4)
    assert rl["traffic"] is None
