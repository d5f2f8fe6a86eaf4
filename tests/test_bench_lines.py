"""bench.py's host-side pieces that need no GPU: the algorithmic flop
counts behind the roofline, the machine-readable lines of the committed ncu
summaries (traffic per launch, pipe fractions, source hash) and the HBM
check against the measured peaks."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SUMMARIES = [("csst100", "k_loglike"), ("csst100_epl", "k_loglike"), ("slacs120", "k_loglike_nc"),
             ("mge32", "k_loglike_nc")]


def test_flop_counts_scale_with_the_work():
    sep = bench.flops_per_eval(100, 100, 4, 21, True, 10000)
    direct = bench.flops_per_eval(100, 100, 4, 21, False, 10000)
    assert direct > sep > 0
    # csst100 by hand: 10^4 pixels x (16 subpixels x (72 + 9) + 2) + 10^4 x
    # (2 channels x 2 x 42 separable taps + 15 sums)
    assert sep == 10000 * (16 * 81 + 2) + 10000 * (2 * 2 * 42 + 15)
    # half the pixels traced: the per-subpixel part halves, the per-pixel part stays
    half = bench.flops_per_eval(100, 100, 4, 21, True, 5000)
    assert sep / 2 < half < sep
    # supersampling 5 x 5 against 4 x 4: the per-subpixel part grows by 25/16
    assert bench.flops_per_eval(100, 100, 5, 21, True, 10000) > sep


def test_multi_flop_count_by_hand():
    from paper_2503_08586_gb300 import workloads as W
    s = W.MULTI_WORKLOADS["slacs120"]
    got = bench.flops_per_eval_multi(s.ny, s.nx, s.sub, s.psf_size, s.psf_kind == "gaussian",
                                     s.comps)
    # per subpixel: grid 4, SIE + shear + lens equation 37, two planes' frames 14,
    # four Sersics 4 x (13 + 1); per pixel: 4 means, 4 columns x 441 taps x 2,
    # 14 weighted sums x 3
    per_sub = 4 + 37 + 14 + 4 * 14
    assert got == 120 * 120 * (16 * per_sub + 4 + 4 * 441 * 2 + 3 * 14)


@pytest.mark.parametrize("workload,kernel", SUMMARIES)
def test_summary_machine_lines_parse(workload, kernel):
    text = open(os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")).read()
    m = re.search(r"traffic_bytes_per_launch: (\d+) source_hash: ([0-9a-f]{16})", text)
    assert m and int(m.group(1)) > 0
    p = re.search(r"pipes: (.*?) source_hash: ([0-9a-f]{16})", text)
    assert p and p.group(2) == m.group(2)
    f = p.group(1).split()
    vals = dict(zip(f[0::2], map(float, f[1::2])))
    assert set(vals) == {"fma_inst", "xu_inst", "xu_cycles", "alu_cycles", "issue"}
    assert all(0.0 < v <= 1.0 for v in vals.values())
    # the reading functions agree with the text when the sources match it
    if m.group(2) == bench.source_hash(kernel):
        assert bench.captured_traffic(workload, kernel) == float(m.group(1))
        assert bench.captured_pipes(workload, kernel)["issue"] == vals["issue"]


def test_hbm_check_against_measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks in this checkout")
    peak = float(json.load(open(path))["hbm_gbs"])
    h = bench.hbm_check(2.0e9, 1000.0)      # 2 GB in one second
    assert h["peak_gbs"] == peak
    assert h["achieved_gbs"] == pytest.approx(2.0)
    assert h["frac"] == pytest.approx(2.0 / peak)
    assert bench.hbm_check(None, 1.0) is None


def test_source_hash_follows_code_not_comments():
    a = "int f(int x) { return x + 1; }  // one more\n/* block\n comment */"
    b = "int f(int x)\n{\n    return x + 1;   // a different comment\n}\n"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_pipe_peaks_from_device_count_and_sampled_clock():
    p = bench.pipe_peaks({"sm_mhz": 1800.0, "sm_max_mhz": 2070.0}, n_sm=152)
    assert p["mhz"] == 1800.0 and p["n_sm"] == 152
    assert p["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 1800e6 / 1e12)
    assert p["mufu_gops"] == pytest.approx(152 * 16 * 1800e6 / 1e9)
    assert "sampled" in p["basis"]
    # no sample under load: nvidia-smi's maximum clock, then the fallback
    assert bench.pipe_peaks({"sm_mhz": None, "sm_max_mhz": 2070.0}, n_sm=100)["mhz"] == 2070.0
    q = bench.pipe_peaks(None, n_sm=100)
    assert q["mhz"] == bench.SM_MAX_MHZ and "no sample" in q["basis"]


def test_transcendental_counts_and_mufu_roof():
    # csst100: 10^4 pixels x 16 subpixels x 9 (SIE sqrt, atan, atanh; two
    # Sersics' sqrt, pow, exp)
    assert bench.transcendentals_per_eval(4, 10000) == 10000 * 16 * 9
    from paper_2503_08586_gb300 import workloads as W
    s = W.MULTI_WORKLOADS["slacs120"]
    # SLACS: the SIE's 3 plus 4 Sersics x 3 per subpixel
    assert bench.transcendentals_per_eval_multi(s.ny, s.nx, s.sub, s.comps) == \
        s.ny * s.nx * s.sub ** 2 * (3 + 4 * 3)
    peaks = bench.pipe_peaks({"sm_mhz": 2000.0}, n_sm=100)
    r = bench.mufu_roof(3.2e9, 1.0, peaks)           # 3.2e9 evaluations in 1 ms
    assert r["achieved"] == pytest.approx(3.2e3)      # Gop/s
    assert r["frac"] == pytest.approx(3.2e3 / (100 * 16 * 2000e6 / 1e9))
