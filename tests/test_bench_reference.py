"""The benchmark's reference arm (the CPU oracle) runs without a GPU: one
JSON line with the contract's keys, on a reduced workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--n", "20000"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "evals/s"
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
                "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_other_ranks_of_the_reference_arm_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--n", "20000"], capture_output=True, text=True, cwd=ROOT, env=env,
                         timeout=600)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_clock_summary_of_nvidia_smi_rows():
    """The clocks record of the JSON line: median SM clock under load, the
    largest max clock, and every throttle reason reported Active."""
    import bench
    rows = [
        ["0", "2070", "2070", "850.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1980", "2070", "1390.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2055", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"],
        ["0", "2070"],                                   # a truncated line is ignored
    ]
    c = bench.summarize_clocks(rows)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = rows[:1] + [["0", "1200", "2070", "1400", "0x40", "Not Active", "Active", "Not Active", "Not Active"]]
    assert bench.summarize_clocks(hot)["reasons"] == ["hw_thermal_slowdown"]
    assert bench.summarize_clocks([])["sm_mhz"] is None


def test_lower_bound_roofline_record():
    """Roofline arithmetic of the benchmark line: 4KD + K FP32 lane
    operations per node x sample (packed subtraction 2, 3-input max 1, half a
    packed FMA 1 per cluster and attribute; one min or max per cluster)
    against SMs x 128 lanes x clock; the measured probe rate beside it; the
    DRAM traffic of a full launch scaled from the N = 5e6 capture."""
    import bench
    r = bench.lb_roofline(11.5, 10_000_000, 8, 5, 256, 152, 2070.0, 2070.0, (4, 256),
                          probe={"fma2_tops": 40.0, "max3_tops": 39.0, "lb_mix_tops": 38.0})
    achieved = (4 * 5 * 8 + 5) * 256 * 1e7 / 11.5e-3 / 1e12
    assert r["ops_per_eval"] == 165
    assert abs(r["achieved"] - achieved) < 1e-9 and abs(r["peak"] - 152 * 128 * 2070e6 / 1e12) < 1e-9
    assert abs(r["frac"] - achieved / r["peak"]) < 1e-12 and 0.9 < r["frac"] < 0.92
    assert abs(r["frac_of_probe"] - achieved / 38.0) < 1e-12
    assert r["traffic"] == 2 * 160_336_896 + 3_938_304 and r["bound"] == "alu"
    assert abs(r["hbm_gbs"] - 1e7 * 8 * 4 / 11.5e-3 / 1e9) < 1e-9
    other = bench.lb_roofline(11.5, 10_000_000, 8, 5, 256, 152, None, 1965.0, (2, 256))
    assert other["traffic"] is None and "fallback" in other["peak_basis"] and "1965" in other["peak_basis"]
    assert "frac_of_probe" not in other
