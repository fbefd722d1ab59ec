"""Host-side arithmetic of bench.py, on CPU: the algorithmic work per node behind the roofline,
the committed ncu record and its staleness check, the clock-sample summary and the bounded
oracle sample."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

RECORD = os.path.join("profiles", "dram_traffic_advected_wave_512x512_p3.json")


def test_volume_kernel_work_per_node_of_the_bench_workload():
    """2D, p = 3, ideal EOS, closed-form recovery: 120 (con2prim) + 14 (two nodal fluxes of 7)
    + 80 (2 N flops x 5 variables x 2 directions) + 40 (four face lines of N = 4 nodes among
    16, 5 variables, 2 N flops each) = 254 flops per node."""
    spec = bench.make_spec("advected_wave")
    assert (spec["dim"], spec["degree"], spec["eos"], spec["c2p"]) == (2, 3, "ideal", "analytic")
    assert bench.volume_kernel_flops_per_node(spec) == 254.0
    # the iterative solvers grow by their per-iteration cost
    it = dict(spec, c2p="iterative")
    assert bench.volume_kernel_flops_per_node(it, 5.0) - bench.volume_kernel_flops_per_node(it, 4.0) == 19.0
    tm = dict(spec, eos="tm", c2p="iterative")
    assert bench.volume_kernel_flops_per_node(tm, 3.0) - bench.volume_kernel_flops_per_node(tm, 2.0) == 14.0


def _copy_record_tree(dst):
    d = json.load(open(os.path.join(ROOT, RECORD)))
    for f in [RECORD] + d["source_files"]:
        os.makedirs(os.path.join(dst, os.path.dirname(f)), exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))
    return d


def test_capture_record_is_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    d = _copy_record_tree(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    fresh = bench.measured_traffic("volume_kernel", "advected_wave")
    k = d["kernels"]["volume_kernel"]
    # the record matches the sources as committed, or is already stale: either way the
    # value is the record's or None, never anything else
    assert fresh in (None, k["dram_bytes_read"] + k["dram_bytes_write"])
    assert bench.measured_traffic("volume_kernel", "kh2d") is None
    assert bench.measured_traffic("no_such_kernel", "advected_wave") is None
    if fresh is not None:
        assert bench.measured_fp64_pipe("volume_kernel", "advected_wave") == pytest.approx(
            k["fp64_pipe_busy_pct"] / 100.0)
    with open(tmp_path / d["source_files"][0], "ab") as fh:
        fh.write(b"\n// changed\n")
    assert bench.measured_traffic("volume_kernel", "advected_wave") is None
    assert bench.measured_fp64_pipe("volume_kernel", "advected_wave") is None


def test_capture_record_traffic_covers_the_state():
    """The volume kernel reads the whole state (5 doubles per node) at least once: a record below
    that would be a mis-scaled capture."""
    d = json.load(open(os.path.join(ROOT, RECORD)))
    spec = bench.make_spec("advected_wave")
    state = 5 * 8 * bench.dof(spec)
    k = d["kernels"]["volume_kernel"]
    assert k["dram_bytes_read"] >= 0.95 * state
    assert 0.0 < k["fp64_pipe_busy_pct"] <= 100.0


def test_clock_summary_takes_the_median_and_the_active_reasons(tmp_path):
    c = bench.ClockSampler(0, str(tmp_path))
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1010.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1005.3, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    open(c.path, "w").write("\n".join(rows) + "\n")
    c.proc = object()  # as if nvidia-smi had run
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert os.path.dirname(c.path) == str(tmp_path)
    assert bench.ClockSampler(0).summary()["sm_mhz"] is None  # never started


def test_clock_summary_keeps_the_timed_region(tmp_path):
    """Samples carry nvidia-smi's timestamp; only those inside the marked window count, and the
    nearest one stands in when the window is shorter than the sampling interval."""
    import datetime
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def row(ms, clock, cap):
        t = (base + datetime.timedelta(milliseconds=ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"0, {clock}, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, {cap}, {t}"
    lines = [row(0, 1400, "Active"), row(50, 2070, "Not Active"), row(100, 2055, "Not Active"),
             row(150, 2070, "Not Active"), row(200, 1500, "Active")]
    t0 = base.timestamp()
    s = bench.summarize_clock_lines(lines, (t0 + 0.04, t0 + 0.16))
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["reasons"] == [] and s["scope"] == "timed region"
    s = bench.summarize_clock_lines(lines, (t0 + 0.101, t0 + 0.109))
    assert s["samples"] == 1 and s["sm_mhz"] == 2055.0 and s["scope"].startswith("nearest")
    s = bench.summarize_clock_lines(lines)
    assert s["samples"] == 5 and s["reasons"] == ["sw_power_cap"]


def test_job_throughput_counts_every_replica():
    assert bench.job_throughput(1, 1000, 10, 3, 1000.0) == 30000.0
    assert bench.job_throughput(4, 1000, 10, 3, 1000.0) == 4 * 30000.0


def test_oracle_sample_never_exceeds_the_workload():
    spec = dict(bench.make_spec("advected_wave"), n_elem=[12, 12])
    s = bench.oracle_sample_spec(spec, target_s=0.05)
    assert all(2 <= a <= b for a, b in zip(s["n_elem"], spec["n_elem"]))
    assert {k: v for k, v in s.items() if k != "n_elem"} == {k: v for k, v in spec.items() if k != "n_elem"}


def test_face_and_update_kernel_work_of_the_bench_workload():
    """Face kernel: two ideal face states (24 + 7 + 15 flops each) and the LLF combination (26)
    = 118 flops per face point; 512 x 512 periodic elements carry 2 x 262144 x 4 face points.
    Update kernel: lift 40 + Shu-Osher (10 + 25 + 25)/3 + admissibility 8 = 68 per node."""
    spec = bench.make_spec("advected_wave")
    assert bench.face_kernel_flops_per_point(spec) == 118.0
    assert bench.face_points(spec) == 2 * 512 * 512 * 4
    assert bench.update_kernel_flops_per_node(spec) == 68.0
    # a non-periodic axis adds one face per line of elements along it
    s = dict(spec, n_elem=[8, 4], bc=[("outflow", "outflow"), ("periodic", "periodic")])
    assert bench.face_points(s) == (32 + 4) * 4 + 32 * 4
    assert bench.face_kernel_flops_per_point(dict(spec, eos="tm", flux="hll")) == 2 * 61.0 + 32.0


def test_kernel_roofline_is_flops_over_time_against_the_peak():
    r = bench.kernel_roofline("face_kernel", 122.0, 2_097_152, 0.5, 1.25)
    assert r["achieved"] == pytest.approx(122.0 * 2_097_152 / 0.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert bench.kernel_roofline("x", 1.0, 1, 0.0, 1.0)["achieved"] is None


def test_oracle_on_all_cores_runs_every_process():
    """Every process steps its own copy of the sample (spawned, so none inherits a CUDA
    context): the job's rate is the sum of theirs, its time the slowest one's."""
    spec = dict(bench.make_spec("advected_wave"), n_elem=[4, 4])
    vn, tn = bench.run_oracle_all_cores(spec, 1, 0, 2)
    assert vn > 0.0 and tn > 0.0
    assert bench.host_cores() >= 1


def test_fp64_alu_peak_from_unit_counts_and_clock():
    """152 SMs x 2 FMA lanes x 2 flops x 2070 MHz = 1.2586 TFLOP/s, GB300's nominal 1.25."""
    assert bench.fp64_alu_peak_tflops(152, 2070.0) == pytest.approx(1.258560)
    assert bench.fp64_alu_peak_tflops(152, 1035.0) == pytest.approx(1.258560 / 2)


def test_smaller_capture_cases_keep_the_workload_and_drop_the_traffic_record():
    """--n shrinks a workload for a profiler capture (n x n, n x 2n, n^3) without changing its
    method choices, and the committed ncu record (taken at the benchmark size) is not applied."""
    for name, n, shape in (("advected_wave", 64, [64, 64]), ("kh2d", 32, [32, 64]), ("kh3d", 16, [16, 16, 16])):
        big, small = bench.make_spec(name), bench.make_spec(name, None, n)
        assert small["n_elem"] == shape
        assert {k: v for k, v in small.items() if k != "n_elem"} == {k: v for k, v in big.items() if k != "n_elem"}
    assert bench.measured_traffic("volume_kernel", "advected_wave_n64") is None
