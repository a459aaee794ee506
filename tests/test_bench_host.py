"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic is
used only for the kernel sources and the workload it was taken on, schedule
names, and the paper's Table 1 figures the --paper-table mode prints beside
its own."""
import json
import os

import bench


def test_recorded_traffic_needs_the_same_sources_and_workload(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    wl = rec["workload"]
    root = tmp_path / "r"
    (root / "profiles").mkdir(parents=True)
    (root / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.ncu_traffic("forward", wl) == rec["kernels"]["forward"]["dram_bytes_per_launch"]
    assert bench.ncu_traffic("forward", "large_256x256x128_fpa2048") is None
    assert bench.ncu_traffic("no_such_kernel", wl) is None
    # a record taken on other kernel sources is ignored
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("forward", wl) is None


def test_schedule_names():
    assert bench.schedule_name(("chunk", 128, 300)) == \
        "chunks of <= 128 tasks, longest first, CTA priority skew 0.3"
    assert bench.schedule_name(("split", 20, 0)) == "balanced split, item overhead 5 tasks"


def test_paper_table1_figures():
    t = bench.PAPER_TABLE1_P4000_S
    assert len(t) == 15 and {w for w, _ in t} == {3, 24, 75}
    assert t[(75, 3100)] == 467.2 and t[(3, 10)] == 0.08 and t[(24, 33)] == 1.6


def test_reference_arm_reports_the_work_it_ran():
    """--impl reference: every step is one full-size oracle EM iteration, so
    steps x ms_per_step is the timed work, and its config has exactly the keys
    and values the repo arm prints for the workload."""
    import subprocess
    import sys
    import synth
    wl = synth.TINY
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--workload", wl.name, "--steps", "3", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    assert abs(line["value"] - 1e3 / line["ms_per_step"]) <= 1e-9 * line["value"]
    assert line["config"] == bench.bench_config(wl, wl.k, 1)
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["value"] == line["value"]
