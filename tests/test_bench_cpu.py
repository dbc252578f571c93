"""bench.py's reference arm on the CPU: one JSON line with the contract's
keys, the same metric string as the GPU arm, and no work on ranks other than
0 under torchrun."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, args=()):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--cpu-seconds", "1", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench
    r = _run(args=("--variant", "plain"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["unit"] == "Gpts/s" and out["higher_is_better"] is True and out["value"] > 0
    assert out["steps"] == 1 and out["warmup"] == 0 and out["dtype"] == "f64"
    assert out["config"]["workload"] == "dipping_300x1000_96shots"
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_summary_parses_reasons():
    """nvidia-smi samples (sm, max, power, active mask, hw_slowdown,
    hw_thermal, sw_thermal, sw_power_cap): median SM clock, the maximum, and
    every throttle reason seen Active."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.out = "\n".join([
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.out = "1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active"
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.out = ""
    assert c.summary()["reasons"] == ["unavailable"]


def test_traffic_record_needs_the_captured_source(tmp_path, monkeypatch):
    """The ncu traffic of a kernel is reported only for the workload it was
    captured on and while the step-kernel sources hash as at the capture."""
    sys.path.insert(0, ROOT)
    import bench
    rec = {"k_bwd_step": {"workload": "w", "source_hash": bench.kernel_source_hash(), "bytes_per_launch": 5.0}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.read_traffic("k_bwd_step", "w") == 5.0
    assert bench.read_traffic("k_bwd_step", "other") is None
    assert bench.read_traffic("k_fwd_step", "w") is None
    rec["k_bwd_step"]["source_hash"] = "0" * 16
    f.write_text(json.dumps(rec))
    assert bench.read_traffic("k_bwd_step", "w") is None


def test_committed_traffic_matches_the_current_kernels():
    """profiles/traffic.json was captured on the step-kernel sources in the
    tree (a kernel change without a new capture reports traffic null)."""
    sys.path.insert(0, ROOT)
    import bench
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert t and all(e["source_hash"] == bench.kernel_source_hash() for e in t.values())
    assert bench.read_traffic("k_bwd_step", "dipping_300x1000_96shots") > 0


def test_traffic_tool_reads_ncu_csv(tmp_path):
    """The traffic tool keys launches by step kind and averages DRAM bytes
    (read + write) over each kind's captured launches."""
    from paper_1406_1864_gb300 import traffic
    assert traffic.key_of("void k_fwd_step<1, 12, 1, 3, 4, 1, 2, 11>(Batch<FwdArgs, T6>)") == \
        "k_fwd_step<offset Hessian>"
    assert traffic.key_of("void k_fwd_step<2, 4, 0, 2, 4, 1, 2, 13>(Batch<FwdArgs, T6>)") == "k_fwd_step"
    assert traffic.key_of("void k_bwd_step<2, 2, 4, 1, 0>(Batch<BwdArgs, T4>)") == "k_bwd_step"
    assert traffic.key_of("void k_offh_level<11, 4>(const float *, Lay2D, int, int, int, float *)") == \
        "k_offh_level"
    assert traffic.key_of("k_prep_c2(...)") is None
    hdr = '"ID","Kernel Name","Metric Name","Metric Value"\n'
    rows = []
    for i, (rd, wr) in enumerate([(100.0, 20.0), (140.0, 40.0)]):
        name = "void k_bwd_step<2, 2, 4, 1, 0>(Batch<BwdArgs, T4>)"
        rows.append(f'"{i}","{name}","dram__bytes_read.sum","{rd:,.0f}"\n')
        rows.append(f'"{i}","{name}","dram__bytes_write.sum","{wr:,.0f}"\n')
    f = tmp_path / "t.csv"
    f.write_text("==PROF== noise\n" + hdr + "".join(rows))
    per = traffic.read_csv(str(f))
    assert list(per) == ["k_bwd_step"] and sorted(per["k_bwd_step"][1]) == [120.0, 180.0]
