"""Host-side logic of the benchmark: the measured-traffic record is used only
while the kernel sources hash to the value stored beside it."""
import os

import bench


def test_traffic_record_follows_kernel_hash(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 64
    prof = tmp_path / "profiles"
    prof.mkdir()
    md = prof / bench.PROFILES[2]
    md.write_text("summary\n\ntraffic_per_launch_bytes: 123456 kernel_sources_sha256 %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.measured_traffic(2) == 123456
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.measured_traffic(2) is None
    assert bench.measured_traffic(5) is None


def test_committed_profiles_parse():
    # every render-kernel summary carries a traffic line in the expected form
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in bench.PROFILES.values():
        for key in ("traffic_per_launch_bytes:", "instructions_per_launch:"):
            lines = [ln for ln in open(os.path.join(root, "profiles", name)) if ln.startswith(key)]
            assert len(lines) == 1, (name, key)
            parts = lines[0].split()
            assert int(parts[1]) > 0 and parts[2] == "kernel_sources_sha256" and len(parts[3]) == 64


def test_code_only_ignores_comments_and_spacing():
    a = "int x = 1;  // one\n/* block\n comment */ int y = x << 2;\n"
    b = "int x = 1;\nint y = x << 2;  // shifted\n"
    assert bench._code_only(a) == bench._code_only(b) == "intx=1;inty=x<<2;"
    assert bench._code_only("int y = x << 3;") != bench._code_only("int y = x << 2;")


def test_reference_arm_line():
    """bench.py --impl reference runs the oracle on the host and prints one
    JSON line with the contract's keys (no GPU needed)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--points", "200000"], capture_output=True, text=True, timeout=600,
                         cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "tiles/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "tiles/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["n_objects"] == 200000 and "workload" in line["config"]
