"""Host-side pieces of bench.py that need no GPU: the profile lookup that
feeds the roofline's measured traffic, the kernel naming, the workload and
the reference arm's bounded oracle sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import bench  # noqa: E402


@pytest.mark.parametrize("workload", ["default", "heading"])
def test_profiled_traffic_needs_the_profiled_sources(tmp_path, monkeypatch, workload):
    kernel = "map_stream_kernel"
    key = (kernel, workload)
    per_frame = 19_000_000
    prof = tmp_path / "p.txt"
    prof.write_text(f"source_sha256_16: {bench.map_source_hash(key)}\n"
                    f"dram_bytes_per_frame: {per_frame}\n")
    monkeypatch.setitem(bench.PROFILES, key, (str(prof), bench.PROFILES[key][1]))
    # the lookup joins profiles/ to the name; an absolute name stays as given
    assert bench.profiled_traffic(900, kernel, workload) == per_frame * 900
    prof.write_text("source_sha256_16: 0000000000000000\ndram_bytes_per_frame: 1\n")
    assert bench.profiled_traffic(900, kernel, workload) is None
    assert bench.profiled_traffic(900, "no_such_kernel") is None
    assert bench.profiled_traffic(900, kernel, "no_such_workload") is None


def test_committed_profiles_name_their_sources():
    for kernel, (name, sources) in bench.PROFILES.items():
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "source_sha256_16:" in text and "dram_bytes_per_frame:" in text, name
        for f in sources:
            assert os.path.exists(os.path.join(ROOT, "paper_2601_07154_gb300", "csrc", f))


def test_workload_config_and_frame_bytes():
    cfg = bench.workload_config()
    assert cfg["width"] == 1920 and cfg["height"] == 1080 and cfg["frames_per_step"] == 900
    assert "ACCEL" in cfg["workload"] and "speed changes" not in cfg["workload"]
    assert "HEADING" in bench.workload_config(workload="heading")["workload"]
    assert "speed changes" in bench.workload_config(workload="accel_in_view")["workload"]
    assert bench.FRAME_BYTES == 1920 * 1080 * 12
    assert 1 <= bench.PIECE_FRAMES <= 64


def test_reference_arm_prints_one_line_on_the_host():
    """--impl reference times the FP64 oracle on the host (no GPU) and prints
    the contract's JSON line with impl, cpu_baseline and e2e."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    rec = json.loads(out[-1])
    assert rec["impl"] == "reference" and rec["unit"] == "frames/s" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["higher_is_better"] is True
