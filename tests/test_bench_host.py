"""Host logic of bench.py that needs no GPU: kernel names from ncu's CSV, the
DRAM-traffic record (ingested from a capture, bytes per voxel, invalid once a
kernel's source changes), the whole-step measured-traffic line, and the
reference arm's JSON line on a tiny sample."""
import csv
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _row(i, kernel, metric, unit, value):
    return [str(i), "1", "python3", "127.0.0.1", kernel, "1", "7", "(512, 1, 1)", "(304, 1, 1)", "0", "10.3",
            "Command line profiler metrics", metric, unit, value]


def test_kernel_short_name():
    assert bench.kernel_short_name("void k_init6<unsigned short, 1>(CUtensorMap_st, Batch, int *)") == "k_init6"
    assert bench.kernel_short_name("ws::k_write6(Batch, const unsigned short *)") == "k_write6"
    assert bench.kernel_short_name("void ws::<unnamed>::k_gradient3d<unsigned short>(const T1 *, int)") == \
        "k_gradient3d"
    assert bench.kernel_short_name("void (anonymous namespace)::k_x(int)") == "k_x"


def test_ingest_and_traffic(tmp_path):
    voxels = 1000
    rows = [HDR]
    # two launches of k_init6 (medians taken), one of each other kernel; mixed units
    rows += [_row(0, "void k_init6<unsigned short, 1>(CUtensorMap_st)", "dram__bytes_read.sum", "Kbyte", "2"),
             _row(0, "void k_init6<unsigned short, 1>(CUtensorMap_st)", "dram__bytes_write.sum", "byte", "6000"),
             _row(1, "void k_init6<unsigned short, 1>(CUtensorMap_st)", "dram__bytes_read.sum", "byte", "2000"),
             _row(1, "void k_init6<unsigned short, 1>(CUtensorMap_st)", "dram__bytes_write.sum", "Kbyte", "6"),
             _row(1, "void k_init6<unsigned short, 1>(CUtensorMap_st)", "gpu__time_duration.sum", "ns", "5"),
             _row(2, "k_chase(Batch)", "dram__bytes_read.sum", "Mbyte", "0.003"),
             _row(2, "k_chase(Batch)", "dram__bytes_write.sum", "byte", "300"),
             _row(3, "void k_rag6<unsigned short, 1>(A)", "dram__bytes_read.sum", "byte", "4000"),
             _row(3, "void k_rag6<unsigned short, 1>(A)", "dram__bytes_write.sum", "byte", "0"),
             _row(4, "ws::k_write6(Batch)", "dram__bytes_read.sum", "byte", "2000"),
             _row(4, "ws::k_write6(Batch)", "dram__bytes_write.sum", "Gbyte", "0.000024"),
             _row(5, "void ws::<unnamed>::k_other(int)", "dram__bytes_read.sum", "byte", "1")]
    src = tmp_path / "dram.csv"
    with open(src, "w", newline="") as f:
        csv.writer(f).writerows(rows)
    out = tmp_path / "traffic.json"
    rec = bench.ingest_ncu(str(src), voxels, str(out))
    assert set(rec) == {"k_init6", "k_chase", "k_rag6", "k_write6"}   # kernels with a known source only
    assert rec["k_init6"]["bytes_per_voxel"] == pytest.approx(8.0) and rec["k_init6"]["launches"] == 2
    assert rec["k_chase"]["bytes_per_voxel"] == pytest.approx(3.3)
    assert rec["k_write6"]["bytes_per_voxel"] == pytest.approx(26.0)
    assert json.load(open(out)) == json.loads(json.dumps(rec))
    # per launch on another volume size: bytes per voxel x voxels
    assert bench.traffic_for("k_rag6", 10 ** 6, str(out)) == pytest.approx(4.0e6)
    pd = bench.path_dram(10 ** 6, 10.0, 1000.0, str(out))
    assert pd["bytes_per_voxel"] == pytest.approx(8.0 + 3.3 + 4.0 + 26.0)
    assert pd["achieved"] == pytest.approx(41.3e6 / 1e-2 / 1e9)
    assert pd["frac"] == pytest.approx(pd["achieved"] / 1000.0)
    # a record taken on other source is not used
    stale = dict(rec)
    stale["k_rag6"] = dict(rec["k_rag6"], source_sha="0" * 16)
    with open(out, "w") as f:
        json.dump(stale, f)
    assert bench.traffic_for("k_rag6", 10 ** 6, str(out)) is None
    assert bench.path_dram(10 ** 6, 10.0, 1000.0, str(out)) is None
    assert bench.traffic_for("k_init6", 10 ** 6, str(tmp_path / "missing.json")) is None


def test_reference_arm_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-side", "16",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 3
    assert rec["value"] == rec["cpu_baseline"]["value"] == rec["e2e"]["value"] > 0
    assert rec["cpu_baseline"]["cores"] == 1


def test_source_hash_ignores_comments(tmp_path):
    """The traffic records stay valid across comment edits of a kernel source
    and not across code edits."""
    a = tmp_path / "a.cuh"
    a.write_text("int f(int x)  // doubles\n{\n    return 2 * x;\n}\n")
    b = tmp_path / "b.cuh"
    b.write_text("// a new header comment\nint f(int x)\n{\n\n    return 2 * x;   // twice\n}\n")
    c = tmp_path / "c.cuh"
    c.write_text("int f(int x)\n{\n    return 3 * x;\n}\n")
    assert bench._code_text(str(a)) == bench._code_text(str(b))
    assert bench._code_text(str(a)) != bench._code_text(str(c))
