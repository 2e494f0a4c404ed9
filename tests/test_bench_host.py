"""Host logic of bench.py that the JSON line rests on: the traffic figure is only
reported for the fill kernel the committed ncu summary was taken on, keyed by a
digest of the kernel's code (its own file and the headers it includes) that
ignores comments and blank lines but not code; and the serving baseline that
runs the oracle on spawned worker processes."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _with_sources(tmp_path, edit):
    """A copy of the kernel sources (and the header they include) with `edit` applied to fill_col3.cu."""
    pkg = tmp_path / "paper_2311_17530_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2311_17530_gb300", "csrc"), pkg / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), tmp_path / "include")
    f = pkg / "csrc" / "fill_col3.cu"
    f.write_text(edit(f.read_text()))
    return str(tmp_path)


def test_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    base = bench.kernel_source_digest("fill_col3")
    root_c = _with_sources(tmp_path / "c", lambda s: s.replace("namespace msadp {", "// a new comment\n\n/* and a block */\nnamespace msadp {", 1))
    monkeypatch.setattr(bench, "ROOT", root_c)
    assert bench.kernel_source_digest("fill_col3") == base
    root_x = _with_sources(tmp_path / "x", lambda s: s.replace("constexpr int SB = 8;", "constexpr int SB = 16;", 1))
    monkeypatch.setattr(bench, "ROOT", root_x)
    assert bench.kernel_source_digest("fill_col3") != base


def test_traffic_only_for_matching_digest(tmp_path, monkeypatch):
    rec = {"fill_col3:k3_protein": {"source_digest": bench.kernel_source_digest("fill_col3"),
                                    "dram_bytes_per_launch": 123}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(rec))
    pkg = tmp_path / "paper_2311_17530_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2311_17530_gb300", "csrc"), pkg / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), tmp_path / "include")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k3_protein", "fill_col3") == 123
    assert bench.measured_traffic("k4_dna", "fill_tiles") is None
    rec["fill_col3:k3_protein"]["source_digest"] = "0" * 16
    (prof / "traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("k3_protein", "fill_col3") is None


def test_serving_cpu_baseline_runs_on_spawned_workers():
    """The serving baseline: the oracle on a prefix of the request stream, one
    request per task, on spawned processes."""
    r = bench.serving_cpu_baseline(3, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == "alignments/s"
    assert r["value"] > 0 and r["cells_per_s"] > 0
    assert "requests 0..2" in r["sample"]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON
    line with the keys the benchmark contract asks of it."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-cells", "2e5"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    for key in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "scaling", "dtype", "data", "config"):
        assert key in d, key
    assert d["config"]["workload"] == "k3_protein_700_760_800"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["value"] > 0


def test_reference_arm_other_ranks_exit_without_work():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_whole_column_limit_matches_the_library():
    """bench.py names the k = 6 whole-column kernel by the same last-axis limit
    the planner and the kernel use."""
    src = open(os.path.join(ROOT, "paper_2311_17530_gb300", "csrc", "internal.h")).read()
    assert f"constexpr int kWideZ = {bench.WIDE_Z};" in src
    assert len(bench.kernel_source_digest("fill_lines_wide")) == 16
