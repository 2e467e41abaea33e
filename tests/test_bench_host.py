"""Host-side helpers of the benchmark: the comment-insensitive source hash that keys recorded
profiler counters to the code they were taken on."""
import bench


def test_strip_c_comments_keeps_code_and_literals():
    src = 'int a = 1; // note "x"\n/* block\n comment */ const char* s = "a//b /* c */";\nchar q = \'"\';  int b;'
    assert bench.strip_c_comments(src) == 'int a = 1; const char* s = "a//b /* c */"; char q = \'"\'; int b;'


def test_comment_edits_keep_the_hash_and_code_edits_change_it(tmp_path, monkeypatch):
    (tmp_path / "paper_1205_5351_gb300" / "csrc").mkdir(parents=True)
    f = tmp_path / "paper_1205_5351_gb300" / "csrc" / bench.SOLVER_SOURCES[0]
    f.write_text("int f(int a) { return a + 1; }  // one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_sha256()
    f.write_text("/* a new\n   comment */\nint f(int a) {\n    return a + 1;   // two\n}\n")
    assert bench.kernel_sources_sha256() == h0
    f.write_text("int f(int a) { return a + 2; }\n")
    h1 = bench.kernel_sources_sha256()
    assert h1 != h0
    # host-only sources are not part of it
    (tmp_path / "paper_1205_5351_gb300" / "csrc" / "tilt_api.cu").write_text("int g() { return 3; }\n")
    assert bench.kernel_sources_sha256() == h1


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) on a two-patch sample."""
    import json
    import os
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--impl",
                          "reference", "--steps", "1", "--warmup", "0", "--patches", "2"],
                         capture_output=True, text=True, timeout=600, check=True)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "patches/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "2 patches" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "patches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_stratified_parity_sample_covers_the_hard_cases():
    # the slowest patch first, then every status-2 patch, then every (class, status, size)
    # stratum before any stratum repeats
    import bench
    from types import SimpleNamespace as NS
    sizes = [(40, 40), (120, 120), (60, 80), (100, 90)] * 10
    patches = [NS(m=m, n=n) for m, n in sizes]
    results = [{"status": (2 if q == 17 else 1 if q % 3 == 0 else 0), "launch_class": q % 2} for q in range(40)]
    lat = [float(q) for q in range(40)]
    lat[9] = 1e6
    idx = bench.stratified_sample(patches, results, lat, 12)
    assert idx[0] == 9 and idx[1] == 17 and len(idx) == 12 and len(set(idx)) == 12
    strata = {(results[q]["launch_class"], results[q]["status"]) for q in idx}
    assert strata == {(r["launch_class"], r["status"]) for r in results}
    assert len(bench.stratified_sample(patches, results, lat, 100)) == 40
