"""Host-side helpers of the benchmark: the comment-insensitive source hash that keys recorded
profiler counters to the code they were taken on."""
import bench


def test_strip_c_comments_keeps_code_and_literals():
    src = 'int a = 1; // note "x"\n/* block\n comment */ const char* s = "a//b /* c */";\nchar q = \'"\';  int b;'
    assert bench.strip_c_comments(src) == 'int a = 1; const char* s = "a//b /* c */"; char q = \'"\'; int b;'


def test_comment_edits_keep_the_hash_and_code_edits_change_it(tmp_path, monkeypatch):
    for d in ("paper_1205_5351_gb300/csrc", "include"):
        (tmp_path / d).mkdir(parents=True)
    f = tmp_path / "include" / "x.h"
    f.write_text("int f(int a) { return a + 1; }  // one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_sha256()
    f.write_text("/* a new\n   comment */\nint f(int a) {\n    return a + 1;   // two\n}\n")
    assert bench.kernel_sources_sha256() == h0
    f.write_text("int f(int a) { return a + 2; }\n")
    assert bench.kernel_sources_sha256() != h0
