"""The kernel-source hash that ties the committed ncu summaries to the code they were taken on
(bench.kernel_source_hash): it covers the code only, so a comment or layout edit keeps a summary
valid and any change to the code itself invalidates it. Host logic only."""
import bench


def test_comments_and_layout_do_not_count():
    a = "int f(int x) {  // the first form\n    return x + 1; /* done */\n}\n"
    b = "// another header line\nint f(int x)\n{\n  return x + 1;\n}  /* a different comment */\n"
    assert bench._code_only(a, "//") == bench._code_only(b, "//")


def test_code_changes_count():
    a = "int f(int x) { return x + 1; }"
    for b in ("int f(int x) { return x + 2; }", "int f(int x) { return x - 1; }", "int f(int y) { return y + 1; }"):
        assert bench._code_only(a, "//") != bench._code_only(b, "//")


def test_literals_keep_comment_markers():
    code = 'const char* s = "a // not a comment /* nor this */"; char q = \'"\'; int n; // gone'
    out = bench._code_only(code, "//")
    assert '"a // not a comment /* nor this */"' in out and "gone" not in out and out.endswith("int n;")
    py = 'x = "# kept"  # dropped\ny = 2'
    assert bench._code_only(py, "#") == 'x = "# kept" y = 2'

