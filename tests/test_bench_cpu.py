"""Host logic of bench.py that decides whether the ncu traffic figure still applies: the digest of
a source ignores comments and whitespace but not code (a figure taken on other code reports as
null)."""
import bench


def _digest_of(tmp_path, text):
    p = tmp_path / "k.cu"
    p.write_text(text)
    return bench._code_digest(str(p))


def test_code_digest_ignores_comments_and_whitespace(tmp_path):
    a = _digest_of(tmp_path, "int f(int x) {\n  return x + 1;  // one more\n}\n")
    b = _digest_of(tmp_path, "/* block\n comment */ int f(int x) { return x + 1; }")
    assert a == b


def test_code_digest_sees_code_changes(tmp_path):
    a = _digest_of(tmp_path, "int f(int x) { return x + 1; }")
    b = _digest_of(tmp_path, "int f(int x) { return x + 2; }")
    assert a != b

