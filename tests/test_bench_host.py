"""Host logic of the bench's roofline figures (no GPU): the algorithmic bytes
per kernel and the DRAM traffic taken from committed ncu captures, which
apply only to the kernel source they were measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_stream_engine_reads_the_set_once_and_writes_the_survivors():
    # rows as qp_read_stats returns them: (t, groups, extended, kept, intermediate)
    rows = [((100, 60000, 250000, 150000, 150000), 140000), ((101, 61000, 252000, 151000, 151000), 150000)]
    b = bench.algorithmic_bytes(rows, 2, 8, lambda t: True, engine="stream")
    E = 16
    assert b[0] == 0 and b[1] == 0 and b[3] == 0
    assert b[2] == (140000 + 150000) * E + (150000 + 151000) * E


def test_algorithmic_bytes_merge_table_engine():
    rows = [((5, 0, 400, 400, 400), 100), ((20, 30, 120, 90, 90), 100)]   # a filling step, then a merging one
    b = bench.algorithmic_bytes(rows, 2, 16, lambda t: t >= 16, engine="hash")
    E = 24
    assert b[0] == 100 * (E + 4) + 30 * 32
    assert b[1] == 100 * (E + 4) + 30 * 16
    assert b[2] == (100 * E + 400 * E) + (30 * (4 + 8 + 32 + 40) + 90 * E)


def _fake_tree(tmp_path, src, rows):
    (tmp_path / "paper_2506_03127_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2506_03127_gb300" / "csrc" / "qp.cu").write_bytes(src)
    (tmp_path / "profiles" / "traffic.txt").write_text("# header\n" + "\n".join(rows) + "\n")


def test_code_hash_ignores_comments_and_layout_but_not_code(tmp_path):
    def h(text):
        f = tmp_path / "k.cu"
        f.write_text(text)
        return bench.code_hash(str(f))
    base = h('int f(int x) {\n    return x + 1;   // one more\n}\nconst char *s = "a // b";\n')
    assert h('// a new comment\nint f(int x) { /* same */ return x + 1; }\nconst char *s = "a // b";\n') == base
    assert h('int f(int x) {\n    return x + 2;\n}\nconst char *s = "a // b";\n') != base
    assert h('int f(int x) {\n    return x + 1;\n}\nconst char *s = "a // c";\n') != base   # inside a string: code
    assert h("char c = '\"'; int g;  // it's\n") == h("char c = '\"';\nint g;\n")


def test_ncu_traffic_applies_only_to_the_captured_code(tmp_path, monkeypatch):
    src = b"__global__ void k() {}   // kernel source\n"
    _fake_tree(tmp_path, src, [])
    sha = bench.code_hash(str(tmp_path / "paper_2506_03127_gb300" / "csrc" / "qp.cu"))
    _rows = [f"spin_boson_structured_dk16 stream_tile {sha} 2340608 0",
             f"tls_ohmic_full_dk12 stream_regular {sha} 400 16",
             "chain3_structured_dk12 stream_tile 0123456789abcdef 777 0"]
    (tmp_path / "profiles" / "traffic.txt").write_text("# header\n" + "\n".join(_rows) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("spin_boson_structured_dk16", False, 150000) == 2340608
    # the regular kernel's capture is scaled by stored paths (25 B per path here)
    assert bench.ncu_traffic("tls_ohmic_full_dk14", True, 1 << 28) == pytest.approx(25.0 * (1 << 28))
    # a row taken on another source does not apply; nor does a missing workload
    assert bench.ncu_traffic("chain3_structured_dk12", False, 1) is None
    assert bench.ncu_traffic("spin_boson_ohmic_dk8", False, 1) is None
    # a comment changes: the rows still apply; the code changes: they go stale
    (tmp_path / "paper_2506_03127_gb300" / "csrc" / "qp.cu").write_bytes(src + b"// edited\n")
    assert bench.ncu_traffic("spin_boson_structured_dk16", False, 150000) == 2340608
    (tmp_path / "paper_2506_03127_gb300" / "csrc" / "qp.cu").write_bytes(src + b"int edited;\n")
    assert bench.ncu_traffic("spin_boson_structured_dk16", False, 150000) is None
