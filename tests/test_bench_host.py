"""Host logic of bench.py (no GPU): the ncu traffic figure of the committed
profile is reported only for the kernel code, radius, tile rows, padded
grid and slab height it was measured on; comments do not count as code."""
import os
import sys

import pytest

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def _profile(tmp_path, src_bytes, radius=4, rows=8, grid="576x576x576"):
    src = tmp_path / "stencil.cu"
    src.write_bytes(src_bytes)
    prof = tmp_path / "profile.md"
    prof.write_text("# summary\n\nradius: %d\ntile_rows: %d\npadded_grid: %s\n"
                    "traffic_ratio_zchunk_16: 1.02\ntraffic_ratio_zchunk_32: 1.04\n"
                    "stencil_code_sha256: %s\n"
                    % (radius, rows, grid, bench.kernel_code_digest(str(src))))
    return str(src), str(prof)


def test_traffic_matches_only_the_profiled_launch(tmp_path, monkeypatch):
    src, prof = _profile(tmp_path, b"kernel source A")
    monkeypatch.setattr(bench, "STENCIL_SRC", src)
    monkeypatch.setattr(bench, "PROFILE", prof)
    g = (576, 576, 576)
    assert bench.profiled_traffic(4, 8, g, 16, 1e9) == pytest.approx(1.02e9)
    assert bench.profiled_traffic(4, 8, g, 32, 2e9) == pytest.approx(2.08e9)
    assert bench.profiled_traffic(4, 8, g, 24, 1e9) is None  # other slab height
    assert bench.profiled_traffic(4, 8, g, None, 1e9) is None  # automatic slabs
    assert bench.profiled_traffic(8, 8, g, 16, 1e9) is None  # other radius
    assert bench.profiled_traffic(4, 16, g, 16, 1e9) is None  # other tile
    assert bench.profiled_traffic(4, 8, (448, 448, 448), 16, 1e9) is None  # other grid
    with open(src, "wb") as f:  # the kernel changed since the capture
        f.write(b"kernel source B")
    assert bench.profiled_traffic(4, 8, g, 16, 1e9) is None


def test_code_digest_ignores_comments_only(tmp_path):
    code = 'int f(int a) {\n    const char* s = "a // b /* c */";\n    return a + 1;\n}\n'
    commented = ('// header\n/* block\n   comment */\nint f(int a) {  // trailing\n\n'
                 '    const char* s = "a // b /* c */";\n    return a + 1;  /* x */\n}\n')
    changed = code.replace("a + 1", "a + 2")
    digests = []
    for i, text in enumerate((code, commented, changed)):
        path = tmp_path / ("k%d.cu" % i)
        path.write_text(text)
        digests.append(bench.kernel_code_digest(str(path)))
    assert digests[0] == digests[1]  # comments and blank lines only
    assert digests[0] != digests[2]  # a code change
    s_lit = tmp_path / "lit.cu"  # a string literal keeps its "//"
    s_lit.write_text(code.replace('"a // b /* c */"', '"a"'))
    assert bench.kernel_code_digest(str(s_lit)) != digests[0]


def test_missing_or_incomplete_profile(tmp_path, monkeypatch):
    src, prof = _profile(tmp_path, b"k")
    monkeypatch.setattr(bench, "STENCIL_SRC", src)
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "absent.md"))
    assert bench.profiled_traffic(4, 8, (576, 576, 576), 16, 1e9) is None
    text = open(prof).read().replace("tile_rows: 8\n", "")
    with open(prof, "w") as f:
        f.write(text)
    monkeypatch.setattr(bench, "PROFILE", prof)
    assert bench.profiled_traffic(4, 8, (576, 576, 576), 16, 1e9) is None


def test_committed_profile_names_its_launch():
    text = open(bench.PROFILE).read()
    for key in ("radius:", "tile_rows:", "padded_grid:", "traffic_ratio_zchunk_",
                "stencil_code_sha256:"):
        assert key in text
    # the profile was taken on the current stencil code
    m = __import__("re").search(r"stencil_code_sha256:\s*([0-9a-f]{64})", text)
    assert m.group(1) == bench.kernel_code_digest(bench.STENCIL_SRC)
