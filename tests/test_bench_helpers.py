"""Host helpers of bench.py: the code digest that ties a committed ncu
summary to the kernel source it was taken on, and the lookup of the profiled
DRAM traffic by workload, tile side and digest."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_digest_ignores_comments_not_code(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) { return x + 1; }  // add one\n/* block\n comment */\n")
    b = tmp_path / "b.cu"
    b.write_text("// header\nint  f(int x)\n{\n    return x + 1;\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_profiled_traffic_matches_tile_and_digest(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1410_5780_gb300" / "csrc").mkdir(parents=True)
    src = tmp_path / "paper_1410_5780_gb300" / "csrc" / "kernels.cu"
    src.write_text("__global__ void k() {}\n")
    digest = bench.code_digest(str(src))
    for name, tile, b, d in (("k_tile_warp_facade.md", 128, 11.0, digest),
                             ("k_tile_warp_facade_tile64.md", 64, 19.0, digest),
                             ("k_tile_warp_tracker.md", 32, 290.0, "stale")):
        rec = {"kernel": "k_tile_warp", "tile": tile, "bytes_per_launch": b, "code_sha256": d}
        (tmp_path / "profiles" / name).write_text(f"# x\n\n<!-- traffic: {json.dumps(rec)} -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("facade", 128) == 11.0
    assert bench.profiled_traffic("facade", 64) == 19.0
    assert bench.profiled_traffic("facade", 32) is None
    assert bench.profiled_traffic("tracker", 32) is None  # taken on other code
    src.write_text("__global__ void k() { }  // same code, new comment\n")
    assert bench.profiled_traffic("facade", 64) == 19.0


def test_committed_summaries_are_found():
    """Every committed k_tile_warp summary names its tile side and the digest
    of the kernels.cu code it was taken on; the bench finds each one taken on
    the current code (a summary of older code reads as null traffic)."""
    import glob
    import re
    paths = glob.glob(os.path.join(ROOT, "profiles", "k_tile_warp_*.md"))
    assert paths
    digest = bench.code_digest(os.path.join(ROOT, "paper_1410_5780_gb300", "csrc", "kernels.cu"))
    for p in paths:
        rec = json.loads(re.search(r"<!-- traffic: (\{.*?\}) -->", open(p).read()).group(1))
        assert rec["tile"] in (32, 64, 128) and len(rec["code_sha256"]) == 64, p
        if rec["code_sha256"] == digest:
            workload = os.path.basename(p)[len("k_tile_warp_"):-3].split("_")[0]
            assert bench.profiled_traffic(workload, rec["tile"]) == rec["bytes_per_launch"], p
