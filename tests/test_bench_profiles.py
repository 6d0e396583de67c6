"""The benchmark's readers of the committed ncu summaries: the dominant
kernel's DRAM traffic per launch and each solve's DRAM bytes are used only
while the library sources hash to the value recorded beside them, and the
%HBM figures are those bytes over the solve time."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _profile(tmp_path, sha, lines):
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "ncu_dram_per_solve.md").write_text(
        "# summary\n\ntext with: a colon\n\n- csrc sha256[:16]: `%s`\n%s\n" % (sha, "\n".join(lines)))
    return tmp_path


def test_dram_reader_checks_the_source_hash(tmp_path, monkeypatch):
    import bench
    real = bench.csrc_sha()
    root = _profile(tmp_path, real, [
        "- sr_fmg_fp64_256 dram bytes per solve: 21643400000",
        "- mixed_sr_512 dram bytes per solve: 7.5e10"])
    # the summary from the temporary tree, the sources' hash from the real one
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "csrc_sha", lambda: real)
    assert bench.ncu_dram_per_solve() == {"sr_fmg_fp64_256": 21643400000.0,
                                          "mixed_sr_512": 7.5e10}
    monkeypatch.setattr(bench, "csrc_sha", lambda: "0000000000000000")
    assert bench.ncu_dram_per_solve() == {}


def test_dram_rate():
    import bench
    r = bench.dram_rate(2.0e10, 10.0, 8000.0)
    assert r["gbs"] == pytest.approx(2000.0)
    assert r["frac_of_measured"] == pytest.approx(0.25)
    assert r["frac_of_nominal_8tbs"] == pytest.approx(0.25)
    assert bench.dram_rate(None, 10.0, 8000.0) is None
    assert bench.dram_rate(2.0e10, 10.0, None)["frac_of_measured"] is None


def test_csrc_sha_covers_the_7_point_sources():
    import hashlib
    import bench
    d = os.path.join(ROOT, "paper_1406_7808_gb300", "csrc")
    names = sorted(x for x in os.listdir(d)
                   if x.endswith((".cu", ".cuh")) and x != "kernels27.cu")
    assert "kernels.cu" in names and "srfmg_device.cuh" in names and "srfmg_api.cu" in names
    h = hashlib.sha256(b"".join(open(os.path.join(d, x), "rb").read() for x in names))
    assert bench.csrc_sha() == h.hexdigest()[:16]
