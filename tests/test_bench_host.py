"""Host-side pieces of bench.py that decide what the JSON line claims: the
recorded DRAM traffic is used only while the kernel sources it was taken on
are unchanged, and the algorithmic bytes of the batched and per-view forms
differ only in the once-per-batch terms."""
import os
import pathlib
import shutil

import pytest

import bench


@pytest.fixture
def scratch(request):
    """A fresh directory under the repository's git-ignored _build/."""
    d = pathlib.Path(bench.ROOT) / "_build" / "test_bench_host" / request.node.name
    shutil.rmtree(d, ignore_errors=True)
    d.mkdir(parents=True)
    yield d
    shutil.rmtree(d, ignore_errors=True)


def _tree(root):
    csrc = root / "paper_2605_05876_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.RASTER_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2605_05876_gb300", "csrc", f), csrc / f)
    (root / "profiles").mkdir()
    return csrc


def test_recorded_traffic_follows_the_source_hash(scratch, monkeypatch):
    csrc = _tree(scratch)
    monkeypatch.setattr(bench, "ROOT", str(scratch))
    h = bench.source_hash()
    (scratch / "profiles" / "traffic.txt").write_text(
        "# kernel workload bytes hash\n"
        f"raster_bwd some_workload 12345 {h}\n"
        "raster_fwd some_workload 999 0123456789ab\n")
    assert bench.recorded_traffic("raster_bwd", "some_workload") == 12345.0
    assert bench.recorded_traffic("raster_bwd", "other_workload") is None
    assert bench.recorded_traffic("raster_fwd", "some_workload") is None     # taken on other sources
    with open(csrc / bench.RASTER_SOURCES[1], "a") as fh:                  # any edit of a rasteriser source
        fh.write("\n// edited\n")
    assert bench.source_hash() != h
    assert bench.recorded_traffic("raster_bwd", "some_workload") is None


def test_missing_traffic_file_reads_as_unmeasured(scratch, monkeypatch):
    _tree(scratch)
    monkeypatch.setattr(bench, "ROOT", str(scratch))
    assert bench.recorded_traffic("raster_bwd", "some_workload") is None


def test_algorithmic_bytes_forms():
    N, V, M, P, E = 1000, 16, 50000, 64000, 4096
    b = bench.algorithmic_bytes(N, V, M, P, E)
    pv = bench.algorithmic_bytes(N, V, M, P, E, per_view=True)
    assert b["total"] == sum(v for k, v in b.items() if k != "total")
    # per view, only the parameters and their gradients are moved once per view
    assert pv["params"] == V * b["params"]
    assert pv["project_bwd"] - b["project_bwd"] == (V - 1) * bench.B_PARAM_GRAD * N
    for k in ("records", "bin_sort", "raster_fwd", "raster_bwd", "gradient_scatter", "env"):
        assert pv[k] == b[k], k
    # the per-record and per-instance terms grow with the views and the instances
    b2 = bench.algorithmic_bytes(N, 2 * V, 2 * M, 2 * P, E)
    for k in ("records", "bin_sort", "raster_fwd", "raster_bwd", "gradient_scatter"):
        assert b2[k] == 2 * b[k], k
