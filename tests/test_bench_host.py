"""Host logic of the benchmark that needs no GPU: the DRAM-traffic records
of the committed ncu summaries (roofline.traffic) and their tie to the
kernel sources they were captured from."""
import os

import pytest

import bench


def _records():
    out = []
    for name in sorted(os.listdir(bench.PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(bench.PROFILES, name)) as f:
            for line in f:
                line = line.strip().strip("`")
                if line.startswith("traffic-record:"):
                    out.append((name, dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)))
    return out


def test_traffic_records_are_complete():
    """Every record names its kernel, block width, rows, bytes, digest and
    source files, and the files exist."""
    recs = _records()
    assert recs, "no traffic records under profiles/"
    for name, kv in recs:
        for key in ("kernel", "n_b", "N", "bytes", "sources", "digest"):
            assert key in kv, (name, key)
        for rel in kv["sources"].split(","):
            assert os.path.exists(os.path.join(bench.ROOT, rel)), (name, rel)
        assert int(kv["bytes"]) > 0 and int(kv["N"]) > 0 and int(kv["n_b"]) > 0
        assert len(kv["digest"]) == 16


def test_benchmark_kernels_have_records():
    """The kernels the benchmark's roofline names (footprint-staged
    double-word and complex-float steps, their gathered forms, the native
    fp64 step) each have a record at n_b = 32."""
    kernels = {kv["kernel"] for _, kv in _records() if kv["n_b"] == "32"}
    for k in ("k_cheb_step_fp_dw", "k_cheb_step_fp_c64", "k_cheb_step_dw", "k_cheb_step_staged_c64"):
        assert k in kernels, k


def _write_record(tmp_path, digest, sources, nbytes=1000, rows=100):
    (tmp_path / "k.md").write_text(
        "traffic-record: kernel=k_test n_b=32 N=%d bytes=%d sources=%s digest=%s\n"
        % (rows, nbytes, ",".join(sources), digest))


def test_record_counts_only_for_unchanged_sources(tmp_path, monkeypatch):
    """A record scales with the row count while its digest equals the
    sources' digest, and is ignored (None) once a source differs."""
    src = ["bench.py"]
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    _write_record(tmp_path, bench.source_digest(src), src)
    traffic, where = bench.profiled_traffic("k_test", 32, 400)
    assert traffic == pytest.approx(4000.0)
    assert where.endswith("k.md")
    assert bench.profiled_traffic("k_test", 16, 400) == (None, None)      # other block width
    _write_record(tmp_path, "0" * 16, src)
    assert bench.profiled_traffic("k_test", 32, 400) == (None, None)      # stale digest
    _write_record(tmp_path, bench.source_digest(src), ["no/such/file.cu"])
    assert bench.profiled_traffic("k_test", 32, 400) == (None, None)      # missing source
