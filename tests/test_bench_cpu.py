"""Host logic of bench.py that needs no GPU: the DRAM-traffic figure is reported only while the kernel,
plan and workload sources are byte-identical to those of the committed capture."""
import bench


def _capture(path, digest, nbytes=123456):
    path.write_text(f"# capture\n\ntraffic_bytes_per_hpsi: {nbytes}\nsources_sha256: {digest}\n")


def test_traffic_reported_for_matching_sources(tmp_path, monkeypatch):
    f = tmp_path / "capture.md"
    _capture(f, bench.sources_digest())
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    value, note = bench.hpsi_traffic()
    assert value == 123456 and "ncu" in note


def test_traffic_null_when_sources_changed(tmp_path, monkeypatch):
    f = tmp_path / "capture.md"
    _capture(f, "0" * 64)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.hpsi_traffic() == (None, "kernel or workload sources changed since the DRAM capture")


def test_traffic_null_without_capture(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.hpsi_traffic()[0] is None
    f = tmp_path / "garbled.md"
    f.write_text("traffic_bytes_per_hpsi: lots\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.hpsi_traffic()[0] is None


def test_digest_covers_every_listed_source(tmp_path, monkeypatch):
    """A copy of the listed sources gives the same digest; changing any one byte of any of them
    changes it."""
    import os
    import shutil
    for rel in bench.TRAFFIC_SOURCES:
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copyfile(os.path.join(bench.ROOT, rel), tmp_path / rel)
    d0 = bench.sources_digest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.sources_digest() == d0
    for rel in bench.TRAFFIC_SOURCES:
        data = (tmp_path / rel).read_bytes()
        (tmp_path / rel).write_bytes(data[:-1] + bytes([data[-1] ^ 1]))
        assert bench.sources_digest() != d0, rel
        (tmp_path / rel).write_bytes(data)
