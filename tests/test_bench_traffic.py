"""The bench's recorded DRAM traffic (profiles/traffic.json) is reported only
for the code it was captured from: the digest of a kernel's sources ignores
comments and whitespace but follows every code change, a record whose
digest no longer matches gives no figure, and a per-unit record scales with
the units of the launch."""
import bench


def _write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_digest_ignores_comments_and_follows_code(tmp_path):
    a = _write(tmp_path, "a.cu", "int f(int x) {\n  return x + 1;  // one\n}\n")
    b = _write(tmp_path, "b.cu", "/* header */\nint f(int x)   {\n\n return x + 1; // other words\n}")
    c = _write(tmp_path, "c.cu", "int f(int x) {\n  return x + 2;  // one\n}\n")
    da = bench.source_digest((a,))
    assert da == bench.source_digest((a,))
    # same code, other comments and spacing (names differ, so compare per name)
    b_as_a = _write(tmp_path, "a.cu", open(b).read())
    assert bench.source_digest((b_as_a,)) == da
    c_as_a = _write(tmp_path, "a.cu", open(c).read())
    assert bench.source_digest((c_as_a,)) != da


def test_recorded_traffic_only_for_matching_code(tmp_path, monkeypatch):
    src = _write(tmp_path, "k.cu", "__global__ void k() {}\n")
    dig = bench.source_digest((src,))
    recs = {
        "per_unit": {"source": dig, "source_files": [src], "bytes_per_unit": 12.5},
        "per_launch": {"source": dig, "source_files": [src], "bytes_per_launch": 4096},
        "stale": {"source": "0" * 16, "source_files": [src], "bytes_per_launch": 4096},
    }
    monkeypatch.setattr(bench, "traffic_record", lambda: recs)
    assert bench.recorded_traffic("per_unit", 1000) == 12500
    assert bench.recorded_traffic("per_launch") == 4096
    assert bench.recorded_traffic("per_launch", 10) is None
    assert bench.recorded_traffic("stale") is None
    assert bench.recorded_traffic("missing", 5) is None


def test_committed_records_name_their_sources():
    recs = bench.traffic_record()
    assert recs, "profiles/traffic.json holds the captured kernels"
    for key, rec in recs.items():
        if not isinstance(rec, dict):
            continue
        assert rec["source_files"] and rec.get("command", "").startswith("ncu ")
        assert "--clock-control none" in rec["command"]
        # exactly one of: bytes per unit, bytes per launch, an event count per launch
        kinds = [k in rec for k in ("bytes_per_unit", "bytes_per_launch", "count_per_launch")]
        assert sum(kinds) == 1, key


def test_recorded_count_checks_the_source_digest(monkeypatch):
    digest = bench.source_digest(bench.RASTER_SOURCES)
    recs = {"fresh": {"source": digest, "source_files": list(bench.RASTER_SOURCES),
                      "count_per_launch": 77},
            "stale": {"source": "0" * 16, "source_files": list(bench.RASTER_SOURCES),
                      "count_per_launch": 77},
            "bytes": {"source": digest, "source_files": list(bench.RASTER_SOURCES),
                      "bytes_per_launch": 5}}
    monkeypatch.setattr(bench, "traffic_record", lambda: recs)
    assert bench.recorded_count("fresh") == 77
    assert bench.recorded_count("stale") is None
    assert bench.recorded_count("bytes") is None
    assert bench.recorded_count("missing") is None
