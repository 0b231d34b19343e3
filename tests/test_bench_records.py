"""Host logic of bench.py's measurement records, on CPU: the per-launch DRAM
traffic it reports comes only from a record taken on the current kernel
sources, and the committed record parses."""
import bench


def test_traffic_record_is_used_only_for_the_current_sources(tmp_path, monkeypatch):
    cur = bench.source_hash()
    rec = tmp_path / "dram_traffic.txt"
    rec.write_text("# comment line\n"
                   f"kernel x_inverse workload large bytes_per_launch 722000000 source {cur}\n"
                   "kernel z_convolve workload large bytes_per_launch 987000000 source 0000000000000000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.ncu_traffic("x_inverse", "large") == 722000000.0
    # a record of other sources, another workload or an unknown kernel is not used
    assert bench.ncu_traffic("z_convolve", "large") is None
    assert bench.ncu_traffic("x_inverse", "yig_wire") is None
    assert bench.ncu_traffic("y_forward", "large") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.txt"))
    assert bench.ncu_traffic("x_inverse", "large") is None


def test_source_hash_follows_the_kernel_sources(tmp_path, monkeypatch):
    src = tmp_path / "csrc"
    src.mkdir()
    (src / "a.cu").write_text("int a;\n")
    monkeypatch.setattr(bench, "SRC_DIR", str(src))
    h0 = bench.source_hash()
    assert len(h0) == 16 and h0 == bench.source_hash()
    (src / "a.cu").write_text("int a; // changed\n")
    assert bench.source_hash() != h0


def test_committed_traffic_record_parses():
    n = 0
    with open(bench.TRAFFIC_FILE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(zip(*[iter(line.split())] * 2))
            assert set(kv) == {"kernel", "workload", "bytes_per_launch", "source"}, line
            assert float(kv["bytes_per_launch"]) > 0
            assert len(kv["source"]) == 16
            n += 1
    assert n >= 5
