"""bench.py's roofline traffic comes from the ncu captures recorded in
profiles/dram_traffic.json, and only while the captured kernel's sources hash
to the value recorded there (host logic only, no GPU)."""
import importlib.util
import json
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profiled_traffic_follows_the_recorded_hash(tmp_path, monkeypatch):
    b = _bench()
    recs = json.loads((ROOT / "profiles" / "dram_traffic.json").read_text())
    assert recs, "no capture recorded"
    for key, rec in recs.items():
        kernel, workload = key.split("@")
        assert kernel in b.KERNEL_SOURCES and len(rec["source_sha16"]) == 16
        assert rec["dram_bytes_per_iteration"] > 0 and rec["summary"].startswith("profiles/")
        assert (ROOT / rec["summary"]).exists()
        got = b.profiled_traffic_per_iteration(kernel, workload)
        if rec["source_sha16"] == b.kernel_source_hash(kernel):
            assert got == rec["dram_bytes_per_iteration"]
        else:
            assert got is None
    # a record whose hash no longer matches the sources gives no traffic
    fake = tmp_path / "dram_traffic.json"
    fake.write_text(json.dumps({"k_persistent@hydro401": {
        "source_sha16": "0" * 16, "dram_bytes_per_iteration": 1.0,
        "summary": "profiles/k_persistent_hydro401.md"}}))
    monkeypatch.setattr(b, "TRAFFIC_FILE", fake)
    assert b.profiled_traffic_per_iteration("k_persistent", "hydro401") is None
