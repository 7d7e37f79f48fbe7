"""bench.py's roofline traffic comes from the committed ncu summary of the
FP64 iteration kernel, and only while the kernel sources hash to the value
recorded there (host logic only, no GPU)."""
import importlib.util
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profiled_traffic_follows_the_recorded_hash():
    b = _bench()
    text = (ROOT / "profiles" / "k_persistent_hydro401.md").read_text().splitlines()
    rec = [l.rsplit(":", 1)[1].strip() for l in text if l.startswith("kernel source sha256[:16]:")]
    dram = [float(l.split(":", 1)[1]) for l in text if l.startswith("dram bytes per iteration:")]
    assert len(rec) == 1 and len(dram) == 1 and len(rec[0]) == 16
    got = b.profiled_traffic_per_iteration()
    if rec[0] == b.kernel_source_hash():
        assert got == dram[0]
    else:
        assert got is None
