"""Host-side pieces of bench.py's roofline (no GPU): the per-phase
algorithmic bytes follow their stated formulas, the committed traffic record
covers the three measured phases and is used only while the phases' sources
hash to the recorded values (null after a change, until it is re-taken), and the second oracle's whole-graph rate is read
from the golden file's header."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_phase_bytes_formulas():
    tm = {"gamma_entries": 1000, "t_members": 100, "edges": 10, "wedges": 7}
    L, M, smin = 8, 10, 500
    b = bench.phase_bytes(tm, L, M, smin)
    assert b["tau"] == 4 * smin + (8 + 4 * L) * M
    assert b["count"] == 4 * 1000 + 100 * 4 * (3 * L + 3) + 10 * (28 + 12 * L + 16 * L * L)
    assert b["cycles"] == 4 * 7
    assert b["cliques"] is None


def test_traffic_record_is_keyed_by_sources(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    for ph in ("tau", "count", "cycles"):
        assert rec[ph]["workload"] == "rmat23" and rec[ph]["dram_bytes_per_unit"] > 0
        current = rec[ph]["sources_sha256"] == bench.phase_sources_sha256(ph)
        want = rec[ph]["dram_bytes_per_unit"] if current else None
        assert bench.committed_traffic("rmat23", ph) == want, ph
        assert bench.committed_traffic("cl1m", ph) is None  # another workload: no figure
    # a changed source disowns the record
    monkeypatch.setattr(bench, "phase_sources_sha256", lambda ph: "0" * 64)
    assert bench.committed_traffic("rmat23", "cycles") is None


def test_recorded_second_oracle_rate():
    rec = bench.recorded_oracle2("rmat23")
    assert rec is not None and rec["cores"] >= 1 and rec["seconds"] > 0
    assert abs(rec["edges_per_s"] - 129338312 / rec["seconds"]) < 1e-6
    assert bench.recorded_oracle2("er1000") is None
