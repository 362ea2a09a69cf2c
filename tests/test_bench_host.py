"""Host-side pieces of bench.py, on the CPU: the byte models behind the
roofline object, the parser of the committed ncu traffic table, and the
reference arm (the oracle on a bounded sample) printing its contract line."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def test_staged_bytes_cover_every_kernel_and_sum_to_the_floor():
    steps = set()
    assert set(bench.ALG_BYTES) <= set(bench.STEP_OF_KERNEL)
    for k, st in bench.STEP_OF_KERNEL.items():
        assert k in bench.ALG_BYTES or k.startswith("scan"), k  # prefix sums: no own model
        parts = st.split("+")
        assert all(s in bench.STAGED_BYTES for s in parts), (k, st)
        assert bench.staged_bytes(k) == sum(bench.STAGED_BYTES[s] for s in parts)
        steps.update(parts)
    assert steps == set(bench.STAGED_BYTES)  # every step has a kernel
    assert bench.STAGED_TOTAL == 85 and bench.COMPULSORY_BYTES == 21
    assert bench.staged_bytes("density") == 40  # rho and nh/delta in one kernel


def test_traffic_table_parses_with_hashes_and_issue_shares():
    rows = bench.parse_traffic()
    assert {"density", "fill_cells", "fill_place", "assign"} <= set(rows)
    for k, (bph, h, issue) in rows.items():
        assert k in bench.ALG_BYTES
        assert 0.0 < bph < 200.0
        assert len(h) == 12 and all(c in "0123456789abcdef" for c in h)
        assert issue is None or 0.0 < issue <= 1.0
    # the density kernel moves about its staged floor (rho never round-trips)
    assert abs(rows["density"][0] - bench.staged_bytes("density")) < 0.2 * 40


def test_source_hash_ignores_comments_and_host_files():
    h = bench.source_hash()
    assert len(h) == 12 and h == bench.source_hash()


def test_reference_arm_prints_its_contract_line():
    out = subprocess.run(
        [sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--events", "8",
         "--lo", "10000", "--hi", "20000", "--steps", "1", "--warmup", "0"],
        capture_output=True, text=True, timeout=600, cwd=str(ROOT))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Mhits/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert e2e["value"] == line["value"]
