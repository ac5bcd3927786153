"""The committed DRAM-traffic records of the X-stream kernels
(profiles/*_traffic.json) belong to the current kernel sources: the bench
reports a record's traffic only while the hash of the sources it was taken
from matches, so a kernel change must come with a new capture."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["c1s", "c2s"])
def test_traffic_record_matches_current_sources(workload):
    import bench
    spec = bench.TRAFFIC_RECORDS[workload]
    with open(os.path.join(ROOT, "profiles", spec["record"])) as f:
        rec = json.load(f)
    assert rec["sources"] == spec["sources"]
    assert rec["sources_sha256"] == bench.sources_sha256(spec["sources"]), (
        f"{spec['record']} was captured from other sources; recapture it with its recorded command")
    assert rec["workload"] == spec["full"] and rec["dram_bytes_per_launch"] > 0
    # traffic is at least the bytes the kernel must read, and not wildly above them
    assert 0.95 <= rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] <= 2.0
