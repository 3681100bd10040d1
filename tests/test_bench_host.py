"""Host-side arithmetic of bench.py's roofline fields (CPU)."""
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_is_the_dram_bytes_of_a_whole_launch():
    """The committed ncu summary stores bytes per cell-update; the bench's
    traffic field is per launch, i.e. times the steps one launch advances
    (two for the temporally blocked kernel).  Entries whose counters predate
    the current kernel sources are reported as null and skipped here."""
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        summary = json.load(f)
    cells = 8192 * 8192
    for name, e in summary.items():
        t = bench.traffic_per_launch(name, cells)
        if t is None:
            assert e.get("source_hash") != bench.kernel_source_hash(name)
            continue
        assert abs(t - e["bytes_per_launch"]) <= 1e-9 * e["bytes_per_launch"], name
        assert abs(e["bytes_per_cell"] * cells * e.get("steps_per_launch", 1) - e["bytes_per_launch"]) <= \
            1e-9 * e["bytes_per_launch"], name
    assert bench.traffic_per_launch("no such kernel", cells) is None


def test_learned_kernel_counters_follow_the_kernel_source():
    """The learned record carries the committed ncu counters of the fused
    learned step only while its sources hash to the value they were taken
    on; otherwise null."""
    import bench
    name = "learned_step_kernel<2,2>"
    with open(os.path.join(ROOT, "profiles", "learned_kernel.json")) as f:
        rec = json.load(f)[name]
    got = bench.kernel_counters(name)
    if got is None:
        assert rec["source_hash"] != bench.kernel_source_hash(name)
    else:
        assert got["tensor_pipe_pct"] == rec["tensor_pipe_pct"]
        assert abs(got["dram_bytes_per_cell_step"] * 152 * 256 * 256 * 64 -
                   (rec["dram_read_bytes"] + rec["dram_write_bytes"])) <= 1e-3 * rec["dram_read_bytes"]
    assert bench.kernel_counters("no such kernel") is None
