"""The committed ncu counters describe the stepping kernel as it is built:
profiles/traffic.txt must carry a line for the current sources' digest (the
bench reports DRAM traffic only then), so a kernel change without a new
capture shows here rather than as a silent null in the bench line."""
import bench
from paper_2604_06947_gb300 import build as B


def test_traffic_counters_match_the_current_kernel():
    for tag, workload in (("k_step_tb:L4:V16:B64", "burgers_lf_2^20_cells_K64"),
                          ("k_step_tb:L2:V8:B128", "upwind_closed_2^24_cells_K64")):
        c = bench.profiled_counters(tag, B.kernel_digest(), workload)
        assert c.get("dram_bytes_per_launch", 0) > 0, "recapture profiles/traffic.txt"
        assert c.get("warp_instructions_per_launch", 0) > 0
