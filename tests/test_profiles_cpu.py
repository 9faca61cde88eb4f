"""The DRAM traffic the bench reports for the descent is the figure of the
committed ncu summary (same kernel, same workload), and every profile summary
names the command that produced it (committed files only)."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_bench_traffic_matches_the_dram_summary():
    txt = open(os.path.join(PROFILES, "dp_task_grid4096.md")).read()

    def num(name, unit):
        m = re.search(name + r" \| ([\d,]+) " + unit, txt)
        return int(m.group(1).replace(",", ""))
    rd = num(r"dram__bytes_read\.sum", "B")
    wr = num(r"dram__bytes_write\.sum", "B")
    total = num(r"traffic \(read \+ write\)", "B")
    assert rd + wr == total
    assert bench.MID_DP_TRAFFIC_BYTES in (None, total)
    assert bench.DESCENT_KERNEL in txt
    if bench.MID_DP_ISSUE is not None:
        assert bench.MID_DP_ISSUE["smsp__inst_executed.sum"] == num(r"smsp__inst_executed\.sum",
                                                                    "warp")
        assert bench.MID_DP_ISSUE["smsp__thread_inst_executed.sum"] == num(
            r"smsp__thread_inst_executed\.sum", "thread")


def test_profile_summaries_name_their_commands():
    names = sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))
    assert names
    for f in names:
        txt = open(os.path.join(PROFILES, f)).read()
        assert "ncu " in txt and "--clock-control none" in txt, f
        cmds = re.findall(r"^(python [^\n]+)$", txt, flags=re.M)
        assert cmds, f
        for c in cmds:
            script = c.split()[1]
            if script.endswith(".py"):
                assert os.path.exists(os.path.join(ROOT, script)), (f, script)
            assert "_work" not in c, (f, c)
