"""The DRAM traffic bench.py reports for the dominant kernel is the figure of the committed ncu
summary it cites (so the two cannot drift apart when a kernel is recaptured)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reported_traffic_matches_the_ncu_summary():
    import bench
    text = open(os.path.join(ROOT, "profiles", "pk_solve1_fp64_1024x1024_ncu.md")).read()
    m = re.search(r"= ([0-9.]+) MB per iteration", text)
    assert m, "the summary states the DRAM bytes per iteration"
    assert abs(bench.NCU_TRAFFIC["kry_persistent"] - float(m.group(1)) * 1e6) < 0.05e6
    # the bench names the summary it takes the figure from
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert "profiles/pk_solve1_fp64_1024x1024_ncu.md" in src


def test_profile_commands_use_committed_entry_points():
    """Every summary gives the command that made it, running bench.py (committed) under ncu."""
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "ncu " in text and "--clock-control none" in text, name
        assert "python bench.py" in text, name
        assert "_work" not in text, name
