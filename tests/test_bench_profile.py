"""The committed ncu summary of the dominant kernel still describes the current sources.

bench.py reports the kernel's measured DRAM traffic only while the sources of the
persistent low-rank kernel hash to the captured version (otherwise "traffic" is null); a
change to those sources must come with a new capture.  CPU only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_lr_profile_matches_current_sources():
    import bench
    per_stage = bench._profiled_traffic(1)
    assert per_stage is not None, "lr_persistent sources changed since the committed ncu capture"
    # the capture read about the algorithmic 340.2 MB of factors per stage
    assert 3.3e8 < per_stage < 3.6e8
    assert bench._profiled_traffic(8) == 8 * per_stage
