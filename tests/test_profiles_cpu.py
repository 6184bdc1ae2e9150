"""The committed ncu summaries that bench.py reads its traffic figures from:
each names a kernel bench.py knows, carries every machine-read field with a
sensible value, and gives the command that made it (running committed files)."""
import glob
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _machine_read(path):
    vals = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals


SUMMARIES = [p for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
             if "source_sha256" in open(p).read()]


def test_there_are_summaries():
    assert len(SUMMARIES) >= 5


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_summary_is_machine_readable(path):
    import bench
    name = os.path.basename(path)[:-3]
    kernel = next(k for k in bench.KERNEL_SOURCES if name.startswith(k + "_"))
    vals = _machine_read(path)
    assert len(vals["source_sha256"]) == 64 and int(vals["source_sha256"], 16) >= 0
    assert float(vals["dram_bytes_per_launch"]) > 0 and float(vals["sweeps_per_launch"]) > 0
    assert vals["traffic_scales_with_sweeps"].split()[0] in ("yes", "no")
    text = open(path).read()
    assert "ncu " in text and "--clock-control none" in text and "python bench.py" in text
    assert kernel in text
