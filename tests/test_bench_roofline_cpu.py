"""The benchmark's roofline arithmetic against the figure the paper prints
(Sec. V-A: 92.4 GB/s of copy bandwidth gives 304 MLUP/s for D3Q19 in FP64;
tests/golden/roofline_skylake.txt)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _golden():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "roofline_skylake.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k] = float(v)
    return vals


def test_paper_roofline_figure():
    g = _golden()
    mlups = bench.roofline_mlups(g["bandwidth_gbs"], int(g["q"]), int(g["bytes_per_value"]))
    assert round(mlups) == g["mlups"], mlups


def test_algorithmic_bytes():
    # D3Q19 FP32: 152 B per cell; the channel adds the 4 B link mask of every cell
    assert bench.algorithmic_bytes(19, 4, 1) == 152
    assert bench.algorithmic_bytes(19, 2, 10, 12) == 19 * 2 * 2 * 10 + 48
    assert bench.algorithmic_bytes(27, 4, 384 ** 3) == 216 * 384 ** 3
