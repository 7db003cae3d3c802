"""Host-side bookkeeping of bench.py that the JSON line relies on (no GPU)."""

import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_box_extents_match_the_library():
    # the class rule the launch count mirrors is the library's own table
    with open(os.path.join(ROOT, "paper_1606_05562_gb300", "csrc", "atdct16_internal.h")) as f:
        text = f.read()
    m = re.search(r"kZonalBoxK\[kZonalBoxClasses\]\s*=\s*\{([^}]*)\}", text)
    assert m is not None
    assert tuple(int(v) for v in m.group(1).split(",")) == bench.BOX_EXTENTS


def test_zonal_launches_per_call():
    # one kernel per non-empty class, then the PSNR finalize
    assert bench.zonal_launches_per_call(bench.R_SWEEP) == 6  # four box extents and the general kernel
    assert bench.zonal_launches_per_call([0]) == 2            # r = 0 runs the general kernel
    assert bench.zonal_launches_per_call([1, 1, 1]) == 2
    assert bench.zonal_launches_per_call([2, 3, 6]) == 2      # all within the 3 x 3 corner
    assert bench.zonal_launches_per_call([6, 7]) == 3         # 7 needs the 6 x 6 corner
    assert bench.zonal_launches_per_call([36, 37]) == 3       # 37 leaves the 8 x 8 corner
    assert bench.zonal_launches_per_call([64, 256, 0]) == 2
