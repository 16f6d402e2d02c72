"""Host-side arithmetic of bench.py (CPU): the group counts its roofline divides by, against the
oracle's own reference grids."""
import os
import sys

import numpy as np

from oracle import htsvd_oracle as O

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _oracle_groups(shape, sub, prm):
    p = O.Params.of(prm)
    total = 0
    for z0, z1 in O.subimage_bounds(shape[0], sub[0]):
        for y0, y1 in O.subimage_bounds(shape[1], sub[1]):
            for x0, x1 in O.subimage_bounds(shape[2], sub[2]):
                total += len(O.volume_reference_positions((z1 - z0, y1 - y0, x1 - x0), p))
    return total


def test_adaptive_volume_group_count_matches_the_oracle_grid():
    prm = dict(ps=4, stride=2, window=5, K=32)
    for shape, sub in (((176, 208, 176), (88, 104, 88)), ((24, 26, 29), (12, 13, 14)), ((41, 17, 30), (20, 100, 7))):
        assert bench.volume_adaptive_groups(shape, sub, 4, 2) == _oracle_groups(shape, sub, prm)
    assert bench.volume_adaptive_groups((176, 208, 176), (88, 104, 88), 4, 2) == 8 * 43 * 51 * 43
    # a single part is the whole volume's grid (the mri176 workload's 87 x 103 x 87 groups)
    assert bench.volume_adaptive_groups((176, 208, 176), (176, 208, 176), 4, 2) == 87 * 103 * 87
    assert np.isfinite(bench.volume_flops_per_group(32))
