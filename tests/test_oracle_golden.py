"""Pins from values the paper prints (tests/golden/): the level-2 example of Fig. 3 and the loop
bounds of Section 5.1, against the oracle's micro-tet enumeration."""
import os

import numpy as np

from oracle import mesh as M

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    out = []
    for line in open(os.path.join(HERE, "golden", "fig3_level2_rows.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            lvl, cls, cnt = line.split()
            out.append((int(lvl), cls, int(cnt)))
    return out


def test_longest_rows_of_fig3():
    groups = {"white_up": [0], "octahedron": [1, 2, 3, 4], "white_down": [5]}
    for level, cls, count in _rows():
        n = 2 ** level
        c, tv = M.micro_tets(n)
        for o in groups[cls]:
            origins = tv[c == o][:, 0, :] - M.CLASS_OFFSETS[o][0]
            # longest row: the x-run at y = z = 0 (Algorithm 2's innermost loop)
            row = origins[(origins[:, 1] == 0) & (origins[:, 2] == 0)]
            assert len(row) == count, (cls, o, len(row))
            assert np.array_equal(np.sort(row[:, 0]), np.arange(count))
