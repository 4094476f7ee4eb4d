"""The tail-error report helper (CPU): shells by |q| in zones, the |q| > 4
zone bucket, and the relative error restricted to values above 1e-3 max."""
import math

import numpy as np

from tail_report import format_rows, tail_report


def test_tail_report_on_a_planted_error():
    grid = dict(q_extent=64, npz=8)          # dp = 2 pi / 8: |q| up to 4 zones per axis
    lx = np.array([32, 40, 48, 63, 0])       # |q_x| = 0, 1, 2, 3.875, 4 zones (l_y = Q/2)
    ly = np.full(5, 32)
    ref = np.array([-1.0, -0.5, -0.1, -1e-4, -2e-3])
    got = ref.copy()
    got[2] += 1e-6                           # 1e-6 of max in the third shell
    got[4] += 2e-6                           # and 2e-6 at |q| = 4 zones exactly
    rows = tail_report(grid, lx, ly, np.zeros(5, int), got, ref, 1.0)
    by = {r[0]: r for r in rows}
    assert by["|q| in [0, 1) zones"][1:3] == (1, 0.0)
    assert math.isclose(by["|q| in [2, 3) zones"][2], 1e-6) and math.isclose(by["|q| in [2, 3) zones"][3], 1e-5)
    assert by["|q| in [3, 4) zones"][3] is None                       # |ref| below 1e-3 max: no relative figure
    assert math.isclose(by["|q| in [4, 5) zones"][2], 2e-6) and math.isclose(by["|q| in [4, 5) zones"][3], 1e-3)
    assert "|q| > 4 zones" not in by                                   # 4 zones is not beyond 4
    assert "max relative err" in format_rows(rows)
