"""Errors in the large-|q| tail, reported apart from the max-normalised bar.

FFT roundoff is of the order of the largest |Im chi| at every output, while
Im chi itself decays with |q| (Sec. 4, Fig. 5): in the far zones the error
relative to the local value grows although the error relative to the maximum
does not.  This splits sampled errors by |q| into shells one zone wide
(2 pi, lattice constant 1) and into |q| > 4 zones, each as max |error| / max
|Im chi| and as the largest relative error where |Im chi| > 1e-3 max.
"""
import math

import numpy as np


def tail_report(grid, lx, ly, m, got, ref, scale):
    """Rows (label, samples, max abs err / scale, max rel err where
    |ref| > 1e-3 scale or None) per one-zone |q| shell and for |q| > 4 zones."""
    Q, npz = grid["q_extent"], grid["npz"]
    dp = 2.0 * math.pi / npz
    q = np.hypot((np.asarray(lx) - Q // 2) * dp, (np.asarray(ly) - Q // 2) * dp) / (2.0 * math.pi)
    err = np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))
    big = np.abs(ref) > 1e-3 * scale
    rows = []

    def row(label, sel):
        if not np.any(sel):
            return
        rel = err[sel & big] / np.abs(np.asarray(ref)[sel & big]) if np.any(sel & big) else None
        rows.append((label, int(sel.sum()), float(err[sel].max() / scale), None if rel is None else float(rel.max())))

    for z in range(int(math.floor(q.max())) + 1):
        row(f"|q| in [{z}, {z + 1}) zones", (q >= z) & (q < z + 1))
    row("|q| > 4 zones", q > 4)
    return rows


def format_rows(rows):
    return "\n".join(f"  {label}: {n} samples, max err {a:.2e} of max"
                     + ("" if r is None else f", max relative err {r:.2e} where |Im chi| > 1e-3 max")
                     for label, n, a, r in rows)
