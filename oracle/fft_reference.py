"""FP64 FFT reference of the whole output (test infrastructure).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` this module serves the
tests and the bench's CPU legs; the library never imports it, and it calls
nothing from the library.

The direct double sum of ``oracle.imchi_samples`` is the oracle; it costs
O(N^2 n_eps) per output, too much for every output of a 1024 x 1024 x 512
grid.  This module evaluates the same discrete Eq. 9 (Sec. 2) for every
output at once the way Sec. 3 does, through the convolution theorem: with the
T = 0 split a = A [e_j < 0], b = A [e_j >= 0] (Appendix A, Eq. A3),

    C(s_x, s_y, m) = sum_{p, j} a(p, j) b(p + s, j + m)
                   = IFFT[ conj(FFT a) FFT b ](s, m),

in FP64 with numpy/scipy, then Im chi(q_l, w_m) = -c C(l - Q/2, m), c = de / (2 pi)
/ npz^2 (Eq. 9 prefactor, readings as in the C oracle).  The transforms are
circular; they equal the linear correlation when no wanted lag wraps onto a
nonzero term:
  * momentum, extended zone (A = 0 outside the grid): lags |s| <= Q/2 of
    length-N sequences are exact on P >= N + Q/2 points (zero padding);
  * momentum, reduced zone: the band is periodic and the circular
    correlation on P = N points is the wanted one;
  * energy: a lives on j < J0 = n_eps/2 and b on j >= J0, so every lag m of a
    length-n_eps circular correlation is exact (a wrapped partner index
    j + m - n_eps < J0 - 1 lands where b = 0): no energy padding.
It is pinned against the direct sum (tests/test_fft_reference.py) to 1e-12 of
the maximum on every output of small grids.
"""
from __future__ import annotations

import math
import os

import numpy as np


def imchi_fft64(A: np.ndarray, grid: dict, q_extent: int | None = None, n_omega: int | None = None,
                workers: int | None = None) -> np.ndarray:
    """Every output Im chi(q_lx, q_ly, w_m), shape [Q, Q, n_omega], FP64, of
    the discrete Eq. 9 for the spectral function A [N, N, n_eps] on `grid`
    (zones, npz, n_eps, e_max), by FFT correlation.  Peak host memory about
    6 complex128 volumes of [P, P, n_eps/2 + 1]."""
    import scipy.fft as sfft

    zones, npz, n_eps, e_max = grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"]
    N = zones * npz
    Q = int(q_extent if q_extent is not None else grid.get("q_extent") or N)
    n_omega = int(n_omega if n_omega is not None else grid.get("n_omega") or n_eps // 2)
    assert A.shape == (N, N, n_eps)
    if workers is None:
        workers = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    P = N if zones == 1 else N + Q // 2
    de = 2.0 * e_max / n_eps
    c = de / (2.0 * math.pi) / float(npz * npz)
    j = np.arange(n_eps)
    occ = 2 * j + 1 < n_eps                        # e_j < 0, decided on integers

    def forward(part):
        # energy (real input), then p_y and p_x zero-padded to P
        f = sfft.rfft(part, axis=2, workers=workers)
        del part
        f = sfft.fft(f, n=P, axis=1, workers=workers, overwrite_x=True)
        return sfft.fft(f, n=P, axis=0, workers=workers, overwrite_x=True)

    fa = forward(np.where(occ, A, 0.0))
    fb = forward(np.where(occ, 0.0, A))
    np.conjugate(fa, out=fa)
    fb *= fa                                        # conj(a^) b^
    del fa
    sl = (np.arange(Q) - Q // 2) % P                # lag l - Q/2 -> circular index
    f = sfft.ifft(fb, axis=0, workers=workers, overwrite_x=True)
    del fb
    f = np.ascontiguousarray(f[sl])
    f = sfft.ifft(f, axis=1, workers=workers, overwrite_x=True)
    f = np.ascontiguousarray(f[:, sl])
    corr = sfft.irfft(f, n=n_eps, axis=2, workers=workers, overwrite_x=True)
    del f
    out = np.ascontiguousarray(corr[:, :, :n_omega])
    del corr
    out *= -c
    return out


def shell_report(grid: dict, got: np.ndarray, ref: np.ndarray, rel_floor: float = 1e-3):
    """Error of a whole output `got` [Q, Q, n_omega] against `ref`: overall
    max |got - ref| / max |ref|, then per one-zone |q| shell (zone width
    2 pi, lattice constant 1) and for |q| > 4 zones, each as max |error| /
    max |ref| and as the largest relative error where |ref| > rel_floor max."""
    Q, npz = ref.shape[0], grid["npz"]
    scale = float(np.abs(ref).max())
    err = np.abs(got.astype(np.float64) - ref)
    rel = np.where(np.abs(ref) > rel_floor * scale, err / np.maximum(np.abs(ref), 1e-300), 0.0)
    err_q = err.max(axis=2)                         # per lag (lx, ly)
    rel_q = rel.max(axis=2)
    big_q = (np.abs(ref) > rel_floor * scale).any(axis=2)
    del err, rel
    s = (np.arange(Q) - Q // 2) / float(npz)       # lag in zones (q / 2 pi)
    qz = np.hypot(s[:, None], s[None, :])
    rows = [("all outputs", int(got.size), float(err_q.max() / scale), float(rel_q.max()))]

    def row(label, sel):
        if np.any(sel):
            rows.append((label, int(sel.sum()) * ref.shape[2], float(err_q[sel].max() / scale),
                         float(rel_q[sel].max()) if np.any(sel & big_q) else None))

    for z in range(int(math.floor(qz.max())) + 1):
        row(f"|q| in [{z}, {z + 1}) zones", (qz >= z) & (qz < z + 1))
    row("|q| > 4 zones", qz > 4)
    return rows
