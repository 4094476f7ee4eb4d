"""The FP64 FFT reference (oracle/fft_reference.py) pinned to the direct sum.

The direct double sum of the discrete Eq. 9 (oracle.imchi_samples) is the
oracle; the FFT reference evaluates the same sum for every output at once
through the convolution theorem (Sec. 3), and is used where the direct sum
is too slow for a whole output (the 1024 x 1024 x 512 precision study).
Here it must reproduce the direct sum on every output of small grids, in
both zone kinds, with ragged lag counts, odd energy counts and a random A
with no symmetry, to 1e-12 of the maximum (FP64 rounding), and on seeded
samples of a larger grid.  Its shell report is checked on planted errors.
"""
import numpy as np
import pytest

import oracle
from oracle.fft_reference import imchi_fft64, shell_report
from paper_1208_3210_gb300 import workloads as wl


def _band(grid, filling=1.1, gamma=0.08):
    b = wl.band_params(filling=filling, gamma=gamma, ff_a=0.9)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    return b


@pytest.mark.parametrize("kw", [
    dict(zones=2, npz=8, n_eps=24, e_max=1.0),                         # extended, Q = N
    dict(zones=1, npz=16, n_eps=20, e_max=1.0),                        # reduced zone (periodic)
    dict(zones=3, npz=6, n_eps=33, e_max=1.5, q_extent=36, n_omega=33),  # all lags, odd n_eps, every transfer
    dict(zones=2, npz=10, n_eps=16, e_max=2.0, q_extent=6, n_omega=3),   # few lags and transfers
    dict(zones=1, npz=8, n_eps=7, e_max=0.8, q_extent=4),              # reduced zone, Q < N, n_eps odd
])
def test_matches_direct_sum_every_output(kw):
    grid = wl.grid_params(kw["zones"], kw["npz"], kw["n_eps"], kw["e_max"], kw.get("n_omega", 0),
                          kw.get("q_extent", 0))
    A = oracle.spectral(_band(grid), grid)
    ref = oracle.imchi_full(A, grid, grid["q_extent"], grid["n_omega"])
    got = imchi_fft64(A, grid)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_random_spectral_function_every_output():
    grid = wl.grid_params(2, 7, 18, 1.0, n_omega=18, q_extent=28)
    A = wl.random_spectral(grid, seed=4).astype(np.float64)
    ref = oracle.imchi_full(A, grid, grid["q_extent"], grid["n_omega"])
    got = imchi_fft64(A, grid)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_matches_direct_sum_samples_larger_grid():
    grid = wl.grid_params(4, 16, 128, 2.0)
    A = oracle.spectral(_band(grid, gamma=0.05), grid)
    lx, ly, m = wl.output_samples(grid, 400, seed=2)
    ref = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    got = imchi_fft64(A, grid)[lx, ly, m]
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_shell_report_on_planted_errors():
    # a known error planted at one lag: the overall row and the right shell see it
    grid = wl.grid_params(8, 4, 8, 1.0)                 # Q = 32 lags of 1/4 zone
    rng = np.random.default_rng(0)
    ref = -rng.uniform(0.5, 1.0, size=(32, 32, 4))
    got = ref.copy()
    got[31, 31, 2] += 1e-3                               # lag (15, 15): |q| = 5.3 zones
    rows = dict((r[0], r) for r in shell_report(grid, got, ref))
    scale = np.abs(ref).max()
    assert rows["all outputs"][2] == pytest.approx(1e-3 / scale)
    assert rows["|q| in [5, 6) zones"][2] == pytest.approx(1e-3 / scale)
    assert rows["|q| > 4 zones"][2] == pytest.approx(1e-3 / scale)
    assert rows["|q| in [0, 1) zones"][2] == 0.0
    assert rows["|q| in [5, 6) zones"][3] == pytest.approx(1e-3 / abs(ref[31, 31, 2]))
