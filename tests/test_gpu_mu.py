"""The chemical-potential solve on the GPU against the oracle's FP64 bisection
(Sec. 3: the Fermi level is placed to hold the filling; the occupation is the
Lorentzian one of Eq. 5).  Covers the three-pass multisection taken for
gamma < 0.02 eV, zones beyond 512 points per axis, the free-electron band,
fillings far from half filling, and a filling the search interval cannot
reach (reported as LINDHARD_ENOCONV by lindhard_plan_status).  Zones of at
most 98 points per axis solve in one CTA of the set-up launch, larger ones in
the multi-CTA passes: both paths are checked on each side of the boundary."""
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _gpu_mu(lh, grid, band):
    import torch
    plan = lh.Plan([grid])
    mu = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    plan.imchi([band], mu_out=mu)
    try:
        plan.status()
    finally:
        plan.close()
    return mu.item()


@pytest.mark.parametrize("gamma", [0.005, 0.01, 0.019, 0.02, 0.2])
@pytest.mark.parametrize("filling", [0.35, 1.04, 1.17, 1.7])
def test_mu_matches_oracle_across_gamma_and_filling(lh, gamma, filling):
    grid = wl.grid_params(2, 32, 16, 1.0)
    band = wl.band_params(filling=filling, gamma=gamma)
    ref = oracle.solve_mu(0, band["t"], band["tp"], band["tpp"], gamma, grid["npz"], filling)
    got = _gpu_mu(lh, grid, band)
    assert abs(got - ref) < 1e-10, (got, ref)


@pytest.mark.parametrize("npz", [6, 1024])
def test_mu_small_and_large_zones(lh, npz):
    """npz = 6 (4 symmetry classes per axis) and one zone of 1024 x 1024
    points (a size the previous point-by-point solve did not accept)."""
    zones = 2 if npz == 6 else 1
    grid = wl.grid_params(zones, npz, 16, 1.0)
    band = wl.band_params(filling=1.1, gamma=0.03)
    ref = oracle.solve_mu(0, band["t"], band["tp"], band["tpp"], 0.03, npz, 1.1)
    got = _gpu_mu(lh, grid, band)
    assert abs(got - ref) < 1e-10, (got, ref)


def test_mu_free_electrons(lh):
    grid = wl.grid_params(4, 16, 16, 2.0)
    band = wl.band_params(filling=0.3, gamma=0.05, kind=1, t=0.0, tp=0.0, tpp=0.0)
    ref = oracle.solve_mu(1, 0.0, 0.0, 0.0, 0.05, 16, 0.3)
    got = _gpu_mu(lh, grid, band)
    assert abs(got - ref) < 1e-10, (got, ref)


def test_unreachable_filling_reports_enoconv(lh):
    """Filling 1.9999 with gamma = 0.2 eV: the Lorentzian tails keep n(mu)
    below it on the whole search interval [-B-3, B+3] eV, so the solve reports
    that it found no chemical potential (a status code, no fault)."""
    grid = wl.grid_params(2, 16, 16, 1.0)
    band = wl.band_params(filling=1.9999, gamma=0.2)
    B = 4 * (abs(band["t"]) + abs(band["tp"]) + abs(band["tpp"]))
    assert oracle.filling(0, band["t"], band["tp"], band["tpp"], 0.2, 16, B + 3.0) < 1.9999
    with pytest.raises(lh.LindhardError, match="ENOCONV"):
        _gpu_mu(lh, grid, band)
    # the plan's status word is per plan: a fresh plan solves a reachable filling
    ok = wl.band_params(filling=1.15, gamma=0.2)
    ref = oracle.solve_mu(0, ok["t"], ok["tp"], ok["tpp"], 0.2, 16, 1.15)
    assert abs(_gpu_mu(lh, grid, ok) - ref) < 1e-10


@pytest.mark.parametrize("gamma", [0.005, 0.019, 0.05])
@pytest.mark.parametrize("npz", [64, 96, 98, 100, 128])
def test_mu_on_both_solve_paths(lh, npz, gamma):
    # npz <= 98: the one-CTA solve (a bracketed Newton iteration and the
    # Halley step in the set-up launch); npz >= 100: the multi-CTA passes
    grid = wl.grid_params(1, npz, 16, 1.0) if npz in (64, 128) else wl.grid_params(2, npz, 16, 1.0)
    band = wl.band_params(filling=1.13, gamma=gamma)
    ref = oracle.solve_mu(0, band["t"], band["tp"], band["tpp"], gamma, npz, 1.13)
    got = _gpu_mu(lh, grid, band)
    assert abs(got - ref) < 1e-10, (npz, gamma, got, ref)


@pytest.mark.parametrize("npz", [16, 128])
def test_enoconv_on_both_solve_paths(lh, npz):
    grid = wl.grid_params(1, npz, 16, 1.0)
    band = wl.band_params(filling=1.9999, gamma=0.2)
    with pytest.raises(lh.LindhardError, match="ENOCONV"):
        _gpu_mu(lh, grid, band)
