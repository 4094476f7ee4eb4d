"""The energy passes with one warp per line (forward: k_fwd_energy_warp,
used for every FP32 grid at T = 0 with an energy FFT of 128, 256 or 512
points; inverse: k_inv_energy_warp, engine variant 2 of the inverse energy
pass) against the FP64 oracle.

Covered: the energy FFT lengths 128, 256 and 512, each with n_eps equal to
the length (no energy padding) and below it (odd n_eps included, so that
e = 0 falls on a grid point); n_omega at half the energies, at all of them
and a ragged few; the caller-supplied-A path; both inverse forms on the same
plan geometry.  Bar: 2e-5 of max|Im chi| (FP32), every output on tiny grids,
seeded samples on the others.
"""
import json

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _band(grid, **kw):
    b = wl.band_params(filling=kw.get("filling", 1.12), gamma=kw.get("gamma", 0.07), ff_a=0.8)
    bo = dict(b)
    bo["mu"] = oracle.solve_mu(bo["kind"], bo["t"], bo["tp"], bo["tpp"], bo["gamma"], grid["npz"], bo["filling"])
    return b, bo


def _plan_out(lh, grid, band, tmp_path, monkeypatch, inv_energy):
    """One forward call with the inverse energy variant pinned through a cache file."""
    import torch
    probe = lh.Plan([grid])
    s = probe.sizes[0]
    probe.close()
    base = (f"{torch.cuda.get_device_name(0)}|P={s.fft_p}|N={s.N}|PE={s.fft_e}|Q={s.q_extent}")
    path = tmp_path / f"tune_{inv_energy}.json"
    path.write_text(json.dumps({base + "|fwd_y": 1, base + "|inv_y": 1, base + "|x_product": 0,
                                base + "|inv_energy": inv_energy}, indent=0))
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
    plan = lh.Plan([grid], autotune=True)
    assert plan.variants()["energy_inv"] == inv_energy
    out = plan.imchi([band])
    plan.status()
    got = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    plan.close()
    return got, s


# N = 96 pads to P = 192 (the autotuner's range, so the inverse variant can be pinned)
@pytest.mark.parametrize("n_eps,n_omega", [(128, 64), (100, 50), (256, 128), (200, 200), (512, 256),
                                           (333, 7), (512, 512)])
def test_energy_warp_passes_match_oracle(lh, tmp_path, monkeypatch, n_eps, n_omega):
    grid = wl.grid_params(2, 48, n_eps, 2.0, n_omega=n_omega)
    band, bo = _band(grid)
    lx, ly, m = wl.output_samples(grid, 250, seed=5, near_origin=4)
    A = oracle.spectral(bo, grid)
    ref = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    del A
    outs = []
    for v in (0, 2):
        got, s = _plan_out(lh, grid, band, tmp_path, monkeypatch, v)
        assert s.fft_e in (128, 256, 512) and s.fft_p == 192
        err = np.abs(got[lx, ly, m] - ref).max() / np.abs(ref).max()
        assert err <= TOL32, (v, err)
        assert got.max() <= TOL32 * np.abs(got).max()          # Im chi <= 0
        assert np.abs(got[:, :, 0]).max() <= TOL32 * np.abs(got).max()   # Im chi(q, 0) = 0
        outs.append(got)
    # the two inverse forms agree over the whole output
    assert np.abs(outs[0] - outs[1]).max() <= TOL32 * np.abs(outs[0]).max()


@pytest.mark.parametrize("n_eps", [128, 90, 256, 512])
def test_energy_warp_caller_supplied_A_every_output(lh, n_eps):
    # a random A with no symmetry through the caller-A path of the warp pass
    grid = wl.grid_params(2, 6, n_eps, 1.0, n_omega=min(n_eps, 40), q_extent=24)
    A = wl.random_spectral(grid, seed=9)
    import torch
    plan = lh.Plan([grid])
    s = plan.sizes[0]
    assert s.fft_e in (128, 256, 512)
    out = plan.imchi(None, A_in=torch.from_numpy(A).cuda().reshape(-1))
    plan.status()
    got = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    plan.close()
    ref = oracle.imchi_full(A.astype(np.float64), grid, grid["q_extent"], grid["n_omega"])
    assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max()


@pytest.mark.parametrize("n_eps", [128, 256])
def test_energy_warp_every_output_small_grid(lh, n_eps):
    # every output of a small generated grid (ragged momentum count: N = 20)
    grid = wl.grid_params(2, 10, n_eps, 1.5, n_omega=n_eps // 2)
    band, bo = _band(grid, gamma=0.09)
    import torch
    plan = lh.Plan([grid])
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = plan.imchi([band], mu_out=mu)
    plan.status()
    s = plan.sizes[0]
    got = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    plan.close()
    assert abs(mu.item() - bo["mu"]) < 1e-10
    ref = oracle.imchi_full(oracle.spectral(bo, grid), grid, grid["q_extent"], grid["n_omega"])
    assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max()
