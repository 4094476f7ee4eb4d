"""The autotuned plan (LINDHARD_PLAN_AUTOTUNE): every engine variant of the
p_y passes (single-column, paired, paired with 12 values per thread) and of
the product pass (default tile, 12 values per thread) agrees with the FP64
oracle, whichever one a cache file pins, and a fresh tune writes its choices
to the cache file named by LINDHARD_TUNE_CACHE.
"""
import json
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32 = 2e-5

# N = 128 with Q = 128 lags (P = 192, a 3 * 2^k length) and one periodic zone
# of 128 points (P = 128): both take the paired-column engine by default.
GRIDS = [wl.grid_params(2, 64, 40, 1.5), wl.grid_params(1, 128, 32, 1.0)]


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _keys(grid, sizes):
    import torch
    base = (f"{torch.cuda.get_device_name(0)}|P={sizes.fft_p}|N={sizes.N}|PE={sizes.fft_e}"
            f"|Q={sizes.q_extent}")
    return base + "|fwd_y", base + "|inv_y", base + "|x_product", base + "|inv_energy"


def _oracle_samples(grid, band, count=250):
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    lx, ly, m = wl.output_samples(grid, count, seed=7)
    A = oracle.spectral(b, grid)
    return (lx, ly, m), oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)


@pytest.mark.parametrize("grid", GRIDS, ids=["zones2_N128_P192", "zones1_N128_P128"])
def test_pinned_variants_match_oracle(lh, grid, tmp_path, monkeypatch):
    import torch
    band = wl.band_params(filling=1.1, gamma=0.06, ff_a=0.7)
    (lx, ly, m), ref = _oracle_samples(grid, band)
    probe = lh.Plan([grid])
    kf, ki, kx, ke = _keys(grid, probe.sizes[0])
    three_pow = probe.sizes[0].fft_p % 3 == 0
    probe.close()
    # (p_y variant, product variant): 0/1/2 = single-column, paired, paired
    # with 12 values per thread; 3/4 = TMA-staged forms of 1/2.  Product:
    # 0/1 = default and 12-value tiles, 2/3 = their TMA-staged forms.  The
    # 12-value tiles exist for 3 * 2^k only.
    # 8/9 and 6/7: the pruned engine on 8 and 4 column pairs (N = Q = 2P/3 only)
    combos = [(0, 0), (1, 0), (3, 2), (5, 4)] + ([(2, 1), (1, 1), (4, 3), (3, 3), (8, 6), (9, 7)] if three_pow else [])
    outs = []
    for j, (vy, vx) in enumerate(combos):
        ve = j % 2   # inverse energy pass: default and TMA-staged forms in turn
        path = tmp_path / f"tune_{vy}{vx}.json"
        path.write_text(json.dumps({kf: vy, ki: vy, kx: vx, ke: ve}, indent=0))
        monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
        plan = lh.Plan([grid], autotune=True)
        out = plan.imchi([band])
        plan.status()
        s = plan.sizes[0]
        got = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
        plan.close()
        err = np.abs(got[lx, ly, m] - ref).max() / np.abs(ref).max()
        assert err <= TOL32, (vy, vx, ve, err)
        outs.append(got)
    # the engines compute the same transforms: agreement well inside the bar
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() <= TOL32 * np.abs(outs[0]).max()
    torch.cuda.synchronize()


def test_fresh_tune_writes_cache_and_matches_default(lh, tmp_path, monkeypatch):
    import torch
    w = wl.WORKLOADS["extended_256x256x256"]
    grid, band = w["grid"], w["band"]
    path = tmp_path / "tune.json"
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
    plan = lh.Plan([grid], autotune=True)
    out_t = plan.imchi([band])
    plan.status()
    kf, ki, kx, ke = _keys(grid, plan.sizes[0])
    plan.close()
    entries = json.loads(path.read_text())
    assert entries[kf] in range(12) and entries[ki] in range(12) and entries[kx] in range(11) and entries[ke] in (0, 1, 2)
    base = lh.Plan([grid])
    out_d = base.imchi([band])
    base.status()
    base.close()
    mx = float(out_d.abs().max())
    assert mx > 0 and not math.isnan(mx)
    assert float((out_t - out_d).abs().max()) <= TOL32 * mx
    del out_t, out_d
    torch.cuda.empty_cache()


def test_tma_variants_full_size_match_default(lh, tmp_path, monkeypatch):
    """The TMA-staged persistent passes on the extended 256 x 256 x 256 grid
    (P = 384, 256-row tiles, many tiles per CTA) against the default engines."""
    import torch
    w = wl.WORKLOADS["extended_256x256x256"]
    grid, band = w["grid"], w["band"]
    base = lh.Plan([grid])
    out_d = base.imchi([band])
    base.status()
    kf, ki, kx, ke = _keys(grid, base.sizes[0])
    base.close()
    mx = float(out_d.abs().max())
    # 10 / 8: the TMA-staged pruned passes (11: two CTAs per SM); 9 / 10: the
    # pipelined product pass
    for vy, vx, ve in [(3, 2, 1), (4, 3, 0), (5, 2, 1), (6, 5, 0), (10, 8, 2), (8, 9, 2), (10, 10, 0), (11, 10, 2)]:
        path = tmp_path / f"tma_{vy}{vx}.json"
        path.write_text(json.dumps({kf: vy, ki: vy, kx: vx, ke: ve}, indent=0))
        monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
        plan = lh.Plan([grid], autotune=True)
        out_t = plan.imchi([band])
        plan.status()
        plan.close()
        assert float((out_t - out_d).abs().max()) <= TOL32 * mx, (vy, vx, ve)
    del out_t, out_d
    torch.cuda.empty_cache()


def test_pinned_entries_stay_with_their_file(lh, tmp_path, monkeypatch):
    # variants pinned in one cache file are used while it is named, and are
    # neither used nor written once the variable names another file
    probe = lh.Plan([GRIDS[1]])
    kf, ki, kx, ke = _keys(GRIDS[1], probe.sizes[0])
    probe.close()
    pinned = tmp_path / "pinned.json"
    pinned.write_text(json.dumps({kf: 0, ki: 0, kx: 0, ke: 0}, indent=0))
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(pinned))
    plan = lh.Plan([GRIDS[1]], autotune=True)
    assert plan.variants() == {"py_fwd": 0, "py_inv": 0, "px_product": 0, "energy_inv": 0}
    plan.close()
    other = tmp_path / "other.json"
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(other))
    plan = lh.Plan([GRIDS[0]], autotune=True)
    plan.close()
    written = json.loads(other.read_text())
    assert written and not any(k in written for k in (kf, ki, kx, ke))
