"""Finite temperature on the GPU (grids with quantity LINDHARD_IMCHI_T or
LINDHARD_SQW): Im chi_T with the occupation difference f(e) - f(e + w)
(Appendix A, Eq. A1) and the dynamical structure factor S(q, w) of Eq. 1,
against the FP64 oracle's direct sums (oracle.thermal_samples).

Bars: FP32 2e-5 of max|ref| per instance (every output on small grids,
seeded samples on the 256^3 workload); FP64 1e-12.  Each case prints the
error it measured.
"""
import json
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32, TOL64 = 2e-5, 1e-12


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _solved(band, grid):
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    return b


def _gpu(lh, grid, band, precision=None, A_in=None):
    g = dict(grid)
    if precision is not None:
        g["precision"] = precision
    plan = lh.Plan([g])
    out = plan.imchi([band], A_in=A_in)
    plan.status()
    s = plan.sizes[0]
    res = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    fft_e = s.fft_e
    plan.close()
    return res, fft_e


CASES = [
    # (grid, band, kT)
    (wl.grid_params(2, 16, 32, 1.5), wl.band_params(filling=1.1, gamma=0.08, ff_a=0.8), 0.05),
    (wl.grid_params(2, 16, 33, 1.5, n_omega=20), wl.band_params(filling=1.2, gamma=0.05, ff_a=1.0), 0.01),
    (wl.grid_params(1, 32, 24, 1.0), wl.band_params(filling=0.9, gamma=0.1), 0.3),
    (wl.grid_params(2, 12, 30, 1.2, q_extent=48), wl.band_params(filling=1.15, gamma=0.06, ff_a=0.6), 0.1),
]
IDS = ["extended_kT0.05", "odd_eps_kT0.01", "reduced_kT0.3", "all_lags_kT0.1"]


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
@pytest.mark.parametrize("grid,band,kT", CASES, ids=IDS)
def test_thermal_against_oracle(lh, grid, band, kT, quantity):
    g = dict(grid, quantity=quantity)
    b = dict(band, kT=kT)
    got, fft_e = _gpu(lh, g, b)
    assert fft_e >= grid["n_eps"] + grid["n_omega"] - 1
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_full(A, grid, grid["q_extent"], grid["n_omega"], kT, quantity)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"quantity {quantity}, kT {kT}: {err:.2e} of max (PE = {fft_e})")
    assert err <= TOL32
    if quantity == 2:
        assert got.min() >= -TOL32 * np.abs(ref).max()      # S >= 0


# energy FFT lengths that take the warp-per-line forward pass with the
# Fermi-weight table: 128 (a power of two, padded), 384 and 768 (24 values a
# thread); small momentum grids and few lags keep the oracle's direct sums short
WARP_CASES = [
    (wl.grid_params(2, 8, 100, 1.5, n_omega=20), 0.05, 128),
    (wl.grid_params(2, 8, 256, 1.5, q_extent=12), 0.025, 384),
    (wl.grid_params(2, 8, 512, 3.0, q_extent=8), 0.025, 768),
]


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
@pytest.mark.parametrize("grid,kT,pe", WARP_CASES, ids=["PE128", "PE384", "PE768"])
def test_thermal_warp_energy_lengths(lh, grid, kT, pe, quantity):
    import torch
    band = wl.band_params(filling=1.1, gamma=0.06, ff_a=0.8)
    g = dict(grid, quantity=quantity)
    got, fft_e = _gpu(lh, g, dict(band, kT=kT))
    assert fft_e == pe
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_full(A, grid, grid["q_extent"], grid["n_omega"], kT, quantity)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"PE {pe}, quantity {quantity}: {err:.2e} of max")
    assert err <= TOL32
    # the same grid with the spectral function supplied by the caller
    N = grid["zones"] * grid["npz"]
    Ar = np.random.default_rng(pe).random((N, N, grid["n_eps"]))
    got_a, _ = _gpu(lh, g, dict(band, kT=kT), A_in=torch.tensor(Ar.ravel(), dtype=torch.float32, device="cuda"))
    ref_a = oracle.thermal_full(Ar.astype(np.float32).astype(np.float64), grid, grid["q_extent"],
                                grid["n_omega"], kT, quantity)
    err_a = np.abs(got_a - ref_a).max() / np.abs(ref_a).max()
    print(f"PE {pe}, quantity {quantity}, caller A: {err_a:.2e} of max")
    assert err_a <= TOL32


# the warp-per-pair inverse energy pass (inverse variant 2) at the 3 * 2^k
# energy lengths, pinned through the tune cache (momentum FFTs of at least 128
# points take the tuned passes), on sampled outputs against the oracle
@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
# (n_omega = PE/2 takes the kernel's half-output form)
@pytest.mark.parametrize("n_eps,n_omega,e_max,kT,pe", [(256, 128, 1.5, 0.025, 384), (512, 256, 3.0, 0.025, 768),
                                                       (193, 192, 1.5, 0.025, 384)],
                         ids=["PE384", "PE768", "PE384_half"])
def test_thermal_warp_inverse_lengths(lh, tmp_path, monkeypatch, n_eps, n_omega, e_max, kT, pe, quantity):
    import torch
    grid = wl.grid_params(2, 64, n_eps, e_max, n_omega=n_omega, q_extent=96, quantity=quantity)
    band = dict(wl.band_params(filling=1.1, gamma=0.06, ff_a=0.8), kT=kT)
    probe = lh.Plan([grid])
    s = probe.sizes[0]
    assert s.fft_e == pe and s.fft_p >= 128
    base = f"{torch.cuda.get_device_name(0)}|P={s.fft_p}|N={s.N}|PE={s.fft_e}|Q={s.q_extent}"
    probe.close()
    lx, ly, m = wl.output_samples(grid, 120, seed=pe + quantity)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_samples(A, grid, grid["q_extent"], kT, quantity, lx, ly, m)
    outs = {}
    for ve in (0, 2):
        path = tmp_path / f"tune_{ve}.json"
        path.write_text(json.dumps({base + "|fwd_y": 1, base + "|inv_y": 1, base + "|x_product": 0,
                                    base + "|inv_energy": ve}, indent=0))
        monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
        plan = lh.Plan([grid], autotune=True)
        out = plan.imchi([band])
        plan.status()
        assert plan.variants()["energy_inv"] == ve
        outs[ve] = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
        plan.close()
        err = np.abs(outs[ve][lx, ly, m] - ref).max() / np.abs(ref).max()
        print(f"PE {pe}, quantity {quantity}, inverse energy variant {ve}: {err:.2e} of max")
        assert err <= TOL32
    # every output: the two inverse passes differ only in rounding order
    scale = np.abs(outs[0]).max()
    assert np.abs(outs[2] - outs[0]).max() <= TOL32 * scale


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
def test_thermal_fp64(lh, quantity):
    grid, band, kT = CASES[0]
    got, _ = _gpu(lh, dict(grid, quantity=quantity), dict(band, kT=kT), precision=lh.FP64)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_full(A, grid, grid["q_extent"], grid["n_omega"], kT, quantity)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"FP64 quantity {quantity}: {err:.2e} of max")
    assert err <= TOL64


def test_thermal_caller_supplied_A(lh):
    # a random A with no symmetry: the odd part C(q, w) - C(-q, -w) is not
    # zero at w = 0, so every lag of the odd-part transform is exercised
    import torch
    grid = wl.grid_params(2, 8, 24, 1.0)
    A = np.random.default_rng(11).random((16, 16, 24))
    kT = 0.08
    for quantity in (1, 2):
        got, _ = _gpu(lh, dict(grid, quantity=quantity), dict(wl.band_params(), kT=kT),
                      A_in=torch.tensor(A.ravel(), dtype=torch.float32, device="cuda"))
        ref = oracle.thermal_full(A.astype(np.float32).astype(np.float64), grid, 16, 12, kT, quantity)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"caller A, quantity {quantity}: {err:.2e} of max")
        assert err <= TOL32


def test_zero_temperature_limit_and_fluctuation_dissipation(lh):
    grid, band, _ = CASES[0]
    de = 2 * grid["e_max"] / grid["n_eps"]
    t0, _ = _gpu(lh, grid, band)
    cold, _ = _gpu(lh, dict(grid, quantity=1), dict(band, kT=de / 4000))
    mx = np.abs(t0).max()
    print(f"kT -> 0 against the T = 0 output: {np.abs(cold - t0).max() / mx:.2e} of max")
    assert np.abs(cold - t0).max() <= TOL32 * mx
    kT = 0.05
    im, _ = _gpu(lh, dict(grid, quantity=1), dict(band, kT=kT))
    s, _ = _gpu(lh, dict(grid, quantity=2), dict(band, kT=kT))
    w = np.arange(grid["n_omega"]) * de
    lhs = s[..., 1:] * (1 - np.exp(-w[1:] / kT))
    err = np.abs(lhs + im[..., 1:] / math.pi).max() / (np.abs(im).max() / math.pi)
    print(f"Eq. 1 on the GPU outputs: {err:.2e} of max|Im chi_T|/pi")
    assert err <= 2 * TOL32


def test_thermal_product_variants(lh, tmp_path, monkeypatch):
    # the odd-part product sits in every product engine: each pinned variant
    # (default, 12-value, TMA-staged forms, high-occupancy tile) against the oracle
    grid = wl.grid_params(2, 64, 24, 1.5, quantity=1)        # P = 192
    band = dict(wl.band_params(filling=1.1, gamma=0.06, ff_a=0.7), kT=0.04)
    import torch
    probe = lh.Plan([grid])
    s = probe.sizes[0]
    base = f"{torch.cuda.get_device_name(0)}|P={s.fft_p}|N={s.N}|PE={s.fft_e}|Q={s.q_extent}"
    probe.close()
    lx, ly, m = wl.output_samples(grid, 200, seed=5)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_samples(A, grid, grid["q_extent"], 0.04, 1, lx, ly, m)
    for vx in (0, 1, 2, 3, 4):
        path = tmp_path / f"tune_{vx}.json"
        path.write_text(json.dumps({base + "|fwd_y": 1, base + "|inv_y": 1, base + "|x_product": vx,
                                    base + "|inv_energy": vx % 2}, indent=0))   # one entry per line
        monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
        plan = lh.Plan([grid], autotune=True)
        out = plan.imchi([band])
        plan.status()
        assert plan.variants()["px_product"] == vx
        got = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
        plan.close()
        err = np.abs(got[lx, ly, m] - ref).max() / np.abs(ref).max()
        print(f"product variant {vx}: {err:.2e} of max")
        assert err <= TOL32


def test_thermal_in_a_mixed_graph_batch(lh):
    """A T = 0 grid, an Im chi_T grid and an S grid in one concurrent,
    graph-captured plan give the bits each gives alone, and a changed kT is
    picked up (the graph is captured again)."""
    g0 = wl.grid_params(2, 16, 32, 1.5)
    grids = [g0, dict(g0, quantity=1), dict(g0, quantity=2)]
    band = wl.band_params(filling=1.1, gamma=0.08, ff_a=0.8)
    bands = [band, dict(band, kT=0.05), dict(band, kT=0.05)]
    plan = lh.Plan(grids, concurrent=True, graph=True)
    out = plan.imchi(bands).cpu().numpy()
    plan.status()
    off = 0
    for g, b in zip(grids, bands):
        alone, _ = _gpu(lh, g, b)
        n = alone.size
        assert np.array_equal(out[off:off + n], alone.ravel().astype(np.float32))
        off += n
    warmer = [band, dict(band, kT=0.2), dict(band, kT=0.2)]
    out2 = plan.imchi(warmer).cpu().numpy()
    plan.status()
    alone, _ = _gpu(lh, grids[2], warmer[2])
    assert np.array_equal(out2[-alone.size:], alone.ravel().astype(np.float32))
    plan.close()


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
def test_thermal_full_size_extended_workload(lh, quantity):
    """The 256 x 256 x 256 workload at kT = 25 meV (PE = 384 >= 256 + 128 - 1):
    seeded samples against the direct sum."""
    import torch
    w = wl.WORKLOADS["extended_256x256x256"]
    grid = dict(w["grid"], quantity=quantity)
    band = dict(w["band"], kT=0.025)
    plan = lh.Plan([grid])
    out = plan.imchi([band])
    plan.status()
    s = plan.sizes[0]
    assert s.fft_e == 384
    got = out.reshape(s.q_extent, s.q_extent, s.n_omega)
    lx, ly, m = wl.output_samples(grid, 300, seed=9)
    A = oracle.spectral(_solved(w["band"], grid), grid)
    ref = oracle.thermal_samples(A, grid, grid["q_extent"], 0.025, quantity, lx, ly, m)
    g = got.cpu().numpy().astype(np.float64)[lx, ly, m]
    err = np.abs(g - ref).max() / np.abs(ref).max()
    print(f"256^3 quantity {quantity}: {err:.2e} of the sample max")
    assert err <= TOL32
    assert torch.isfinite(got).all()
    plan.close()
    del out, got
    torch.cuda.empty_cache()


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
@pytest.mark.parametrize("cfg", [dict(zones=1, npz=32, n_eps=48, e_max=1.0, q_extent=32, n_omega=48),
                                 dict(zones=2, npz=16, n_eps=40, e_max=1.5, q_extent=64, n_omega=40)],
                         ids=["reduced", "extended_all_lags"])
def test_thermal_sum_rule(lh, cfg, quantity):
    # summed over every lag the finite-temperature outputs factorise into
    # Fermi-weighted energy correlations of the density of states D(e): the
    # library's FP64 reduction of its own output against its own D, and its D
    # side against numpy on the oracle's A
    grid = dict(wl.grid_params(cfg["zones"], cfg["npz"], cfg["n_eps"], cfg["e_max"], n_omega=cfg["n_omega"],
                               q_extent=cfg["q_extent"]), quantity=quantity)
    kT = 0.06
    band = dict(wl.band_params(filling=1.1, gamma=0.08, ff_a=1.0), kT=kT)
    plan = lh.Plan([grid])
    out = plan.imchi([band])
    sq, dc = plan.sum_rule(0, out, band=band)
    plan.status()
    sq, dc = sq.cpu().numpy(), dc.cpu().numpy()
    scale = np.abs(dc).max()
    assert scale > 0
    err = np.abs(sq - dc).max() / scale
    A = oracle.spectral(_solved(band, grid), grid)
    D = A.sum(axis=(0, 1))
    n, de = grid["n_eps"], 2 * grid["e_max"] / grid["n_eps"]
    e = -grid["e_max"] + (np.arange(n) + 0.5) * de
    f, fe = 1 / (np.exp(e / kT) + 1), 1 / (np.exp(-e / kT) + 1)
    c = de / (2 * math.pi) / grid["npz"] ** 2
    if quantity == 1:
        ref = np.array([-c * np.sum(D[: n - m] * D[m:] * (f[: n - m] - f[m:])) for m in range(grid["n_omega"])])
    else:
        ref = np.array([c / math.pi * np.sum(D[: n - m] * D[m:] * f[: n - m] * fe[m:]) for m in range(grid["n_omega"])])
    err_d = np.abs(dc - ref).max() / np.abs(ref).max()
    print(f"quantity {quantity}: sum over q against the DOS side {err:.2e}, DOS side against numpy {err_d:.2e}")
    assert err <= 1e-5 and err_d <= 1e-6
    plan.close()


def test_thermal_tensor_core_precision_and_noalloc(lh):
    """The finite-temperature weights and the odd-part product combine with
    the tensor-core inverse p_y pass and with the entry that allocates
    nothing."""
    import torch
    grid = wl.grid_params(2, 32, 16, 1.0, q_extent=128, quantity=1)   # every lag: P = 128, a tensor-core length
    band = dict(wl.band_params(filling=1.1, gamma=0.06, ff_a=0.8), kT=0.05)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_full(A, grid, grid["q_extent"], grid["n_omega"], 0.05, 1)
    mx = np.abs(ref).max()
    tc, _ = _gpu(lh, grid, band, precision=lh.SPLITBF16_TC)
    e_tc = np.abs(tc - ref).max() / mx
    out = torch.empty(grid["q_extent"] ** 2 * grid["n_omega"], dtype=torch.float32, device="cuda")
    lh.imchi_noalloc(grid, band, out=out)
    torch.cuda.synchronize()
    na = out.reshape(ref.shape).cpu().numpy().astype(np.float64)
    e_na = np.abs(na - ref).max() / mx
    print(f"Im chi_T: tensor-core inverse p_y {e_tc:.2e}, no-allocation entry {e_na:.2e} of max")
    assert e_tc <= TOL32 and e_na <= TOL32


@pytest.mark.parametrize("grid,kT", [(wl.grid_params(2, 8, 2, 1.0, n_omega=2), 0.1),
                                     (wl.grid_params(2, 8, 24, 1.0, n_omega=24), 0.05),
                                     (wl.grid_params(2, 8, 24, 1.0), 1.0),
                                     (wl.grid_params(2, 8, 24, 1.0), 1e-7),
                                     (wl.grid_params(1, 16, 9, 1.0, n_omega=9, q_extent=2), 0.2)],
                         ids=["n_eps2", "n_omega_eq_n_eps", "kT_1eV", "kT_1e-7", "one_lag_pair"])
@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
def test_thermal_edge_cases(lh, grid, kT, quantity):
    # the smallest energy grid, every transfer kept (PE >= 2 n_eps - 1), a
    # temperature as large as the window's half-width (the odd part C(q, w) -
    # C(-q, -w) then cancels to about w/4kT of either term, the most FP32
    # rounding it amplifies here) and one far below the half cell (weights
    # exactly 0 or 1), the smallest lag window
    band = dict(wl.band_params(filling=1.1, gamma=0.1, ff_a=0.5), kT=kT)
    got, fft_e = _gpu(lh, dict(grid, quantity=quantity), band)
    assert fft_e >= grid["n_eps"] + grid["n_omega"] - 1
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.thermal_full(A, grid, grid["q_extent"], grid["n_omega"], kT, quantity)
    mx = np.abs(ref).max()
    assert mx > 0
    err = np.abs(got - ref).max() / mx
    print(f"n_eps {grid['n_eps']}, n_omega {grid['n_omega']}, kT {kT}, quantity {quantity}: {err:.2e} of max")
    assert err <= TOL32
