"""The large extended-zone workload that bench.py times by default: 8 x 8
zones of 128 points (1024 x 1024 momenta), 512 energies on [-3, 3] eV,
gamma = 0.03 eV, momentum FFTs of 1536 points (N + Q/2), energy FFT of 512.

Every engine variant the autotuner can pick for this geometry runs here,
each pinned through a tune-cache file (the other passes on the variants the
tuner picked on GB300), against the FP64 oracle's direct sums on stratified
seeded samples (bar 2e-5 of the sample maximum, which is at most the true
maximum); and the autotuned plan itself, tuned afresh exactly as the bench
tunes it, on the same samples.  Whole-output properties (Im chi <= 0 and
Im chi(q, 0) = 0, both within the bar) are checked for every plan.
"""
import json

import numpy as np
import pytest

import oracle
from tail_report import format_rows, tail_report
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32 = 2e-5
NAME = "large_1024x1024x512"
# variants the autotuner tries at P = 1536 (a 3 * 2^k length >= 384), per pass
CANDIDATES = {"fwd_y": [0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11], "inv_y": [0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11],
              "x_product": [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10], "inv_energy": [0, 1, 2]}
# the passes not under test run the variants the tuner chose on GB300
TUNED = {"fwd_y": 3, "inv_y": 3, "x_product": 5, "inv_energy": 0}


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


@pytest.fixture(scope="module")
def ref():
    """Oracle samples of the workload, computed once for every plan below."""
    w = wl.WORKLOADS[NAME]
    grid, band = w["grid"], dict(w["band"])
    band["mu"] = oracle.solve_mu(band["kind"], band["t"], band["tp"], band["tpp"], band["gamma"], grid["npz"],
                                 band["filling"])
    lx, ly, m = wl.output_samples(grid, 600, seed=3)
    A = oracle.spectral(band, grid)
    vals = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    del A
    return dict(grid=grid, band=w["band"], mu=band["mu"], lx=lx, ly=ly, m=m, vals=vals)


def _keys(sizes):
    import torch
    base = (f"{torch.cuda.get_device_name(0)}|P={sizes.fft_p}|N={sizes.N}|PE={sizes.fft_e}"
            f"|Q={sizes.q_extent}")
    return {p: f"{base}|{p}" for p in ("fwd_y", "inv_y", "x_product", "inv_energy")}


def _check(lh, plan, ref, label):
    """Run the plan once; compare the sampled outputs with the oracle and
    check the whole-output properties; returns the sampled outputs."""
    import torch
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = plan.imchi([ref["band"]], mu_out=mu)
    plan.status()
    s = plan.sizes[0]
    out = out.reshape(s.q_extent, s.q_extent, s.n_omega)
    mx = float(out.abs().max())
    assert mx > 0
    assert float(out.max()) <= TOL32 * mx, label
    assert float(out[:, :, 0].abs().max()) <= TOL32 * mx, label
    idx = [torch.from_numpy(a.astype(np.int64)).cuda() for a in (ref["lx"], ref["ly"], ref["m"])]
    got = out[idx[0], idx[1], idx[2]].double().cpu().numpy()
    del out
    torch.cuda.empty_cache()
    assert abs(mu.item() - ref["mu"]) < 1e-10, label
    scale = np.abs(ref["vals"]).max()
    err = np.abs(got - ref["vals"]).max() / scale
    print(f"{label}: {got.size} samples, max err {err:.3e} of sample max")
    assert err <= TOL32, f"{label}: max err {err:.3e}"
    return got, err


@pytest.mark.parametrize("pass_,variant", [(p, v) for p, vs in CANDIDATES.items() for v in vs])
def test_each_variant_matches_oracle(lh, ref, tmp_path, monkeypatch, pass_, variant):
    probe = lh.Plan([ref["grid"]])
    keys = _keys(probe.sizes[0])
    assert probe.sizes[0].fft_p == 1536 and probe.sizes[0].fft_e == 512
    probe.close()
    pins = dict(TUNED, **{pass_: variant})
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({keys[p]: v for p, v in pins.items()}, indent=0))
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(path))
    plan = lh.Plan([ref["grid"]], autotune=True)
    names = {"fwd_y": "py_fwd", "inv_y": "py_inv", "x_product": "px_product", "inv_energy": "energy_inv"}
    assert plan.variants() == {names[p]: v for p, v in pins.items()}
    _check(lh, plan, ref, f"{pass_}={variant}")
    plan.close()


def test_autotuned_plan_matches_oracle(lh, ref, tmp_path, monkeypatch):
    """A fresh tune (the procedure the bench's plan runs) and its choices."""
    monkeypatch.setenv("LINDHARD_TUNE_CACHE", str(tmp_path / "fresh.json"))
    plan = lh.Plan([ref["grid"]], autotune=True)
    chosen = plan.variants()
    got, err = _check(lh, plan, ref, f"autotuned {chosen}")
    plan.close()
    scale = np.abs(ref["vals"]).max()
    print(format_rows(tail_report(ref["grid"], ref["lx"], ref["ly"], ref["m"], got, ref["vals"], scale)))
