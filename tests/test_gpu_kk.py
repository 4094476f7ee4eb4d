"""Kramers-Kronig real part and RPA susceptibility on the GPU (Sec. 4) against
the FP64 oracle (oracle.kk_real, oracle.rpa).

The pass is checked on its own (its input is the GPU's Im chi, so only the
Kramers-Kronig sum and the RPA arithmetic are measured) and end to end (Im chi
from the oracle's direct sum).  Bars: the FP32 SIMT form within 1e-6
max|Re chi| of the FP64 sum of the same input, the tensor-core form (far field
in BF16 hi/lo products, near band in FP32) within 2e-5 max|Re chi|, chi_RPA
within 1e-5 max|chi_RPA| of the FP64 formula applied to the GPU's own chi.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_TC, TOL_SIMT, TOL_RPA = 2e-5, 1e-6, 1e-5


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _imchi(lh, grid, band):
    plan = lh.Plan([grid])
    out = plan.imchi([band])
    plan.status()
    return plan, out


def _check_pass(lh, plan, out, grid, v0, variants=(0, 1)):
    s = plan.sizes[0]
    im = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    re_ref = oracle.kk_real(im)
    mx = np.abs(re_ref).max()
    assert mx > 0
    res = {}
    for v in variants:
        re, rp = plan.kk_rpa(out, v0=v0, variant=v)
        plan.status()
        re = re.cpu().numpy().astype(np.float64)
        rp = rp.cpu().numpy().astype(np.complex128)
        err = np.abs(re - re_ref).max() / mx
        rp_ref = oracle.rpa(re, im, 2 * math.pi / grid["npz"], v0)
        err_rpa = np.abs(rp - rp_ref).max() / np.abs(rp_ref).max()
        assert err <= (TOL_TC if v == 0 else TOL_SIMT), (v, err)
        assert err_rpa <= TOL_RPA, (v, err_rpa)
        res[v] = (re, rp, err)
    return im, res


@pytest.mark.parametrize("n_eps,n_omega", [(48, 24), (64, 48), (66, 33), (256, 128), (512, 256)])
def test_kk_rpa_against_oracle_on_the_gpu_output(lh, n_eps, n_omega):
    grid = wl.grid_params(2, 8, n_eps, 1.5, n_omega=n_omega)
    band = wl.band_params(filling=1.1, gamma=0.08, ff_a=0.8)
    plan, out = _imchi(lh, grid, band)
    _, res = _check_pass(lh, plan, out, grid, v0=0.05)
    print(f"n_omega={n_omega}: tensor-core {res[0][2]:.2e}, FP32 SIMT {res[1][2]:.2e} of max|Re chi|")
    plan.close()


def test_kk_rpa_end_to_end_against_the_direct_sum(lh):
    grid = wl.grid_params(2, 12, 64, 1.5, n_omega=32)
    band = wl.band_params(filling=1.15, gamma=0.06, ff_a=1.0)
    plan, out = _imchi(lh, grid, band)
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    im_ref = oracle.imchi_full(oracle.spectral(b, grid), grid, grid["q_extent"], grid["n_omega"])
    re_ref = oracle.kk_real(im_ref)
    v0 = 0.05
    rp_ref = oracle.rpa(re_ref, im_ref, 2 * math.pi / grid["npz"], v0)
    for v in (0, 1):
        re, rp = plan.kk_rpa(out, v0=v0, variant=v)
        plan.status()
        e_re = np.abs(re.cpu().numpy() - re_ref).max() / np.abs(re_ref).max()
        e_rp = np.abs(rp.cpu().numpy() - rp_ref).max() / np.abs(rp_ref).max()
        print(f"variant {v}: Re chi {e_re:.2e}, chi_RPA {e_rp:.2e}")
        assert e_re <= 3e-5 and e_rp <= 1e-4, (v, e_re, e_rp)
    plan.close()


def test_rpa_limits(lh):
    grid = wl.grid_params(2, 8, 32, 1.0)
    band = wl.band_params(filling=1.1, gamma=0.1)
    plan, out = _imchi(lh, grid, band)
    s = plan.sizes[0]
    im = out.reshape(s.q_extent, s.q_extent, s.n_omega)
    for v in (0, 1):
        re, rp = plan.kk_rpa(out, v0=0.0, variant=v)        # no interaction: chi_RPA = chi
        assert np.array_equal(rp.real.cpu().numpy(), re.cpu().numpy())
        assert np.array_equal(rp.imag.cpu().numpy(), im.cpu().numpy())
        _, rp = plan.kk_rpa(out, v0=0.3, variant=v)         # q = 0 (lag Q/2, Q/2): V infinite, chi_RPA -> 0
        assert float(rp[s.q_extent // 2, s.q_extent // 2].abs().max()) == 0.0
    plan.status()
    plan.close()


def test_kk_size_limits(lh):
    grid = wl.grid_params(1, 16, 600, 1.0, n_omega=300)
    band = wl.band_params(filling=1.1, gamma=0.1)
    plan, out = _imchi(lh, grid, band)
    with pytest.raises(lh.LindhardError, match="EUNSUPPORTED"):
        plan.kk_rpa(out, v0=0.1, variant=0)                 # tensor-core form: n_omega <= 256
    _check_pass(lh, plan, out, grid, v0=0.1, variants=(1,))
    plan.close()


def test_kk_rpa_full_size_extended_workload(lh):
    """The 256 x 256 x 256 workload (n_omega = 128): both forms agree, and
    seeded lines match the FP64 sum of the GPU's own Im chi."""
    import torch
    w = wl.WORKLOADS["extended_256x256x256"]
    plan, out = _imchi(lh, w["grid"], w["band"])
    s = plan.sizes[0]
    re0, rp0 = plan.kk_rpa(out, v0=0.05, variant=0)
    re1, rp1 = plan.kk_rpa(out, v0=0.05, variant=1)
    plan.status()
    mx = float(re1.abs().max())
    d = float((re0 - re1).abs().max()) / mx
    print(f"extended: tensor-core vs FP32 SIMT {d:.2e} of max|Re chi|")
    assert d <= TOL_TC
    rng = np.random.default_rng(3)
    lines = rng.integers(0, s.q_extent * s.q_extent, 300)
    im = out.reshape(-1, s.n_omega).cpu().numpy().astype(np.float64)[lines]
    ref = oracle.kk_real(im)
    got = re1.reshape(-1, s.n_omega).cpu().numpy().astype(np.float64)[lines]
    assert np.abs(got - ref).max() <= TOL_SIMT * max(np.abs(ref).max(), 1e-30) * 10
    plan.close()
    del out, re0, re1, rp0, rp1
    torch.cuda.empty_cache()
