"""lindhard_imchi_noalloc: the forward entry point for callers that cannot
allocate device memory (a framework owning the memory pool, hosts that forbid
allocation after start-up, code that must not synchronise the device).

Its results must match the plan-based lindhard_imchi within the FP32 parity
tolerance on consecutive calls (the shared scratch array keeps the previous
call's contents), it must leave the device's free memory unchanged, and it
must reject grids whose intermediates do not fit its fixed array.
"""
import numpy as np
import pytest

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


def _grid(zones, npz, n_eps, e_max):
    N = zones * npz
    return dict(zones=zones, npz=npz, n_eps=n_eps, e_max=e_max, n_omega=n_eps // 2, q_extent=N)


def _plan_result(lh, grid, band):
    import torch
    plan = lh.Plan([grid])
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = plan.imchi([band], mu_out=mu)
    plan.status()
    res = out.cpu().numpy().astype(np.float64), mu.item()
    plan.close()
    return res


def test_noalloc_matches_plan_on_consecutive_calls(lh):
    import torch
    cases = [(wl.WORKLOADS["reduced_32x32x48"]["grid"], wl.WORKLOADS["reduced_32x32x48"]["band"]),
             (_grid(2, 32, 128, 2.0), wl.band_params(filling=1.1, gamma=0.08, ff_a=1.0))]
    refs = [_plan_result(lh, g, b) for g, b in cases]
    outs = [torch.empty(r[0].size, dtype=torch.float32, device="cuda") for r in refs]
    mus = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in refs]
    # first call on the device looks up the scratch array's address
    lh.imchi_noalloc(cases[0][0], cases[0][1], out=outs[0], mu_out=mus[0])
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    # two calls in a row on each grid, alternating grids, results checked each time
    for rep in range(2):
        for i, (g, b) in enumerate(cases):
            outs[i].fill_(float("nan"))
            lh.imchi_noalloc(g, b, out=outs[i], mu_out=mus[i])
            torch.cuda.synchronize()
            got = outs[i].cpu().numpy().astype(np.float64)
            ref, ref_mu = refs[i]
            scale = np.abs(ref).max()
            err = np.abs(got - ref).max() / scale
            assert err <= TOL32, f"case {i} call {rep}: err {err:.3e}"
            assert abs(mus[i].item() - ref_mu) < 1e-12
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_caller_supplied_spectral_function(lh):
    import torch
    grid = _grid(2, 8, 24, 1.0)
    A = torch.from_numpy(wl.random_spectral(grid, seed=9)).cuda().reshape(-1)
    plan = lh.Plan([grid])
    ref = plan.imchi(None, A_in=A).cpu().numpy()
    plan.close()
    out = torch.empty(ref.size, dtype=torch.float32, device="cuda")
    for _ in range(2):
        lh.imchi_noalloc(grid, None, out=out, A_in=A)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max()


def test_noalloc_rejects_grids_beyond_its_scratch(lh):
    import torch
    grid = _grid(2, 64, 128, 2.0)          # needs about 54 MiB of intermediates
    band = wl.band_params()
    out = torch.empty(128 * 128 * 64, dtype=torch.float32, device="cuda")
    with pytest.raises(lh.LindhardError) as ei:
        lh.imchi_noalloc(grid, band, out=out)
    assert ei.value.status == lh.EINVAL
    assert "bytes of scratch" in str(ei.value)
