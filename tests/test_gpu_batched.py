"""Batched plans: instances on concurrent streams, and the whole batch
recorded once into a CUDA graph and replayed.  The kernels are the same as in
a sequential plan, so every output must be bit-identical to it, across graph
replays and re-recordings after the band values change."""
import numpy as np
import pytest

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


def _grids():
    return [wl.grid_params(2, 8, 24, 1.0), wl.grid_params(1, 16, 16, 1.0), wl.grid_params(4, 6, 20, 2.0),
            wl.grid_params(2, 32, 64, 2.0), wl.grid_params(4, 16, 32, 2.0, q_extent=128, n_omega=32)]


def _bands(shift=0.0):
    return [wl.band_params(filling=1.05 + shift, gamma=0.1, ff_a=1.0), wl.band_params(filling=1.15, gamma=0.05),
            wl.band_params(filling=1.17, gamma=0.15 + shift, ff_a=1.0), wl.band_params(filling=1.1, gamma=0.08),
            wl.band_params(filling=1.12, gamma=0.06, ff_a=0.5)]


def _run(plan, bands, out, mu):
    import torch
    plan.imchi(bands, out=out, mu_out=mu)
    plan.status()
    torch.cuda.synchronize()
    return out.cpu().numpy().copy(), mu.cpu().numpy().copy()


def test_concurrent_and_graph_match_sequential(lh):
    import torch
    grids = _grids()
    seq = lh.Plan(grids)
    con = lh.Plan(grids, concurrent=True)
    gra = lh.Plan(grids, graph=True)
    n = seq.out_elems()
    outs = {k: torch.empty(n, dtype=torch.float32, device="cuda") for k in ("s", "c", "g")}
    mus = {k: torch.empty(5, dtype=torch.float64, device="cuda") for k in ("s", "c", "g")}
    for shift in (0.0, 0.0, 0.01, 0.01, 0.0):      # replay, re-record, replay, re-record
        b = _bands(shift)
        ref, ref_mu = _run(seq, b, outs["s"], mus["s"])
        got_c, mu_c = _run(con, b, outs["c"], mus["c"])
        outs["g"].fill_(float("nan"))
        got_g, mu_g = _run(gra, b, outs["g"], mus["g"])
        assert np.array_equal(ref, got_c) and np.array_equal(ref, got_g)
        assert np.array_equal(ref_mu, mu_c) and np.array_equal(ref_mu, mu_g)
    for pl in (seq, con, gra):
        pl.close()


def test_concurrent_backward_matches_sequential(lh):
    import torch
    grids = _grids()[:3]
    bands = _bands()[:3]
    seq = lh.Plan(grids, backward=True)
    con = lh.Plan(grids, backward=True, concurrent=True)
    w = torch.rand(seq.out_elems(), dtype=torch.float32, device="cuda")
    res = []
    for pl in (seq, con):
        dA = torch.empty(pl.a_elems(), dtype=torch.float32, device="cuda")
        dp = torch.empty(15, dtype=torch.float64, device="cuda")
        pl.backward(w, bands=bands, dA=dA, dparams=dp)
        pl.status()
        res.append((dA.cpu().numpy(), dp.cpu().numpy()))
        pl.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_batched_workload_builds(lh):
    # the 64-instance benchmark workload: plan creation and one graph call
    import torch
    grids, bands = wl.batched_workload(64)
    plan = lh.Plan(grids, graph=True)
    out = torch.empty(plan.out_elems(), dtype=torch.float32, device="cuda")
    mu = torch.empty(64, dtype=torch.float64, device="cuda")
    plan.imchi(bands, out=out, mu_out=mu)
    plan.status()
    assert torch.isfinite(out).all() and float(out.max()) <= 2e-5 * float(out.abs().max())
    plan.close()
