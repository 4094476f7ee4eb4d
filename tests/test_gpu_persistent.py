"""The persistent batch launch (LINDHARD_PLAN_PERSISTENT): every instance's
five transform passes in one launch whose CTAs claim (instance, pass, tile)
items from a device queue, each item waiting (bounded) for its instance's
previous pass.

Checked: a mixed batch (momentum FFTs of 192, 384 and 768 points, energy
FFTs of 128 and 256 with and without energy padding, transfers at half the
energies and not) against the FP64 oracle per instance and against the plain
plan; graph replay; every one of the 64 instances of the batched workload
against the oracle's direct sums at seeded samples (the form the bench
times); and a wait made to run out on purpose (a completion counter asked for
one more tile than exists, a 20 us limit): the call ends, lindhard_plan_status
reports LINDHARD_ETIMEOUT without a fault, and the next call is correct.
"""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32 = 2e-5

MIXED = [wl.grid_params(2, 64, 128, 2.0), wl.grid_params(4, 32, 256, 2.0),
         wl.grid_params(2, 128, 128, 1.5, n_omega=50), wl.grid_params(4, 64, 200, 2.0, n_omega=100),
         wl.grid_params(4, 128, 256, 2.0)]
MIXED_BANDS = [wl.band_params(filling=f, gamma=g_, ff_a=1.0)
               for f, g_ in zip((1.04, 1.10, 1.16, 1.12, 1.17), (0.12, 0.05, 0.18, 0.03, 0.08))]


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _split(plan, out):
    res, off = [], 0
    for s in plan.sizes:
        res.append(out[off:off + s.out_elems].reshape(s.q_extent, s.q_extent, s.n_omega))
        off += s.out_elems
    return res


def _oracle_samples(grid, band, count, seed):
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    lx, ly, m = wl.output_samples(grid, count, seed=seed, near_origin=4)
    A = oracle.spectral(b, grid)
    ref = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    return (lx, ly, m), ref, b["mu"]


def test_mixed_batch_matches_oracle_and_plain_plan(lh):
    import torch
    plan = lh.Plan(MIXED, persistent=True)
    mu = torch.zeros(len(MIXED), dtype=torch.float64, device="cuda")
    out = plan.imchi(MIXED_BANDS, mu_out=mu)
    plan.status()
    got = [x.cpu().numpy().astype(np.float64) for x in _split(plan, out)]
    plain = lh.Plan(MIXED)
    ref_plain = [x.cpu().numpy().astype(np.float64) for x in _split(plain, plain.imchi(MIXED_BANDS))]
    plain.status()
    plain.close()
    plan.close()
    for i, (g, b) in enumerate(zip(MIXED, MIXED_BANDS)):
        (lx, ly, m), ref, mu_ref = _oracle_samples(g, b, 300, seed=i)
        assert abs(mu[i].item() - mu_ref) < 1e-10
        err = np.abs(got[i][lx, ly, m] - ref).max() / np.abs(ref).max()
        assert err <= TOL32, (i, err)
        mx = np.abs(ref_plain[i]).max()
        assert np.abs(got[i] - ref_plain[i]).max() <= TOL32 * mx, i
        assert got[i].max() <= TOL32 * mx and np.abs(got[i][:, :, 0]).max() <= TOL32 * mx


def test_graph_replay_bit_identical(lh):
    import torch
    eager = lh.Plan(MIXED, persistent=True)
    a = eager.imchi(MIXED_BANDS).clone()
    eager.status()
    eager.close()
    plan = lh.Plan(MIXED, persistent=True, graph=True)
    out = torch.empty_like(a)
    for _ in range(3):
        plan.imchi(MIXED_BANDS, out=out)
    plan.status()
    assert torch.equal(out, a)
    # new band values re-record the graph
    b2 = [dict(b, gamma=b["gamma"] * 1.1) for b in MIXED_BANDS]
    plan.imchi(b2, out=out)
    plan.status()
    assert not torch.equal(out, a)
    plan.close()


def test_batched_64_every_instance_against_oracle(lh):
    """The 64-instance batched workload as the bench runs it (persistent launch
    replayed as a graph): every instance against the oracle at seeded samples,
    and Im chi <= 0 and Im chi(q, 0) = 0 over every instance's output."""
    import torch
    grids, bands = wl.batched_workload(64)
    plan = lh.Plan(grids, persistent=True, graph=True, autotune=True)
    mu = torch.zeros(len(grids), dtype=torch.float64, device="cuda")
    out = torch.empty(sum(s.out_elems for s in plan.sizes), dtype=torch.float32, device="cuda")
    for _ in range(2):
        plan.imchi(bands, out=out, mu_out=mu)
    plan.status()
    parts = [x.cpu().numpy().astype(np.float64) for x in _split(plan, out)]
    plan.close()
    worst = 0.0
    for i, (g, b, got) in enumerate(zip(grids, bands, parts)):
        (lx, ly, m), ref, mu_ref = _oracle_samples(g, b, 24, seed=100 + i)
        assert abs(mu[i].item() - mu_ref) < 1e-10, i
        err = np.abs(got[lx, ly, m] - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err <= TOL32, (i, g, err)
        mx = np.abs(got).max()
        assert got.max() <= TOL32 * mx and np.abs(got[:, :, 0]).max() <= TOL32 * mx, i
    print(f"batched_64: worst instance error {worst:.2e} of its sample maximum")


def test_wait_runs_out_and_reports_timeout(lh):
    import torch
    grids, bands = MIXED[:2], MIXED_BANDS[:2]
    plan = lh.Plan(grids, persistent=True)
    good = plan.imchi(bands).clone()
    plan.status()
    plan.set_wait_limit(20_000, stall_instance=1)      # 20 us; instance 1's first wait cannot be met
    t0 = time.perf_counter()
    plan.imchi(bands)
    with pytest.raises(lh.LindhardError) as info:
        plan.status()
    assert info.value.status == lh.ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    plan.set_wait_limit(0, -1)                         # default limit, no stall
    again = plan.imchi(bands)
    plan.status()
    assert torch.equal(again, good)
    plan.close()
