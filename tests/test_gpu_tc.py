"""The tensor-core form (precision LINDHARD_SPLITBF16_TC): the inverse p_y
pass runs both stages of P = R1 R2 as matrix products on the tensor cores,
operands split into BF16 hi + lo, three products (hi.hi + lo.hi + hi.lo)
accumulated in FP32.  Every compiled length is checked against the FP64
oracle (every output on the small grids, seeded samples on the large ones)
and against the FP32 SIMT path over the whole output, at the FP32 bar of
2e-5 max|Im chi|; each case prints the errors it measured.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 2e-5

# (momentum FFT length, grid, oracle check: "full" or a sample count)
CASES = [
    (128, dict(zones=2, npz=32, n_eps=16, e_max=1.0, q_extent=128, n_omega=8), "full"),
    (192, dict(zones=2, npz=48, n_eps=16, e_max=1.0, q_extent=96, n_omega=8), "full"),
    (256, dict(zones=1, npz=256, n_eps=16, e_max=1.0, q_extent=256, n_omega=8), 200),
    (384, wl.WORKLOADS["extended_256x256x256"]["grid"], 300),
    (512, dict(zones=4, npz=64, n_eps=16, e_max=2.0, q_extent=512, n_omega=8), 150),
    (768, dict(zones=4, npz=128, n_eps=16, e_max=2.0, q_extent=512, n_omega=8), 100),
    (1024, dict(zones=8, npz=64, n_eps=16, e_max=2.0, q_extent=1024, n_omega=8), 80),
    (1536, dict(zones=8, npz=128, n_eps=16, e_max=3.0, q_extent=1024, n_omega=8), 60),
]


@pytest.fixture(scope="module")
def lh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard


def _run(lh, grid, band, precision):
    plan = lh.Plan([grid], precision=precision)
    out = plan.imchi([band])
    plan.status()
    s = plan.sizes[0]
    res = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    info = (s.fft_p, plan.variants()["py_inv"])
    plan.close()
    return res, info


@pytest.mark.parametrize("P,grid,check", CASES, ids=[f"P{c[0]}" for c in CASES])
def test_tensor_core_inverse_pass(lh, P, grid, check):
    import torch
    band = wl.band_params(filling=1.1, gamma=0.06, ff_a=0.8)
    ref32, (p32, v32) = _run(lh, grid, band, lh.FP32)
    tc, (ptc, vtc) = _run(lh, grid, band, lh.SPLITBF16_TC)
    assert p32 == ptc == P and vtc == 7 and v32 != 7
    mx = np.abs(ref32).max()
    assert mx > 0 and not math.isnan(mx)
    d32 = np.abs(tc - ref32).max() / mx
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    A = oracle.spectral(b, grid)
    Q = grid["q_extent"] or grid["zones"] * grid["npz"]
    if check == "full":
        ref = oracle.imchi_full(A, grid, Q, grid["n_omega"] or grid["n_eps"] // 2)
        e_tc = np.abs(tc - ref).max() / np.abs(ref).max()
        e_32 = np.abs(ref32 - ref).max() / np.abs(ref).max()
    else:
        lx, ly, m = wl.output_samples(grid, check, seed=3)
        ref = oracle.imchi_samples(A, grid, Q, lx, ly, m)
        scale = np.abs(ref).max()
        e_tc = np.abs(tc[lx, ly, m] - ref).max() / scale
        e_32 = np.abs(ref32[lx, ly, m] - ref).max() / scale
    print(f"P={P}: tensor-core vs oracle {e_tc:.2e}, FP32 SIMT vs oracle {e_32:.2e}, "
          f"tensor-core vs FP32 SIMT {d32:.2e} (of max|Im chi|)")
    assert e_tc <= TOL and d32 <= TOL
    torch.cuda.empty_cache()


def test_tensor_core_batched_graph(lh):
    """Two tensor-core instances of different lengths in one graph-captured
    concurrent plan give the same bits as each run alone."""
    import torch
    grids = [dict(CASES[0][1], precision=lh.SPLITBF16_TC), dict(CASES[1][1], precision=lh.SPLITBF16_TC)]
    bands = [wl.band_params(filling=1.05, gamma=0.1, ff_a=1.0), wl.band_params(filling=1.15, gamma=0.05)]
    plan = lh.Plan(grids, graph=True)
    out = plan.imchi(bands).cpu().numpy()
    again = plan.imchi(bands).cpu().numpy()
    plan.status()
    plan.close()
    assert np.array_equal(out, again)
    off = 0
    for g, b in zip(grids, bands):
        alone, _ = _run(lh, g, b, lh.SPLITBF16_TC)
        n = alone.size
        assert np.array_equal(out[off:off + n], alone.reshape(-1).astype(np.float32))
        off += n
    torch.cuda.synchronize()
