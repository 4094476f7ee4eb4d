"""Precision study on the large extended-zone workload (8 x 8 zones of 128
points, 512 energies on [-3, 3] eV, gamma = 0.03 eV): the FP32 SIMT form and
the split-BF16 tensor-core form (LINDHARD_SPLITBF16_TC), every one of the
268 M outputs against the FP64 FFT reference of the discrete Eq. 9
(oracle/fft_reference.py), itself checked here against the FP64 direct sums
at seeded samples of this grid.

The bar is 2e-5 of max|Im chi| over the whole output.  The error is also
reported per one-zone |q| shell and beyond 4 zones, against the maximum and
relative to the local value where |Im chi| > 1e-3 max: FFT roundoff scales
with the maximum, while Im chi decays with |q| (Sec. 4, Fig. 5), so the
relative error in the far zones grows although the error against the maximum
does not.  With LINDHARD_PRECISION_REPORT naming a file the rows are written
there as JSON.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.fft_reference import imchi_fft64, shell_report
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


def test_whole_grid_error_fp32_and_tensor_core(lh):
    import torch
    w = wl.WORKLOADS["large_1024x1024x512"]
    grid, band = w["grid"], w["band"]
    b = dict(band)
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    A = oracle.spectral(b, grid)
    ref = imchi_fft64(A, grid)
    # the FFT reference at this size against the direct sums: FP64 roundoff
    # of transforms over 1536 x 1536 x 512 points (measured 1.5e-11 of the
    # maximum), six orders of magnitude inside the bar it serves
    lx, ly, m = wl.output_samples(grid, 150, seed=13)
    direct = oracle.imchi_samples(A, grid, Q, lx, ly, m)
    del A
    ref_err = np.abs(ref[lx, ly, m] - direct).max() / np.abs(direct).max()
    print(f"FP64 FFT reference against the direct sums: {ref_err:.2e} of the sample maximum")
    assert ref_err <= 1e-10
    report = {}
    for name, prec in (("fp32", lh.FP32), ("split_bf16_tc", lh.SPLITBF16_TC)):
        plan = lh.Plan([grid], precision=prec, autotune=True)
        out = plan.imchi([band])
        plan.status()
        got = out.reshape(Q, Q, n_omega).cpu().numpy()
        variants = plan.variants()
        plan.close()
        del out
        torch.cuda.empty_cache()
        rows = shell_report(grid, got, ref)
        del got
        report[name] = {"variants": variants, "rows": rows}
        print(f"{name} {variants}")
        for label, n, a, r in rows:
            print(f"  {label}: {n} outputs, max err {a:.2e} of max"
                  + ("" if r is None else f", max relative err {r:.2e} where |Im chi| > 1e-3 max"))
        assert rows[0][2] <= TOL32, (name, rows[0])
    path = os.environ.get("LINDHARD_PRECISION_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(report, f, indent=1)
