"""The seeded input module (CPU): every workload is reproducible from its seed,
the sampled output indices stay inside the output and reach every transfer
stratum and the far |q| shells, and the batched workload has the stated mix."""
import numpy as np

from paper_1208_3210_gb300 import workloads as wl


def test_output_samples_are_in_range_seeded_and_stratified():
    for name in ("reduced_32x32x48", "extended_256x256x256", "large_1024x1024x512"):
        g = wl.WORKLOADS[name]["grid"]
        lx, ly, m = wl.output_samples(g, 400, seed=3)
        again = wl.output_samples(g, 400, seed=3)
        assert all(np.array_equal(a, b) for a, b in zip((lx, ly, m), again))
        assert lx.dtype == np.int32 and ly.dtype == np.int32 and m.dtype == np.int32
        Q, n_omega = g["q_extent"], g["n_omega"]
        assert lx.min() >= 0 and lx.max() < Q and ly.min() >= 0 and ly.max() < Q
        assert m.min() >= 0 and m.max() < n_omega
        assert m.min() == 0 and m.max() >= n_omega // 2          # low and high transfers
        # the far shells are sampled, not only the peak around q = 0
        r = np.hypot(lx - Q // 2, ly - Q // 2)
        assert r.max() > 0.6 * np.hypot(Q / 2, Q / 2)


def test_batched_workload_mix():
    grids, bands = wl.batched_workload(64, seed=0)
    again = wl.batched_workload(64, seed=0)
    assert grids == again[0] and bands == again[1]
    assert len(grids) == 64
    Ns = {g["zones"] * g["npz"] for g in grids}
    assert Ns <= {128, 256, 512} and len(Ns) > 1
    assert {g["zones"] for g in grids} <= {2, 4}
    assert {g["n_eps"] for g in grids} <= {128, 256}
    assert all(0.02 <= b["gamma"] <= 0.2 for b in bands)
    assert {b["filling"] for b in bands} == set(wl.BATCH_FILLINGS)


def test_grid_params_defaults_and_extras():
    g = wl.grid_params(4, 64, 256, 2.0)
    assert g["n_omega"] == 128 and g["q_extent"] == 256
    g = wl.grid_params(2, 8, 24, 1.0, n_omega=5, q_extent=16, quantity=2)
    assert g["n_omega"] == 5 and g["q_extent"] == 16 and g["quantity"] == 2
    b = wl.band_params(filling=1.1, gamma=0.07, kT=0.03)
    assert b["kT"] == 0.03 and np.isnan(b["mu"])
