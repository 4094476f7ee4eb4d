"""The energy-direct form (LINDHARD_PLAN_ENERGY_DIRECT): the paper's own
arrangement of Sec. 3, a 2D momentum FFT per energy plane and the energy sum
of Eq. 9 done directly per momentum frequency, against the FP64 oracle's
direct double sum (every output of small grids, seeded samples at full size)
and against the 3D FFT form.  Bar: 2e-5 of max|Im chi| (FP32); each case
prints the error it measured.
"""
import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 2e-5


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


def _run(lh, grid, band, direct=True, A_in=None):
    plan = lh.Plan([grid], energy_direct=direct)
    out = plan.imchi([band], A_in=A_in)
    plan.status()
    s = plan.sizes[0]
    res = out.reshape(s.q_extent, s.q_extent, s.n_omega).cpu().numpy().astype(np.float64)
    plan.close()
    return res


CASES = [
    # n_omega <= 32, 64, 128: one, two and four transfers per lane
    wl.grid_params(2, 16, 32, 1.5),
    wl.grid_params(2, 16, 33, 1.5, n_omega=20),                # odd n_eps: e = 0 is empty
    wl.grid_params(1, 32, 24, 1.0),                            # reduced zone, P = N
    wl.grid_params(2, 12, 30, 1.2, q_extent=48),               # every lag, P = 48
    wl.grid_params(2, 8, 64, 1.5, n_omega=64),                 # transfers beyond n_eps / 2
    wl.grid_params(2, 8, 160, 2.0, n_omega=100),
]
IDS = ["extended", "odd_eps", "reduced", "all_lags", "n_omega_eq_n_eps", "n_omega_100"]


@pytest.mark.parametrize("grid", CASES, ids=IDS)
def test_direct_against_oracle(lh, grid):
    band = wl.band_params(filling=1.1, gamma=0.08, ff_a=0.8)
    got = _run(lh, grid, band)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.imchi_full(A, grid, grid["q_extent"], grid["n_omega"])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"{grid['zones']}x{grid['npz']} n_eps {grid['n_eps']} n_omega {grid['n_omega']}: {err:.2e} of max")
    assert err <= TOL


@pytest.mark.parametrize("n_eps,n_omega", [(512, 256), (1024, 512)], ids=["R8", "R16"])
def test_direct_long_energy_axis(lh, n_eps, n_omega):
    # eight and sixteen transfers per lane; seeded samples against the direct sum
    grid = wl.grid_params(2, 8, n_eps, 2.0, n_omega=n_omega)
    band = wl.band_params(filling=1.1, gamma=0.05, ff_a=0.8)
    got = _run(lh, grid, band)
    lx, ly, m = wl.output_samples(grid, 400, seed=4)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    err = np.abs(got[lx, ly, m] - ref).max() / np.abs(ref).max()
    print(f"n_eps {n_eps}, n_omega {n_omega}: {err:.2e} of the sample max")
    assert err <= TOL


def test_direct_caller_supplied_A(lh):
    import torch
    grid = wl.grid_params(2, 8, 24, 1.0)
    A = np.random.default_rng(12).random((16, 16, 24))
    got = _run(lh, grid, wl.band_params(), A_in=torch.tensor(A.ravel(), dtype=torch.float32, device="cuda"))
    ref = oracle.imchi_full(A.astype(np.float32).astype(np.float64), grid, 16, 12)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"caller A: {err:.2e} of max")
    assert err <= TOL


def test_direct_full_size_against_the_3d_form(lh):
    """The 256 x 256 x 256 workload: the whole output against the 3D FFT form,
    and seeded samples against the oracle."""
    import torch
    w = wl.WORKLOADS["extended_256x256x256"]
    grid, band = w["grid"], w["band"]
    d = _run(lh, grid, band, direct=True)
    f = _run(lh, grid, band, direct=False)
    mx = np.abs(f).max()
    diff = np.abs(d - f).max() / mx
    lx, ly, m = wl.output_samples(grid, 300, seed=8)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.imchi_samples(A, grid, grid["q_extent"], lx, ly, m)
    e_d = np.abs(d[lx, ly, m] - ref).max() / np.abs(ref).max()
    e_f = np.abs(f[lx, ly, m] - ref).max() / np.abs(ref).max()
    print(f"256^3: direct vs 3D {diff:.2e} of max; against the oracle: direct {e_d:.2e}, 3D {e_f:.2e}")
    assert diff <= TOL and e_d <= TOL
    assert np.all(d <= TOL * mx) and np.abs(d[..., 0]).max() <= TOL * mx   # Im chi <= 0, Im chi(q, 0) = 0
    torch.cuda.empty_cache()


def test_direct_graph_batch_bit_identical(lh):
    grids = [CASES[0], CASES[1], CASES[3]]
    bands = [wl.band_params(filling=1.05, gamma=0.1, ff_a=1.0), wl.band_params(filling=1.15, gamma=0.05),
             wl.band_params(filling=1.1, gamma=0.07, ff_a=0.5)]
    plan = lh.Plan(grids, graph=True, energy_direct=True)
    out = plan.imchi(bands).cpu().numpy()
    again = plan.imchi(bands).cpu().numpy()
    plan.status()
    plan.close()
    assert np.array_equal(out, again)
    off = 0
    for g, b in zip(grids, bands):
        alone = _run(lh, g, b)
        n = alone.size
        assert np.array_equal(out[off:off + n], alone.ravel().astype(np.float32))
        off += n


@pytest.mark.parametrize("grid", [wl.grid_params(2, 8, 2, 1.0, n_omega=2),
                                  wl.grid_params(2, 8, 7, 1.0, n_omega=7, q_extent=2),
                                  wl.grid_params(1, 16, 3, 1.0, n_omega=3),
                                  wl.grid_params(3, 8, 17, 1.3, n_omega=9, q_extent=48)],
                         ids=["n_eps2", "one_lag_pair", "reduced_n_eps3", "three_zones_all_lags"])
def test_direct_edge_cases(lh, grid):
    # the smallest energy grids (one occupied and one empty plane; odd counts),
    # the smallest lag window and an odd zone count, every output against the oracle
    band = wl.band_params(filling=1.1, gamma=0.1, ff_a=0.5)
    got = _run(lh, grid, band)
    A = oracle.spectral(_solved(band, grid), grid)
    ref = oracle.imchi_full(A, grid, grid["q_extent"], grid["n_omega"])
    mx = np.abs(ref).max()
    assert mx > 0
    err = np.abs(got - ref).max() / mx
    print(f"n_eps {grid['n_eps']}, n_omega {grid['n_omega']}, Q {grid['q_extent']}: {err:.2e} of max")
    assert err <= TOL
