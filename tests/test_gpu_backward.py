"""Parity of the adjoint (lindhard_imchi_backward) with the FP64 oracle.

dL/dA is compared with the oracle's direct adjoint sums (every point on small
grids, seeded samples at the gradient workload's full size) within
2e-5 max|dL/dA_oracle|; dL/d(t, t', t'', mu, gamma) with the oracle's chain
rule within 1e-4 of sum |dL/dA dA/dtheta| (the sum has cancellations); at full
size the bilinear identity <dL/da, a> = <dL/db, b> = L and central differences
of the forward loss (h = 1e-4 eV) hold.
"""
import math

import numpy as np
import pytest

import oracle
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


def _grid(zones, npz, n_eps, e_max=1.0, Q=0, n_omega=0):
    N = zones * npz
    return dict(zones=zones, npz=npz, n_eps=n_eps, e_max=e_max, n_omega=n_omega or n_eps // 2, q_extent=Q or N)


def _oracle_band(band, grid):
    b = dict(band)
    if math.isnan(b.get("mu", float("nan"))):
        b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["filling"])
    return b


def _gpu_backward(lh, grid, band, w, A=None):
    import torch
    plan = lh.Plan([grid], backward=True)
    s = plan.sizes[0]
    w_t = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda().reshape(-1)
    dA = torch.empty(s.a_elems, dtype=torch.float32, device="cuda")
    dp = None if A is not None else torch.zeros(5, dtype=torch.float64, device="cuda")
    A_t = None if A is None else torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda().reshape(-1)
    plan.backward(w_t, bands=None if A is not None else [band], A_in=A_t, dA=dA, dparams=dp)
    plan.status()
    out = dA.cpu().numpy().astype(np.float64).reshape(s.N, s.N, s.n_eps)
    dpn = None if dp is None else dp.cpu().numpy()
    plan.close()
    return out, dpn


@pytest.mark.parametrize("cfg", [dict(zones=1, npz=16, n_eps=24), dict(zones=2, npz=12, n_eps=20),
                                 dict(zones=3, npz=6, n_eps=17, Q=36, n_omega=17)])
def test_dA_matches_oracle_random_A(lh, cfg):
    grid = _grid(**cfg)
    A = wl.random_spectral(grid, seed=2)
    w = wl.loss_weights(grid, seed=4, dtype=np.float64)
    got, _ = _gpu_backward(lh, grid, None, w, A=A)
    ref = oracle.grad_A_full(A.astype(np.float64), grid, grid["q_extent"], w.astype(np.float32).astype(np.float64))
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= TOL32, err


@pytest.mark.parametrize("cfg", [dict(zones=1, npz=16, n_eps=32), dict(zones=2, npz=12, n_eps=24, e_max=1.5)])
def test_dA_and_dparams_match_oracle_generated_A(lh, cfg):
    grid = _grid(**cfg)
    band = wl.band_params(filling=1.12, gamma=0.08, ff_a=0.8)
    w = wl.loss_weights(grid, seed=5, dtype=np.float64).astype(np.float32).astype(np.float64)
    got, dp = _gpu_backward(lh, grid, band, w)
    b = _oracle_band(band, grid)
    A = oracle.spectral(b, grid)
    gref = oracle.grad_A_full(A, grid, grid["q_extent"], w)
    err = np.abs(got - gref).max() / np.abs(gref).max()
    assert err <= TOL32, err
    d = oracle.spectral_dtheta(b, grid)
    for r in range(5):
        terms = gref * d[r]
        ref = terms.sum()
        assert abs(dp[r] - ref) <= 1e-4 * np.abs(terms).sum(), (r, dp[r], ref)


def test_reduced_zone_workload_gradient(lh):
    w0 = wl.WORKLOADS["reduced_32x32x48"]
    grid, band = w0["grid"], w0["band"]
    w = wl.loss_weights(grid, seed=0, dtype=np.float64).astype(np.float32).astype(np.float64)
    got, dp = _gpu_backward(lh, grid, band, w)
    b = _oracle_band(band, grid)
    A = oracle.spectral(b, grid)
    gref = oracle.grad_A_full(A, grid, grid["q_extent"], w)
    assert np.abs(got - gref).max() <= TOL32 * np.abs(gref).max()
    d = oracle.spectral_dtheta(b, grid)
    for r in range(5):
        terms = gref * d[r]
        assert abs(dp[r] - terms.sum()) <= 1e-4 * np.abs(terms).sum()


def test_gradient_workload_full_size(lh):
    """The extended 256 x 256 x 256 geometry with seeded w ~ U[0, 1]."""
    import torch
    w0 = wl.WORKLOADS["extended_256x256x256"]
    grid, band = w0["grid"], w0["band"]
    w = wl.loss_weights(grid, seed=0)
    plan = lh.Plan([grid], backward=True)
    s = plan.sizes[0]
    w_t = torch.from_numpy(w).cuda().reshape(-1)
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    chi = plan.imchi([band], mu_out=mu)
    dA = torch.empty(s.a_elems, dtype=torch.float32, device="cuda")
    dp = torch.zeros(5, dtype=torch.float64, device="cuda")
    plan.backward(w_t, bands=[band], dA=dA, dparams=dp)
    plan.status()
    L = float((chi.double() * w_t.double()).sum())
    # sampled dL/dA against the oracle's adjoint sums
    b = _oracle_band(band, grid)
    assert abs(mu.item() - b["mu"]) < 1e-10
    A = oracle.spectral(b, grid)
    ix, iy, jj = wl.spectral_samples(grid, 300, seed=3)
    # include points near the Fermi surface where |dL/dA| is largest
    ref = oracle.grad_A_samples(A, grid, s.q_extent, w.astype(np.float64), ix, iy, jj)
    got = dA.reshape(s.N, s.N, s.n_eps).cpu().numpy()[ix, iy, jj].astype(np.float64)
    gmax = float(dA.abs().max())
    assert np.abs(got - ref).max() <= TOL32 * gmax
    # bilinear identity over the whole grid: <dL/da, a> = <dL/db, b> = L
    A_t = torch.from_numpy(A).cuda()
    dA3 = dA.reshape(s.N, s.N, s.n_eps).double()
    occ = torch.arange(s.n_eps, device="cuda") * 2 + 1 < s.n_eps
    La = float((dA3 * A_t)[:, :, occ].sum())
    Lb = float((dA3 * A_t)[:, :, ~occ].sum())
    assert La == pytest.approx(L, rel=2e-5) and Lb == pytest.approx(L, rel=2e-5)
    # chain rule through Eqs. 4-5 at full size, with the oracle's dA/dtheta
    d = oracle.spectral_dtheta(b, grid)
    for r in range(5):
        terms = dA3 * torch.from_numpy(d[r]).cuda()
        assert abs(dp[r].item() - float(terms.sum())) <= 1e-4 * float(terms.abs().sum())
    # central differences of the forward loss (mu held fixed), h = 1e-4 eV
    names = ["t", "tp", "tpp", "mu", "gamma"]
    h = 1e-4
    for r, name in enumerate(names):
        bp, bm = dict(b), dict(b)
        bp["filling"] = bm["filling"] = float("nan")
        bp[name] += h
        bm[name] -= h
        Lp = float((plan.imchi([bp]).double() * w_t.double()).sum())
        Lm = float((plan.imchi([bm]).double() * w_t.double()).sum())
        fd = (Lp - Lm) / (2 * h)
        assert dp[r].item() == pytest.approx(fd, rel=2e-2, abs=2e-3 * abs(L)), (name, dp[r].item(), fd)
    plan.close()


def test_autograd_function(lh):
    """torch.autograd through ImChiFunction: the parameter gradient matches the
    oracle's FP64 chain rule."""
    import torch
    grid = _grid(2, 12, 24, e_max=1.5)
    band = wl.band_params(filling=1.12, gamma=0.08, ff_a=0.8)
    b = _oracle_band(band, grid)
    plan = lh.Plan([grid], backward=True)
    params = torch.tensor([[b["t"], b["tp"], b["tpp"], b["mu"], b["gamma"]]], dtype=torch.float64,
                          requires_grad=True)
    w_np = wl.loss_weights(grid, seed=6)
    w = torch.from_numpy(w_np).cuda().reshape(-1)
    chi = lh.ImChiFunction.apply(params, plan, [band])
    L = (chi.double() * w.double()).sum()
    L.backward()
    g = params.grad.numpy()[0]
    # oracle gradient (FP64 chain rule through Eqs. 4-5)
    A = oracle.spectral(b, grid)
    gref = oracle.grad_A_full(A, grid, grid["q_extent"], w_np.astype(np.float64))
    d = oracle.spectral_dtheta(b, grid)
    for r in range(5):
        terms = gref * d[r]
        assert abs(g[r] - terms.sum()) <= 1e-4 * np.abs(terms).sum(), (r, g[r], terms.sum())
    plan.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_at_fixed_filling(lh, kind):
    """dL/dtheta at fixed filling = dL/dtheta at fixed mu + dL/dmu dmu/dtheta
    (lindhard_dmu_dparams), against central differences of the FP64 oracle
    loss with mu solved again from the filling at every step (h = 1e-4 eV)."""
    grid = _grid(2, 8, 24, 1.2)
    if kind == 0:
        band = wl.band_params(filling=1.1, gamma=0.08, ff_a=0.9)
    else:
        band = wl.band_params(filling=0.4, gamma=0.1, ff_a=0.0, kind=1, t=0.0, tp=0.0, tpp=0.0)
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    w = np.random.default_rng(9).uniform(0, 1, (Q, Q, n_omega)).astype(np.float32).astype(np.float64)
    _, dp = _gpu_backward(lh, grid, band, w)
    b = _oracle_band(band, grid)
    plan = lh.Plan([grid])
    dmu = plan.dmu_dparams(band, b["mu"])
    plan.close()
    ref = oracle.dmu_dparams(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], grid["npz"], b["mu"])
    assert np.allclose(dmu, ref, rtol=1e-10, atol=1e-14), (dmu, ref)
    total = np.array([dp[0], dp[1], dp[2], dp[4]]) + dp[3] * dmu      # d/d(t, t', t'', gamma)

    def loss(bb):
        bb = dict(bb)
        bb["mu"] = oracle.solve_mu(bb["kind"], bb["t"], bb["tp"], bb["tpp"], bb["gamma"], grid["npz"], bb["filling"])
        return oracle.loss(oracle.spectral(bb, grid), grid, Q, w)

    h = 1e-4
    for r, name in enumerate(["t", "tp", "tpp", "gamma"]):
        if kind == 1 and r < 3:
            assert dmu[r] == 0.0
            continue
        up, dn = dict(band), dict(band)
        up[name] += h
        dn[name] -= h
        fd = (loss(up) - loss(dn)) / (2 * h)
        scale = abs(fd) + abs(dp[r if r < 3 else 4]) + abs(dp[3] * dmu[r])
        print(f"kind {kind} d/d{name}: total {total[r]:.6e}, central difference {fd:.6e}")
        assert abs(total[r] - fd) <= 2e-4 * scale, (name, total[r], fd)


# --- finite temperature (Appendix A, Eq. A1; Eq. 1) ------------------------------

def _gpu_backward_thermal(lh, grid, band, w, A=None):
    import torch
    plan = lh.Plan([grid], backward=True)
    s = plan.sizes[0]
    w_t = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda().reshape(-1)
    dA = torch.empty(s.a_elems, dtype=torch.float32, device="cuda")
    dp = None if A is not None else torch.zeros(5, dtype=torch.float64, device="cuda")
    A_t = None if A is None else torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda().reshape(-1)
    plan.backward(w_t, bands=[band], A_in=A_t, dA=dA, dparams=dp)
    plan.status()
    out = dA.cpu().numpy().astype(np.float64).reshape(s.N, s.N, s.n_eps)
    dpn = None if dp is None else dp.cpu().numpy()
    fft_e = s.fft_e
    plan.close()
    return out, dpn, fft_e


# energy FFTs of 48 (3 * 2^4) and 32 points (n_eps + n_omega - 1 = 35 and 29)
THERMAL_CFGS = [(dict(zones=2, npz=8, n_eps=24, e_max=1.5), 48), (dict(zones=1, npz=16, n_eps=20), 32)]


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
@pytest.mark.parametrize("cfg,pe", THERMAL_CFGS, ids=["PE48", "PE32"])
def test_thermal_dA_matches_oracle_random_A(lh, cfg, pe, quantity):
    grid = dict(_grid(**cfg), quantity=quantity)
    kT = 0.05
    band = dict(wl.band_params(filling=1.12, gamma=0.08, ff_a=0.8), kT=kT)
    A = wl.random_spectral(grid, seed=3)
    w = wl.loss_weights(grid, seed=6, dtype=np.float64).astype(np.float32).astype(np.float64)
    got, _, fft_e = _gpu_backward_thermal(lh, grid, band, w, A=A)
    assert fft_e == pe
    ref = oracle.thermal_grad_A_full(A.astype(np.float32).astype(np.float64), grid, grid["q_extent"], w, kT, quantity)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"PE {pe}, quantity {quantity}, caller A: dL/dA {err:.2e} of max")
    assert err <= TOL32, err


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
@pytest.mark.parametrize("cfg,pe", THERMAL_CFGS, ids=["PE48", "PE32"])
def test_thermal_dA_and_dparams_match_oracle_generated_A(lh, cfg, pe, quantity):
    grid = dict(_grid(**cfg), quantity=quantity)
    kT = 0.04
    band = dict(wl.band_params(filling=1.1, gamma=0.07, ff_a=0.8), kT=kT)
    w = wl.loss_weights(grid, seed=8, dtype=np.float64).astype(np.float32).astype(np.float64)
    got, dp, fft_e = _gpu_backward_thermal(lh, grid, band, w)
    assert fft_e == pe
    b = _oracle_band(band, grid)
    A = oracle.spectral(b, grid)
    gref = oracle.thermal_grad_A_full(A, grid, grid["q_extent"], w, kT, quantity)
    err = np.abs(got - gref).max() / np.abs(gref).max()
    print(f"PE {pe}, quantity {quantity}: dL/dA {err:.2e} of max")
    assert err <= TOL32, err
    d = oracle.spectral_dtheta(b, grid)
    for r in range(5):
        terms = gref * d[r]
        ref = terms.sum()
        assert abs(dp[r] - ref) <= 1e-4 * np.abs(terms).sum(), (r, dp[r], ref)


@pytest.mark.parametrize("quantity", [0, 1, 2], ids=["imchi", "imchi_T", "S"])
def test_pruned_product_geometry_against_oracle_samples(lh, quantity):
    # N = Q = 2P/3 (P = 192): the adjoint's p_x products run on the pruned
    # engine (weights loaded as rows [0, Q) and phase-shifted, the inverse
    # keeping p_x < N); seeded cells against the oracle's adjoint sums
    import torch
    grid = dict(_grid(2, 64, 24, 1.5), quantity=quantity)
    band = wl.band_params(filling=1.1, gamma=0.07, ff_a=0.8)
    kT = 0.05 if quantity else 0.0
    if quantity:
        band = dict(band, kT=kT)
    w = wl.loss_weights(grid, seed=9, dtype=np.float64).astype(np.float32).astype(np.float64)
    plan = lh.Plan([grid], backward=True)
    s = plan.sizes[0]
    assert s.fft_p == 192 and s.N == 128 and s.q_extent == 128
    w_t = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda().reshape(-1)
    dA = torch.empty(s.a_elems, dtype=torch.float32, device="cuda")
    plan.backward(w_t, bands=[band], dA=dA)
    plan.status()
    got = dA.cpu().numpy().astype(np.float64).reshape(s.N, s.N, s.n_eps)
    plan.close()
    b = _oracle_band(band, grid)
    A = oracle.spectral(b, grid)
    rng = np.random.default_rng(12)
    ix, iy, jj = rng.integers(0, 128, 300), rng.integers(0, 128, 300), rng.integers(0, 24, 300)
    if quantity:
        ref = oracle.thermal_grad_A_samples(A, grid, 128, w, kT, quantity, ix, iy, jj)
    else:
        ref = oracle.grad_A_samples(A, grid, 128, w, ix, iy, jj)
    scale = np.abs(ref).max()
    err = np.abs(got[ix, iy, jj] - ref).max() / scale
    print(f"quantity {quantity}: dL/dA {err:.2e} of the samples' max")
    assert err <= TOL32, err
