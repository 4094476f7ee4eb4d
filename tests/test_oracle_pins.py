"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form worked out by hand, an exact identity of Eq. 9, a different algorithm
(the convolution theorem that the paper's method relies on, Sec. 3), a
symmetry of the lattice, or a continuum limit (Appendix A, the free-fermion
form of Sec. 2).  Together they are chosen so that a dropped term, a wrong
sign or index, a transposed operand or a wrong prefactor fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1208_3210_gb300 import workloads as wl

T, TP, TPP = 0.42, -0.10, 0.065


def _grid(zones, npz, n_eps, e_max):
    return dict(zones=zones, npz=npz, n_eps=n_eps, e_max=e_max)


def _band(mu, gamma, ff_a=0.0, kind=0):
    return dict(kind=kind, t=T, tp=TP, tpp=TPP, mu=mu, gamma=gamma, ff_a=ff_a)


def _fft_correlation(A, grid, Q, n_omega):
    """Im chi through the convolution theorem (Sec. 3, the B(r, w) product):
    zero-padded FP64 numpy FFTs, a conjugate product and an inverse FFT.
    An algorithm independent of the oracle's direct double sum."""
    N, _, n_eps = A.shape
    j = np.arange(n_eps)
    occ = (2 * j + 1 < n_eps)
    a = A * occ[None, None, :]
    b = A * (~occ)[None, None, :]
    periodic = grid["zones"] == 1
    P = N if periodic else 2 * N
    PE = 2 * n_eps
    fa = np.fft.fftn(a, s=(P, P, PE), axes=(0, 1, 2))
    fb = np.fft.fftn(b, s=(P, P, PE), axes=(0, 1, 2))
    corr = np.fft.ifftn(np.conj(fa) * fb).real
    s = (np.arange(Q) - Q // 2) % P
    _, _, _, c = oracle.grid_sizes(grid["zones"], grid["npz"], n_eps, grid["e_max"])
    return -c * corr[np.ix_(s, s, np.arange(n_omega))]


# --- the band and the rigid-band chemical potential -------------------------

def test_band_high_symmetry_points():
    # Substituting Gamma = (0,0), X = (pi,0), M = (pi,pi) into the band by hand.
    assert oracle.band(0, T, TP, TPP, 0.0, 0.0) == pytest.approx(-4 * T - 4 * TP - 4 * TPP, abs=1e-14)
    assert oracle.band(0, T, TP, TPP, math.pi, 0.0) == pytest.approx(4 * TP - 4 * TPP, abs=1e-14)
    assert oracle.band(0, T, TP, TPP, math.pi, math.pi) == pytest.approx(4 * T - 4 * TP - 4 * TPP, abs=1e-14)
    assert oracle.band(1, 0, 0, 0, 0.3, -0.4) == pytest.approx(0.125, abs=1e-15)


def test_mu_half_filling_particle_hole():
    # Nearest-neighbour band: eps(k + (pi,pi)) = -eps(k), so one electron per
    # site puts mu at exactly 0 for any broadening (rigid band, Sec. 3).
    for npz in (16, 32):
        assert abs(oracle.solve_mu(0, T, 0.0, 0.0, 0.05, npz, 1.0)) < 1e-12


def test_filling_measure_free_electrons():
    # n = 2 Int d^2p/(2pi)^2 Theta(mu - p^2/2) = mu/pi in the gamma -> 0 limit:
    # pins the 2/npz^2 measure of d^2p/(2 pi)^2.
    n = oracle.filling(1, 0, 0, 0, 1e-3, 256, 1.0)
    assert n == pytest.approx(1.0 / math.pi, rel=2e-3)


def test_filling_monotone_and_solved():
    fills = [oracle.filling(0, T, TP, TPP, 0.05, 32, mu) for mu in np.linspace(-2, 2, 41)]
    assert all(b > a for a, b in zip(fills, fills[1:]))
    mu = oracle.solve_mu(0, T, TP, TPP, 0.05, 32, 1.15)
    assert oracle.filling(0, T, TP, TPP, 0.05, 32, mu) == pytest.approx(1.15, abs=1e-12)
    with pytest.raises(ValueError):
        oracle.solve_mu(0, T, TP, TPP, 0.05, 32, 2.5)


# --- the spectral function (Eqs. 4-5) -------------------------------------------

def test_lorentzian_weight_and_form_factor():
    # Midpoint sum of A over the window -> |M|^2 [atan((E-xi)/g) + atan((E+xi)/g)]/pi.
    grid = _grid(2, 8, 4000, 1.0)
    mu, gamma, ff = 0.05, 0.05, 1.0
    A = oracle.spectral(_band(mu, gamma, ff), grid)
    N, dp, de, _ = oracle.grid_sizes(2, 8, 4000, 1.0)
    for ix, iy in [(8, 8), (3, 11), (15, 0)]:
        px, py = (ix - N // 2) * dp, (iy - N // 2) * dp
        xi = oracle.band(0, T, TP, TPP, px, py) - mu
        m2 = math.exp(-(px * px + py * py) * ff * ff / 8)
        exact = m2 * (math.atan((1 - xi) / gamma) + math.atan((1 + xi) / gamma)) / math.pi
        assert A[ix, iy].sum() * de == pytest.approx(exact, rel=1e-5)


# --- Eq. 9 itself -----------------------------------------------------------------

@pytest.mark.parametrize("zones,npz,n_eps", [(1, 8, 12), (2, 4, 10), (2, 4, 9), (3, 4, 8)])
def test_direct_sum_equals_fft_correlation(zones, npz, n_eps):
    # P1: the direct double sum and the convolution-theorem route agree to
    # rounding, for the reduced (wrapping) and extended (truncating) zones and
    # for an odd energy count (e = 0 on the grid goes to the empty part).
    grid = _grid(zones, npz, n_eps, 1.0)
    mu = oracle.solve_mu(0, T, TP, TPP, 0.1, npz, 1.15)
    A = oracle.spectral(_band(mu, 0.1, 0.7), grid)
    N = zones * npz
    for Q, n_omega in [(N, n_eps // 2), (N if zones == 1 else 2 * N, n_eps)]:
        direct = oracle.imchi_full(A, grid, Q, n_omega)
        ref = _fft_correlation(A, grid, Q, n_omega)
        scale = np.abs(ref).max()
        assert scale > 0
        np.testing.assert_allclose(direct, ref, rtol=0, atol=1e-12 * scale)


def test_random_spectral_function_matches_shift_and_multiply():
    # A with no symmetry (the caller-supplied-A path): explicit array shifts.
    grid = _grid(2, 3, 7, 1.0)
    A = wl.random_spectral(grid, seed=3).astype(np.float64)
    N, n_eps = 6, 7
    _, _, _, c = oracle.grid_sizes(2, 3, 7, 1.0)
    Q, n_omega = 2 * N, n_eps
    direct = oracle.imchi_full(A, grid, Q, n_omega)
    j = np.arange(n_eps)
    a = A * (2 * j + 1 < n_eps)
    b = A * (2 * j + 1 >= n_eps)
    for l in [(0, 0), (1, 11), (6, 6), (9, 2), (11, 11)]:
        sx, sy = l[0] - Q // 2, l[1] - Q // 2
        for m in range(n_omega):
            acc = 0.0
            for ix in range(N):
                for iy in range(N):
                    if 0 <= ix + sx < N and 0 <= iy + sy < N:
                        acc += float(np.dot(a[ix, iy, : n_eps - m], b[ix + sx, iy + sy, m:]))
            assert direct[l[0], l[1], m] == pytest.approx(-c * acc, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("zones,npz,n_eps", [(1, 8, 16), (2, 6, 12), (2, 6, 11)])
def test_sum_rule(zones, npz, n_eps):
    # P2: summing Eq. 9 over all q factorises into the energy correlation of
    # the occupied and empty densities of states:
    #   sum_q Im chi(q, w_m) = -c sum_j D_a(e_j) D_b(e_{j+m}).
    grid = _grid(zones, npz, n_eps, 1.5)
    A = oracle.spectral(_band(0.05, 0.08, 1.0), grid)
    N, _, _, c = oracle.grid_sizes(zones, npz, n_eps, 1.5)
    Q = N if zones == 1 else 2 * N
    chi = oracle.imchi_full(A, grid, Q, n_eps)
    j = np.arange(n_eps)
    D = A.sum(axis=(0, 1))
    Da = D * (2 * j + 1 < n_eps)
    Db = D * (2 * j + 1 >= n_eps)
    for m in range(n_eps):
        rhs = -c * float(np.dot(Da[: n_eps - m], Db[m:]))
        assert chi[:, :, m].sum() == pytest.approx(rhs, rel=1e-12, abs=1e-15)


def test_square_lattice_symmetry():
    # P3: the band and |M|^2 are invariant under the square group, so is Im chi.
    # Reduced zone: exact.  Extended zone: exact under x <-> y; reflections hold
    # up to the unpaired edge row of the even grid (|M|^2 there ~ 1e-3 here).
    grid = _grid(1, 12, 16, 1.0)
    mu = oracle.solve_mu(0, T, TP, TPP, 0.05, 12, 1.15)
    A = oracle.spectral(_band(mu, 0.05), grid)
    chi = oracle.imchi_full(A, grid, 12, 8)
    scale = np.abs(chi).max()
    np.testing.assert_allclose(chi, chi.transpose(1, 0, 2), atol=1e-13 * scale)
    refl = np.roll(chi[::-1], 1, axis=0)  # l -> -l (mod 12) about l = Q/2
    np.testing.assert_allclose(chi, refl, atol=1e-13 * scale)
    grid = _grid(3, 6, 12, 1.5)
    A = oracle.spectral(_band(mu, 0.05, ff_a=1.0), grid)
    chi = oracle.imchi_full(A, grid, 18, 6)
    scale = np.abs(chi).max()
    np.testing.assert_allclose(chi, chi.transpose(1, 0, 2), atol=1e-13 * scale)
    inner = chi[1:, 1:]
    np.testing.assert_allclose(inner, inner[::-1, ::-1], atol=2e-3 * scale)


def test_zero_energy_transfer_and_sign():
    # P4: with the T = 0 split the occupied and empty supports are disjoint, so
    # Im chi(q, 0) = 0 exactly; every term is >= 0, so Im chi <= 0.
    grid = _grid(2, 6, 14, 1.0)
    A = oracle.spectral(_band(0.0, 0.1, 1.0), grid)
    chi = oracle.imchi_full(A, grid, 12, 14)
    assert np.all(chi[:, :, 0] == 0.0)
    assert np.all(chi <= 0.0)
    assert chi.min() < 0.0


def test_two_level_appendix_a():
    # P5: one occupied momentum p1 and one empty momentum p2 (a caller-supplied
    # A).  Im chi is nonzero only at q in {0, p2 - p1, p1 - p2}; at q = p2 - p1
    # it is -(1/(2 pi npz^2)) times the midpoint sum of L(e - xi1) L(e + w - xi2)
    # over [-w, 0], which converges to the integral of Eq. A3 as de^2.
    from scipy.integrate import quad

    zones, npz, e_max, gamma = 2, 4, 1.0, 0.05
    xi1, xi2 = -0.2, 0.25
    p1, p2 = (2, 5), (6, 3)

    def lor(e, xi):
        return gamma / (math.pi * ((e - xi) ** 2 + gamma ** 2))

    errs = []
    for n_eps in (200, 400, 800):
        grid = _grid(zones, npz, n_eps, e_max)
        N, dp, de, _ = oracle.grid_sizes(zones, npz, n_eps, e_max)
        e = -e_max + (np.arange(n_eps) + 0.5) * de
        A = np.zeros((N, N, n_eps))
        A[p1] = lor(e, xi1)
        A[p2] = lor(e, xi2)
        Q = 2 * N
        m = n_eps // 4                      # w = e_max / 2
        w = m * de
        lq = (p2[0] - p1[0] + Q // 2, p2[1] - p1[1] + Q // 2)
        val = oracle.imchi_samples(A, grid, Q, [lq[0]], [lq[1]], [m])[0]
        integral = quad(lambda x: lor(x, xi1) * lor(x + w, xi2), -w, 0.0, points=[xi1, xi2 - w], limit=200)[0]
        errs.append(abs(val / (-integral / (2 * math.pi * npz * npz)) - 1.0))
        full = oracle.imchi_full(A, grid, Q, m + 1)
        nz = {tuple(x) for x in np.argwhere(np.abs(full[:, :, m]) > 0)}
        assert nz == {(Q // 2, Q // 2), lq, (p1[0] - p2[0] + Q // 2, p1[1] - p2[1] + Q // 2)}
    assert errs[-1] < 2e-4
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_free_electron_lindhard_limit():
    # P6: for xi = p^2/2 - mu and gamma -> 0, Eq. 9 in 2D becomes
    #   Im chi = -2/((2 pi)^3 q) [sqrt((kF^2 - p0^2)_+) - sqrt((kF^2 - (p0+q)^2)_+)],
    # p0 = w/q - q/2, kF^2 = 2 mu (delta(w - q(p_par + q/2)) fixes p_par, and
    # the p_perp measure is the difference of two chords).  Pins the absolute
    # scale de/(2 pi) * 1/npz^2 and the occupation split; the error falls as
    # gamma shrinks.
    mu = 1.0

    def closed(q, w):
        p0 = w / q - q / 2
        return -(2 / q) * (math.sqrt(max(2 * mu - p0 * p0, 0)) - math.sqrt(max(2 * mu - (p0 + q) ** 2, 0))) \
            / (2 * math.pi) ** 3

    errs = []
    for gamma, n_eps in ((0.1, 160), (0.05, 320)):
        grid = _grid(2, 192, n_eps, 0.8)
        N, dp, de, _ = oracle.grid_sizes(2, 192, n_eps, 0.8)
        A = oracle.spectral(dict(kind=1, t=0, tp=0, tpp=0, mu=mu, gamma=gamma, ff_a=0.0), grid)
        lq, m = int(round(1.0 / dp)), int(round(0.5 / de))
        val = oracle.imchi_samples(A, grid, N, [N // 2 + lq], [N // 2], [m])[0]
        errs.append(abs(val / closed(lq * dp, m * de) - 1.0))
        del A
    assert errs[1] < 0.015
    assert errs[0] / errs[1] > 2.5


# --- the adjoint --------------------------------------------------------------------

def _small_case(zones=2, npz=4, n_eps=10, seed=1):
    grid = _grid(zones, npz, n_eps, 1.0)
    mu = oracle.solve_mu(0, T, TP, TPP, 0.1, npz, 1.15)
    band = _band(mu, 0.1, 0.8)
    A = oracle.spectral(band, grid)
    N = zones * npz
    Q, n_omega = N, n_eps // 2
    w = np.random.default_rng(seed).uniform(0, 1, (Q, Q, n_omega))
    return grid, band, A, Q, w


@pytest.mark.parametrize("n_eps", [10, 11])
@pytest.mark.parametrize("zones", [1, 2])
def test_grad_A_central_difference_is_exact(zones, n_eps):
    # L is a quadratic form in A, so a central difference in A is exact up to
    # rounding: (L(A + hE) - L(A - hE)) / 2h = dL/dA . E.  An odd energy count
    # puts a cell at e = 0 (empty by the split): every cell is probed there.
    grid, band, A, Q, w = _small_case(zones=zones, npz=6 if zones == 1 else 4, n_eps=n_eps)
    g = oracle.grad_A_full(A, grid, Q, w)
    rng = np.random.default_rng(7)
    h = 0.05
    cells = [(int(rng.integers(0, A.shape[0])), int(rng.integers(0, A.shape[1])), int(rng.integers(0, A.shape[2])))
             for _ in range(6)]
    if n_eps % 2:
        cells += [(int(rng.integers(0, A.shape[0])), int(rng.integers(0, A.shape[1])), j)
                  for j in (n_eps // 2 - 1, n_eps // 2, n_eps // 2 + 1)]
    for ix, iy, j in cells:
        Ap, Am = A.copy(), A.copy()
        Ap[ix, iy, j] += h
        Am[ix, iy, j] -= h
        fd = (oracle.loss(Ap, grid, Q, w) - oracle.loss(Am, grid, Q, w)) / (2 * h)
        assert g[ix, iy, j] == pytest.approx(fd, rel=1e-9, abs=1e-13)


def test_grad_A_bilinear_identity():
    # L = a^T K b with a, b the occupied and empty parts of A, so
    # <dL/da, a> = <dL/db, b> = L.
    grid, band, A, Q, w = _small_case()
    g = oracle.grad_A_full(A, grid, Q, w)
    L = oracle.loss(A, grid, Q, w)
    j = np.arange(A.shape[2])
    occ = (2 * j + 1 < A.shape[2])
    assert float(np.sum((g * A)[:, :, occ])) == pytest.approx(L, rel=1e-12)
    assert float(np.sum((g * A)[:, :, ~occ])) == pytest.approx(L, rel=1e-12)


def test_grad_params_central_difference():
    # dL/d(t, t', t'', mu, gamma) through Eqs. 4-5 against central differences
    # of the oracle loss with h = 1e-4 eV (truncation ~ h^2/gamma^2 ~ 1e-6).
    grid, band, A, Q, w = _small_case()
    g = oracle.grad_params(A, band, grid, Q, w)
    names = ["t", "tp", "tpp", "mu", "gamma"]
    h = 1e-4
    for r, name in enumerate(names):
        bp, bm = dict(band), dict(band)
        bp[name] += h
        bm[name] -= h
        fd = (oracle.loss(oracle.spectral(bp, grid), grid, Q, w)
              - oracle.loss(oracle.spectral(bm, grid), grid, Q, w)) / (2 * h)
        assert g[r] == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(fd) + 1e-12)


# --- Kramers-Kronig real part and RPA (Sec. 4) -----------------------------------

def _oscillator(w, w0, gamma, s=1.0):
    """A causal response with its poles in the lower half plane:
    chi(w) = -s / (w0^2 - w^2 - i gamma w), Im chi < 0 for w > 0 (the sign of
    Im chi of Eq. 9); its real part is fixed by analyticity."""
    d = (w0 ** 2 - w ** 2) ** 2 + (gamma * w) ** 2
    return -s * (w0 ** 2 - w ** 2) / d, -s * gamma * w / d


@pytest.mark.parametrize("gamma", [0.2, 0.5])
def test_kk_reproduces_the_real_part_of_a_causal_response(gamma):
    # Re chi from Im chi alone against the closed form.  Maclaurin's rule
    # converges faster than any power of the step for an analytic response, so
    # what remains is the window's tail, (2/pi) Int_W^inf Im chi(w')/w' dw' ~
    # (2/pi) gamma / (3 W^3): doubling the window W cuts it about eightfold.
    def err(h, W):
        w = np.arange(int(round(W / h))) * h
        re_ref, im = _oscillator(w, 1.0, gamma)
        re = oracle.kk_real(im[None, :])[0]
        keep = w <= 3.0
        return np.abs(re[keep] - re_ref[keep]).max() / np.abs(re_ref[keep]).max()
    e40, e80 = err(0.01, 40.0), err(0.01, 80.0)
    tail = 2.0 / math.pi * gamma / (3 * 40.0 ** 3)
    assert e40 < 2 * tail + 1e-7, (e40, tail)
    assert e80 < e40 / 4, (e40, e80)
    assert err(0.04, 40.0) < 1e-3


def test_kk_static_lindhard_response_is_negative():
    # Re chi(q, 0) = (4/pi) sum_{k odd} Im chi_k / k with Im chi <= 0 (Eq. 9):
    # the static Lindhard response is negative wherever Im chi is not zero
    grid = _grid(2, 12, 32, 1.5)
    b = _band(oracle.solve_mu(0, T, TP, TPP, 0.08, 12, 1.1), 0.08, 1.0)
    A = oracle.spectral(b, grid)
    im = oracle.imchi_full(A, grid, 24, 16)
    re = oracle.kk_real(im)
    assert (re[:, :, 0] <= 0).all()
    assert re[:, :, 0].min() < 0


def test_rpa_shifts_the_pole_to_the_plasmon_frequency():
    # chi_L = -s / (w0^2 - w^2 - i g w) gives chi_RPA = chi_L / (1 - V chi_L)
    # = -s / (w0^2 + V s - w^2 - i g w): the peak of -Im chi_RPA moves from w0
    # to sqrt(w0^2 + V s) (the plasmon of Sec. 4), with V = v0 / |q|^2.
    h, w0, g, s, v0, dp = 0.002, 1.0, 0.02, 1.0, 1.25, 1.0
    w = np.arange(int(round(20.0 / h))) * h
    _, im1 = _oscillator(w, w0, g, s)
    Q = 2
    im = np.broadcast_to(im1, (Q, Q, w.size)).copy()
    re = oracle.kk_real(im)
    chi = oracle.rpa(re, im, dp, v0)
    # lag (1, 0): q = (0, -dp), V = v0 / dp^2; lag (0, 0): q = (-dp, -dp), V = v0 / (2 dp^2)
    for (lx, ly), V in (((1, 0), v0 / dp ** 2), ((0, 0), v0 / (2 * dp ** 2))):
        peak = w[np.argmax(-chi[lx, ly].imag)]
        assert abs(peak - math.sqrt(w0 ** 2 + V * s)) < 5 * h, (lx, ly, peak)
    assert np.all(chi[1, 1] == 0)                     # q = 0: V infinite, chi_RPA -> 0
    same = oracle.rpa(re, im, dp, 0.0)                # no interaction: chi_RPA = chi_L
    assert np.array_equal(same, re + 1j * im)


# --- dmu/dtheta at fixed filling (the implicit gradient of the rigid band) ----------

@pytest.mark.parametrize("kind,fill,gamma", [(0, 1.15, 0.05), (0, 0.7, 0.2), (1, 0.3, 0.1)])
def test_dmu_dparams_matches_central_differences_of_the_mu_solve(kind, fill, gamma):
    # the analytic implicit-function derivative against central differences of
    # the oracle's own bisection for mu (a different computation of the same
    # quantity); h = 1e-4 eV leaves a truncation of order h^2
    npz = 24
    th = [T, TP, TPP, gamma] if kind == 0 else [0.0, 0.0, 0.0, gamma]
    mu = oracle.solve_mu(kind, *th[:3], gamma, npz, fill)
    got = oracle.dmu_dparams(kind, *th[:3], gamma, npz, mu)
    h = 1e-4
    for r in range(4):
        if kind == 1 and r < 3:
            assert got[r] == 0.0           # free electrons: no hoppings
            continue
        up, dn = list(th), list(th)
        up[r] += h
        dn[r] -= h
        fd = (oracle.solve_mu(kind, *up[:3], up[3], npz, fill) - oracle.solve_mu(kind, *dn[:3], dn[3], npz, fill)) / (2 * h)
        assert abs(got[r] - fd) <= 1e-6 * max(1.0, abs(fd)), (r, got[r], fd)


# --- envelope of -Im chi along the [100] cut (Sec. 4, Fig. 5) -----------------------

def _spiky_cut(Q, npz, k, floor=0.05):
    """-Im chi on the [100] cut equal to 1 / (1 + (q/k)^2) at the zone centres
    q = 2 pi n and to a small fraction of it elsewhere: the zone maxima lie
    exactly on the Lorentzian envelope."""
    dp = 2 * math.pi / npz
    q = (np.arange(Q) - Q // 2) * dp
    env = 1.0 / (1.0 + (q / k) ** 2)
    centre = ((np.arange(Q) - Q // 2) % npz) == 0
    im = np.zeros((Q, Q, 3))
    im[:, Q // 2, 2] = -np.where(centre, env, floor * env)
    return im


@pytest.mark.parametrize("k", [1.3, 4.0, 11.0])
def test_envelope_recovers_a_lorentzian_envelope(k):
    Q, npz = 512, 32
    k0, qs, ys = oracle.envelope_k0(_spiky_cut(Q, npz, k), npz, 2)
    assert abs(k0 - k) <= 1e-6 * k, (k0, k)
    assert np.allclose(qs, 2 * math.pi * np.arange(len(qs)))      # one point per zone, at its centre
    # the fit sees only the cut at l_y = Q/2 and transfer m, scaled freely
    im = _spiky_cut(Q, npz, k) * 7.5
    im[:, : Q // 2, :] = -3.0
    im[:, Q // 2, :2] = -9.0
    assert abs(oracle.envelope_k0(im, npz, 2)[0] - k) <= 1e-6 * k


def test_envelope_takes_each_zone_whole():
    # a zone is the lag window [G_n - npz/2, G_n + npz/2) around its
    # reciprocal lattice vector: with each zone's spike a quarter zone left of
    # G_n, the maxima sit there (a window shifted by half a zone would take
    # the next zone's spike instead)
    Q, npz, k = 256, 16, 5.0
    dp = 2 * math.pi / npz
    lag = np.arange(Q) - Q // 2
    q = lag * dp
    spike = (lag + npz // 4) % npz == 0
    im = np.zeros((Q, Q, 2))
    im[:, Q // 2, 1] = -np.where(spike, 1.0 / (1.0 + (q / k) ** 2), 0.01)
    k0, qs, ys = oracle.envelope_k0(im, npz, 1)
    assert np.allclose(qs, 2 * math.pi * (np.arange(len(qs)) - 0.25))
    env = 1.0 / (1.0 + (qs / k) ** 2)
    assert np.allclose(ys, env / env.max(), rtol=1e-14)          # the spikes, normalised by the largest
    assert 0 < k0 < Q * dp


def test_envelope_of_the_lindhard_response_decays():
    # on an extended grid the zone maxima of -Im chi fall off with q (the form
    # factor |M(p)|^2 and the band) and the fitted k0 is finite and positive
    grid = _grid(4, 8, 24, 1.5)
    b = _band(oracle.solve_mu(0, T, TP, TPP, 0.08, 8, 1.1), 0.08, 1.0)
    im = oracle.imchi_full(oracle.spectral(b, grid), grid, 32, 12)
    k0, qs, ys = oracle.envelope_k0(im, 8, 6)
    assert 0 < k0 < 32 * 2 * math.pi / 8 and ys.max() == 1.0
    assert ys[-1] < ys[0]
    with pytest.raises(ValueError):              # omega = 0: Im chi vanishes identically
        oracle.envelope_k0(im, 8, 0)


# --- finite temperature: Im chi_T and S(q, w) (Eq. 1, Appendix A Eq. A1) -----------

def _fermi(grid, kT):
    n_eps = grid["n_eps"]
    e = -grid["e_max"] + (np.arange(n_eps) + 0.5) * (2 * grid["e_max"] / n_eps)
    return 1.0 / (np.exp(e / kT) + 1.0), 1.0 / (np.exp(-e / kT) + 1.0)


def _thermal_fft(A, grid, Q, n_omega, kT):
    """Im chi_T and S through the convolution theorem: C(q, w) = sum A f (p, e)
    A (1 - f) (p + q, e + w) over every lag by zero-padded FP64 numpy FFTs;
    Im chi_T = -c [C(q, w) - C(-q, -w)], S = (c/pi) C(q, w)."""
    N, _, n_eps = A.shape
    f, fe = _fermi(grid, kT)
    periodic = grid["zones"] == 1
    P = N if periodic else 2 * N
    PE = 2 * n_eps
    fa = np.fft.fftn(A * f, s=(P, P, PE), axes=(0, 1, 2))
    fb = np.fft.fftn(A * fe, s=(P, P, PE), axes=(0, 1, 2))
    corr = np.fft.ifftn(np.conj(fa) * fb).real
    s = (np.arange(Q) - Q // 2) % P
    sn = (-(np.arange(Q) - Q // 2)) % P
    m = np.arange(n_omega)
    C = corr[np.ix_(s, s, m)]
    Cn = corr[np.ix_(sn, sn, (-m) % PE)]
    _, _, _, c = oracle.grid_sizes(grid["zones"], grid["npz"], n_eps, grid["e_max"])
    return -c * (C - Cn), c / math.pi * C


def _thermal_case(zones, npz, n_eps, e_max, gamma=0.1, ff_a=0.8):
    grid = _grid(zones, npz, n_eps, e_max)
    b = _band(oracle.solve_mu(0, T, TP, TPP, gamma, npz, 1.1), gamma, ff_a)
    return grid, oracle.spectral(b, grid)


def test_thermal_zero_temperature_limit():
    # kT far below the half cell de/2: every grid occupation is exactly 0 or 1
    # and the finite-temperature sums reduce term by term to Eq. 9
    grid, A = _thermal_case(2, 8, 24, 1.5)
    Q, nw = 16, 12
    kT = (2 * 1.5 / 24) / 4000
    ref = oracle.imchi_full(A, grid, Q, nw)
    im = oracle.thermal_full(A, grid, Q, nw, kT, oracle.IMCHI_T)
    s = oracle.thermal_full(A, grid, Q, nw, kT, oracle.SQW)
    assert np.array_equal(im, ref)
    assert np.allclose(s[..., 1:], -ref[..., 1:] / math.pi, rtol=1e-14, atol=0)
    assert np.all(s[..., 0] == 0.0)


@pytest.mark.parametrize("zones,npz,n_eps,kT", [(2, 8, 24, 0.03), (2, 8, 23, 0.3), (1, 16, 20, 0.1)])
def test_thermal_against_fft_correlation(zones, npz, n_eps, kT):
    grid, A = _thermal_case(zones, npz, n_eps, 1.5)
    Q = zones * npz if zones == 1 else 2 * zones * npz
    nw = n_eps // 2
    im_fft, s_fft = _thermal_fft(A, grid, Q, nw, kT)
    im = oracle.thermal_full(A, grid, Q, nw, kT, oracle.IMCHI_T)
    s = oracle.thermal_full(A, grid, Q, nw, kT, oracle.SQW)
    assert np.abs(im - im_fft).max() <= 1e-12 * np.abs(im_fft).max()
    assert np.abs(s - s_fft).max() <= 1e-12 * np.abs(s_fft).max()
    assert np.abs(im[..., 0]).max() <= 1e-13 * np.abs(im).max()     # Im chi_T(q, 0) = 0 (inversion-symmetric A)


def test_fluctuation_dissipation_and_detailed_balance():
    # Eq. 1: S (1 - exp(-w/kT)) = -Im chi_T / pi; and S(-q, -w) = exp(-w/kT) S(q, w),
    # on a random A with no symmetry
    grid = _grid(2, 6, 18, 1.2)
    A = np.random.default_rng(5).random((12, 12, 18))
    kT, Q = 0.15, 24
    de = 2 * 1.2 / 18
    rng = np.random.default_rng(6)
    lx, ly = rng.integers(1, Q, 60), rng.integers(1, Q, 60)
    m = rng.integers(1, 10, 60)
    im = oracle.thermal_samples(A, grid, Q, kT, oracle.IMCHI_T, lx, ly, m)
    s = oracle.thermal_samples(A, grid, Q, kT, oracle.SQW, lx, ly, m)
    boltz = np.exp(-m * de / kT)
    assert np.allclose(s * (1 - boltz), -im / math.pi, rtol=1e-12, atol=0)
    s_rev = oracle.thermal_samples(A, grid, Q, kT, oracle.SQW, Q - lx, Q - ly, -m)
    im_rev = oracle.thermal_samples(A, grid, Q, kT, oracle.IMCHI_T, Q - lx, Q - ly, -m)
    assert np.allclose(s_rev, boltz * s, rtol=1e-12, atol=0)
    assert np.allclose(im_rev, -im, rtol=1e-12, atol=0)


def test_thermal_high_temperature_limit():
    # kT >> the window: f(e) - f(e + w) -> w / 4kT and f (1 - f) -> 1/4, so
    # both reduce to the unweighted correlation of A with itself
    grid, A = _thermal_case(2, 6, 16, 1.0)
    Q, nw, kT = 12, 8, 1e6
    _, _, de, c = oracle.grid_sizes(2, 6, 16, 1.0)
    lx, ly, m = [a.ravel() for a in np.meshgrid(np.arange(Q), np.arange(Q), np.arange(1, nw), indexing="ij")]
    N = 12
    plain = np.zeros(lx.size)
    for k in range(lx.size):
        sx, sy = lx[k] - Q // 2, ly[k] - Q // 2
        x0, x1 = max(0, -sx), min(N, N - sx)
        y0, y1 = max(0, -sy), min(N, N - sy)
        a = A[x0:x1, y0:y1, : 16 - m[k]]
        b = A[x0 + sx:x1 + sx, y0 + sy:y1 + sy, m[k]:]
        plain[k] = np.sum(a * b)
    im = oracle.thermal_samples(A, grid, Q, kT, oracle.IMCHI_T, lx, ly, m)
    s = oracle.thermal_samples(A, grid, Q, kT, oracle.SQW, lx, ly, m)
    w = m * de
    assert np.allclose(im * 4 * kT / w, -c * plain, rtol=1e-9, atol=0)
    assert np.allclose(s * 4 * math.pi / c, plain, rtol=1e-5, atol=0)


def test_thermal_sum_rule():
    # summed over every lag the momentum correlation factorises into densities
    # of states D(e_j) = sum_p A(p, e_j):
    #   sum_q Im chi_T(q, w_m) = -c sum_j D_j D_{j+m} [f_j - f_{j+m}]
    grid, A = _thermal_case(2, 6, 20, 1.5)
    Q, nw, kT = 24, 10, 0.07
    _, _, _, c = oracle.grid_sizes(2, 6, 20, 1.5)
    im = oracle.thermal_full(A, grid, Q, nw, kT, oracle.IMCHI_T)
    D = A.sum(axis=(0, 1))
    f, _ = _fermi(grid, kT)
    for mm in range(nw):
        ref = -c * sum(D[j] * D[j + mm] * (f[j] - f[j + mm]) for j in range(20 - mm))
        assert abs(im[..., mm].sum() - ref) <= 1e-12 * max(abs(ref), np.abs(im).max())


# --- the finite-temperature adjoint (thermal_grad_A_samples) ---------------------

def _thermal_loss(A, grid, Q, w, kT, quantity):
    return float(np.sum(w * oracle.thermal_full(A, grid, Q, w.shape[2], kT, quantity)))


@pytest.mark.parametrize("zones", [1, 2])
@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
def test_thermal_grad_A_central_difference_is_exact(zones, quantity):
    # Eq. A1 and Eq. 1 are quadratic forms in A, so a central difference in A
    # is exact up to rounding: (L(A + hE) - L(A - hE)) / 2h = dL/dA . E
    grid, band, A, Q, w = _small_case(zones=zones, npz=6 if zones == 1 else 4)
    kT = 0.15
    g = oracle.thermal_grad_A_full(A, grid, Q, w, kT, quantity)
    rng = np.random.default_rng(11)
    h = 0.05
    for _ in range(6):
        ix, iy, j = (int(rng.integers(0, A.shape[0])), int(rng.integers(0, A.shape[1])),
                     int(rng.integers(0, A.shape[2])))
        Ap, Am = A.copy(), A.copy()
        Ap[ix, iy, j] += h
        Am[ix, iy, j] -= h
        fd = (_thermal_loss(Ap, grid, Q, w, kT, quantity) - _thermal_loss(Am, grid, Q, w, kT, quantity)) / (2 * h)
        assert g[ix, iy, j] == pytest.approx(fd, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("quantity", [1, 2], ids=["imchi_T", "S"])
def test_thermal_grad_A_homogeneity(quantity):
    # L is homogeneous of degree 2 in A: <dL/dA, A> = 2 L (Euler)
    grid, band, A, Q, w = _small_case()
    g = oracle.thermal_grad_A_full(A, grid, Q, w, 0.08, quantity)
    L = _thermal_loss(A, grid, Q, w, 0.08, quantity)
    assert float(np.sum(g * A)) == pytest.approx(2 * L, rel=1e-12)


def test_thermal_grad_A_zero_temperature_limit():
    # kT far below the half cell: occupations exactly 0 or 1, Im chi_T = Im chi
    # term by term, so the adjoints agree with the T = 0 one
    grid, band, A, Q, w = _small_case()
    kT = (2 * 1.0 / grid["n_eps"]) / 4000
    g = oracle.thermal_grad_A_full(A, grid, Q, w, kT, oracle.IMCHI_T)
    ref = oracle.grad_A_full(A, grid, Q, w)
    assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()
