"""FP64 CPU oracle for the FFT Lindhard susceptibility.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_1208_3210_gb300`` never imports it, and the two share no code.

The arithmetic lives in ``lindhard_oracle.c`` (plain loops in FP64, OpenMP over
independent outputs); this module compiles it with gcc on first use and wraps
it with numpy arrays.  Every function states the passage of Wang et al. it
follows.  Conventions (the readings of the paper) are the ones documented in
the C file: p_i = (i - N/2) 2pi/npz, e_j = -E + (j + 1/2) 2E/n_eps,
w_m = m de, q_l = (l - Q/2) 2pi/npz, measure 1/npz^2 per grid point.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lindhard_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblindhard_oracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp, IEEE arithmetic kept)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.lo_band.restype = ctypes.c_double
            lib.lo_band.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5
            lib.lo_filling.restype = ctypes.c_double
            lib.lo_filling.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_double]
            lib.lo_mu.restype = ctypes.c_int
            lib.lo_mu.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_double, _dp]
            lib.lo_spectral.restype = None
            lib.lo_spectral.argtypes = ([ctypes.c_int] + [ctypes.c_double] * 6
                                        + [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp])
            lib.lo_dmu_dparams.restype = None
            lib.lo_dmu_dparams.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_double, _dp]
            lib.lo_kk_real.restype = None
            lib.lo_kk_real.argtypes = [ctypes.c_long, ctypes.c_int, _dp, _dp]
            lib.lo_rpa.restype = None
            lib.lo_rpa.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            lib.lo_imchi_samples.restype = None
            lib.lo_imchi_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                             ctypes.c_int, ctypes.c_long, _ip, _ip, _ip, _dp]
            lib.lo_thermal_samples.restype = None
            lib.lo_thermal_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_long, _ip, _ip,
                                               _ip, _dp]
            lib.lo_grad_A_samples.restype = None
            lib.lo_grad_A_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                              ctypes.c_int, ctypes.c_int, _dp, ctypes.c_long, _ip, _ip, _ip, _dp]
            lib.lo_thermal_grad_A_samples.restype = None
            lib.lo_thermal_grad_A_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                                      ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                                      ctypes.c_long, _ip, _ip, _ip, _dp]
            lib.lo_spectral_dtheta.restype = None
            lib.lo_spectral_dtheta.argtypes = ([ctypes.c_double] * 6
                                               + [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp])
            lib.lo_num_threads.restype = ctypes.c_int
            lib.lo_num_threads.argtypes = []
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def dmu_dparams(kind, t, tp, tpp, gamma, npz, mu) -> np.ndarray:
    """dmu/d(t, t', t'', gamma) at fixed filling (implicit function theorem on
    the rigid-band count of Sec. 3); see lo_dmu_dparams."""
    out = np.zeros(4)
    _load().lo_dmu_dparams(int(kind), float(t), float(tp), float(tpp), float(gamma), int(npz), float(mu), _d(out))
    return out


def kk_real(im: np.ndarray) -> np.ndarray:
    """Re chi from Im chi along the last axis (transfers w_m = m de) by the
    Kramers-Kronig relation of Sec. 4 in Maclaurin's discretisation (odd Im chi
    in w, zero beyond the window); see lo_kk_real."""
    im = np.ascontiguousarray(im, dtype=np.float64)
    n_omega = im.shape[-1]
    out = np.empty_like(im)
    _load().lo_kk_real(ctypes.c_long(im.size // n_omega), n_omega, _d(im), _d(out))
    return out


def rpa(re: np.ndarray, im: np.ndarray, dp: float, v0: float) -> np.ndarray:
    """chi_RPA = chi / (1 - V_q chi), V_q = v0 / |q|^2 (Sec. 4), for chi on the
    lag grid [Q][Q][n_omega]; returns [Q][Q][n_omega] complex."""
    re = np.ascontiguousarray(re, dtype=np.float64)
    im = np.ascontiguousarray(im, dtype=np.float64)
    Q, _, n_omega = re.shape
    out = np.empty(re.shape + (2,), dtype=np.float64)
    _load().lo_rpa(Q, n_omega, float(dp), float(v0), _d(re), _d(im), _d(out))
    return out[..., 0] + 1j * out[..., 1]


def num_threads() -> int:
    """OpenMP threads the oracle uses (for reporting the CPU baseline)."""
    return int(_load().lo_num_threads())


def band(kind: int, t: float, tp: float, tpp: float, px: float, py: float) -> float:
    """eps0(p) in eV (tight binding, kind 0; free electrons |p|^2/2, kind 1)."""
    return float(_load().lo_band(int(kind), t, tp, tpp, px, py))


def filling(kind, t, tp, tpp, gamma, npz, mu) -> float:
    """Electrons per site incl. spin at chemical potential mu (rigid band, Sec. 3)."""
    return float(_load().lo_filling(int(kind), t, tp, tpp, gamma, int(npz), mu))


def solve_mu(kind, t, tp, tpp, gamma, npz, fill) -> float:
    """mu with filling(mu) == fill, FP64 bisection (rigid band, Sec. 3)."""
    out = ctypes.c_double(0.0)
    rc = _load().lo_mu(int(kind), t, tp, tpp, gamma, int(npz), fill, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"filling {fill} outside (0, 2)")
    return out.value


def grid_sizes(zones: int, npz: int, n_eps: int, e_max: float):
    """N, dp, de and the Eq. 9 prefactor c = de/(2 pi) / npz^2."""
    N = zones * npz
    dp = 2.0 * math.pi / npz
    de = 2.0 * e_max / n_eps
    c = de / (2.0 * math.pi) / float(npz * npz)
    return N, dp, de, c


def spectral(band_p: dict, grid: dict) -> np.ndarray:
    """A(p_i, e_j) in FP64, shape [N, N, n_eps] (Eqs. 4-5).

    band_p: kind, t, tp, tpp, mu, gamma, ff_a.  grid: zones, npz, n_eps, e_max."""
    N = grid["zones"] * grid["npz"]
    A = np.empty((N, N, grid["n_eps"]), dtype=np.float64)
    _load().lo_spectral(int(band_p.get("kind", 0)), band_p["t"], band_p["tp"], band_p["tpp"], band_p["mu"],
                        band_p["gamma"], band_p.get("ff_a", 0.0), grid["zones"], grid["npz"], grid["n_eps"],
                        grid["e_max"], _d(A))
    return A


def imchi_samples(A: np.ndarray, grid: dict, q_extent: int, lx, ly, m) -> np.ndarray:
    """The discrete Eq. 9 at the given output indices (direct double sum, FP64)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    lx = np.ascontiguousarray(lx, dtype=np.int32)
    ly = np.ascontiguousarray(ly, dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = lx.size
    assert ly.size == n and m.size == n
    N = grid["zones"] * grid["npz"]
    assert A.shape == (N, N, grid["n_eps"])
    out = np.empty(n, dtype=np.float64)
    _load().lo_imchi_samples(grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"], _d(A), int(q_extent),
                             n, _i(lx), _i(ly), _i(m), _d(out))
    return out


def imchi_full(A: np.ndarray, grid: dict, q_extent: int, n_omega: int) -> np.ndarray:
    """Every output of the discrete Eq. 9, shape [Q, Q, n_omega] (small grids only)."""
    Q = q_extent
    lx, ly, m = np.meshgrid(np.arange(Q), np.arange(Q), np.arange(n_omega), indexing="ij")
    return imchi_samples(A, grid, Q, lx.ravel(), ly.ravel(), m.ravel()).reshape(Q, Q, n_omega)


IMCHI_T, SQW = 1, 2


def thermal_samples(A: np.ndarray, grid: dict, q_extent: int, kT: float, quantity: int, lx, ly, m) -> np.ndarray:
    """Finite temperature kT > 0 (Eq. 1, Eq. A1) at the given output indices
    (direct double sum, FP64): quantity IMCHI_T gives Im chi_T with the
    occupation difference f(e) - f(e + w); SQW gives the dynamical structure
    factor S(q, w) = -(1/pi) Im chi_T / (1 - exp(-w/kT)), summed as
    (c/pi) sum A A f(e) [1 - f(e + w)].  m may be negative."""
    assert kT > 0 and quantity in (IMCHI_T, SQW)
    A = np.ascontiguousarray(A, dtype=np.float64)
    lx = np.ascontiguousarray(lx, dtype=np.int32)
    ly = np.ascontiguousarray(ly, dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = lx.size
    assert ly.size == n and m.size == n
    N = grid["zones"] * grid["npz"]
    assert A.shape == (N, N, grid["n_eps"])
    out = np.empty(n, dtype=np.float64)
    _load().lo_thermal_samples(grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"], _d(A), int(q_extent),
                               float(kT), int(quantity), n, _i(lx), _i(ly), _i(m), _d(out))
    return out


def thermal_full(A: np.ndarray, grid: dict, q_extent: int, n_omega: int, kT: float, quantity: int) -> np.ndarray:
    """Every output of thermal_samples, shape [Q, Q, n_omega] (small grids only)."""
    Q = q_extent
    lx, ly, m = np.meshgrid(np.arange(Q), np.arange(Q), np.arange(n_omega), indexing="ij")
    return thermal_samples(A, grid, Q, kT, quantity, lx.ravel(), ly.ravel(), m.ravel()).reshape(Q, Q, n_omega)


def grad_A_samples(A: np.ndarray, grid: dict, q_extent: int, w: np.ndarray, ix, iy, j) -> np.ndarray:
    """dL/dA at sample points for L = sum w * Im chi (adjoint of Eq. 9)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Q = q_extent
    assert w.shape[0] == Q and w.shape[1] == Q
    n_omega = w.shape[2]
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    out = np.empty(ix.size, dtype=np.float64)
    _load().lo_grad_A_samples(grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"], _d(A), Q, n_omega,
                              _d(w), ix.size, _i(ix), _i(iy), _i(j), _d(out))
    return out


def grad_A_full(A: np.ndarray, grid: dict, q_extent: int, w: np.ndarray) -> np.ndarray:
    """dL/dA at every grid point, shape [N, N, n_eps] (small grids only)."""
    N = grid["zones"] * grid["npz"]
    ix, iy, j = np.meshgrid(np.arange(N), np.arange(N), np.arange(grid["n_eps"]), indexing="ij")
    return grad_A_samples(A, grid, q_extent, w, ix.ravel(), iy.ravel(), j.ravel()).reshape(N, N, grid["n_eps"])


def thermal_grad_A_samples(A: np.ndarray, grid: dict, q_extent: int, w: np.ndarray, kT: float, quantity: int,
                           ix, iy, j) -> np.ndarray:
    """dL/dA at sample points for L = sum w * X, X = Im chi_T (IMCHI_T) or
    S(q, w) (SQW) at temperature kT (adjoint of Eq. A1 / Eq. 1 as
    thermal_samples sums them)."""
    assert kT > 0 and quantity in (IMCHI_T, SQW)
    A = np.ascontiguousarray(A, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Q = q_extent
    assert w.shape[0] == Q and w.shape[1] == Q
    n_omega = w.shape[2]
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    out = np.empty(ix.size, dtype=np.float64)
    _load().lo_thermal_grad_A_samples(grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"], _d(A), Q, n_omega,
                                      float(kT), int(quantity), _d(w), ix.size, _i(ix), _i(iy), _i(j), _d(out))
    return out


def thermal_grad_A_full(A: np.ndarray, grid: dict, q_extent: int, w: np.ndarray, kT: float,
                        quantity: int) -> np.ndarray:
    """thermal_grad_A_samples at every grid point, shape [N, N, n_eps] (small grids only)."""
    N = grid["zones"] * grid["npz"]
    ix, iy, j = np.meshgrid(np.arange(N), np.arange(N), np.arange(grid["n_eps"]), indexing="ij")
    return thermal_grad_A_samples(A, grid, q_extent, w, kT, quantity, ix.ravel(), iy.ravel(),
                                  j.ravel()).reshape(N, N, grid["n_eps"])


def spectral_dtheta(band_p: dict, grid: dict) -> np.ndarray:
    """dA/d(t, t', t'', mu, gamma), shape [5, N, N, n_eps] (tight binding)."""
    N = grid["zones"] * grid["npz"]
    out = np.empty((5, N, N, grid["n_eps"]), dtype=np.float64)
    _load().lo_spectral_dtheta(band_p["t"], band_p["tp"], band_p["tpp"], band_p["mu"], band_p["gamma"],
                               band_p.get("ff_a", 0.0), grid["zones"], grid["npz"], grid["n_eps"],
                               grid["e_max"], _d(out))
    return out


def grad_params(A: np.ndarray, band_p: dict, grid: dict, q_extent: int, w: np.ndarray) -> np.ndarray:
    """dL/d(t, t', t'', mu, gamma) = sum_{p,j} dL/dA(p,j) dA(p,j)/dtheta (chain rule
    through Eqs. 4-5; mu is held as an independent parameter)."""
    g = grad_A_full(A, grid, q_extent, w)
    d = spectral_dtheta(band_p, grid)
    return np.array([float(np.sum(g * d[r])) for r in range(5)])


def loss(A: np.ndarray, grid: dict, q_extent: int, w: np.ndarray) -> float:
    """L = sum_{l,m} w(l,m) Im chi(q_l, w_m) from the direct sum (small grids only)."""
    chi = imchi_full(A, grid, q_extent, w.shape[2])
    return float(np.sum(w * chi))


def envelope_k0(imchi: np.ndarray, npz: int, m: int):
    """Envelope of -Im chi along the [100] cut (Sec. 4, Fig. 5): the cut is
    q = (q_x, 0), lags l_x with l_y = Q/2, at transfer index m.  Each zone
    n >= 0 of the reciprocal lattice along the cut (lag offsets
    [n npz - npz/2, n npz + npz/2) from Q/2) that the lag window holds whole
    contributes its maximum of
    -Im chi and where it sits; normalised by the largest of them, the points
    are fitted by the Lorentzian shape 1 / (1 + (q/k0)^2) in least squares over
    the points with q > 0.  The one-parameter fit is a golden-section search
    over ln k0 in [ln dp, ln (Q dp)], 200 steps.  Returns (k0 in units of 1/a,
    q of the zone maxima, normalised maxima)."""
    Q = imchi.shape[0]
    dp = 2.0 * math.pi / npz
    cut = -np.asarray(imchi[:, Q // 2, m], dtype=np.float64)
    qs, ys = [], []
    n = 0
    while True:
        lo = Q // 2 + n * npz - npz // 2
        hi = lo + npz
        if lo < 0 or hi > Q:         # only zones the lag window holds whole
            break
        seg = cut[lo:hi]
        i = int(np.argmax(seg))      # first index of the maximum
        qs.append((lo + i - Q // 2) * dp)
        ys.append(seg[i])
        n += 1
    qs, ys = np.array(qs), np.array(ys)
    if len(ys) == 0 or not ys.max() > 0:
        raise ValueError("-Im chi has no positive zone maximum on the cut")
    ys = ys / ys.max()
    keep = qs > 0

    def cost(lk):
        k = math.exp(lk)
        return float(np.sum((ys[keep] - 1.0 / (1.0 + (qs[keep] / k) ** 2)) ** 2))

    a, b = math.log(dp), math.log(Q * dp)
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = cost(c), cost(d)
    for _ in range(200):
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = cost(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = cost(d)
    return math.exp(0.5 * (a + b)), qs, ys
