"""Seeded synthetic inputs for the FFT Lindhard susceptibility workloads.

This module holds parameter sets and random draws only: no step of the
susceptibility calculation lives here.  It is the one module that both the
GPU library's callers and the FP64 oracle's callers use, so that both sides
see identical inputs.

The paper's own inputs (the KKR-LDA CuO2 band of NCCO and its electron
momentum density, Sec. 3) are not available; a single-band square-lattice
tight-binding band with a Gaussian momentum-density envelope stands in for
them, on momentum grids that span several Brillouin zones as in Sec. 4.
"""
from __future__ import annotations

import math

import numpy as np

# Tight-binding band standing in for the CuO2 band of Sec. 3 (eV); it spans
# [-1.54, 1.82] eV, close to the band range the paper quotes for NCCO.
BAND_TB = dict(kind=0, t=0.42, tp=-0.10, tpp=0.065)


def band_params(filling=1.15, gamma=0.05, ff_a=0.0, mu=float("nan"), **over):
    """One instance's physics: hoppings, filling (electrons/site incl. spin),
    Lorentzian half-width gamma (eV), form-factor length ff_a (0 => |M|^2 = 1).
    mu is solved from the filling when it is NaN."""
    p = dict(BAND_TB)
    p.update(filling=float(filling), gamma=float(gamma), ff_a=float(ff_a), mu=float(mu))
    p.update(over)
    return p


def grid_params(zones, npz, n_eps, e_max, n_omega=0, q_extent=0, **extra):
    """One instance's grid: zones per axis, points per zone per axis, energy
    count and half-window.  n_omega = 0 => n_eps // 2, q_extent = 0 => N.
    extra: optional keys passed through (precision, quantity)."""
    N = zones * npz
    return dict(zones=int(zones), npz=int(npz), n_eps=int(n_eps), e_max=float(e_max),
                n_omega=int(n_omega) if n_omega else int(n_eps) // 2,
                q_extent=int(q_extent) if q_extent else int(N), **extra)


# The five workloads.  Sizes follow the problem statement of each:
#   reduced   : one zone, 32 x 32 k-points, 48 energies on [-1, 1] eV
#   extended  : 4 x 4 zones x 64 points/zone (256 x 256), 256 energies on [-2, 2] eV
#   large     : 8 x 8 zones x 128 points/zone (1024 x 1024), 512 energies on [-3, 3] eV
#   batched   : 64 instances of mixed filling, broadening and size
#   gradient  : the extended geometry with a seeded weight w(q, w)
WORKLOADS = {
    "reduced_32x32x48": dict(band=band_params(filling=1.15, gamma=0.05, ff_a=0.0),
                             grid=grid_params(1, 32, 48, 1.0)),
    "extended_256x256x256": dict(band=band_params(filling=1.15, gamma=0.05, ff_a=1.0),
                                 grid=grid_params(4, 64, 256, 2.0)),
    "large_1024x1024x512": dict(band=band_params(filling=1.15, gamma=0.03, ff_a=1.0),
                                grid=grid_params(8, 128, 512, 3.0)),
}

# Fillings of the batched workload: x in {0.04, 0.06, ..., 0.16, 0.17}, plus one.
BATCH_FILLINGS = [1.04, 1.06, 1.08, 1.10, 1.12, 1.14, 1.16, 1.17]


def batched_instances(count=64, seed=0):
    """The batched workload: `count` independent instances with seeded
    broadening in [0.02, 0.2] eV, N in {128, 256, 512}, 2 or 4 zones,
    128 or 256 energies on [-2, 2] eV, fillings cycled over BATCH_FILLINGS."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        gamma = float(rng.uniform(0.02, 0.2))
        N = int(rng.choice([128, 256, 512]))
        zones = int(rng.choice([2, 4]))
        n_eps = int(rng.choice([128, 256]))
        out.append(dict(band=band_params(filling=BATCH_FILLINGS[i % len(BATCH_FILLINGS)], gamma=gamma, ff_a=1.0),
                        grid=grid_params(zones, N // zones, n_eps, 2.0)))
    return out


def batched_workload(count=64, seed=0):
    """(grids, bands) of the batched workload, in instance order."""
    inst = batched_instances(count, seed)
    return [x["grid"] for x in inst], [x["band"] for x in inst]


def loss_weights(grid, seed=0, dtype=np.float32):
    """w(q_l, w_m) ~ U[0, 1], shape [Q, Q, n_omega], for L = sum w Im chi."""
    rng = np.random.default_rng(seed)
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    return rng.uniform(0.0, 1.0, size=(Q, Q, n_omega)).astype(dtype)


def output_samples(grid, count, seed=0, near_origin=8):
    """Seeded output indices (lx, ly, m), stratified by energy transfer and by
    |q| shell, plus every m at a block of lags around q = 0 where |Im chi| peaks.
    Returns int32 arrays lx, ly, m."""
    rng = np.random.default_rng(seed)
    Q, n_omega = grid["q_extent"], grid["n_omega"]
    lx, ly, m = [], [], []
    # a small block around the origin, all energies
    h = max(1, near_origin // 2)
    for dx in range(-h, h):
        for dy in range(-h, h):
            for mm in range(0, n_omega, max(1, n_omega // 16)):
                lx.append(Q // 2 + dx)
                ly.append(Q // 2 + dy)
                m.append(mm)
    # stratified remainder: energy strata x radial shells
    n_shell, n_e = 8, 8
    rest = max(0, count - len(lx))
    per = max(1, rest // (n_shell * n_e))
    rmax = math.hypot(Q / 2, Q / 2)
    for s in range(n_shell):
        for e in range(n_e):
            k = 0
            while k < per:
                x = int(rng.integers(0, Q))
                y = int(rng.integers(0, Q))
                r = math.hypot(x - Q / 2, y - Q / 2) / rmax
                if int(r * n_shell) != s and not (s == n_shell - 1 and r >= 1.0):
                    continue
                lx.append(x)
                ly.append(y)
                lo = e * n_omega // n_e
                hi = max(lo + 1, (e + 1) * n_omega // n_e)
                m.append(int(rng.integers(lo, hi)))
                k += 1
    return (np.asarray(lx, np.int32), np.asarray(ly, np.int32), np.asarray(m, np.int32))


def spectral_samples(grid, count, seed=0):
    """Seeded grid points (ix, iy, j) at which dL/dA is compared."""
    rng = np.random.default_rng(seed)
    N = grid["zones"] * grid["npz"]
    return (rng.integers(0, N, count).astype(np.int32), rng.integers(0, N, count).astype(np.int32),
            rng.integers(0, grid["n_eps"], count).astype(np.int32))


def random_spectral(grid, seed=0, dtype=np.float32):
    """A caller-supplied A(p, e) >= 0 with no lattice symmetry, shape
    [N, N, n_eps] (exercises the path that takes A instead of generating it)."""
    rng = np.random.default_rng(seed)
    N = grid["zones"] * grid["npz"]
    return rng.uniform(0.0, 1.0, size=(N, N, grid["n_eps"])).astype(dtype)
