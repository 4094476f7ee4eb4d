"""Python binding of liblindhard.so (include/lindhard.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
Python parameters to the C structs, passes torch tensors' device pointers and
the current CUDA stream, and maps status codes to exceptions.  There is no
fallback: if the library cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblindhard.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOCONV, EUNSUPPORTED = range(7)
FP32, SPLITBF16_TC, FP64 = 0, 1, 2
IMCHI, IMCHI_T, SQW = 0, 1, 2          # lindhard_quantity
PLAN_BACKWARD, PLAN_CONCURRENT, PLAN_GRAPH, PLAN_AUTOTUNE, PLAN_ENERGY_DIRECT, PLAN_PERSISTENT = 1, 2, 4, 8, 16, 32
_STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT",
                 ENOCONV: "ENOCONV", EUNSUPPORTED: "EUNSUPPORTED"}

# Exported symbols, in the order include/lindhard.h declares them.
SYMBOLS = ("lindhard_plan_create", "lindhard_plan_sizes", "lindhard_plan_workspace_bytes", "lindhard_imchi",
           "lindhard_imchi_f64", "lindhard_imchi_backward", "lindhard_plan_profile", "lindhard_plan_profile_passes",
           "lindhard_plan_pass_times",
           "lindhard_sum_rule", "lindhard_dmu_dparams", "lindhard_envelope_k0", "lindhard_kk_rpa",
           "lindhard_plan_set_wait_limit", "lindhard_plan_variants", "lindhard_plan_status", "lindhard_plan_destroy",
           "lindhard_imchi_noalloc", "lindhard_last_error")
NOALLOC_SCRATCH_BYTES = 32 << 20
NUM_PASSES = 7
PASS_NAMES = ("tables", "mu_solve", "energy_fwd", "py_fwd", "px_product", "py_inv", "energy_inv")


class LindhardError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Band(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("tp", ctypes.c_double), ("tpp", ctypes.c_double),
                ("mu", ctypes.c_double), ("filling", ctypes.c_double), ("gamma", ctypes.c_double),
                ("ff_a", ctypes.c_double), ("band_kind", ctypes.c_int), ("reserved", ctypes.c_int),
                ("kT", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("zones", ctypes.c_int), ("pts_per_zone", ctypes.c_int), ("n_eps", ctypes.c_int),
                ("e_max", ctypes.c_double), ("n_omega", ctypes.c_int), ("q_extent", ctypes.c_int),
                ("precision", ctypes.c_int), ("quantity", ctypes.c_int)]


class Sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in ("N", "n_eps", "n_omega", "q_extent", "fft_p", "fft_e",
                                                 "out_elems", "a_elems", "hbm_bytes_forward",
                                                 "kernels_forward")]


_lib = None


def load(path: str = LIB_PATH):
    """Load liblindhard.so (build it first with paper_1208_3210_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_1208_3210_gb300.build.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.lindhard_plan_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_uint, ctypes.POINTER(vp)]
        lib.lindhard_plan_sizes.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Sizes)]
        lib.lindhard_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.lindhard_imchi.argtypes = [vp, ctypes.POINTER(Band), vp, vp, vp, vp]
        lib.lindhard_imchi_f64.argtypes = [vp, ctypes.POINTER(Band), vp, vp, vp, vp]
        lib.lindhard_imchi_backward.argtypes = [vp, ctypes.POINTER(Band), vp, vp, vp, vp, vp]
        lib.lindhard_plan_profile.argtypes = [vp, ctypes.c_int]
        lib.lindhard_plan_profile_passes.argtypes = [vp, ctypes.c_uint]
        lib.lindhard_plan_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        lib.lindhard_plan_status.argtypes = [vp, vp]
        lib.lindhard_plan_variants.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.lindhard_plan_destroy.argtypes = [vp]
        lib.lindhard_plan_destroy.restype = None
        lib.lindhard_last_error.restype = ctypes.c_char_p
        lib.lindhard_imchi_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Band), vp, vp, vp, vp]
        lib.lindhard_imchi_noalloc.restype = ctypes.c_int
        lib.lindhard_sum_rule.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Band), vp, vp, vp, vp, vp]
        lib.lindhard_sum_rule.restype = ctypes.c_int
        lib.lindhard_dmu_dparams.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Band), ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double), vp]
        lib.lindhard_dmu_dparams.restype = ctypes.c_int
        lib.lindhard_envelope_k0.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
        lib.lindhard_envelope_k0.restype = ctypes.c_int
        lib.lindhard_kk_rpa.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_double, ctypes.c_int, vp]
        lib.lindhard_kk_rpa.restype = ctypes.c_int
        for name in ("lindhard_plan_create", "lindhard_plan_sizes", "lindhard_plan_workspace_bytes",
                     "lindhard_imchi", "lindhard_imchi_f64", "lindhard_imchi_backward", "lindhard_plan_profile",
                     "lindhard_plan_pass_times", "lindhard_plan_status", "lindhard_plan_set_wait_limit"):
            getattr(lib, name).restype = ctypes.c_int
        lib.lindhard_plan_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_int]
        _lib = lib
    return _lib


def _check(status: int):
    if status != OK:
        raise LindhardError(status, load().lindhard_last_error().decode())


def make_grid(zones, npz, n_eps, e_max, n_omega=0, q_extent=0, precision=FP32, quantity=IMCHI) -> Grid:
    return Grid(int(zones), int(npz), int(n_eps), float(e_max), int(n_omega), int(q_extent), int(precision),
                int(quantity))


def make_band(t=0.42, tp=-0.10, tpp=0.065, mu=float("nan"), filling=1.15, gamma=0.05, ff_a=0.0,
              kind=0, kT=0.0, **_ignored) -> Band:
    return Band(float(t), float(tp), float(tpp), float(mu), float(filling), float(gamma), float(ff_a), int(kind), 0,
                float(kT))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def imchi_noalloc(grid: dict, band=None, out=None, A_in=None, mu_out=None, stream=None):
    """One forward call through lindhard_imchi_noalloc, which allocates no
    device memory: for callers that cannot allocate when they need Im chi.
    `out` (float32, Q*Q*n_omega elements) must be supplied by the caller; all
    intermediates live in the library's fixed 32 MiB device array, so calls
    that could overlap on the GPU must be serialised."""
    g = make_grid(grid["zones"], grid["npz"], grid["n_eps"], grid["e_max"], grid.get("n_omega", 0),
                  grid.get("q_extent", 0), FP32, grid.get("quantity", IMCHI))
    b = None if band is None else (band if isinstance(band, Band) else make_band(**band))
    _check(load().lindhard_imchi_noalloc(ctypes.byref(g), None if b is None else ctypes.byref(b), _ptr(A_in),
                                         _ptr(out), _ptr(mu_out), _stream(stream)))
    return out


class Plan:
    """A lindhard_plan for one or more instance grids (dicts with zones, npz,
    n_eps, e_max and optional n_omega, q_extent, precision, quantity)."""

    def __init__(self, grids: Sequence[dict], precision: int = FP32, backward: bool = False,
                 concurrent: bool = False, graph: bool = False, autotune: bool = False,
                 energy_direct: bool = False, persistent: bool = False):
        lib = load()
        self.grids = [make_grid(g["zones"], g["npz"], g["n_eps"], g["e_max"], g.get("n_omega", 0),
                                g.get("q_extent", 0), g.get("precision", precision), g.get("quantity", IMCHI))
                      for g in grids]
        self.batch = len(self.grids)
        arr = (Grid * self.batch)(*self.grids)
        h = ctypes.c_void_p()
        flags = (PLAN_BACKWARD if backward else 0) | (PLAN_CONCURRENT if concurrent else 0) | \
            (PLAN_GRAPH if graph else 0) | (PLAN_AUTOTUNE if autotune else 0) | \
            (PLAN_ENERGY_DIRECT if energy_direct else 0) | (PLAN_PERSISTENT if persistent else 0)
        _check(lib.lindhard_plan_create(arr, self.batch, flags, ctypes.byref(h)))
        self._h = h
        self.sizes = []
        for i in range(self.batch):
            s = Sizes()
            _check(lib.lindhard_plan_sizes(h, i, ctypes.byref(s)))
            self.sizes.append(s)
        self.precision = self.grids[0].precision

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(load().lindhard_plan_workspace_bytes(self._h, ctypes.byref(n)))
        return n.value

    def out_elems(self) -> int:
        return sum(s.out_elems for s in self.sizes)

    def a_elems(self) -> int:
        return sum(s.a_elems for s in self.sizes)

    def _bands(self, bands):
        if bands is None:
            return None
        if isinstance(bands, dict):
            bands = [bands]
        assert len(bands) == self.batch
        return (Band * self.batch)(*[b if isinstance(b, Band) else make_band(**b) for b in bands])

    def imchi(self, bands=None, out=None, A_in=None, mu_out=None, stream=None):
        """Im chi for every instance into `out` (device tensor, concatenated
        [Q][Q][n_omega] blocks).  Allocates `out` when it is None."""
        import torch
        f64 = self.precision == FP64
        dt = torch.float64 if f64 else torch.float32
        if out is None:
            out = torch.empty(self.out_elems(), dtype=dt, device="cuda")
        assert out.dtype == dt and out.is_cuda and out.is_contiguous() and out.numel() == self.out_elems()
        if A_in is not None:
            assert A_in.dtype == dt and A_in.is_cuda and A_in.is_contiguous() and A_in.numel() == self.a_elems()
        if mu_out is not None:
            assert mu_out.dtype == torch.float64 and mu_out.is_cuda and mu_out.numel() >= self.batch
        fn = load().lindhard_imchi_f64 if f64 else load().lindhard_imchi
        _check(fn(self._h, self._bands(bands), _ptr(A_in), _ptr(out), _ptr(mu_out), _stream(stream)))
        return out

    def backward(self, w, bands=None, A_in=None, dA=None, dparams=None, stream=None):
        """Adjoint for L = sum w * X (X the grids' quantity: Im chi, Im chi_T or
        S(q, w)): fills dA (float32, A layout) and/or dparams (float64,
        [batch][5] = dL/d(t, t', t'', mu, gamma))."""
        assert w.dtype.is_floating_point and w.is_cuda and w.is_contiguous() and w.numel() == self.out_elems()
        if dA is not None:
            assert dA.is_cuda and dA.is_contiguous() and dA.numel() == self.a_elems()
        if dparams is not None:
            assert dparams.is_cuda and dparams.numel() >= 5 * self.batch
        _check(load().lindhard_imchi_backward(self._h, self._bands(bands), _ptr(A_in), _ptr(w), _ptr(dA),
                                              _ptr(dparams), _stream(stream)))
        return dA, dparams

    def profile(self, enable: bool = True, passes=None):
        """Start (or stop) per-pass CUDA-event timing of every pass, or of the
        named passes only (names as in PASS_NAMES); clears accumulated times."""
        if passes is None:
            _check(load().lindhard_plan_profile(self._h, 1 if enable else 0))
        else:
            mask = sum(1 << PASS_NAMES.index(n) for n in passes) if enable else 0
            _check(load().lindhard_plan_profile_passes(self._h, mask))

    def pass_times(self):
        """{pass name: (total ms, launches)} since profiling was enabled."""
        ms = (ctypes.c_double * NUM_PASSES)()
        n = (ctypes.c_longlong * NUM_PASSES)()
        _check(load().lindhard_plan_pass_times(self._h, ms, n))
        return {PASS_NAMES[i]: (ms[i], n[i]) for i in range(NUM_PASSES)}

    def sum_rule(self, index, out_i, band=None, A_in=None, stream=None):
        """(sum_q Im chi(q, w_m), -c sum_j D_a(e_j) D_b(e_{j+m})) in FP64 for
        instance `index` (its output slice `out_i`)."""
        import torch
        n_omega = self.sizes[index].n_omega
        sq = torch.empty(n_omega, dtype=torch.float64, device="cuda")
        dc = torch.empty(n_omega, dtype=torch.float64, device="cuda")
        b = None if band is None else (band if isinstance(band, Band) else make_band(**band))
        _check(load().lindhard_sum_rule(self._h, int(index), None if b is None else ctypes.byref(b), _ptr(A_in),
                                        _ptr(out_i), _ptr(sq), _ptr(dc), _stream(stream)))
        return sq, dc

    def dmu_dparams(self, band, mu, index=0, stream=None):
        """dmu/d(t, t', t'', gamma) at fixed filling, at chemical potential mu
        (numpy float64 [4])."""
        import numpy as np
        b = band if isinstance(band, Band) else make_band(**band)
        out = (ctypes.c_double * 4)()
        _check(load().lindhard_dmu_dparams(self._h, int(index), ctypes.byref(b), float(mu), out, _stream(stream)))
        return np.array(list(out))

    def envelope_k0(self, out_i, m, index=0, stream=None):
        """k0 of the Lorentzian envelope 1 / (1 + (q/k0)^2) of -Im chi along the
        [100] cut at transfer index m, with the zone maxima (q, normalised
        -Im chi) it was fitted to."""
        import numpy as np
        s = self.sizes[index]
        cap = s.q_extent // max(1, self.grids[index].pts_per_zone) + 2
        k0 = ctypes.c_double()
        q = (ctypes.c_double * cap)()
        y = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(load().lindhard_envelope_k0(self._h, int(index), _ptr(out_i), int(m), ctypes.byref(k0), q, y, cap,
                                           ctypes.byref(n), _stream(stream)))
        k = min(n.value, cap)
        return k0.value, np.array(list(q)[:k]), np.array(list(y)[:k])

    def kk_rpa(self, out_i, index=0, v0=0.0, rpa=True, variant=0, stream=None):
        """Re chi by Kramers-Kronig and chi_RPA = chi / (1 - v0/|q|^2 chi) for
        instance `index` from its Im chi block `out_i` (device float32
        [Q][Q][n_omega] or flat).  variant 0: tensor cores (n_omega <= 256);
        1: FP32 SIMT.  Returns (Re chi, chi_RPA as complex64 or None), shaped
        [Q][Q][n_omega]."""
        import torch
        s = self.sizes[index]
        shape = (s.q_extent, s.q_extent, s.n_omega)
        assert out_i.dtype == torch.float32 and out_i.is_cuda and out_i.is_contiguous()
        assert out_i.numel() == s.out_elems
        re = torch.empty(shape, dtype=torch.float32, device="cuda")
        rp = torch.empty(shape + (2,), dtype=torch.float32, device="cuda") if rpa else None
        _check(load().lindhard_kk_rpa(self._h, int(index), _ptr(out_i), _ptr(re), _ptr(rp), float(v0), int(variant),
                                      _stream(stream)))
        return re, (torch.view_as_complex(rp) if rpa else None)

    def status(self, stream=None):
        _check(load().lindhard_plan_status(self._h, _stream(stream)))

    def set_wait_limit(self, wait_ns: int = 0, stall_instance: int = -1):
        """Bounded-wait limit of a persistent plan (ns; 0 = the default 1 s);
        stall_instance >= 0 makes that instance's first dependency wait run out
        (a test of the timeout path)."""
        _check(load().lindhard_plan_set_wait_limit(self._h, int(wait_ns), int(stall_instance)))

    def variants(self, index=0):
        """Engine variants of instance `index`: {"py_fwd", "py_inv", "px_product", "energy_inv"}."""
        v = (ctypes.c_int * 4)()
        _check(load().lindhard_plan_variants(self._h, index, v))
        return {"py_fwd": v[0], "py_inv": v[1], "px_product": v[2], "energy_inv": v[3]}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lindhard_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- autograd ---------------------------------------------------------------------

PARAM_NAMES = ("t", "tp", "tpp", "mu", "gamma")


class ImChiFunction:
    """torch.autograd.Function over the library's forward and adjoint calls.

    ``ImChiFunction.apply(params, plan, band)``: params is a float64 tensor of
    shape [batch, 5] holding (t, t', t'', mu, gamma) per instance (mu is used
    as given, so the gradient is the partial derivative at fixed mu); band
    supplies the rest of each instance (ff_a, band_kind).  Returns the
    concatenated Im chi (float32).  backward() calls lindhard_imchi_backward
    with w = grad_output and returns dL/dparams.  The plan must be created with
    backward=True."""

    _cls = None

    @classmethod
    def _get(cls):
        if cls._cls is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, params, plan, bands):
                    ctx.plan = plan
                    ctx.device = params.device
                    ctx.bands = _bands_with(params, bands)
                    return plan.imchi(ctx.bands)

                @staticmethod
                def backward(ctx, grad_out):
                    plan = ctx.plan
                    dp = torch.zeros(5 * plan.batch, dtype=torch.float64, device="cuda")
                    plan.backward(grad_out.contiguous().float(), bands=ctx.bands, dparams=dp)
                    return dp.reshape(plan.batch, 5).to(ctx.device), None, None

            cls._cls = _F
        return cls._cls

    @classmethod
    def apply(cls, params, plan, bands):
        return cls._get().apply(params, plan, bands)


def _bands_with(params, bands):
    """Bands with (t, t', t'', mu, gamma) taken from params[i] and the filling
    unset, so that mu is used as given."""
    vals = params.detach().double().cpu().numpy().reshape(-1, 5)
    if isinstance(bands, dict):
        bands = [bands]
    out = []
    for i, b in enumerate(bands):
        d = dict(b)
        d.update(t=float(vals[i, 0]), tp=float(vals[i, 1]), tpp=float(vals[i, 2]), mu=float(vals[i, 3]),
                 gamma=float(vals[i, 4]), filling=float("nan"))
        out.append(d)
    return out
