"""The C ABI library: it loads, exports every function include/*.h declares,
and rejects bad arguments on the host before touching the GPU (no GPU needed)."""
import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        for m in re.finditer(r"\b(lindhard_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1208_3210_gb300 import build, lindhard
    build.build()
    return lindhard.load()


def test_library_exports_every_declared_function(lib):
    from paper_1208_3210_gb300 import lindhard
    declared = _declared_functions()
    assert declared, "no functions found in include/*.h"
    assert declared == set(lindhard.SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def _create(lib, grid):
    from paper_1208_3210_gb300 import lindhard as lh
    h = ctypes.c_void_p()
    st = lib.lindhard_plan_create(ctypes.byref(grid), 1, 0, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,expect", [
    (dict(zones=0, npz=32, n_eps=48, e_max=1.0), 1),
    (dict(zones=1, npz=31, n_eps=48, e_max=1.0), 1),          # odd points per zone
    (dict(zones=1, npz=24, n_eps=48, e_max=1.0), 6),          # reduced zone not a power of two
    (dict(zones=1, npz=8, n_eps=48, e_max=1.0), 6),           # below the smallest FFT
    (dict(zones=2, npz=32, n_eps=1, e_max=1.0), 1),
    (dict(zones=2, npz=32, n_eps=48, e_max=0.0), 1),
    (dict(zones=2, npz=32, n_eps=48, e_max=float("nan")), 1),
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, n_omega=49), 1),
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, q_extent=7), 1),
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, q_extent=130), 1),
    (dict(zones=1, npz=32, n_eps=48, e_max=1.0, q_extent=34), 1),
    (dict(zones=64, npz=128, n_eps=48, e_max=1.0), 6),        # N beyond the compiled FFT range
    (dict(zones=2, npz=96, n_eps=48, e_max=1.0, precision=2), 6),  # FP64 only up to length 256
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, precision=1), 6),  # no tensor-core form for P = 96
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, precision=3), 6),  # no such precision
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, quantity=3), 1),   # no such quantity
    (dict(zones=2, npz=32, n_eps=48, e_max=1.0, quantity=-1), 1),
    (dict(zones=1, npz=32, n_eps=200, e_max=1.0, quantity=2, precision=2), 6),  # finite T pads PE to 512 > 256 (FP64)
])
def test_plan_rejects_bad_grids_on_host(lib, kw, expect):
    from paper_1208_3210_gb300 import lindhard as lh
    g = lh.make_grid(kw["zones"], kw["npz"], kw["n_eps"], kw["e_max"], kw.get("n_omega", 0),
                     kw.get("q_extent", 0), kw.get("precision", 0), kw.get("quantity", 0))
    st, h = _create(lib, g)
    assert st == expect, lib.lindhard_last_error().decode()
    assert not h.value
    assert lib.lindhard_last_error().decode()


def test_tensor_core_precision_rejects_backward_plans(lib):
    # N = 128 pads to P = 192, a length with a tensor-core form; the backward
    # pass is built for LINDHARD_FP32 only (checked before any CUDA call)
    from paper_1208_3210_gb300 import lindhard as lh
    g = lh.make_grid(2, 64, 16, 1.0, 0, 0, lh.SPLITBF16_TC)
    h = ctypes.c_void_p()
    st = lib.lindhard_plan_create(ctypes.byref(g), 1, lh.PLAN_BACKWARD, ctypes.byref(h))
    assert st == lh.EUNSUPPORTED and not h.value
    assert "backward" in lib.lindhard_last_error().decode()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.lindhard_plan_create(None, 1, 0, ctypes.byref(h)) == 1
    assert lib.lindhard_imchi(None, None, None, None, None, None) == 1
    assert lib.lindhard_plan_status(None, None) == 1
    assert lib.lindhard_kk_rpa(None, 0, None, None, None, 0.0, 0, None) == 1
    assert lib.lindhard_envelope_k0(None, 0, None, 0, None, None, None, 0, None, None) == 1
    assert lib.lindhard_dmu_dparams(None, 0, None, 0.0, None, None) == 1
    assert lib.lindhard_plan_set_wait_limit(None, 0, -1) == 1
    lib.lindhard_plan_destroy(None)


@pytest.mark.parametrize("kw,flags,msg", [
    (dict(), 32 | 1, "forward only"),                                   # persistent + backward
    (dict(), 32 | 16, "forward only"),                                  # persistent + energy-direct
    (dict(precision=2), 32, "persistent batch launch takes"),           # FP64
    (dict(quantity=1), 32, "persistent batch launch takes"),            # finite temperature
    (dict(zones=1, npz=128), 32, "persistent batch launch takes"),      # reduced zone
    (dict(q_extent=64), 32, "persistent batch launch takes"),           # Q != N: padding not one third
    (dict(n_eps=1024), 32, "persistent batch launch takes"),            # energy FFT of 1024
])
def test_persistent_plan_rejections_on_host(lib, kw, flags, msg):
    from paper_1208_3210_gb300 import lindhard as lh
    g = lh.make_grid(kw.get("zones", 2), kw.get("npz", 64), kw.get("n_eps", 128), 1.0, 0, kw.get("q_extent", 0),
                     kw.get("precision", 0), kw.get("quantity", 0))
    h = ctypes.c_void_p()
    st = lib.lindhard_plan_create(ctypes.byref(g), 1, flags, ctypes.byref(h))
    assert st == lh.EUNSUPPORTED and not h.value
    assert msg in lib.lindhard_last_error().decode()


@pytest.mark.parametrize("quantity,kT,a_in,band,msg", [
    (0, 0.05, False, True, "kT must be 0"),                  # T = 0 grid with a temperature
    (1, 0.0, False, True, "need kT > 0"),                    # finite-temperature grid at kT = 0
    (2, float("nan"), False, True, "kT must be finite"),
    (2, -0.1, False, True, "kT must be finite"),
    (1, 0.05, True, False, "need bands"),                    # caller A, but no band for kT
    (2, 0.0, True, True, "need kT > 0"),                     # caller A: kT still read and checked
])
def test_temperature_arguments_on_host(lib, quantity, kT, a_in, band, msg):
    # The no-allocation entry checks grid and band before it touches a device.
    # The call gets a made-up device address for its buffers, so it runs in a
    # child process that sees no GPU: should the host checks ever let a case
    # through, the child's first CUDA call fails there instead of a kernel
    # writing through that address on a shared GPU.
    import subprocess
    import sys
    code = f"""
import ctypes, sys
sys.path.insert(0, {ROOT!r})
from paper_1208_3210_gb300 import lindhard as lh
lib = lh.load()
g = lh.make_grid(2, 16, 32, 1.0, quantity={quantity})
b = lh.make_band(kT={kT!r})
fake = ctypes.c_void_p(256)
st = lib.lindhard_imchi_noalloc(ctypes.byref(g), {'ctypes.byref(b)' if band else 'None'},
                                {'fake' if a_in else 'None'}, fake, None, None)
print(st)
print(lib.lindhard_last_error().decode())
"""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code.replace("nan", "float('nan')")], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    st, err = r.stdout.split("\n", 1)
    from paper_1208_3210_gb300 import lindhard as lh
    assert int(st) == lh.EINVAL
    assert msg in err


@pytest.mark.parametrize("kw,flags,msg", [
    (dict(), 1 | 16, "forward only"),                                   # with LINDHARD_PLAN_BACKWARD
    (dict(precision=2), 16, "energy-direct form takes"),                # FP64
    (dict(precision=1), 16, "energy-direct form takes"),                # tensor-core precision
    (dict(quantity=2), 16, "energy-direct form takes"),                 # finite temperature
    (dict(n_eps=2048), 16, "energy-direct form takes"),                 # n_eps > 1024
    (dict(n_eps=1024, n_omega=600), 16, "energy-direct form takes"),    # n_omega > 512
])
def test_energy_direct_plan_rejections_on_host(lib, kw, flags, msg):
    from paper_1208_3210_gb300 import lindhard as lh
    g = lh.make_grid(2, 64, kw.get("n_eps", 32), 1.0, kw.get("n_omega", 0), 0, kw.get("precision", 0),
                     kw.get("quantity", 0))
    h = ctypes.c_void_p()
    st = lib.lindhard_plan_create(ctypes.byref(g), 1, flags, ctypes.byref(h))
    assert st == lh.EUNSUPPORTED and not h.value
    assert msg in lib.lindhard_last_error().decode()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of lindhard_band, lindhard_grid and lindhard_sizes
    have the sizes and field offsets the C compiler gives the header's structs."""
    import subprocess
    from paper_1208_3210_gb300 import lindhard as lh
    fields = {"lindhard_band": (lh.Band, [f[0] for f in lh.Band._fields_]),
              "lindhard_grid": (lh.Grid, [f[0] for f in lh.Grid._fields_]),
              "lindhard_sizes": (lh.Sizes, [f[0] for f in lh.Sizes._fields_])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lindhard.h"', "int main(void) {"]
    for name, (_, names) in fields.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in names:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, (cls, names) in fields.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in names:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
