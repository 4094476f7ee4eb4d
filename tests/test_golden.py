"""Stored expected values: the reduced-zone fixture is reproduced by the oracle,
and the tight-binding stand-in spans the band range the paper quotes."""
import json
import math
import os

import numpy as np

import oracle
from paper_1208_3210_gb300 import workloads as wl

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_reduced_zone_fixture_reproduced():
    w = wl.WORKLOADS["reduced_32x32x48"]
    b, g = dict(w["band"]), w["grid"]
    ref = np.load(os.path.join(HERE, "reduced_32x32x48.npz"))
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], g["npz"], b["filling"])
    assert b["mu"] == float(ref["mu"])
    chi = oracle.imchi_full(oracle.spectral(b, g), g, g["q_extent"], g["n_omega"])
    np.testing.assert_allclose(chi, ref["imchi"], rtol=0, atol=1e-14 * np.abs(ref["imchi"]).max())


def test_stand_in_band_range_near_paper():
    # Sec. 3: the NCCO CuO2 band spans about -1.4 .. 1.9 eV.  The stand-in's
    # extremes sit at Gamma and M; they agree to within 0.15 eV.
    paper = json.load(open(os.path.join(HERE, "paper_values.json")))["cuo2_band_range_eV"]["value"]
    b = wl.BAND_TB
    lo = oracle.band(0, b["t"], b["tp"], b["tpp"], 0.0, 0.0)
    hi = oracle.band(0, b["t"], b["tp"], b["tpp"], math.pi, math.pi)
    assert abs(lo - paper[0]) < 0.15 and abs(hi - paper[1]) < 0.15
