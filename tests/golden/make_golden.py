"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Calls only ``oracle`` (for arithmetic) and the seeded-input module (for the
parameters).  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1208_3210_gb300 import workloads as wl  # noqa: E402


def reduced_zone():
    w = wl.WORKLOADS["reduced_32x32x48"]
    b, g = dict(w["band"]), w["grid"]
    b["mu"] = oracle.solve_mu(b["kind"], b["t"], b["tp"], b["tpp"], b["gamma"], g["npz"], b["filling"])
    A = oracle.spectral(b, g)
    chi = oracle.imchi_full(A, g, g["q_extent"], g["n_omega"])
    np.savez_compressed(os.path.join(HERE, "reduced_32x32x48.npz"), imchi=chi, mu=np.float64(b["mu"]))


if __name__ == "__main__":
    reduced_zone()
