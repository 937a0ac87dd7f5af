"""Writes mie_spheres.json: Mie-series Q_ext, Q_sca, <cos theta> and S11 at
0, 1, ..., 180 degrees for the homogeneous spheres of the workloads, from the
oracle's Mie code alone (oracle/mie.py, Bohren-Huffman formulation).  The
benchmark reads the file to state the DDA error against Mie (Sec. 3.1:
relative Q_ext error, maximum and RMS relative S11 error over the angles)
without running the oracle; tests/test_oracle_scatter_mie.py checks that the
file still equals what the oracle computes.

Run from the repository root:  python tests/golden/make_mie_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import mie  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mie_spheres.json")

# (size parameter x, real refractive index m): x = 3 m = 1.5 (16^3 sphere),
# x = 40 m = 1.05 (134^3), x = 20 m = 2 (128^3), x = 40 m = 2 (256^3),
# x = 160 m = 1.05 (536^3)
SPHERES = [(3.0, 1.5), (40.0, 1.05), (20.0, 2.0), (40.0, 2.0), (160.0, 1.05)]


def cases():
    th = np.linspace(0.0, 180.0, 181)
    out = []
    for x, m in SPHERES:
        qe, qs, _, g = mie.efficiencies(x, m)
        out.append({"x": x, "m": m, "qext": float(qe), "qsca": float(qs), "g": float(g),
                    "s11": [float(v) for v in mie.s11(x, m, th)]})
    return out


def main():
    doc = {"note": "Mie series of oracle/mie.py (Bohren-Huffman formulation, the Mie code the "
                   "paper compares the DDA with in Sec. 3.1); S11 at theta = 0, 1, ..., 180 "
                   "degrees, incident intensity 1, S11 = (|S1|^2 + |S2|^2) / 2.",
           "theta_deg": [float(t) for t in np.linspace(0.0, 180.0, 181)],
           "spheres": cases()}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
