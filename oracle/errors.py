"""O12: the accuracy measures of Sec. 3.2 / Sec. 4.

Relative errors of integral quantities (Fig. 4, 5), and the maximum and
root-mean-square relative errors of S11(theta) over the scattering angles
(Figs. 6, 7).  Reading for the paper's silent points: the RMS is uniform over
the supplied angles (0..180 degrees in 1-degree steps, both ends included).
"""
import numpy as np


def rel_error(value, exact):
    return abs(value - exact) / abs(exact)


def s11_errors(s11, s11_exact):
    """(max, rms) of |S11 - S11_exact| / S11_exact over the angles."""
    e = np.abs(np.asarray(s11) - np.asarray(s11_exact)) / np.abs(np.asarray(s11_exact))
    return float(np.max(e)), float(np.sqrt(np.mean(e * e)))
