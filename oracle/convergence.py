"""Verification formulas of Sec. 4.1."""

import numpy as np


def observed_order(E_coarse, E_fine, ratio):
    """b = ln(E_m / E_{m+1}) / ln(delta)  (Eq 4.1)."""
    return float(np.log(E_coarse / E_fine) / np.log(ratio))


def richardson_order(f_m, f_m1, f_m2, ratio):
    """b = ln((f_m - f_{m+1}) / (f_{m+1} - f_{m+2})) / ln(delta), three grid levels
    with a constant refinement ratio and no exact solution (Eq 4.2)."""
    return float(np.log((f_m - f_m1) / (f_m1 - f_m2)) / np.log(ratio))


def gci(f_m, f_m1, ratio, order, Fs=1.25):
    """Grid convergence index of the finer grid (Eq 4.3), safety factor 1.25."""
    eps = (f_m - f_m1) / f_m1
    return float(Fs * abs(eps) / (ratio ** order - 1.0))
