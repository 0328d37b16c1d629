"""Flame-sheet (Burke-Schumann) state relation with the regularisation of Sec. 3.5.

Parameters (paper notation):
  S   generalised stoichiometric coefficient (Eq 2.34);
  Q   generalised heat release (Eq 2.36);
  k   regularisation sharpness, k = ln((1-tol)/tol) / (2 eps) (text after Eq 3.34);
  sigma = 0.7 transport exponent (Eq 2.50).

Reading of the conventional configuration inputs: the stoichiometric conventional mixture fraction Z_st maps to S = 1/Z_st - 1 (the
rescaled flame sits at Z = 1, Eq 2.34), and the adiabatic flame-to-ambient
temperature ratio maps to Q through T_flame = 1 + Q/(S+1) (Eq 3.37 at Z = 1 with
H = H_inf = 1 + (S+1)/Q).
"""

import numpy as np


def derived_parameters(Z_st, density_ratio, eps, tol, Le_F=1.0, Le_O=1.0, gamma=1.4):
    S = 1.0 / Z_st - 1.0
    Q = (density_ratio - 1.0) * (S + 1.0)
    k = np.log((1.0 - tol) / tol) / (2.0 * eps)                  # text after Eq 3.34
    N_F = (1.0 - Le_F) / (S * Le_F)                              # text after Eq 2.37
    N_O = (Le_O - 1.0) / Le_O
    zeta = (S + 1.0) * (gamma - 1.0) / (gamma * Q)               # text after Eq 2.45
    return dict(S=S, Q=Q, k=k, N_F=N_F, N_O=N_O, zeta=zeta, Le_F=Le_F, Le_O=Le_O)


def Nprime_eps(Z, fp):
    """N' of the p0 equation (Eq 2.39), N'_F = -1/S, N'_O = 1, regularised with
    the same theta_eps as N (Eq 3.35b)."""
    return (-1.0 / fp["S"] - 1.0) * theta_eps(Z, fp["k"]) + 1.0


def theta_eps(Z, k):
    """Regularised Heaviside around the flame Z = 1 (Eq 3.34)."""
    return 0.5 * (1.0 + np.tanh(k * (Z - 1.0)))


def lewis_eps(Z, fp):
    """Le_eps(Z) (Eq 3.35a)."""
    return (fp["Le_F"] - fp["Le_O"]) * theta_eps(Z, fp["k"]) + fp["Le_O"]


def N_eps(Z, fp):
    """N_eps(Z) (Eq 3.35b)."""
    return (fp["N_F"] - fp["N_O"]) * theta_eps(Z, fp["k"]) + fp["N_O"]


def F_sharp(Z, S):
    """Unregularised F(Z) (Eq 3.37)."""
    return np.where(Z > 1.0, (1.0 - Z) / S, Z - 1.0)


def F_eps_unshifted(Z, S, k):
    """Closed form of the integral of the regularised slope (Eq 3.41)."""
    x = k * (Z - 1.0)
    return ((-(S + 1.0) * np.log(np.cosh(x)) / k) + (S - 1.0) * (Z - 1.0)) / (2.0 * S)


def F_eps(Z, S, k):
    """Eq 3.41 translated to the levels of F far from the flame.

    For |k(Z-1)| -> infinity, ln cosh x = |x| - ln 2 + o(1), so Eq 3.41 exceeds
    Eq 3.37 by (S+1) ln 2 / (2 S k) on both sides of the flame; subtracting this
    constant is the translation the text after Eq 3.41 asks for (same shift on
    both sides, so the slopes of Eq 3.39 are untouched)."""
    return F_eps_unshifted(Z, S, k) - (S + 1.0) * np.log(2.0) / (2.0 * S * k)


def temperature(Z, H, fp):
    """T_eps = Q/(S+1) [F_eps(Z) + H]  (Eq 3.42)."""
    return fp["Q"] / (fp["S"] + 1.0) * (F_eps(Z, fp["S"], fp["k"]) + H)


def kappa(T, sigma, transport=0, C=0.0):
    """kappa = mu = rho D as a function of T: the power law T^sigma (Eq 2.50),
    or with transport = 1 Sutherland's law T^(3/2) (1 + C) / (T + C) (Eq 4.12),
    C the Sutherland constant over the reference temperature."""
    if transport == 1:
        return T ** 1.5 * (1.0 + C) / (T + C)
    return T ** sigma


def density(p0, T):
    """Ideal-gas law p0 = rho T (Eq 2.49)."""
    return p0 / T


def closed_p0(mass, T_interior, dV):
    """Enclosed system: p0 * int(1/T) dV = m (Eq 2.40, midpoint rule Eq 3.22);
    dV is the cell volume, or an array of them on a stretched grid."""
    if np.ndim(dV) == 0:
        return mass / (np.sum(1.0 / T_interior) * dV)
    return mass / np.sum(dV / T_interior)
