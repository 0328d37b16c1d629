"""Heat-release objective of the flame sheet (test infrastructure: only tests,
the smoke check and the benchmark's CPU baseline use this package).

The paper defines no objective; this is the heat-release rate of the
Burke-Schumann flame sheet with unit Lewis numbers.  With T = Q/(S+1) (F_eps(Z)
+ H) (Eq 3.42) and H, Z both obeying the same diffusion operator, the source
that the regularised sheet puts into the temperature equation is

    omega = -Q/(S+1) F_eps''(Z) kappa |grad Z|^2 / Pe,

F_eps'' the curvature of the regularised F (Eq 3.41; the level shift after
Eq 3.41 does not change it).  The objective of a run is the time integral over
the domain, J = sum_{n=1..N} dt sum_cells omega(level n) dV (midpoint rule,
Eq 3.22), with grad Z by the centred difference delta_2 (Eq 3.21, n = 2).

Pinned (tests/test_oracle_pins.py): F_eps'' against second differences of
Eq 3.41 itself, omega against -d^2T/dZ^2 kappa |grad Z|^2 / Pe of the state
relation, delta_2 of a linear field.

The oracle's derivative of J is taken by the complex step (Squire and Trapp,
SIAM Review 40, 1998): for a map that is real-analytic in its input,
Im J(c + i h e) / h is dJ/dc . e up to O(h^2) with no subtraction, so any
h far below the rounding scale gives it to rounding.  Every operation of the
step on the path from the burner profile to J is analytic (products, sums,
powers of T, log cosh and tanh of Z, the linear Poisson solve), and the
oracle's arrays take the dtype of their values, so the perturbation travels
through the step.  Pinned against central differences of J.
"""

import numpy as np

from .operators import V, diff2, integrate


def F_eps_second_derivative(Z, S, k):
    """d^2 F_eps / dZ^2 of Eq 3.41: -(S+1) k / (2 S cosh^2(k (Z - 1)))."""
    x = k * (Z - 1.0)
    return -(S + 1.0) * k / (2.0 * S * np.cosh(x) ** 2)


def heat_release_rate(pb, Z, kappa):
    """omega on the interior cells from padded Z (ghosts filled) and kappa."""
    g, fp = pb.g, pb.fp
    grad2 = sum(diff2(Z, g, j) ** 2 for j in range(g.dim))
    Fpp = F_eps_second_derivative(V(Z, g), fp["S"], fp["k"])
    return -fp["Q"] / (fp["S"] + 1.0) * Fpp * V(kappa, g) * grad2 / pb.Pe


def heat_release(pb, st):
    """sum over the interior cells of omega dV at the level held by st."""
    return integrate(heat_release_rate(pb, st.Z, st.kappa), pb.g)


def objective(pb, st, nsteps, advance):
    """J = sum_{n=1..nsteps} dt * heat_release(level n), stepping st with
    ``advance`` (the oracle's one-step function)."""
    dt = pb.prm["dt"]
    J = 0.0
    for _ in range(nsteps):
        st = advance(pb, st)
        J += dt * heat_release(pb, st)
    return J


def complex_step_derivative(J, c, e, h=1e-20):
    """dJ/dc . e at c for a real-analytic objective J evaluated on complex
    input: Im J(c + i h e) / h."""
    c = np.asarray(c, dtype=float)
    e = np.asarray(e, dtype=float)
    return float(np.imag(J(c + 1j * h * e))) / h
