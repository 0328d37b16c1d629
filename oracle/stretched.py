"""Stretched tensor-product grids (Eq 4.18) and the collocated operators of
Sec. 3.2 (Eqs 3.20-3.22) on them -- the non-uniform counterpart of
``operators.py``, for the cavity's clustered grids.

Oracle code: test infrastructure only (imported by the tests, never by the
package).  Arrays here are interior arrays (no ghost layer), x the last axis;
an axis is described by its face coordinates.

Reading of Eq 4.18.  As printed, x~ = (1 + tanh(alpha (x - 1/2))) /
(2 tanh(alpha / 2)) does not map [0, 1] onto itself and does not tend to the
identity as alpha -> 0, which the text after it states.  The map used here,
x~ = (1 + tanh(alpha (x - 1/2)) / tanh(alpha / 2)) / 2, does both and differs
from the printed one by a constant, so the spacings (all the grid study uses)
are the same.  It is applied to the faces x = i / n; cell centres are the
midpoints of their faces (the centroid of a cell, the point the midpoint rule
of Eq 3.22 evaluates).
"""

import numpy as np
from scipy.optimize import brentq


def tanh_faces(n, alpha):
    """Face coordinates of Eq 4.18 on [0, 1]: n + 1 values, clustered at both
    ends for alpha > 0 (uniform for alpha = 0)."""
    s = np.arange(n + 1) / n
    if alpha == 0.0:
        return s
    return 0.5 * (1.0 + np.tanh(alpha * (s - 0.5)) / np.tanh(0.5 * alpha))


def spacing_ratio(n, alpha):
    dx = np.diff(tanh_faces(n, alpha))
    return float(dx.max() / dx.min())


def alpha_for_ratio(n, ratio):
    """alpha of Eq 4.18 whose largest spacing is ``ratio`` times its smallest
    (found numerically, as the text after Eq 4.18 describes)."""
    if ratio <= 1.0:
        return 0.0
    return brentq(lambda a: spacing_ratio(n, a) - ratio, 1e-6, 20.0, xtol=1e-14)


class Axis:
    """One direction of a tensor grid: faces xf (n + 1), centres xc (n, the
    face midpoints) and widths dx (n)."""

    def __init__(self, faces):
        self.xf = np.asarray(faces, dtype=float)
        self.n = len(self.xf) - 1
        self.xc = 0.5 * (self.xf[1:] + self.xf[:-1])
        self.dx = np.diff(self.xf)


def _along(a, axis, fn):
    """Apply a 1D operator ``fn`` along numpy axis ``axis`` of ``a``."""
    return np.moveaxis(fn(np.moveaxis(a, axis, -1)), -1, axis)


def interp_to_faces(phi, ax, axis=-1):
    """Eq 3.20 with n = 1 at the interior faces (n - 1 values): the linear
    interpolant of the two neighbouring centre values at the face."""
    def f(p):
        xl, xr, xfa = ax.xc[:-1], ax.xc[1:], ax.xf[1:-1]
        return ((xfa - xl) * p[..., 1:] + (xr - xfa) * p[..., :-1]) / (xr - xl)
    return _along(phi, axis, f)


def diff_to_faces(phi, ax, axis=-1):
    """Eq 3.21 with n = 1 at the interior faces: the centre difference over the
    centre distance."""
    return _along(phi, axis, lambda p: (p[..., 1:] - p[..., :-1]) / (ax.xc[1:] - ax.xc[:-1]))


def faces_diff_to_cells(q, ax, axis=-1):
    """Eq 3.21 with n = 1 at the centres from all n + 1 face values: the face
    difference over the cell width."""
    return _along(q, axis, lambda p: (p[..., 1:] - p[..., :-1]) / ax.dx)


def diff2(phi, ax, axis=-1):
    """Eq 3.21 with n = 2 at the centres 1 .. n - 2 (the neighbours' difference
    over their distance)."""
    return _along(phi, axis, lambda p: (p[..., 2:] - p[..., :-2]) / (ax.xc[2:] - ax.xc[:-2]))


def volumes(axes):
    """Cell volumes dV (the weights of Eq 3.22), x the last axis."""
    w = np.ones(())
    for d, ax in enumerate(axes):
        shp = [1] * len(axes)
        shp[len(axes) - 1 - d] = ax.n
        w = w * ax.dx.reshape(shp)
    return w


def integrate(phi, axes):
    """Eq 3.22: the midpoint rule with the cells' volumes."""
    return float(np.sum(phi * volumes(axes)))


def laplacian_neumann(P, axes):
    """The pressure operator sum_j delta_1(delta_1 P / delta_1 x_j) / delta_1 x_j
    (Eqs 3.9 and 3.24) with zero flux through every boundary face (the
    homogeneous Neumann condition of the solid and inflow sides)."""
    out = np.zeros_like(P)
    nd = len(axes)
    for d, ax in enumerate(axes):
        axis = nd - 1 - d
        g = diff_to_faces(P, ax, axis)
        pad = [(0, 0)] * nd
        pad[axis] = (1, 1)
        out = out + faces_diff_to_cells(np.pad(g, pad), ax, axis)
    return out


def solve_neumann(b, axes):
    """The zero-mean solution (volume-weighted mean) of laplacian_neumann(P) =
    b - mean(b), by a dense least-squares solve of the operator with the
    constant mode constrained (small grids only)."""
    shape = b.shape
    N = b.size
    A = np.zeros((N, N))
    e = np.zeros(N)
    for k in range(N):
        e[k] = 1.0
        A[:, k] = laplacian_neumann(e.reshape(shape), axes).ravel()
        e[k] = 0.0
    w = volumes(axes).ravel() * np.ones(N)
    rhs = b.ravel() - np.sum(b.ravel() * w) / np.sum(w)
    M = np.block([[A, w[:, None]], [w[None, :], np.zeros((1, 1))]])
    sol = np.linalg.solve(M, np.concatenate([rhs, [0.0]]))
    return sol[:N].reshape(shape)


def cell_divergence(F, axes):
    """delta_1 F_j / delta_1 x_j summed over directions (Eq 3.24): ``F[d]`` holds
    the n_d + 1 face values of direction d, boundary faces included."""
    nd = len(axes)
    return sum(faces_diff_to_cells(F[d], ax, nd - 1 - d) for d, ax in enumerate(axes))


def project(Fs, axes, drho_dt=None):
    """Eqs 3.23-3.24 on a closed box: P solves
    delta_1(delta_1 P / delta_1 x_j) / delta_1 x_j = delta_1 Fs_j / delta_1 x_j + d_t rho
    with zero flux through the boundary, and the returned faces are
    F_j = Fs_j - delta_1 P / delta_1 x_j (boundary faces kept).  Returns (F, P)."""
    nd = len(axes)
    rhs = cell_divergence(Fs, axes)
    if drho_dt is not None:
        rhs = rhs + drho_dt
    P = solve_neumann(rhs, axes)
    F = []
    for d, ax in enumerate(axes):
        axis = nd - 1 - d
        pad = [(0, 0)] * nd
        pad[axis] = (1, 1)
        F.append(Fs[d] - np.pad(diff_to_faces(P, ax, axis), pad))
    return F, P
