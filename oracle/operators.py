"""Collocated-grid operators of Sec. 3.2 (Eqs 3.20-3.22), uniform spacing.

Layout (oracle-only convention): a cell field is a numpy array of shape
``(n_z+2, n_y+2, n_x+2)`` in 3D or ``(n_y+2, n_x+2)`` in 2D -- x is the last
(fastest) axis -- with one ghost layer on each side (padded index 0 and n_d+1
are ghosts, interior cells are 1..n_d; the ghost convention of Eq 3.45).

Interface data along direction j (Fig. 1: the auxiliary flux F_j lives on the
j-interfaces) is held as a "face view": an array whose j-extent is n_j+1
(interface between padded cells f-1 and f, f = 1..n_j+1) and whose other
extents are the interior cells.  A padded face array stores the same values at
padded indices f = 1..n_j+1 along j.

Directions are numbered d = 0 (x_1), 1 (x_2), 2 (x_3).
"""

import numpy as np


class Grid:
    """Uniform Cartesian grid on [0, L_0] x [0, L_1] (x [0, L_2]) with n_d cells."""

    def __init__(self, n, L):
        self.dim = len(n)
        assert self.dim in (2, 3) and len(L) == self.dim
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.h = tuple(self.L[d] / self.n[d] for d in range(self.dim))
        self.dV = float(np.prod(self.h))
        self.shape = tuple(self.n[d] + 2 for d in reversed(range(self.dim)))

    def ax(self, d):
        """numpy axis of direction d (x is the last axis)."""
        return self.dim - 1 - d

    def zeros(self):
        return np.zeros(self.shape)

    def centres(self, d):
        """Cell-centre coordinate of direction d on the padded array (ghosts included)."""
        x = (np.arange(self.n[d] + 2) - 0.5) * self.h[d]
        shp = [1] * self.dim
        shp[self.ax(d)] = self.n[d] + 2
        return np.broadcast_to(x.reshape(shp), self.shape)

    def unit(self, d, k=1):
        off = [0] * self.dim
        off[d] = k
        return off


def V(a, g, off=None, face=None):
    """View of padded array ``a`` over the interior cells -- or, with ``face=j``,
    over padded indices 1..n_j+1 along j and the interior along the other
    directions -- shifted by the integer offset vector ``off``."""
    sl = [None] * g.dim
    for d in range(g.dim):
        lo, hi = 1, g.n[d] + 1
        if face == d:
            hi = g.n[d] + 2
        o = off[d] if off is not None else 0
        sl[g.ax(d)] = slice(lo + o, hi + o)
    return a[tuple(sl)]


def pad(interior_values, g):
    """New padded array with the given interior values and zero ghosts."""
    a = g.zeros()
    V(a, g)[...] = interior_values
    return a


# ---------------------------------------------------------------------------
# Eq 3.20 / Eq 3.21 with n = 1 (odd operators), centre -> interface.
# On a uniform grid the weights of Eq 3.20 are 1/2, 1/2.
# ---------------------------------------------------------------------------
def interp_to_faces(phi, g, j):
    """bar(phi)^{1x_j} on every j-interface (needs the ghost cells along j)."""
    return 0.5 * (V(phi, g, off=g.unit(j, -1), face=j) + V(phi, g, face=j))


def diff_to_faces(phi, g, j):
    """delta_1 phi / delta_1 x_j on every j-interface."""
    return (V(phi, g, face=j) - V(phi, g, off=g.unit(j, -1), face=j)) / g.h[j]


# Interface -> centre (odd operators applied to face views).
def _lo_hi(fv, g, j):
    a = g.ax(j)
    n = g.n[j]
    lo = [slice(None)] * g.dim
    hi = [slice(None)] * g.dim
    lo[a] = slice(0, n)
    hi[a] = slice(1, n + 1)
    return fv[tuple(lo)], fv[tuple(hi)]


def faces_interp_to_cells(fv, g, j):
    """bar(.)^{1x_j} at the cell centres from the two j-interfaces of each cell."""
    lo, hi = _lo_hi(fv, g, j)
    return 0.5 * (lo + hi)


def faces_diff_to_cells(fv, g, j):
    """delta_1 (.) / delta_1 x_j at the cell centres from the two j-interfaces."""
    lo, hi = _lo_hi(fv, g, j)
    return (hi - lo) / g.h[j]


# ---------------------------------------------------------------------------
# Eq 3.21 with n = 2 (even operator), centre -> centre.
# ---------------------------------------------------------------------------
def diff2(phi, g, j, off=None, face=None):
    """delta_2 phi / delta_2 x_j at the cells selected by ``V(.., off, face)``."""
    base = list(off) if off is not None else [0] * g.dim
    plus = list(base)
    plus[j] += 1
    minus = list(base)
    minus[j] -= 1
    return (V(phi, g, off=plus, face=face) - V(phi, g, off=minus, face=face)) / (2.0 * g.h[j])


# ---------------------------------------------------------------------------
# Eq 3.22: midpoint-rule integration over the interior cells.
# ---------------------------------------------------------------------------
def integrate(phi_interior, g):
    return float(np.sum(phi_interior) * g.dV)
