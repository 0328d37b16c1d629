"""Collocated-grid operators of Sec. 3.2 (Eqs 3.20-3.22) on a uniform grid or
on a tensor-product grid with arbitrary face coordinates (the tanh-stretched
grids of Eq 4.18).

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

On a stretched grid cell centres are the midpoints of their faces.  A ghost
cell sits where the boundary condition puts its value: mirrored about the end
face on a non-periodic side (so the mirror ghosts of Eqs 3.43-3.44 give the
boundary value and the zero gradient at the face), and one period away on a
periodic side (Eq 3.45).  The uniform grid keeps its own arithmetic (weights
1/2, spacing h) so that its results do not depend on the general path.
"""

import numpy as np


class Grid:
    """Cartesian grid on [0, L_0] x [0, L_1] (x [0, L_2]) with n_d cells:
    uniform, or with the face coordinates ``faces[d]`` (n_d + 1 values from 0
    to L_d) of each direction; ``periodic[d]`` places the ghost cells of a
    stretched grid."""

    def __init__(self, n, L, faces=None, periodic=None):
        self.dim = len(n)
        assert self.dim in (2, 3) and len(L) == self.dim
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.shape = tuple(self.n[d] + 2 for d in reversed(range(self.dim)))
        self.uniform = faces is None
        if self.uniform:
            self.h = tuple(self.L[d] / self.n[d] for d in range(self.dim))
            self.dV = float(np.prod(self.h))
            return
        self.h = None                          # no single spacing: fail loudly if used
        self.xf, self.xc, self.dx = [], [], []
        for d in range(self.dim):
            xf = np.asarray(faces[d], dtype=float)
            n_d = self.n[d]
            assert xf.shape == (n_d + 1,) and np.all(np.diff(xf) > 0)
            assert abs(xf[0]) < 1e-14 and abs(xf[-1] - self.L[d]) < 1e-12 * self.L[d]
            w = np.diff(xf)
            xc = np.empty(n_d + 2)
            dx = np.empty(n_d + 2)
            xc[1:-1] = 0.5 * (xf[1:] + xf[:-1])
            dx[1:-1] = w
            if periodic is not None and periodic[d]:
                xc[0], xc[-1] = xc[n_d] - self.L[d], xc[1] + self.L[d]
                dx[0], dx[-1] = w[-1], w[0]
            else:
                xc[0], xc[-1] = 2.0 * xf[0] - xc[1], 2.0 * xf[-1] - xc[n_d]
                dx[0], dx[-1] = w[0], w[-1]
            self.xf.append(xf)
            self.xc.append(xc)
            self.dx.append(dx)
        dV = np.ones(())
        for d in range(self.dim):
            dV = dV * self._along(d, self.dx[d][1:-1])
        self.dV = dV                           # interior cell volumes (Eq 3.22)

    def ax(self, d):
        """numpy axis of direction d (x is the last axis)."""
        return self.dim - 1 - d

    def _along(self, d, x):
        """1D array ``x`` shaped to broadcast along direction d."""
        shp = [1] * self.dim
        shp[self.ax(d)] = len(x)
        return np.asarray(x).reshape(shp)

    def zeros(self, dtype=float):
        return np.zeros(self.shape, dtype=dtype)

    def centres(self, d):
        """Cell-centre coordinate of direction d on the padded array (ghosts included)."""
        if self.uniform:
            x = (np.arange(self.n[d] + 2) - 0.5) * self.h[d]
        else:
            x = self.xc[d]
        return np.broadcast_to(self._along(d, x), self.shape)

    def padded_centres(self, d):
        """1D cell-centre coordinates of direction d, ghosts included."""
        if self.uniform:
            return (np.arange(self.n[d] + 2) - 0.5) * self.h[d]
        return self.xc[d]

    def volume(self):
        """Volume of the domain."""
        if self.uniform:
            return float(np.prod([self.n[d] * self.h[d] for d in range(self.dim)]))
        return float(np.sum(self.dV))

    def mean(self, a):
        """Mean of an interior array: the plain mean on a uniform grid, the
        volume-weighted one (Eq 3.22) otherwise."""
        if self.uniform:
            return a.mean()
        return float(np.sum(a * self.dV)) / float(np.sum(self.dV))

    def face_area(self, j):
        """Area of each j-interface of one end layer: a scalar on a uniform
        grid, an array of the end layer's shape otherwise."""
        if self.uniform:
            return self.dV / self.h[j]
        a = np.ones(())
        for d in range(self.dim):
            if d != j:
                a = a * self._along(d, self.dx[d][1:-1])
        return np.squeeze(a, axis=self.ax(j))

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


def dtype_of(*arrays):
    """float64, or complex128 when any argument is complex (the oracle then
    carries a complex-step perturbation through the step)."""
    return np.result_type(np.float64, *[np.asarray(a).dtype for a in arrays])


def pad(interior_values, g):
    """New padded array with the given interior values and zero ghosts."""
    a = g.zeros(dtype_of(interior_values))
    V(a, g)[...] = interior_values
    return a


# ---------------------------------------------------------------------------
# Eq 3.20 / Eq 3.21 with n = 1 (odd operators), centre -> interface.
# On a uniform grid the weights of Eq 3.20 are 1/2, 1/2.
# ---------------------------------------------------------------------------
def centres_to_faces(lo, hi, g, j):
    """Eq 3.20 with n = 1 at every j-interface from the values ``lo`` and
    ``hi`` at the centres on either side of it (face views of the cells
    f - 1 and f along j)."""
    if g.uniform:
        return 0.5 * (lo + hi)
    xl, xr = g._along(j, g.xc[j][:-1]), g._along(j, g.xc[j][1:])
    xf = g._along(j, g.xf[j])
    return ((xf - xl) * hi + (xr - xf) * lo) / (xr - xl)


def interp_to_faces(phi, g, j):
    """bar(phi)^{1x_j} on every j-interface (needs the ghost cells along j)."""
    return centres_to_faces(V(phi, g, off=g.unit(j, -1), face=j), V(phi, g, face=j), g, j)


def diff_to_faces(phi, g, j):
    """delta_1 phi / delta_1 x_j on every j-interface."""
    lo, hi = V(phi, g, off=g.unit(j, -1), face=j), V(phi, g, face=j)
    if g.uniform:
        return (hi - lo) / g.h[j]
    return (hi - lo) / g._along(j, g.xc[j][1:] - g.xc[j][:-1])


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
    if g.uniform:
        return 0.5 * (lo + hi)
    xl, xr = g._along(j, g.xf[j][:-1]), g._along(j, g.xf[j][1:])
    xc = g._along(j, g.xc[j][1:-1])
    return ((xc - xl) * hi + (xr - xc) * lo) / (xr - xl)


def faces_diff_to_cells(fv, g, j):
    """delta_1 (.) / delta_1 x_j at the cell centres from the two j-interfaces."""
    lo, hi = _lo_hi(fv, g, j)
    if g.uniform:
        return (hi - lo) / g.h[j]
    return (hi - lo) / g._along(j, g.dx[j][1:-1])


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
    diff = V(phi, g, off=plus, face=face) - V(phi, g, off=minus, face=face)
    if g.uniform:
        return diff / (2.0 * g.h[j])
    # along j the selected cells are the interior ones (the offset and the face
    # selection of every caller are along other directions)
    assert base[j] == 0 and face != j
    return diff / g._along(j, g.xc[j][2:] - g.xc[j][:-2])


# ---------------------------------------------------------------------------
# Eq 3.22: midpoint-rule integration over the interior cells.
# ---------------------------------------------------------------------------
def integrate(phi_interior, g):
    r = np.sum(phi_interior) * g.dV if g.uniform else np.sum(phi_interior * g.dV)
    return complex(r) if np.iscomplexobj(r) else float(r)
