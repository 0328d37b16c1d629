"""Ghost-cell boundary conditions (Sec. 3.6, Eqs 3.43-3.46) and the boundary
mass fluxes of the projection (Sec. 3.3).

Boundary kinds of a domain side:
  PERIODIC  Eq 3.45 (both sides of the direction must be periodic);
  INFLOW    Dirichlet v = v_in, Z = Z_in, H = H_in (Eq 3.43); known mass flux rho_in v_in;
  OUTFLOW   zero normal gradient of v, Z, H (Eq 3.44, Phi = 0); mass flux extrapolated
            from the adjacent cell and shifted uniformly so that global mass is
            conserved (text after Eq 4.22);
  WALL      no-slip v = 0 (Eq 3.43), zero-gradient Z, H (Eq 3.44); zero mass flux;
  SLIP      symmetry plane: normal velocity 0 (Eq 3.43), tangential velocity and
            Z, H zero-gradient (Eq 3.44), zero mass flux (Eqs 4.22a-b).
  WALL_T    isothermal no-slip wall (the heated and cooled walls of Eq 4.16):
            v = 0, Dirichlet Z = Z_in (the inflow value, air) and H = H_wall of
            that side (Eq 3.43), so kappa takes the wall state's value; zero
            mass flux.
An INFLOW face whose adjacent interior cell is inside the immersed body mask is
a WALL face (the burner foot closes the inlet under it).
"""

import numpy as np

PERIODIC, INFLOW, OUTFLOW, WALL, SLIP, WALL_T = 0, 1, 2, 3, 4, 5


def _slab(a, g, d, idx):
    """Full padded slab of ``a`` at padded index ``idx`` along direction d."""
    sl = [slice(None)] * g.dim
    sl[g.ax(d)] = idx
    return a[tuple(sl)]


def _layers(g, d, side):
    """(ghost, first, second, third) padded indices for a side of direction d."""
    n = g.n[d]
    return (0, 1, 2, 3) if side == 0 else (n + 1, n, n - 1, n - 2)


class Boundary:
    """Per-face boundary kinds (a full padded slab per side) plus inflow data."""

    def __init__(self, g, bc, inflow_v, inflow_Z, inflow_H, chi=None, wall_H=None):
        self.g = g
        # Dirichlet H of each side's isothermal wall, [d][side]
        self.wall_H = [[float(wall_H[d][s]) if wall_H is not None else 0.0 for s in (0, 1)]
                       for d in range(g.dim)]
        self.bc = [tuple(bc[d]) for d in range(g.dim)]
        self.inflow_v = [float(inflow_v[d]) for d in range(g.dim)]
        self.inflow_Z = float(inflow_Z)
        self.inflow_H = float(inflow_H)
        self.kinds = {}
        for d in range(g.dim):
            lo, hi = self.bc[d]
            assert (lo == PERIODIC) == (hi == PERIODIC), "periodic must pair"
            for side in (0, 1):
                kind = self.bc[d][side]
                shp = _slab(g.zeros(), g, d, 0).shape
                arr = np.full(shp, kind, dtype=np.int64)
                if kind == INFLOW and chi is not None:
                    first = _layers(g, d, side)[1]
                    arr[_slab(chi, g, d, first) > 0] = WALL
                self.kinds[(d, side)] = arr

    def periodic(self, d):
        return self.bc[d][0] == PERIODIC

    # ------------------------------------------------------------------
    def fill(self, phi, what, comp=None, kappa_in=None, kappa_wall=None):
        """Fill all ghost cells of ``phi`` in place.

        ``what`` is "Z", "H", "kappa" or "v" (then ``comp`` is the velocity
        component).  For "kappa" the Dirichlet value is ``kappa_in``, the
        transport coefficient of the inflow state, so the interface value of kappa
        on an inflow side is kappa_in (Eq 3.43 applied to kappa); other sides take
        its zero-gradient ghost (Eq 3.44), and an isothermal wall's side the
        transport coefficient of the wall state, kappa_wall[d][side].
        Directions are filled in order 0, 1, 2 over full padded slabs, so edge and
        corner ghosts end up consistent with every side they touch."""
        g = self.g
        for d in range(g.dim):
            n = g.n[d]
            if self.periodic(d):                                    # Eq 3.45
                _slab(phi, g, d, 0)[...] = _slab(phi, g, d, n)
                _slab(phi, g, d, n + 1)[...] = _slab(phi, g, d, 1)
                continue
            for side in (0, 1):
                ghost, first = _layers(g, d, side)[:2]
                a1 = _slab(phi, g, d, first)
                kind = self.kinds[(d, side)]
                if what == "Z":
                    dirichlet = self.inflow_Z
                elif what == "H":
                    dirichlet = self.inflow_H
                elif what == "kappa":
                    dirichlet = kappa_in if kappa_in is not None else 0.0   # no inflow side
                else:
                    dirichlet = self.inflow_v[comp]
                mirror_in = 2.0 * dirichlet - a1                     # Eq 3.43 (Phi = inflow)
                mirror_zero = -a1                                    # Eq 3.43 (Phi = 0)
                zero_grad = a1                                       # Eq 3.44 (Phi = 0)
                if what == "v":
                    wall = mirror_zero
                    slip = mirror_zero if comp == d else zero_grad
                    wall_t = mirror_zero
                else:
                    wall = zero_grad
                    slip = zero_grad
                    if what == "Z":
                        wall_t = mirror_in
                    elif what == "H":
                        wall_t = 2.0 * self.wall_H[d][side] - a1
                    else:
                        kw = kappa_wall[d][side] if kappa_wall is not None else 0.0
                        wall_t = 2.0 * kw - a1
                out = np.select(
                    [kind == INFLOW, kind == OUTFLOW, kind == WALL, kind == SLIP, kind == WALL_T],
                    [mirror_in, zero_grad, wall, slip, wall_t])
                _slab(phi, g, d, ghost)[...] = out

    def fill_pressure(self, P):
        """Ghost cells of P: periodic copy (Eq 3.45) or quadratic extrapolation
        from the first three interior cells (Eqs 3.27-3.28)."""
        g = self.g
        for d in range(g.dim):
            n = g.n[d]
            if self.periodic(d):
                _slab(P, g, d, 0)[...] = _slab(P, g, d, n)
                _slab(P, g, d, n + 1)[...] = _slab(P, g, d, 1)
                continue
            for side in (0, 1):
                i0, i1, i2, i3 = _layers(g, d, side)
                if g.uniform:
                    x0, x1, x2, x3 = [(i - 0.5) * g.h[d] for i in (i0, i1, i2, i3)]
                else:                                                # stretched: the centres
                    x0, x1, x2, x3 = [g.xc[d][i] for i in (i0, i1, i2, i3)]
                A = (x2 - x0) * (x3 - x0) / ((x2 - x1) * (x3 - x1))
                B = (x1 - x0) * (x3 - x0) / ((x1 - x2) * (x3 - x2))
                C = (x1 - x0) * (x2 - x0) / ((x1 - x3) * (x2 - x3))
                _slab(P, g, d, i0)[...] = (A * _slab(P, g, d, i1) + B * _slab(P, g, d, i2)
                                           + C * _slab(P, g, d, i3))

    # ------------------------------------------------------------------
    def face_kind_view(self, d, side):
        """Boundary kind restricted to the interior range of the other directions
        (the shape of one end layer of a d-face view)."""
        g = self.g
        arr = self.kinds[(d, side)]
        sl = []
        for dd in reversed(range(g.dim)):
            if dd == d:
                continue
            sl.append(slice(1, g.n[dd] + 1))
        return arr[tuple(sl)]


def face_end(fv, g, d, side):
    """The boundary layer (first or last interface) of a d-face view."""
    sl = [slice(None)] * g.dim
    sl[g.ax(d)] = 0 if side == 0 else g.n[d]
    return fv[tuple(sl)]


def cell_end(a_interior, g, d, side):
    """First or last interior layer of an interior-shaped array along d."""
    sl = [slice(None)] * g.dim
    sl[g.ax(d)] = 0 if side == 0 else g.n[d] - 1
    return a_interior[tuple(sl)]
