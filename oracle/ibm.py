"""Mass-flux immersed boundary (Sec. 3.4): shifted mask chi, targets v_ib, Z_ib,
H_ib, and mass source S_m.

* Shifted characteristic function (text after Eq 3.30, Iwakami): the body is
  extended into the fluid by the Brinkman length s = Da_ib^(1/2); a cell has
  chi = 1 iff the signed distance of its centre to the body is <= s.
* Radial ejection (Eqs 4.19-4.20): for a circle (2D) / sphere (3D) of radius R,
  v_ib = U_b (x - c)/r and S_m = chi (dim-1) rho_b U_b / r, which is the
  divergence of rho_b v_ib (Eq 4.19 is the 2D case).
* Slot burner (rectangular body ejecting through its top face, +x_2): the
  profile U(x_1) = U_b [1 - ((x_1 - c_1)/(a_1 + s))^2]_+ times an optional
  piecewise-linear modulation sampled uniformly across the shifted width;
  v_ib = (0, U(x_1) (x_2 - y_lo)/(y_hi - y_lo)) with y_lo, y_hi the shifted
  bottom and top of the body; S_m = rho_b U(x_1)/(n_col dx_2) on the n_col masked
  cells of each column, so that the discrete integral of S_m (Eq 3.22) equals the
  prescribed ejected mass flow sum_i rho_b U(x_1,i) dx_1 exactly.
"""

import numpy as np

from .operators import V

NONE, SLOT, SPHERE = 0, 1, 2


def build(g, geo):
    """Return dict(chi (padded, 0/1 float), vib (list of padded arrays),
    Sm (interior), Z_ib, H_ib, Da_ib) or None when there is no body."""
    if geo is None or geo.get("kind", NONE) == NONE:
        return None
    dim = g.dim
    s = np.sqrt(geo["Da_ib"])
    c = [float(geo["center"][d]) for d in range(dim)]
    x = [g.centres(d) for d in range(dim)]
    rho_b = float(geo["rho_b"])
    U_b = float(geo["U_b"])
    vib = [g.zeros() for _ in range(dim)]
    Sm_full = g.zeros()

    if geo["kind"] == SPHERE:
        R = float(geo["radius"])
        r = np.sqrt(sum((x[d] - c[d]) ** 2 for d in range(dim)))
        chi = (r - R <= s).astype(float)                          # shifted mask
        rs = np.where(r > 0.0, r, 1.0)
        for d in range(dim):
            vib[d] = chi * U_b * (x[d] - c[d]) / rs                # Eq 4.20
        Sm_full = chi * (dim - 1) * rho_b * U_b / rs               # Eq 4.19 (and its 3D form)
    elif geo["kind"] == SLOT:
        a = [float(geo["half"][d]) for d in range(dim)]
        q = [np.abs(x[d] - c[d]) - a[d] for d in range(dim)]
        outside = np.sqrt(sum(np.maximum(q[d], 0.0) ** 2 for d in range(dim)))
        inside = np.minimum(np.max(np.stack(q), axis=0), 0.0)
        sd = outside + inside                                      # signed distance to the box
        chi = (sd <= s).astype(float)
        # ejection profile across the transverse directions (all but x_2)
        prof = np.ones(g.shape)
        for d in range(dim):
            if d == 1:
                continue
            prof = prof * (1.0 - ((x[d] - c[d]) / (a[d] + s)) ** 2)
        prof = np.maximum(prof, 0.0)
        samples = geo.get("profile")
        if samples is not None and len(samples) > 0:
            samples = np.asarray(samples, dtype=float)
            lo, hi = c[0] - a[0] - s, c[0] + a[0] + s
            xs = np.linspace(lo, hi, len(samples))
            prof = prof * np.interp(x[0], xs, samples)
        U = U_b * prof
        y_lo, y_hi = c[1] - a[1] - s, c[1] + a[1] + s
        vib[1] = chi * U * (x[1] - y_lo) / (y_hi - y_lo)
        # number of masked interior cells per column (fixed x_1, x_3)
        chi_int = V(chi, g)
        n_col = np.sum(chi_int, axis=g.ax(1), keepdims=True)
        n_col_safe = np.where(n_col > 0, n_col, 1.0)
        Sm_int = chi_int * rho_b * V(U, g) / (n_col_safe * g.h[1])
        Sm_full = g.zeros()
        V(Sm_full, g)[...] = Sm_int
    else:
        raise ValueError("unknown body kind")

    return dict(chi=chi, vib=vib, Sm=V(Sm_full, g).copy(), Z_ib=float(geo["Z_ib"]),
                H_ib=float(geo["H_ib"]), Da_ib=float(geo["Da_ib"]))
