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
* Body given by surface markers (the marker form of the immersed boundary,
  Sec. 3.4): marker m carries its position x_m, unit outward normal n_m, normal
  ejection speed U_m and surface element A_m (length in 2D, area in 3D).  A
  cell centre p is matched with its nearest marker (least |p - x_m|^2, the
  lowest index on a tie); its signed distance to the body is the normal
  offset (p - x_m).n_m, so chi = 1 iff that offset is <= s; v_ib = U_m n_m
  there (outward normal ejection, the radial form of Eq 4.20 when the markers
  lie on a sphere).  Cells outside the markers' bounding box widened by 2s
  are outside the shifted body.  The ejected flow rho_b U_m A_m of each marker
  is spread uniformly over the N_m masked interior cells matched with it,
  S_m = rho_b U_m A_m / (N_m dV), so the discrete integral of S_m equals the
  total sum_m rho_b U_m A_m exactly; every marker needs N_m >= 1 (markers no
  denser than the cells).
* Coaxial cylinders (the Taylor-Couette flow of Sec. 4.2.3), axis along x_3
  through the centre: the inner cylinder r <= R_1 turns rigidly with surface
  speed U_b (counter-clockwise about +x_3), the outer body r >= R_2 is at
  rest, the fluid fills the gap.  With r the distance in the x_1-x_2 plane,
  each solid is extended into the gap by s: chi = 1 iff r - R_1 <= s or
  R_2 - r <= s; v_ib = (U_b / R_1)(-(x_2 - c_2), x_1 - c_1) in the inner
  body, 0 in the outer; no mass source.  r is formed with explicitly
  rounded squares and sum (the mask is an integer decision).
"""

import numpy as np

from .operators import V

NONE, SLOT, SPHERE, MARKERS, COUETTE = 0, 1, 2, 3, 4


def nearest_markers(pts, X):
    """Index of the nearest marker of every point (first minimum of the squared
    distance, summed over the directions in order), by brute force in chunks."""
    out = np.empty(len(pts), dtype=np.int64)
    for a in range(0, len(pts), 4096):
        P = pts[a:a + 4096]
        d2 = None
        for d in range(X.shape[1]):
            t = P[:, d:d + 1] - X[None, :, d]
            d2 = t * t if d2 is None else d2 + t * t
        out[a:a + 4096] = np.argmin(d2, axis=1)
    return out


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
            samples = np.asarray(samples)
            samples = samples.astype(complex if np.iscomplexobj(samples) else float)
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
        Sm_full = g.zeros(Sm_int.dtype)
        V(Sm_full, g)[...] = Sm_int
    elif geo["kind"] == MARKERS:
        M = np.asarray(geo["markers"], dtype=float).reshape(-1, 2 * dim + 2)
        X, Nrm, Um, Am = M[:, :dim], M[:, dim:2 * dim], M[:, 2 * dim], M[:, 2 * dim + 1]
        lo = X.min(axis=0) - 2.0 * s
        hi = X.max(axis=0) + 2.0 * s
        pts = np.stack([x[d].ravel() for d in range(dim)], axis=1)
        inbox = np.all((pts >= lo) & (pts <= hi), axis=1)
        near = np.full(len(pts), -1, dtype=np.int64)
        near[inbox] = nearest_markers(pts[inbox], X)
        m = near[inbox]
        off = None
        for d in range(dim):
            t = (pts[inbox, d] - X[m, d]) * Nrm[m, d]
            off = t if off is None else off + t
        chi_flat = np.zeros(len(pts))
        chi_flat[inbox] = (off <= s).astype(float)
        chi = chi_flat.reshape(g.shape)
        near = near.reshape(g.shape)
        safe = np.where(near >= 0, near, 0)
        for d in range(dim):
            vib[d] = chi * Um[safe] * Nrm[safe, d]
        chi_int = V(chi, g)
        near_int = V(near, g)
        counts = np.bincount(near_int[chi_int > 0].ravel(), minlength=len(M))
        if np.any(counts == 0):
            raise ValueError("a marker has no masked cell matched with it (markers denser than the cells)")
        mi = np.where(near_int >= 0, near_int, 0)
        Sm_int = chi_int * (rho_b * Um[mi] * Am[mi] / (counts[mi] * g.dV))
        Sm_full = g.zeros()
        V(Sm_full, g)[...] = Sm_int
    elif geo["kind"] == COUETTE:
        R1, R2 = float(geo["radius"]), float(geo["half"][0])
        dx, dy = x[0] - c[0], x[1] - c[1]
        r = np.sqrt(dx * dx + dy * dy)
        inner = r - R1 <= s
        chi = (inner | (R2 - r <= s)).astype(float)
        w = np.where(inner, U_b / R1, 0.0)
        vib[0] = -w * dy
        vib[1] = w * dx
    else:
        raise ValueError("unknown body kind")

    return dict(chi=chi, vib=vib, Sm=V(Sm_full, g).copy(), Z_ib=float(geo["Z_ib"]),
                H_ib=float(geo["H_ib"]), Da_ib=float(geo["Da_ib"]))
