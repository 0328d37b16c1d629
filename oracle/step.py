"""One time step of the low-Mach fractional-step method (Sec. 3.1, Eqs 3.1-3.19)
with the collocated spatial discretisation of Sec. 3.2 (Eqs 3.23-3.26).

Unknowns (Eqs 2.42-2.50): velocity v, rescaled mixture fraction Z, excess
enthalpy H, P = p dt (Eq 3.8c), thermodynamic pressure p0(t); derived T, rho,
kappa from the flame-sheet state relation.

Readings where the paper is silent or ambiguous (each one is also listed with
the design notes of the package):
 * Eq 3.3 writes v^n inside the (n-1) residual; the (n-1) residual of Eq 3.1 is
   used instead: the full right-hand side of the previous step is stored and
   reused.
 * Eq 3.26a's interpolation index: v_i is interpolated along x_j onto the
   j-interface, delta_1(F_j bar(v_i)^{1x_j}) / delta_1 x_j.
 * The convective terms at level n use the interface fluxes F^n of the
   projection that produced v^n; at t = 0, F^0 = bar(rho^0 v^0) (P = 0).
 * Viscous stress (Eq 2.46) on the j-interface: kappa by Eq 3.20; d v_i/d x_j by
   delta_1 across the interface; tangential derivatives d v_j / d x_i (i != j) and
   the divergence's tangential parts by the interface average (Eq 3.20: 1/2 and
   1/2 on a uniform grid) of the cell-centred delta_2 derivatives; then delta_1
   across the cell (a composition of odd operators, text after Eq 3.26).
 * Penalisation terms (Eqs 3.30-3.32) join the other forcing terms of their
   equation (Z, H: inside the 1/rho bracket of Eqs 3.2/3.4) and get the same
   AB2 / AM2 treatment.
 * Start-up (text after Eq 3.19): step 0 uses Euler in the predictor; the
   backward-difference rates of rho (Eqs 3.11, 3.19) and p0 (Eqs 3.5, 3.14) use
   the highest order the stored history allows (0th, 1st, then 2nd order).
 * Enclosed systems take p0 from Eq 2.40 with the initial mass m = int rho^0 dV,
   p0^0 = 1; open systems take p0 = 1 (Eq 2.41).
 * Semi-enclosed systems (closed_system = 2) advance p0 by the ODE of Eq 2.38
   with the stages of the scalars: AB2 in the predictor (Euler on step 0),
   AM2 in the corrector, its right-hand side G evaluated on the level's
   fields.  The volume integrals are cell sums of the discrete operators the
   residuals use: div(kappa grad .) as in Eq 3.26b's diffusive part, div v as
   the sum of the cell-centred delta_2 derivatives (which telescopes to the
   boundary values of v), and N' regularised like N (Eq 3.35b).  The
   projection's mass balance is then closed only up to the ODE's truncation
   error; the mean of b is removed as for every other kind.
 * The outflow interfaces' mass flux is the adjacent cell's provisional
   momentum, shifted by one uniform amount so that the discrete global mass
   balance closes exactly (text after Eq 4.22); the mean of b is then removed
   (augmented-matrix solution, Sec. 3.3).
 * ``incompressible``: T = rho = kappa = p0 = 1 regardless of Z, H -- the
   constant-density runs of Secs 4.2-4.3 (Re = Pe/Pr in the viscous term).
 * ``stretch`` (alpha of Eq 4.18 per direction, 0 for uniform) gives the
   tanh-stretched grids of the cavity (Sec. 4.3.1): every operator takes the
   non-uniform weights of Eqs 3.20-3.22, the mean of b and of P is
   volume-weighted, and the Poisson equation is solved by a sparse
   factorisation.  Immersed bodies are not built on stretched grids.
"""

import copy

import numpy as np

from . import flame, poisson
from .boundary import (Boundary, PERIODIC, INFLOW, OUTFLOW, WALL, SLIP, WALL_T, face_end, cell_end)
from .ibm import build as build_ibm
from .operators import (Grid, V, pad, dtype_of, centres_to_faces, interp_to_faces, diff_to_faces,
                        faces_interp_to_cells, faces_diff_to_cells, diff2, integrate)
from .stretched import tanh_faces


class Problem:
    """Static data of a run: grid, parameters, boundary, body."""

    def __init__(self, prm, geo=None):
        self.prm = dict(prm)
        dim = int(prm["dim"])
        alpha = [float(a) for a in prm.get("stretch", [0.0] * dim)[:dim]]
        if any(a != 0.0 for a in alpha):
            if geo is not None:
                raise NotImplementedError("immersed bodies on stretched grids are not built")
            faces = [prm["L"][d] * tanh_faces(prm["n"][d], alpha[d]) for d in range(dim)]
            per = [prm["bc"][d][0] == PERIODIC for d in range(dim)]
            self.g = Grid(prm["n"][:dim], prm["L"][:dim], faces=faces, periodic=per)
        else:
            self.g = Grid(prm["n"][:dim], prm["L"][:dim])
        g = self.g
        self.fp = flame.derived_parameters(prm["Z_st"], prm["density_ratio"], prm["eps_reg"],
                                           prm["tol_reg"], prm["Le_F"], prm["Le_O"], prm["gamma"])
        self.Pe = prm["Re"] * prm["Pr"]
        self.ibm = build_ibm(g, geo)
        chi = self.ibm["chi"] if self.ibm is not None else None
        self.bnd = Boundary(g, prm["bc"][:dim], prm["inflow_v"][:dim], prm["inflow_Z"],
                            prm["inflow_H"], chi, prm.get("wall_H"))
        self.transport = int(prm.get("transport", 0))
        self.suth_C = float(prm.get("sutherland_C", 0.0))
        self.periodic = [self.bnd.periodic(d) for d in range(dim)]
        self.incompressible = bool(prm.get("incompressible", 0))
        self.has_inflow = any(prm["bc"][d][s] == INFLOW for d in range(dim) for s in (0, 1))
        self.closed = int(prm.get("closed_system", 0)) == 1
        self.semi = int(prm.get("closed_system", 0)) == 2 and not self.incompressible

    # -- state relation (Sec. 3.5, Eqs 2.49-2.50, 2.40-2.41) ------------------
    def thermo_at(self, Z, H, p0):
        """(T, rho, kappa) for a given p0: T and rho on the interior cells (ghosts
        unused), kappa with its ghost cells filled by the boundary rule."""
        g = self.g
        if self.incompressible:
            one = np.ones(g.shape)
            return one, one.copy(), one.copy()
        T = pad(flame.temperature(V(Z, g), V(H, g), self.fp), g)        # Eq 3.42
        rho = pad(flame.density(p0, V(T, g)), g)                         # Eq 2.49
        kap = pad(self.kappa_of(V(T, g)), g)                             # Eq 2.50 / 4.12
        self.bnd.fill(kap, "kappa", kappa_in=self.inflow_kappa() if self.has_inflow else None,
                      kappa_wall=self.wall_kappa())
        return T, rho, kap

    def thermo(self, Z, H, mass, p0_ode=None):
        """(T, rho, kappa, p0): p0 from Eq 2.40 (enclosed), Eq 2.41 (open) or
        the value p0_ode the ODE of Eq 2.38 gave (semi-enclosed)."""
        g = self.g
        if self.incompressible:
            return self.thermo_at(Z, H, 1.0) + (1.0,)
        if self.semi:
            p0 = float(p0_ode)
        elif self.closed:
            T = flame.temperature(V(Z, g), V(H, g), self.fp)
            p0 = flame.closed_p0(mass, T, g.dV)
        else:
            p0 = 1.0
        return self.thermo_at(Z, H, p0) + (p0,)

    def inflow_temperature(self):
        return float(flame.temperature(np.array(self.prm["inflow_Z"]),
                                       np.array(self.prm["inflow_H"]), self.fp))

    def kappa_of(self, T):
        return flame.kappa(T, self.prm["sigma"], self.transport, self.suth_C)

    def inflow_kappa(self):
        return float(self.kappa_of(self.inflow_temperature()))

    def wall_kappa(self):
        """kappa of each isothermal wall's state (Z_in, H_wall of the side), [d][side]."""
        out = []
        for d in range(self.g.dim):
            row = []
            for s in (0, 1):
                if self.prm["bc"][d][s] != WALL_T or self.incompressible:
                    row.append(1.0)
                    continue
                T = flame.temperature(np.array(self.prm["inflow_Z"]), np.array(self.bnd.wall_H[d][s]), self.fp)
                row.append(float(self.kappa_of(T)))
            out.append(row)
        return out

    def inflow_density(self, p0):
        if self.incompressible:
            return 1.0
        return float(flame.density(p0, self.inflow_temperature()))


class State:
    """Time level n plus the multistep history (Eqs 3.1, 3.5, 3.11)."""

    def __init__(self):
        self.v = None        # list of padded arrays
        self.Z = self.H = self.T = self.rho = self.kappa = self.P = None
        self.F = None        # list of padded interface arrays
        self.p0_hist = []    # [p0^n, p0^(n-1), p0^(n-2)]
        self.rho_prev = None
        self.R_prev = None
        self.G_prev = None   # right-hand side of Eq 2.38 at the previous level
        self.mass = None
        self.nstep = 0
        self.t = 0.0

    def copy(self):
        return copy.deepcopy(self)


# -----------------------------------------------------------------------------
def initial_state(pb, v0, Z0, H0):
    """State at t = 0 from interior arrays v0 (list), Z0, H0."""
    g, bnd = pb.g, pb.bnd
    st = State()
    st.v = [pad(v0[d], g) for d in range(g.dim)]
    for d in range(g.dim):
        bnd.fill(st.v[d], "v", d)
    st.Z = pad(Z0, g)
    st.H = pad(H0, g)
    bnd.fill(st.Z, "Z")
    bnd.fill(st.H, "H")
    T, rho, kap = pb.thermo_at(st.Z, st.H, 1.0)                      # p0^0 = 1
    st.T, st.rho, st.kappa = T, rho, kap
    st.mass = integrate(V(rho, g), g)
    st.p0_hist = [1.0]
    st.P = g.zeros()
    mom = [V(rho, g) * V(st.v[d], g) for d in range(g.dim)]
    Ft = _provisional_fluxes(pb, mom, 1.0)
    st.F = []
    for j in range(g.dim):
        Fj = g.zeros(dtype_of(Ft[j]))
        V(Fj, g, face=j)[...] = Ft[j]
        st.F.append(Fj)
    return st


# -----------------------------------------------------------------------------
def residuals(pb, v, Z, H, rho, kap, F, p0dot):
    """Right-hand sides at one time level (interior arrays).

    Rv[i] = Res_v,i + f_v,i + F_v,i    (Eqs 3.8a-b, 3.26a, 3.29-3.30)
    RZ    = Res_Z  (Eq 3.2 with F_Z of Eq 3.31, Eq 3.26b)
    RH    = Res_H + f_H  (Eqs 3.4a-b with F_H of Eq 3.32, Eq 3.26b)"""
    g, prm, fp = pb.g, pb.prm, pb.fp
    dim = g.dim
    Pe = pb.Pe
    PrPe = prm["Pr"] / Pe
    rho_c = V(rho, g)
    kap_c = V(kap, g)
    ibm = pb.ibm
    Fv = [V(F[j], g, face=j) for j in range(dim)]
    kf = [interp_to_faces(kap, g, j) for j in range(dim)]
    dt_ = dtype_of(*v, Z, H, rho, kap, *F)

    Rv = []
    for i in range(dim):
        conv = np.zeros(rho_c.shape, dtype=dt_)
        visc = np.zeros(rho_c.shape, dtype=dt_)
        for j in range(dim):
            # Eq 3.26a: delta_1 (F_j bar(v_i)^{1x_j}) / delta_1 x_j
            conv += faces_diff_to_cells(Fv[j] * interp_to_faces(v[i], g, j), g, j)
            # Eq 2.46 on the j-interfaces
            dvi_dxj = diff_to_faces(v[i], g, j)
            if i == j:
                dvj_dxi = dvi_dxj
            else:
                dvj_dxi = centres_to_faces(diff2(v[j], g, i, off=g.unit(j, -1), face=j),
                                           diff2(v[j], g, i, face=j), g, j)
            tau = kf[j] * (dvi_dxj + dvj_dxi)
            if i == j:
                div = diff_to_faces(v[j], g, j)
                for k in range(dim):
                    if k != j:
                        div = div + centres_to_faces(diff2(v[k], g, k, off=g.unit(j, -1), face=j),
                                                     diff2(v[k], g, k, face=j), g, j)
                tau = tau - (2.0 / 3.0) * kf[j] * div
            visc += faces_diff_to_cells(tau, g, j)
        R = -conv + PrPe * visc
        if i == 1 and prm["inv_Fr2"] != 0.0:
            R = R + prm["inv_Fr2"] * (1.0 - rho_c)                    # Eq 3.8b
        if ibm is not None:                                          # Eq 3.30
            chi = V(ibm["chi"], g)
            R = R - chi * PrPe / ibm["Da_ib"] * kap_c * (V(v[i], g) - V(ibm["vib"][i], g))
        Rv.append(R)

    def convective(phi):                                             # Eq 3.26b
        out = np.zeros(rho_c.shape, dtype=dt_)
        for j in range(dim):
            out += faces_interp_to_cells(Fv[j] * diff_to_faces(phi, g, j), g, j)
        return out

    def diffusive(phi):                                              # div(kappa grad phi)
        out = np.zeros(rho_c.shape, dtype=dt_)
        for j in range(dim):
            out += faces_diff_to_cells(kf[j] * diff_to_faces(phi, g, j), g, j)
        return out

    Zc = V(Z, g)
    Hc = V(H, g)
    Le = flame.lewis_eps(Zc, fp)                                     # Eq 3.35a
    Nn = flame.N_eps(Zc, fp)                                         # Eq 3.35b
    dZ = diffusive(Z)
    bracket_Z = -convective(Z) + dZ / (Le * Pe)
    bracket_H = -convective(H) + diffusive(H) / Pe + fp["zeta"] * p0dot + Nn * dZ / Pe
    if ibm is not None:
        chi = V(ibm["chi"], g)
        bracket_Z = bracket_Z - chi * kap_c * (Zc - ibm["Z_ib"]) / (Le * Pe * ibm["Da_ib"])  # Eq 3.31
        bracket_H = bracket_H - chi * kap_c * (Hc - ibm["H_ib"]) / (Pe * ibm["Da_ib"])       # Eq 3.32
    return dict(v=Rv, Z=bracket_Z / rho_c, H=bracket_H / rho_c)


# -----------------------------------------------------------------------------
def _provisional_fluxes(pb, mom, p0):
    """Interface mass fluxes of the provisional momentum (first term of Eq 3.23),
    with the known boundary fluxes on non-periodic sides (before the outflow
    shift).  ``mom`` is a list of interior arrays."""
    g, bnd = pb.g, pb.bnd
    rho_in = pb.inflow_density(p0)
    out = []
    for j in range(g.dim):
        m = pad(mom[j], g)
        if bnd.periodic(j):
            bnd_fill_periodic(m, g, j)
        Fj = interp_to_faces(m, g, j)
        if not bnd.periodic(j):
            for side in (0, 1):
                kind = bnd.face_kind_view(j, side)
                adj = cell_end(mom[j], g, j, side)
                val = np.select([kind == INFLOW, kind == OUTFLOW, kind == WALL, kind == SLIP],
                                [rho_in * bnd.inflow_v[j] + 0.0 * adj, adj, 0.0 * adj, 0.0 * adj])
                face_end(Fj, g, j, side)[...] = val
        out.append(Fj)
    return out


def bnd_fill_periodic(a, g, j):
    n = g.n[j]
    ax = g.ax(j)
    s0 = [slice(None)] * g.dim
    s1 = [slice(None)] * g.dim
    s0[ax], s1[ax] = 0, n
    a[tuple(s0)] = a[tuple(s1)]
    s0[ax], s1[ax] = n + 1, 1
    a[tuple(s0)] = a[tuple(s1)]


def project(pb, mom, rho, drho, p0):
    """Pressure step: Eqs 3.9-3.11 / 3.17-3.19 through Eqs 3.23-3.25.

    Returns (P padded with ghosts, F list of padded interface arrays,
    v list of padded arrays with ghosts, b)."""
    g, bnd = pb.g, pb.bnd
    dim = g.dim
    Ft = _provisional_fluxes(pb, mom, p0)
    Sm = pb.ibm["Sm"] if pb.ibm is not None else 0.0
    # global mass balance: sum (d_t rho - S_m) dV + net outward boundary flow = 0
    total = integrate(drho - Sm, g)
    out_area = 0.0
    for j in range(dim):
        if bnd.periodic(j):
            continue
        dA = g.face_area(j)
        for side in (0, 1):
            sign = -1.0 if side == 0 else 1.0
            kind = bnd.face_kind_view(j, side)
            if g.uniform:
                total += sign * np.sum(face_end(Ft[j], g, j, side)) * dA
                out_area += float(np.sum(kind == OUTFLOW)) * dA
            else:
                total += sign * np.sum(face_end(Ft[j], g, j, side) * dA)
                out_area += float(np.sum((kind == OUTFLOW) * dA))
    if out_area > 0.0:
        c = -total / out_area
        for j in range(dim):
            if bnd.periodic(j):
                continue
            for side in (0, 1):
                sign = -1.0 if side == 0 else 1.0
                kind = bnd.face_kind_view(j, side)
                end = face_end(Ft[j], g, j, side)
                end[...] = np.where(kind == OUTFLOW, end + sign * c, end)
    # Eq 3.24 (+ S_m, Eq 3.33): L P = d_t rho + sum_j delta_1 Ft_j - S_m
    b = drho - Sm
    for j in range(dim):
        b = b + faces_diff_to_cells(Ft[j], g, j)
    b = b - g.mean(b)
    P_int = poisson.solve(b, g, pb.periodic)
    P = pad(P_int, g)
    bnd.fill_pressure(P)
    F = []
    for j in range(dim):
        Fj_face = Ft[j] - diff_to_faces(P, g, j)                      # Eq 3.23
        if not bnd.periodic(j):
            for side in (0, 1):
                face_end(Fj_face, g, j, side)[...] = face_end(Ft[j], g, j, side)
        Fj = g.zeros(dtype_of(Fj_face))
        V(Fj, g, face=j)[...] = Fj_face
        F.append(Fj)
    v = []
    for i in range(dim):
        vi = pad((mom[i] - diff2(P, g, i)) / V(rho, g), g)            # Eq 3.25
        bnd.fill(vi, "v", i)
        v.append(vi)
    return P, F, v, b


def p0_rate(pb, v, Z, H, kap, p0):
    """Right-hand side of Eq 2.38,
    G = gamma / V { Q/(S+1) / Pe int [div(kappa grad H) + N' div(kappa grad Z)] dV
                    - p0 int div v dV },
    the integrals as cell sums of the discrete operators (padded inputs with
    their ghost cells filled)."""
    g, fp = pb.g, pb.fp
    dim = g.dim
    kf = [interp_to_faces(kap, g, j) for j in range(dim)]

    def diffusive(phi):
        out = np.zeros(V(phi, g).shape, dtype=dtype_of(phi, kap))
        for j in range(dim):
            out += faces_diff_to_cells(kf[j] * diff_to_faces(phi, g, j), g, j)
        return out

    heat = integrate(diffusive(H) + flame.Nprime_eps(V(Z, g), fp) * diffusive(Z), g)
    div = integrate(sum(diff2(v[j], g, j) for j in range(dim)), g)
    vol = g.volume()
    return pb.prm["gamma"] / vol * (fp["Q"] / (fp["S"] + 1.0) / pb.Pe * heat - p0 * div)


def _ddt_rho(rho_new, rho_n, rho_prev, dt, n):
    """Backward difference of rho: Eq 3.11 / 3.19 (first order on step 0)."""
    if n == 0:
        return (rho_new - rho_n) / dt
    return (3.0 * rho_new - 4.0 * rho_n + rho_prev) / (2.0 * dt)


def _p0dot_level_n(hist, dt):
    """d_t p0 at level n (Eq 3.5) from [p0^n, p0^(n-1), p0^(n-2)]."""
    if len(hist) >= 3:
        return (3.0 * hist[0] - 4.0 * hist[1] + hist[2]) / (2.0 * dt)
    if len(hist) == 2:
        return (hist[0] - hist[1]) / dt
    return 0.0


def _p0dot_star(p0s, hist, dt):
    """d_t p0 at the predicted level (Eq 3.14)."""
    if len(hist) >= 2:
        return (3.0 * p0s - 4.0 * hist[0] + hist[1]) / (2.0 * dt)
    return (p0s - hist[0]) / dt


def advance(pb, st, return_star=False):
    """Advance ``st`` (not modified) by one step; returns the new State
    (and the predicted fields when ``return_star``)."""
    g, bnd, prm = pb.g, pb.bnd, pb.prm
    dim = g.dim
    dt = float(prm["dt"])
    n = st.nstep
    rho_n = V(st.rho, g)
    mom_n = [rho_n * V(st.v[i], g) for i in range(dim)]

    # ---------------- predictor (Eqs 3.1-3.11) ----------------
    p0dot_n = _p0dot_level_n(st.p0_hist, dt)
    Rn = residuals(pb, st.v, st.Z, st.H, st.rho, st.kappa, st.F, p0dot_n)
    if n == 0 or st.R_prev is None:
        cZ, cH, cv = Rn["Z"], Rn["H"], Rn["v"]                         # Euler start
    else:
        Rp = st.R_prev
        cZ = 1.5 * Rn["Z"] - 0.5 * Rp["Z"]                              # Eq 3.1
        cH = 1.5 * Rn["H"] - 0.5 * Rp["H"]                              # Eq 3.3
        cv = [1.5 * Rn["v"][i] - 0.5 * Rp["v"][i] for i in range(dim)]  # Eq 3.10
    Zs = pad(V(st.Z, g) + dt * cZ, g)
    Hs = pad(V(st.H, g) + dt * cH, g)
    bnd.fill(Zs, "Z")
    bnd.fill(Hs, "H")
    p0_ode = None
    if pb.semi:                                                          # Eq 2.38, AB2
        G_n = p0_rate(pb, st.v, st.Z, st.H, st.kappa, st.p0_hist[0])
        cG = G_n if (n == 0 or st.G_prev is None) else 1.5 * G_n - 0.5 * st.G_prev
        p0_ode = st.p0_hist[0] + dt * cG
    Ts, rhos, kaps, p0s = pb.thermo(Zs, Hs, st.mass, p0_ode)            # Eq 3.6
    mom_t = [mom_n[i] + dt * cv[i] for i in range(dim)]                 # rho* v~ (Eq 3.10)
    drho = _ddt_rho(V(rhos, g), rho_n, None if st.rho_prev is None else V(st.rho_prev, g), dt, n)
    Ps, Fs, vs, _ = project(pb, mom_t, rhos, drho, p0s)                 # Eqs 3.9, 3.23-3.25

    # ---------------- corrector (Eqs 3.12-3.19) ----------------
    p0dot_s = _p0dot_star(p0s, st.p0_hist, dt)
    Rs = residuals(pb, vs, Zs, Hs, rhos, kaps, Fs, p0dot_s)
    Z1 = pad(V(st.Z, g) + 0.5 * dt * (Rs["Z"] + Rn["Z"]), g)            # Eq 3.12
    H1 = pad(V(st.H, g) + 0.5 * dt * (Rs["H"] + Rn["H"]), g)            # Eq 3.13
    bnd.fill(Z1, "Z")
    bnd.fill(H1, "H")
    if pb.semi:                                                          # Eq 2.38, AM2
        G_s = p0_rate(pb, vs, Zs, Hs, kaps, p0s)
        p0_ode = st.p0_hist[0] + 0.5 * dt * (G_s + G_n)
    T1, rho1, kap1, p01 = pb.thermo(Z1, H1, st.mass, p0_ode)            # Eq 3.15
    mom_b = [mom_n[i] + 0.5 * dt * (Rs["v"][i] + Rn["v"][i]) for i in range(dim)]  # Eq 3.18
    drho1 = _ddt_rho(V(rho1, g), rho_n, None if st.rho_prev is None else V(st.rho_prev, g), dt, n)
    P1, F1, v1, _ = project(pb, mom_b, rho1, drho1, p01)                # Eqs 3.17, 3.23-3.25

    new = State()
    new.v, new.Z, new.H, new.T, new.rho, new.kappa = v1, Z1, H1, T1, rho1, kap1
    new.P, new.F = P1, F1
    new.p0_hist = ([p01] + st.p0_hist)[:3]
    new.rho_prev = st.rho.copy()
    new.R_prev = Rn
    new.G_prev = G_n if pb.semi else None
    new.mass = st.mass
    new.nstep = n + 1
    new.t = st.t + dt
    if return_star:
        star = dict(v=vs, Z=Zs, H=Hs, T=Ts, rho=rhos, P=Ps, F=Fs, p0=p0s)
        return new, star
    return new


def run(pb, st, nsteps):
    for _ in range(nsteps):
        st = advance(pb, st)
    return st
