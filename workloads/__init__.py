"""Seeded synthetic workloads (input recipes) shared by the tests, the bench and
the oracle checks.

This module only builds inputs: the parameter record, the body description and
the initial fields.  It holds none of the solver's arithmetic -- the state
relation, the boundary treatment, the mask, the fluxes and the Poisson solve
are implemented separately by the oracle and by the CUDA path.

Conventions of the recipes (paper variables; Eqs 2.34-2.37, 4.21):
  S = 1/Z_st - 1, Q = (ratio - 1)(S + 1)  so that the flame (Z = 1) temperature
  is the density ratio; ambient air and fuel at T = 1, hence
  H_inf = H_ib = 1 + (S+1)/Q ("zero excess enthalpy"), Z_air = 0, Z_fuel = S + 1.
Initial fields are interior arrays of shape (n_y, n_x) / (n_z, n_y, n_x), x fastest.

Workloads
  taylor_green(n, dt)   Taylor-Green vortex (Eqs 4.4-4.6), constant density.
  periodic_blobs(...)   2D doubly periodic enclosed box, 8 Gaussian mixture-fraction
                        blobs, solenoidal random velocity (rms 0.1), 64x64.
  slot_burner(...)      2D planar slot burner, 256x512 on [0,1]x[0,2].
  sphere_burner(...)    3D spherical porous burner, 192^3 on [0,1]^3.
  marker_burner(...)    the porous burner (circle in 2D, sphere in 3D) given by
                        surface markers instead of its analytic shape.
  heated_cavity(...)    the differentially heated square cavity of Sec. 4.3
                        (Eqs 4.8-4.17): isothermal side walls, adiabatic top and
                        bottom, Sutherland transport, buoyancy, enclosed.
"""

import numpy as np

PERIODIC, INFLOW, OUTFLOW, WALL, SLIP, WALL_T = 0, 1, 2, 3, 4, 5
IBM_NONE, IBM_SLOT, IBM_SPHERE, IBM_MARKERS, IBM_COUETTE = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1

SEED = 20260101


def _base_params():
    return dict(
        dim=2, n=[0, 0, 1], L=[1.0, 1.0, 1.0],
        bc=[[PERIODIC, PERIODIC], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC]],
        inflow_v=[0.0, 0.0, 0.0], inflow_Z=0.0, inflow_H=0.0,
        Re=100.0, Pr=0.7, inv_Fr2=0.0, Le_F=1.0, Le_O=1.0, gamma=1.4, sigma=0.7,
        Z_st=0.055, density_ratio=7.0, eps_reg=0.5, tol_reg=1e-3,
        closed_system=0, incompressible=0, dt=0.0,
        precision=FP64, poisson_rtol=1e-10, poisson_max_iter=200, mg_sweeps=0, mg_tail_cells=0,
        stage_tile_x=0, transport=0, sutherland_C=0.0, wall_H=[[0.0, 0.0], [0.0, 0.0], [0.0, 0.0]])


def paper_scalars(Z_st, ratio):
    """(S, Q, H_inf, Z_fuel) of the recipe conventions above."""
    S = 1.0 / Z_st - 1.0
    Q = (ratio - 1.0) * (S + 1.0)
    return S, Q, 1.0 + (S + 1.0) / Q, S + 1.0


def cell_centres(n, L):
    """Coordinates of interior cell centres, one array per direction."""
    dim = len(n)
    axes = [(np.arange(n[d]) + 0.5) * (L[d] / n[d]) for d in range(dim)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")     # (z), y, x order
    return list(reversed(grids))                             # x, y, (z)


def stable_dt(n, L, Re, Pr, ratio, sigma, U, cfl, Da_ib=None, dim=2):
    """Fixed time step of a run: CFL-scaled minimum of the convective limit,
    the explicit-diffusion limit at the hottest, lightest state (kappa = T_f^sigma,
    rho = 1/T_f) and, with a body, the penalisation limit dt <= Re Da_ib."""
    h = min(L[d] / n[d] for d in range(dim))
    T_f = ratio
    kap_max = T_f ** sigma
    rho_min = 1.0 / T_f
    lim = [h / U, h * h * Re * min(1.0, Pr) * rho_min / (2.0 * dim * kap_max)]
    if Da_ib is not None:
        lim.append(Re * Da_ib * rho_min / kap_max)
    return cfl * min(lim)


def _solenoidal_2d(rng, n, L, kmax, rms):
    """delta_2-curl of a random periodic streamfunction (modes 0 < |k| <= kmax),
    scaled to the requested rms speed."""
    x, y = cell_centres(n, L)
    psi = np.zeros(x.shape)
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            k2 = kx * kx + ky * ky
            if k2 == 0 or k2 > kmax * kmax:
                continue
            amp = rng.normal() / np.sqrt(k2)
            ph = rng.uniform(0.0, 2.0 * np.pi)
            psi += amp * np.cos(2.0 * np.pi * (kx * x / L[0] + ky * y / L[1]) + ph)
    hx, hy = L[0] / n[0], L[1] / n[1]
    u = (np.roll(psi, -1, axis=0) - np.roll(psi, 1, axis=0)) / (2.0 * hy)
    v = -(np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1)) / (2.0 * hx)
    s = rms / np.sqrt(np.mean(u * u + v * v))
    return u * s, v * s


def taylor_green(n=50, dt=4e-3, Re=100.0):
    """Taylor-Green vortex on the unit periodic square (Sec. 4.2): exact
    velocity of Eqs 4.4-4.5 at t = 0; constant density."""
    prm = _base_params()
    prm.update(dim=2, n=[n, n, 1], L=[1.0, 1.0, 1.0], Re=Re, Pr=1.0, incompressible=1, dt=dt,
               poisson_rtol=1e-13)
    x, y = cell_centres((n, n), (1.0, 1.0))
    u = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    v = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    fields = dict(v=[u, v], Z=np.zeros_like(u), H=np.ones_like(u))
    return prm, None, fields


def taylor_green_exact(n, t, Re=100.0):
    """Eqs 4.4-4.6 at the cell centres."""
    x, y = cell_centres((n, n), (1.0, 1.0))
    e1 = np.exp(-8 * np.pi ** 2 * t / Re)
    e2 = np.exp(-16 * np.pi ** 2 * t / Re)
    u = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * e1
    v = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y) * e1
    p = 0.25 * (np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) * e2
    return u, v, p


def periodic_blobs(n=64, seed=SEED, cfl=0.4, nblobs=8):
    """2D doubly periodic enclosed box: Z_c = clip(sum of 8 Gaussian blobs, 0, 1)
    with amplitude U[0.3,1], width U[0.05,0.15] L, centre U[0,1)^2 (minimum-image
    periodic distance); H = H_inf; velocity the delta_2-curl of a random
    streamfunction (|k| <= 4) scaled to rms 0.1; Z_st = 0.055, density ratio 7,
    Le = 1, Re = 100, Pr = 0.7; enclosed (p0 from the mass constraint)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prm = _base_params()
    ny = nx = n
    prm.update(dim=2, n=[nx, ny, 1], L=[1.0, 1.0, 1.0], Re=100.0, Pr=0.7, closed_system=1)
    S, Q, H_inf, Z_fuel = paper_scalars(prm["Z_st"], prm["density_ratio"])
    x, y = cell_centres((nx, ny), (1.0, 1.0))
    Zc = np.zeros(x.shape)
    for _ in range(nblobs):
        a = rng.uniform(0.3, 1.0)
        s = rng.uniform(0.05, 0.15)
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        dx = (x - cx + 0.5) % 1.0 - 0.5
        dy = (y - cy + 0.5) % 1.0 - 0.5
        Zc += a * np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
    Zc = np.clip(Zc, 0.0, 1.0)
    u, v = _solenoidal_2d(rng, (nx, ny), (1.0, 1.0), 4, 0.1)
    Umax = float(np.max(np.sqrt(u * u + v * v)))
    prm["dt"] = stable_dt((nx, ny), (1.0, 1.0), prm["Re"], prm["Pr"], prm["density_ratio"],
                          prm["sigma"], Umax, cfl)
    fields = dict(v=[u, v], Z=Z_fuel * Zc, H=np.full(x.shape, H_inf))
    return prm, None, fields


def filling_chamber(n=64, U_in=0.1, cfl=0.4, closed_system=2, dim=2):
    """Semi-enclosed chamber (Eq 2.38): the unit square (cube), periodic in x
    (and z), air (Z = 0, H = H_inf) entering through the whole bottom side at
    v_2 = U_in, a no-slip wall on top, no outlet, so that p0 rises as the
    chamber fills.  It holds a Gaussian fuel blob (peak Z = Z_fuel, width 0.1,
    centre (0.5, 0.6[, 0.5])) burning in air moving at v_2 = U_in;
    Z_st = 0.055, density ratio 7, Le = 1, Re = 100, Pr = 0.7."""
    prm = _base_params()
    bc = [[PERIODIC, PERIODIC], [INFLOW, WALL], [PERIODIC, PERIODIC]]
    prm.update(dim=dim, n=[n, n, n if dim == 3 else 1], L=[1.0, 1.0, 1.0], Re=100.0, Pr=0.7, bc=bc,
               inflow_v=[0.0, U_in, 0.0], closed_system=closed_system)
    S, Q, H_inf, Z_fuel = paper_scalars(prm["Z_st"], prm["density_ratio"])
    prm.update(inflow_Z=0.0, inflow_H=H_inf)
    shape = (n,) * dim
    xs = cell_centres(shape, (1.0,) * dim)
    centre = (0.5, 0.6, 0.5)
    r2 = sum((xs[d] - centre[d]) ** 2 for d in range(dim))
    Z = Z_fuel * np.exp(-r2 / (2.0 * 0.1 ** 2))
    prm["dt"] = stable_dt(shape, (1.0,) * dim, prm["Re"], prm["Pr"], prm["density_ratio"], prm["sigma"],
                          max(U_in, 0.1), cfl, dim=dim)
    v = [np.zeros(Z.shape) for _ in range(dim)]
    v[1][...] = U_in
    fields = dict(v=v, Z=Z, H=np.full(Z.shape, H_inf))
    return prm, None, fields


def slot_burner(nx=256, ny=512, cfl=0.4, Re=200.0, profile=None, U_coflow=0.2, Z_st=0.055, density_ratio=7.0,
                Da_ib=1e-4):
    """2D planar slot burner: [0,1] x [0,2], periodic in x; bottom inflow of air
    (v = (0, U_coflow), Z = 0, H = H_inf) outside the burner foot; top outflow.
    Immersed rectangular burner 0.1 x 0.3 standing on the bottom boundary at
    x = 0.5 (centre (0.5, 0.15), half-sizes (0.05, 0.15)), ejecting fuel
    (Z = S+1, T = 1) through its top face with a parabolic mass-flux profile of
    peak U_b = 1; Da_ib = 1e-4.  Initial state: fuel at rest inside the
    (unshifted) burner box, falling off outside it as a Gaussian of the distance
    to the box (width max(0.04, 10 dy)), and coflow air far from it."""
    prm = _base_params()
    prm.update(dim=2, n=[nx, ny, 1], L=[1.0, 2.0, 1.0], Re=Re, Pr=0.7,
               bc=[[PERIODIC, PERIODIC], [INFLOW, OUTFLOW], [PERIODIC, PERIODIC]],
               inflow_v=[0.0, U_coflow, 0.0], Z_st=Z_st, density_ratio=density_ratio)
    S, Q, H_inf, Z_fuel = paper_scalars(prm["Z_st"], prm["density_ratio"])
    prm.update(inflow_Z=0.0, inflow_H=H_inf)
    Da = Da_ib
    geo = dict(kind=IBM_SLOT, center=[0.5, 0.15, 0.0], half=[0.05, 0.15, 0.0], radius=0.0,
               Da_ib=Da, rho_b=1.0, U_b=1.0, Z_ib=Z_fuel, H_ib=H_inf,
               profile=None if profile is None else list(profile))
    x, y = cell_centres((nx, ny), (1.0, 2.0))
    # distance to the (unshifted) burner box; Gaussian fall-off of the fuel
    # outside it, wide enough (>= 10 cells) that the Z = 1 flame is resolved
    dx = np.maximum(np.abs(x - 0.5) - 0.05, 0.0)
    dy = np.maximum(y - 0.3, 0.0)
    dist = np.sqrt(dx * dx + dy * dy)
    w = max(0.04, 10.0 * 2.0 / ny)
    shape = np.exp(-dist * dist / (2.0 * w * w))
    u = np.zeros(x.shape)
    v = U_coflow * (1.0 - shape)
    Z = Z_fuel * shape
    H = np.full(x.shape, H_inf)
    prm["dt"] = stable_dt((nx, ny), (1.0, 2.0), Re, prm["Pr"], prm["density_ratio"],
                          prm["sigma"], 1.0, cfl, Da_ib=Da)
    return prm, geo, dict(v=[u, v], Z=Z, H=H)


def bump_basis(geo, Da_ib, n_bumps=64, n_profile=256):
    """Gaussian bumps evenly spaced across the shifted slot face [lo, hi]
    (centres at the midpoints of n_bumps equal parts, standard deviation one
    part), sampled at n_profile uniform points of [lo, hi]: the profile samples
    are A @ c with A[k, m] = phi_m(x_k) / sum_m' phi_m'(x_k), so the ejected
    flux is U_base(x) sum_m c_m phi_m / sum_m phi_m (c = 1: the plain parabola)."""
    s = np.sqrt(Da_ib)
    lo = geo["center"][0] - geo["half"][0] - s
    hi = geo["center"][0] + geo["half"][0] + s
    xk = np.linspace(lo, hi, n_profile)
    part = (hi - lo) / n_bumps
    xm = lo + (np.arange(n_bumps) + 0.5) * part
    phi = np.exp(-0.5 * ((xk[:, None] - xm[None, :]) / part) ** 2)
    return phi / phi.sum(axis=1, keepdims=True)


def slot_bumps(nx=128, ny=256, n_bumps=64, n_profile=256, seed=SEED, Da_ib=1e-4):
    """Slot burner (the 2D slot geometry, FP64) whose ejected mass-flux profile
    is parametrised by n_bumps Gaussian bumps (bump_basis); coefficients
    c_m ~ U[0.8, 1.2] (seeded).  Returns (prm, geo, fields, basis, c)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.uniform(0.8, 1.2, n_bumps)
    prm, geo, f = slot_burner(nx, ny, Da_ib=Da_ib)
    prm["precision"] = FP64
    A = bump_basis(geo, Da_ib, n_bumps, n_profile)
    geo["profile"] = list(A @ c)
    return prm, geo, f, A, c


BATCH_GRIDS = ((64, 128), (96, 192), (128, 256))


def batched_flames(count=256, seed=SEED, precision=MIXED):
    """Independent 2D slot-burner flames of uneven sizes: grid drawn uniformly
    from 64x128, 96x192, 128x256; inlet Re ~ U[50, 400]; Z_st ~ U[0.04, 0.08];
    density ratio ~ U[4, 8].  Da_ib = max(1e-4, (2 dx)^2), so the Brinkman
    layer sqrt(Da_ib) spans at least two cells on the coarsest grids.
    Returns a list of (prm, geo, fields)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        nx, ny = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
        Re = float(rng.uniform(50.0, 400.0))
        Z_st = float(rng.uniform(0.04, 0.08))
        ratio = float(rng.uniform(4.0, 8.0))
        Da = max(1e-4, (2.0 / nx) ** 2)
        prm, geo, f = slot_burner(nx, ny, Re=Re, Z_st=Z_st, density_ratio=ratio, Da_ib=Da)
        prm["precision"] = precision
        out.append((prm, geo, f))
    return out


def sphere_burner(n=192, cfl=0.4, Re=150.0, seed=SEED, rms=0.01):
    """3D spherical porous burner: [0,1]^3, outflow on all sides; sphere of
    radius 0.1 at the centre ejecting fuel radially with U_b = 1; quiescent air
    plus a seeded solenoidal perturbation of rms 0.01 (delta_2-curl of a random
    vector potential with modes |k| <= 3); fuel inside the sphere, falling off
    outside it as a Gaussian of the distance (width max(0.04, 10 dx))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prm = _base_params()
    prm.update(dim=3, n=[n, n, n], L=[1.0, 1.0, 1.0], Re=Re, Pr=0.7,
               bc=[[OUTFLOW, OUTFLOW]] * 3)
    S, Q, H_inf, Z_fuel = paper_scalars(prm["Z_st"], prm["density_ratio"])
    prm.update(inflow_Z=0.0, inflow_H=H_inf)
    Da = 1e-4
    geo = dict(kind=IBM_SPHERE, center=[0.5, 0.5, 0.5], half=[0.0, 0.0, 0.0], radius=0.1,
               Da_ib=Da, rho_b=1.0, U_b=1.0, Z_ib=Z_fuel, H_ib=H_inf, profile=None)
    x, y, z = cell_centres((n, n, n), (1.0, 1.0, 1.0))
    h = 1.0 / n
    A = [np.zeros(x.shape) for _ in range(3)]
    for c in range(3):
        for _ in range(6):
            k = rng.integers(-3, 4, size=3)
            if not k.any():
                continue
            ph = rng.uniform(0, 2 * np.pi)
            A[c] += rng.normal() * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + ph)

    def d2(a, d):
        ax = 2 - d
        return (np.roll(a, -1, axis=ax) - np.roll(a, 1, axis=ax)) / (2 * h)
    u = d2(A[2], 1) - d2(A[1], 2)
    v = d2(A[0], 2) - d2(A[2], 0)
    w = d2(A[1], 0) - d2(A[0], 1)
    s = rms / np.sqrt(np.mean(u * u + v * v + w * w))
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    dist = np.maximum(r - 0.1, 0.0)
    width = max(0.04, 10.0 / n)
    Z = Z_fuel * np.exp(-dist * dist / (2.0 * width * width))
    H = np.full(x.shape, H_inf)
    prm["dt"] = stable_dt((n, n, n), (1.0, 1.0, 1.0), Re, prm["Pr"], prm["density_ratio"],
                          prm["sigma"], 1.0, cfl, Da_ib=Da, dim=3)
    return prm, geo, dict(v=[u * s, v * s, w * s], Z=Z, H=H)


def circle_markers(center, R, count, U_b=1.0):
    """Markers on a circle: count equal arcs, each marker at its arc's midpoint
    with the outward radial normal, ejection speed U_b and arc length 2 pi R /
    count.  Rows (x, y, n_x, n_y, U, A)."""
    th = 2.0 * np.pi * (np.arange(count) + 0.5) / count
    nx, ny = np.cos(th), np.sin(th)
    A = np.full(count, 2.0 * np.pi * R / count)
    return np.stack([center[0] + R * nx, center[1] + R * ny, nx, ny, np.full(count, U_b), A], axis=1)


def sphere_markers(center, R, count, U_b=1.0):
    """Markers on a sphere: the Fibonacci lattice (equal-area points), outward
    radial normals, ejection speed U_b and area 4 pi R^2 / count each.  Rows
    (x, y, z, n_x, n_y, n_z, U, A)."""
    k = np.arange(count)
    nz = 1.0 - (2.0 * k + 1.0) / count
    rr = np.sqrt(1.0 - nz * nz)
    ph = k * np.pi * (3.0 - np.sqrt(5.0))
    nx, ny = rr * np.cos(ph), rr * np.sin(ph)
    A = np.full(count, 4.0 * np.pi * R * R / count)
    return np.stack([center[0] + R * nx, center[1] + R * ny, center[2] + R * nz, nx, ny, nz,
                     np.full(count, U_b), A], axis=1)


def taylor_couette_exact(x, y, c=(0.0, 0.0)):
    """Exact Taylor-Couette velocity for R_2 = 2 R_1 = 2 (Sec. 4.2.3):
    v_theta = (4 - r^2)/(3 r) in the gap 1 <= r <= 2, rigid rotation
    v_theta = r inside the inner cylinder, rest outside the outer one."""
    dx, dy = x - c[0], y - c[1]
    r = np.sqrt(dx * dx + dy * dy)
    rs = np.where(r > 0.0, r, 1.0)
    vt = np.where(r < 1.0, r, np.where(r <= 2.0, (4.0 - r * r) / (3.0 * rs), 0.0))
    return -vt * dy / rs, vt * dx / rs


def taylor_couette(n=128, Re=1.0, Da_ib=1e-3, L=5.0, cfl=0.4, dim=2, nz=8):
    """Taylor-Couette flow (Sec. 4.2.3): constant density, coaxial cylinders of
    radii 1 and 2 (eta = 1/2) centred in the periodic box [0, L]^2 (times
    nz cells of the same spacing along the axis x_3 in 3D), the inner one
    turning with unit surface speed, the outer one at rest; penalised with
    the shifted mask at Da_ib.  The initial velocity is the exact solution
    (rigid rotation in the inner body, rest in the outer)."""
    prm = _base_params()
    h = L / n
    nn = [n, n, nz if dim == 3 else 1]
    Ls = [L, L, h * nz if dim == 3 else 1.0]
    prm.update(dim=dim, n=nn, L=Ls, Re=Re, Pr=1.0, incompressible=1)
    c = [0.5 * L, 0.5 * L, 0.5 * Ls[2]]
    geo = dict(kind=IBM_COUETTE, center=c[:dim], half=[2.0, 0.0, 0.0], radius=1.0, Da_ib=Da_ib,
               rho_b=1.0, U_b=1.0, Z_ib=0.0, H_ib=0.0)
    xs = cell_centres(tuple(nn[:dim]), tuple(Ls[:dim]))
    u, v = taylor_couette_exact(xs[0], xs[1], c)
    vel = [u, v] + ([np.zeros(u.shape)] if dim == 3 else [])
    prm["dt"] = cfl * min(h / 1.0, h * h * Re / (2.0 * dim), Re * Da_ib)
    fields = dict(v=vel, Z=np.zeros(u.shape), H=np.zeros(u.shape))
    return prm, geo, fields


def marker_burner(n=64, dim=2, spacing=1.5, cfl=0.4, Re=150.0, seed=SEED, rms=0.01):
    """The porous burner given by surface markers: a circle (2D, n x n) or a
    sphere (3D, n^3) of radius 0.1 at the centre of the unit box, outflow on all
    sides, markers about ``spacing`` cells apart ejecting fuel with U_b = 1.
    3D: the sphere_burner recipe with its body replaced by markers.  2D: quiescent
    air plus a solenoidal perturbation of rms 0.01, fuel inside the circle
    falling off outside it as a Gaussian of the distance."""
    R, h = 0.1, 1.0 / n
    if dim == 3:
        prm, geo, f = sphere_burner(n, cfl=cfl, Re=Re, seed=seed, rms=rms)
        count = int(round(4.0 * np.pi * R * R / (spacing * h) ** 2))
        M = sphere_markers([0.5, 0.5, 0.5], R, count)
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        prm = _base_params()
        prm.update(dim=2, n=[n, n, 1], L=[1.0, 1.0, 1.0], Re=Re, Pr=0.7, bc=[[OUTFLOW, OUTFLOW]] * 2 +
                   [[PERIODIC, PERIODIC]])
        S, Q, H_inf, Z_fuel = paper_scalars(prm["Z_st"], prm["density_ratio"])
        prm.update(inflow_Z=0.0, inflow_H=H_inf)
        geo = dict(kind=IBM_SPHERE, center=[0.5, 0.5, 0.0], half=[0.0, 0.0, 0.0], radius=R, Da_ib=1e-4,
                   rho_b=1.0, U_b=1.0, Z_ib=Z_fuel, H_ib=H_inf, profile=None)
        u, v = _solenoidal_2d(rng, (n, n), (1.0, 1.0), 3, rms)
        x, y = cell_centres((n, n), (1.0, 1.0))
        dist = np.maximum(np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2) - R, 0.0)
        width = max(0.04, 10.0 / n)
        f = dict(v=[u, v], Z=Z_fuel * np.exp(-dist * dist / (2.0 * width * width)), H=np.full(x.shape, H_inf))
        prm["dt"] = stable_dt((n, n), (1.0, 1.0), Re, prm["Pr"], prm["density_ratio"], prm["sigma"], 1.0, cfl,
                              Da_ib=1e-4, dim=2)
        count = int(round(2.0 * np.pi * R / (spacing * h)))
        M = circle_markers([0.5, 0.5], R, count)
    geo = dict(geo, kind=IBM_MARKERS, markers=M)
    return prm, geo, f


def heated_cavity(n=64, Ra=1e2, eps=0.6, gravity=True, ny=None, cfl=0.4, T0=None, h_min=None):
    """Differentially heated square cavity (Sec. 4.3): unit square, left wall at
    T_H = 1 + eps, right wall at T_C = 1 - eps (isothermal no-slip walls,
    Eq 4.16a-b), adiabatic no-slip top and bottom (Eq 4.16c); Pr = 0.71,
    gamma = 1.4, Sutherland transport with C = 110.5 K / 600 K (Eq 4.12),
    Pe = Pr Ra^(1/2) (Eq 4.10, so Re = Ra^(1/2)), Fr = (2 Pr eps)^(1/2)
    (Eq 4.11); enclosed (p0 from the mass, Eq 4.13).  Air only (Z = 0) with the
    convenient Q = S + 1, so H = T + 1 (Eq 4.16) and the quiescent initial
    state at T = 1 has H = 2 (Eq 4.17).  gravity=False and ny > 0 (periodic in
    x_2) give the one-dimensional conduction slab used as a pin; T0 (an
    interior array) replaces the uniform initial temperature; h_min (the
    smallest cell width of a stretched grid) sets the explicit limits of dt
    instead of 1/n."""
    ny = n if ny is None else ny
    prm = _base_params()
    Re = Ra ** 0.5
    Pr = 0.71
    bc_y = [WALL, WALL] if ny == n and gravity else [PERIODIC, PERIODIC]
    if not gravity and ny != n:
        bc_y = [PERIODIC, PERIODIC]
    prm.update(dim=2, n=[n, ny, 1], L=[1.0, float(ny) / n if bc_y[0] == PERIODIC else 1.0, 1.0],
               bc=[[WALL_T, WALL_T], bc_y, [PERIODIC, PERIODIC]], Re=Re, Pr=Pr,
               inv_Fr2=(1.0 / (2.0 * Pr * eps)) if gravity else 0.0, gamma=1.4, transport=1,
               sutherland_C=110.5 / 600.0, density_ratio=2.0, closed_system=1, inflow_Z=0.0, inflow_H=2.0,
               wall_H=[[2.0 + eps, 2.0 - eps], [0.0, 0.0], [0.0, 0.0]])
    x, y = cell_centres((n, ny), (1.0, prm["L"][1]))
    T = np.ones(x.shape) if T0 is None else np.asarray(T0, dtype=float)
    fields = dict(v=[np.zeros(x.shape), np.zeros(x.shape)], Z=np.zeros(x.shape), H=T + 1.0)
    # explicit diffusion limit at the hottest, lightest state: kappa(T_H), rho ~ 1/T_H
    TH = 1.0 + eps
    C = prm["sutherland_C"]
    kap_max = TH ** 1.5 * (1.0 + C) / (TH + C)
    h = 1.0 / n if h_min is None else float(h_min)
    lim = [h / 1.0, h * h * Re * min(1.0, Pr) * (1.0 / TH) / (4.0 * kap_max)]
    prm["dt"] = cfl * min(lim)
    return prm, None, fields
