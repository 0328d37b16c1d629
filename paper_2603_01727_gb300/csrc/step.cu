// Kernels of one predictor / corrector stage of the low-Mach step (everything
// but the Poisson solve).  Paper references: temporal scheme Eqs 3.1-3.19,
// collocated operators Eqs 3.20-3.26, boundary ghosts Eqs 3.43-3.46 and
// 3.27-3.28, penalisation Eqs 3.30-3.33, flame-sheet state Eqs 3.34-3.42.
//
// Layout: every cell field is a padded x-fastest array (one ghost layer per
// active direction); the interface flux F_j of direction j is stored at the
// padded index of the cell on the high side of the interface, so cell c has its
// low j-interface at c and its high one at c + s_j.  The pressure P and the
// Poisson right-hand side b are compact interior arrays.

#include <cmath>

#include "step.cuh"

namespace lm {

namespace {

constexpr int NT = kThreads;

__device__ __forceinline__ void padded_coords(const Geom& g, long long c, int q[3]) {
    q[0] = (int)(c % g.p[0]);
    long long r = c / g.p[0];
    q[1] = (int)(r % g.p[1]);
    q[2] = (int)(r / g.p[1]);
}

// Slab position (the two other padded coordinates) of padded cell c for direction d.
__device__ __forceinline__ long long slab_index(const Geom& g, int d, const int q[3]) {
    const int a = (d == 0) ? 1 : 0;
    const int b = (d == 2) ? 1 : 2;
    return (long long)q[a] + (long long)g.p[a] * q[b];
}

__device__ __forceinline__ long long compact_stride(const Geom& g, int d) {
    return d == 0 ? 1LL : (d == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
}

// ----------------------------------------------------------------------------
// Ghost cells of one direction d (Eqs 3.43-3.45; kappa: see Bnd docs).
// ----------------------------------------------------------------------------
__global__ void k_ghost(Geom g, Phys ph, const uint8_t* __restrict__ klo, const uint8_t* __restrict__ khi,
                        int d, int periodic, GhostJob job) {
    const int a = (d == 0) ? 1 : 0;
    const int b = (d == 2) ? 1 : 2;
    const long long nslab = (long long)g.p[a] * g.p[b];
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nslab) return;
    const int ca = (int)(q % g.p[a]);
    const int cb = (int)(q / g.p[a]);
    const long long base = (long long)ca * g.s[a] + (long long)cb * g.s[b];
    const int n = g.n[d];
    const long long sd = g.s[d];
    const long long i_g0 = base, i_1 = base + sd, i_n = base + (long long)n * sd, i_gh = base + (long long)(n + 1) * sd;
    for (int f = 0; f < job.nf; ++f) {
        double* x = job.f[f];
        const int what = job.what[f];
        if (periodic) {
            x[i_g0] = x[i_n];
            x[i_gh] = x[i_1];
            continue;
        }
        double dv;
        if (what == GW_Z) dv = ph.inflow_Z;
        else if (what == GW_H) dv = ph.inflow_H;
        else if (what == GW_KAPPA) dv = ph.kappa_in;
        else dv = ph.inflow_v[what - GW_V0];
        const bool vel = what >= GW_V0;
        const bool normal = vel && (what - GW_V0 == d);
        for (int side = 0; side < 2; ++side) {
            const long long ig = side ? i_gh : i_g0;
            const long long ia = side ? i_n : i_1;
            const int kind = side ? khi[q] : klo[q];
            const double adj = x[ia];
            double out;
            if (kind == BC_INFLOW) out = 2.0 * dv - adj;
            else if (kind == BC_OUTFLOW) out = adj;
            else if (kind == BC_WALL) out = vel ? -adj : adj;
            else out = normal ? -adj : adj;  // BC_SLIP
            x[ig] = out;
        }
    }
}

// ----------------------------------------------------------------------------
// Flame-sheet state relation (Eqs 3.41-3.42 with the level translation, 2.49,
// 2.50) at the interior cells; block partials of sum(1/T) for Eq 2.40.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double temperature(const Phys& ph, double z, double h) {
    const double x = ph.k * (z - 1.0);
    const double ax = fabs(x);
    // ln cosh x + ln 2 = |x| + log1p(exp(-2|x|)): Eq 3.41 minus its level shift
    const double F = (-(ph.S + 1.0) * (ax + log1p(exp(-2.0 * ax))) / ph.k + (ph.S - 1.0) * (z - 1.0)) /
                     (2.0 * ph.S);
    return ph.Q / (ph.S + 1.0) * (F + h);
}

__global__ void k_state(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ H,
                        double* __restrict__ T, double* __restrict__ rho, double* __restrict__ kap,
                        double* __restrict__ part, int* status, double* sc, int p0_slot) {
    __shared__ double sm[NT / 32];
    double acc = 0.0;
    int bad = 0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        double Tv, kv;
        if (ph.incompressible) {
            Tv = 1.0;
            kv = 1.0;
        } else {
            Tv = temperature(ph, Z[c], H[c]);
            kv = pow(Tv, ph.sigma);
        }
        T[c] = Tv;
        kap[c] = kv;
        if (!ph.closed) rho[c] = ph.incompressible ? 1.0 : 1.0 / Tv;
        acc += 1.0 / Tv;
        if (!(Tv > 0.0) || !(Tv < 1e300)) bad = 1;
    }
    if (bad) atomicOr(status, ST_NAN);
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
    if (blockIdx.x == 0 && threadIdx.x == 0 && !ph.closed) sc[p0_slot] = 1.0;
}

// Enclosed system: p0 = m / (sum(1/T) dV) (Eq 2.40), rho = p0 / T (Eq 2.49).
__global__ void k_density(Geom g, const double* __restrict__ T, double* __restrict__ rho,
                          const double* __restrict__ part, int np, double* sc, int p0_slot) {
    __shared__ double sm[NT / 32];
    const double s = sum_partials<NT>(part, np, sm);
    const double p0 = sc[SC_MASS] / (s * g.dV);
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        rho[c] = p0 / T[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[p0_slot] = p0;
}

// ----------------------------------------------------------------------------
// Residuals at one level and the AB2 / AM2 combination (Eqs 3.1-3.4, 3.7-3.8,
// 3.10, 3.12-3.13, 3.16, 3.18; convection Eq 3.26; penalisation Eqs 3.30-3.32).
// ----------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(NT) k_residual(Geom g, Phys ph, ResidArgs a) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    int ct[3];
    interior_coords(g, t, ct);
    (void)ct;

    // dp0/dt for the H source (Eqs 3.5, 3.14)
    const double p0dot =
        (a.wden != 0.0) ? (a.w0 * a.sc[a.p0a] + a.w1 * a.sc[a.p0b] + a.w2 * a.sc[a.p0c]) / a.wden : 0.0;

    const double rho_c = a.rho[c];
    const double kap_c = a.kap[c];
    const double Zc = a.Z[c], Hc = a.H[c];

    // scalar convection (Eq 3.26b) and diffusion div(kappa grad .)
    double convZ = 0.0, convH = 0.0, difZ = 0.0, difH = 0.0;
    double kf_lo[DIM], kf_hi[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const double ih = g.ih[j];
        const double Flo = a.F[j][c], Fhi = a.F[j][c + s];
        kf_lo[j] = 0.5 * (a.kap[c - s] + kap_c);
        kf_hi[j] = 0.5 * (kap_c + a.kap[c + s]);
        const double dZlo = (Zc - a.Z[c - s]) * ih, dZhi = (a.Z[c + s] - Zc) * ih;
        const double dHlo = (Hc - a.H[c - s]) * ih, dHhi = (a.H[c + s] - Hc) * ih;
        convZ += 0.5 * (Flo * dZlo + Fhi * dZhi);
        convH += 0.5 * (Flo * dHlo + Fhi * dHhi);
        difZ += (kf_hi[j] * dZhi - kf_lo[j] * dZlo) * ih;
        difH += (kf_hi[j] * dHhi - kf_lo[j] * dHlo) * ih;
    }

    // momentum: convection Eq 3.26a, viscous stress Eq 2.46 on the interfaces
    double Rv[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const double* vi = a.v[i];
        double conv = 0.0, visc = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const double ih = g.ih[j];
            const double Flo = a.F[j][c], Fhi = a.F[j][c + s];
            conv += (Fhi * (0.5 * (vi[c] + vi[c + s])) - Flo * (0.5 * (vi[c - s] + vi[c]))) * ih;
            double tau_f[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const long long ca = side ? c : c - s;   // cell below the interface
                const long long cb = ca + s;             // cell above
                const double kf = side ? kf_hi[j] : kf_lo[j];
                const double dvi = (vi[cb] - vi[ca]) * ih;
                double dvj;
                if (i == j) {
                    dvj = dvi;
                } else {
                    const long long si = g.s[i];
                    const double* vj = a.v[j];
                    const double da = (vj[ca + si] - vj[ca - si]) * (0.5 * g.ih[i]);
                    const double db = (vj[cb + si] - vj[cb - si]) * (0.5 * g.ih[i]);
                    dvj = 0.5 * (da + db);
                }
                double tau = kf * (dvi + dvj);
                if (i == j) {
                    double div = (a.v[j][cb] - a.v[j][ca]) * ih;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        if (k == j) continue;
                        const long long sk = g.s[k];
                        const double* vk = a.v[k];
                        const double da = (vk[ca + sk] - vk[ca - sk]) * (0.5 * g.ih[k]);
                        const double db = (vk[cb + sk] - vk[cb - sk]) * (0.5 * g.ih[k]);
                        div = div + 0.5 * (da + db);
                    }
                    tau = tau - (2.0 / 3.0) * kf * div;
                }
                tau_f[side] = tau;
            }
            visc += (tau_f[1] - tau_f[0]) * ih;
        }
        double R = -conv + ph.PrPe * visc;
        if (i == 1 && ph.inv_Fr2 != 0.0) R = R + ph.inv_Fr2 * (1.0 - rho_c);          // Eq 3.8b
        if (a.ibm && a.chi[c]) R = R - ph.PrPe * a.inv_Da * kap_c * (vi[c] - a.vib[i][c]);  // Eq 3.30
        Rv[i] = R;
    }

    // Lewis and N coefficients (Eq 3.35)
    double Le = ph.Le_O, Nn = ph.N_O;
    if (ph.Le_F != ph.Le_O) {
        const double th = 0.5 * (1.0 + tanh(ph.k * (Zc - 1.0)));
        Le = (ph.Le_F - ph.Le_O) * th + ph.Le_O;
        Nn = (ph.N_F - ph.N_O) * th + ph.N_O;
    }
    const double Pe = ph.Pe;
    double bZ = -convZ + difZ / (Le * Pe);
    double bH = -convH + difH / Pe + ph.zeta * p0dot + Nn * difZ / Pe;
    if (a.ibm && a.chi[c]) {
        bZ = bZ - kap_c * (Zc - a.Z_ib) / (Le * Pe) * a.inv_Da;                 // Eq 3.31
        bH = bH - kap_c * (Hc - a.H_ib) / Pe * a.inv_Da;                         // Eq 3.32
    }
    const double RZ = bZ / rho_c;
    const double RH = bH / rho_c;

    // combination
    const double dt = a.dt;
    const double rb = a.rhob[c];
    if (a.mode == MODE_CORR) {
#pragma unroll
        for (int i = 0; i < DIM; ++i) a.mo[i][c] = rb * a.vb[i][c] + 0.5 * dt * (Rv[i] + a.Rrd[i][c]);
        a.Zo[c] = a.Zb[c] + 0.5 * dt * (RZ + a.Rrd[3][c]);
        a.Ho[c] = a.Hb[c] + 0.5 * dt * (RH + a.Rrd[4][c]);
    } else {
        const bool ab2 = (a.mode == MODE_PRED_AB2);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            const double cv = ab2 ? (1.5 * Rv[i] - 0.5 * a.Rrd[i][c]) : Rv[i];
            a.Rst[i][c] = Rv[i];
            a.mo[i][c] = rb * a.vb[i][c] + dt * cv;
        }
        const double cZ = ab2 ? (1.5 * RZ - 0.5 * a.Rrd[3][c]) : RZ;
        const double cH = ab2 ? (1.5 * RH - 0.5 * a.Rrd[4][c]) : RH;
        a.Rst[3][c] = RZ;
        a.Rst[4][c] = RH;
        a.Zo[c] = a.Zb[c] + dt * cZ;
        a.Ho[c] = a.Hb[c] + dt * cH;
    }
}

// ----------------------------------------------------------------------------
// Interface mass fluxes of the provisional momentum (first term of Eq 3.23) and
// block partials of the global mass balance (Eq 3.24 + S_m, Eq 3.33).
// ----------------------------------------------------------------------------
template <int DIM>
__global__ void k_face_flux(Geom g, Phys ph, Bnd bnd, FluxArgs a) {
    __shared__ double sm[NT / 32];
    const double rho_in = ph.incompressible ? 1.0 : a.sc[a.p0_slot] / ph.rho_in_T;
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        int ct[3], q[3];
        interior_coords(g, t, ct);
        padded_coords(g, c, q);
        if (a.correct) {
            const double drho = (a.bdf_c0 * a.rho_new[c] + a.bdf_c1 * a.rho_n[c] +
                                 (a.bdf_c2 != 0.0 ? a.bdf_c2 * a.rho_prev[c] : 0.0)) / a.bdf_den;
            const double Sm = a.Sm ? a.Sm[c] : 0.0;
            acc += (drho - Sm) * g.dV;
        }
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const int n = g.n[j];
            const double* m = a.mom[j];
            const double dA = g.dV * g.ih[j];
            if (ct[j] > 0 || g.periodic[j]) {
                const long long cl = (ct[j] > 0) ? c - s : c + (long long)(n - 1) * s;
                a.F[j][c] = 0.5 * (m[cl] + m[c]);
            } else {
                const int kind = bnd.kind[j][0][slab_index(g, j, q)];
                const double val = (kind == BC_INFLOW) ? rho_in * ph.inflow_v[j] : (kind == BC_OUTFLOW) ? m[c] : 0.0;
                a.F[j][c] = val;
                acc += -val * dA;
            }
            if (ct[j] == n - 1) {
                if (g.periodic[j]) {
                    a.F[j][c + s] = 0.5 * (m[c] + m[c - (long long)(n - 1) * s]);
                } else {
                    const int kind = bnd.kind[j][1][slab_index(g, j, q)];
                    const double val =
                        (kind == BC_INFLOW) ? rho_in * ph.inflow_v[j] : (kind == BC_OUTFLOW) ? m[c] : 0.0;
                    a.F[j][c + s] = val;
                    acc += val * dA;
                }
            }
        }
    }
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) a.part[blockIdx.x] = acc;
}

// Uniform shift of the outflow fluxes closing the mass balance, then
// b = d_t rho + sum_j delta_1 F_j / delta_1 x_j - S_m  (Eq 3.24 with S_m).
template <int DIM>
__global__ void k_rhs(Geom g, Bnd bnd, FluxArgs a, int np) {
    __shared__ double sm[NT / 32];
    const double total = sum_partials<NT>(a.part, np, sm);
    const double area = a.sc[SC_OUT_AREA];
    const double shift = (area > 0.0) ? -total / area : 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        int ct[3], q[3];
        interior_coords(g, t, ct);
        padded_coords(g, c, q);
        const double drho = (a.bdf_c0 * a.rho_new[c] + a.bdf_c1 * a.rho_n[c] +
                             (a.bdf_c2 != 0.0 ? a.bdf_c2 * a.rho_prev[c] : 0.0)) / a.bdf_den;
        const double Sm = a.Sm ? a.Sm[c] : 0.0;
        double b = drho - Sm;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            if (!g.periodic[j]) {
                if (ct[j] == 0 && bnd.kind[j][0][slab_index(g, j, q)] == BC_OUTFLOW) a.F[j][c] = a.F[j][c] - shift;
                if (ct[j] == g.n[j] - 1 && bnd.kind[j][1][slab_index(g, j, q)] == BC_OUTFLOW)
                    a.F[j][c + s] = a.F[j][c + s] + shift;
            }
            b = b + (a.F[j][c + s] - a.F[j][c]) * g.ih[j];
        }
        a.b[t] = b;
    }
}

// ----------------------------------------------------------------------------
// Projection: F_j = Ft_j - delta_1 P / delta_1 x_j on the interfaces that carry
// a pressure term (Eq 3.23), v_i = (rho v~_i - delta_2 P / delta_2 x_i) / rho
// (Eq 3.25) with P ghosts by quadratic extrapolation (Eqs 3.27-3.28).
// ----------------------------------------------------------------------------
template <int DIM>
__global__ void k_project(Geom g, ProjArgs a) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    int ct[3];
    interior_coords(g, t, ct);
    const double Pc = a.P[t];
    const double rho = a.rho[c];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const long long st = compact_stride(g, j);
        const int n = g.n[j];
        const double ih = g.ih[j];
        double Pm, Pp;
        if (ct[j] > 0) Pm = a.P[t - st];
        else if (g.periodic[j]) Pm = a.P[t + (long long)(n - 1) * st];
        else Pm = a.eA * Pc + a.eB * a.P[t + st] + a.eC * a.P[t + 2 * st];
        if (ct[j] < n - 1) Pp = a.P[t + st];
        else if (g.periodic[j]) Pp = a.P[t - (long long)(n - 1) * st];
        else Pp = a.eA * Pc + a.eB * a.P[t - st] + a.eC * a.P[t - 2 * st];
        if (ct[j] > 0 || g.periodic[j]) a.F[j][c] = a.F[j][c] - (Pc - Pm) * ih;
        if (ct[j] == n - 1 && g.periodic[j]) a.F[j][c + s] = a.F[j][c + s] - (Pp - Pc) * ih;
        a.v[j][c] = (a.mom[j][c] - (Pp - Pm) / (2.0 * g.h[j])) / rho;
    }
}

__global__ void k_momentum(Geom g, const double* __restrict__ rho, const double* v0, const double* v1,
                           const double* v2, double* m0, double* m1, double* m2) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    const double r = rho[c];
    m0[c] = r * v0[c];
    m1[c] = r * v1[c];
    if (g.dim == 3) m2[c] = r * v2[c];
}

__global__ void k_sum_interior(Geom g, const double* __restrict__ x, double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT)
        acc += x[pad_index(g, t)];
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_store_sum(const double* part, int np, double scale, double* dst) {
    __shared__ double sm[NT / 32];
    const double s = sum_partials<NT>(part, np, sm);
    if (threadIdx.x == 0) *dst = s * scale;
}

__global__ void k_rotate_p0(double* sc) {
    sc[SC_P0_NM2] = sc[SC_P0_NM1];
    sc[SC_P0_NM1] = sc[SC_P0_N];
    sc[SC_P0_N] = sc[SC_P0_NEW];
}

__global__ void k_copy_scalar(const double* src, double* dst, int n) {
    if (threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
}

__global__ void k_or_status(const int* flag, int bit, int* status) {
    if (*flag) atomicOr(status, bit);
}

// ----------------------------------------------------------------------------
// Immersed body (set-up): shifted mask, v_ib, U profile, S_m (Eqs 3.30-3.33,
// 4.19-4.20).  Evaluated on every padded cell (ghosts included: the inlet's
// wall override reads the mask of the first interior layer only).
// ----------------------------------------------------------------------------
__global__ void k_ibm_cells(Geom g, IbmDev b, uint8_t* chi, double* vib0, double* vib1, double* vib2,
                            double* U, double* Sm) {
    const long long c = (long long)blockIdx.x * NT + threadIdx.x;
    if (c >= g.npad) return;
    int q[3];
    padded_coords(g, c, q);
    double x[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < g.dim; ++d) x[d] = ((double)q[d] - 0.5) * g.h[d];
    double* vib[3] = {vib0, vib1, vib2};
    bool interior = true;
    for (int d = 0; d < g.dim; ++d)
        if (q[d] < 1 || q[d] > g.n[d]) interior = false;
    if (b.kind == 2) {  // sphere / circle, radial ejection
        double r2 = 0.0;
        for (int d = 0; d < g.dim; ++d) r2 += (x[d] - b.c[d]) * (x[d] - b.c[d]);
        const double r = sqrt(r2);
        const double m = (r - b.radius <= b.s) ? 1.0 : 0.0;
        const double rs = (r > 0.0) ? r : 1.0;
        chi[c] = (uint8_t)(m != 0.0);
        for (int d = 0; d < g.dim; ++d) vib[d][c] = m * b.U_b * (x[d] - b.c[d]) / rs;
        Sm[c] = interior ? m * (double)(g.dim - 1) * b.rho_b * b.U_b / rs : 0.0;
        U[c] = 0.0;
    } else {  // slot ejecting through its +x_2 face
        double qd[3], out2 = 0.0, qmax = -1e300;
        for (int d = 0; d < g.dim; ++d) {
            qd[d] = fabs(x[d] - b.c[d]) - b.half[d];
            const double mq = qd[d] > 0.0 ? qd[d] : 0.0;
            out2 = out2 + mq * mq;
            qmax = qd[d] > qmax ? qd[d] : qmax;
        }
        const double sd = sqrt(out2) + (qmax < 0.0 ? qmax : 0.0);
        const double m = (sd <= b.s) ? 1.0 : 0.0;
        double prof = 1.0;
        for (int d = 0; d < g.dim; ++d) {
            if (d == 1) continue;
            const double r = (x[d] - b.c[d]) / (b.half[d] + b.s);
            prof = prof * (1.0 - r * r);
        }
        prof = prof > 0.0 ? prof : 0.0;
        if (b.n_profile > 0) {
            const double lo = b.c[0] - b.half[0] - b.s, hi = b.c[0] + b.half[0] + b.s;
            double mod;
            if (x[0] <= lo) mod = b.profile[0];
            else if (x[0] >= hi) mod = b.profile[b.n_profile - 1];
            else {
                const double pos = (x[0] - lo) / (hi - lo) * (double)(b.n_profile - 1);
                int i0 = (int)floor(pos);
                if (i0 > b.n_profile - 2) i0 = b.n_profile - 2;
                const double fr = pos - (double)i0;
                mod = b.profile[i0] + fr * (b.profile[i0 + 1] - b.profile[i0]);
            }
            prof = prof * mod;
        }
        const double Uv = b.U_b * prof;
        const double ylo = b.c[1] - b.half[1] - b.s, yhi = b.c[1] + b.half[1] + b.s;
        chi[c] = (uint8_t)(m != 0.0);
        for (int d = 0; d < g.dim; ++d) vib[d][c] = 0.0;
        vib[1][c] = m * Uv * (x[1] - ylo) / (yhi - ylo);
        U[c] = Uv;
        Sm[c] = 0.0;
    }
}

// Slot source per x_2-column: S_m = rho_b U / (n_col h_2) on the masked cells.
__global__ void k_slot_source(Geom g, IbmDev b, const uint8_t* chi, const double* U, double* Sm) {
    const long long col = (long long)blockIdx.x * NT + threadIdx.x;
    const long long ncol = (long long)g.n[0] * (g.dim == 3 ? g.n[2] : 1);
    if (col >= ncol) return;
    const int i = (int)(col % g.n[0]) + 1;
    const int k = (g.dim == 3) ? (int)(col / g.n[0]) + 1 : 0;
    const long long base = (long long)i + (long long)k * g.s[2];
    int cnt = 0;
    for (int j = 1; j <= g.n[1]; ++j) cnt += chi[base + (long long)j * g.s[1]];
    const double nc = cnt > 0 ? (double)cnt : 1.0;
    for (int j = 1; j <= g.n[1]; ++j) {
        const long long c = base + (long long)j * g.s[1];
        Sm[c] = (double)chi[c] * b.rho_b * U[c] / (nc * g.h[1]);
    }
}

// Boundary kinds per slab position; an inflow face over a masked first
// interior cell is a wall.  Partials count outflow interface area.
__global__ void k_bkinds(Geom g, int d, int bc_lo, int bc_hi, const uint8_t* chi, uint8_t* klo, uint8_t* khi,
                         double* part) {
    __shared__ double sm[NT / 32];
    const int a = (d == 0) ? 1 : 0;
    const int b = (d == 2) ? 1 : 2;
    const long long nslab = (long long)g.p[a] * g.p[b];
    double area = 0.0;
    const double dA = g.dV * g.ih[d];
    for (long long q = (long long)blockIdx.x * NT + threadIdx.x; q < nslab; q += (long long)gridDim.x * NT) {
        const int ca = (int)(q % g.p[a]);
        const int cb = (int)(q / g.p[a]);
        const long long base = (long long)ca * g.s[a] + (long long)cb * g.s[b];
        int klo_v = bc_lo, khi_v = bc_hi;
        if (chi) {
            if (klo_v == BC_INFLOW && chi[base + g.s[d]]) klo_v = BC_WALL;
            if (khi_v == BC_INFLOW && chi[base + (long long)g.n[d] * g.s[d]]) khi_v = BC_WALL;
        }
        klo[q] = (uint8_t)klo_v;
        khi[q] = (uint8_t)khi_v;
        const bool inner_a = (g.dim == 2 && a == 2) || (ca >= 1 && ca <= g.n[a]);
        const bool inner_b = (g.dim == 2 && b == 2) || (cb >= 1 && cb <= g.n[b]);
        if (inner_a && inner_b) area += ((klo_v == BC_OUTFLOW) + (khi_v == BC_OUTFLOW)) * dA;
    }
    area = block_sum<NT>(area, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = area;
}

// Pack interior cells (face_dir < 0) or the interfaces of direction face_dir
// of a padded array into a compact x-fastest array.
__global__ void k_pack(Geom g, const double* __restrict__ src, double* __restrict__ dst, int face_dir) {
    long long m[3] = {g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1};
    if (face_dir >= 0) m[face_dir] += 1;
    const long long tot = m[0] * m[1] * m[2];
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= tot) return;
    const long long i = t % m[0], j = (t / m[0]) % m[1], k = t / (m[0] * m[1]);
    const long long kz = (g.dim == 3) ? k + 1 : 0;
    dst[t] = src[(i + 1) + (j + 1) * g.s[1] + kz * g.s[2]];
}

__global__ void k_unpack(Geom g, const double* __restrict__ src, double* __restrict__ dst) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    dst[pad_index(g, t)] = src[t];
}

__global__ void k_u8_to_double(Geom g, const uint8_t* __restrict__ src, double* __restrict__ dst) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    dst[t] = (double)src[pad_index(g, t)];
}

}  // namespace

int reduce_grid(const Geom& g) { return reduce_blocks(g.ncell); }

void launch_ghost(const Geom& g, const Bnd& bnd, const Phys& ph, const GhostJob& job, cudaStream_t s,
                  int* launches) {
    for (int d = 0; d < g.dim; ++d) {
        const int a = (d == 0) ? 1 : 0;
        const int b = (d == 2) ? 1 : 2;
        const long long nslab = (long long)g.p[a] * g.p[b];
        k_ghost<<<blocks_for(nslab), NT, 0, s>>>(g, ph, bnd.kind[d][0], bnd.kind[d][1], d, g.periodic[d], job);
        ++*launches;
    }
}

void launch_state(const Geom& g, const Phys& ph, const double* Z, const double* H, double* T, double* rho,
                  double* kap, double* sc, int p0_slot, double* part, int* status, cudaStream_t s,
                  int* launches) {
    const int rb = reduce_grid(g);
    k_state<<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, part, status, sc, p0_slot);
    ++*launches;
    if (ph.closed) {
        k_density<<<rb, NT, 0, s>>>(g, T, rho, part, rb, sc, p0_slot);
        ++*launches;
    }
}

void launch_residual(const Geom& g, const Phys& ph, const ResidArgs& a, cudaStream_t s, int* launches) {
    if (g.dim == 3)
        k_residual<3><<<blocks_for(g.ncell), NT, 0, s>>>(g, ph, a);
    else
        k_residual<2><<<blocks_for(g.ncell), NT, 0, s>>>(g, ph, a);
    ++*launches;
}

void launch_flux_rhs(const Geom& g, const Phys& ph, const Bnd& bnd, const FluxArgs& a, cudaStream_t s,
                     int* launches) {
    const int rb = reduce_grid(g);
    if (g.dim == 3)
        k_face_flux<3><<<rb, NT, 0, s>>>(g, ph, bnd, a);
    else
        k_face_flux<2><<<rb, NT, 0, s>>>(g, ph, bnd, a);
    ++*launches;
    if (!a.correct) return;
    if (g.dim == 3)
        k_rhs<3><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    else
        k_rhs<2><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    ++*launches;
}

void launch_project(const Geom& g, const ProjArgs& a, cudaStream_t s, int* launches) {
    if (g.dim == 3)
        k_project<3><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
    else
        k_project<2><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
    ++*launches;
}

void launch_momentum(const Geom& g, const double* rho, double* const v[3], double* mom[3], cudaStream_t s,
                     int* launches) {
    k_momentum<<<blocks_for(g.ncell), NT, 0, s>>>(g, rho, v[0], v[1], v[2], mom[0], mom[1], mom[2]);
    ++*launches;
}

void launch_sum(const Geom& g, const double* x, double* part, cudaStream_t s, int* launches) {
    k_sum_interior<<<reduce_grid(g), NT, 0, s>>>(g, x, part);
    ++*launches;
}

void launch_store_sum(const double* part, int np, double scale, double* dst, cudaStream_t s, int* launches) {
    k_store_sum<<<1, NT, 0, s>>>(part, np, scale, dst);
    ++*launches;
}

void launch_rotate_p0(double* sc, cudaStream_t s, int* launches) {
    k_rotate_p0<<<1, 1, 0, s>>>(sc);
    ++*launches;
}

void launch_copy_scalar(const double* src, double* dst, int n, cudaStream_t s, int* launches) {
    k_copy_scalar<<<1, 32, 0, s>>>(src, dst, n);
    ++*launches;
}

void launch_or_status(const int* src_flag, int bit, int* status, cudaStream_t s, int* launches) {
    k_or_status<<<1, 1, 0, s>>>(src_flag, bit, status);
    ++*launches;
}

void launch_ibm(const Geom& g, const IbmDev& b, uint8_t* chi, double* vib[3], double* U, double* Sm,
                cudaStream_t s) {
    k_ibm_cells<<<blocks_for(g.npad), NT, 0, s>>>(g, b, chi, vib[0], vib[1], vib[2], U, Sm);
    if (b.kind == 1) {
        const long long ncol = (long long)g.n[0] * (g.dim == 3 ? g.n[2] : 1);
        k_slot_source<<<blocks_for(ncol), NT, 0, s>>>(g, b, chi, U, Sm);
    }
}

void launch_bkinds(const Geom& g, const int bc[3][2], const uint8_t* chi, uint8_t* kind[3][2], double* part,
                   double* sc, cudaStream_t s) {
    // sum of the outflow area over the directions, accumulated through partial buffers
    int np_total = 0;
    for (int d = 0; d < g.dim; ++d) {
        const int a = (d == 0) ? 1 : 0;
        const int b = (d == 2) ? 1 : 2;
        const long long nslab = (long long)g.p[a] * g.p[b];
        int nb = blocks_for(nslab);
        if (nb > 256) nb = 256;
        k_bkinds<<<nb, NT, 0, s>>>(g, d, bc[d][0], bc[d][1], chi, kind[d][0], kind[d][1], part + np_total);
        np_total += nb;
    }
    k_store_sum<<<1, NT, 0, s>>>(part, np_total, 1.0, sc + SC_OUT_AREA);
}

void launch_pack(const Geom& g, const double* padded, double* compact, int face_dir, cudaStream_t s) {
    long long m[3] = {g.n[0], g.n[1], g.dim == 3 ? g.n[2] : 1};
    if (face_dir >= 0) m[face_dir] += 1;
    k_pack<<<blocks_for(m[0] * m[1] * m[2]), NT, 0, s>>>(g, padded, compact, face_dir);
}

void launch_unpack(const Geom& g, const double* compact, double* padded, cudaStream_t s) {
    k_unpack<<<blocks_for(g.ncell), NT, 0, s>>>(g, compact, padded);
}

void launch_u8_to_double(const Geom& g, const uint8_t* padded, double* compact, cudaStream_t s) {
    k_u8_to_double<<<blocks_for(g.ncell), NT, 0, s>>>(g, padded, compact);
}

}  // namespace lm
