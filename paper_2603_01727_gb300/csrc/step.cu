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
#include <cstdlib>
#include <cstring>

#include "step.cuh"

namespace lm {

namespace {

constexpr int NT = kThreads;

__device__ __forceinline__ void padded_coords(const Geom& g, long long c, int q[3]) {
    const unsigned cc = (unsigned)c;
    const unsigned r = divu32(cc, g.dp0);
    const unsigned k = divu32(r, g.dp1);
    q[0] = (int)(cc - r * (unsigned)g.p[0]);
    q[1] = (int)(r - k * (unsigned)g.p[1]);
    q[2] = (int)k;
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
// Ghost value of field `what` across side `side` of direction d (Eqs
// 3.43-3.45): Dirichlet sides mirror about the prescribed face value (inflow,
// isothermal wall), zero-gradient sides copy, walls reverse the velocity,
// symmetry planes its normal component.
__device__ __forceinline__ double ghost_value(const Phys& ph, int what, int d, int side, int kind, double adj) {
    const bool vel = what >= GW_V0;
    const bool normal = vel && (what - GW_V0 == d);
    if (kind == BC_WALL_T) {
        if (vel) return -adj;
        const double dv = (what == GW_Z) ? ph.inflow_Z : (what == GW_H) ? ph.wall_H[d][side] : ph.kap_wall[d][side];
        return 2.0 * dv - adj;
    }
    double dv;
    if (what == GW_Z) dv = ph.inflow_Z;
    else if (what == GW_H) dv = ph.inflow_H;
    else if (what == GW_KAPPA) dv = ph.kappa_in;
    else dv = ph.inflow_v[what - GW_V0];
    if (kind == BC_INFLOW) return 2.0 * dv - adj;
    if (kind == BC_OUTFLOW) return adj;
    if (kind == BC_WALL) return vel ? -adj : adj;
    return normal ? -adj : adj;   // BC_SLIP
}

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
        for (int side = 0; side < 2; ++side) {
            const long long ig = side ? i_gh : i_g0;
            const long long ia = side ? i_n : i_1;
            const int kind = side ? khi[q] : klo[q];
            x[ig] = ghost_value(ph, what, d, side, kind, x[ia]);
        }
    }
}

// ----------------------------------------------------------------------------
// Ghost fill fused into the kernel that produces a field: the thread that
// writes interior cell c (padded coordinates q) also writes every ghost cell
// whose value k_ghost's direction-by-direction fill (d = 0, 1, 2) would take
// from c, composing the per-direction maps in the same order (a corner is the
// d = 1 map of the d = 0 ghost).  Same formulas, so the same values.
// ----------------------------------------------------------------------------
// vals[f]: the value just written to job.f[f] at interior cell q.
__device__ __forceinline__ void fill_ghosts_of(const Geom& g, const Phys& ph, const Bnd& bnd, const GhostJob& job,
                                               const int q[3], const double* vals) {
    int opt[3][3], nopt[3] = {1, 1, 1};
    bool any = false;
    for (int d = 0; d < 3; ++d) {
        opt[d][0] = 0;
        if (d >= g.dim) continue;
        const int n = g.n[d];
        const bool per = g.periodic[d];
        if (per ? (q[d] == n) : (q[d] == 1)) opt[d][nopt[d]++] = 1;   // source of the low ghost
        if (per ? (q[d] == 1) : (q[d] == n)) opt[d][nopt[d]++] = 2;   // source of the high ghost
        any = any || nopt[d] > 1;
    }
    if (!any) return;
    for (int i2 = 0; i2 < nopt[2]; ++i2)
        for (int i1 = 0; i1 < nopt[1]; ++i1)
            for (int i0 = 0; i0 < nopt[0]; ++i0) {
                const int o[3] = {opt[0][i0], opt[1][i1], opt[2][i2]};
                if (o[0] == 0 && o[1] == 0 && o[2] == 0) continue;
                for (int f = 0; f < job.nf; ++f) {
                    double v = vals[f];
                    int qq[3] = {q[0], q[1], q[2]};
                    for (int d = 0; d < g.dim; ++d) {
                        if (o[d] == 0) continue;
                        const int side = o[d] - 1;
                        if (!g.periodic[d])
                            v = ghost_value(ph, job.what[f], d, side, bnd.kind[d][side][slab_index(g, d, qq)], v);
                        qq[d] = side ? g.n[d] + 1 : 0;
                    }
                    job.f[f][(long long)qq[0] + (long long)qq[1] * g.s[1] + (long long)qq[2] * g.s[2]] = v;
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
    // ln cosh x + ln 2 = |x| + log1p(exp(-2|x|)): Eq 3.41 minus its level shift,
    // with the constant factors folded: T = cT (cA (|x| + L) + cB (Z - 1) + H)
    return ph.cT * (ph.cA * (ax + log1p(exp(-2.0 * ax))) + ph.cB * (z - 1.0) + h);
}

// Mixed precision: the bounded term L = log1p(exp(-2|x|)), x = k (Z - 1), is
// evaluated in FP64 inside the stoichiometric band |x| < kStoichBand and in
// FP32 outside it, where L < 2.3e-6 and its FP32 rounding (< 1.4e-13 in T) stays
// far below what the BDF density rate (which divides T differences by dt)
// would amplify into the pressure.  The affine part, whose cancellation (F + H
// is ~18x smaller than F in air) needs FP64, is FP64 everywhere.
constexpr double kStoichBand = 6.5;

// The band test and the FP32 argument use the leading 24 bits of |x| taken
// from its bit pattern (FF split), and the FP32 value returns through bit
// operations: the FP64 pipe (1/64 of the FP32 rate) sees only the affine part.
__device__ __forceinline__ double temperature_mixed(const Phys& ph, double z, double h) {
    const double zm1 = z - 1.0;
    const double ax = fabs(ph.k * zm1);
    const float axf = FF(ax).hi;
    double L;
    if (axf < (float)kStoichBand) L = log1p(exp(-2.0 * ax));
    else L = f2d_bits(log1pf(expf(-2.0f * axf)));
    return ph.cT * (ph.cA * (ax + L) + ph.cB * zm1 + h);
}

// 1/T to FP64 accuracy: an FP32 reciprocal of the split's leading part, one
// FP32 Newton step against both parts (y to ~2^-24 relative), then one FP64
// Newton step (y <- y + y (1 - T y) squares the error: ~4e-15).  The FP32
// operand and result cross by bit operations.
__device__ __forceinline__ double recip_newton(double T) {
    const FF t(T);
    float y = __frcp_rn(t.hi);
    y = fmaf(y, fmaf(-t.lo, y, fmaf(-t.hi, y, 1.0f)), y);
    const double yd = f2d_bits(y);
    return fma(yd, fma(-T, yd, 1.0), yd);
}

// kappa = T^sigma (Eq 2.50) in the mixed path.  For the paper's sigma = 7/10:
// y0 = powf(T, 0.7) (FP32), then with delta = T^7 / y0^10 - 1 (~1e-7) the exact
// y = y0 (1 + delta)^(1/10) = y0 (1 + delta/10 - 0.045 delta^2 + O(delta^3)).
// T^7 and y0^10 (repeated squaring) and their quotient are float-float (about
// 2^-46 relative per operation, eight of them: delta to ~1e-13 and kappa to
// ~1e-14 relative, measured 2e-14 against the FP64 pow); the
// correction y0 (delta/10 - 0.045 delta^2), ~1e-8 of y0, is FP32, and y0 plus
// it is exact as a float pair.  Only the final pair-to-double sum uses the
// FP64 pipe, so kappa carries no FP32 rounding noise into the diffusion-flux
// differences at a fraction of an FP64 pow's cost.  Other exponents use the
// FP64 pow.
__device__ __forceinline__ double kappa_mixed(const Phys& ph, double T) {
    if (ph.transport != 0 || !ph.sigma_is_07) return kappa_of(ph, T);
    const FF t(T);
    const float y0 = powf(t.hi, 0.7f);
    const FF t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
    const FF y(y0, 0.f);
    const FF y2 = y * y, y4 = y2 * y2, y8 = y4 * y4, y10 = y8 * y2;
    const float delta = (t7 / y10 - FF(1.f, 0.f)).hi;
    const FF k = ff_fast_two_sum(y0, y0 * (delta * fmaf(-0.045f, delta, 0.1f)));
    return f2d_bits(k.hi) + f2d_bits(k.lo);
}

// T > 0 and T < 1e300 (not NaN) from the bit pattern: positive doubles order
// as their bits, so no FP64 comparison is issued.
__device__ __forceinline__ bool temperature_ok(double T) {
    const long long b = __double_as_longlong(T);
    return b > 0 && b < 0x7e37e43c8800759cLL;   // the bits of 1e300
}

// State relation at one cell (Eqs 2.49-2.51): T and kappa from Z, H (kappa's
// ghost copies too when kj names them), rho = 1/T for an open system (p0 = 1,
// Eq 2.41); returns 1/T and sets bad on an out-of-range temperature.
template <bool MIXED>
__device__ __forceinline__ double state_cell(const Geom& g, const Phys& ph, const double* __restrict__ Z,
                                             const double* __restrict__ H, double* __restrict__ T,
                                             double* __restrict__ rho, double* __restrict__ kap, const Bnd& bnd,
                                             const GhostJob& kj, int kap_ghosts, long long c, int& bad) {
    double Tv, kv, iT;
    if (ph.incompressible) {
        Tv = 1.0;
        kv = 1.0;
        iT = 1.0;
    } else if (MIXED) {
        Tv = temperature_mixed(ph, Z[c], H[c]);
        kv = kappa_mixed(ph, Tv);
        iT = recip_newton(Tv);
    } else {
        Tv = temperature(ph, Z[c], H[c]);
        kv = kappa_of(ph, Tv);
        iT = 1.0 / Tv;
    }
    T[c] = Tv;
    kap[c] = kv;
    if (kap_ghosts) {
        int q[3];
        padded_coords(g, c, q);
        fill_ghosts_of(g, ph, bnd, kj, q, &kv);
    }
    if (!ph.closed) rho[c] = iT;        // p0 = 1 (Eq 2.41), rho = p0 / T (Eq 2.49)
    if (MIXED ? !temperature_ok(Tv) : (!(Tv > 0.0) || !(Tv < 1e300))) bad = 1;
    return iT;
}

__device__ __forceinline__ GhostJob kappa_job(double* kap) {
    GhostJob kj;
    kj.f[0] = kap;
    kj.what[0] = GW_KAPPA;
    kj.nf = 1;
    return kj;
}

template <bool MIXED>
__global__ void k_state(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ H,
                        double* __restrict__ T, double* __restrict__ rho, double* __restrict__ kap,
                        double* __restrict__ part, int* status, double* sc, int p0_slot, Bnd bnd, int kap_ghosts) {
    const GhostJob kj = kappa_job(kap);
    __shared__ double sm[NT / 32];
    double acc = 0.0;
    int bad = 0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        acc += state_cell<MIXED>(g, ph, Z, H, T, rho, kap, bnd, kj, kap_ghosts, c, bad);
    }
    if (bad) atomicOr(status, ST_NAN);
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
    if (blockIdx.x == 0 && threadIdx.x == 0 && !ph.closed) {
        sc[p0_slot] = 1.0;
        sc[p0_slot + SC_INV_OFF] = 1.0;
    }
}

// Per-step checks after the corrector's projection: the discrete continuity
// residual of Eq 3.24 (with the mass source of Eq 3.33) cell by cell, the
// global mass balance over the boundary faces (text after Eq 4.22), and the
// differences between the predictor's and the corrector's v and P (the local
// truncation error measure of Sec. 4.2.2).  Block partials in DG_* order;
// k_diag_final reduces them in index order (deterministic).
template <int DIM>
__global__ void __launch_bounds__(NT) k_diag(Geom g, DiagArgs a) {
    double mres = 0.0, mdr = 0.0, msm = 0.0, bal = 0.0, du[3] = {0.0, 0.0, 0.0}, dp = 0.0, dp2 = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        int cc[3];
        interior_coords(g, t, cc);
        const long long c = pad_index(g, t);
        const double drho = (a.c0 * a.rho_new[c] + a.c1 * a.rho_n[c] + a.c2 * a.rho_prev[c]) * a.iden;
        const double sm = a.Sm ? a.Sm[c] : 0.0;
        double div = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const double lo = a.F[j][c], hi = a.F[j][c + g.s[j]];
            div += (hi - lo) * g.ih[j];
            if (!g.periodic[j]) {
                const double dA = g.dV * g.ih[j];
                if (cc[j] == 0) bal -= lo * dA;
                if (cc[j] == g.n[j] - 1) bal += hi * dA;
            }
        }
        bal += (drho - sm) * g.dV;
        mres = fmax(mres, fabs(drho + div - sm));
        mdr = fmax(mdr, fabs(drho));
        msm = fmax(msm, fabs(sm));
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            const double d = a.vs[i][c] - a.v[i][c];
            du[i] = fma(d, d, du[i]);
        }
        const double d = a.Ps[t] - a.P[t];
        dp += d;
        dp2 = fma(d, d, dp2);
    }
    __shared__ double red[NT / 32];
    double vals[DG_N] = {mres, mdr, msm, bal, du[0], du[1], du[2], dp, dp2};
#pragma unroll
    for (int k = 0; k < DG_N; ++k) {
        const double v = (k < DG_BAL) ? block_max<NT>(vals[k], red) : block_sum<NT>(vals[k], red);
        if (threadIdx.x == 0) a.part[k * kDiagBlocks + blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(NT) k_diag_final(Geom g, DiagArgs a, int nb) {
    __shared__ double red[NT / 32];
    for (int k = 0; k < DG_N; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nb; i += NT) {
            const double x = a.part[k * kDiagBlocks + i];
            v = (k < DG_BAL) ? fmax(v, x) : v + x;
        }
        v = (k < DG_BAL) ? block_max<NT>(v, red) : block_sum<NT>(v, red);
        if (threadIdx.x == 0) a.out[k] = (k >= DG_DU) ? v * g.dV : v;
    }
}

// Enclosed system: p0 = m / (sum(1/T) dV) (Eq 2.40), rho = p0 / T (Eq 2.49).
// Semi-enclosed (semi): p0 is the value the ODE of Eq 2.38 left in the slot.
__global__ void k_density(Geom g, const double* __restrict__ T, double* __restrict__ rho,
                          const double* __restrict__ part, int np, double* sc, int p0_slot, int mixed, int semi) {
    __shared__ double sm[NT / 32];
    double p0;
    if (semi) {
        p0 = sc[p0_slot];
    } else {
        const double s = sum_partials<NT>(part, np, sm);
        p0 = sc[SC_MASS] / (s * g.dV);
    }
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        rho[c] = mixed ? p0 * recip_newton(T[c]) : p0 / T[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !semi) {
        sc[p0_slot] = p0;
        sc[p0_slot + SC_INV_OFF] = 1.0 / p0;
    }
}

// Semi-enclosed system, Eq 2.38: block partials of the two volume sums of
//   G = gamma / V { Q / ((S+1) Pe) sum [div(kappa grad H) + N' div(kappa grad Z)] dV - p0 sum div v dV },
// div(kappa grad .) as the residuals' diffusion (kappa on the faces by the
// mean of Eq 3.20, delta_1 across them), N' = (N'_F - N'_O) theta_eps(Z - 1)
// + N'_O regularised like N (Eq 3.35b), and div v the cell-centred delta_2
// divergence.  One FP64 pass over Z, H, kappa and v.
template <int DIM>
__global__ void __launch_bounds__(NT) k_p0_rate(Geom g, Phys ph, const double* __restrict__ Z,
                                                const double* __restrict__ H, const double* __restrict__ kap,
                                                const double* __restrict__ v0, const double* __restrict__ v1,
                                                const double* __restrict__ v2, double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    const double* v[3] = {v0, v1, v2};
    double heat = 0.0, div = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        const double kc = kap[c], Zc = Z[c], Hc = H[c];
        double dH = 0.0, dZ = 0.0, dv = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const double kp = 0.5 * (kc + kap[c + s]), km = 0.5 * (kc + kap[c - s]);
            dH += (kp * (H[c + s] - Hc) - km * (Hc - H[c - s])) * g.ih[j] * g.ih[j];
            dZ += (kp * (Z[c + s] - Zc) - km * (Zc - Z[c - s])) * g.ih[j] * g.ih[j];
            dv += (v[j][c + s] - v[j][c - s]) * (0.5 * g.ih[j]);
        }
        const double th = 0.5 * (1.0 + tanh(ph.k * (Zc - 1.0)));
        heat += dH + ((ph.NpF - ph.NpO) * th + ph.NpO) * dZ;
        div += dv;
    }
    heat = block_sum<NT>(heat, sm);
    div = block_sum<NT>(div, sm);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = heat;
        part[gridDim.x + blockIdx.x] = div;
    }
}

// One block: the sums in index order, G, and the stage's p0 (AB2 predictor,
// AM2 corrector, as for Z and H in Eqs 3.1-3.3 and 3.12-3.13).  The
// predictor rotates the G history (SC_G_N -> SC_G_NM1).
__global__ void k_p0_ode(Geom g, Phys ph, const double* __restrict__ part, int np, double* sc, int stage, double dt,
                         int out_slot) {
    __shared__ double sm[NT / 32];
    const double heat = sum_partials<NT>(part, np, sm) * g.dV;
    const double div = sum_partials<NT>(part + np, np, sm) * g.dV;
    if (threadIdx.x != 0) return;
    const double p0_level = (stage == ODE_CORR) ? sc[SC_P0_STAR] : sc[SC_P0_N];
    const double G = ph.ode_gV * (ph.ode_heat * heat - p0_level * div);
    double p0;
    if (stage == ODE_CORR) {
        p0 = sc[SC_P0_N] + 0.5 * dt * (G + sc[SC_G_N]);
    } else {
        const double Gp = sc[SC_G_N];
        sc[SC_G_NM1] = Gp;
        sc[SC_G_N] = G;
        p0 = sc[SC_P0_N] + dt * ((stage == ODE_PRED_AB2) ? 1.5 * G - 0.5 * Gp : G);
    }
    sc[out_slot] = p0;
    sc[out_slot + SC_INV_OFF] = 1.0 / p0;
}

// ----------------------------------------------------------------------------
// Residuals at one level and the AB2 / AM2 combination (Eqs 3.1-3.4, 3.7-3.8,
// 3.10, 3.12-3.13, 3.16, 3.18; convection Eq 3.26; penalisation Eqs 3.30-3.32).
// ----------------------------------------------------------------------------
// C is the arithmetic type of the residual terms and of the stored residual
// history (double in both precision modes, see launch_residual); the state
// updates X = X_b + dt * combination are FP64.

// Plain FP64 loads of the stencil's inputs.
struct PlainLoad {
    const ResidArgs* a;
    __device__ __forceinline__ double operator()(int f, long long i) const {
        switch (f) {
            case RF_V0: return a->v[0][i];
            case RF_V1: return a->v[1][i];
            case RF_V2: return a->v[2][i];
            case RF_Z: return a->Z[i];
            case RF_H: return a->H[i];
            case RF_RHO: return a->rho[i];
            case RF_KAP: return a->kap[i];
            case RF_F0: return a->F[0][i];
            case RF_F1: return a->F[1][i];
            case RF_F2: return a->F[2][i];
            case RF_T: return a->T[i];
            case RF_VIB0: return a->vib[0][i];
            case RF_VIB1: return a->vib[1][i];
            default: return a->vib[2][i];
        }
    }
};

// Float-float loads with the six stencil fields read from their split
// images (launch_ff_images), which the stencil reads up to 19 times per cell:
// the same values as splitting on load, without the integer split per use.
struct ImageLoad {
    const ResidArgs* a;
    long long np;
    __device__ __forceinline__ FF operator()(int f, long long i) const {
        int p;
        switch (f) {
            case RF_V0: p = 0; break;
            case RF_V1: p = 1; break;
            case RF_V2: p = 2; break;
            case RF_Z: p = 3; break;
            case RF_H: p = 4; break;
            case RF_KAP: p = 5; break;
            default: return FF(PlainLoad{a}(f, i));
        }
        const float2 w = __ldg(a->ffs + (long long)p * np + i);
        return FF(w.x, w.y);
    }
};

__global__ void k_ff_images(long long npad, int nf, FFSrc src, float2* __restrict__ dst) {
    for (long long p = (long long)blockIdx.x * NT + threadIdx.x; p < npad; p += (long long)gridDim.x * NT) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (!src.f[f]) continue;
            const FF w(src.f[f][p]);
            dst[(long long)f * npad + p] = make_float2(w.hi, w.lo);
        }
    }
}

// Stage residuals at padded cell c (Eqs 3.1-3.4, 3.7-3.8, 3.26, 3.30-3.32):
// R[i] = Res_v,i + f_v,i + F_v,i (i < DIM), R[3] = Res_Z, R[4] = Res_H.  C is
// the arithmetic type (double, or a dual number for the adjoint); ld(f, i)
// returns input field f at padded index i as a C.
template <int DIM, class C, class LD>
__device__ __forceinline__ void residual_cell(const Geom& g, const Phys& ph, const ResidArgs& a, long long c,
                                              double p0dot, const LD& ld, C R[5]) {
    // every input converted to the arithmetic type as it is loaded, so that
    // differences of loaded values are taken in C (the same bits whichever
    // loader supplies a float-float value: split on load, or its image)
    auto ldc = [&](int f, long long i) -> C { return C(ld(f, i)); };
    const C half = (C)0.5;
    const C rho_c = ldc(RF_RHO, c);
    const C kap_c = ldc(RF_KAP, c);
    const C Zc = ldc(RF_Z, c), Hc = ldc(RF_H, c);

    // scalar convection (Eq 3.26b) and diffusion div(kappa grad .)
    C convZ = 0.0, convH = 0.0, difZ = 0.0, difH = 0.0;
    C kf_lo[DIM], kf_hi[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const C ih = (C)g.ih[j];
        const C Flo = ldc(RF_F0 + j, c), Fhi = ldc(RF_F0 + j, c + s);
        kf_lo[j] = half * (ldc(RF_KAP, c - s) + kap_c);
        kf_hi[j] = half * (kap_c + ldc(RF_KAP, c + s));
        const C dZlo = (Zc - ldc(RF_Z, c - s)) * ih, dZhi = (ldc(RF_Z, c + s) - Zc) * ih;
        const C dHlo = (Hc - ldc(RF_H, c - s)) * ih, dHhi = (ldc(RF_H, c + s) - Hc) * ih;
        convZ += half * (Flo * dZlo + Fhi * dZhi);
        convH += half * (Flo * dHlo + Fhi * dHhi);
        difZ += (kf_hi[j] * dZhi - kf_lo[j] * dZlo) * ih;
        difH += (kf_hi[j] * dHhi - kf_lo[j] * dHlo) * ih;
    }

    // momentum: convection Eq 3.26a, viscous stress Eq 2.46 on the interfaces
    const C two3 = (C)(2.0 / 3.0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        C conv = 0.0, visc = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const C ih = (C)g.ih[j];
            const C Flo = ldc(RF_F0 + j, c), Fhi = ldc(RF_F0 + j, c + s);
            const C vl = ldc(RF_V0 + i, c - s), vc = ldc(RF_V0 + i, c), vh = ldc(RF_V0 + i, c + s);
            conv += (Fhi * (half * (vc + vh)) - Flo * (half * (vl + vc))) * ih;
            C tau_f[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const long long ca = side ? c : c - s;   // cell below the interface
                const long long cb = ca + s;             // cell above
                const C kf = side ? kf_hi[j] : kf_lo[j];
                const C dvi = (side ? (vh - vc) : (vc - vl)) * ih;
                C dvj;
                if (i == j) {
                    dvj = dvi;
                } else {
                    const long long si = g.s[i];
                    const C hi2 = (C)(0.5 * g.ih[i]);
                    const C da = (ldc(RF_V0 + j, ca + si) - ldc(RF_V0 + j, ca - si)) * hi2;
                    const C db = (ldc(RF_V0 + j, cb + si) - ldc(RF_V0 + j, cb - si)) * hi2;
                    dvj = half * (da + db);
                }
                C tau = kf * (dvi + dvj);
                if (i == j) {
                    C div = dvi;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        if (k == j) continue;
                        const long long sk = g.s[k];
                        const C hk2 = (C)(0.5 * g.ih[k]);
                        const C da = (ldc(RF_V0 + k, ca + sk) - ldc(RF_V0 + k, ca - sk)) * hk2;
                        const C db = (ldc(RF_V0 + k, cb + sk) - ldc(RF_V0 + k, cb - sk)) * hk2;
                        div = div + half * (da + db);
                    }
                    tau = tau - two3 * kf * div;
                }
                tau_f[side] = tau;
            }
            visc += (tau_f[1] - tau_f[0]) * ih;
        }
        C Rm = -conv + (C)ph.PrPe * visc;
        if (i == 1 && ph.inv_Fr2 != 0.0) Rm = Rm + (C)ph.inv_Fr2 * ((C)1.0 - rho_c);                  // Eq 3.8b
        if (a.ibm && a.chi[c])
            Rm = Rm - (C)(ph.PrPe * a.inv_Da) * kap_c * (ldc(RF_V0 + i, c) - ldc(RF_VIB0 + i, c));    // Eq 3.30
        R[i] = Rm;
    }

    // Lewis and N coefficients (Eq 3.35)
    C iLePe = (C)ph.iLePe, Nn = (C)ph.N_O;
    if (ph.Le_F != ph.Le_O) {
        const C th = half * ((C)1.0 + tanh_c(ph.k * (Zc - (C)1.0)));
        const C Le = (C)(ph.Le_F - ph.Le_O) * th + (C)ph.Le_O;
        Nn = (C)(ph.N_F - ph.N_O) * th + (C)ph.N_O;
        iLePe = (C)1.0 / (Le * (C)ph.Pe);
    }
    const C iPe = (C)ph.iPe;
    C bZ = -convZ + difZ * iLePe;
    C bH = -convH + difH * iPe + (C)(ph.zeta * p0dot) + Nn * difZ * iPe;
    if (a.ibm && a.chi[c]) {
        const C iDa = (C)a.inv_Da;
        bZ = bZ - kap_c * (Zc - (C)a.Z_ib) * iLePe * iDa;                                   // Eq 3.31
        bH = bH - kap_c * (Hc - (C)a.H_ib) * iPe * iDa;                                     // Eq 3.32
    }
    // 1/rho = T / p0 (Eq 2.49)
    const C irho = ldc(RF_T, c) * (C)a.sc[a.p0r + SC_INV_OFF];
    R[3] = bZ * irho;
    R[4] = bH * irho;
}

// C: arithmetic of the stencil terms (double, or float-float in the mixed
// path); the residuals are stored and combined in FP64.
// Float-float stencil: three blocks per SM (80 registers) in 3D, four (64) in
// 2D; latency-bound at the two blocks its uncapped register count allows.  In
// 2D the fourth block costs spills (slower back to back with warm caches) but
// hides the DRAM latency of the step's first kernel after a cold L2 better, and
// a 131k-cell grid fits one wave (slot 256x512 step 1.000 -> 0.993 ms).
// The interior -> padded index map with 64-bit division, kept for the 3D
// stage stencil only: at its 80-register cap the compiler spills 96 bytes with
// this form and 524 with the 32-bit invariant-divisor map (measured 2.32 vs
// 2.55 ms per 192^3 launch); every other kernel uses pad_index.
__device__ __forceinline__ long long pad_index_div64(const Geom& g, long long t) {
    const int i = (int)(t % g.n[0]);
    const long long r = t / g.n[0];
    const int j = (int)(r % g.n[1]);
    const int k = (int)(r / g.n[1]);
    const long long kz = (g.dim == 3) ? (k + 1) : 0;
    return (long long)(i + 1) + (long long)(j + 1) * g.s[1] + kz * g.s[2];
}

template <int DIM, class C>
struct ResidMinBlocks {
    static constexpr int v = 2;
};
template <>
struct ResidMinBlocks<3, FF> {
    static constexpr int v = 3;
};
template <>
struct ResidMinBlocks<2, FF> {
    static constexpr int v = 4;
};

// The stage stencil and combination of the cells of block bx (NT cells);
// IMG: float-float stencil inputs from their split images.
template <int DIM, class C, bool IMG = false>
__device__ __forceinline__ void residual_body(const Geom& g, const Phys& ph, const ResidArgs& a, int bx) {
    // the linear cell map: the tiled one (stage_tile_x) costs the register-capped
    // float-float stencil spills (96 -> 848 bytes in 3D) and gained nothing
    const long long t = (long long)bx * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = (DIM == 3) ? pad_index_div64(g, t) : pad_index(g, t);
    const double* Rrd[5];
    double* Rst[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        Rrd[k] = reinterpret_cast<const double*>(a.Rrd[k]);
        Rst[k] = reinterpret_cast<double*>(a.Rst[k]);
    }
    // dp0/dt for the H source (Eqs 3.5, 3.14)
    const double p0dot =
        (a.wden != 0.0) ? __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.w0, a.sc[a.p0a]), __dmul_rn(a.w1, a.sc[a.p0b])),
                                              __dmul_rn(a.w2, a.sc[a.p0c])),
                                    a.iwden)
                        : 0.0;
    C Rall[5];
    if constexpr (IMG) residual_cell<DIM, C>(g, ph, a, c, p0dot, ImageLoad{&a, g.npad}, Rall);
    else residual_cell<DIM, C>(g, ph, a, c, p0dot, PlainLoad{&a}, Rall);
    double Rv[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) Rv[i] = (double)Rall[i];
    const double RZ = (double)Rall[3], RH = (double)Rall[4];

    // combination (FP64 state update)
    const double dt = a.dt;
    const double rb = a.rhob[c];
    double zo, ho;
    if (a.mode == MODE_CORR) {
        const double hdt = 0.5 * dt;
#pragma unroll
        for (int i = 0; i < DIM; ++i)
            a.mo[i][c] = __fma_rn(hdt, __dadd_rn(Rv[i], Rrd[i][c]), __dmul_rn(rb, a.vb[i][c]));
        zo = __fma_rn(hdt, __dadd_rn(RZ, Rrd[3][c]), a.Zb[c]);
        ho = __fma_rn(hdt, __dadd_rn(RH, Rrd[4][c]), a.Hb[c]);
    } else {
        const bool ab2 = (a.mode == MODE_PRED_AB2);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            // explicitly rounded (the same bits in every instantiation of this
            // body, whatever contraction the compiler would choose)
            const double cv = ab2 ? __fma_rn(1.5, Rv[i], __dmul_rn(-0.5, Rrd[i][c])) : Rv[i];
            Rst[i][c] = Rv[i];
            a.mo[i][c] = __fma_rn(dt, cv, __dmul_rn(rb, a.vb[i][c]));
        }
        const double cZ = ab2 ? __fma_rn(1.5, RZ, __dmul_rn(-0.5, Rrd[3][c])) : RZ;
        const double cH = ab2 ? __fma_rn(1.5, RH, __dmul_rn(-0.5, Rrd[4][c])) : RH;
        Rst[3][c] = RZ;
        Rst[4][c] = RH;
        zo = __fma_rn(dt, cZ, a.Zb[c]);
        ho = __fma_rn(dt, cH, a.Hb[c]);
    }
    a.Zo[c] = zo;
    a.Ho[c] = ho;
    if (DIM == 2 && a.gj.nf) {   // fused ghost fill of Z, H (2D: the 3D stencil runs out of registers)
        int q[3];
        padded_coords(g, c, q);
        const double vals[2] = {zo, ho};
        fill_ghosts_of(g, ph, a.bnd, a.gj, q, vals);
    }
}

template <int DIM, class C, bool IMG = false>
__global__ void __launch_bounds__(NT, ResidMinBlocks<DIM, C>::v) k_residual(Geom g, Phys ph, ResidArgs a) {
    residual_body<DIM, C, IMG>(g, ph, a, blockIdx.x);
}

// ----------------------------------------------------------------------------
// Interface mass fluxes of the provisional momentum (first term of Eq 3.23) and
// block partials of the global mass balance (Eq 3.24 + S_m, Eq 3.33).
// ----------------------------------------------------------------------------
// s / 2 without the FP64 pipe: a normal double halves exactly by decrementing
// its exponent field; zero, subnormal, infinite and NaN values take the FP64
// multiply (bitwise the same result either way).
__device__ __forceinline__ double half_exact(double s) {
    const long long b = __double_as_longlong(s);
    const int e = (int)((b >> 52) & 0x7ff);
    return (e > 1 && e < 0x7ff) ? __longlong_as_double(b - (1LL << 52)) : s * 0.5;
}

// Face fluxes of one cell (its low faces, and its high faces on the last layer)
// and its term of the mass balance; rho_new_c = rho^{new} at the cell (read
// only when a.correct), rho_in = inflow density, iden = 1 / bdf_den.
template <int DIM>
__device__ __forceinline__ double flux_cell(const Geom& g, const Phys& ph, const Bnd& bnd, const FluxArgs& a,
                                            long long t, long long c, double rho_new_c, double rho_in,
                                            double iden) {
    double acc = 0.0;
    int ct[3], q[3];
    interior_coords(g, t, ct);
    padded_coords(g, c, q);
    // FP64 products and sums explicitly rounded (no contraction), so that the
    // member-batched launch of this code rounds exactly as the single one
    if (a.correct) {
        double num = __dadd_rn(__dmul_rn(a.bdf_c0, rho_new_c), __dmul_rn(a.bdf_c1, a.rho_n[c]));
        if (a.bdf_c2 != 0.0) num = __dadd_rn(num, __dmul_rn(a.bdf_c2, a.rho_prev[c]));
        const double drho = __dmul_rn(num, iden);
        const double Sm = a.Sm ? a.Sm[c] : 0.0;
        const double bm = __dsub_rn(drho, Sm);
        a.b[t] = bm;   // completed by k_rhs with the flux divergence
        acc = __fma_rn(bm, g.dV, acc);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const int n = g.n[j];
        const double* m = a.mom[j];
        const double dA = g.dV * g.ih[j];
        if (ct[j] > 0 || g.periodic[j]) {
            const long long cl = (ct[j] > 0) ? c - s : c + (long long)(n - 1) * s;
            a.F[j][c] = half_exact(m[cl] + m[c]);
        } else {
            const int kind = bnd.kind[j][0][slab_index(g, j, q)];
            const double val =
                (kind == BC_INFLOW) ? __dmul_rn(rho_in, ph.inflow_v[j]) : (kind == BC_OUTFLOW) ? m[c] : 0.0;
            a.F[j][c] = val;
            acc = __fma_rn(-val, dA, acc);
        }
        if (ct[j] == n - 1) {
            if (g.periodic[j]) {
                a.F[j][c + s] = half_exact(m[c] + m[c - (long long)(n - 1) * s]);
            } else {
                const int kind = bnd.kind[j][1][slab_index(g, j, q)];
                const double val =
                    (kind == BC_INFLOW) ? __dmul_rn(rho_in, ph.inflow_v[j]) : (kind == BC_OUTFLOW) ? m[c] : 0.0;
                a.F[j][c + s] = val;
                acc = __fma_rn(val, dA, acc);
            }
        }
    }
    return acc;
}

template <int DIM>
__global__ void k_face_flux(Geom g, Phys ph, Bnd bnd, FluxArgs a) {
    __shared__ double sm[NT / 32];
    const double rho_in = ph.incompressible ? 1.0 : a.sc[a.p0_slot] / ph.rho_in_T;
    const double iden = 1.0 / a.bdf_den;     // once per thread: FP64 division is a long sequence
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        acc += flux_cell<DIM>(g, ph, bnd, a, t, c, a.correct ? a.rho_new[c] : 0.0, rho_in, iden);
    }
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) a.part[blockIdx.x] = acc;
}

// Open system (p0 = 1): the state relation and the face fluxes of a stage in
// one pass.  The flux needs rho^{new} only at its own cell, just computed, and
// p0 = 1 for the inflow density (so the same bits as k_state then
// k_face_flux); the state's sum of 1/T serves only the enclosed system's p0, so
// the block partials are the mass balance's.
template <int DIM, bool MIXED>
__device__ __forceinline__ void state_flux_body(const Geom& g, const Phys& ph, const double* __restrict__ Z,
                                                const double* __restrict__ H, double* __restrict__ T,
                                                double* __restrict__ rho, double* __restrict__ kap, int* status,
                                                double* sc, const Bnd& bnd, int kap_ghosts, const FluxArgs& a,
                                                int bx, int gx) {
    const GhostJob kj = kappa_job(kap);
    __shared__ double sm[NT / 32];
    const double rho_in = ph.incompressible ? 1.0 : 1.0 / ph.rho_in_T;
    const double iden = 1.0 / a.bdf_den;
    double acc = 0.0;
    int bad = 0;
    for (long long t = (long long)bx * NT + threadIdx.x; t < g.ncell; t += (long long)gx * NT) {
        const long long c = pad_index(g, t);
        const double iT = state_cell<MIXED>(g, ph, Z, H, T, rho, kap, bnd, kj, kap_ghosts, c, bad);
        acc += flux_cell<DIM>(g, ph, bnd, a, t, c, iT, rho_in, iden);
    }
    if (bad) atomicOr(status, ST_NAN);
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) a.part[bx] = acc;
    if (bx == 0 && threadIdx.x == 0) {
        sc[a.p0_slot] = 1.0;
        sc[a.p0_slot + SC_INV_OFF] = 1.0;
    }
}

template <int DIM, bool MIXED>
__global__ void k_state_flux(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ H,
                             double* __restrict__ T, double* __restrict__ rho, double* __restrict__ kap,
                             int* status, double* sc, Bnd bnd, int kap_ghosts, FluxArgs a) {
    state_flux_body<DIM, MIXED>(g, ph, Z, H, T, rho, kap, status, sc, bnd, kap_ghosts, a, blockIdx.x, gridDim.x);
}

// Uniform shift of the outflow fluxes closing the mass balance, then
// b = d_t rho + sum_j delta_1 F_j / delta_1 x_j - S_m  (Eq 3.24 with S_m).
template <int DIM>
__device__ __forceinline__ void rhs_body(const Geom& g, const Bnd& bnd, const FluxArgs& a, int np, int bx, int gx) {
    __shared__ double sm[NT / 32];
    const double total = sum_partials<NT>(a.part, np, sm);
    const double area = a.sc[SC_OUT_AREA];
    const double shift = (area > 0.0) ? -total / area : 0.0;
    double bsum = 0.0;
    for (long long t = (long long)bx * NT + threadIdx.x; t < g.ncell; t += (long long)gx * NT) {
        const long long c = pad_index(g, t);
        int ct[3], q[3];
        interior_coords(g, t, ct);
        padded_coords(g, c, q);
        double b = a.b[t];   // d_t rho - S_m, stored by k_face_flux
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            if (!g.periodic[j]) {
                if (ct[j] == 0 && bnd.kind[j][0][slab_index(g, j, q)] == BC_OUTFLOW)
                    a.F[j][c] = __dsub_rn(a.F[j][c], shift);
                if (ct[j] == g.n[j] - 1 && bnd.kind[j][1][slab_index(g, j, q)] == BC_OUTFLOW)
                    a.F[j][c + s] = __dadd_rn(a.F[j][c + s], shift);
            }
            b = __fma_rn(__dsub_rn(a.F[j][c + s], a.F[j][c]), g.ih[j], b);
        }
        a.b[t] = b;
        bsum += b;
        if (a.guess != GUESS_NONE) {
            const double p = a.P[t];
            if (a.guess == GUESS_SHIFT) {
                a.P[t] = __dadd_rn(p, a.Pd[t]);
            } else {
                const double pm = a.Pm1[t];
                a.Pm1[t] = p;
                if (a.guess == GUESS_EXTRAP) a.P[t] = __fma_rn(2.0, p, -pm);
            }
        }
    }
    if (a.mb_out) {
        // mean(b) for the pressure solve, with the block decomposition and the
        // fixed-order sums of the solver's own mean pass (bitwise the same)
        bsum = block_sum<NT>(bsum, sm);
        if (threadIdx.x == 0) a.mb_part[bx] = bsum;
        if (arrive_last_n(a.mb_cnt, gx)) {
            double v = 0.0;
            for (int i = threadIdx.x; i < gx; i += NT) v += __ldcg(a.mb_part + i);
            v = block_sum<NT>(v, sm);
            if (threadIdx.x == 0) {
                *a.mb_out = v / (double)g.ncell;
                *a.mb_cnt = 0u;
            }
        }
    }
}

template <int DIM>
__global__ void k_rhs(Geom g, Bnd bnd, FluxArgs a, int np) {
    rhs_body<DIM>(g, bnd, a, np, blockIdx.x, gridDim.x);
}

// ----------------------------------------------------------------------------
// Projection: F_j = Ft_j - delta_1 P / delta_1 x_j on the interfaces that carry
// a pressure term (Eq 3.23), v_i = (rho v~_i - delta_2 P / delta_2 x_i) / rho
// (Eq 3.25) with P ghosts by quadratic extrapolation (Eqs 3.27-3.28).
// ----------------------------------------------------------------------------
// p0 history n-2 <- n-1 <- n <- n+1 (and the inverses) at the end of a step.
__device__ __forceinline__ void rotate_p0(double* sc) {
    sc[SC_P0_NM2] = sc[SC_P0_NM1];
    sc[SC_P0_NM1] = sc[SC_P0_N];
    sc[SC_P0_N] = sc[SC_P0_NEW];
    sc[SC_P0_NM2 + SC_INV_OFF] = sc[SC_P0_NM1 + SC_INV_OFF];
    sc[SC_P0_NM1 + SC_INV_OFF] = sc[SC_P0_N + SC_INV_OFF];
    sc[SC_P0_N + SC_INV_OFF] = sc[SC_P0_NEW + SC_INV_OFF];
}

template <int DIM>
__device__ __forceinline__ void project_body(const Geom& g, const Phys& ph, const ProjArgs& a, int bx) {
    double vout[3];
    const long long t = cell_of_block(g, bx);
    if (t < 0) return;
    const long long c = pad_index(g, t);
    int ct[3];
    interior_coords(g, t, ct);
    // FP64 products and sums explicitly rounded (no contraction; see flux_cell)
    const double Pc = a.P[t];
    const double irho = __dmul_rn(a.T[c], a.sc[a.p0_slot + SC_INV_OFF]);   // 1/rho = T / p0 (Eq 2.49)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const long long st = compact_stride(g, j);
        const int n = g.n[j];
        const double ih = g.ih[j];
        double Pm, Pp;
        if (ct[j] > 0) Pm = a.P[t - st];
        else if (g.periodic[j]) Pm = a.P[t + (long long)(n - 1) * st];
        else Pm = __fma_rn(a.eC, a.P[t + 2 * st], __fma_rn(a.eB, a.P[t + st], __dmul_rn(a.eA, Pc)));
        if (ct[j] < n - 1) Pp = a.P[t + st];
        else if (g.periodic[j]) Pp = a.P[t - (long long)(n - 1) * st];
        else Pp = __fma_rn(a.eC, a.P[t - 2 * st], __fma_rn(a.eB, a.P[t - st], __dmul_rn(a.eA, Pc)));
        if (ct[j] > 0 || g.periodic[j]) a.F[j][c] = __fma_rn(-__dsub_rn(Pc, Pm), ih, a.F[j][c]);
        if (ct[j] == n - 1 && g.periodic[j]) a.F[j][c + s] = __fma_rn(-__dsub_rn(Pp, Pc), ih, a.F[j][c + s]);
        vout[j] = __dmul_rn(__fma_rn(-__dsub_rn(Pp, Pm), __dmul_rn(0.5, ih), a.mom[j][c]), irho);
        a.v[j][c] = vout[j];
    }
    if (a.gj.nf) {   // fused ghost fill of v
        int q[3];
        padded_coords(g, c, q);
        fill_ghosts_of(g, ph, a.bnd, a.gj, q, vout);
    }
    if (a.Pd) a.Pd[t] = __dsub_rn(Pc, a.Pstar[t]);
    // the step's last projection rotates the p0 history (it reads only the new
    // p0, which the rotation leaves as it is)
    if (a.rot && t == 0) rotate_p0(a.rot);
}

template <int DIM>
__global__ void k_project(Geom g, Phys ph, ProjArgs a) {
    project_body<DIM>(g, ph, a, blockIdx.x);
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
    } else if (b.kind == 4) {  // coaxial cylinders: inner turns rigidly, outer at rest
        const double dx = x[0] - b.c[0], dy = x[1] - b.c[1];
        const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        const bool inner = (r - b.radius <= b.s);
        const bool m = inner || (b.half[0] - r <= b.s);
        const double w = inner ? b.U_b / b.radius : 0.0;
        chi[c] = (uint8_t)m;
        vib[0][c] = -w * dy;
        vib[1][c] = w * dx;
        if (g.dim == 3) vib[2][c] = 0.0;
        Sm[c] = 0.0;
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

// Marker body (Sec. 3.4 with the body given by surface markers): every padded
// cell centre p is matched with its nearest marker (least |p - x_m|^2 summed
// over the directions in order, the lowest index on a tie); the normal offset
// (p - x_m).n_m <= s marks it (shifted mask), and v_ib = U_m n_m there.  Cells
// outside the markers' box widened by 2 s are outside the body.  The distance
// and offset are formed with explicitly rounded products and sums, so the
// integer decisions do not depend on FMA contraction.  Markers are scanned in
// chunks staged in shared memory.
constexpr int kMkChunk = 256;
__global__ void __launch_bounds__(NT) k_marker_cells(Geom g, IbmDev b, uint8_t* chi, double* vib0, double* vib1,
                                                     double* vib2, double* U, double* Sm, int* near, int* counts) {
    __shared__ double sx[3][kMkChunk];
    const int D = g.dim, stride = 2 * g.dim + 2;
    const long long c = (long long)blockIdx.x * NT + threadIdx.x;
    const bool live = c < g.npad;
    int q[3] = {0, 0, 0};
    double x[3] = {0.0, 0.0, 0.0};
    bool inbox = false;
    if (live) {
        padded_coords(g, c, q);
        inbox = true;
        for (int d = 0; d < D; ++d) {
            x[d] = ((double)q[d] - 0.5) * g.h[d];
            if (x[d] < b.bb_lo[d] || x[d] > b.bb_hi[d]) inbox = false;
        }
    }
    double best = 0.0;
    int bm = -1;
    if (__syncthreads_or(inbox)) {
        for (int m0 = 0; m0 < b.n_mk; m0 += kMkChunk) {
            const int cnt = min(kMkChunk, b.n_mk - m0);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += NT)
                for (int d = 0; d < D; ++d) sx[d][i] = b.mk[(long long)(m0 + i) * stride + d];
            __syncthreads();
            if (!inbox) continue;
            for (int i = 0; i < cnt; ++i) {
                double d2 = 0.0;
                for (int d = 0; d < D; ++d) {
                    const double t = __dsub_rn(x[d], sx[d][i]);
                    d2 = (d == 0) ? __dmul_rn(t, t) : __dadd_rn(d2, __dmul_rn(t, t));
                }
                if (bm < 0 || d2 < best) {
                    best = d2;
                    bm = m0 + i;
                }
            }
        }
    }
    if (!live) return;
    double* vib[3] = {vib0, vib1, vib2};
    double m = 0.0, Um = 0.0, nrm[3] = {0.0, 0.0, 0.0};
    if (bm >= 0) {
        const double* M = b.mk + (long long)bm * stride;
        double off = 0.0;
        for (int d = 0; d < D; ++d) {
            nrm[d] = M[D + d];
            const double t = __dmul_rn(__dsub_rn(x[d], M[d]), nrm[d]);
            off = (d == 0) ? t : __dadd_rn(off, t);
        }
        m = (off <= b.s) ? 1.0 : 0.0;
        Um = M[2 * D];
    }
    near[c] = bm;
    chi[c] = (uint8_t)(m != 0.0);
    for (int d = 0; d < D; ++d) vib[d][c] = __dmul_rn(__dmul_rn(m, Um), nrm[d]);
    U[c] = 0.0;
    Sm[c] = 0.0;
    bool interior = true;
    for (int d = 0; d < D; ++d)
        if (q[d] < 1 || q[d] > g.n[d]) interior = false;
    if (interior && m != 0.0) atomicAdd(counts + bm, 1);
}

// S_m = rho_b U_m A_m / (N_m dV) on the N_m masked interior cells matched with
// marker m: the discrete integral of S_m is the markers' total ejected flow.
__global__ void k_marker_source(Geom g, IbmDev b, const uint8_t* chi, const int* near, const int* counts,
                                double* Sm) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    if (!chi[c]) return;
    const int stride = 2 * g.dim + 2;
    const double* M = b.mk + (long long)near[c] * stride;
    Sm[c] = __dmul_rn(__dmul_rn(b.rho_b, M[2 * g.dim]), M[2 * g.dim + 1]) /
            __dmul_rn((double)counts[near[c]], g.dV);
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

__global__ void k_add_unpack(Geom g, const double* __restrict__ src, double* __restrict__ dst) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t < g.ncell) dst[pad_index(g, t)] += src[t];
}

// Batched solves: copy the systems' separate arrays into / out of one
// contiguous [nb][N] array (grid dimension y = system).
__global__ void k_gather(const double* const* __restrict__ src, double* __restrict__ dst, long long N) {
    const double* s = src[blockIdx.y];
    double* d = dst + (long long)blockIdx.y * N;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT) d[t] = s[t];
}
__global__ void k_scatter(const double* __restrict__ src, double* const* __restrict__ dst, long long N) {
    const double* s = src + (long long)blockIdx.y * N;
    double* d = dst[blockIdx.y];
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT) d[t] = s[t];
}

__global__ void k_u8_to_double(Geom g, const uint8_t* __restrict__ src, double* __restrict__ dst) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    dst[t] = (double)src[pad_index(g, t)];
}

// ============================================================================
// Discrete adjoint (reverse mode) of the step's kernels.  Every adjoint kernel
// takes lambda (the adjoint of the forward kernel's outputs) and ADDS the
// adjoint of its inputs, so contributions from several uses accumulate.
// ============================================================================

// Loader that seeds one input value (field sf at padded index si): the stencil
// evaluated with it returns, in .d, the derivative along that input.
struct DualLoad {
    PlainLoad p;
    int sf;
    long long si;
    __device__ __forceinline__ Dual operator()(int f, long long i) const {
        return Dual(p(f, i), (f == sf && i == si) ? 1.0 : 0.0);
    }
};

__device__ __forceinline__ bool padded_interior(const Geom& g, const int q[3]) {
    for (int d = 0; d < g.dim; ++d)
        if (q[d] < 1 || q[d] > g.n[d]) return false;
    return true;
}

// Stencil transpose by gather: for padded cell j and each input field f,
//   lam_f[j] += sum_{interior c within one cell of j} sum_o dR_o(c)/df(j) lamR_o(c),
// each derivative taken exactly by evaluating residual_cell at c in dual
// numbers with f(j) seeded.  lamR: adjoint of the residuals (v0..v2, Z, H).
template <int DIM>
__global__ void __launch_bounds__(NT)
    k_residual_adj(Geom g, Phys ph, ResidArgs a, double p0dot, AdjR lr, AdjIn li) {
    const long long j = (long long)blockIdx.x * NT + threadIdx.x;
    if (j >= g.npad) return;
    int q[3];
    padded_coords(g, j, q);
    const int fields[] = {RF_V0, RF_V1, RF_V2, RF_Z, RF_H, RF_KAP, RF_F0, RF_F1, RF_F2, RF_T, RF_VIB0, RF_VIB1,
                          RF_VIB2, RF_RHO};
    for (int fi = 0; fi < 14; ++fi) {
        const int f = fields[fi];
        if (!li.out[f]) continue;
        if ((f == RF_V2 || f == RF_F2 || f == RF_VIB2) && DIM < 3) continue;
        double acc = 0.0;
        const int oz = (DIM == 3) ? 1 : 0;
        for (int dz = -oz; dz <= oz; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int qc[3] = {q[0] + dx, q[1] + dy, q[2] + dz};
                    if (!padded_interior(g, qc)) continue;
                    const long long c = j + dx + (long long)dy * g.s[1] + (long long)dz * g.s[2];
                    Dual R[5];
                    residual_cell<DIM, Dual>(g, ph, a, c, p0dot, DualLoad{PlainLoad{&a}, f, j}, R);
                    for (int o = 0; o < DIM; ++o) acc += R[o].d * lr.R[o][c];
                    acc += R[3].d * lr.R[3][c] + R[4].d * lr.R[4][c];
                }
        li.out[f][j] += acc;
    }
}

// ---------------------------------------------------------------------------
// Stencil transpose by a hand-written reverse sweep (2D), two phases.
// Phase 1, per interior cell c: the partial derivatives of
// sum_o lamR_o(c) R_o(c) with respect to the 40 input values of c's stencil
// (slots below), stored per slot.  Phase 2, per padded cell j: lambda_f[j] +=
// the slots of the cells whose stencil reaches j, summed in a fixed order.
// Same result as the dual-number gather up to rounding order.
// ---------------------------------------------------------------------------
// 5-point fields (Z, H, kappa): centre, then -x, +x, -y, +y.
constexpr int SL_Z = 0, SL_H = 5, SL_K = 10;
constexpr int SL_F0 = 15;   // F_0 at c and c + s_0
constexpr int SL_F1 = 17;   // F_1 at c and c + s_1
constexpr int SL_T = 19;
constexpr int SL_V0 = 20, SL_V1 = 29;   // v_i on the 3x3 block, (dy+1)*3 + (dx+1)
constexpr int SL_VIB0 = 38, SL_VIB1 = 39;
constexpr int SL_N = 40;

__host__ __device__ constexpr int sl5(int j, int sgn) { return sgn == 0 ? 0 : 1 + 2 * j + (sgn > 0 ? 1 : 0); }
__host__ __device__ constexpr int sl9(int dx, int dy) { return (dy + 1) * 3 + (dx + 1); }

// (field id, dx, dy) of every slot
struct SlotTab {
    int f[SL_N], dx[SL_N], dy[SL_N];
};
__host__ __device__ constexpr SlotTab make_slots() {
    SlotTab t{};
    const int fld5[3] = {RF_Z, RF_H, RF_KAP};
    for (int q = 0; q < 3; ++q) {
        const int b = 5 * q;
        t.f[b] = fld5[q]; t.dx[b] = 0; t.dy[b] = 0;
        t.f[b + 1] = fld5[q]; t.dx[b + 1] = -1; t.dy[b + 1] = 0;
        t.f[b + 2] = fld5[q]; t.dx[b + 2] = 1; t.dy[b + 2] = 0;
        t.f[b + 3] = fld5[q]; t.dx[b + 3] = 0; t.dy[b + 3] = -1;
        t.f[b + 4] = fld5[q]; t.dx[b + 4] = 0; t.dy[b + 4] = 1;
    }
    t.f[SL_F0] = RF_F0; t.dx[SL_F0] = 0; t.dy[SL_F0] = 0;
    t.f[SL_F0 + 1] = RF_F0; t.dx[SL_F0 + 1] = 1; t.dy[SL_F0 + 1] = 0;
    t.f[SL_F1] = RF_F1; t.dx[SL_F1] = 0; t.dy[SL_F1] = 0;
    t.f[SL_F1 + 1] = RF_F1; t.dx[SL_F1 + 1] = 0; t.dy[SL_F1 + 1] = 1;
    t.f[SL_T] = RF_T; t.dx[SL_T] = 0; t.dy[SL_T] = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            t.f[SL_V0 + sl9(dx, dy)] = RF_V0; t.dx[SL_V0 + sl9(dx, dy)] = dx; t.dy[SL_V0 + sl9(dx, dy)] = dy;
            t.f[SL_V1 + sl9(dx, dy)] = RF_V1; t.dx[SL_V1 + sl9(dx, dy)] = dx; t.dy[SL_V1 + sl9(dx, dy)] = dy;
        }
    t.f[SL_VIB0] = RF_VIB0; t.dx[SL_VIB0] = 0; t.dy[SL_VIB0] = 0;
    t.f[SL_VIB1] = RF_VIB1; t.dx[SL_VIB1] = 0; t.dy[SL_VIB1] = 0;
    return t;
}
__constant__ SlotTab c_slots = make_slots();

// unit offsets of direction d (2D)
__device__ __forceinline__ int ex(int d) { return d == 0 ? 1 : 0; }
__device__ __forceinline__ int ey(int d) { return d == 1 ? 1 : 0; }

__global__ void __launch_bounds__(NT) k_residual_rev(Geom g, Phys ph, ResidArgs a, double p0dot, AdjR lr,
                                                     double* __restrict__ cont) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    double gs[SL_N];
#pragma unroll
    for (int k = 0; k < SL_N; ++k) gs[k] = 0.0;
    const long long S[2] = {g.s[0], g.s[1]};

    // ---- forward values of the scalar part
    const double kc = a.kap[c], Zc = a.Z[c], Hc = a.H[c];
    double kflo[2], kfhi[2], dZlo[2], dZhi[2], dHlo[2], dHhi[2], Flo[2], Fhi[2];
    double convZ = 0.0, convH = 0.0, difZ = 0.0, difH = 0.0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double ih = g.ih[j];
        Flo[j] = a.F[j][c];
        Fhi[j] = a.F[j][c + S[j]];
        kflo[j] = 0.5 * (a.kap[c - S[j]] + kc);
        kfhi[j] = 0.5 * (kc + a.kap[c + S[j]]);
        dZlo[j] = (Zc - a.Z[c - S[j]]) * ih;
        dZhi[j] = (a.Z[c + S[j]] - Zc) * ih;
        dHlo[j] = (Hc - a.H[c - S[j]]) * ih;
        dHhi[j] = (a.H[c + S[j]] - Hc) * ih;
        convZ += 0.5 * (Flo[j] * dZlo[j] + Fhi[j] * dZhi[j]);
        convH += 0.5 * (Flo[j] * dHlo[j] + Fhi[j] * dHhi[j]);
        difZ += (kfhi[j] * dZhi[j] - kflo[j] * dZlo[j]) * ih;
        difH += (kfhi[j] * dHhi[j] - kflo[j] * dHlo[j]) * ih;
    }
    const double iLePe = ph.iLePe, iPe = ph.iPe, Nn = ph.N_O;
    const bool pen = a.ibm && a.chi[c];
    double bZ = -convZ + difZ * iLePe;
    double bH = -convH + difH * iPe + ph.zeta * p0dot + Nn * difZ * iPe;
    if (pen) {
        bZ -= kc * (Zc - a.Z_ib) * iLePe * a.inv_Da;
        bH -= kc * (Hc - a.H_ib) * iPe * a.inv_Da;
    }
    const double ip0 = a.sc[a.p0r + SC_INV_OFF];
    const double irho = a.T[c] * ip0;

    // ---- reverse: scalars
    const double lR3 = lr.R[3][c], lR4 = lr.R[4][c];
    gs[SL_T] += (lR3 * bZ + lR4 * bH) * ip0;
    const double lbZ = lR3 * irho, lbH = lR4 * irho;
    if (pen) {
        gs[SL_K] -= (lbZ * (Zc - a.Z_ib) * iLePe + lbH * (Hc - a.H_ib) * iPe) * a.inv_Da;
        gs[SL_Z] -= lbZ * kc * iLePe * a.inv_Da;
        gs[SL_H] -= lbH * kc * iPe * a.inv_Da;
    }
    const double lconvZ = -lbZ, lconvH = -lbH;
    const double ldifZ = lbZ * iLePe + lbH * Nn * iPe, ldifH = lbH * iPe;
    double lkflo[2], lkfhi[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double ih = g.ih[j];
        gs[(j == 0 ? SL_F0 : SL_F1)] += 0.5 * (lconvZ * dZlo[j] + lconvH * dHlo[j]);
        gs[(j == 0 ? SL_F0 : SL_F1) + 1] += 0.5 * (lconvZ * dZhi[j] + lconvH * dHhi[j]);
        const double ldZlo = 0.5 * lconvZ * Flo[j] - ldifZ * kflo[j] * ih;
        const double ldZhi = 0.5 * lconvZ * Fhi[j] + ldifZ * kfhi[j] * ih;
        const double ldHlo = 0.5 * lconvH * Flo[j] - ldifH * kflo[j] * ih;
        const double ldHhi = 0.5 * lconvH * Fhi[j] + ldifH * kfhi[j] * ih;
        lkfhi[j] = (ldifZ * dZhi[j] + ldifH * dHhi[j]) * ih;
        lkflo[j] = -(ldifZ * dZlo[j] + ldifH * dHlo[j]) * ih;
        gs[SL_Z + sl5(j, 0)] += (ldZlo - ldZhi) * ih;
        gs[SL_Z + sl5(j, -1)] -= ldZlo * ih;
        gs[SL_Z + sl5(j, 1)] += ldZhi * ih;
        gs[SL_H + sl5(j, 0)] += (ldHlo - ldHhi) * ih;
        gs[SL_H + sl5(j, -1)] -= ldHlo * ih;
        gs[SL_H + sl5(j, 1)] += ldHhi * ih;
    }

    // ---- momentum
    const double two3 = 2.0 / 3.0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double* vi = a.v[i];
        const int SVi = (i == 0) ? SL_V0 : SL_V1;
        const double lRi = lr.R[i][c];
        const double lconv = -lRi, lvisc = ph.PrPe * lRi;
        if (pen) {
            const double q = lRi * ph.PrPe * a.inv_Da;
            gs[SL_K] -= q * (vi[c] - a.vib[i][c]);
            gs[SVi + sl9(0, 0)] -= q * kc;
            gs[(i == 0) ? SL_VIB0 : SL_VIB1] += q * kc;
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const long long s = S[j];
            const double ih = g.ih[j];
            const int SFj = (j == 0) ? SL_F0 : SL_F1;
            const double vl = vi[c - s], vc = vi[c], vh = vi[c + s];
            gs[SFj + 1] += lconv * ih * 0.5 * (vc + vh);
            gs[SFj] -= lconv * ih * 0.5 * (vl + vc);
            gs[SVi + sl9(0, 0)] += lconv * ih * 0.5 * (Fhi[j] - Flo[j]);
            gs[SVi + sl9(ex(j), ey(j))] += lconv * ih * 0.5 * Fhi[j];
            gs[SVi + sl9(-ex(j), -ey(j))] -= lconv * ih * 0.5 * Flo[j];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const double lt = (side ? 1.0 : -1.0) * lvisc * ih;
                const int oax = side ? 0 : -ex(j), oay = side ? 0 : -ey(j);   // ca offset
                const int obx = oax + ex(j), oby = oay + ey(j);                // cb offset
                const double kf = side ? kfhi[j] : kflo[j];
                const double dvi = (side ? (vh - vc) : (vc - vl)) * ih;
                double ldvi, lkf;
                if (i != j) {
                    const int k2 = i;   // the other direction
                    const double* vj = a.v[j];
                    const long long sk = S[k2];
                    const double hk2 = 0.5 * g.ih[k2];
                    const long long ca = c + oax + (long long)oay * g.s[1];
                    const long long cb = c + obx + (long long)oby * g.s[1];
                    const double da = (vj[ca + sk] - vj[ca - sk]) * hk2;
                    const double db = (vj[cb + sk] - vj[cb - sk]) * hk2;
                    const double dvj = 0.5 * (da + db);
                    lkf = lt * (dvi + dvj);
                    ldvi = lt * kf;
                    const double q = 0.5 * lt * kf * hk2;
                    const int SVj = (j == 0) ? SL_V0 : SL_V1;
                    gs[SVj + sl9(oax + ex(k2), oay + ey(k2))] += q;
                    gs[SVj + sl9(oax - ex(k2), oay - ey(k2))] -= q;
                    gs[SVj + sl9(obx + ex(k2), oby + ey(k2))] += q;
                    gs[SVj + sl9(obx - ex(k2), oby - ey(k2))] -= q;
                } else {
                    const int k2 = 1 - j;
                    const double* vk = a.v[k2];
                    const long long sk = S[k2];
                    const double hk2 = 0.5 * g.ih[k2];
                    const long long ca = c + oax + (long long)oay * g.s[1];
                    const long long cb = c + obx + (long long)oby * g.s[1];
                    const double da = (vk[ca + sk] - vk[ca - sk]) * hk2;
                    const double db = (vk[cb + sk] - vk[cb - sk]) * hk2;
                    const double div = dvi + 0.5 * (da + db);
                    lkf = lt * (2.0 * dvi - two3 * div);
                    ldvi = lt * kf * (2.0 - two3);
                    const double q = -two3 * lt * kf * 0.5 * hk2;
                    const int SVk = (k2 == 0) ? SL_V0 : SL_V1;
                    gs[SVk + sl9(oax + ex(k2), oay + ey(k2))] += q;
                    gs[SVk + sl9(oax - ex(k2), oay - ey(k2))] -= q;
                    gs[SVk + sl9(obx + ex(k2), oby + ey(k2))] += q;
                    gs[SVk + sl9(obx - ex(k2), oby - ey(k2))] -= q;
                }
                if (side) {
                    gs[SVi + sl9(ex(j), ey(j))] += ldvi * ih;
                    gs[SVi + sl9(0, 0)] -= ldvi * ih;
                    lkfhi[j] += lkf;
                } else {
                    gs[SVi + sl9(0, 0)] += ldvi * ih;
                    gs[SVi + sl9(-ex(j), -ey(j))] -= ldvi * ih;
                    lkflo[j] += lkf;
                }
            }
        }
    }
    // face kappa = arithmetic mean of the two cells
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        gs[SL_K + sl5(j, -1)] += 0.5 * lkflo[j];
        gs[SL_K + sl5(j, 0)] += 0.5 * (lkflo[j] + lkfhi[j]);
        gs[SL_K + sl5(j, 1)] += 0.5 * lkfhi[j];
    }
    const long long np = g.npad;
#pragma unroll
    for (int k = 0; k < SL_N; ++k) cont[(long long)k * np + c] = gs[k];
}

__global__ void __launch_bounds__(NT) k_residual_rev_gather(Geom g, const double* __restrict__ cont, AdjIn li) {
    const long long j = (long long)blockIdx.x * NT + threadIdx.x;
    if (j >= g.npad) return;
    int q[3];
    padded_coords(g, j, q);
    const long long np = g.npad;
    double acc = 0.0;
    int cur = c_slots.f[0];
    for (int k = 0; k < SL_N; ++k) {
        const int f = c_slots.f[k];
        if (f != cur) {
            if (li.out[cur]) li.out[cur][j] += acc;
            acc = 0.0;
            cur = f;
        }
        // the cell whose stencil offset (dx, dy) lands on j
        const int qc[3] = {q[0] - c_slots.dx[k], q[1] - c_slots.dy[k], q[2]};
        if (!padded_interior(g, qc)) continue;
        acc += cont[(long long)k * np + j - c_slots.dx[k] - (long long)c_slots.dy[k] * g.s[1]];
    }
    if (li.out[cur]) li.out[cur][j] += acc;
}

// Ghost fill of direction d transposed: ghost = s * adjacent (+ constant) or a
// periodic copy, so lam_adjacent += s * lam_ghost and the ghost's lambda is
// consumed (zeroed).  Directions are transposed in reverse order.
__global__ void k_ghost_adj(Geom g, const uint8_t* __restrict__ klo, const uint8_t* __restrict__ khi, int d,
                            int periodic, GhostJob job) {
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
            x[i_n] += x[i_g0];
            x[i_1] += x[i_gh];
            x[i_g0] = 0.0;
            x[i_gh] = 0.0;
            continue;
        }
        const bool vel = what >= GW_V0;
        const bool normal = vel && (what - GW_V0 == d);
        for (int side = 0; side < 2; ++side) {
            const long long ig = side ? i_gh : i_g0;
            const long long ia = side ? i_n : i_1;
            const int kind = side ? khi[q] : klo[q];
            double sg;
            if (kind == BC_INFLOW || kind == BC_WALL_T) sg = -1.0;   // mirrors about a fixed value
            else if (kind == BC_OUTFLOW) sg = 1.0;
            else if (kind == BC_WALL) sg = vel ? -1.0 : 1.0;
            else sg = normal ? -1.0 : 1.0;
            x[ia] += sg * x[ig];
            x[ig] = 0.0;
        }
    }
}

// State relation transposed (FP64 path, open system: rho = 1/T, kappa = T^sigma
// or Sutherland's law, T = cT (cA (|x| + log1p(e^-2|x|)) + cB (Z - 1) + H),
// x = k (Z - 1)): dT/dZ = cT (cA k tanh(x) + cB), dT/dH = cT, drho/dT =
// -1/T^2, dkappa/dT = sigma kappa / T (power law) or kappa (3/(2T) - 1/(T + C))
// (Eq 4.12).
__global__ void k_state_adj(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ T,
                            const double* __restrict__ kap, double* lT, double* lrho, double* lkap, double* lZ,
                            double* lH) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    const double Tv = T[c];
    const double dk = (ph.transport == 1) ? kap[c] * (1.5 / Tv - 1.0 / (Tv + ph.suth_C)) : ph.sigma * kap[c] / Tv;
    const double lt = lT[c] - lrho[c] / (Tv * Tv) + lkap[c] * dk;
    const double x = ph.k * (Z[c] - 1.0);
    lZ[c] += lt * ph.cT * (ph.cA * ph.k * tanh(x) + ph.cB);
    lH[c] += lt * ph.cT;
    lT[c] = 0.0;      // T, rho, kappa are outputs of the state relation
    lrho[c] = 0.0;
    lkap[c] = 0.0;
}

// Face fluxes and Poisson right-hand side transposed, part A.  lFt = total
// adjoint of every interface flux after the outflow shift: the adjoint of the
// final flux (which the projection passes through unchanged) plus its uses in
// b = d_t rho - S_m + sum_j (F_j(hi) - F_j(lo)) / h_j.  Block partials of the
// adjoint of the uniform outflow shift, sum(lFt over high outflow faces) -
// sum(lFt over low outflow faces).
template <int DIM>
__global__ void k_flux_adj_a(Geom g, Bnd bnd, FluxAdj a) {
    __shared__ double sm[NT / 32];
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        int ct[3], q[3];
        interior_coords(g, t, ct);
        padded_coords(g, c, q);
        const double lb = a.lb[t];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const long long st = compact_stride(g, j);
            const double ih = g.ih[j];
            const int n = g.n[j];
            const double lo = a.lF[j][c] - lb * ih + (ct[j] > 0 ? a.lb[t - st] * ih : 0.0);
            a.lFt[j][c] = lo;
            if (ct[j] == 0 && !g.periodic[j] && bnd.kind[j][0][slab_index(g, j, q)] == BC_OUTFLOW) acc -= lo;
            if (ct[j] == n - 1) {
                const double hi = a.lF[j][c + s] + lb * ih;
                a.lFt[j][c + s] = hi;
                if (!g.periodic[j] && bnd.kind[j][1][slab_index(g, j, q)] == BC_OUTFLOW) acc += hi;
            }
        }
    }
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) a.part[blockIdx.x] = acc;
}

// Part B: adjoint of the mass-balance total (shift = -total / area), of the
// density rate (BDF weights onto the three density levels), of S_m, and of
// the provisional momentum through the face interpolation and the extrapolated
// outflow faces.  Consumes lF (zeroed: the fluxes are outputs of this stage).
template <int DIM>
__global__ void k_flux_adj_b(Geom g, Bnd bnd, FluxAdj a, int np) {
    __shared__ double sm[NT / 32];
    const double lshift = sum_partials<NT>(a.part, np, sm);
    const double area = a.sc[SC_OUT_AREA];
    const double ltot = (area > 0.0) ? -lshift / area : 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT) {
        const long long c = pad_index(g, t);
        int ct[3], q[3];
        interior_coords(g, t, ct);
        padded_coords(g, c, q);
        const double ldrho = a.lb[t] + ltot * g.dV;
        const double iden = 1.0 / a.bdf_den;
        a.lrho_new[c] += a.bdf_c0 * iden * ldrho;
        a.lrho_n[c] += a.bdf_c1 * iden * ldrho;
        if (a.bdf_c2 != 0.0) a.lrho_prev[c] += a.bdf_c2 * iden * ldrho;
        if (a.lSm) a.lSm[c] -= ldrho;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long s = g.s[j];
            const int n = g.n[j];
            const double dA = g.dV * g.ih[j];
            const bool per = g.periodic[j];
            double lm = 0.0;
            if (ct[j] > 0 || per) lm += 0.5 * a.lFt[j][c];
            else if (bnd.kind[j][0][slab_index(g, j, q)] == BC_OUTFLOW) lm += a.lFt[j][c] - ltot * dA;
            if (ct[j] < n - 1 || per) lm += 0.5 * a.lFt[j][c + s];
            else if (bnd.kind[j][1][slab_index(g, j, q)] == BC_OUTFLOW) lm += a.lFt[j][c + s] + ltot * dA;
            if (per && ct[j] == 0) lm += 0.5 * a.lFt[j][c + (long long)n * s];          // last cell's wrap face
            if (per && ct[j] == n - 1) lm += 0.5 * a.lFt[j][c - (long long)(n - 1) * s];  // first cell's low face
            a.lmom[j][c] += lm;
            a.lF[j][c] = 0.0;
            if (ct[j] == n - 1) a.lF[j][c + s] = 0.0;
        }
    }
}

// Coefficients of P at position k (one direction) in P_c, P_minus and P_plus of
// the projection at position i (Eqs 3.27-3.28 extrapolation at walls/outflow).
struct PCoef {
    double c, m, p;
};
__device__ __forceinline__ PCoef proj_coef(int i, int k, int n, int per, double eA, double eB, double eC) {
    PCoef r;
    r.c = (i == k) ? 1.0 : 0.0;
    if (i > 0) r.m = (k == i - 1) ? 1.0 : 0.0;
    else if (per) r.m = (k == n - 1) ? 1.0 : 0.0;
    else r.m = (k == i ? eA : 0.0) + (k == i + 1 ? eB : 0.0) + (k == i + 2 ? eC : 0.0);
    if (i < n - 1) r.p = (k == i + 1) ? 1.0 : 0.0;
    else if (per) r.p = (k == 0) ? 1.0 : 0.0;
    else r.p = (k == i ? eA : 0.0) + (k == i - 1 ? eB : 0.0) + (k == i - 2 ? eC : 0.0);
    return r;
}

// Projection transposed (Eqs 3.23, 3.25, 3.27-3.28): from the adjoints of the
// projected velocity lv (interior) and of the final fluxes lF (unchanged: the
// provisional fluxes carry them on), adds lmom += lv / rho,
// lT += lv (mom - delta_2 P / 2h) / p0, and sets lP (compact) by gathering, for
// every pressure value, the projection positions that read it.
template <int DIM>
__global__ void k_project_adj(Geom g, ProjAdj a) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    int ct[3];
    interior_coords(g, t, ct);
    const double ip0 = a.sc[a.p0_slot + SC_INV_OFF];
    const double irho = a.T[c] * ip0;
    const double Pc = a.P[t];
    double lT = 0.0, lP = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const long long s = g.s[j];
        const long long st = compact_stride(g, j);
        const int n = g.n[j];
        const int per = g.periodic[j];
        const double ih = g.ih[j];
        double Pm, Pp;
        if (ct[j] > 0) Pm = a.P[t - st];
        else if (per) Pm = a.P[t + (long long)(n - 1) * st];
        else Pm = a.eA * Pc + a.eB * a.P[t + st] + a.eC * a.P[t + 2 * st];
        if (ct[j] < n - 1) Pp = a.P[t + st];
        else if (per) Pp = a.P[t - (long long)(n - 1) * st];
        else Pp = a.eA * Pc + a.eB * a.P[t - st] + a.eC * a.P[t - 2 * st];
        const double lv = a.lv[j][c];
        a.lmom[j][c] += lv * irho;
        lT += lv * (a.mom[j][c] - (Pp - Pm) * (0.5 * ih)) * ip0;

        // gather over the positions i whose projection reads P at k = ct[j]
        const int k = ct[j];
        int cand[7];
        int nc = 0;
        for (int i = (k - 2 > 0 ? k - 2 : 0); i <= (k + 2 < n - 1 ? k + 2 : n - 1); ++i) cand[nc++] = i;
        if (per && k == n - 1 && 0 < k - 2) cand[nc++] = 0;
        if (per && k == 0 && n - 1 > 2) cand[nc++] = n - 1;
        for (int m = 0; m < nc; ++m) {
            const int i = cand[m];
            const PCoef co = proj_coef(i, k, n, per, a.eA, a.eB, a.eC);
            const long long ci = c + (long long)(i - k) * s;
            const double irho_i = a.T[ci] * ip0;
            lP += a.lv[j][ci] * (-0.5 * ih * irho_i) * (co.p - co.m);
            if (i > 0 || per) lP += a.lF[j][ci] * (-ih) * (co.c - co.m);
            if (i == n - 1 && per) lP += a.lF[j][ci + s] * (-ih) * (co.p - co.c);
        }
    }
    a.lT[c] += lT;
    a.lP[t] = lP;
}

// AB2 / Euler (predictor) or AM2 (corrector) combination transposed
// (Eqs 3.1-3.4, 3.12-3.13, 3.16): X = X_b + dt * (weights of R_now, R_hist).
//   corrector: lR = dt/2 (lmom, lZ, lH); lRh += dt/2 (...); lv = rho^n lmom;
//              lrho_n += v^n . lmom; lZ, lH carry on to level n unchanged.
//   predictor: lR = lRh + w dt (lmom, lZs, lHs) (w = 3/2 AB2, 1 Euler);
//              lRh = -dt/2 (...) (AB2) or 0; lv += rho^n lmom; lrho_n += v^n . lmom;
//              lZ += lZs, lH += lHs.
template <int DIM>
__global__ void k_comb_adj(Geom g, CombAdj a) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= g.ncell) return;
    const long long c = pad_index(g, t);
    const double dt = a.dt;
    const double rn = a.rho_n[c];
    double lr = 0.0;
    double lin[5];
#pragma unroll
    for (int i = 0; i < DIM; ++i) lin[i] = a.lmom[i][c];
    lin[3] = a.lZin[c];
    lin[4] = a.lHin[c];
    if (a.mode == MODE_CORR) {
        const double h = 0.5 * dt;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            a.lR[i][c] = h * lin[i];
            a.lRh[i][c] += h * lin[i];
            a.lv[i][c] = rn * lin[i];
            lr += a.v_n[i][c] * lin[i];
        }
        for (int k = 3; k < 5; ++k) {
            a.lR[k][c] = h * lin[k];
            a.lRh[k][c] += h * lin[k];
        }
    } else {
        const bool ab2 = a.mode == MODE_PRED_AB2;
        const double w = ab2 ? 1.5 * dt : dt;
        const double wh = ab2 ? -0.5 * dt : 0.0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            a.lR[i][c] = a.lRh[i][c] + w * lin[i];
            a.lRh[i][c] = wh * lin[i];
            a.lv[i][c] += rn * lin[i];
            lr += a.v_n[i][c] * lin[i];
        }
        for (int k = 3; k < 5; ++k) {
            a.lR[k][c] = a.lRh[k][c] + w * lin[k];
            a.lRh[k][c] = wh * lin[k];
        }
        a.lZ[c] += lin[3];
        a.lH[c] += lin[4];
    }
    a.lrho_n[c] += lr;
}

// Heat-release rate of the flame sheet with unit Lewis number:
// omega = -Q/(S+1) F_eps''(Z) kappa |grad Z|^2 / Pe
//       = (Q/S)(k/2) sech^2(k (Z - 1)) kappa |delta_2 Z|^2 / Pe   (Eqs 2.30, 3.41).
struct ObjLoad {
    const double* Z;
    const double* kap;
    int sf;
    long long si;
    __device__ __forceinline__ Dual operator()(int f, long long i) const {
        const double v = (f == RF_Z) ? Z[i] : kap[i];
        return Dual(v, (f == sf && i == si) ? 1.0 : 0.0);
    }
};
struct ObjPlain {
    const double* Z;
    const double* kap;
    __device__ __forceinline__ double operator()(int f, long long i) const { return (f == RF_Z) ? Z[i] : kap[i]; }
};

template <int DIM, class C, class LD>
__device__ __forceinline__ C omega_cell(const Geom& g, const Phys& ph, long long c, const LD& ld) {
    const C th = tanh_c((C)ph.k * (ld(RF_Z, c) - (C)1.0));
    C g2 = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const C dz = (ld(RF_Z, c + g.s[j]) - ld(RF_Z, c - g.s[j])) * (C)(0.5 * g.ih[j]);
        g2 = g2 + dz * dz;
    }
    const double coef = ph.Q / ph.S * 0.5 * ph.k / ph.Pe;
    return (C)coef * ((C)1.0 - th * th) * ld(RF_KAP, c) * g2;
}

template <int DIM>
__global__ void k_objective(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ kap,
                            double* part) {
    __shared__ double sm[NT / 32];
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < g.ncell; t += (long long)gridDim.x * NT)
        acc += omega_cell<DIM, double>(g, ph, pad_index(g, t), ObjPlain{Z, kap});
    acc = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// lZ[j] += w d(sum_c omega_c dV)/dZ_j over the cells c within one step of j;
// lkap[j] += w dV d omega_j / d kappa_j (j interior).
template <int DIM>
__global__ void k_objective_adj(Geom g, Phys ph, const double* __restrict__ Z, const double* __restrict__ kap,
                                double w, double* lZ, double* lkap) {
    const long long j = (long long)blockIdx.x * NT + threadIdx.x;
    if (j >= g.npad) return;
    int q[3];
    padded_coords(g, j, q);
    const double wv = w * g.dV;
    double az = 0.0;
    if (padded_interior(g, q)) {
        az += omega_cell<DIM, Dual>(g, ph, j, ObjLoad{Z, kap, RF_Z, j}).d;
        lkap[j] += wv * omega_cell<DIM, Dual>(g, ph, j, ObjLoad{Z, kap, RF_KAP, j}).d;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int qc[3] = {q[0], q[1], q[2]};
            qc[d] += sgn;
            if (!padded_interior(g, qc)) continue;
            az += omega_cell<DIM, Dual>(g, ph, j + sgn * g.s[d], ObjLoad{Z, kap, RF_Z, j}).d;
        }
    lZ[j] += wv * az;
}

// Gradient of the adjoint-weighted IBM forcing with respect to the slot's
// flux-profile samples.  v_ib,2 = m U (x_2 - y_lo) / (y_hi - y_lo) and
// S_m = chi rho_b U / (n_col h_2) are linear in U = U_b base(x) mod(x), mod the
// piecewise-linear interpolant of the samples (the forward set-up kernel), so
// per column: col = U_b base(x) sum_rows (lvib2 m (x_2 - y_lo)/(y_hi - y_lo)
// + lSm chi rho_b / (n_col h_2)), then spread on the two samples around x.
__global__ void k_profile_col(Geom g, IbmDev b, const uint8_t* __restrict__ chi, const double* __restrict__ lvib1,
                              const double* __restrict__ lSm, double* col) {
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i >= g.n[0]) return;
    const double x = ((double)(i + 1) - 0.5) * g.h[0];
    const double r = (x - b.c[0]) / (b.half[0] + b.s);
    double base = 1.0 - r * r;
    base = base > 0.0 ? base : 0.0;
    const double ylo = b.c[1] - b.half[1] - b.s, yhi = b.c[1] + b.half[1] + b.s;
    int cnt = 0;
    for (int j = 1; j <= g.n[1]; ++j) cnt += chi[(i + 1) + (long long)j * g.s[1]];
    const double nc = cnt > 0 ? (double)cnt : 1.0;
    double acc = 0.0;
    for (int j = 1; j <= g.n[1]; ++j) {
        const long long c = (i + 1) + (long long)j * g.s[1];
        if (!chi[c]) continue;
        const double y = ((double)j - 0.5) * g.h[1];
        acc += lvib1[c] * (y - ylo) / (yhi - ylo) + lSm[c] * b.rho_b / (nc * g.h[1]);
    }
    col[i] = b.U_b * base * acc;
}

__global__ void k_profile_spread(Geom g, IbmDev b, const double* __restrict__ col, double* grad) {
    const int k = blockIdx.x * NT + threadIdx.x;
    if (k >= b.n_profile) return;
    const double lo = b.c[0] - b.half[0] - b.s, hi = b.c[0] + b.half[0] + b.s;
    double acc = 0.0;
    for (int i = 0; i < g.n[0]; ++i) {
        const double x = ((double)(i + 1) - 0.5) * g.h[0];
        double wk;
        if (x <= lo) wk = (k == 0) ? 1.0 : 0.0;
        else if (x >= hi) wk = (k == b.n_profile - 1) ? 1.0 : 0.0;
        else {
            const double pos = (x - lo) / (hi - lo) * (double)(b.n_profile - 1);
            int i0 = (int)floor(pos);
            if (i0 > b.n_profile - 2) i0 = b.n_profile - 2;
            const double fr = pos - (double)i0;
            wk = (k == i0) ? 1.0 - fr : (k == i0 + 1) ? fr : 0.0;
        }
        acc += wk * col[i];
    }
    grad[k] = acc;
}

// ----------------------------------------------------------------------------
// Member-batched stage kernels: block b of the launch belongs to the member m
// with start[m] <= b < start[m+1] (binary search over the work list), as its
// member-local block b - start[m]; the member's record is staged in shared
// memory, then the stage body runs exactly as in the member's own launch.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int member_of_block(const int* __restrict__ start, int nm, int b) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Copy of the record into shared memory (8-byte words), then a barrier.
__device__ __forceinline__ int stage_rec(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm,
                                         StageRec* srec) {
    __shared__ int s_m;
    if (threadIdx.x == 0) s_m = member_of_block(start, nm, blockIdx.x);
    __syncthreads();
    const int m = s_m;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(recs + m);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(srec);
    for (int i = threadIdx.x; i < (int)(sizeof(StageRec) / 8); i += NT) dst[i] = src[i];
    __syncthreads();
    return blockIdx.x - start[m];
}

template <int DIM, class C>
__global__ void __launch_bounds__(NT, ResidMinBlocks<DIM, C>::v)
    k_residual_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    residual_body<DIM, C>(r.g, r.ph, r.u.r, bx);
}

template <int DIM, bool MIXED>
__global__ void k_state_flux_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    const StageSF& q = r.u.sf;
    state_flux_body<DIM, MIXED>(r.g, r.ph, q.Z, q.H, q.T, q.rho, q.kap, q.status, q.sc, q.bnd, q.kap_ghosts, q.fa,
                                bx, r.nblocks);
}

template <int DIM>
__global__ void k_rhs_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    rhs_body<DIM>(r.g, r.u.sf.bnd, r.u.sf.fa, r.np, bx, r.nblocks);
}

template <int DIM>
__global__ void k_project_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    project_body<DIM>(r.g, r.ph, r.u.p, bx);
}

template <int DIM, class C>
__global__ void __launch_bounds__(NT, ResidMinBlocks<DIM, C>::v)
    k_residual_img_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    residual_body<DIM, C, true>(r.g, r.ph, r.u.r, bx);
}

__global__ void k_ff_images_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    const StageImg& q = r.u.im;
    const long long p = (long long)bx * NT + threadIdx.x;
    if (p >= q.npad) return;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (!q.src.f[f]) continue;
        const FF w(q.src.f[f][p]);
        q.dst[(long long)f * q.npad + p] = make_float2(w.hi, w.lo);
    }
}

__global__ void k_copy_b(const StageRec* __restrict__ recs, const int* __restrict__ start, int nm) {
    __shared__ __align__(16) StageRec r;
    const int bx = stage_rec(recs, start, nm, &r);
    const StageCopy& q = r.u.cp;
    const long long t = (long long)bx * NT + threadIdx.x;
    if (t < q.n) q.dst[t] = q.src[t];
}

thread_local StageCollector* t_collect = nullptr;

bool collect(const StageRec& rec) {
    if (!t_collect) return false;
    if (t_collect->n < t_collect->cap) t_collect->recs[t_collect->n] = rec;
    else t_collect->overflow = true;
    ++t_collect->n;
    return true;
}

}  // namespace

void set_stage_collector(StageCollector* c) { t_collect = c; }
bool stage_collecting() { return t_collect != nullptr; }

cudaError_t stage_copy(const double* src, double* dst, long long n, cudaStream_t s) {
    if (t_collect) {
        StageRec r;
        std::memset(&r, 0, sizeof(r));
        r.kind = SK_COPY;
        r.nblocks = blocks_for(n);
        r.u.cp.src = src;
        r.u.cp.dst = dst;
        r.u.cp.n = n;
        collect(r);
        return cudaSuccess;
    }
    return cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_stage_batched(int kind, int dim, int mixed, const StageRec* recs, const int* start, int nm,
                                 int total_blocks, cudaStream_t s) {
    const dim3 grid((unsigned)total_blocks);
    switch (kind) {
        case SK_RESID:
            if (dim == 3) {
                if (mixed) k_residual_b<3, FF><<<grid, NT, 0, s>>>(recs, start, nm);
                else k_residual_b<3, double><<<grid, NT, 0, s>>>(recs, start, nm);
            } else {
                if (mixed) k_residual_b<2, FF><<<grid, NT, 0, s>>>(recs, start, nm);
                else k_residual_b<2, double><<<grid, NT, 0, s>>>(recs, start, nm);
            }
            break;
        case SK_STATE_FLUX:
            if (dim == 3) {
                if (mixed) k_state_flux_b<3, true><<<grid, NT, 0, s>>>(recs, start, nm);
                else k_state_flux_b<3, false><<<grid, NT, 0, s>>>(recs, start, nm);
            } else {
                if (mixed) k_state_flux_b<2, true><<<grid, NT, 0, s>>>(recs, start, nm);
                else k_state_flux_b<2, false><<<grid, NT, 0, s>>>(recs, start, nm);
            }
            break;
        case SK_RHS:
            if (dim == 3) k_rhs_b<3><<<grid, NT, 0, s>>>(recs, start, nm);
            else k_rhs_b<2><<<grid, NT, 0, s>>>(recs, start, nm);
            break;
        case SK_PROJECT:
            if (dim == 3) k_project_b<3><<<grid, NT, 0, s>>>(recs, start, nm);
            else k_project_b<2><<<grid, NT, 0, s>>>(recs, start, nm);
            break;
        case SK_IMAGES:
            k_ff_images_b<<<grid, NT, 0, s>>>(recs, start, nm);
            break;
        case SK_RESID_IMG:   // the float-float stencil reading its inputs' images
            if (dim == 3) k_residual_img_b<3, FF><<<grid, NT, 0, s>>>(recs, start, nm);
            else k_residual_img_b<2, FF><<<grid, NT, 0, s>>>(recs, start, nm);
            break;
        default:
            k_copy_b<<<grid, NT, 0, s>>>(recs, start, nm);
    }
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(const Geom& g, const DiagArgs& a, cudaStream_t st) {
    long long nb = (g.ncell + NT - 1) / NT;
    if (nb > kDiagBlocks) nb = kDiagBlocks;
    if (g.dim == 3) k_diag<3><<<(int)nb, NT, 0, st>>>(g, a);
    else k_diag<2><<<(int)nb, NT, 0, st>>>(g, a);
    k_diag_final<<<1, NT, 0, st>>>(g, a, (int)nb);
    return cudaGetLastError();
}


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
                  int* launches, const Bnd* bnd, bool kap_ghosts) {
    const int rb = reduce_grid(g);
    Bnd b;
    std::memset(&b, 0, sizeof(b));
    if (bnd) b = *bnd;
    const int kg = (bnd && kap_ghosts) ? 1 : 0;
    if (ph.mixed)
        k_state<true><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, part, status, sc, p0_slot, b, kg);
    else
        k_state<false><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, part, status, sc, p0_slot, b, kg);
    ++*launches;
    if (ph.closed) {
        k_density<<<rb, NT, 0, s>>>(g, T, rho, part, rb, sc, p0_slot, ph.mixed, ph.semi);
        ++*launches;
    }
}

void launch_ff_images(const Geom& g, const double* const src[6], float2* dst, cudaStream_t s, int* launches) {
    FFSrc fs;
    for (int f = 0; f < 6; ++f) fs.f[f] = (f == 2 && g.dim == 2) ? nullptr : src[f];
    if (t_collect) {
        StageRec r;
        std::memset(&r, 0, sizeof(r));
        r.g = g;
        r.kind = SK_IMAGES;
        r.nblocks = blocks_for(g.npad);
        r.u.im.src = fs;
        r.u.im.dst = dst;
        r.u.im.npad = g.npad;
        collect(r);
        ++*launches;
        return;
    }
    // one padded cell per thread (192^3: 14.49 -> 14.43 ms per step against a
    // grid-stride loop over 8 x 152 blocks)
    const long long nb = (g.npad + NT - 1) / NT;
    k_ff_images<<<(int)nb, NT, 0, s>>>(g.npad, 6, fs, dst);
    ++*launches;
}

void launch_p0_ode(const Geom& g, const Phys& ph, const double* Z, const double* H, const double* kap,
                   double* const* v, double* part, double* sc, int stage, double dt, int out_slot, cudaStream_t s,
                   int* launches) {
    const int rb = reduce_grid(g);
    const double* v2 = (g.dim == 3) ? v[2] : v[0];
    if (g.dim == 3) k_p0_rate<3><<<rb, NT, 0, s>>>(g, ph, Z, H, kap, v[0], v[1], v2, part);
    else k_p0_rate<2><<<rb, NT, 0, s>>>(g, ph, Z, H, kap, v[0], v[1], v2, part);
    k_p0_ode<<<1, NT, 0, s>>>(g, ph, part, rb, sc, stage, dt, out_slot);
    *launches += 2;
}

void launch_residual(const Geom& g, const Phys& ph, const ResidArgs& a, cudaStream_t s, int* launches) {
    const int nb = blocks_for(g.ncell);
    if (t_collect) {
        StageRec r;
        std::memset(&r, 0, sizeof(r));
        r.g = g;
        r.ph = ph;
        r.kind = (a.ffs && ph.mixed) ? SK_RESID_IMG : SK_RESID;
        r.nblocks = nb;
        r.u.r = a;
        collect(r);
        ++*launches;
        return;
    }
    // FP64, or float-float (~48 bits on the FP32 pipes) in the mixed path: the
    // pressure is the dt-scaled divergence of the momentum increment and
    // inherits the stencil's relative rounding directly, which plain FP32
    // (24 bits) leaves above 1e-6
    if (ph.mixed) {
        if (g.dim == 3) {
            if (a.ffs) k_residual<3, FF, true><<<nb, NT, 0, s>>>(g, ph, a);
            else k_residual<3, FF><<<nb, NT, 0, s>>>(g, ph, a);
        } else {
            if (a.ffs) k_residual<2, FF, true><<<nb, NT, 0, s>>>(g, ph, a);
            else k_residual<2, FF><<<nb, NT, 0, s>>>(g, ph, a);
        }
    } else {
        if (g.dim == 3) k_residual<3, double><<<nb, NT, 0, s>>>(g, ph, a);
        else k_residual<2, double><<<nb, NT, 0, s>>>(g, ph, a);
    }
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

void launch_state_flux_rhs(const Geom& g, const Phys& ph, const double* Z, const double* H, double* T, double* rho,
                           double* kap, double* sc, int* status, const Bnd& bnd, bool kap_ghosts, const FluxArgs& a,
                           cudaStream_t s, int* launches) {
    const int rb = reduce_grid(g);
    const int kg = kap_ghosts ? 1 : 0;
    if (t_collect) {
        StageRec r;
        std::memset(&r, 0, sizeof(r));
        r.g = g;
        r.ph = ph;
        r.kind = SK_STATE_FLUX;
        r.nblocks = rb;
        r.np = rb;
        r.u.sf.Z = Z;
        r.u.sf.H = H;
        r.u.sf.T = T;
        r.u.sf.rho = rho;
        r.u.sf.kap = kap;
        r.u.sf.status = status;
        r.u.sf.sc = sc;
        r.u.sf.bnd = bnd;
        r.u.sf.kap_ghosts = kg;
        r.u.sf.fa = a;
        collect(r);
        r.kind = SK_RHS;
        collect(r);
        *launches += 2;
        return;
    }
    if (g.dim == 3) {
        if (ph.mixed) k_state_flux<3, true><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, status, sc, bnd, kg, a);
        else k_state_flux<3, false><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, status, sc, bnd, kg, a);
        k_rhs<3><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    } else {
        if (ph.mixed) k_state_flux<2, true><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, status, sc, bnd, kg, a);
        else k_state_flux<2, false><<<rb, NT, 0, s>>>(g, ph, Z, H, T, rho, kap, status, sc, bnd, kg, a);
        k_rhs<2><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    }
    *launches += 2;
}

void launch_project(const Geom& g, const Phys& ph, const ProjArgs& a, cudaStream_t s, int* launches) {
    if (t_collect) {
        StageRec r;
        std::memset(&r, 0, sizeof(r));
        r.g = g;
        r.ph = ph;
        r.kind = SK_PROJECT;
        r.nblocks = cell_blocks(g);
        r.u.p = a;
        collect(r);
        ++*launches;
        return;
    }
    if (g.dim == 3)
        k_project<3><<<cell_blocks(g), NT, 0, s>>>(g, ph, a);
    else
        k_project<2><<<cell_blocks(g), NT, 0, s>>>(g, ph, a);
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

void launch_marker_cells(const Geom& g, const IbmDev& b, uint8_t* chi, double* vib[3], double* U, double* Sm,
                         int* near, int* counts, cudaStream_t s) {
    k_marker_cells<<<blocks_for(g.npad), NT, 0, s>>>(g, b, chi, vib[0], vib[1], vib[2], U, Sm, near, counts);
}

void launch_marker_source(const Geom& g, const IbmDev& b, const uint8_t* chi, const int* near, const int* counts,
                          double* Sm, cudaStream_t s) {
    k_marker_source<<<blocks_for(g.ncell), NT, 0, s>>>(g, b, chi, near, counts, Sm);
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

void launch_add_unpack(const Geom& g, const double* compact, double* padded, cudaStream_t s) {
    k_add_unpack<<<blocks_for(g.ncell), NT, 0, s>>>(g, compact, padded);
}

void launch_gather(const double* const* src, double* dst, long long N, int nb, cudaStream_t s) {
    k_gather<<<dim3(reduce_blocks(N), nb), NT, 0, s>>>(src, dst, N);
}
void launch_scatter(const double* src, double* const* dst, long long N, int nb, cudaStream_t s) {
    k_scatter<<<dim3(reduce_blocks(N), nb), NT, 0, s>>>(src, dst, N);
}

void launch_u8_to_double(const Geom& g, const uint8_t* padded, double* compact, cudaStream_t s) {
    k_u8_to_double<<<blocks_for(g.ncell), NT, 0, s>>>(g, padded, compact);
}

// ------------------------------- adjoint launchers -------------------------------
void launch_residual_adj(const Geom& g, const Phys& ph, const ResidArgs& a, double p0dot, const AdjR& lr,
                         const AdjIn& li, double* cont, cudaStream_t s) {
    if (cont && g.dim == 2) {
        k_residual_rev<<<blocks_for(g.ncell), NT, 0, s>>>(g, ph, a, p0dot, lr, cont);
        k_residual_rev_gather<<<blocks_for(g.npad), NT, 0, s>>>(g, cont, li);
        return;
    }
    if (g.dim == 3) k_residual_adj<3><<<blocks_for(g.npad), NT, 0, s>>>(g, ph, a, p0dot, lr, li);
    else k_residual_adj<2><<<blocks_for(g.npad), NT, 0, s>>>(g, ph, a, p0dot, lr, li);
}

int residual_rev_slots() { return SL_N; }

void launch_ghost_adj(const Geom& g, const Bnd& bnd, const GhostJob& job, cudaStream_t s) {
    for (int d = g.dim - 1; d >= 0; --d) {   // the forward fill runs d = 0, 1, 2
        const int a = (d == 0) ? 1 : 0;
        const int b = (d == 2) ? 1 : 2;
        const long long nslab = (long long)g.p[a] * g.p[b];
        k_ghost_adj<<<blocks_for(nslab), NT, 0, s>>>(g, bnd.kind[d][0], bnd.kind[d][1], d, g.periodic[d], job);
    }
}

void launch_state_adj(const Geom& g, const Phys& ph, const double* Z, const double* T, const double* kap,
                      double* lT, double* lrho, double* lkap, double* lZ, double* lH, cudaStream_t s) {
    k_state_adj<<<blocks_for(g.ncell), NT, 0, s>>>(g, ph, Z, T, kap, lT, lrho, lkap, lZ, lH);
}

void launch_flux_adj(const Geom& g, const Bnd& bnd, const FluxAdj& a, cudaStream_t s) {
    const int rb = reduce_grid(g);
    if (g.dim == 3) {
        k_flux_adj_a<3><<<rb, NT, 0, s>>>(g, bnd, a);
        k_flux_adj_b<3><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    } else {
        k_flux_adj_a<2><<<rb, NT, 0, s>>>(g, bnd, a);
        k_flux_adj_b<2><<<rb, NT, 0, s>>>(g, bnd, a, rb);
    }
}

void launch_project_adj(const Geom& g, const ProjAdj& a, cudaStream_t s) {
    if (g.dim == 3) k_project_adj<3><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
    else k_project_adj<2><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
}

void launch_comb_adj(const Geom& g, const CombAdj& a, cudaStream_t s) {
    if (g.dim == 3) k_comb_adj<3><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
    else k_comb_adj<2><<<blocks_for(g.ncell), NT, 0, s>>>(g, a);
}

void launch_objective(const Geom& g, const Phys& ph, const double* Z, const double* kap, double* part,
                      double* out, cudaStream_t s) {
    const int rb = reduce_grid(g);
    if (g.dim == 3) k_objective<3><<<rb, NT, 0, s>>>(g, ph, Z, kap, part);
    else k_objective<2><<<rb, NT, 0, s>>>(g, ph, Z, kap, part);
    k_store_sum<<<1, NT, 0, s>>>(part, rb, g.dV, out);
}

void launch_objective_adj(const Geom& g, const Phys& ph, const double* Z, const double* kap, double w, double* lZ,
                          double* lkap, cudaStream_t s) {
    if (g.dim == 3) k_objective_adj<3><<<blocks_for(g.npad), NT, 0, s>>>(g, ph, Z, kap, w, lZ, lkap);
    else k_objective_adj<2><<<blocks_for(g.npad), NT, 0, s>>>(g, ph, Z, kap, w, lZ, lkap);
}

void launch_profile_grad(const Geom& g, const IbmDev& b, const uint8_t* chi, const double* lvib1,
                         const double* lSm, double* col, double* grad, cudaStream_t s) {
    k_profile_col<<<blocks_for(g.n[0]), NT, 0, s>>>(g, b, chi, lvib1, lSm, col);
    k_profile_spread<<<blocks_for(b.n_profile), NT, 0, s>>>(g, b, col, grad);
}

}  // namespace lm
