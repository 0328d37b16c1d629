// C ABI of the low-Mach flame-sheet step (include/lowmach.h) and the host-side
// orchestration of one time step: the predictor / corrector launch sequence of
// paper Sec. 3.1 (Eqs 3.1-3.19), CUDA-graph capture of a whole step with one
// conditional while node per pressure solve, and the t = 0 initialisation.

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/lowmach.h"
#include "poisson.cuh"
#include "step.cuh"

using namespace lm;

namespace {

constexpr int kMaxProfile = 4096;

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// Discrete adjoint state: lambda arrays (padded layout unless noted) and the
// forward values of the recomputed step that its transposes read.
struct AdjWs {
    double* Lv[3];          // lambda of v at the level being stepped back to
    double* Lvs[3];         // lambda of v*
    double *LZ, *LH, *LZs, *LHs, *LT, *Lkap;
    double* LF[3];          // lambda of the interface fluxes
    double* LFt[3];         // scratch of the flux transpose
    double* LRh[5];         // lambda of the stored residual history
    double* LR[5];          // lambda of the stage residual being transposed
    double* Lm[3];          // lambda of the provisional momentum
    double* Lr[3];          // rotating lambda of the density levels
    int i_rho, i_prev;      // Lr roles: rho at the level, rho one level below
    double* Lvib[3];        // accumulated lambda of v_ib over all steps
    double* LSm;            // accumulated lambda of S_m over all steps
    double *LP, *Lb;        // compact: lambda of P and of the Poisson rhs
    double* v0[3];          // level-n forward values
    double *Z0, *H0, *T0, *kap0, *rho0;
    double* F0[3];
    double* m0[3];          // predictor values: provisional momentum, T*, kappa*, P*, F*
    double *Ts, *kaps, *Ps;
    double* rhos;           // rho* (read by the buoyancy term of the corrector's stencil)
    double* Fs[3];
    double *col, *grad, *obj, *rep, *part;
    double* cont;           // scratch of the reverse stencil sweep (slots x padded cells)
    int use_dual;           // 1: exact dual-number stencil transpose (LOWMACH_ADJ_DUAL=1)
    char* lam_base;         // lambda region (zeroed by begin)
    size_t lam_bytes;
};

struct sim {
    sim_params_t prm;
    Geom g;
    Phys ph;
    cudaStream_t stream;   // caller's stream (work is enqueued here)
    cudaStream_t cap;      // private stream used for graph capture
    cudaStream_t side;     // private stream used to capture while-node bodies

    double* v[3];
    double* vs[3];
    double *Z, *H, *Zs, *Hs, *T, *kap;
    double* rho[3];
    double* mom[3];
    double* F[3];
    double* R[2][5];
    double* vib[3];
    double *Sm, *U;
    double *P, *b, *io;
    double* Pstar;         // the predictor's P of the last step (per-step checks)
    double *Pm1, *Pd;      // warm-start history: P of the step before, P - P* of the last step
    long long hist_from = 0;   // the step from which that history is being kept (set-up or load)
    double* diag;          // per-step check partials and results
    double* part;
    double* part2;
    double* ode_part;                     // block partials of Eq 2.38's sums (semi-enclosed)
    float2* ffs;                          // 3D mixed: float-float images of the stencil inputs (or null)
    double* sc;
    double* profile;
    int* status;
    uint8_t* chi;
    uint8_t* kind[3][2];

    PoissonPlan pp;
    std::vector<double> minv;
    Bnd bnd;
    double eA, eB, eC;

    int ibm_active;
    double Z_ib, H_ib, Da;

    int fields_set;        // bit mask of U, V, W, Z, H set since create
    bool need_init;
    long long nstep;
    int rho_base;
    double t;

    int launches_last;
    int launches_fixed_graph[6];
    int body_launches;
    cudaGraphExec_t gexec[6];
    bool gvalid[6];
    int use_graph;

    IbmDev ibm;            // body description of the last set-up (device profile copy)
    AdjWs adj;
    bool adj_active;
    bool adj_save;         // the eager step copies its predictor values into adj
    // Adjoint steps run their pressure solves (recompute: predictor,
    // corrector; transpose: lambda_P -> lambda_b) as captured one-solve
    // graphs instead of the host-driven loop.
    bool solve_graphs;
    cudaGraphExec_t solve_exec[3];
    bool solve_valid[3];
    int solve_fixed[3], solve_body[3];   // kernels of a solve graph outside / per loop iteration
    cudaStream_t save_stream = nullptr;   // private stream: the restart blob's early part (sim_step_save)
    cudaEvent_t ev_early = nullptr;   // recorded in a step once the early state arrays are final

    char err[512];
};

namespace {

sim_status fail(sim_t* s, sim_status st, const char* fmt, ...) {
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->err, sizeof(s->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(s, SIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

Geom make_geom(const sim_params_t* p) {
    Geom g;
    std::memset(&g, 0, sizeof(g));
    g.dim = p->dim;
    for (int d = 0; d < 3; ++d) {
        const bool act = d < p->dim;
        g.n[d] = act ? p->n[d] : 1;
        g.p[d] = act ? p->n[d] + 2 : 1;
        g.h[d] = act ? p->L[d] / p->n[d] : 1.0;
        g.ih[d] = 1.0 / g.h[d];
        g.ih2[d] = g.ih[d] * g.ih[d];
        g.periodic[d] = act ? (p->bc[d][0] == SIM_BC_PERIODIC) : 0;
    }
    g.s[0] = 1;
    g.s[1] = g.p[0];
    g.s[2] = (long long)g.p[0] * g.p[1];
    g.npad = (long long)g.p[0] * g.p[1] * g.p[2];
    g.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    g.dV = 1.0;
    for (int d = 0; d < p->dim; ++d) g.dV *= g.h[d];
    g.dn0 = make_divu32((unsigned)g.n[0]);
    g.dn1 = make_divu32((unsigned)g.n[1]);
    g.dp0 = make_divu32((unsigned)g.p[0]);
    g.dp1 = make_divu32((unsigned)g.p[1]);
    g.tile_x = p->stage_tile_x;
    return g;
}

double host_temperature(const Phys& ph, double z, double h) {
    const double x = ph.k * (z - 1.0);
    const double ax = std::fabs(x);
    const double F =
        (-(ph.S + 1.0) * (ax + std::log1p(std::exp(-2.0 * ax))) / ph.k + (ph.S - 1.0) * (z - 1.0)) / (2.0 * ph.S);
    return ph.Q / (ph.S + 1.0) * (F + h);
}

Phys make_phys(const sim_params_t* p) {
    Phys ph;
    std::memset(&ph, 0, sizeof(ph));
    ph.S = 1.0 / p->Z_st - 1.0;                                  // Eq 2.34 with Z_st
    ph.Q = (p->density_ratio - 1.0) * (ph.S + 1.0);              // flame temperature = ratio
    ph.k = std::log((1.0 - p->tol_reg) / p->tol_reg) / (2.0 * p->eps_reg);  // text after Eq 3.34
    ph.Pe = p->Re * p->Pr;
    ph.PrPe = p->Pr / ph.Pe;
    ph.zeta = (ph.S + 1.0) * (p->gamma - 1.0) / (p->gamma * ph.Q);
    ph.Le_F = p->Le_F;
    ph.Le_O = p->Le_O;
    ph.N_F = (1.0 - p->Le_F) / (ph.S * p->Le_F);
    ph.N_O = (p->Le_O - 1.0) / p->Le_O;
    ph.cA = -(ph.S + 1.0) / (2.0 * ph.S * ph.k);                 // Eq 3.41 folded into Eq 3.42
    ph.cB = (ph.S - 1.0) / (2.0 * ph.S);
    ph.cT = ph.Q / (ph.S + 1.0);
    ph.iPe = 1.0 / ph.Pe;
    ph.iLePe = 1.0 / (p->Le_O * ph.Pe);
    ph.mixed = (p->precision == SIM_MIXED);
    ph.sigma_is_07 = (p->sigma == 0.7);
    ph.sigma = p->sigma;
    ph.transport = p->transport;
    ph.suth_C = p->sutherland_C;
    ph.inv_Fr2 = p->inv_Fr2;
    for (int d = 0; d < 3; ++d) ph.inflow_v[d] = p->inflow_v[d];
    ph.inflow_Z = p->inflow_Z;
    ph.inflow_H = p->inflow_H;
    ph.incompressible = p->incompressible;
    ph.closed = p->closed_system != 0 && !p->incompressible;
    ph.semi = p->closed_system == 2 && !p->incompressible;
    ph.NpF = -1.0 / ph.S;                                        // Eq 2.39
    ph.NpO = 1.0;
    {
        double vol = 1.0;
        for (int d = 0; d < p->dim; ++d) vol *= p->L[d];
        ph.ode_gV = p->gamma / vol;                              // Eq 2.38
        ph.ode_heat = ph.Q / ((ph.S + 1.0) * ph.Pe);
    }
    bool inflow = false;
    for (int d = 0; d < p->dim; ++d)
        for (int q = 0; q < 2; ++q) inflow |= (p->bc[d][q] == SIM_BC_INFLOW);
    if (p->incompressible) {
        ph.rho_in_T = 1.0;
        ph.kappa_in = 1.0;
    } else if (inflow) {
        ph.rho_in_T = host_temperature(ph, p->inflow_Z, p->inflow_H);
        ph.kappa_in = kappa_of(ph, ph.rho_in_T);
    } else {
        ph.rho_in_T = 1.0;
        ph.kappa_in = 1.0;
    }
    // isothermal walls: Dirichlet H of the side, kappa of the wall state (Z_in, H_wall)
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 2; ++q) {
            ph.wall_H[d][q] = p->wall_H[d][q];
            ph.kap_wall[d][q] = 1.0;
            if (d < p->dim && p->bc[d][q] == SIM_BC_WALL_T && !p->incompressible)
                ph.kap_wall[d][q] = kappa_of(ph, host_temperature(ph, p->inflow_Z, p->wall_H[d][q]));
        }
    return ph;
}

const char* validate(const sim_params_t* p) {
    if (!p) return "null parameters";
    if (p->dim != 2 && p->dim != 3) return "dim must be 2 or 3";
    for (int d = 0; d < p->dim; ++d) {
        if (p->n[d] < 4) return "every extent must be >= 4 cells";
        if (!(p->L[d] > 0.0)) return "domain lengths must be > 0";
        for (int q = 0; q < 2; ++q)
            if (p->bc[d][q] < SIM_BC_PERIODIC || p->bc[d][q] > SIM_BC_WALL_T) return "unknown boundary kind";
        if ((p->bc[d][0] == SIM_BC_PERIODIC) != (p->bc[d][1] == SIM_BC_PERIODIC))
            return "a periodic side needs a periodic partner";
    }
    if (!(p->dt > 0.0)) return "dt must be > 0";
    if (!(p->Re > 0.0) || !(p->Pr > 0.0)) return "Re and Pr must be > 0";
    if (!p->incompressible) {
        if (!(p->Z_st > 0.0 && p->Z_st < 1.0)) return "Z_st must lie in (0, 1)";
        if (!(p->density_ratio > 1.0)) return "density_ratio must be > 1";
        if (!(p->eps_reg > 0.0)) return "eps_reg must be > 0";
        if (!(p->tol_reg > 0.0 && p->tol_reg < 0.5)) return "tol_reg must lie in (0, 0.5)";
        if (!(p->Le_F > 0.0 && p->Le_O > 0.0)) return "Lewis numbers must be > 0";
        if (!(p->gamma > 1.0)) return "gamma must be > 1";
    }
    if (!(p->poisson_rtol > 0.0 && p->poisson_rtol < 1.0)) return "poisson_rtol must lie in (0, 1)";
    if (p->poisson_max_iter < 1) return "poisson_max_iter must be >= 1";
    if (p->mg_sweeps < 0 || p->mg_sweeps > 2) return "mg_sweeps must be 0 (default), 1 or 2";
    if (p->mg_tail_cells < 0) return "mg_tail_cells must be >= 0";
    if (p->transport != 0 && p->transport != 1) return "transport must be 0 (power law) or 1 (Sutherland)";
    if (p->transport == 1 && !(p->sutherland_C >= 0.0)) return "sutherland_C must be >= 0";
    if (p->stage_tile_x != 0 && (p->stage_tile_x < 8 || p->stage_tile_x > 256 ||
                                 (p->stage_tile_x & (p->stage_tile_x - 1)) != 0))
        return "stage_tile_x must be 0 or a power of two from 8 to 256";
    if (p->precision != SIM_FP64 && p->precision != SIM_MIXED) return "precision must be SIM_FP64 or SIM_MIXED";
    if (p->closed_system < 0 || p->closed_system > 2)
        return "closed_system must be 0 (open), 1 (enclosed) or 2 (semi-enclosed)";
    if (p->closed_system == 1) {
        for (int d = 0; d < p->dim; ++d)
            for (int q = 0; q < 2; ++q)
                if (p->bc[d][q] == SIM_BC_INFLOW || p->bc[d][q] == SIM_BC_OUTFLOW)
                    return "an enclosed system cannot have inflow or outflow sides";
    }
    if (p->closed_system == 2) {
        for (int d = 0; d < p->dim; ++d)
            for (int q = 0; q < 2; ++q)
                if (p->bc[d][q] == SIM_BC_OUTFLOW)
                    return "a semi-enclosed system has no outflow sides (its outflow would close the mass balance)";
    }
    return nullptr;
}

// Walk the workspace layout; with s != nullptr assign the pointers.
size_t layout(const sim_params_t* p, sim_t* s, char* base) {
    const Geom g = make_geom(p);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* ptr = base ? base + off : nullptr;
        off += a256(bytes);
        return ptr;
    };
    const size_t fpad = sizeof(double) * (size_t)g.npad;
    const size_t fcmp = sizeof(double) * (size_t)g.ncell;
    long long maxface = 0;
    for (int d = 0; d < g.dim; ++d) {
        long long m = g.ncell / g.n[d] * (g.n[d] + 1);
        if (m > maxface) maxface = m;
    }
    long long maxslab = 0;
    for (int d = 0; d < 3; ++d) {
        const int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
        const long long m = (long long)g.p[a] * g.p[b];
        if (m > maxslab) maxslab = m;
    }
    const int D = g.dim;
    sim_t tmp;
    sim_t* t = s ? s : &tmp;
    auto F = [&](double** dst) { *dst = (double*)take(fpad); };
    // the restart state first, in the order and with the padding of the
    // restart blob (state_segments), so that the blob's body is one
    // contiguous image of the workspace: the arrays final once the
    // corrector's state relation has run, then those the step's end writes
    F(&t->Z); F(&t->H); F(&t->T); F(&t->kap);
    for (int r = 0; r < 3; ++r) F(&t->rho[r]);
    for (int k = 0; k < 2; ++k) {
        for (int d = 0; d < D; ++d) F(&t->R[k][d]);
        F(&t->R[k][3]);
        F(&t->R[k][4]);
    }
    for (int d = 0; d < D; ++d) F(&t->v[d]);
    for (int d = 0; d < D; ++d) F(&t->F[d]);
    {
        double* q = (double*)take(fcmp);
        if (s) s->P = q;
        q = (double*)take(sizeof(double) * SC_NSCAL);
        if (s) s->sc = q;
        int* st = (int*)take(sizeof(int) * 8);
        if (s) s->status = st;
    }
    {
        double* q = (double*)take(fcmp);
        if (s) s->Pm1 = q;
        q = (double*)take(fcmp);
        if (s) s->Pd = q;
    }
    for (int d = 0; d < D; ++d) F(&t->vs[d]);
    F(&t->Zs); F(&t->Hs);
    for (int d = 0; d < D; ++d) F(&t->mom[d]);
    for (int d = 0; d < D; ++d) F(&t->vib[d]);
    F(&t->Sm);
    F(&t->U);
    {
        // mixed path: the stage stencil's float-float input images
        float2* im = nullptr;
        if (p->precision == SIM_MIXED) im = (float2*)take(sizeof(float2) * 6 * (size_t)g.npad);
        if (s) s->ffs = im;
    }
    {
        double* q = (double*)take(fcmp);
        if (s) s->Pstar = q;
        q = (double*)take(sizeof(double) * (size_t)(DG_N * kDiagBlocks + DG_N));
        if (s) s->diag = q;
        q = (double*)take(fcmp);
        if (s) s->b = q;
        q = (double*)take(sizeof(double) * (size_t)(maxface > g.ncell ? maxface : g.ncell));
        if (s) s->io = q;
        q = (double*)take(sizeof(double) * kMaxPartials);
        if (s) s->part = q;
        q = (double*)take(sizeof(double) * kMaxPartials);
        if (s) s->part2 = q;
        q = (double*)take(sizeof(double) * 2 * kMaxPartials);
        if (s) s->ode_part = q;
        q = (double*)take(sizeof(double) * kMaxProfile);
        if (s) s->profile = q;
        uint8_t* c = (uint8_t*)take((size_t)g.npad);
        if (s) s->chi = c;
        for (int d = 0; d < 3; ++d)
            for (int q2 = 0; q2 < 2; ++q2) {
                uint8_t* k = (uint8_t*)take((size_t)maxslab);
                if (s) s->kind[d][q2] = k;
            }
    }
    const char* err = nullptr;
    int periodic[3] = {g.periodic[0], g.periodic[1], g.periodic[2]};
    const size_t pb = poisson_plan_bytes(g.dim, g.n, periodic, p->precision == SIM_MIXED, p->mg_tail_cells, nullptr, nullptr, &err);
    if (pb == 0) return 0;
    off += a256(pb);
    return off;
}

char* poisson_ws(const sim_params_t* p, char* base) {
    // the Poisson plan sits at the end of the layout
    const Geom g = make_geom(p);
    const char* err = nullptr;
    int periodic[3] = {g.periodic[0], g.periodic[1], g.periodic[2]};
    const size_t pb = a256(poisson_plan_bytes(g.dim, g.n, periodic, p->precision == SIM_MIXED, p->mg_tail_cells,
                                              nullptr, nullptr, &err));
    return base + layout(p, nullptr, nullptr) - pb;
}

// --------------------------- launch sequences -------------------------------
void ghost(sim_t* s, std::initializer_list<std::pair<double*, int>> fields, cudaStream_t st, int* L) {
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (auto& f : fields) {
        job.f[job.nf] = f.first;
        job.what[job.nf] = f.second;
        ++job.nf;
    }
    launch_ghost(s->g, s->bnd, s->ph, job, st, L);
}

GhostJob job_of(sim_t* s, std::initializer_list<std::pair<double*, int>> fields) {
    (void)s;
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (auto& f : fields) {
        job.f[job.nf] = f.first;
        job.what[job.nf] = f.second;
        ++job.nf;
    }
    return job;
}

GhostJob job_v(sim_t* s, double* const* v) {
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (int d = 0; d < s->g.dim; ++d) {
        job.f[d] = v[d];
        job.what[d] = GW_V0 + d;
    }
    job.nf = s->g.dim;
    return job;
}

void ghost_v(sim_t* s, double* const* v, cudaStream_t st, int* L) {
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (int d = 0; d < s->g.dim; ++d) {
        job.f[d] = v[d];
        job.what[d] = GW_V0 + d;
    }
    job.nf = s->g.dim;
    launch_ghost(s->g, s->bnd, s->ph, job, st, L);
}

cudaError_t enqueue_init(sim_t* s, cudaStream_t st) {
    int L = 0;
    const Geom& g = s->g;
    double* rho0 = s->rho[s->rho_base];
    ghost_v(s, s->v, st, &L);
    ghost(s, {{s->Z, GW_Z}, {s->H, GW_H}}, st, &L);
    Phys ph0 = s->ph;
    ph0.closed = 0;                                      // p0^0 = 1
    launch_state(g, ph0, s->Z, s->H, s->T, rho0, s->kap, s->sc, SC_P0_N, s->part, s->status, st, &L);
    ghost(s, {{s->kap, GW_KAPPA}}, st, &L);
    launch_sum(g, rho0, s->part, st, &L);
    launch_store_sum(s->part, reduce_grid(g), g.dV, s->sc + SC_MASS, st, &L);
    launch_momentum(g, rho0, s->v, s->mom, st, &L);
    FluxArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    for (int d = 0; d < g.dim; ++d) {
        fa.mom[d] = s->mom[d];
        fa.F[d] = s->F[d];
    }
    fa.sc = s->sc;
    fa.p0_slot = SC_P0_N;
    fa.part = s->part;
    fa.correct = 0;
    launch_flux_rhs(g, s->ph, s->bnd, fa, st, &L);
    cudaError_t e = cudaMemsetAsync(s->P, 0, sizeof(double) * (size_t)g.ncell, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->Pm1, 0, sizeof(double) * (size_t)g.ncell, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->Pd, 0, sizeof(double) * (size_t)g.ncell, st);
    if (e != cudaSuccess) return e;
    double ones[3] = {1.0, 1.0, 1.0};
    e = cudaMemcpyAsync(s->sc + SC_P0_NM1, ones, sizeof(double) * 2, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s->sc + SC_G_N, 0, sizeof(double) * 2, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s->status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Capture a solve's prologue and its CG loop as a conditional while node on
// st (being captured); the loop body is captured on side into the node's body
// graph.  body_launch: kernels per iteration.
cudaError_t capture_while_solve(PoissonPlan* pl, const double* b, double* x, cudaStream_t st, cudaStream_t side,
                                int* body_launch, int mean_ready) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph_h;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph_h, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, graph_h, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    e = poisson_enqueue_prologue(pl, b, x, st, (unsigned long long)h, mean_ready);
    if (e != cudaSuccess) return e;
    // the first iterations ahead of the loop (no per-iteration loop cost); an
    // iteration after convergence changes nothing (its update kernels test the
    // done flag) and the loop then does not run
    const int prefix = poisson_prefix_iters(pl);
    for (int u = 0; u < prefix && e == cudaSuccess; ++u) e = poisson_enqueue_body(pl, x, st, (unsigned long long)h);
    if (e != cudaSuccess) return e;
    e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph_h, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph_h, dv.data(), nullptr, dv.size(), &np);
    if (e != cudaSuccess) return e;
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(side, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    const int before = pl->launches;
    e = poisson_enqueue_body(pl, x, side, (unsigned long long)h);
    cudaGraph_t body_out = bodyg;
    cudaError_t e2 = cudaStreamEndCapture(side, &body_out);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    *body_launch = pl->launches - before;
    return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// One solve as its own graph (prologue, while node, epilogue), captured once
// on the simulation's capture stream: 0 and 1 the step's predictor and
// corrector solves (b -> P), 2 the adjoint's transposed solve.
sim_status launch_solve_graph(sim_t* s, int which, cudaStream_t st) {
    if (!s->solve_valid[which]) {
        PoissonPlan* pl = &s->pp;
        const double* b = which == 2 ? s->adj.LP : s->b;
        double* x = which == 2 ? s->adj.Lb : s->P;
        double* rep = which == 2 ? s->adj.rep : s->sc + (which == 0 ? SC_ITERS_PRED : SC_ITERS_CORR);
        CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed));
        int body = 0;
        pl->launches = 0;
        cudaError_t e = capture_while_solve(pl, b, x, s->cap, s->side, &body, which != 2);
        // P keeps the rounding-level mean the solve leaves (only its differences
        // act; sim_get removes it); the adjoint's transposed solve is zero-mean
        if (e == cudaSuccess) e = poisson_enqueue_epilogue(pl, x, s->cap, rep, s->status, ST_NOCONV, which == 2);
        s->solve_body[which] = body;
        s->solve_fixed[which] = pl->launches - body;
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s->cap, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(s, SIM_ECUDA, "solve graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&s->solve_exec[which], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(s, SIM_ECUDA, "solve graph instantiate: %s", cudaGetErrorString(e));
        s->solve_valid[which] = true;
    }
    CK(cudaGraphLaunch(s->solve_exec[which], st));
    return SIM_OK;
}

void drop_solve_graphs(sim_t* s) {
    for (int k = 0; k < 3; ++k)
        if (s->solve_valid[k]) {
            cudaGraphExecDestroy(s->solve_exec[k]);
            s->solve_valid[k] = false;
        }
}

// Pressure solve of one stage; graph mode adds a conditional while node whose
// condition the prologue and every iteration set on the device.
cudaError_t enqueue_poisson(sim_t* s, cudaStream_t st, bool graph, int iter_slot, int* L, int* body_launch) {
    PoissonPlan* pl = &s->pp;
    pl->launches = 0;
    cudaError_t e;
    if (!graph && s->solve_graphs) {
        const sim_status ss = launch_solve_graph(s, iter_slot == SC_ITERS_PRED ? 0 : 1, st);
        return ss == SIM_OK ? cudaGetLastError() : cudaErrorUnknown;
    }
    if (pl->persist) {
        // the whole solve in one cooperative launch (graph and eager alike)
        *body_launch = 0;
        e = poisson_enqueue_persistent(pl, s->b, s->P, st, 1);
        if (e != cudaSuccess) return e;
    } else if (!graph) {
        e = poisson_enqueue_prologue(pl, s->b, s->P, st, 0ULL, 1);
        if (e != cudaSuccess) return e;
        int done = 0;
        for (int guard = 0; guard <= pl->max_iter + 1; ++guard) {
            e = cudaMemcpyAsync(&done, pl->ictl + PI_DONE, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            if (done) break;
            const int before = pl->launches;
            e = poisson_enqueue_body(pl, s->P, st, 0ULL);
            if (e != cudaSuccess) return e;
            *body_launch = pl->launches - before;
        }
    } else {
        e = capture_while_solve(pl, s->b, s->P, st, s->side, body_launch, 1);
        if (e != cudaSuccess) return e;
    }
    // iterations / residual into the step's scalar slots and non-convergence
    // into the status word; P keeps the rounding-level mean the solve leaves
    // (every correction is zero-mean; only P's differences act), sim_get
    // removes it
    e = poisson_enqueue_epilogue(pl, s->P, st, s->sc + iter_slot, s->status, ST_NOCONV, 0);
    if (e != cudaSuccess) return e;
    // in graph mode the body is counted per executed iteration at query time
    *L += graph ? pl->launches - *body_launch : pl->launches;
    return cudaGetLastError();
}

struct Roles {
    double *rho_n, *rho_prev, *rho_new;
    double* Rn[5];
    double* Rp[5];
};

Roles roles(sim_t* s, long long n) {
    Roles r;
    const int b = s->rho_base;
    r.rho_n = s->rho[b];
    r.rho_new = s->rho[(b + 1) % 3];
    r.rho_prev = s->rho[(b + 2) % 3];
    for (int k = 0; k < 5; ++k) {
        r.Rn[k] = s->R[n & 1][k];
        r.Rp[k] = s->R[(n + 1) & 1][k];
    }
    return r;
}

ResidArgs resid_common(sim_t* s) {
    ResidArgs a;
    std::memset(&a, 0, sizeof(a));
    a.chi = s->chi;
    for (int d = 0; d < s->g.dim; ++d) a.vib[d] = s->vib[d];
    a.Z_ib = s->Z_ib;
    a.H_ib = s->H_ib;
    a.inv_Da = s->ibm_active ? 1.0 / s->Da : 0.0;
    a.ibm = s->ibm_active;
    a.sc = s->sc;
    a.dt = s->prm.dt;
    return a;
}

// The mixed stage stencil reads float-float images of its inputs (one split
// per value instead of one per use); LOWMACH_FF_IMAGES=0 splits on load (the
// same bits: the stencil converts each value as it loads it).
bool use_ff_images(const sim_t* s) {
    if (!s->ffs) return false;
    const char* e = std::getenv("LOWMACH_FF_IMAGES");
    return !(e && e[0] == '0');
}

// Warm-started pressure solves (LOWMACH_EXTRAP=1; off by default): the
// predictor's solve starts from the linear extrapolation 2 P^n - P^(n-1) of
// the last two steps' pressures, the corrector's from P* + (P^n - P*^n), the
// predictor's pressure shifted by the last step's predictor-corrector
// difference, once two (one) steps of history exist since the set-up or the
// last state load (the restart blob does not carry it: a reloaded run takes
// plain guesses for two steps, and matches an uninterrupted one to the
// solvers' tolerance, not bitwise).  Both are initial guesses
// only: every solve still runs to its tolerance.  Measured on the 256x512
// slot burner: 12.95 instead of 14.10 CG iterations per step over 300 steps
// (0.859 against 0.899 ms), but 16.1 instead of 15.55 over the first 25
// (the start-up transient defeats the extrapolation); on the 192^3 sphere
// burner 22.0 instead of 22.55 over 25 steps, yet 0.15 ms slower (the extra
// passes over P in the right-hand side and projection kernels).
bool use_extrap() {
    const char* e = std::getenv("LOWMACH_EXTRAP");
    return e && e[0] == '1';
}

// Sections of a step, in order: SEC_PRED (predictor up to the right-hand
// side), SEC_POIS_PRED (its pressure solve), SEC_MID (predictor projection to
// the corrector's right-hand side), SEC_POIS_CORR, SEC_END (corrector
// projection, ghosts, p0 rotation).  A batch runs the solves of same-grid
// members as one batched solve between the other sections.
enum StepSec : int { SEC_PRED = 0, SEC_POIS_PRED = 1, SEC_MID = 2, SEC_POIS_CORR = 3, SEC_END = 4 };

cudaError_t enqueue_step_sections(sim_t* s, long long n, cudaStream_t st, bool graph, int* L, int* body, int first,
                                  int last) {
    auto on = [&](int k) { return k >= first && k <= last; };
    const Geom& g = s->g;
    const int D = g.dim;
    const double dt = s->prm.dt;
    Roles r = roles(s, n);

    // ---------------- predictor ----------------
    ResidArgs a = resid_common(s);
    for (int d = 0; d < D; ++d) {
        a.v[d] = s->v[d];
        a.vb[d] = s->v[d];
        a.F[d] = s->F[d];
        a.mo[d] = s->mom[d];
    }
    a.Z = s->Z;
    a.H = s->H;
    a.rho = r.rho_n;
    a.kap = s->kap;
    a.Zb = s->Z;
    a.Hb = s->H;
    a.rhob = r.rho_n;
    for (int k = 0; k < 5; ++k) {
        a.Rst[k] = r.Rn[k];
        a.Rrd[k] = r.Rp[k];
    }
    a.Zo = s->Zs;
    a.Ho = s->Hs;
    a.mode = (n == 0) ? MODE_PRED_EULER : MODE_PRED_AB2;
    a.p0a = SC_P0_N;
    a.p0b = SC_P0_NM1;
    a.p0c = SC_P0_NM2;
    a.T = s->T;              // T^n
    a.p0r = SC_P0_N;
    if (n == 0) {
        a.wden = 0.0;
    } else if (n == 1) {
        a.w0 = 1.0; a.w1 = -1.0; a.w2 = 0.0; a.wden = dt;
    } else {
        a.w0 = 3.0; a.w1 = -4.0; a.w2 = 1.0; a.wden = 2.0 * dt;
    }
    a.iwden = (a.wden != 0.0) ? 1.0 / a.wden : 0.0;
    // ghost cells of Z*, H*, kappa, v are filled by the kernels that write them
    a.bnd = s->bnd;
    a.gj = job_of(s, {{s->Zs, GW_Z}, {s->Hs, GW_H}});
    a.ffs = use_ff_images(s) ? s->ffs : nullptr;
    if (D == 3) a.gj.nf = 0;   // 3D: separate ghost fills (the 3D kernels run faster without)
    FluxArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    for (int d = 0; d < D; ++d) {
        fa.mom[d] = s->mom[d];
        fa.F[d] = s->F[d];
    }
    fa.rho_new = r.rho_new;
    fa.rho_n = r.rho_n;
    fa.rho_prev = r.rho_prev;
    fa.Sm = s->ibm_active ? s->Sm : nullptr;
    if (n == 0) {
        fa.bdf_c0 = 1.0; fa.bdf_c1 = -1.0; fa.bdf_c2 = 0.0; fa.bdf_den = dt;
    } else {
        fa.bdf_c0 = 3.0; fa.bdf_c1 = -4.0; fa.bdf_c2 = 1.0; fa.bdf_den = 2.0 * dt;
    }
    fa.sc = s->sc;
    fa.p0_slot = SC_P0_STAR;
    fa.part = s->part;
    fa.b = s->b;
    fa.correct = 1;
    const bool extrap = use_extrap();
    fa.P = s->P;
    fa.Pm1 = s->Pm1;
    fa.Pd = s->Pd;
    const long long hn = n - s->hist_from;   // steps of warm-start history
    fa.guess = !extrap ? GUESS_NONE : (hn >= 2) ? GUESS_EXTRAP : (hn == 1) ? GUESS_COPY : GUESS_NONE;
    // k_rhs leaves mean(b) in the plan's scratch word (the solve's prologue
    // then runs no mean pass)
    poisson_meanb_target(&s->pp, &fa.mb_part, &fa.mb_cnt, &fa.mb_out);
    // an open system (p0 = 1) forms its state and face fluxes in one kernel
    const bool fuse = !s->ph.closed;
    if (on(SEC_PRED)) {
        // semi-enclosed: p0* from Eq 2.38 on level n's fields
        if (s->ph.semi)
            launch_p0_ode(g, s->ph, s->Z, s->H, s->kap, s->v, s->ode_part, s->sc,
                          n == 0 ? ODE_PRED_EULER : ODE_PRED_AB2, dt, SC_P0_STAR, st, L);
        if (a.ffs) {
            const double* src[6] = {s->v[0], s->v[1], D == 3 ? s->v[2] : nullptr, s->Z, s->H, s->kap};
            launch_ff_images(g, src, s->ffs, st, L);
        }
        launch_residual(g, s->ph, a, st, L);
        if (D == 3) ghost(s, {{s->Zs, GW_Z}, {s->Hs, GW_H}}, st, L);
        if (fuse) {
            launch_state_flux_rhs(g, s->ph, s->Zs, s->Hs, s->T, r.rho_new, s->kap, s->sc, s->status, s->bnd, D == 2,
                                  fa, st, L);
            if (D == 3) ghost(s, {{s->kap, GW_KAPPA}}, st, L);
        } else {
            launch_state(g, s->ph, s->Zs, s->Hs, s->T, r.rho_new, s->kap, s->sc, SC_P0_STAR, s->part, s->status, st,
                         L, &s->bnd, D == 2);
            if (D == 3) ghost(s, {{s->kap, GW_KAPPA}}, st, L);
            launch_flux_rhs(g, s->ph, s->bnd, fa, st, L);
        }
    }
    cudaError_t e = cudaSuccess;
    if (on(SEC_POIS_PRED)) e = enqueue_poisson(s, st, graph, SC_ITERS_PRED, L, body);
    if (e != cudaSuccess) return e;
    ProjArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    for (int d = 0; d < D; ++d) {
        pa.F[d] = s->F[d];
        pa.mom[d] = s->mom[d];
        pa.v[d] = s->vs[d];
    }
    pa.P = s->P;
    pa.rho = r.rho_new;
    pa.T = s->T;             // T*
    pa.sc = s->sc;
    pa.p0_slot = SC_P0_STAR;
    pa.eA = s->eA;
    pa.eB = s->eB;
    pa.eC = s->eC;
    pa.bnd = s->bnd;
    pa.gj = job_v(s, s->vs);
    if (D == 3) pa.gj.nf = 0;   // 3D: separate ghost fills (measured faster there)
    if (on(SEC_MID)) {
        launch_project(g, s->ph, pa, st, L);
        if (D == 3) ghost_v(s, s->vs, st, L);
        // P* kept for the predictor-corrector difference (per-step checks)
        e = stage_copy(s->P, s->Pstar, g.ncell, st);
        if (e != cudaSuccess) return e;
        // semi-enclosed: p0^{n+1} from Eq 2.38 on the predicted fields
        // (kappa* is overwritten by the corrector's state relation)
        if (s->ph.semi)
            launch_p0_ode(g, s->ph, s->Zs, s->Hs, s->kap, s->vs, s->ode_part, s->sc, ODE_CORR, dt, SC_P0_NEW,
                          st, L);
    }
    if (on(SEC_MID) && s->adj_save) {
        // predictor values read by the reverse pass (overwritten by the corrector)
        const size_t fp = sizeof(double) * (size_t)g.npad;
        for (int d = 0; d < D && e == cudaSuccess; ++d) {
            e = cudaMemcpyAsync(s->adj.m0[d], s->mom[d], fp, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(s->adj.Fs[d], s->F[d], fp, cudaMemcpyDeviceToDevice, st);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->adj.Ts, s->T, fp, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->adj.rhos, r.rho_new, fp, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->adj.kaps, s->kap, fp, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->adj.Ps, s->P, sizeof(double) * (size_t)g.ncell, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }

    // ---------------- corrector ----------------
    ResidArgs c = resid_common(s);
    for (int d = 0; d < D; ++d) {
        c.v[d] = s->vs[d];
        c.vb[d] = s->v[d];
        c.F[d] = s->F[d];
        c.mo[d] = s->mom[d];
    }
    c.Z = s->Zs;
    c.H = s->Hs;
    c.rho = r.rho_new;      // rho* (overwritten by rho^{n+1} below, after this kernel)
    c.kap = s->kap;         // kappa*
    c.Zb = s->Z;
    c.Hb = s->H;
    c.rhob = r.rho_n;
    for (int k = 0; k < 5; ++k) c.Rrd[k] = r.Rn[k];
    c.Zo = s->Z;
    c.Ho = s->H;
    c.mode = MODE_CORR;
    c.p0a = SC_P0_STAR;
    c.p0b = SC_P0_N;
    c.p0c = SC_P0_NM1;
    c.T = s->T;              // T*
    c.p0r = SC_P0_STAR;
    if (n == 0) {
        c.w0 = 1.0; c.w1 = -1.0; c.w2 = 0.0; c.wden = dt;
    } else {
        c.w0 = 3.0; c.w1 = -4.0; c.w2 = 1.0; c.wden = 2.0 * dt;
    }
    c.iwden = 1.0 / c.wden;
    c.bnd = s->bnd;
    c.gj = job_of(s, {{s->Z, GW_Z}, {s->H, GW_H}});
    c.ffs = a.ffs;
    fa.guess = (extrap && hn >= 1) ? GUESS_SHIFT : GUESS_NONE;
    if (D == 3) c.gj.nf = 0;
    fa.p0_slot = SC_P0_NEW;
    if (on(SEC_MID)) {
        if (c.ffs) {
            const double* src[6] = {s->vs[0], s->vs[1], D == 3 ? s->vs[2] : nullptr, s->Zs, s->Hs, s->kap};
            launch_ff_images(g, src, s->ffs, st, L);
        }
        launch_residual(g, s->ph, c, st, L);
        if (D == 3) ghost(s, {{s->Z, GW_Z}, {s->H, GW_H}}, st, L);
        if (fuse) {
            launch_state_flux_rhs(g, s->ph, s->Z, s->H, s->T, r.rho_new, s->kap, s->sc, s->status, s->bnd, D == 2, fa,
                                  st, L);
            if (D == 3) ghost(s, {{s->kap, GW_KAPPA}}, st, L);
        } else {
            launch_state(g, s->ph, s->Z, s->H, s->T, r.rho_new, s->kap, s->sc, SC_P0_NEW, s->part, s->status, st, L,
                         &s->bnd, D == 2);
            if (D == 3) ghost(s, {{s->kap, GW_KAPPA}}, st, L);
            launch_flux_rhs(g, s->ph, s->bnd, fa, st, L);
        }
        // Z, H, T, kappa, rho and the stored residuals -- the early part of the
        // restart blob -- are final from here on (sim_step_save copies them
        // while the corrector's solve runs)
        if (first == SEC_PRED && last == SEC_END && s->ev_early) {
            const cudaError_t er = cudaEventRecordWithFlags(s->ev_early, st,
                                                            graph ? cudaEventRecordExternal : cudaEventRecordDefault);
            if (er != cudaSuccess) return er;
        }
    }
    if (on(SEC_POIS_CORR)) e = enqueue_poisson(s, st, graph, SC_ITERS_CORR, L, body);
    if (e != cudaSuccess) return e;
    for (int d = 0; d < D; ++d) pa.v[d] = s->v[d];
    pa.p0_slot = SC_P0_NEW;  // T^{n+1}, p0^{n+1}
    pa.gj = job_v(s, s->v);
    if (D == 3) pa.gj.nf = 0;
    if (extrap) {         // the corrector's projection keeps P - P* for the next step's guess
        pa.Pd = s->Pd;
        pa.Pstar = s->Pstar;
    }
    if (on(SEC_END)) {
        pa.rot = s->sc;   // the projection's block 0 rotates the p0 history at its end
        launch_project(g, s->ph, pa, st, L);
        if (D == 3) ghost_v(s, s->v, st, L);
    }
    return cudaGetLastError();
}

// Enqueue step number n (predictor + corrector).  graph: being captured on st.
cudaError_t enqueue_step(sim_t* s, long long n, cudaStream_t st, bool graph, int* L, int* body) {
    return enqueue_step_sections(s, n, st, graph, L, body, SEC_PRED, SEC_END);
}

void after_step(sim_t* s) {
    s->rho_base = (s->rho_base + 1) % 3;
    s->nstep += 1;
    s->t += s->prm.dt;
}

sim_status capture_phase(sim_t* s, int phase) {
    int L = 0, body = 0;
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = enqueue_step(s, s->nstep, s->cap, true, &L, &body);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(s, SIM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return fail(s, SIM_ECUDA, "end capture: %s", cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&s->gexec[phase], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(s, SIM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    s->gvalid[phase] = true;
    s->launches_fixed_graph[phase] = L;
    s->body_launches = body;
    return SIM_OK;
}

sim_status check_device_status(sim_t* s) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (st & ST_NAN) return fail(s, SIM_ENAN, "non-finite or non-positive temperature in the state");
    if (st & ST_NOCONV) return fail(s, SIM_ENOCONV, "a pressure solve did not reach poisson_rtol in %d iterations",
                                    s->prm.poisson_max_iter);
    return SIM_OK;
}

}  // namespace

// adjoint helpers (defined with the adjoint entry points below)
namespace {
ResidArgs adj_resid_args(sim_t* s, double* const* v, const double* Z, const double* H, const double* kap,
                         double* const* F, const double* T, const double* rho);
AdjIn adj_in(sim_t* s, double* const* lv, double* lZ, double* lH, double* lrho);
}  // namespace

// ============================== C ABI ========================================
extern "C" {

sim_status sim_workspace_size(const sim_params_t* prm, size_t* bytes) {
    if (!bytes) return SIM_EINVAL;
    if (validate(prm)) return SIM_EINVAL;
    const size_t b = layout(prm, nullptr, nullptr);
    if (b == 0) return SIM_EINVAL;
    *bytes = b;
    return SIM_OK;
}

namespace {
std::vector<std::pair<void*, size_t>> state_segments(sim_t* s);
char* state_image(const std::vector<std::pair<void*, size_t>>& seg, size_t* bytes);
}  // namespace

sim_status sim_create(const sim_params_t* prm, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                      sim_t** out) {
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    const char* bad = validate(prm);
    if (bad) return SIM_EINVAL;
    const size_t need = layout(prm, nullptr, nullptr);
    if (need == 0) return SIM_EINVAL;
    if (!d_workspace || workspace_bytes < need) return SIM_ENOMEM;
    if (((uintptr_t)d_workspace & 255) != 0) return SIM_EINVAL;
    sim_t* s = new sim_t();   // value-initialised: every plain member starts at zero
    s->prm = *prm;
    s->g = make_geom(prm);
    s->ph = make_phys(prm);
    s->stream = (cudaStream_t)cuda_stream;
    {
        // LOWMACH_NO_GRAPH=1 keeps every step on the host-driven launch path
        const char* ng = std::getenv("LOWMACH_NO_GRAPH");
        s->use_graph = !(ng && ng[0] == '1');
    }
    layout(prm, s, (char*)d_workspace);
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 2; ++q) {
            s->bnd.kind[d][q] = s->kind[d][q];
            s->bnd.bc[d][q] = (d < prm->dim) ? prm->bc[d][q] : SIM_BC_PERIODIC;
        }
    // Eq 3.28 on the first three cell centres of a side (uniform spacing)
    {
        const double h = 1.0;
        const double x0 = -0.5 * h, x1 = 0.5 * h, x2 = 1.5 * h, x3 = 2.5 * h;
        s->eA = (x2 - x0) * (x3 - x0) / ((x2 - x1) * (x3 - x1));
        s->eB = (x1 - x0) * (x3 - x0) / ((x1 - x2) * (x3 - x2));
        s->eC = (x1 - x0) * (x2 - x0) / ((x1 - x3) * (x2 - x3));
    }
    const char* err = nullptr;
    int periodic[3] = {s->g.periodic[0], s->g.periodic[1], s->g.periodic[2]};
    char* pws = poisson_ws(prm, (char*)d_workspace);
    const int* nn = s->g.n;
    if (!poisson_plan_init(&s->pp, prm->dim, nn, s->g.h, periodic, prm->precision == SIM_MIXED, prm->mg_sweeps,
                           prm->mg_tail_cells, prm->poisson_rtol,
                           prm->poisson_max_iter, pws,
                           (size_t)((char*)d_workspace + need - pws), &s->minv, &err)) {
        delete s;
        return SIM_EINVAL;
    }
    sim_status st = SIM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->save_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_early, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        // release whatever was created before the failure
        if (s->cap) cudaStreamDestroy(s->cap);
        if (s->side) cudaStreamDestroy(s->side);
        if (s->save_stream) cudaStreamDestroy(s->save_stream);
        if (s->ev_early) cudaEventDestroy(s->ev_early);
        delete s;
        return SIM_ECUDA;
    }
    if (!poisson_upload_coarse(&s->pp, s->minv, s->stream, &err)) {
        sim_destroy(s);
        return SIM_ECUDA;
    }
    // no body yet: boundary kinds from the sides alone
    int bc[3][2];
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 2; ++q) bc[d][q] = s->bnd.bc[d][q];
    {
        // the restart-state arrays and the padding between them (a blob's
        // body is their contiguous image, padding included)
        size_t nimg = 0;
        char* img = state_image(state_segments(s), &nimg);
        e = img ? cudaMemsetAsync(img, 0, nimg, s->stream) : cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->sc, 0, sizeof(double) * SC_NSCAL, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->status, 0, sizeof(int) * 8, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->chi, 0, (size_t)s->g.npad, s->stream);
    if (e == cudaSuccess) {
        launch_bkinds(s->g, bc, nullptr, s->kind, s->part, s->sc, s->stream);
        e = cudaStreamSynchronize(s->stream);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        sim_destroy(s);
        return SIM_ECUDA;
    }
    s->need_init = true;
    *out = s;
    return st;
}

sim_status sim_set_ibm_geometry(sim_t* s, const sim_ibm_t* geo) {
    if (!s) return SIM_EINVAL;
    int bc[3][2];
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 2; ++q) bc[d][q] = s->bnd.bc[d][q];
    for (int k = 0; k < 6; ++k)
        if (s->gvalid[k]) {
            cudaGraphExecDestroy(s->gexec[k]);
            s->gvalid[k] = false;
        }
    if (!geo || geo->kind == SIM_IBM_NONE) {
        s->ibm_active = 0;
        CK(cudaMemsetAsync(s->chi, 0, (size_t)s->g.npad, s->stream));
        launch_bkinds(s->g, bc, nullptr, s->kind, s->part, s->sc, s->stream);
        CK(cudaStreamSynchronize(s->stream));
        CK(cudaGetLastError());
        return SIM_OK;
    }
    if (geo->kind != SIM_IBM_SLOT && geo->kind != SIM_IBM_SPHERE && geo->kind != SIM_IBM_MARKERS &&
        geo->kind != SIM_IBM_COUETTE)
        return fail(s, SIM_EINVAL, "unknown body kind %d", geo->kind);
    if (geo->kind == SIM_IBM_COUETTE && !(geo->radius > 0.0 && geo->half[0] > geo->radius))
        return fail(s, SIM_EINVAL, "coaxial cylinders need 0 < radius < half[0]");
    if (s->ph.semi)
        return fail(s, SIM_EINVAL, "a semi-enclosed system takes no immersed body (Eq 2.38 has no penalisation "
                                   "or mass-source terms)");
    const int mk_stride = 2 * s->g.dim + 2;
    if (geo->kind == SIM_IBM_MARKERS &&
        (geo->n_markers < 1 || !geo->markers || (long long)geo->n_markers * mk_stride > s->g.npad))
        return fail(s, SIM_EINVAL, "markers: need 1 to %lld rows of %d doubles", s->g.npad / mk_stride, mk_stride);
    if (!(geo->Da_ib > 0.0)) return fail(s, SIM_EINVAL, "Da_ib must be > 0");
    if (geo->n_profile < 0 || geo->n_profile > kMaxProfile || (geo->n_profile > 0 && !geo->profile) ||
        geo->n_profile == 1)
        return fail(s, SIM_EINVAL, "profile must have 0 or 2..%d samples", kMaxProfile);
    if (s->prm.dt >= s->prm.Re * geo->Da_ib)
        return fail(s, SIM_EUNSTABLE, "dt = %g >= Re Da_ib = %g (explicit penalisation limit)", s->prm.dt,
                    s->prm.Re * geo->Da_ib);
    IbmDev b;
    std::memset(&b, 0, sizeof(b));
    b.kind = geo->kind;
    for (int d = 0; d < 3; ++d) {
        b.c[d] = geo->center[d];
        b.half[d] = geo->half[d];
    }
    b.radius = geo->radius;
    b.s = std::sqrt(geo->Da_ib);
    b.rho_b = geo->rho_b;
    b.U_b = geo->U_b;
    b.n_profile = geo->n_profile;
    if (geo->n_profile > 0) {
        CK(cudaMemcpyAsync(s->profile, geo->profile, sizeof(double) * geo->n_profile, cudaMemcpyHostToDevice,
                           s->stream));
        b.profile = s->profile;
    }
    if (geo->kind == SIM_IBM_MARKERS) {
        // set-up scratch: the marker rows in the first momentum array, the
        // nearest-marker index per padded cell and the per-marker counts in
        // the predictor velocity arrays (all rewritten by every step)
        const int D = s->g.dim;
        b.n_mk = geo->n_markers;
        for (int d = 0; d < 3; ++d) {
            b.bb_lo[d] = 0.0;
            b.bb_hi[d] = 0.0;
        }
        for (int d = 0; d < D; ++d) {
            double lo = geo->markers[d], hi = geo->markers[d];
            for (int m = 1; m < geo->n_markers; ++m) {
                const double v = geo->markers[(size_t)m * mk_stride + d];
                lo = v < lo ? v : lo;
                hi = v > hi ? v : hi;
            }
            b.bb_lo[d] = lo - 2.0 * b.s;
            b.bb_hi[d] = hi + 2.0 * b.s;
        }
        CK(cudaMemcpyAsync(s->mom[0], geo->markers, sizeof(double) * (size_t)geo->n_markers * mk_stride,
                           cudaMemcpyHostToDevice, s->stream));
        b.mk = s->mom[0];
        int* near = reinterpret_cast<int*>(s->vs[0]);
        int* counts = reinterpret_cast<int*>(s->vs[1]);
        CK(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)geo->n_markers, s->stream));
        launch_marker_cells(s->g, b, s->chi, s->vib, s->U, s->Sm, near, counts, s->stream);
        CK(cudaGetLastError());
        std::vector<int> hc((size_t)geo->n_markers);
        CK(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (int m = 0; m < geo->n_markers; ++m)
            if (hc[(size_t)m] == 0) {
                s->ibm_active = 0;
                CK(cudaMemsetAsync(s->chi, 0, (size_t)s->g.npad, s->stream));
                launch_bkinds(s->g, bc, nullptr, s->kind, s->part, s->sc, s->stream);
                CK(cudaStreamSynchronize(s->stream));
                return fail(s, SIM_EINVAL, "marker %d has no masked cell matched with it (markers denser than "
                            "the cells)", m);
            }
        launch_marker_source(s->g, b, s->chi, near, counts, s->Sm, s->stream);
        b.mk = nullptr;   // the scratch is reused by the steps
    } else {
        launch_ibm(s->g, b, s->chi, s->vib, s->U, s->Sm, s->stream);
    }
    s->ibm = b;
    launch_bkinds(s->g, bc, s->chi, s->kind, s->part, s->sc, s->stream);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    s->ibm_active = 1;
    s->Z_ib = geo->Z_ib;
    s->H_ib = geo->H_ib;
    s->Da = geo->Da_ib;
    return SIM_OK;
}

sim_status sim_fields(sim_t* s, int id, void* buf, int dir, int on_device) {
    if (!s || !buf) return SIM_EINVAL;
    const Geom& g = s->g;
    const int D = g.dim;
    cudaStream_t st = s->stream;
    const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind d2h = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t cells = sizeof(double) * (size_t)g.ncell;
    if (dir == SIM_SET) {
        double* dst = nullptr;
        int bit = 0;
        if (id >= SIM_FIELD_U && id <= SIM_FIELD_W) {
            if (id - SIM_FIELD_U >= D) return fail(s, SIM_EINVAL, "no W component in 2D");
            dst = s->v[id - SIM_FIELD_U];
            bit = 1 << id;
        } else if (id == SIM_FIELD_Z) {
            dst = s->Z;
            bit = 1 << 3;
        } else if (id == SIM_FIELD_H) {
            dst = s->H;
            bit = 1 << 4;
        } else {
            return fail(s, SIM_EINVAL, "field %d cannot be set (only U, V, W, Z, H)", id);
        }
        CK(cudaMemcpyAsync(s->io, buf, cells, h2d, st));
        launch_unpack(g, s->io, dst, st);
        CK(cudaGetLastError());
        if (!on_device) CK(cudaStreamSynchronize(st));
        s->fields_set |= bit;
        s->need_init = true;
        return SIM_OK;
    }
    if (dir != SIM_GET) return fail(s, SIM_EINVAL, "dir must be SIM_GET or SIM_SET");
    size_t bytes = cells;
    if (id >= SIM_FIELD_U && id <= SIM_FIELD_W) {
        if (id - SIM_FIELD_U >= D) return fail(s, SIM_EINVAL, "no W component in 2D");
        launch_pack(g, s->v[id - SIM_FIELD_U], s->io, -1, st);
    } else if (id == SIM_FIELD_Z) {
        launch_pack(g, s->Z, s->io, -1, st);
    } else if (id == SIM_FIELD_H) {
        launch_pack(g, s->H, s->io, -1, st);
    } else if (id == SIM_FIELD_T) {
        launch_pack(g, s->T, s->io, -1, st);
    } else if (id == SIM_FIELD_RHO) {
        launch_pack(g, s->rho[s->rho_base], s->io, -1, st);
    } else if (id == SIM_FIELD_KAPPA) {
        launch_pack(g, s->kap, s->io, -1, st);
    } else if (id == SIM_FIELD_P) {
        // the zero-mean P of Eqs 3.17 / 3.24 (the stored P carries the
        // rounding-level mean the solves leave)
        CK(cudaMemcpyAsync(s->io, s->P, cells, cudaMemcpyDeviceToDevice, st));
        CK(poisson_enqueue_remove_mean(&s->pp, (double*)s->io, st));
    } else if (id >= SIM_FIELD_FX && id <= SIM_FIELD_FZ) {
        const int d = id - SIM_FIELD_FX;
        if (d >= D) return fail(s, SIM_EINVAL, "no z faces in 2D");
        launch_pack(g, s->F[d], s->io, d, st);
        bytes = sizeof(double) * (size_t)(g.ncell / g.n[d] * (g.n[d] + 1));
    } else if (id == SIM_FIELD_CHI) {
        launch_u8_to_double(g, s->chi, s->io, st);
    } else if (id == SIM_FIELD_SM) {
        if (s->ibm_active)
            launch_pack(g, s->Sm, s->io, -1, st);
        else
            CK(cudaMemsetAsync(s->io, 0, cells, st));
    } else {
        return fail(s, SIM_EINVAL, "unknown field %d", id);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(buf, s->io, bytes, d2h, st));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return SIM_OK;
}

sim_status sim_step(sim_t* s, int nsteps) {
    if (!s || nsteps < 0) return SIM_EINVAL;
    const int need = (s->g.dim == 3) ? 0x1f : 0x1b;
    if ((s->fields_set & need) != need) return fail(s, SIM_ESTATE, "set U, V, (W,) Z, H before stepping");
    if (s->need_init) {
        // level 0 starts the rotation afresh: the set-up writes rho^0 into the
        // buffer the first step reads as rho^n, whatever a previous run left
        s->nstep = 0;
        s->rho_base = 0;
        s->t = 0.0;
        s->hist_from = 0;
        CK(enqueue_init(s, s->stream));
        s->need_init = false;
        for (int k = 0; k < 6; ++k)
            if (s->gvalid[k]) {
                cudaGraphExecDestroy(s->gexec[k]);
                s->gvalid[k] = false;
            }
    }
    for (int it = 0; it < nsteps; ++it) {
        const long long n = s->nstep;
        // eager until the launch sequence is the steady one (the first two
        // steps; with warm starts, also the first two after a state load)
        if (n < 2 || !s->use_graph || (use_extrap() && n - s->hist_from < 2)) {
            int L = 0, body = 0;
            CK(enqueue_step(s, n, s->stream, false, &L, &body));
            s->launches_last = L;
        } else {
            // the launch sequence depends on n only through the rotating roles
            const int phase = (int)(n % 6);
            if (!s->gvalid[phase]) {
                sim_status st = capture_phase(s, phase);
                if (st != SIM_OK) return st;
            }
            CK(cudaGraphLaunch(s->gexec[phase], s->stream));
            s->launches_last = -(s->launches_fixed_graph[phase] + 1);  // resolved by sim_query
        }
        after_step(s);
    }
    return SIM_OK;
}

sim_status sim_sync(sim_t* s) {
    if (!s) return SIM_EINVAL;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return check_device_status(s);
}

namespace {
// Per-step checks of the last completed step, from the state: rho^{n+1},
// rho^n, rho^{n-1} are the three rotating levels; the step's own rate rule
// (first order on the first step, Eq 3.11 / 3.19 after).
sim_status run_diagnostics(sim_t* s, double* res) {
    const Geom& g = s->g;
    DiagArgs a;
    std::memset(&a, 0, sizeof(a));
    const int b = s->rho_base;
    a.rho_new = s->rho[b];
    a.rho_n = s->rho[(b + 2) % 3];
    a.rho_prev = s->rho[(b + 1) % 3];
    const double dt = s->prm.dt;
    if (s->nstep == 1) {
        a.c0 = 1.0; a.c1 = -1.0; a.c2 = 0.0; a.iden = 1.0 / dt;
    } else {
        a.c0 = 3.0; a.c1 = -4.0; a.c2 = 1.0; a.iden = 1.0 / (2.0 * dt);
    }
    for (int d = 0; d < g.dim; ++d) {
        a.F[d] = s->F[d];
        a.v[d] = s->v[d];
        a.vs[d] = s->vs[d];
    }
    a.Sm = s->ibm_active ? s->Sm : nullptr;
    a.P = s->P;
    a.Ps = s->Pstar;
    a.part = s->diag;
    a.out = s->diag + DG_N * kDiagBlocks;
    CK(launch_diagnostics(g, a, s->stream));
    CK(cudaMemcpyAsync(res, a.out, sizeof(double) * DG_N, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return SIM_OK;
}
}  // namespace

sim_status sim_query(sim_t* s, int what, double* out) {
    if (!s || !out) return SIM_EINVAL;
    CK(cudaStreamSynchronize(s->stream));
    auto dev = [&](int slot, double* v) -> sim_status {
        CK(cudaMemcpy(v, s->sc + slot, sizeof(double), cudaMemcpyDeviceToHost));
        return SIM_OK;
    };
    switch (what) {
        case SIM_Q_TIME: *out = s->t; return SIM_OK;
        case SIM_Q_DT: *out = s->prm.dt; return SIM_OK;
        case SIM_Q_P0: return dev(SC_P0_N, out);
        case SIM_Q_STEPS: *out = (double)s->nstep; return SIM_OK;
        case SIM_Q_ITERS_PRED: return dev(SC_ITERS_PRED, out);
        case SIM_Q_RESID_PRED: return dev(SC_RELRES_PRED, out);
        case SIM_Q_ITERS_CORR: return dev(SC_ITERS_CORR, out);
        case SIM_Q_RESID_CORR: return dev(SC_RELRES_CORR, out);
        case SIM_Q_MASS: return dev(SC_MASS, out);
        case SIM_Q_NCELLS: *out = (double)s->g.ncell; return SIM_OK;
        case SIM_Q_MG_LEVELS: *out = (double)s->pp.nlev; return SIM_OK;
        case SIM_Q_TAIL_NX: *out = (double)s->pp.lev[s->pp.top].n[0]; return SIM_OK;
        case SIM_Q_TAIL_NY: *out = (double)s->pp.lev[s->pp.top].n[1]; return SIM_OK;
        case SIM_Q_TAIL_FDM: *out = (double)s->pp.fdm; return SIM_OK;
        case SIM_Q_TAIL_NZ: *out = (double)(s->g.dim == 3 ? s->pp.lev[s->pp.top].n[2] : 1); return SIM_OK;
        case SIM_Q_KERNEL_LAUNCHES: {
            if (s->launches_last >= 0) {
                *out = (double)s->launches_last;
                return SIM_OK;
            }
            double ip = 0, ic = 0;
            sim_status st = dev(SC_ITERS_PRED, &ip);
            if (st != SIM_OK) return st;
            st = dev(SC_ITERS_CORR, &ic);
            if (st != SIM_OK) return st;
            // the step graph's fixed part holds the iterations captured ahead of
            // each solve's loop; the loops ran the rest
            *out = (double)(-s->launches_last - 1) +
                   (poisson_loop_iters(&s->pp, ip) + poisson_loop_iters(&s->pp, ic)) * s->body_launches;
            return SIM_OK;
        }
        case SIM_Q_DIV_RESID:
        case SIM_Q_DIV_SCALE:
        case SIM_Q_MASS_BALANCE:
        case SIM_Q_PC_DIFF_U:
        case SIM_Q_PC_DIFF_V:
        case SIM_Q_PC_DIFF_W:
        case SIM_Q_PC_DIFF_P: {
            if (s->nstep < 1 || s->need_init) return fail(s, SIM_ESTATE, "per-step checks need a completed step");
            double r[DG_N];
            const sim_status st = run_diagnostics(s, r);
            if (st != SIM_OK) return st;
            const double N = (double)s->g.ncell;
            switch (what) {
                case SIM_Q_DIV_RESID: *out = r[DG_MAXRES]; break;
                case SIM_Q_DIV_SCALE: *out = r[DG_MAXDRHO] + r[DG_MAXSM]; break;
                case SIM_Q_MASS_BALANCE: *out = r[DG_BAL]; break;
                case SIM_Q_PC_DIFF_U: *out = std::sqrt(r[DG_DU]); break;
                case SIM_Q_PC_DIFF_V: *out = std::sqrt(r[DG_DU + 1]); break;
                case SIM_Q_PC_DIFF_W: *out = s->g.dim == 3 ? std::sqrt(r[DG_DU + 2]) : 0.0; break;
                default: {
                    // P is unique up to a constant: the difference's mean is removed
                    const double sd = r[DG_DP] / s->g.dV, m = sd / N;
                    *out = std::sqrt(std::fmax(r[DG_DP2] - m * sd * s->g.dV, 0.0));
                }
            }
            return SIM_OK;
        }
        default: return fail(s, SIM_EINVAL, "unknown query %d", what);
    }
}

sim_status sim_time_kernel(sim_t* s, int kernel, int reps) {
    if (!s || reps < 0) return SIM_EINVAL;
    if (s->need_init || s->nstep < 1) return fail(s, SIM_ESTATE, "time kernels after the first step");
    const Geom& g = s->g;
    const int D = g.dim;
    const long long n = s->nstep;
    Roles r = roles(s, n);
    int L = 0;
    for (int it = 0; it < reps; ++it) {
        switch (kernel) {
            case SIM_K_RESIDUAL: {
                ResidArgs a = resid_common(s);
                for (int d = 0; d < D; ++d) {
                    a.v[d] = s->v[d];
                    a.vb[d] = s->v[d];
                    a.F[d] = s->F[d];
                    a.mo[d] = s->mom[d];
                }
                a.Z = s->Z;
                a.H = s->H;
                a.rho = r.rho_n;
                a.kap = s->kap;
                a.Zb = s->Z;
                a.Hb = s->H;
                a.rhob = r.rho_n;
                for (int k = 0; k < 5; ++k) {
                    a.Rst[k] = r.Rn[k];
                    a.Rrd[k] = r.Rp[k];
                }
                a.Zo = s->Zs;
                a.Ho = s->Hs;
                a.mode = MODE_PRED_AB2;
                a.p0a = SC_P0_N;
                a.p0b = SC_P0_NM1;
                a.p0c = SC_P0_NM2;
                a.T = s->T;
                a.p0r = SC_P0_N;
                a.w0 = 3.0; a.w1 = -4.0; a.w2 = 1.0; a.wden = 2.0 * s->prm.dt;
                a.iwden = 1.0 / a.wden;
                // the stencil variant the step runs (its inputs' images as the
                // last stage left them)
                a.ffs = use_ff_images(s) ? s->ffs : nullptr;
                launch_residual(g, s->ph, a, s->stream, &L);
                break;
            }
            case SIM_K_MG_DOWN: CK(poisson_launch_single(&s->pp, 0, s->stream)); break;
            case SIM_K_CG_MATVEC: CK(poisson_launch_single(&s->pp, 1, s->stream)); break;
            case SIM_K_MG_UP: CK(poisson_launch_single(&s->pp, 2, s->stream)); break;
            case SIM_K_MG_TAIL: CK(poisson_launch_single(&s->pp, 3, s->stream)); break;
            case SIM_K_STATE: {
                // T, kappa of Z*, H* into residual scratch (the next predictor rewrites it)
                Phys ph = s->ph;
                ph.closed = 0;
                launch_state(g, ph, s->Zs, s->Hs, r.Rn[3], r.rho_new, r.Rn[4], s->sc, SC_P0_STAR, s->part,
                             s->status, s->stream, &L);
                break;
            }
            case SIM_K_PROJECT: {
                ProjArgs pa;
                std::memset(&pa, 0, sizeof(pa));
                for (int d = 0; d < D; ++d) {
                    pa.F[d] = r.Rn[d];   // residual scratch stands in for the interface fluxes
                    pa.mom[d] = s->mom[d];
                    pa.v[d] = s->vs[d];
                }
                pa.P = s->pp.q;          // Krylov scratch as the pressure argument
                pa.rho = r.rho_n;
                pa.T = s->T;
                pa.sc = s->sc;
                pa.p0_slot = SC_P0_N;
                pa.eA = s->eA;
                pa.eB = s->eB;
                pa.eC = s->eC;
                launch_project(g, s->ph, pa, s->stream, &L);
                break;
            }
            case SIM_K_RESIDUAL_REV: {
                // reverse stencil sweep and gather of the predictor stage (adds into lambda)
                if (!s->adj_active) return fail(s, SIM_ESTATE, "time the reverse stencil after sim_adjoint_begin");
                AdjWs& A = s->adj;
                AdjR lr;
                for (int k = 0; k < 5; ++k) lr.R[k] = A.LR[k];
                const ResidArgs a = adj_resid_args(s, s->v, s->Z, s->H, s->kap, s->F, s->T, r.rho_n);
                launch_residual_adj(g, s->ph, a, 0.0, lr, adj_in(s, A.Lv, A.LZ, A.LH, nullptr),
                                    A.use_dual ? nullptr : A.cont,
                                    s->stream);
                L += 2;
                break;
            }
            default: return fail(s, SIM_EINVAL, "unknown kernel id %d", kernel);
        }
    }
    CK(cudaGetLastError());
    return SIM_OK;
}

// ----------------------------- restart state ---------------------------------
namespace {
struct StateHeader {
    char magic[8];
    int version, dim, n[3], rho_base;
    long long nstep;
    double t, dt;
    int ibm_active, pad_;
};

// Segments of the restart blob: (device pointer, bytes), in a fixed order.
std::vector<std::pair<void*, size_t>> state_segments(sim_t* s) {
    const Geom& g = s->g;
    const size_t fpad = sizeof(double) * (size_t)g.npad;
    std::vector<std::pair<void*, size_t>> seg;
    // final once the corrector's state relation has run (kEarlySegments(dim))
    seg.push_back({s->Z, fpad});
    seg.push_back({s->H, fpad});
    seg.push_back({s->T, fpad});
    seg.push_back({s->kap, fpad});
    for (int r = 0; r < 3; ++r) seg.push_back({s->rho[r], fpad});
    for (int k = 0; k < 2; ++k) {
        for (int d = 0; d < g.dim; ++d) seg.push_back({s->R[k][d], fpad});
        seg.push_back({s->R[k][3], fpad});
        seg.push_back({s->R[k][4], fpad});
    }
    // written at the step's end
    for (int d = 0; d < g.dim; ++d) seg.push_back({s->v[d], fpad});
    for (int d = 0; d < g.dim; ++d) seg.push_back({s->F[d], fpad});
    seg.push_back({s->P, sizeof(double) * (size_t)g.ncell});
    seg.push_back({s->sc, sizeof(double) * SC_NSCAL});
    seg.push_back({s->status, sizeof(int) * 8});
    return seg;
}

// The blob's body as one contiguous image of the workspace's state arrays
// (layout carves them first, in blob order, with the blob's padding): its
// start and length, or null.
char* state_image(const std::vector<std::pair<void*, size_t>>& seg, size_t* bytes) {
    char* base = (char*)seg[0].first;
    size_t off = 0;
    for (auto& q : seg) {
        if ((char*)q.first != base + off) return nullptr;
        off += a256(q.second);
    }
    *bytes = off;
    return base;
}

void fill_header(const sim_t* s, StateHeader* h) {
    std::memset(h, 0, sizeof(*h));
    std::memcpy(h->magic, "LMSTATE", 8);
    h->version = 2;
    h->dim = s->g.dim;
    for (int d = 0; d < 3; ++d) h->n[d] = s->g.n[d];
    h->rho_base = s->rho_base;
    h->nstep = s->nstep;
    h->t = s->t;
    h->dt = s->prm.dt;
    h->ibm_active = s->ibm_active;
}

size_t state_bytes(sim_t* s) {
    size_t b = a256(sizeof(StateHeader));
    for (auto& q : state_segments(s)) b += a256(q.second);
    return b;
}
}  // namespace

sim_status sim_state_size(const sim_t* cs, size_t* bytes) {
    if (!cs || !bytes) return SIM_EINVAL;
    *bytes = state_bytes(const_cast<sim_t*>(cs));
    return SIM_OK;
}

sim_status sim_state_save(sim_t* s, void* buf, int on_device) {
    if (!s || !buf) return SIM_EINVAL;
    if (s->need_init) return fail(s, SIM_ESTATE, "no state yet: step once after setting the fields");
    StateHeader h;
    fill_header(s, &h);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char* out = (char*)buf;
    if (on_device) CK(cudaMemcpyAsync(out, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream));
    const auto seg = state_segments(s);
    size_t nimg = 0;
    char* img = state_image(seg, &nimg);
    if (img) {
        // one copy of the contiguous state image
        CK(cudaMemcpyAsync(out + a256(sizeof(StateHeader)), img, nimg, k, s->stream));
    } else {
        size_t off = a256(sizeof(StateHeader));
        for (auto& q : seg) {
            CK(cudaMemcpyAsync(out + off, q.first, q.second, k, s->stream));
            off += a256(q.second);
        }
    }
    CK(cudaStreamSynchronize(s->stream));
    if (!on_device) std::memcpy(out, &h, sizeof(h));   // a host blob's header, written by the host
    return SIM_OK;
}

sim_status sim_step_save(sim_t* s, void* buf, int on_device) {
    if (!s || !buf) return SIM_EINVAL;
    const sim_status st = sim_step(s, 1);
    if (st != SIM_OK) return st;
    const auto seg = state_segments(s);
    size_t nimg = 0;
    char* img = state_image(seg, &nimg);
    if (!img) return sim_state_save(s, buf, on_device);
    // the arrays final after the corrector's state relation lead the image
    const int ne = 7 + 2 * (s->g.dim + 2);
    size_t nearly = 0;
    for (int i = 0; i < ne; ++i) nearly += a256(seg[(size_t)i].second);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char* out = (char*)buf + a256(sizeof(StateHeader));
    CK(cudaStreamWaitEvent(s->save_stream, s->ev_early, 0));
    CK(cudaMemcpyAsync(out, img, nearly, k, s->save_stream));
    // From here the early copy may be writing into the caller's buffer: every
    // return, failed or not, first waits for it, so the buffer is free again
    // when the call returns.
    const char* what = nullptr;
    cudaError_t e = cudaMemcpyAsync(out + nearly, img + nearly, nimg - nearly, k, s->stream);
    if (e != cudaSuccess) what = "cudaMemcpyAsync (late part)";
    StateHeader h;
    fill_header(s, &h);
    if (!what && on_device) {
        e = cudaMemcpyAsync(buf, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) what = "cudaMemcpyAsync (header)";
    }
    const cudaError_t e_save = cudaStreamSynchronize(s->save_stream);
    if (!what) {
        e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) what = "cudaStreamSynchronize (step stream)";
    }
    if (!what && e_save != cudaSuccess) {
        e = e_save;
        what = "cudaStreamSynchronize (save stream)";
    }
    if (what) return fail(s, SIM_ECUDA, "sim_step_save: %s: %s", what, cudaGetErrorString(e));
    if (!on_device) std::memcpy(buf, &h, sizeof(h));
    return SIM_OK;
}

sim_status sim_state_load(sim_t* s, const void* buf, int on_device) {
    if (!s || !buf) return SIM_EINVAL;
    StateHeader h;
    if (on_device)
        CK(cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDeviceToHost));
    else
        std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "LMSTATE", 8) != 0 || h.version != 2 || h.dim != s->g.dim || h.dt != s->prm.dt ||
        h.n[0] != s->g.n[0] || h.n[1] != s->g.n[1] || h.n[2] != s->g.n[2] || h.ibm_active != s->ibm_active)
        return fail(s, SIM_EINVAL, "restart blob does not match this simulation");
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const char* in = (const char*)buf;
    const auto seg = state_segments(s);
    size_t nimg = 0;
    char* img = state_image(seg, &nimg);
    if (img) {
        CK(cudaMemcpyAsync(img, in + a256(sizeof(StateHeader)), nimg, k, s->stream));
    } else {
        size_t off = a256(sizeof(StateHeader));
        for (auto& q : seg) {
            CK(cudaMemcpyAsync(q.first, in + off, q.second, k, s->stream));
            off += a256(q.second);
        }
    }
    if (!on_device) CK(cudaStreamSynchronize(s->stream));
    s->rho_base = h.rho_base;
    s->nstep = h.nstep;
    s->hist_from = h.nstep;
    s->t = h.t;
    s->need_init = false;
    s->fields_set = 0x1f;
    return SIM_OK;
}

const char* sim_last_error(const sim_t* s) { return s ? s->err : "null handle"; }

void sim_destroy(sim_t* s) {
    if (!s) return;
    drop_solve_graphs(s);
    for (int k = 0; k < 6; ++k)
        if (s->gvalid[k]) cudaGraphExecDestroy(s->gexec[k]);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->save_stream) cudaStreamDestroy(s->save_stream);
    if (s->ev_early) cudaEventDestroy(s->ev_early);
    delete s;
}

// ----------------------- stand-alone pressure solve --------------------------
sim_status sim_poisson_workspace_size(int dim, const int n[3], const int periodic[3], size_t* bytes) {
    if (!n || !periodic || !bytes || (dim != 2 && dim != 3)) return SIM_EINVAL;
    for (int d = 0; d < dim; ++d)
        if (n[d] < 2) return SIM_EINVAL;
    int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    const char* err = nullptr;
    const size_t b = poisson_plan_bytes(dim, nn, periodic, 0, 0, nullptr, nullptr, &err);
    if (b == 0) return SIM_EINVAL;
    *bytes = b;
    return SIM_OK;
}

sim_status sim_poisson_solve(int dim, const int n[3], const double h[3], const int periodic[3], const double* d_b,
                             double* d_P, double rtol, int max_iter, void* d_workspace, size_t workspace_bytes,
                             void* cuda_stream, int* iters, double* rel_resid) {
    if (!n || !h || !periodic || !d_b || !d_P || !d_workspace || (dim != 2 && dim != 3)) return SIM_EINVAL;
    if (!(rtol > 0.0 && rtol < 1.0) || max_iter < 1) return SIM_EINVAL;
    int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    double hh[3] = {h[0], h[1], dim == 3 ? h[2] : 1.0};
    int per[3] = {periodic[0] != 0, periodic[1] != 0, dim == 3 ? (periodic[2] != 0) : 0};
    for (int d = 0; d < dim; ++d)
        if (nn[d] < 2 || !(hh[d] > 0.0)) return SIM_EINVAL;
    const char* err = nullptr;
    const size_t need = poisson_plan_bytes(dim, nn, per, 0, 0, nullptr, nullptr, &err);
    if (need == 0) return SIM_EINVAL;
    if (workspace_bytes < need) return SIM_ENOMEM;
    PoissonPlan pl;
    std::vector<double> minv;
    if (!poisson_plan_init(&pl, dim, nn, hh, per, 0, 0, 0, rtol, max_iter, d_workspace, workspace_bytes, &minv, &err))
        return SIM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!poisson_upload_coarse(&pl, minv, st, &err)) return SIM_ECUDA;
    cudaError_t e = poisson_solve_host_loop(&pl, d_b, d_P, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SIM_ECUDA;
    double sc[PS_NSCAL];
    int ic[PI_NINT];
    if (cudaMemcpy(sc, pl.scal, sizeof(sc), cudaMemcpyDeviceToHost) != cudaSuccess) return SIM_ECUDA;
    if (cudaMemcpy(ic, pl.ictl, sizeof(ic), cudaMemcpyDeviceToHost) != cudaSuccess) return SIM_ECUDA;
    if (iters) *iters = (int)sc[PS_ITERS];
    if (rel_resid) *rel_resid = sc[PS_RELRES];
    return ic[PI_NOCONV] ? SIM_ENOCONV : SIM_OK;
}

}  // extern "C"

// ------------------------------ discrete adjoint -----------------------------
namespace {

// Adjoint workspace layout: the lambda region first (zeroed by begin), then the
// saved forward values.  Returns the bytes used (a null base only measures).
size_t adj_layout(const sim_t* s, AdjWs* A, char* base) {
    const Geom& g = s->g;
    const int D = g.dim;
    const size_t fpad = sizeof(double) * (size_t)g.npad;
    const size_t fcmp = sizeof(double) * (size_t)g.ncell;
    size_t off = 0;
    auto take = [&](size_t bytes) -> double* {
        double* p = base ? (double*)(base + off) : nullptr;
        off += a256(bytes);
        return p;
    };
    AdjWs tmp;
    AdjWs& a = A ? *A : tmp;
    std::memset(&a, 0, sizeof(a));
    for (int d = 0; d < D; ++d) a.Lv[d] = take(fpad);
    for (int d = 0; d < D; ++d) a.Lvs[d] = take(fpad);
    a.LZ = take(fpad); a.LH = take(fpad); a.LZs = take(fpad); a.LHs = take(fpad);
    a.LT = take(fpad); a.Lkap = take(fpad);
    for (int d = 0; d < D; ++d) a.LF[d] = take(fpad);
    for (int d = 0; d < D; ++d) a.LFt[d] = take(fpad);
    for (int k = 0; k < 5; ++k)
        if (k < D || k >= 3) {
            a.LRh[k] = take(fpad);
            a.LR[k] = take(fpad);
        }
    for (int d = 0; d < D; ++d) a.Lm[d] = take(fpad);
    for (int r = 0; r < 3; ++r) a.Lr[r] = take(fpad);
    for (int d = 0; d < D; ++d) a.Lvib[d] = take(fpad);
    a.LSm = take(fpad);
    a.LP = take(fcmp);
    a.Lb = take(fcmp);
    a.lam_base = base;
    a.lam_bytes = off;
    for (int d = 0; d < D; ++d) a.v0[d] = take(fpad);
    a.Z0 = take(fpad); a.H0 = take(fpad); a.T0 = take(fpad); a.kap0 = take(fpad); a.rho0 = take(fpad);
    for (int d = 0; d < D; ++d) a.F0[d] = take(fpad);
    for (int d = 0; d < D; ++d) a.m0[d] = take(fpad);
    a.Ts = take(fpad); a.kaps = take(fpad); a.rhos = take(fpad);
    a.Ps = take(fcmp);
    for (int d = 0; d < D; ++d) a.Fs[d] = take(fpad);
    a.col = take(sizeof(double) * (size_t)g.n[0]);
    a.grad = take(sizeof(double) * kMaxProfile);
    a.obj = take(sizeof(double) * 4);
    a.rep = take(sizeof(double) * 4);
    a.part = take(sizeof(double) * kMaxPartials);
    a.cont = take(fpad * (size_t)residual_rev_slots());
    return off;
}

// The adjoint covers the FP64 2D open-system step with unit Lewis numbers and
// no gravity; null when supported, else the reason.
const char* adj_unsupported(const sim_t* s) {
    if (s->g.dim != 2) return "the adjoint step is 2D only";
    if (s->prm.precision != SIM_FP64) return "the adjoint step needs precision SIM_FP64";
    if (s->ph.closed) return "the adjoint step needs an open system (p0 = 1)";
    if (s->ph.incompressible) return "the adjoint step needs the variable-density model";
    return nullptr;
}

void adj_ghost(sim_t* s, std::initializer_list<std::pair<double*, int>> fields, cudaStream_t st) {
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (auto& f : fields) {
        job.f[job.nf] = f.first;
        job.what[job.nf] = f.second;
        ++job.nf;
    }
    launch_ghost_adj(s->g, s->bnd, job, st);
}

void adj_ghost_v(sim_t* s, double* const* lv, cudaStream_t st) {
    GhostJob job;
    std::memset(&job, 0, sizeof(job));
    for (int d = 0; d < s->g.dim; ++d) {
        job.f[d] = lv[d];
        job.what[d] = GW_V0 + d;
    }
    job.nf = s->g.dim;
    launch_ghost_adj(s->g, s->bnd, job, st);
}

// The pressure solve maps b to the zero-mean P = M A^+ M b (M removes the
// mean, A the symmetric compact Laplacian), a symmetric operator: its
// transpose is the same solve applied to lambda_P.
cudaError_t adj_poisson(sim_t* s, const double* lP, double* lb, cudaStream_t st) {
    if (s->solve_graphs && lP == s->adj.LP && lb == s->adj.Lb)
        return launch_solve_graph(s, 2, st) == SIM_OK ? cudaGetLastError() : cudaErrorUnknown;
    PoissonPlan* pl = &s->pp;
    cudaError_t e = poisson_enqueue_prologue(pl, lP, lb, st, 0ULL, 0);
    if (e != cudaSuccess) return e;
    int done = 0;
    for (int guard = 0; guard <= pl->max_iter + 1; ++guard) {
        e = cudaMemcpyAsync(&done, pl->ictl + PI_DONE, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (done) break;
        e = poisson_enqueue_body(pl, lb, st, 0ULL);
        if (e != cudaSuccess) return e;
    }
    return poisson_enqueue_epilogue(pl, lb, st, s->adj.rep, s->status, ST_NOCONV, 1);
}

ResidArgs adj_resid_args(sim_t* s, double* const* v, const double* Z, const double* H, const double* kap,
                         double* const* F, const double* T, const double* rho) {
    ResidArgs a = resid_common(s);
    for (int d = 0; d < s->g.dim; ++d) {
        a.v[d] = v[d];
        a.F[d] = F[d];
    }
    a.Z = Z;
    a.H = H;
    a.kap = kap;
    a.T = T;
    a.rho = rho;             // the stage's input density (read by the buoyancy term only)
    a.p0r = SC_P0_N;         // open system: p0 = 1 in every slot
    return a;
}

AdjIn adj_in(sim_t* s, double* const* lv, double* lZ, double* lH, double* lrho) {
    AdjWs& A = s->adj;
    AdjIn li;
    std::memset(&li, 0, sizeof(li));
    for (int d = 0; d < s->g.dim; ++d) {
        li.out[RF_V0 + d] = lv[d];
        li.out[RF_F0 + d] = A.LF[d];
        if (s->ibm_active) li.out[RF_VIB0 + d] = A.Lvib[d];
    }
    li.out[RF_Z] = lZ;
    li.out[RF_H] = lH;
    li.out[RF_KAP] = A.Lkap;
    li.out[RF_T] = A.LT;
    li.out[RF_RHO] = lrho;   // buoyancy only (null without gravity)
    return li;
}

}  // namespace

extern "C" {

sim_status sim_objective(sim_t* s, double* out) {
    if (!s || !out) return SIM_EINVAL;
    if (s->need_init) return fail(s, SIM_ESTATE, "no state yet: step once after setting the fields");
    launch_objective(s->g, s->ph, s->Z, s->kap, s->part, s->io, s->stream);
    CK(cudaMemcpyAsync(out, s->io, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return SIM_OK;
}

sim_status sim_adjoint_workspace_size(const sim_t* s, size_t* bytes) {
    if (!s || !bytes) return SIM_EINVAL;
    *bytes = adj_layout(s, nullptr, nullptr);
    return SIM_OK;
}

sim_status sim_adjoint_begin(sim_t* s, void* d_workspace, size_t workspace_bytes) {
    if (!s) return SIM_EINVAL;
    const char* why = adj_unsupported(s);
    if (why) return fail(s, SIM_EINVAL, "%s", why);
    const size_t need = adj_layout(s, nullptr, nullptr);
    if (!d_workspace || workspace_bytes < need) return fail(s, SIM_ENOMEM, "adjoint workspace needs %zu bytes", need);
    if (((uintptr_t)d_workspace & 255) != 0) return fail(s, SIM_EINVAL, "adjoint workspace must be 256-byte aligned");
    adj_layout(s, &s->adj, (char*)d_workspace);
    s->adj.i_rho = 0;
    s->adj.i_prev = 1;
    {
        // the hand-written reverse sweep of the stage stencil covers Le_F ==
        // Le_O without gravity; differential diffusion (the regularised
        // Le_eps(Z), N_eps(Z) of Eq 3.35) and buoyancy (Eq 3.8b, through the
        // stage's density) take the exact dual-number gather
        const char* dual = std::getenv("LOWMACH_ADJ_DUAL");
        s->adj.use_dual =
            ((dual && dual[0] == '1') || s->ph.Le_F != s->ph.Le_O || s->ph.inv_Fr2 != 0.0) ? 1 : 0;
    }
    CK(cudaMemsetAsync(s->adj.lam_base, 0, s->adj.lam_bytes, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->adj_active = true;
    drop_solve_graphs(s);        // captured against the previous adjoint workspace
    s->solve_graphs = true;
    return SIM_OK;
}

sim_status sim_adjoint_end(sim_t* s) {
    if (!s) return SIM_EINVAL;
    s->adj_active = false;
    s->solve_graphs = false;
    drop_solve_graphs(s);
    std::memset(&s->adj, 0, sizeof(s->adj));
    return SIM_OK;
}

sim_status sim_adjoint_step(sim_t* s, double objective_weight, double* dJ_dprofile) {
    if (!s) return SIM_EINVAL;
    if (!s->adj_active) return fail(s, SIM_ESTATE, "sim_adjoint_begin first");
    if (s->need_init) return fail(s, SIM_ESTATE, "no state yet: load a saved state or step once");
    AdjWs& A = s->adj;
    const Geom& g = s->g;
    const Phys& ph = s->ph;
    const int D = g.dim;
    const double dt = s->prm.dt;
    const long long n = s->nstep;
    cudaStream_t st = s->stream;
    const size_t fpad = sizeof(double) * (size_t)g.npad;
    const Roles r = roles(s, n);
    int La = 0;   // kernels enqueued by this call

    // level-n values, then the step recomputed with its predictor values saved
    for (int d = 0; d < D; ++d) {
        CK(cudaMemcpyAsync(A.v0[d], s->v[d], fpad, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(A.F0[d], s->F[d], fpad, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaMemcpyAsync(A.Z0, s->Z, fpad, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(A.H0, s->H, fpad, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(A.T0, s->T, fpad, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(A.kap0, s->kap, fpad, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(A.rho0, r.rho_n, fpad, cudaMemcpyDeviceToDevice, st));
    {
        int L = 0, body = 0;
        s->adj_save = true;
        cudaError_t e = enqueue_step(s, n, st, false, &L, &body);
        s->adj_save = false;
        CK(e);
        La += L;
        after_step(s);
    }
    // s->vs = v*, s->Zs / Hs = Z* / H*, s->mom = corrector momentum, s->Z / H / T /
    // kap / P = level n+1; A.m0 / Ts / kaps / Ps / Fs = predictor values.
    double* Lrho = A.Lr[A.i_rho];                 // lambda rho^{n+1}, then rho*
    double* Lrn = A.Lr[A.i_prev];                 // lambda rho^n
    const int i_free = 3 - A.i_rho - A.i_prev;
    double* Lrp = A.Lr[i_free];                   // lambda rho^{n-1} (zero on entry)
    const double bc0 = 1.0, bc1 = n == 0 ? -1.0 : -4.0;
    const double bdf[4] = {n == 0 ? bc0 : 3.0, bc1, n == 0 ? 0.0 : 1.0, n == 0 ? dt : 2.0 * dt};

    // objective term of level n+1
    if (objective_weight != 0.0) {
        launch_objective_adj(g, ph, s->Z, s->kap, objective_weight, A.LZ, A.Lkap, st);
        La += 1;
    }

    const bool grav = ph.inv_Fr2 != 0.0;
    for (int stage = 1; stage >= 0; --stage) {   // corrector, then predictor
        const bool corr = stage == 1;
        double* const* lv = corr ? A.Lv : A.Lvs;
        // projection^T (ghost fill of the projected velocity first)
        adj_ghost_v(s, lv, st);
        for (int d = 0; d < D; ++d) CK(cudaMemsetAsync(A.Lm[d], 0, fpad, st));
        ProjAdj pj;
        std::memset(&pj, 0, sizeof(pj));
        for (int d = 0; d < D; ++d) {
            pj.lv[d] = lv[d];
            pj.lF[d] = A.LF[d];
            pj.mom[d] = corr ? s->mom[d] : A.m0[d];
            pj.lmom[d] = A.Lm[d];
        }
        pj.P = corr ? s->P : A.Ps;
        pj.T = corr ? s->T : A.Ts;
        pj.sc = s->sc;
        pj.p0_slot = SC_P0_N;
        pj.lT = A.LT;
        pj.lP = A.LP;
        pj.eA = s->eA;
        pj.eB = s->eB;
        pj.eC = s->eC;
        launch_project_adj(g, pj, st);
        // pressure solve^T
        s->pp.launches = 0;
        CK(adj_poisson(s, A.LP, A.Lb, st));
        La += D + 1 + (s->solve_graphs ? 0 : s->pp.launches);
        // face fluxes and right-hand side^T
        FluxAdj fa;
        std::memset(&fa, 0, sizeof(fa));
        for (int d = 0; d < D; ++d) {
            fa.lF[d] = A.LF[d];
            fa.lFt[d] = A.LFt[d];
            fa.lmom[d] = A.Lm[d];
        }
        fa.lb = A.Lb;
        fa.lrho_new = Lrho;
        fa.lrho_n = Lrn;
        fa.lrho_prev = Lrp;
        fa.lSm = s->ibm_active ? A.LSm : nullptr;
        fa.bdf_c0 = bdf[0];
        fa.bdf_c1 = bdf[1];
        fa.bdf_c2 = bdf[2];
        fa.bdf_den = bdf[3];
        fa.sc = s->sc;
        fa.part = A.part;
        launch_flux_adj(g, s->bnd, fa, st);
        La += 2 + 2 * D + 2;       // flux (2), kappa and Z/H ghost fills (2 x D), state, combination
        // state relation^T (kappa ghosts first), then the Z, H ghost fill^T
        double* lZo = corr ? A.LZ : A.LZs;
        double* lHo = corr ? A.LH : A.LHs;
        adj_ghost(s, {{A.Lkap, GW_KAPPA}}, st);
        launch_state_adj(g, ph, corr ? s->Z : s->Zs, corr ? s->T : A.Ts, corr ? s->kap : A.kaps, A.LT, Lrho,
                         A.Lkap, lZo, lHo, st);
        adj_ghost(s, {{lZo, GW_Z}, {lHo, GW_H}}, st);
        // combination^T
        CombAdj cb;
        std::memset(&cb, 0, sizeof(cb));
        for (int d = 0; d < D; ++d) {
            cb.lmom[d] = A.Lm[d];
            cb.lv[d] = A.Lv[d];
            cb.v_n[d] = A.v0[d];
        }
        cb.lZin = lZo;
        cb.lHin = lHo;
        for (int k = 0; k < 5; ++k) {
            cb.lR[k] = A.LR[k];
            cb.lRh[k] = A.LRh[k];
        }
        cb.lZ = A.LZ;
        cb.lH = A.LH;
        cb.lrho_n = Lrn;
        cb.rho_n = A.rho0;
        cb.dt = dt;
        cb.mode = corr ? MODE_CORR : (n == 0 ? MODE_PRED_EULER : MODE_PRED_AB2);
        launch_comb_adj(g, cb, st);
        // stencil^T at the stage's input level
        AdjR lr;
        for (int k = 0; k < 5; ++k) lr.R[k] = A.LR[k];
        if (corr) {
            for (int d = 0; d < D; ++d) CK(cudaMemsetAsync(A.Lvs[d], 0, fpad, st));
            CK(cudaMemsetAsync(A.LZs, 0, fpad, st));
            CK(cudaMemsetAsync(A.LHs, 0, fpad, st));
            // the stencil read rho* (buoyancy): its lambda joins Lrho, which the
            // corrector's state relation^T has consumed and zeroed and the
            // predictor's flux and state relation^T use next as lambda rho*
            const ResidArgs a = adj_resid_args(s, s->vs, s->Zs, s->Hs, A.kaps, A.Fs, A.Ts, A.rhos);
            launch_residual_adj(g, ph, a, 0.0, lr, adj_in(s, A.Lvs, A.LZs, A.LHs, grav ? Lrho : nullptr),
                                A.use_dual ? nullptr : A.cont, st);
        } else {
            const ResidArgs a = adj_resid_args(s, A.v0, A.Z0, A.H0, A.kap0, A.F0, A.T0, A.rho0);
            launch_residual_adj(g, ph, a, 0.0, lr, adj_in(s, A.Lv, A.LZ, A.LH, grav ? Lrn : nullptr),
                                A.use_dual ? nullptr : A.cont, st);
        }
        La += A.use_dual ? 1 : 2;
    }
    // density roles one level down; the consumed rho buffer is zero again
    A.i_rho = A.i_prev;
    A.i_prev = i_free;
    s->launches_last = La;
    CK(cudaGetLastError());
    if (dJ_dprofile) {
        if (!s->ibm_active || s->ibm.kind != SIM_IBM_SLOT || s->ibm.n_profile < 2)
            return fail(s, SIM_EINVAL, "dJ_dprofile needs a slot body with a flux profile");
        launch_profile_grad(g, s->ibm, s->chi, A.Lvib[1], A.LSm, A.col, A.grad, st);
        s->launches_last += 2;
        CK(cudaMemcpyAsync(dJ_dprofile, A.grad, sizeof(double) * s->ibm.n_profile, cudaMemcpyDeviceToHost, st));
    }
    const sim_status st_dev = check_device_status(s);
    if (st_dev != SIM_OK) return st_dev;
    if (s->solve_graphs) {
        // kernels of the graph-launched solves: their loops ran the reported
        // iterations (the last transposed solve's count for both) less those
        // captured ahead of the loop, which solve_fixed holds
        double it[4] = {0.0, 0.0, 0.0, 0.0};
        CK(cudaMemcpy(&it[0], s->sc + SC_ITERS_PRED, sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&it[1], s->sc + SC_ITERS_CORR, sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&it[2], A.rep, sizeof(double), cudaMemcpyDeviceToHost));
        for (int k = 0; k < 3; ++k) it[k] = poisson_loop_iters(&s->pp, it[k]);
        s->launches_last += s->solve_fixed[0] + (int)(s->solve_body[0] * it[0]) + s->solve_fixed[1] +
                            (int)(s->solve_body[1] * it[1]) + 2 * (s->solve_fixed[2] + (int)(s->solve_body[2] * it[2]));
    }
    return SIM_OK;
}

// Adjoint of a state field at the current level, interior cells (or faces)
// as for sim_fields: get copies it out, set adds buf to it.
sim_status sim_adjoint_field(sim_t* s, int id, double* buf, int dir) {
    if (!s || !buf || (dir != SIM_GET && dir != SIM_SET)) return SIM_EINVAL;
    if (!s->adj_active) return fail(s, SIM_ESTATE, "sim_adjoint_begin first");
    AdjWs& A = s->adj;
    const Geom& g = s->g;
    double* f = nullptr;
    int face = -1;
    switch (id) {
        case SIM_FIELD_U: f = A.Lv[0]; break;
        case SIM_FIELD_V: f = A.Lv[1]; break;
        case SIM_FIELD_Z: f = A.LZ; break;
        case SIM_FIELD_H: f = A.LH; break;
        case SIM_FIELD_T: f = A.LT; break;
        case SIM_FIELD_RHO: f = A.Lr[A.i_rho]; break;
        case SIM_FIELD_KAPPA: f = A.Lkap; break;
        case SIM_FIELD_SM: f = A.LSm; break;
        case SIM_FIELD_FX: f = A.LF[0]; face = 0; break;
        case SIM_FIELD_FY: f = A.LF[1]; face = 1; break;
        default: return fail(s, SIM_EINVAL, "no adjoint for field %d", id);
    }
    long long m = 1;
    for (int d = 0; d < g.dim; ++d) m *= g.n[d] + (d == face ? 1 : 0);
    const size_t bytes = sizeof(double) * (size_t)m;
    if (dir == SIM_GET) {
        launch_pack(g, f, s->io, face, s->stream);
        CK(cudaMemcpyAsync(buf, s->io, bytes, cudaMemcpyDeviceToHost, s->stream));
    } else {
        if (face >= 0) return fail(s, SIM_EINVAL, "adjoint seeds are cell fields");
        CK(cudaMemcpyAsync(s->io, buf, bytes, cudaMemcpyHostToDevice, s->stream));
        launch_add_unpack(g, s->io, f, s->stream);
    }
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return SIM_OK;
}

sim_status sim_poisson_batch_workspace_size(const int n[2], const int periodic[2], int nb, int precision,
                                            size_t* bytes) {
    if (!n || !periodic || !bytes || nb < 1 || (precision != SIM_FP64 && precision != SIM_MIXED)) return SIM_EINVAL;
    const int nn[3] = {n[0], n[1], 1};
    const int per[3] = {periodic[0] != 0, periodic[1] != 0, 0};
    const char* err = nullptr;
    const size_t b = poisson_plan_bytes_batch(2, nn, per, precision == SIM_MIXED, 0, nb, nullptr, nullptr, &err);
    if (b == 0) return SIM_EINVAL;
    *bytes = b;
    return SIM_OK;
}

sim_status sim_poisson_solve_batch(const int n[2], const double h[2], const int periodic[2], int nb, int precision,
                                   const double* d_b, double* d_P, double rtol, int max_iter, void* d_workspace,
                                   size_t workspace_bytes, void* cuda_stream, int* iters, double* rel_resid) {
    if (!n || !h || !periodic || !d_b || !d_P || !d_workspace || nb < 1) return SIM_EINVAL;
    if (precision != SIM_FP64 && precision != SIM_MIXED) return SIM_EINVAL;
    if (!(rtol > 0.0 && rtol < 1.0) || max_iter < 1) return SIM_EINVAL;
    const int nn[3] = {n[0], n[1], 1};
    const double hh[3] = {h[0], h[1], 1.0};
    const int per[3] = {periodic[0] != 0, periodic[1] != 0, 0};
    for (int d = 0; d < 2; ++d)
        if (nn[d] < 2 || !(hh[d] > 0.0)) return SIM_EINVAL;
    const int mixed = precision == SIM_MIXED;
    const char* err = nullptr;
    const size_t need = poisson_plan_bytes_batch(2, nn, per, mixed, 0, nb, nullptr, nullptr, &err);
    if (need == 0) return SIM_EINVAL;
    if (workspace_bytes < need) return SIM_ENOMEM;
    PoissonPlan pl;
    std::vector<double> minv;
    if (!poisson_plan_init_batch(&pl, 2, nn, hh, per, mixed, 0, 0, rtol, max_iter, nb, d_workspace, workspace_bytes,
                                 &minv, &err))
        return SIM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!poisson_upload_coarse(&pl, minv, st, &err)) return SIM_ECUDA;
    cudaError_t e = poisson_solve_host_loop(&pl, d_b, d_P, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SIM_ECUDA;
    std::vector<double> sc((size_t)nb * PS_NSCAL);
    std::vector<int> ic((size_t)nb * PI_NINT);
    if (cudaMemcpy(sc.data(), pl.scal, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SIM_ECUDA;
    if (cudaMemcpy(ic.data(), pl.ictl, sizeof(int) * ic.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SIM_ECUDA;
    int noconv = 0;
    for (int k = 0; k < nb; ++k) {
        if (iters) iters[k] = (int)sc[(size_t)k * PS_NSCAL + PS_ITERS];
        if (rel_resid) rel_resid[k] = sc[(size_t)k * PS_NSCAL + PS_RELRES];
        noconv |= ic[(size_t)k * PI_NINT + PI_NOCONV];
    }
    return noconv ? SIM_ENOCONV : SIM_OK;
}

// ------------------------------ batches --------------------------------------
// Many independent simulations advanced by one CUDA graph per step: each
// simulation's whole step (its kernels and its two pressure-solve while nodes)
// is captured on its own forked stream, so the graph holds one independent
// branch per simulation and the GPU runs their latency-bound chains
// concurrently.  Simulations must step in lockstep (same step count).
}  // extern "C"

// Members of a batch with the same grid and pressure-solver settings share
// one batched solve per stage (one launch per multigrid level and CG update
// for all of them) when the batch has a workspace.
struct BatchGroup {
    std::vector<int> members;
    PoissonPlan pl;
    std::vector<double> minv;
    double* bb;                  // contiguous right-hand sides [nb][N]
    double* xb;                  // contiguous solutions (warm start in, answer out)
    const double** bptr;         // device table: each member's b
    double** xptr;               // device table: each member's P
    double** rep[2];             // device tables: each member's predictor / corrector report slots
    int** status;                // device table: each member's status word
    cudaStream_t st, side;
    cudaEvent_t ev;
    int fixed_launches;          // kernels of one solve outside its loop
    int body_launches;           // kernels per iteration
};

struct sim_batch {
    std::vector<sim_t*> sims;
    cudaStream_t stream;         // caller's stream (the batch graph runs here)
    cudaStream_t cap;            // capture origin
    cudaEvent_t fork;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t gexec[6];
    bool gvalid[6];
    std::vector<BatchGroup> groups;
    std::vector<int> group_of;   // member -> group, or -1 (own solves)
    // Member-batched stage kernels: the grouped members (2D, open systems)
    // run each stage kernel as one launch over all of them; per phase, the
    // records of every launch position and their work lists (device).
    std::vector<int> staged;     // members whose stage kernels are batched
    StageRec* stab;              // [6 phases][kStagePos][staged] records
    int* swork;                  // [6 phases][kStagePos][staged + 1] block starts
    int stage_launches[6];       // batched launches of a phase's graph
    int last_phase;
    std::vector<int> stage_blocks;   // host copy of the last tables' block starts
    std::vector<int> stage_kinds;    // kind of each launch position
    char err[512];
};

namespace {

// Members whose pressure solves can be batched together: same 2D grid,
// spacing, sides and solver settings (precision, sweeps, coarse level,
// tolerance, iteration cap).
std::vector<std::vector<int>> batch_groups(sim_t* const* sims, int n) {
    std::vector<std::vector<int>> out;
    auto same = [](const sim_t* a, const sim_t* b) {
        const PoissonPlan &p = a->pp, &q = b->pp;
        return a->g.dim == 2 && b->g.dim == 2 && a->g.n[0] == b->g.n[0] && a->g.n[1] == b->g.n[1] &&
               a->g.h[0] == b->g.h[0] && a->g.h[1] == b->g.h[1] && a->g.periodic[0] == b->g.periodic[0] &&
               a->g.periodic[1] == b->g.periodic[1] && p.mg_fp32 == q.mg_fp32 && p.sweeps == q.sweeps &&
               p.top == q.top && p.rtol == q.rtol && p.max_iter == q.max_iter &&
               (p.r32 != nullptr) == (q.r32 != nullptr) && p.nlev > 1;
    };
    std::vector<int> used((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        if (used[(size_t)i] || sims[i]->g.dim != 2 || sims[i]->pp.nlev < 2) continue;
        std::vector<int> g{i};
        used[(size_t)i] = 1;
        for (int j = i + 1; j < n; ++j)
            if (!used[(size_t)j] && same(sims[i], sims[j])) {
                g.push_back(j);
                used[(size_t)j] = 1;
            }
        if (g.size() >= 2) out.push_back(g);
    }
    return out;
}

constexpr int kStagePos = 16;   // launch positions of one step's stage kernels (at most)

// Members whose stage kernels can run as batched launches: every member that
// is in a solve group, when all of them are 2D open systems (their stage is
// the stencil, the fused state relation and fluxes, the right-hand side and
// the projection); LOWMACH_NO_STAGE_BATCH=1 keeps one launch per member.
std::vector<int> staged_members(sim_t* const* sims, int n, const std::vector<std::vector<int>>& groups) {
    std::vector<int> out;
    const char* e = std::getenv("LOWMACH_NO_STAGE_BATCH");
    if (e && e[0] == '1') return out;
    for (const auto& g : groups)
        for (int k : g) {
            if (sims[k]->g.dim != 2 || sims[k]->ph.closed || sims[k]->ph.mixed != sims[groups[0][0]]->ph.mixed)
                return std::vector<int>();
            out.push_back(k);
        }
    std::sort(out.begin(), out.end());
    return out;
}

size_t stage_table_bytes(int nstaged) {
    if (nstaged == 0) return 0;
    return a256(sizeof(StageRec) * (size_t)6 * kStagePos * nstaged) +
           a256(sizeof(int) * (size_t)6 * kStagePos * (nstaged + 1));
}

// Workspace bytes of one group (plan, contiguous b and x, pointer tables).
size_t group_bytes(const sim_t* s0, int nb, const char** err) {
    const PoissonPlan& p = s0->pp;
    const int per[3] = {s0->g.periodic[0], s0->g.periodic[1], 0};
    const size_t pb = poisson_plan_bytes_batch(2, s0->g.n, per, p.mg_fp32, s0->prm.mg_tail_cells, nb, nullptr,
                                               nullptr, err);
    if (pb == 0) return 0;
    return a256(pb) + 2 * a256(sizeof(double) * (size_t)nb * (size_t)s0->g.ncell) + 5 * a256(sizeof(void*) * nb);
}

sim_status bfail(sim_batch_t* b, sim_status st, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return bfail(b, SIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void batch_drop_graphs(sim_batch_t* b) {
    for (int k = 0; k < 6; ++k)
        if (b->gvalid[k]) {
            cudaGraphExecDestroy(b->gexec[k]);
            b->gvalid[k] = false;
        }
}

// One stage's batched solve of a group, captured on G.st: gather b and the
// warm start, prologue + while node, epilogue, scatter, per-member reports.
cudaError_t batch_group_solve(BatchGroup& G, int which) {
    const int nb = (int)G.members.size();
    const long long N = G.pl.N;
    G.pl.launches = 0;
    launch_gather(G.bptr, G.bb, N, nb, G.st);
    launch_gather((const double* const*)G.xptr, G.xb, N, nb, G.st);
    int body = 0;
    cudaError_t e = capture_while_solve(&G.pl, G.bb, G.xb, G.st, G.side, &body, 0);
    if (e != cudaSuccess) return e;
    e = poisson_enqueue_epilogue(&G.pl, G.xb, G.st, nullptr, nullptr, 0, 0);
    if (e != cudaSuccess) return e;
    launch_scatter(G.xb, G.xptr, N, nb, G.st);
    e = poisson_enqueue_batch_report(&G.pl, G.rep[which], G.status, ST_NOCONV, G.st);
    G.body_launches = body;
    G.fixed_launches = G.pl.launches - body + 3;   // + gathers and scatter
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Records of the staged members' stage kernels for one phase: each member's
// sections are enqueued with a collector installed (nothing is launched), the
// records of each launch position are stored side by side with the position's
// work list (block starts), and both go to the phase's device tables.
sim_status batch_stage_tables(sim_batch_t* b, int phase, int npos[3]) {
    const int secs[3][2] = {{SEC_PRED, SEC_PRED}, {SEC_MID, SEC_MID}, {SEC_END, SEC_END}};
    const int ns = (int)b->staged.size();
    std::vector<StageRec> all((size_t)kStagePos * ns);
    std::vector<int> starts((size_t)kStagePos * (ns + 1), 0);
    std::vector<StageRec> buf(kStagePos);
    int base = 0;
    for (int k = 0; k < 3; ++k) {
        npos[k] = 0;
        for (int j = 0; j < ns; ++j) {
            sim_t* s = b->sims[(size_t)b->staged[(size_t)j]];
            StageCollector col{buf.data(), 0, kStagePos - base, false};
            set_stage_collector(&col);
            int L = 0, body = 0;
            const cudaError_t e = enqueue_step_sections(s, s->nstep, s->cap, true, &L, &body, secs[k][0], secs[k][1]);
            set_stage_collector(nullptr);
            if (e != cudaSuccess) return bfail(b, SIM_ECUDA, "stage records: %s", cudaGetErrorString(e));
            if (col.overflow) return bfail(b, SIM_EINVAL, "stage records: more than %d launches", kStagePos);
            if (j == 0) npos[k] = col.n;
            if (col.n != npos[k]) return bfail(b, SIM_EINVAL, "stage records differ between members");
            for (int i = 0; i < col.n; ++i) {
                if (j > 0 && buf[(size_t)i].kind != all[(size_t)(base + i) * ns].kind)
                    return bfail(b, SIM_EINVAL, "stage records differ between members");
                all[(size_t)(base + i) * ns + j] = buf[(size_t)i];
            }
        }
        for (int i = 0; i < npos[k]; ++i) {
            int* st = starts.data() + (size_t)(base + i) * (ns + 1);
            for (int j = 0; j < ns; ++j) st[j + 1] = st[j] + all[(size_t)(base + i) * ns + j].nblocks;
        }
        base += npos[k];
    }
    StageRec* dtab = b->stab + (size_t)phase * kStagePos * ns;
    int* dwork = b->swork + (size_t)phase * kStagePos * (ns + 1);
    BCK(cudaMemcpy(dtab, all.data(), sizeof(StageRec) * (size_t)base * ns, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(dwork, starts.data(), sizeof(int) * (size_t)base * (ns + 1), cudaMemcpyHostToDevice));
    b->stage_blocks.assign(starts.begin(), starts.end());
    b->stage_kinds.assign((size_t)base, 0);
    for (int i = 0; i < base; ++i) b->stage_kinds[(size_t)i] = all[(size_t)i * ns].kind;
    return SIM_OK;
}

// The batch step as one graph: per-member sections on forked streams, joined
// before and after each stage's batched solves (one forked stream per group).
// The staged members' stage kernels run as member-batched launches on the
// capture stream, alongside the other members' sections.
sim_status batch_capture(sim_batch_t* b, int phase) {
    const int ns = (int)b->staged.size();
    int npos[3] = {0, 0, 0};
    if (ns > 0) {
        const sim_status st = batch_stage_tables(b, phase, npos);
        if (st != SIM_OK) return st;
    }
    std::vector<char> staged(b->sims.size(), 0);
    for (int k : b->staged) staged[(size_t)k] = 1;
    const int mixed = ns > 0 ? b->sims[(size_t)b->staged[0]]->ph.mixed : 0;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaSuccess;
    const int secs[3][2] = {{SEC_PRED, SEC_POIS_PRED}, {SEC_MID, SEC_POIS_CORR}, {SEC_END, SEC_END}};
    for (size_t i = 0; i < b->sims.size(); ++i) {
        b->sims[i]->launches_fixed_graph[phase] = 0;
        b->sims[i]->body_launches = 0;
    }
    b->stage_launches[phase] = 0;
    int base = 0;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->fork, b->cap);
        for (size_t i = 0; i < b->sims.size() && e == cudaSuccess; ++i) {
            if (staged[i]) continue;
            sim_t* s = b->sims[i];
            const bool batched = b->group_of[i] >= 0;
            // a batched member leaves its solve to the group
            const int last = (batched && k < 2) ? secs[k][0] : secs[k][1];
            e = cudaStreamWaitEvent(s->cap, b->fork, 0);
            int L = 0, body = 0;
            if (e == cudaSuccess) e = enqueue_step_sections(s, s->nstep, s->cap, true, &L, &body, secs[k][0], last);
            s->launches_fixed_graph[phase] += L;
            if (!batched && body > 0) s->body_launches = body;
            if (e == cudaSuccess) e = cudaEventRecord(b->join[i], s->cap);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[i], 0);
        }
        // the staged members' stage kernels, one launch per position
        for (int p = 0; p < npos[k] && e == cudaSuccess; ++p) {
            const int pos = base + p;
            const StageRec* recs = b->stab + ((size_t)phase * kStagePos + pos) * ns;
            const int* work = b->swork + ((size_t)phase * kStagePos + pos) * (ns + 1);
            const int total = b->stage_blocks[(size_t)pos * (ns + 1) + ns];
            e = launch_stage_batched(b->stage_kinds[(size_t)pos], 2, mixed, recs, work, ns, total, b->cap);
            b->stage_launches[phase] += 1;
        }
        base += npos[k];
        if (k == 2 || b->groups.empty()) continue;
        if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->cap);
        for (BatchGroup& G : b->groups) {
            if (e == cudaSuccess) e = cudaStreamWaitEvent(G.st, b->fork, 0);
            if (e == cudaSuccess) e = batch_group_solve(G, k);
            if (e == cudaSuccess) e = cudaEventRecord(G.ev, G.st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, G.ev, 0);
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(b, SIM_ECUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->gexec[phase], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, SIM_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    b->gvalid[phase] = true;
    return SIM_OK;
}

}  // namespace

extern "C" {

sim_status sim_batch_workspace_size(sim_t* const* sims, int n, size_t* bytes) {
    if (!sims || n < 1 || !bytes) return SIM_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!sims[i]) return SIM_EINVAL;
    size_t total = 0;
    const char* err = nullptr;
    const auto groups = batch_groups(sims, n);
    for (const auto& g : groups) {
        const size_t gb = group_bytes(sims[g[0]], (int)g.size(), &err);
        if (gb == 0) return SIM_EINVAL;
        total += gb;
    }
    total += stage_table_bytes((int)staged_members(sims, n, groups).size());
    *bytes = total;
    return SIM_OK;
}

sim_status sim_batch_create(sim_t* const* sims, int n, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                            sim_batch_t** out) {
    if (!out || !sims || n < 1) return SIM_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
            if (!sims[i] || sims[i] == sims[j]) return SIM_EINVAL;
    if (!sims[0]) return SIM_EINVAL;
    if (d_workspace && ((uintptr_t)d_workspace & 255) != 0) return SIM_EINVAL;
    size_t need = 0;
    if (d_workspace) {
        const sim_status st = sim_batch_workspace_size(sims, n, &need);
        if (st != SIM_OK) return st;
        if (workspace_bytes < need) return SIM_ENOMEM;
    }
    sim_batch_t* b = new sim_batch();
    b->sims.assign(sims, sims + n);
    b->stream = (cudaStream_t)cuda_stream;
    b->join.assign((size_t)n, nullptr);
    b->group_of.assign((size_t)n, -1);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        sim_batch_destroy(b);
        return SIM_ECUDA;
    }
    if (d_workspace) {
        // batched solves of same-grid members: plans, contiguous vectors and
        // device pointer tables carved from the workspace
        char* cur = (char*)d_workspace;
        const char* err = nullptr;
        for (const auto& gm : batch_groups(sims, n)) {
            b->groups.emplace_back();
            BatchGroup& G = b->groups.back();
            std::memset(&G.pl, 0, sizeof(G.pl));
            G.members = gm;
            const int nb = (int)gm.size();
            const sim_t* s0 = sims[gm[0]];
            const size_t gb = group_bytes(s0, nb, &err);
            const int per[3] = {s0->g.periodic[0], s0->g.periodic[1], 0};
            const size_t pb = a256(poisson_plan_bytes_batch(2, s0->g.n, per, s0->pp.mg_fp32, s0->prm.mg_tail_cells,
                                                            nb, nullptr, nullptr, &err));
            bool ok = poisson_plan_init_batch(&G.pl, 2, s0->g.n, s0->g.h, per, s0->pp.mg_fp32, s0->pp.sweeps,
                                              s0->prm.mg_tail_cells, s0->pp.rtol, s0->pp.max_iter, nb, cur, pb,
                                              &G.minv, &err);
            if (ok) ok = poisson_upload_coarse(&G.pl, G.minv, b->stream, &err);
            if (!ok) {
                sim_batch_destroy(b);
                return SIM_EINVAL;
            }
            char* q = cur + pb;
            const size_t vb = a256(sizeof(double) * (size_t)nb * (size_t)s0->g.ncell), tb = a256(sizeof(void*) * nb);
            G.bb = (double*)q;
            G.xb = (double*)(q + vb);
            G.bptr = (const double**)(q + 2 * vb);
            G.xptr = (double**)(q + 2 * vb + tb);
            G.rep[0] = (double**)(q + 2 * vb + 2 * tb);
            G.rep[1] = (double**)(q + 2 * vb + 3 * tb);
            G.status = (int**)(q + 2 * vb + 4 * tb);
            cur += gb;
            std::vector<const void*> tab[5];
            for (int k : gm) {
                sim_t* m = sims[k];
                b->group_of[(size_t)k] = (int)b->groups.size() - 1;
                tab[0].push_back(m->b);
                tab[1].push_back(m->P);
                tab[2].push_back(m->sc + SC_ITERS_PRED);
                tab[3].push_back(m->sc + SC_ITERS_CORR);
                tab[4].push_back(m->status);
            }
            void* dst[5] = {(void*)G.bptr, (void*)G.xptr, (void*)G.rep[0], (void*)G.rep[1], (void*)G.status};
            for (int t = 0; t < 5 && e == cudaSuccess; ++t)
                e = cudaMemcpyAsync(dst[t], tab[t].data(), sizeof(void*) * nb, cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) {
                sim_batch_destroy(b);
                return SIM_ECUDA;
            }
        }
        b->staged = staged_members(sims, n, batch_groups(sims, n));
        if (!b->staged.empty()) {
            const int ns = (int)b->staged.size();
            b->stab = (StageRec*)cur;
            b->swork = (int*)(cur + a256(sizeof(StageRec) * (size_t)6 * kStagePos * ns));
        }
    }
    *out = b;
    return SIM_OK;
}

// Kernels the last batch step launched, after sim_batch_sync: the members'
// own kernels plus, per group, its solves' kernels (the loop runs as long as
// its slowest member).
sim_status sim_batch_query_launches(sim_batch_t* b, double* out) {
    if (!b || !out) return SIM_EINVAL;
    double total = 0.0;
    for (sim_t* s : b->sims) {
        double v = 0.0;
        const sim_status st = sim_query(s, SIM_Q_KERNEL_LAUNCHES, &v);
        if (st != SIM_OK) return bfail(b, st, "%s", s->err);
        total += v;
    }
    for (const BatchGroup& G : b->groups) {
        double itp = 0.0, itc = 0.0;
        for (int k : G.members) {
            double a = 0.0, c = 0.0;
            sim_query(b->sims[(size_t)k], SIM_Q_ITERS_PRED, &a);
            sim_query(b->sims[(size_t)k], SIM_Q_ITERS_CORR, &c);
            itp = a > itp ? a : itp;
            itc = c > itc ? c : itc;
        }
        total += 2.0 * G.fixed_launches +
                 G.body_launches * (poisson_loop_iters(&G.pl, itp) + poisson_loop_iters(&G.pl, itc));
    }
    total += b->stage_launches[b->last_phase];
    *out = total;
    return SIM_OK;
}

sim_status sim_batch_step(sim_batch_t* b, int nsteps) {
    if (!b || nsteps < 0) return SIM_EINVAL;
    // set-up and the first two (eager) steps go through each simulation's own path
    for (sim_t* s : b->sims) {
        const int need = (s->g.dim == 3) ? 0x1f : 0x1b;
        if ((s->fields_set & need) != need) return bfail(b, SIM_ESTATE, "a simulation has no fields set");
        if (s->need_init) batch_drop_graphs(b);
    }
    int done = 0;
    while (done < nsteps && (b->sims[0]->need_init || b->sims[0]->nstep < 2)) {
        for (sim_t* s : b->sims) {
            const sim_status st = sim_step(s, 1);
            if (st != SIM_OK) return bfail(b, st, "simulation step: %s", s->err);
        }
        ++done;
    }
    if (done == nsteps) return SIM_OK;
    const long long n0 = b->sims[0]->nstep;
    const int rb0 = b->sims[0]->rho_base;
    for (sim_t* s : b->sims)
        if (s->nstep != n0 || s->rho_base != rb0 || s->need_init)
            return bfail(b, SIM_ESTATE, "the simulations of a batch must step in lockstep");
    // the batch stream follows each simulation's stream, and vice versa at the end
    for (size_t i = 0; i < b->sims.size(); ++i) {
        BCK(cudaEventRecord(b->join[i], b->sims[i]->stream));
        BCK(cudaStreamWaitEvent(b->stream, b->join[i], 0));
    }
    for (; done < nsteps; ++done) {
        const int phase = (int)(b->sims[0]->nstep % 6);
        if (!b->gvalid[phase]) {
            const sim_status st = batch_capture(b, phase);
            if (st != SIM_OK) return st;
        }
        BCK(cudaGraphLaunch(b->gexec[phase], b->stream));
        b->last_phase = phase;
        for (sim_t* s : b->sims) {
            s->launches_last = -(s->launches_fixed_graph[phase] + 1);
            after_step(s);
        }
    }
    BCK(cudaEventRecord(b->fork, b->stream));
    for (sim_t* s : b->sims) BCK(cudaStreamWaitEvent(s->stream, b->fork, 0));
    return SIM_OK;
}

sim_status sim_batch_sync(sim_batch_t* b) {
    if (!b) return SIM_EINVAL;
    BCK(cudaStreamSynchronize(b->stream));
    for (sim_t* s : b->sims) {
        const sim_status st = sim_sync(s);
        if (st != SIM_OK) return bfail(b, st, "%s", s->err);
    }
    return SIM_OK;
}

const char* sim_batch_last_error(const sim_batch_t* b) { return b ? b->err : "null handle"; }

void sim_batch_destroy(sim_batch_t* b) {
    if (!b) return;
    batch_drop_graphs(b);
    for (BatchGroup& G : b->groups) {
        if (G.st) cudaStreamDestroy(G.st);
        if (G.side) cudaStreamDestroy(G.side);
        if (G.ev) cudaEventDestroy(G.ev);
    }
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
