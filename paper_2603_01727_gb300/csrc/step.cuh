// Kernels of one predictor / corrector stage (everything but the Poisson
// solve) and their host launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lm {

// Device scalar slots of a simulation.
enum : int {
    SC_P0_N = 0, SC_P0_NM1 = 1, SC_P0_NM2 = 2, SC_P0_STAR = 3, SC_P0_NEW = 4,
    SC_MASS = 5, SC_OUT_AREA = 6,
    SC_ITERS_PRED = 8, SC_RELRES_PRED = 9, SC_ITERS_CORR = 10, SC_RELRES_CORR = 11,
    SC_G_N = 12, SC_G_NM1 = 13,   // right-hand side of Eq 2.38 at levels n, n-1 (semi-enclosed)
    SC_INV_OFF = 16,      // slot p0_slot + SC_INV_OFF holds 1 / p0 of that slot (slots 16..20)
    SC_NSCAL = 32
};
// Device status bits (int word).
enum : int { ST_NOCONV = 1, ST_NAN = 2 };

enum Mode : int { MODE_PRED_EULER = 0, MODE_PRED_AB2 = 1, MODE_CORR = 2 };

// Boundary description on the device: per direction and side, the kind of
// every position of the full padded slab (uint8), plus ghost-fill job lists.
struct Bnd {
    const uint8_t* kind[3][2];
    int bc[3][2];
};

// What a ghost-filled field is: scalar Z, H, kappa, or velocity component c.
enum GhostWhat : int { GW_Z = 0, GW_H = 1, GW_KAPPA = 2, GW_V0 = 3 };
constexpr int kMaxGhostFields = 6;
struct GhostJob {
    double* f[kMaxGhostFields];
    int what[kMaxGhostFields];
    int nf;
};

// Per-step checks (paper Eq 3.24, the global mass balance stated after
// Eq 4.22, and the predictor-corrector differences of Sec. 4.2.2), computed on
// demand from the state after a step.
enum : int {
    DG_MAXRES = 0,   // max |d_t rho + sum_j delta_1 F_j / delta_1 x_j - S_m|
    DG_MAXDRHO = 1,  // max |d_t rho|
    DG_MAXSM = 2,    // max |S_m|
    DG_BAL = 3,      // sum (d_t rho - S_m) dV + net outward boundary flux
    DG_DU = 4,       // sum (v*_i - v_i)^2 dV, i = 0, 1, 2
    DG_DP = 7,       // sum (P* - P)
    DG_DP2 = 8,      // sum (P* - P)^2
    DG_N = 9
};
constexpr int kDiagBlocks = 608;
struct DiagArgs {
    const double* rho_new;
    const double* rho_n;
    const double* rho_prev;
    double c0, c1, c2, iden;   // d_t rho = (c0 rho_new + c1 rho_n + c2 rho_prev) * iden
    const double* F[3];
    const double* Sm;          // may be null
    const double* v[3];        // corrector velocity (padded)
    const double* vs[3];       // predictor velocity (padded)
    const double* P;           // compact P^{n+1}
    const double* Ps;          // compact P* of the same step
    double* part;              // DG_N x kDiagBlocks partials
    double* out;               // DG_N results (sums already times dV)
};
cudaError_t launch_diagnostics(const Geom& g, const DiagArgs& a, cudaStream_t st);

struct ResidArgs {
    const double* v[3];
    const double* Z;
    const double* H;
    const double* rho;
    const double* kap;
    const double* F[3];
    const double* Zb;
    const double* Hb;
    const double* rhob;
    const double* vb[3];
    void* Rst[5];            // stored residuals (v0, v1, v2, Z, H), of the kernel's arithmetic type
    const void* Rrd[5];      // previous (AB2) or level-n (corrector) residuals
    const double* T;         // temperature of the residual's level (1/rho = T / p0)
    int p0r;                 // p0 slot of the residual's level
    double* Zo;
    double* Ho;
    double* mo[3];
    const uint8_t* chi;
    const double* vib[3];
    Bnd bnd;                 // boundary kinds for the fused ghost fill of Zo, Ho
    GhostJob gj;             // {Zo, Ho} to ghost-fill in the kernel (nf = 0: none)
    double Z_ib, H_ib, inv_Da;
    int ibm;
    const double* sc;
    int p0a, p0b, p0c;
    double w0, w1, w2, wden;  // dp0/dt = (w0 sc[a] + w1 sc[b] + w2 sc[c]) / wden (wden = 0: zero)
    double iwden;             // 1 / wden
    int mode;
    double dt;
    // mixed path: float-float images (hi, lo) of v0, v1, v2, Z, H and kappa,
    // six planes of npad float2 written by launch_ff_images (null: the
    // stencil splits each double as it loads it)
    const float2* ffs;
};

struct FluxArgs {
    const double* mom[3];    // provisional momentum (padded layout, interior valid)
    double* F[3];            // out: interface fluxes (padded face layout)
    const double* rho_new;
    const double* rho_n;
    const double* rho_prev;
    const double* Sm;        // may be null
    double bdf_c0, bdf_c1, bdf_c2, bdf_den;  // d_t rho = (c0 new + c1 n + c2 prev) / den
    const double* sc;
    int p0_slot;             // p0 of the stage (inflow density p0 / T_in)
    double* part;            // partial sums of the global mass balance
    double* b;               // right-hand side (compact)
    int correct;             // 1: shift outflow fluxes, build b; 0: fluxes only (t = 0)
    // k_rhs: mean(b) into *mb_out (block partials mb_part, last-block counter
    // mb_cnt), when mb_out is not null
    double* mb_part;
    unsigned int* mb_cnt;
    double* mb_out;
    // initial guess of the stage's pressure solve, formed in place in P
    // (compact) by k_rhs: GUESS_COPY keeps P in Pm1; GUESS_EXTRAP also sets
    // P = 2 P - Pm1 (linear extrapolation from the last two steps' pressures);
    // GUESS_SHIFT adds Pd (the last step's P - P*) to the predictor's P*
    int guess;
    double* P;
    double* Pm1;
    const double* Pd;
};
enum { GUESS_NONE = 0, GUESS_COPY = 1, GUESS_EXTRAP = 2, GUESS_SHIFT = 3 };

struct ProjArgs {
    double* F[3];
    const double* P;         // compact
    const double* mom[3];
    const double* rho;
    const double* T;         // temperature of the stage (1/rho = T / p0)
    const double* sc;
    int p0_slot;
    double* v[3];
    double eA, eB, eC;       // quadratic extrapolation coefficients (Eq 3.28)
    Bnd bnd;                 // boundary kinds for the fused ghost fill of v
    GhostJob gj;             // v components to ghost-fill in the kernel (nf = 0: none)
    double* rot;             // not null: rotate the p0 history in these scalars (the step's end)
    double* Pd;              // not null: Pd = P - Pstar (the corrector's projection)
    const double* Pstar;
};

// Fields read by the stage stencil, by loader id.
enum : int {
    RF_V0 = 0, RF_V1 = 1, RF_V2 = 2, RF_Z = 3, RF_H = 4, RF_RHO = 5, RF_KAP = 6,
    RF_F0 = 7, RF_F1 = 8, RF_F2 = 9, RF_T = 10, RF_VIB0 = 11, RF_VIB1 = 12, RF_VIB2 = 13, RF_N = 14
};

// Adjoint (reverse-mode) arguments: lambda of the stage residuals (padded,
// interior cells) and the lambda arrays of the stencil's inputs (padded; null
// entries are not needed), indexed by the stencil's field ids (v0..v2, Z, H,
// rho, kappa, F0..F2, T, v_ib0..v_ib2).
struct AdjR {
    const double* R[5];
};
struct AdjIn {
    double* out[RF_N];
};
struct FluxAdj {
    double* lF[3];            // in: adjoint of the final fluxes (consumed, zeroed)
    double* lFt[3];           // scratch: total adjoint of each shifted flux
    const double* lb;         // in: adjoint of b (compact)
    double* lmom[3];          // out (+=): provisional momentum
    double* lrho_new;         // out (+=): density of the stage
    double* lrho_n;           // out (+=): density at level n
    double* lrho_prev;        // out (+=): density at level n-1 (BDF2 only)
    double* lSm;              // out (+=): mass source (may be null)
    double bdf_c0, bdf_c1, bdf_c2, bdf_den;
    const double* sc;
    double* part;
};
struct ProjAdj {
    const double* lv[3];      // in: adjoint of the projected velocity (interior)
    const double* lF[3];      // in: adjoint of the final fluxes
    const double* P;          // forward pressure (compact)
    const double* mom[3];     // forward provisional momentum
    const double* T;          // forward temperature of the stage
    const double* sc;
    int p0_slot;
    double* lmom[3];          // out (+=)
    double* lT;               // out (+=)
    double* lP;               // out (=, compact)
    double eA, eB, eC;
};
struct CombAdj {
    const double* lmom[3];    // in: adjoint of the stage's momentum output
    const double* lZin;       // in: adjoint of the stage's Z output
    const double* lHin;
    double* lR[5];            // out (=): adjoint of the stage's residual
    double* lRh[5];           // in/out: adjoint of the stored level-n residual
    double* lv[3];            // out: adjoint of v^n (= in the corrector, += in the predictor)
    double* lZ;               // out (+=, predictor only): adjoint of Z^n
    double* lH;
    double* lrho_n;           // out (+=)
    const double* rho_n;      // forward rho^n
    const double* v_n[3];     // forward v^n
    double dt;
    int mode;
};
void launch_ghost(const Geom& g, const Bnd& bnd, const Phys& ph, const GhostJob& job, cudaStream_t s,
                  int* launches);
// bnd / kap_ghosts (optional): ghost-fill kappa in the same kernel.
void launch_state(const Geom& g, const Phys& ph, const double* Z, const double* H, double* T,
                  double* rho, double* kap, double* sc, int p0_slot, double* part, int* status,
                  cudaStream_t s, int* launches, const Bnd* bnd = nullptr, bool kap_ghosts = false);
void launch_residual(const Geom& g, const Phys& ph, const ResidArgs& a, cudaStream_t s, int* launches);
void launch_flux_rhs(const Geom& g, const Phys& ph, const Bnd& bnd, const FluxArgs& a, cudaStream_t s,
                     int* launches);
// Open systems (p0 = 1, a.correct): state relation + face fluxes in one kernel,
// then the right-hand side; the same results as launch_state + launch_flux_rhs.
void launch_state_flux_rhs(const Geom& g, const Phys& ph, const double* Z, const double* H, double* T, double* rho,
                           double* kap, double* sc, int* status, const Bnd& bnd, bool kap_ghosts,
                           const FluxArgs& a, cudaStream_t s, int* launches);
void launch_project(const Geom& g, const Phys& ph, const ProjArgs& a, cudaStream_t s, int* launches);
void launch_momentum(const Geom& g, const double* rho, double* const v[3], double* mom[3], cudaStream_t s,
                     int* launches);
void launch_sum(const Geom& g, const double* x, double* part, cudaStream_t s, int* launches);
struct FFSrc {
    const double* f[6];
};
// Float-float images of a stage's stencil inputs (padded, ghosts included):
// dst plane f (npad float2) = the (hi, lo) split of src[f], f = v0, v1, v2,
// Z, H, kappa (src[2] unused in 2D).
void launch_ff_images(const Geom& g, const double* const src[6], float2* dst, cudaStream_t s, int* launches);
// Semi-enclosed system: G of Eq 2.38 on one level's fields (padded, ghosts
// filled; v[d] for d < dim) and the stage update of p0 it feeds: stage 0 the
// predictor's Euler step (step 0), 1 its AB2 step, 2 the corrector's AM2 step.
// Writes p0 (and 1/p0) into out_slot; part holds 2 * reduce_grid(g) doubles.
enum { ODE_PRED_EULER = 0, ODE_PRED_AB2 = 1, ODE_CORR = 2 };
void launch_p0_ode(const Geom& g, const Phys& ph, const double* Z, const double* H, const double* kap,
                   double* const* v, double* part, double* sc, int stage, double dt, int out_slot, cudaStream_t s,
                   int* launches);
void launch_store_sum(const double* part, int np, double scale, double* dst, cudaStream_t s, int* launches);
void launch_copy_scalar(const double* src, double* dst, int n, cudaStream_t s, int* launches);
void launch_or_status(const int* src_flag, int bit, int* status, cudaStream_t s, int* launches);

// Member-batched stage kernels (a batch of simulations): one launch of a
// stage kernel covers every member, whatever its grid.  Each member keeps the
// block decomposition of its own launch (nblocks blocks); a work list of
// consecutive block ranges (start[m] .. start[m+1]) maps a block of the batched
// launch to its member and member-local block, so every member computes
// exactly what its own launch would (bitwise).  The members' arguments are
// records in device memory.
enum StageKind : int { SK_RESID = 0, SK_STATE_FLUX = 1, SK_RHS = 2, SK_PROJECT = 3, SK_COPY = 4, SK_IMAGES = 5,
                       SK_RESID_IMG = 6 };
struct StageSF {
    const double* Z;
    const double* H;
    double* T;
    double* rho;
    double* kap;
    int* status;
    double* sc;
    Bnd bnd;
    int kap_ghosts;
    FluxArgs fa;
};
struct StageCopy {
    const double* src;
    double* dst;
    long long n;
};
struct StageImg {
    FFSrc src;
    float2* dst;
    long long npad;
};
struct StageRec {
    Geom g;
    Phys ph;
    int kind;
    int nblocks;             // blocks of the member's own launch
    int np;                  // SK_RHS: partials of the mass balance
    union {
        ResidArgs r;
        StageSF sf;          // SK_STATE_FLUX and SK_RHS (FluxArgs, bnd)
        ProjArgs p;
        StageCopy cp;
        StageImg im;
    } u;
};
// Records collected instead of launched: while a collector is installed on the
// calling thread, launch_residual, launch_state_flux_rhs, launch_project and
// stage_copy append their member's record (SK_STATE_FLUX then SK_RHS for the
// state relation with the right-hand side) and launch nothing.
struct StageCollector {
    StageRec* recs;
    int n, cap;
    bool overflow;
};
void set_stage_collector(StageCollector* c);
// True while a collector is installed on the calling thread.
bool stage_collecting();
// D2D copy of n doubles as a step element (collected like the kernels).
cudaError_t stage_copy(const double* src, double* dst, long long n, cudaStream_t s);
// One batched launch of kind k over nm members: recs[m] (device), start[m]
// the first block of member m (start[nm] = total blocks, device and host
// copies), dim and mixed as for the members' own launches.
cudaError_t launch_stage_batched(int kind, int dim, int mixed, const StageRec* recs, const int* start,
                                 int nm, int total_blocks, cudaStream_t s);

// Immersed body and boundary kinds (set-up time).
struct IbmDev {
    int kind;
    double c[3], half[3], radius, s, rho_b, U_b;
    const double* profile;  // device copy (may be null)
    int n_profile;
    // marker body (kind 3): rows (x[dim], n[dim], U, A), device copy valid
    // during set-up only; bounding box of the positions widened by 2 s
    const double* mk;
    int n_mk;
    double bb_lo[3], bb_hi[3];
};
void launch_ibm(const Geom& g, const IbmDev& b, uint8_t* chi, double* vib[3], double* U, double* Sm,
                cudaStream_t s);
// Marker body, in two parts around the host's check that every marker has a
// masked cell: nearest marker, mask and v_ib of every padded cell plus the
// per-marker counts of masked interior cells (counts zeroed by the caller);
// then S_m from the counts.
void launch_marker_cells(const Geom& g, const IbmDev& b, uint8_t* chi, double* vib[3], double* U, double* Sm,
                         int* near, int* counts, cudaStream_t s);
void launch_marker_source(const Geom& g, const IbmDev& b, const uint8_t* chi, const int* near, const int* counts,
                          double* Sm, cudaStream_t s);
void launch_bkinds(const Geom& g, const int bc[3][2], const uint8_t* chi, uint8_t* kind[3][2],
                   double* part, double* sc, cudaStream_t s);

// Pack / unpack between the padded layout and compact interior / face arrays.
void launch_pack(const Geom& g, const double* padded, double* compact, int face_dir, cudaStream_t s);
void launch_unpack(const Geom& g, const double* compact, double* padded, cudaStream_t s);
void launch_u8_to_double(const Geom& g, const uint8_t* padded, double* compact, cudaStream_t s);
// Batched solves: nb device arrays of N doubles (src[k] / dst[k], device
// pointer tables) to and from one contiguous [nb][N] array.
void launch_gather(const double* const* src, double* dst, long long N, int nb, cudaStream_t s);
void launch_scatter(const double* src, double* const* dst, long long N, int nb, cudaStream_t s);
void launch_add_unpack(const Geom& g, const double* compact, double* padded, cudaStream_t s);

// Adjoint (reverse-mode) launchers; every one adds the adjoint of its forward
// kernel's inputs given the adjoint of its outputs.
// Stencil transpose: with cont (residual_rev_slots() padded arrays of
// scratch, 2D), the hand-written reverse sweep and its gather; with cont null,
// the exact dual-number gather (any dimension; the checker of the former).
void launch_residual_adj(const Geom& g, const Phys& ph, const ResidArgs& a, double p0dot, const AdjR& lr,
                         const AdjIn& li, double* cont, cudaStream_t s);
int residual_rev_slots();
void launch_ghost_adj(const Geom& g, const Bnd& bnd, const GhostJob& job, cudaStream_t s);
void launch_state_adj(const Geom& g, const Phys& ph, const double* Z, const double* T, const double* kap,
                      double* lT, double* lrho, double* lkap, double* lZ, double* lH, cudaStream_t s);
void launch_flux_adj(const Geom& g, const Bnd& bnd, const FluxAdj& a, cudaStream_t s);
void launch_project_adj(const Geom& g, const ProjAdj& a, cudaStream_t s);
void launch_comb_adj(const Geom& g, const CombAdj& a, cudaStream_t s);
void launch_objective(const Geom& g, const Phys& ph, const double* Z, const double* kap, double* part,
                      double* out, cudaStream_t s);
void launch_objective_adj(const Geom& g, const Phys& ph, const double* Z, const double* kap, double w, double* lZ,
                          double* lkap, cudaStream_t s);
void launch_profile_grad(const Geom& g, const IbmDev& b, const uint8_t* chi, const double* lvib1,
                         const double* lSm, double* col, double* grad, cudaStream_t s);

int reduce_grid(const Geom& g);

}  // namespace lm
