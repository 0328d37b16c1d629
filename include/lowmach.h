/*
 * lowmach.h -- C ABI of the GB300 (sm_103a) implementation of one time step of
 * the low-Mach-number flame-sheet solver of Severino, Fachini, Gennaro,
 * Rodriguez & Souza, "Numerical method for strongly variable-density flows at
 * low Mach number: flame-sheet regularisation and a mass-flux immersed boundary
 * method" (arXiv 2603.01727).
 *
 * The method (paper Secs 2.4-3.6): zero-Mach-number reacting flow in the
 * Burke-Schumann limit with unknowns v, Z, H, P = p dt and p0(t); a
 * predictor (Adams-Bashforth 2) / corrector (Adams-Moulton 2) fractional step
 * (Eqs 3.1-3.19) on a collocated Cartesian grid with auxiliary interface mass
 * fluxes (Eqs 3.20-3.26); a Poisson equation for P per stage (Eqs 3.9, 3.17,
 * 3.24); Brinkman-penalised immersed bodies with a mass source (Eqs 3.29-3.33);
 * and the regularised flame-sheet state relation (Eqs 3.34-3.42).
 *
 * Conventions shared by every entry point
 *   - All floating-point data is IEEE binary64 unless stated otherwise.
 *   - Cell fields are x-fastest arrays of the interior cells only, n[0]*n[1]
 *     (2D) or n[0]*n[1]*n[2] (3D) entries: index i + n0*(j + n1*k).
 *     Interface (face) fields along direction d have n[d]+1 entries along d
 *     and n entries along the others, x fastest.
 *   - Device memory is never allocated by the library.  The caller passes one
 *     device workspace of at least sim_workspace_size() bytes (256-byte
 *     aligned) to sim_create and keeps it alive until sim_destroy.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  sim_step returns after enqueueing
 *     the work and checking the previous step's device status word.
 *   - Errors are returned as sim_status codes; nothing aborts or throws
 *     across the ABI; sim_last_error() gives a human-readable reason.
 */
#ifndef LOWMACH_H
#define LOWMACH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim sim_t;

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = -1,     /* invalid argument or unsupported configuration            */
    SIM_ENOMEM = -2,     /* workspace smaller than sim_workspace_size()              */
    SIM_ECUDA = -3,      /* a CUDA runtime call failed                               */
    SIM_ENOCONV = -4,    /* a Poisson solve hit poisson_max_iter before rtol         */
    SIM_ENAN = -5,       /* a non-finite value appeared in the state                 */
    SIM_EUNSTABLE = -6,  /* dt violates the explicit penalisation limit dt < Re Da_ib */
    SIM_ESTATE = -7      /* call out of order (e.g. step before the fields are set)  */
} sim_status;

/* Boundary kinds of a domain side (paper Sec. 3.6, Eqs 3.43-3.46). */
enum {
    SIM_BC_PERIODIC = 0, /* Eq 3.45; both sides of a direction must be periodic       */
    SIM_BC_INFLOW = 1,   /* Dirichlet v, Z, H (Eq 3.43); known mass flux rho_in v_in  */
    SIM_BC_OUTFLOW = 2,  /* zero-gradient v, Z, H (Eq 3.44); extrapolated mass flux,
                            shifted uniformly to close the global mass balance
                            (text after Eq 4.22)                                      */
    SIM_BC_WALL = 3,     /* no-slip v = 0, zero-gradient Z, H, zero mass flux        */
    SIM_BC_SLIP = 4,     /* symmetry plane (Eqs 4.22a-b): v_n = 0, zero-gradient rest */
    SIM_BC_WALL_T = 5    /* isothermal no-slip wall (Eq 4.16a-b): v = 0, Dirichlet
                            Z = inflow_Z and H = wall_H of the side, zero mass flux */
};

enum { SIM_FP64 = 0, SIM_MIXED = 1 };
enum { SIM_IBM_NONE = 0, SIM_IBM_SLOT = 1, SIM_IBM_SPHERE = 2, SIM_IBM_MARKERS = 3, SIM_IBM_COUETTE = 4 };

/* Run parameters (paper notation, Eqs 2.42-2.50). */
typedef struct {
    int dim;                 /* 2 or 3                                                  */
    int n[3];                /* interior cells per direction (n[2] ignored in 2D)       */
    double L[3];             /* domain lengths; uniform spacing h_d = L_d / n_d         */
    int bc[3][2];            /* SIM_BC_* of the low / high side of each direction       */
    double inflow_v[3];      /* Dirichlet velocity of SIM_BC_INFLOW sides               */
    double inflow_Z;         /* Dirichlet rescaled mixture fraction of inflow sides     */
    double inflow_H;         /* Dirichlet excess enthalpy of inflow sides               */
    double Re, Pr;           /* Reynolds (Re = Pe/Pr) and Prandtl numbers               */
    double inv_Fr2;          /* 1/Fr^2 of the buoyancy term (Eq 3.8b)                   */
    double Le_F, Le_O;       /* fuel / oxidiser Lewis numbers (Eq 3.35)                 */
    double gamma;            /* ratio of specific heats (zeta, text after Eq 2.45)      */
    double sigma;            /* transport exponent, kappa = T^sigma (Eq 2.50)           */
    int transport;           /* 0: kappa = T^sigma; 1: Sutherland's law
                                kappa = T^(3/2) (1 + C) / (T + C) (Eq 4.12)             */
    double sutherland_C;     /* C of Sutherland's law (its constant over the
                                reference temperature, e.g. 110.5 K / 600 K)            */
    double wall_H[3][2];     /* Dirichlet H of SIM_BC_WALL_T sides [direction][side]   */
    double Z_st;             /* stoichiometric conventional mixture fraction: S = 1/Z_st - 1 */
    double density_ratio;    /* flame / ambient temperature: Q = (ratio - 1)(S + 1)     */
    double eps_reg, tol_reg; /* regularisation: k = ln((1-tol)/tol) / (2 eps) (Eq 3.34)  */
    int closed_system;       /* 0: open, p0 = 1 (Eq 2.41); 1: enclosed, p0 from the mass
                                constraint (Eq 2.40), no inflow or outflow sides;
                                2: semi-enclosed, p0 advanced by the ODE of Eq 2.38
                                (AB2 predictor, AM2 corrector), inflow sides allowed,
                                no outflow sides and no immersed body               */
    int incompressible;      /* 1: T = rho = kappa = p0 = 1 (constant-density runs)     */
    double dt;               /* fixed time step (> 0)                                   */
    int precision;           /* SIM_FP64: every kernel in FP64.  SIM_MIXED: the stage
                                stencil in float-float arithmetic (pairs of FP32,
                                about 48 bits) with FP64 residual storage and state
                                updates; the multigrid preconditioner and the CG
                                iteration in FP32 with a reliable update of the FP64
                                solution and residual every iteration (the stopping
                                test stays FP64); the state relation FP64-accurate,
                                FP64 near stoichiometry                                */
    double poisson_rtol;     /* stop when ||r||_2 / ||f||_2 <= rtol (0 < rtol < 1)      */
    int poisson_max_iter;    /* PCG iteration cap (>= 1)                                */
    /* Multigrid tuning (0 = library default): red-black sweeps per pre / post
     * smoothing of the 2D fused kernels (1 or 2), and the largest level (cells)
     * handled by the one-block coarse solve.  Results depend on them only
     * through the iteration count (the stopping test is unchanged). */
    int mg_sweeps;
    int mg_tail_cells;
    /* Cell tile of a block in the projection kernel: 0 = 256 consecutive
     * interior cells (x fastest); otherwise the x extent TX of a TX x (256/TX)
     * tile of cells (x by rows of y, z), TX one of 8, 16, 32, 64, 128, 256.
     * Results do not depend on it (the kernel is cell-local); it sets the
     * blocks' reuse of P's neighbours. */
    int stage_tile_x;
} sim_params_t;

/* Immersed burner (paper Sec. 3.4; Eqs 3.30-3.33, 4.19-4.21).  The mask is the
 * set of cells whose centre lies within sqrt(Da_ib) of the body (shifted
 * characteristic function).  SLOT: box [center-half, center+half] ejecting
 * through its +x_2 face with U(x_1) = U_b [1 - ((x_1-c_1)/(half_1+s))^2]_+ times
 * the piecewise-linear interpolant of profile[0..n_profile-1] sampled uniformly
 * over the shifted width (profile may be NULL); v_ib = (0, U (x_2-y_lo)/(y_hi-y_lo)),
 * S_m = rho_b U / (n_col h_2) on the n_col masked cells of each column.
 * SPHERE (circle in 2D): v_ib = U_b (x-c)/r, S_m = (dim-1) rho_b U_b / r.
 * MARKERS: a body given by n_markers surface markers, row m of `markers`
 * being (x[dim], n[dim], U, A): position, unit outward normal, normal ejection
 * speed and surface element (arc length in 2D, area in 3D).  Every cell centre
 * p is matched with its nearest marker (least |p - x_m|^2, lowest index on a
 * tie); p is in the shifted body iff (p - x_m).n_m <= sqrt(Da_ib), and there
 * v_ib = U_m n_m.  Cells outside the markers' bounding box widened by
 * 2 sqrt(Da_ib) are outside.  Marker m's flow rho_b U_m A_m is spread
 * uniformly over the N_m masked interior cells matched with it,
 * S_m = rho_b U_m A_m / (N_m dV); SIM_EINVAL if some N_m = 0 (markers denser
 * than the cells) or if 2 dim + 2 times n_markers exceeds the padded cell
 * count.  center, half, radius, U_b and the profile are unused.
 * COUETTE (the Taylor-Couette flow of Sec. 4.2.3): coaxial cylinders along
 * x_3 through center, inner radius R_1 = radius turning rigidly with surface
 * speed U_b (counter-clockwise about +x_3), outer radius R_2 = half[0] at
 * rest; with r the distance in the x_1-x_2 plane, the mask is r - R_1 <= s or
 * R_2 - r <= s (s = sqrt(Da_ib)), v_ib = (U_b/R_1)(-(x_2-c_2), x_1-c_1) in the
 * inner body and 0 in the outer, S_m = 0.  SIM_EINVAL unless
 * 0 < radius < half[0]. */
typedef struct {
    int kind;                /* SIM_IBM_*                                              */
    double center[3];
    double half[3];          /* SLOT half-sizes; COUETTE: half[0] = outer radius R_2    */
    double radius;           /* SPHERE radius; COUETTE: inner radius R_1               */
    double Da_ib;            /* immersed-boundary Darcy number (> 0)                   */
    double rho_b, U_b;       /* ejected density and velocity scale                     */
    double Z_ib, H_ib;       /* body targets in the paper's variables (Eq 4.21)        */
    int n_profile;           /* number of profile samples (0: none)                    */
    const double *profile;   /* host pointer, copied during the call                   */
    int n_markers;           /* MARKERS: number of markers                             */
    const double *markers;   /* MARKERS: host pointer to n_markers rows of 2 dim + 2
                                doubles, copied during the call                        */
} sim_ibm_t;

/* Field identifiers for sim_fields. */
enum {
    SIM_FIELD_U = 0, SIM_FIELD_V = 1, SIM_FIELD_W = 2,   /* velocity components        */
    SIM_FIELD_Z = 3, SIM_FIELD_H = 4,                     /* transported scalars        */
    SIM_FIELD_T = 5, SIM_FIELD_RHO = 6,                   /* state relation outputs     */
    SIM_FIELD_P = 7,                                      /* P = p dt, zero mean        */
    SIM_FIELD_FX = 8, SIM_FIELD_FY = 9, SIM_FIELD_FZ = 10,/* interface mass fluxes (faces) */
    SIM_FIELD_CHI = 11,                                   /* mask (0/1 as double)       */
    SIM_FIELD_SM = 12,                                    /* mass source S_m            */
    SIM_FIELD_KAPPA = 13
};
enum { SIM_GET = 0, SIM_SET = 1 };

/* Scalars for sim_query. */
enum {
    SIM_Q_TIME = 0, SIM_Q_DT = 1, SIM_Q_P0 = 2, SIM_Q_STEPS = 3,
    SIM_Q_ITERS_PRED = 4, SIM_Q_ITERS_CORR = 5,     /* PCG iterations of the last step */
    SIM_Q_RESID_PRED = 6, SIM_Q_RESID_CORR = 7,     /* final ||r||/||f|| of the last step */
    SIM_Q_MASS = 8, SIM_Q_NCELLS = 9, SIM_Q_MG_LEVELS = 10,
    SIM_Q_KERNEL_LAUNCHES = 11,                     /* kernels enqueued by the last sim_step */
    SIM_Q_TAIL_NX = 12, SIM_Q_TAIL_NY = 13,         /* shape of the top coarse level solved in one block */
    SIM_Q_TAIL_FDM = 14,                            /* 1: that level is solved by fast diagonalisation */
    SIM_Q_TAIL_NZ = 15,                             /* its z extent (1 in 2D) */
    /* Per-step checks of the last completed step, computed on demand from the
     * state (one pass over the grid; SIM_ESTATE before the first step):     */
    SIM_Q_DIV_RESID = 16,     /* max |d_t rho + sum_j delta_1 F_j / delta_1 x_j - S_m|
                                 over the cells: the discrete continuity of Eq 3.24
                                 with the mass source of Eq 3.33, d_t rho by the
                                 step's own rule (Eq 3.19; first order on step 1);
                                 bounded by the pressure solve's residual        */
    SIM_Q_DIV_SCALE = 17,     /* max |d_t rho| + max |S_m|: a scale for the above */
    SIM_Q_MASS_BALANCE = 18,  /* sum (d_t rho - S_m) dV + net outward flux of F
                                 through the domain boundary: the global mass
                                 balance closed by the outflow correction (text
                                 after Eq 4.22); zero up to rounding            */
    SIM_Q_PC_DIFF_U = 19,     /* L2 norms, sqrt(sum e^2 dV), of the difference  */
    SIM_Q_PC_DIFF_V = 20,     /* between the predicted and corrected velocity   */
    SIM_Q_PC_DIFF_W = 21,     /* components and P (P after removing the mean of  */
    SIM_Q_PC_DIFF_P = 22      /* the difference): the local truncation error
                                 measure of Sec. 4.2.2 (Table 2)                */
};

/* Bytes of device workspace sim_create needs for these parameters. */
sim_status sim_workspace_size(const sim_params_t *prm, size_t *bytes);

/* Validate prm, derive S, Q, k, Pe, zeta, N_F, N_O (paper Eqs 2.34-2.37, 3.34),
 * lay out every device array inside d_workspace and build the multigrid
 * hierarchy of the pressure solver.  No body until sim_set_ibm_geometry; no
 * state until the fields U, V, (W,) Z, H are set with sim_fields. */
sim_status sim_create(const sim_params_t *prm, void *d_workspace, size_t workspace_bytes,
                      void *cuda_stream, sim_t **out);

/* Set (or with geo == NULL / kind == SIM_IBM_NONE, clear) the immersed body:
 * computes chi, v_ib and S_m on the device (paper Sec. 3.4).  Returns
 * SIM_EUNSTABLE if dt >= Re Da_ib (explicit penalisation limit, text after
 * Eq 3.30).  Must precede the first sim_step after the fields are set. */
sim_status sim_set_ibm_geometry(sim_t *sim, const sim_ibm_t *geo);

/* Copy a field between the library and buf (interior cells / faces, layout
 * above).  dir = SIM_GET copies out, SIM_SET copies in (only U, V, W, Z, H may
 * be set; setting them starts a new run at t = 0 from those fields: T, rho,
 * kappa, F^0 and the mass are derived at the next sim_step).  on_device = 1:
 * buf is a device pointer, else a host pointer.  Synchronous with respect to
 * the host for on_device = 0. */
sim_status sim_fields(sim_t *sim, int field_id, void *buf, int dir, int on_device);

/* Advance nsteps time steps (predictor + corrector each, Eqs 3.1-3.19).  The
 * first step of a run uses Euler in the predictor (text after Eq 3.19). */
sim_status sim_step(sim_t *sim, int nsteps);

/* Wait for the enqueued work and return the device status: SIM_ENOCONV if a
 * Poisson solve did not reach rtol, SIM_ENAN if a non-finite value appeared. */
sim_status sim_sync(sim_t *sim);

/* Read one scalar (SIM_Q_*); synchronises the stream. */
sim_status sim_query(sim_t *sim, int what, double *out);

/* Restart state (checkpoint / resume): every array and scalar the next step
 * reads -- v, Z, H, T, kappa, rho^n and rho^(n-1), the interface fluxes F^n, the
 * stored residuals of the last predictor, P, p0 history, mass, step counter and
 * time -- in one opaque little-endian blob of sim_state_size() bytes with a
 * header that identifies the grid.  save copies the blob out (synchronises);
 * load copies it in and the next sim_step continues from it exactly as if the
 * run had never stopped (SIM_EINVAL if the header does not match this grid).
 * buf is a device pointer when on_device = 1, else a host pointer.  The
 * blob's body is one contiguous image of the workspace's state arrays, so it
 * moves in one copy (fastest from pinned host memory); both calls return once
 * a host buffer may be reused.  Blob format version 2: a 256-byte-aligned
 * header, then the segments in this order, each padded to 256 bytes: Z, H, T,
 * kappa, rho (three levels), the stored residuals of the last two steps (the
 * arrays final after the corrector's state relation, first), then v, F, P,
 * the scalars and the status words.  Blobs of version 1 (v and F first) are
 * refused with SIM_EINVAL. */
sim_status sim_state_size(const sim_t *sim, size_t *bytes);
sim_status sim_state_save(sim_t *sim, void *buf, int on_device);
sim_status sim_state_load(sim_t *sim, const void *buf, int on_device);
/* One step (sim_step(sim, 1)) whose restart blob -- the state after the step,
 * as sim_state_save writes it -- goes to buf while the step runs: the arrays
 * that are final once the corrector's state relation has run (Z, H, T,
 * kappa, rho, the stored residuals) are copied on a private stream during the
 * corrector's pressure solve, the rest after the step.  buf as for
 * sim_state_save (sim_state_size() bytes); synchronises.  On every return,
 * an error included, both copies have finished, so the caller may free or
 * reuse buf at once. */
sim_status sim_step_save(sim_t *sim, void *buf, int on_device);

/* Kernel timing support: enqueue `reps` back-to-back launches of one kernel of
 * the next step with that step's arguments (no synchronisation), so a caller
 * can bracket them with CUDA events on the stream.  Only scratch of the step is
 * written (stage temporaries, Krylov and multigrid vectors), never the state.
 * kernel: SIM_K_* below.  Returns SIM_ESTATE before the first step. */
enum {
    SIM_K_RESIDUAL = 0,   /* predictor stencil pass (residuals + AB2 update)             */
    SIM_K_MG_DOWN = 1,    /* fine level: red, black, residual, restriction (one kernel)  */
    SIM_K_CG_MATVEC = 2,  /* CG direction update + operator application + dot product   */
    SIM_K_MG_UP = 3,      /* fine level: prolongation-add, black, red (one kernel)        */
    SIM_K_STATE = 4,      /* flame-sheet state relation                                  */
    SIM_K_PROJECT = 5,    /* interface fluxes + cell velocities (projection)             */
    SIM_K_MG_TAIL = 6,    /* coarse multigrid levels in one thread block                 */
    SIM_K_RESIDUAL_REV = 7 /* adjoint: reverse stencil sweep + gather (after
                              sim_adjoint_begin; adds into the adjoint state)            */
};
sim_status sim_time_kernel(sim_t *sim, int kernel, int reps);

/* Reason of the last failing call on this handle (static storage of the handle). */
const char *sim_last_error(const sim_t *sim);

void sim_destroy(sim_t *sim);

/* ---------------------------------------------------------------------------
 * Heat-release objective and the discrete adjoint of the time step.
 * The paper has no adjoint; this is the exact transpose (reverse mode) of the
 * step as discretised here (Eqs 3.1-3.19, 3.20-3.28, 3.30-3.33, 3.41-3.42).
 *   objective: *out = sum over interior cells of omega dV at the current level,
 *            omega = (Q/S)(k/2) sech^2(k (Z - 1)) kappa |delta_2 Z|^2 / Pe, the
 *            heat-release rate of the flame sheet for Le = 1 (-Q/(S+1) F_eps''(Z)
 *            kappa |grad Z|^2 / Pe from Eqs 2.30 and 3.41).  Host out; synchronous.
 *   adjoint_workspace_size / begin: device memory (caller-owned, 256-byte
 *            aligned, live until end) for the adjoint state lambda and the
 *            recomputed step's values.  begin zeroes lambda and the accumulated
 *            forcing adjoints.  Supported: dim 2, SIM_FP64, open system, no
 *            incompressible switch (SIM_EINVAL else); Le_F != Le_O and
 *            inv_Fr2 != 0 transpose the stage stencil by its exact
 *            dual-number gather.
 *   adjoint_step: the simulation must hold the state of some level n (e.g. from
 *            sim_state_load).  Recomputes step n (the simulation ends at level
 *            n+1), adds objective_weight * d(objective at n+1)/d(state n+1) to
 *            lambda, and transposes step n: lambda becomes the adjoint of the
 *            level-n state, and the adjoints of v_ib and S_m are accumulated.
 *            Call it for n = N-1, ..., 0 with the matching states to get the
 *            gradient of sum_n w_n objective(n) + <seed, state N>.  dJ_dprofile
 *            (host, n_profile doubles, or NULL) receives the gradient with
 *            respect to the slot's profile samples accumulated so far (slot body
 *            with a profile only).  Synchronous; SIM_ENOCONV if a transposed
 *            pressure solve did not converge.
 *   adjoint_field: dir = SIM_GET copies the adjoint of a state field at the
 *            current level to host buf (interior cells, or faces for FX / FY;
 *            SIM_FIELD_SM: the accumulated adjoint of S_m); SIM_SET adds host
 *            buf to it (cell fields U, V, Z, H, T, RHO, KAPPA: a seed).
 * ------------------------------------------------------------------------- */
sim_status sim_objective(sim_t *sim, double *out);
sim_status sim_adjoint_workspace_size(const sim_t *sim, size_t *bytes);
sim_status sim_adjoint_begin(sim_t *sim, void *d_workspace, size_t workspace_bytes);
sim_status sim_adjoint_step(sim_t *sim, double objective_weight, double *dJ_dprofile);
sim_status sim_adjoint_field(sim_t *sim, int field_id, double *buf, int dir);
sim_status sim_adjoint_end(sim_t *sim);

/* ---------------------------------------------------------------------------
 * Batches of independent simulations (many flames, e.g. of uneven grid sizes).
 * One CUDA graph per step holds every simulation's whole step as an
 * independent branch (forked streams at capture), so their latency-bound
 * kernel chains run concurrently on the GPU.  The paper has no counterpart:
 * each simulation is the paper's step unchanged; only the launching differs.
 *   create:  sims (host array of n distinct handles, n >= 1) is copied; the
 *            simulations stay owned by the caller and must outlive the batch.
 *            Work is enqueued on cuda_stream.
 *   step:    advances every simulation nsteps steps; the first two steps of a
 *            run go through each simulation's own launch path, later ones one
 *            batch graph launch per step.  The simulations must be in lockstep
 *            (SIM_ESTATE otherwise).  Do not call a member simulation's own
 *            functions while a batch step may be in flight: sim_batch_sync first.
 *   sync:    waits and returns the first failing member's device status.
 * ------------------------------------------------------------------------- */
typedef struct sim_batch sim_batch_t;
/* Batched pressure solves.  Members with the same 2D grid, spacing, sides
 * and solver settings form a group whose two solves per step run as one
 * batched solve (sim_poisson_solve_batch's kernels: one launch per multigrid
 * level and CG update for the whole group), with bitwise the results of
 * their own solves.  That needs a device workspace of
 * sim_batch_workspace_size bytes (caller-owned, 256-byte aligned, live until
 * destroy); with d_workspace NULL every member keeps its own solves.
 * query_launches (after sync): kernels the last batch step launched. */
sim_status sim_batch_workspace_size(sim_t *const *sims, int n, size_t *bytes);
sim_status sim_batch_create(sim_t *const *sims, int n, void *d_workspace, size_t workspace_bytes,
                            void *cuda_stream, sim_batch_t **out);
sim_status sim_batch_query_launches(sim_batch_t *batch, double *out);
sim_status sim_batch_step(sim_batch_t *batch, int nsteps);
sim_status sim_batch_sync(sim_batch_t *batch);
const char *sim_batch_last_error(const sim_batch_t *batch);
void sim_batch_destroy(sim_batch_t *batch);

/* ---------------------------------------------------------------------------
 * Stand-alone pressure solve (the step's dominant kernel, paper Eqs 3.9/3.24):
 * zero-mean P with sum_d delta_1(delta_1 P/delta_1 x_d)/delta_1 x_d = b - mean(b)
 * on a uniform grid; periodic[d] != 0 selects a periodic direction, else
 * homogeneous Neumann (known boundary mass flux, Sec. 3.3).  Multigrid-
 * preconditioned conjugate gradients to ||r||_2/||f||_2 <= rtol; P holds the
 * warm start on entry.  d_b and d_P are device arrays of n0*n1(*n2) doubles.
 * The workspace (device, >= sim_poisson_workspace_size bytes, 256-byte
 * aligned) holds the multigrid hierarchy and the Krylov vectors.  iters and
 * rel_resid (host pointers, may be NULL) receive the iteration count and the
 * final relative residual; the call synchronises the stream.
 * Returns SIM_ENOCONV if max_iter was reached first.
 * ------------------------------------------------------------------------- */
sim_status sim_poisson_workspace_size(int dim, const int n[3], const int periodic[3],
                                      size_t *bytes);
sim_status sim_poisson_solve(int dim, const int n[3], const double h[3], const int periodic[3],
                             const double *d_b, double *d_P, double rtol, int max_iter,
                             void *d_workspace, size_t workspace_bytes, void *cuda_stream,
                             int *iters, double *rel_resid);

/* Batched stand-alone pressure solve: nb independent systems on the same 2D
 * grid (periodic / Neumann sides as above), advanced together: one launch per
 * multigrid level and CG update serves every system, with per-system
 * scalars, convergence test and iteration count; a system that has converged
 * stops updating while the others continue.  d_b and d_P hold nb consecutive
 * n0*n1 arrays (system k at offset k*n0*n1).  precision: SIM_FP64 (FP64
 * multigrid) or SIM_MIXED (FP32 multigrid and inner CG with FP64 reliable
 * updates, as in sim_params_t).  Each system gets the same iterates it would
 * get solved alone.  iters (nb ints) and rel_resid (nb doubles), host
 * pointers that may be NULL, receive the per-system results; the call
 * synchronises the stream.  Returns SIM_EINVAL for nb < 1, a 3D grid or a grid
 * that does not coarsen, SIM_ENOCONV if some system reached max_iter first. */
sim_status sim_poisson_batch_workspace_size(const int n[2], const int periodic[2], int nb, int precision,
                                            size_t *bytes);
sim_status sim_poisson_solve_batch(const int n[2], const double h[2], const int periodic[2], int nb,
                                   int precision, const double *d_b, double *d_P, double rtol, int max_iter,
                                   void *d_workspace, size_t workspace_bytes, void *cuda_stream, int *iters,
                                   double *rel_resid);

/* ---------------------------------------------------------------------------
 * Pressure solve without any allocation (no counterpart in the paper; an
 * interface convenience).  Same operator, arguments, results and status codes
 * as sim_poisson_solve, minus the workspace: the scratch lives in one static
 * device array of SIM_NOALLOC_SCRATCH_BYTES inside this library, held on every
 * GPU that loads the library until the process exits.
 *
 * For callers that cannot call cudaMalloc or lend a workspace: a plug-in whose
 * host application owns all device memory, a process under a fixed device
 * memory budget, or a latency-critical loop that cannot take the implicit
 * device synchronisation of cudaMalloc / cudaFree.  The call itself allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * - The first call on a device looks up the array's device address with that
 *   device current (one-time set-up); make that first call before any stream
 *   capture on the device.  The address is kept for the life of the process,
 *   so cudaDeviceReset between calls is not supported: a reset reloads the
 *   module and the kept address would no longer name the array.
 * - Returns SIM_ENOMEM, before touching the GPU, when the grid needs more than
 *   SIM_NOALLOC_SCRATCH_BYTES of scratch (sim_poisson_workspace_size gives the
 *   need; about 40 bytes per cell, e.g. 2D grids up to roughly 400 000 cells).
 * - Every call shares the one array: the used part is cleared at the start of
 *   each call, and calls that overlap on the GPU (different streams, or other
 *   host threads) race on it -- serialise them.
 * - Synchronises cuda_stream before returning (like sim_poisson_solve).
 * ------------------------------------------------------------------------- */
#define SIM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
sim_status sim_poisson_solve_noalloc(int dim, const int n[3], const double h[3], const int periodic[3],
                                     const double *d_b, double *d_P, double rtol, int max_iter,
                                     void *cuda_stream, int *iters, double *rel_resid);

#ifdef __cplusplus
}
#endif
#endif /* LOWMACH_H */
