// Pressure Poisson solver of the projection (paper Eqs 3.9, 3.17, 3.24):
// multigrid-preconditioned conjugate gradients for the compact Laplacian on a
// uniform grid with periodic / homogeneous-Neumann sides, zero-mean solution.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "common.cuh"

namespace lm {

constexpr int kMaxLevels = 16;
constexpr long long kMaxCoarse = 1024;   // cells of the directly-solved coarsest level
constexpr long long kCoarsenAbove = 64;  // keep coarsening while a level has more cells

// Geometry and operator coefficients of one multigrid level, in the
// multigrid's arithmetic type T.  A = -L: (A u)_c = diag_c u_c - sum w_d u_nb.
// diag / invd are indexed by the neighbour-count class c_0 + 3 c_1 + 9 c_2,
// c_d in {0, 1, 2} = neighbours that exist along d (Neumann sides drop one).
template <class T>
struct LvT {
    int n[3];
    int per[3];
    int N;
    T w[3];
    T diag[27];
    T invd[27];
    DivU32 dn0, dn1;   // division by n[0], n[1] (compact index -> coordinates)
};

// Host view of a level: shape plus its device arrays.
struct MgLevel {
    int n[3];
    int periodic[3];
    long long N;
    double h[3], ih2[3];
    void* upre;   // pre-smoothed correction   (T, levels 1 .. top-1; level 0: plan u0pre)
    void* upost;  // post-smoothed correction  (T, levels 1 .. top; level top: tail output)
    void* f;      // right-hand side            (T, levels 1 .. top)
};

// Device scalars of one solve (indices into PoissonPlan::scal).
enum : int {
    PS_FF = 0,        // ||f||^2
    PS_RR = 1,        // ||r||^2 of the current iterate
    PS_RZ = 2,        // r.z of the current iteration
    PS_BETA = 3,
    PS_MEANZ = 4,
    PS_MEANB = 5,
    PS_ITERS = 6,     // iterations done (as a double, for reporting)
    PS_RELRES = 7,    // sqrt(rr/ff) at exit
    PS_ALPHA = 8,
    PS_MEANX = 9,
    PS_MEANR = 10,    // mean of the current CG residual (removed before the preconditioner)
    PS_NSCAL = 16
};
// PI_IT: CG iterations of the solve (its parity selects the search-direction
// buffer); PI_TOTAL: the same count for the iteration cap.
enum : int { PI_IT = 0, PI_DONE = 1, PI_NOCONV = 2, PI_ZERO = 3, PI_TOTAL = 5, PI_NINT = 8 };
constexpr int kNumCounters = 12;         // last-block counters (one per reducing kernel kind), barrier words

struct PoissonPlan {
    int dim;
    int nlev;
    int top;              // first level of the single-block tail (levels top .. nlev-1)
    int mg_fp32;          // 1: multigrid in FP32, else FP64
    int sweeps;           // red-black sweeps per pre / post smoothing (2D kernels)
    int mg3_tiles;        // 1: cube-tile 3D level kernels instead of the z-marching ones
    long long mg3_min_cells;  // 3D levels with fewer cells use the cube tiles
    int mg3_sweeps;       // 1: those levels on whole-level colour-sweep passes instead of z-marching
    int k3s_zc;           // consecutive planes per block of the colour-sweep passes
    MgLevel lev[kMaxLevels];
    long long N;          // fine cells
    double* r;            // FP64 Krylov vectors on the fine level
    double* p[2];         // search direction, double-buffered by iteration parity
    double* q;
    void* z;              // preconditioned residual (T)
    void* u0pre;          // pre-smoothed fine-level correction (T)
    // Refinement mode (mg_fp32): the CG's search direction, operator
    // application and preconditioner run in FP32; every iteration folds its
    // correction e = alpha p into the FP64 x, updates the FP64 residual
    // (r -= A e, float-float), replaces the FP32 residual with it and applies
    // the FP64 stopping test (a reliable update every iteration).
    float* r32;           // FP32 copy of the FP64 residual
    float* p32[2];        // search direction, double-buffered
    float* q32;
    double* part0;        // partial sums (npart entries each)
    double* part1;
    double* part2;
    int npart;
    double* scal;         // PS_* scalars
    int* ictl;            // PI_* integer control words
    unsigned int* cnt;    // last-block counters
    void* levtab;         // LvT<T>[nlev] on the device (tail)
    double* Minv;         // dense pseudo-inverse of the coarsest operator
    float* Minv_f;        // the same in FP32
    long long Nc;
    size_t tail_smem;     // dynamic shared memory of the tail kernel
    int tail_off_u[kMaxLevels], tail_off_f[kMaxLevels], tail_off_r;   // tail smem offsets (elements)
    double rtol;
    int max_iter;
    int launches;         // kernels enqueued by the last enqueue (host-side count)
    size_t levtab_bytes;
    unsigned char levtab_host[kMaxLevels * sizeof(LvT<double>)];   // host copy of levtab
    // fast-diagonalisation solve of the top coarse level (FP32 multigrid)
    int fdm;
    float* fdm_tab;       // S_x, S_x^T (nx x nx, eigenvectors as columns), S_y, S_y^T (ny x ny),
                          // [3D: S_z, S_z^T (nz x nz)], inverse eigenvalue sums (x fastest, 0 for
                          // the null mode)
    size_t fdm_tab_floats;
    size_t fdm_smem;
    // Batch of nb independent systems on the same grid (nb = 1: one system).
    // Every per-solve array above holds nb consecutive copies (vectors and
    // level arrays by their length, scal by PS_NSCAL, ictl by PI_NINT, cnt by
    // kNumCounters, partial sums by npart); the kernels take the system index
    // from one grid dimension.  bdone: 1 once every system has converged.
    int nb;
    int* bdone;
    int prefix;           // CG iterations a graph solve captures ahead of its while node
    // Persistent solve (one 2D system, FP32 multigrid with reliable updates,
    // fast-diagonalisation top level): the whole solve in one cooperative
    // launch of persist_grid blocks (all resident), phases separated by grid
    // barriers instead of kernel boundaries.
    int persist;
    int persist_grid;
    int pdl;              // 1: the solver's kernels launch with programmatic dependent launch
};

// Workspace bytes for a grid (no allocation).
// tail_cells (and sweeps below): multigrid tuning, 0 = default.
size_t poisson_plan_bytes(int dim, const int n[3], const int periodic[3], int mg_fp32, int tail_cells,
                          int* nlev_out, long long* Nc_out, const char** err);

// Carve a plan out of ws (256-byte aligned, >= poisson_plan_bytes) and compute
// the coarsest-level inverse and the level tables on the host; minv_host gets
// the coarse inverse followed (fast-diagonalisation plans) by S_x, S_x^T, S_y, S_y^T and the
// inverse eigenvalue sums.
bool poisson_plan_init(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                       int mg_fp32, int sweeps, int tail_cells, double rtol, int max_iter, void* ws,
                       size_t ws_bytes, std::vector<double>* minv_host, const char** err);

// The same for a batch of nb independent systems on one 2D grid (nb >= 1).
size_t poisson_plan_bytes_batch(int dim, const int n[3], const int periodic[3], int mg_fp32, int tail_cells, int nb,
                                int* nlev_out, long long* Nc_out, const char** err);
bool poisson_plan_init_batch(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                             int mg_fp32, int sweeps, int tail_cells, double rtol, int max_iter, int nb, void* ws,
                             size_t ws_bytes, std::vector<double>* minv_host, const char** err);

// Iterations a graph-captured solve runs ahead of its while node (0 for a
// batch or a one-level grid), and the while node's iterations for a solve of
// iters iterations.
int poisson_prefix_iters(const PoissonPlan* pl);
double poisson_loop_iters(const PoissonPlan* pl, double iters);

// Device flag a host-driven loop polls: 1 once the solve (every system of a
// batch) has finished.
const int* poisson_done_flag(const PoissonPlan* pl);

// Batches: copy each system's iteration count and final relative residual to
// rep[k][0..1] and OR status_bit into *status[k] when system k did not
// converge (rep, status: device arrays of nb device pointers).
cudaError_t poisson_enqueue_batch_report(PoissonPlan* pl, double* const* rep, int* const* status, int status_bit,
                                         cudaStream_t s);

// Copy the host-prepared tables into the plan's device buffers (synchronises s).
bool poisson_upload_coarse(PoissonPlan* pl, const std::vector<double>& minv_host, cudaStream_t s,
                           const char** err);

// Enqueue the pieces of a solve of L x = b - mean(b) (b, x: device arrays of N
// doubles; x holds the warm start).  The convergence test of the prologue and
// of each iteration sets the conditional of a while node when graph_handle != 0
// (the body is then being captured into that node's body graph); with
// graph_handle == 0 the loop is host-driven.
// mean_ready: mean(b) is already in the plan's scratch word (written by the
// kernel that formed b, through poisson_meanb_target), so no mean pass runs.
cudaError_t poisson_enqueue_prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s,
                                     unsigned long long graph_handle, int mean_ready);
// Where a kernel producing b can leave mean(b) for a single-system plan: its
// block partials, its last-block counter and the scratch word.
void poisson_meanb_target(PoissonPlan* pl, double** part, unsigned int** cnt, double** out);
cudaError_t poisson_enqueue_body(PoissonPlan* pl, double* x, cudaStream_t s, unsigned long long graph_handle);
// Zero-mean x (remove_mean; the solve itself keeps x's mean, since every
// correction is zero-mean, up to rounding); optionally report iterations /
// relative residual into rep[0], rep[1] and OR status_bit into *status on
// non-convergence.
cudaError_t poisson_enqueue_epilogue(PoissonPlan* pl, double* x, cudaStream_t s, double* rep, int* status,
                                     int status_bit, int remove_mean);
// x -= mean(x) on one system of the plan's grid (its scratch words).
cudaError_t poisson_enqueue_remove_mean(PoissonPlan* pl, double* x, cudaStream_t s);
// Single kernels for timing (scratch only): 0 = fine-level down sweep,
// 1 = CG direction update + operator application, 2 = fine-level up sweep,
// 3 = coarse-level tail.
cudaError_t poisson_launch_single(PoissonPlan* pl, int which, cudaStream_t s);
// Host-driven complete solve (prologue, body until done, epilogue).
// The whole solve of a persistent plan (pl->persist) in one cooperative launch
// (after a reset of its barrier words); mean_ready as for the prologue.  The
// epilogue is enqueued separately.
cudaError_t poisson_enqueue_persistent(PoissonPlan* pl, const double* b, double* x, cudaStream_t s, int mean_ready);
cudaError_t poisson_solve_host_loop(PoissonPlan* pl, const double* b, double* x, cudaStream_t s);

}  // namespace lm
