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

struct MgLevel {
    int n[3];
    int periodic[3];
    double h[3], ih2[3];
    long long N;
    double* u;   // correction (level >= 1)
    double* f;   // right-hand side (level >= 1)
    double* r;   // residual scratch
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
    PS_NSCAL = 16
};
enum : int { PI_IT = 0, PI_DONE = 1, PI_NOCONV = 2, PI_ZERO = 3, PI_NINT = 8 };

struct PoissonPlan {
    int dim;
    int nlev;
    MgLevel lev[kMaxLevels];
    long long N;          // fine cells
    double* r;            // Krylov vectors on the fine level
    double* z;
    double* p;
    double* q;
    double* part0;        // partial sums
    double* part1;
    double* part2;
    double* scal;         // PS_* scalars
    int* ictl;            // PI_* integer control words
    double* Minv;         // dense inverse of the coarsest operator (+ J/N)
    long long Nc;
    double rtol;
    int max_iter;
    int launches;         // kernels enqueued by the last enqueue (host-side count)
};

// Level shapes and workspace bytes for a grid (no allocation).
size_t poisson_plan_bytes(int dim, const int n[3], const int periodic[3], int* nlev_out,
                          long long* Nc_out, const char** err);

// Carve a plan out of ws (256-byte aligned, >= poisson_plan_bytes) and compute
// the coarsest-level inverse on the host (returned in minv_host).  h is the
// fine spacing.
bool poisson_plan_init(PoissonPlan* pl, int dim, const int n[3], const double h[3],
                       const int periodic[3], double rtol, int max_iter, void* ws,
                       size_t ws_bytes, std::vector<double>* minv_host, const char** err);

// Copy the coarsest inverse into the plan's device buffer (synchronises s).
bool poisson_upload_coarse(PoissonPlan* pl, const std::vector<double>& minv_host, cudaStream_t s,
                           const char** err);

// Enqueue the pieces of a solve of L x = b - mean(b) (b, x: device arrays of N
// doubles; x holds the warm start).  The PCG loop body sets the conditional of
// a while node when graph_handle != 0 (the body is then being captured into
// that node's body graph); with graph_handle == 0 the loop is host-driven.
cudaError_t poisson_enqueue_prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s);
cudaError_t poisson_enqueue_ctrl_init(PoissonPlan* pl, cudaStream_t s, unsigned long long graph_handle,
                                      int use_graph);
cudaError_t poisson_enqueue_body(PoissonPlan* pl, double* x, cudaStream_t s,
                                 unsigned long long graph_handle);
cudaError_t poisson_enqueue_epilogue(PoissonPlan* pl, double* x, cudaStream_t s);
// Single kernels of the fine level for timing: 0 = one smoother colour,
// 1 = operator application + dot, 2 = residual + restriction to level 1.
cudaError_t poisson_launch_single(PoissonPlan* pl, int which, cudaStream_t s);
// Host-driven complete solve (prologue, body until done, epilogue).
cudaError_t poisson_solve_host_loop(PoissonPlan* pl, const double* b, double* x, cudaStream_t s);

}  // namespace lm
