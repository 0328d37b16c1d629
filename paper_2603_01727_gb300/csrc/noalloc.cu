// Pressure solve that allocates nothing: the same multigrid-preconditioned CG
// as sim_poisson_solve, with its scratch (Krylov vectors, multigrid levels,
// partial sums, coarsest-level inverse) in one file-scope device array instead
// of a caller-provided workspace.
//
// Who needs it: callers that may not call cudaMalloc (or have no allocator to
// lend a workspace) -- a plug-in running inside a host application that owns
// all device memory and forbids side allocations, a process under a fixed
// device-memory budget, or a latency-critical loop that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree.
//
// The array is kNoAllocScratchBytes (SIM_NOALLOC_SCRATCH_BYTES) long and lives
// in every GPU that loads this library until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// shadow object), so the first call on each device looks the device address up
// with cudaGetSymbolAddress while that device is current and caches it.  The
// cache is never invalidated: a cudaDeviceReset between calls (which reloads
// the module) is not supported, as the header states.

#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lowmach.h"
#include "poisson.cuh"

using namespace lm;

namespace {

constexpr size_t kNoAllocScratchBytes = SIM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];   // device address of the array, per device ordinal

}  // namespace

static __device__ __align__(256) unsigned char g_poisson_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_poisson_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sim_status sim_poisson_solve_noalloc(int dim, const int n[3], const double h[3], const int periodic[3],
                                                const double* d_b, double* d_P, double rtol, int max_iter,
                                                void* cuda_stream, int* iters, double* rel_resid) {
    if (!n || !h || !periodic || !d_b || !d_P || (dim != 2 && dim != 3)) return SIM_EINVAL;
    if (!(rtol > 0.0 && rtol < 1.0) || max_iter < 1) return SIM_EINVAL;
    int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    double hh[3] = {h[0], h[1], dim == 3 ? h[2] : 1.0};
    int per[3] = {periodic[0] != 0, periodic[1] != 0, dim == 3 ? (periodic[2] != 0) : 0};
    for (int d = 0; d < dim; ++d)
        if (nn[d] < 2 || !(hh[d] > 0.0)) return SIM_EINVAL;
    const char* err = nullptr;
    const size_t need = poisson_plan_bytes(dim, nn, per, 0, 0, nullptr, nullptr, &err);
    if (need == 0) return SIM_EINVAL;
    if (need > kNoAllocScratchBytes) return SIM_ENOMEM;   // grid too large for the static scratch

    void* ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) return SIM_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents; start every call from zeros
    if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) return SIM_ECUDA;
    PoissonPlan pl;
    std::vector<double> minv;
    if (!poisson_plan_init(&pl, dim, nn, hh, per, 0, 0, 0, rtol, max_iter, ws, kNoAllocScratchBytes, &minv, &err))
        return SIM_EINVAL;
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
