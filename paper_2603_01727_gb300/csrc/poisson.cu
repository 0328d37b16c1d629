// Multigrid-preconditioned conjugate gradients for the pressure equation of
// the projection, L P = b - mean(b) with L = sum_d delta_1(delta_1 . / delta_1 x_d)
// / delta_1 x_d (paper Eqs 3.9, 3.17, 3.24; homogeneous Neumann on sides with a
// known boundary mass flux, Sec. 3.3; zero-mean solution selected as by the
// augmented-matrix method).  The paper solves this system with a sparse direct
// solver; here it is solved iteratively on the device:
//
//   A = -L (symmetric positive semi-definite, null space = constants);
//   CG on the mean-zero subspace in FP64, preconditioned by one symmetric
//   V-cycle in T = double or float: red-black Gauss-Seidel from a zero guess
//   (pre: red, black; post: black, red), cell-centred bilinear / trilinear
//   prolongation P and restriction R = P^T / 2^dim, the operator
//   re-discretised on every level, and an exact dense solve of the coarsest
//   level (pseudo-inverse through A_c + c 1 1^T).
//
// Kernel structure (one CG iteration):
//   fine levels   one "down" kernel per level: a tile of the level plus a
//                 3-cell halo in shared memory; red from zero, black, residual,
//                 restriction to the next level's right-hand side;
//                 one "up" kernel per level: tile plus a 2-cell halo;
//                 prolongation-add, black, red;
//   coarse levels one single-block "tail" kernel holding every level from
//                 `top` down in shared memory;
//   CG            direction update fused with the operator application
//                 (p double-buffered by iteration parity), then the x / r
//                 update with the convergence test.
// Every reduction is a fixed-order two-stage sum: block partials, then the
// last block to finish sums them in index order, so a solve is bitwise
// reproducible run to run.  The last block also writes the CG scalars and sets
// the while-node conditional.

#include <algorithm>
#include <climits>
#include <type_traits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "poisson.cuh"

namespace lm {

namespace {

// Programmatic dependent launch: every kernel of the solver is launched with
// programmatic stream serialisation, so the next kernel of the chain is
// scheduled while this one drains.  Each kernel therefore waits for its
// predecessor's completion (and memory flush) before touching global memory
// (pdl_wait, first statement), and lets its own successor launch at once
// (pdl_trigger).  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// PDL for the launches of the plan being enqueued (set by each entry point
// from the plan, on the enqueuing host thread).
thread_local bool g_pdl = true;

struct PdlScope {
    bool saved;
    explicit PdlScope(const PoissonPlan* pl) : saved(g_pdl) { g_pdl = pl->pdl != 0; }
    ~PdlScope() { g_pdl = saved; }
};

bool pdl_enabled() { return g_pdl; }

template <typename... KArgs, typename... Args>
void launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

constexpr int NTV = kThreads;            // block size of the pointwise kernels
constexpr int kTailThreads = 512;
constexpr long long kTailCellsF32 = 4096;   // largest level handled by the tail (FP32)
constexpr long long kTailCellsF64 = 128;    // (FP64: one SM's FP64 rate is 1/64 of FP32)
constexpr size_t kTailSmemMax = 200 * 1024;
constexpr long long kMg3MinCells = 1LL << 20;   // smallest 3D level on the z-marching kernels
constexpr long long kMg3SweepMinCells = 1LL << 17;   // ... on the colour-sweep passes

template <int DIM>
struct Tile;
template <>
struct Tile<2> {
    static constexpr int CX = 16, CY = 8, CZ = 1, NT = 256;
};
template <>
struct Tile<3> {
    static constexpr int CX = 8, CY = 4, CZ = 4, NT = 512;
};

// Fine tile of a block (twice the coarse tile) plus a halo of H cells.
template <int DIM, int H>
struct Box {
    static constexpr int FX = 2 * Tile<DIM>::CX, FY = 2 * Tile<DIM>::CY, FZ = (DIM == 3) ? 2 * Tile<DIM>::CZ : 1;
    static constexpr int SX = FX + 2 * H, SY = FY + 2 * H, SZ = (DIM == 3) ? FZ + 2 * H : 1;
    static constexpr int SN = SX * SY * SZ;
    static constexpr int S1 = SX, S2 = SX * SY;   // shared-memory strides of y and z
};

// Compact index -> coordinates of a level by its invariant-divisor
// multiplications (no integer division instruction sequence).
template <class LV>
__device__ __forceinline__ void coords(const LV& L, int t, int c[3]) {
    const unsigned r = divu32((unsigned)t, L.dn0);
    const unsigned k = divu32(r, L.dn1);
    c[0] = (int)((unsigned)t - r * (unsigned)L.n[0]);
    c[1] = (int)(r - k * (unsigned)L.n[1]);
    c[2] = (int)k;
}

__device__ __forceinline__ int wrapi(int g, int n) {
    const int m = g % n;
    return m < 0 ? m + n : m;
}

// Shared-memory cell s of a box with origin o (global coordinates, unwrapped):
// validity (inside the domain or periodic), compact global index (wrapped),
// neighbour-count class, ownership (inside the block's tile and the domain).
template <class T, int DIM>
__device__ __forceinline__ bool cell_info(const LvT<T>& L, const int o[3], const int s[3], int H, int F[3],
                                          int* gi, int* cl, bool* owned) {
    bool valid = true, own = true;
    int idx = 0, c = 0, stride = 1, p3 = 1;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int n = L.n[d];
        const int g = o[d] + s[d];
        int gw = g;
        const bool in = (g >= 0 && g < n);
        if (!in) {
            if (L.per[d]) gw = wrapi(g, n);
            else valid = false;
        }
        own = own && in && s[d] >= H && s[d] < H + F[d];
        idx += gw * stride;
        stride *= n;
        c += (L.per[d] ? 2 : (int)(gw > 0) + (int)(gw < n - 1)) * p3;
        p3 *= 3;
    }
    *gi = idx;
    *cl = c;
    *owned = own && valid;
    return valid;
}

template <class T, int DIM, class B>
__device__ __forceinline__ T off_box(const LvT<T>& L, const T* su, int i) {
    T off = L.w[0] * (su[i - 1] + su[i + 1]) + L.w[1] * (su[i - B::S1] + su[i + B::S1]);
    if (DIM == 3) off += L.w[2] * (su[i - B::S2] + su[i + B::S2]);
    return off;
}

// 1D weights of R = P^T / 2 (times 2) for coarse index I and offset a = 0..3
// (fine index 2I-1+a); Neumann ends drop the outside fine cell and give the
// end cell the reflected weight.
__device__ __forceinline__ float rweight(int a, int I, int Nc, int periodic) {
    float w = (a == 1 || a == 2) ? 0.75f : 0.25f;
    if (!periodic) {
        if (I == 0) {
            if (a == 0) w = 0.0f;
            if (a == 1) w = 1.0f;
        }
        if (I == Nc - 1) {
            if (a == 3) w = 0.0f;
            if (a == 2) w = 1.0f;
        }
    }
    return w;
}

// Coarse neighbour pair of fine index g (wrapped) for bilinear prolongation.
__device__ __forceinline__ void pro_pair(int g, int Nc, int per, int* I, int* J) {
    const int i = g >> 1;
    int j = (g & 1) ? i + 1 : i - 1;
    if (j < 0) j = per ? Nc - 1 : i;
    if (j >= Nc) j = per ? 0 : i;
    *I = i;
    *J = j;
}

template <class T, int DIM>
__device__ __forceinline__ T prolong_at(const LvT<T>& C, const T* __restrict__ uc, const int gw[3]) {
    int I[3] = {0, 0, 0}, J[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) pro_pair(gw[d], C.n[d], C.per[d], &I[d], &J[d]);
    const T a = (T)0.75, b = (T)0.25;
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    auto plane = [&](int k) {
        const int o = nxy * k;
        return a * (a * uc[I[0] + nx * I[1] + o] + b * uc[J[0] + nx * I[1] + o]) +
               b * (a * uc[I[0] + nx * J[1] + o] + b * uc[J[0] + nx * J[1] + o]);
    };
    if (DIM == 3) return a * plane(I[2]) + b * plane(J[2]);
    return plane(0);
}

// Last block of the whole grid to arrive (arrive_last_n, common.cuh, counts the
// blocks of one system of a batch on that system's counter).
__device__ __forceinline__ bool arrive_last(unsigned int* cnt) {
    return arrive_last_n(cnt, gridDim.x * gridDim.y * gridDim.z);
}

// Batches: the system of a block (grid dimension y of the vector kernels, z
// of the 2D level kernels) and the offsets of its control words.
__device__ __forceinline__ void batch_ctl(int fb, double** scal, int** ictl, unsigned int** cnt) {
    *scal += (long long)fb * PS_NSCAL;
    *ictl += (long long)fb * PI_NINT;
    *cnt += (long long)fb * kNumCounters;
}

template <int NT>
__device__ __forceinline__ double sum_parts_cg(const double* part, int np, double* smem) {
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += NT) v += __ldcg(part + i);
    return block_sum<NT>(v, smem);
}

// The same for two partial arrays of np entries in one pass.
template <int NT>
__device__ __forceinline__ void sum_parts2_cg(const double* pa, const double* pb, int np, double* smem2, double* A,
                                              double* B) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < np; i += NT) {
        a += __ldcg(pa + i);
        b += __ldcg(pb + i);
    }
    block_sum2_t<NT, double>(a, b, smem2);
    *A = a;
    *B = b;
}

__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ---------------------------------------------------------------------------
// down: red from zero, black, residual, restriction (one level)
// ---------------------------------------------------------------------------
template <class T, class TF, int DIM>
__global__ void __launch_bounds__(Tile<DIM>::NT) k_mg_down(LvT<T> L, LvT<T> C, const TF* __restrict__ f,
                                                           T* __restrict__ upre, T* __restrict__ fc,
                                                           const double* __restrict__ scal_r) {
    pdl_wait();
    pdl_trigger();
    // fine level: the CG residual enters the preconditioner with its mean removed
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    constexpr int H = 3;
    using B = Box<DIM, H>;
    constexpr int NT = Tile<DIM>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sf = reinterpret_cast<T*>(smraw);
    T* su = sf + B::SN;
    const int o[3] = {(int)blockIdx.x * B::FX - H, (int)blockIdx.y * B::FY - H,
                      (DIM == 3) ? (int)blockIdx.z * B::FZ - H : 0};
    int F[3] = {B::FX, B::FY, B::FZ};
    const int par0 = (o[0] + o[1] + o[2]) & 1;

    // load f on the whole box; red cells from a zero guess: u = f / diag
    for (int i = threadIdx.x; i < B::SN; i += NT) {
        const int s[3] = {i % B::SX, (i / B::SX) % B::SY, i / B::S2};
        int gi, cl;
        bool own;
        T fv = (T)0, uv = (T)0;
        if (cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) {
            fv = (T)(f[gi] - mr);
            if (((par0 + s[0] + s[1] + s[2]) & 1) == 0) uv = fv * L.invd[cl];
        }
        sf[i] = fv;
        su[i] = uv;
    }
    __syncthreads();
    // black cells on the box minus one layer
    {
        constexpr int W = B::FX + 4, RY = B::FY + 4, RZ = (DIM == 3) ? B::FZ + 4 : 1, HW = W / 2;
        for (int k = threadIdx.x; k < HW * RY * RZ; k += NT) {
            const int row = k / HW;
            const int sy = 1 + row % RY;
            const int sz = (DIM == 3) ? 1 + row / RY : 0;
            const int sx = 1 + 2 * (k % HW) + ((1 - par0 - sy - sz - 1) & 1);
            const int s[3] = {sx, sy, sz};
            int gi, cl;
            bool own;
            if (!cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) continue;
            const int i = sx + B::S1 * sy + B::S2 * sz;
            su[i] = (sf[i] + off_box<T, DIM, B>(L, su, i)) * L.invd[cl];
        }
    }
    __syncthreads();
    // residual on the box minus two layers (overwrites f); store the tile's u
    {
        constexpr int W = B::FX + 2, RY = B::FY + 2, RZ = (DIM == 3) ? B::FZ + 2 : 1;
        for (int k = threadIdx.x; k < W * RY * RZ; k += NT) {
            const int sx = 2 + k % W;
            const int sy = 2 + (k / W) % RY;
            const int sz = (DIM == 3) ? 2 + k / (W * RY) : 0;
            const int s[3] = {sx, sy, sz};
            int gi, cl;
            bool own;
            const int i = sx + B::S1 * sy + B::S2 * sz;
            if (!cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) continue;
            const T u = su[i];
            sf[i] = sf[i] - (L.diag[cl] * u - off_box<T, DIM, B>(L, su, i));
            if (own) upre[gi] = u;
        }
    }
    __syncthreads();
    // restriction of the tile's coarse cells
    constexpr int CX = Tile<DIM>::CX, CY = Tile<DIM>::CY, CZ = (DIM == 3) ? Tile<DIM>::CZ : 1;
    for (int c = threadIdx.x; c < CX * CY * CZ; c += NT) {
        const int cx = c % CX, cy = (c / CX) % CY, cz = c / (CX * CY);
        const int I[3] = {(int)blockIdx.x * CX + cx, (int)blockIdx.y * CY + cy,
                          (DIM == 3) ? (int)blockIdx.z * CZ + cz : 0};
        if (I[0] >= C.n[0] || I[1] >= C.n[1] || (DIM == 3 && I[2] >= C.n[2])) continue;
        T acc = (T)0;
        const int az_n = (DIM == 3) ? 4 : 1;
        for (int az = 0; az < az_n; ++az) {
            T wz = (T)1;
            int sz = 0;
            if (DIM == 3) {
                wz = (T)rweight(az, I[2], C.n[2], C.per[2]);
                if (wz == (T)0) continue;
                sz = 2 * cz + 2 + az;
            }
            for (int ay = 0; ay < 4; ++ay) {
                const T wy = (T)rweight(ay, I[1], C.n[1], C.per[1]);
                if (wy == (T)0) continue;
                const int sy = 2 * cy + 2 + ay;
                T row = (T)0;
#pragma unroll
                for (int ax = 0; ax < 4; ++ax) {
                    const T wx = (T)rweight(ax, I[0], C.n[0], C.per[0]);
                    row += wx * sf[(2 * cx + 2 + ax) + B::S1 * sy + B::S2 * sz];
                }
                acc += wz * wy * row;
            }
        }
        fc[I[0] + C.n[0] * (I[1] + C.n[1] * I[2])] = acc * (T)((DIM == 3) ? 0.125 : 0.25);
    }
}

// ---------------------------------------------------------------------------
// up: prolongation-add, black, red (one level); on the fine level also the
// partial sums of r.z and sum z, finished by the last block (beta, mean z).
// ---------------------------------------------------------------------------
template <class T, class TF, int DIM, bool FINE>
__global__ void __launch_bounds__(Tile<DIM>::NT)
    k_mg_up(LvT<T> L, LvT<T> C, const T* __restrict__ upre, const TF* __restrict__ f, const T* __restrict__ uc,
            T* __restrict__ upost, double* part_rz, double* part_sz, double* scal, const int* ictl,
            unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    const TF mr = FINE ? (TF)scal[PS_MEANR] : (TF)0;   // fine level: residual mean removed
    constexpr int H = 2;
    using B = Box<DIM, H>;
    constexpr int NT = Tile<DIM>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sf = reinterpret_cast<T*>(smraw);
    T* su = sf + B::SN;
    const int o[3] = {(int)blockIdx.x * B::FX - H, (int)blockIdx.y * B::FY - H,
                      (DIM == 3) ? (int)blockIdx.z * B::FZ - H : 0};
    int F[3] = {B::FX, B::FY, B::FZ};
    const int par0 = (o[0] + o[1] + o[2]) & 1;

    for (int i = threadIdx.x; i < B::SN; i += NT) {
        const int s[3] = {i % B::SX, (i / B::SX) % B::SY, i / B::S2};
        int gi, cl;
        bool own;
        T fv = (T)0, uv = (T)0;
        if (cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) {
            fv = (T)(f[gi] - mr);
            int gw[3] = {0, 0, 0};
            int rem = gi;
            gw[0] = rem % L.n[0];
            rem /= L.n[0];
            gw[1] = rem % L.n[1];
            gw[2] = rem / L.n[1];
            uv = upre[gi] + prolong_at<T, DIM>(C, uc, gw);
        }
        sf[i] = fv;
        su[i] = uv;
    }
    __syncthreads();
    // black on the box minus one layer
    {
        constexpr int W = B::FX + 2, RY = B::FY + 2, RZ = (DIM == 3) ? B::FZ + 2 : 1, HW = W / 2;
        for (int k = threadIdx.x; k < HW * RY * RZ; k += NT) {
            const int row = k / HW;
            const int sy = 1 + row % RY;
            const int sz = (DIM == 3) ? 1 + row / RY : 0;
            const int sx = 1 + 2 * (k % HW) + ((1 - par0 - sy - sz - 1) & 1);
            const int s[3] = {sx, sy, sz};
            int gi, cl;
            bool own;
            if (!cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) continue;
            const int i = sx + B::S1 * sy + B::S2 * sz;
            su[i] = (sf[i] + off_box<T, DIM, B>(L, su, i)) * L.invd[cl];
        }
    }
    __syncthreads();
    // red on the tile
    {
        constexpr int W = B::FX, RY = B::FY, RZ = B::FZ, HW = W / 2;
        for (int k = threadIdx.x; k < HW * RY * RZ; k += NT) {
            const int row = k / HW;
            const int sy = 2 + row % RY;
            const int sz = (DIM == 3) ? 2 + row / RY : 0;
            const int sx = 2 + 2 * (k % HW) + ((0 - par0 - sy - sz - 2) & 1);
            const int s[3] = {sx, sy, sz};
            int gi, cl;
            bool own;
            if (!cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own)) continue;
            const int i = sx + B::S1 * sy + B::S2 * sz;
            su[i] = (sf[i] + off_box<T, DIM, B>(L, su, i)) * L.invd[cl];
        }
    }
    __syncthreads();
    TF rz = (TF)0, sz = (TF)0;
    {
        constexpr int W = B::FX, RY = B::FY, RZ = B::FZ;
        for (int k = threadIdx.x; k < W * RY * RZ; k += NT) {
            const int s[3] = {2 + k % W, 2 + (k / W) % RY, (DIM == 3) ? 2 + k / (W * RY) : 0};
            int gi, cl;
            bool own;
            cell_info<T, DIM>(L, o, s, H, F, &gi, &cl, &own);
            if (!own) continue;
            const T u = su[s[0] + B::S1 * s[1] + B::S2 * s[2]];
            upost[gi] = u;
            if (FINE) {
                rz = fma(f[gi] - mr, (TF)u, rz);
                sz += (TF)u;
            }
        }
    }
    if (FINE) {
        __shared__ double red[2 * (NT / 32)];
        __shared__ float redf[2 * (NT / 32)];
        double brz, bsz;
        block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (threadIdx.x == 0) {
            part_rz[block_linear()] = brz;
            part_sz[block_linear()] = bsz;
        }
        if (arrive_last(cnt)) {
            double RZ, SZ;
            sum_parts2_cg<NT>(part_rz, part_sz, nb, red, &RZ, &SZ);
            if (threadIdx.x == 0) {
                const int it = ictl[PI_IT];
                scal[PS_BETA] = (it == 0) ? 0.0 : RZ / scal[PS_RZ];
                scal[PS_RZ] = RZ;
                scal[PS_MEANZ] = SZ / (double)L.N;
                *cnt = 0u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// CG: p = (z - mean z) + beta p_old (p_new buffer by parity), q = A p, p.q;
// the last block forms alpha = r.z / p.q.
// ---------------------------------------------------------------------------
template <class T, int DIM, class V>
__global__ void __launch_bounds__(Tile<DIM>::NT)
    k_cg_pq(LvT<V> L, const T* __restrict__ z, V* p0, V* p1, V* __restrict__ q, double* part, double* scal,
            const int* ictl, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    constexpr int H = 1;
    using B = Box<DIM, H>;
    constexpr int NT = Tile<DIM>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sp = reinterpret_cast<V*>(smraw);
    const int it = ictl[PI_IT];
    const V* pold = (it & 1) ? p0 : p1;
    V* pnew = (it & 1) ? p1 : p0;
    const V beta = (V)scal[PS_BETA], mz = (V)scal[PS_MEANZ];
    const int o[3] = {(int)blockIdx.x * B::FX - H, (int)blockIdx.y * B::FY - H,
                      (DIM == 3) ? (int)blockIdx.z * B::FZ - H : 0};
    int F[3] = {B::FX, B::FY, B::FZ};
    for (int i = threadIdx.x; i < B::SN; i += NT) {
        const int s[3] = {i % B::SX, (i / B::SX) % B::SY, i / B::S2};
        int gi, cl;
        bool own;
        V pv = (V)0;
        if (cell_info<V, DIM>(L, o, s, H, F, &gi, &cl, &own)) {
            pv = (V)z[gi] - mz;
            if (it > 0) pv = fma(beta, pold[gi], pv);
        }
        sp[i] = pv;
    }
    __syncthreads();
    V pq = (V)0;
    {
        constexpr int W = B::FX, RY = B::FY, RZ = B::FZ;
        for (int k = threadIdx.x; k < W * RY * RZ; k += NT) {
            const int s[3] = {1 + k % W, 1 + (k / W) % RY, (DIM == 3) ? 1 + k / (W * RY) : 0};
            int gi, cl;
            bool own;
            cell_info<V, DIM>(L, o, s, H, F, &gi, &cl, &own);
            if (!own) continue;
            const int i = s[0] + B::S1 * s[1] + B::S2 * s[2];
            const V pv = sp[i];
            const V qv = L.diag[cl] * pv - off_box<V, DIM, B>(L, sp, i);
            pnew[gi] = pv;
            q[gi] = qv;
            pq = fma(pv, qv, pq);
        }
    }
    __shared__ double red[NT / 32];
    __shared__ float redf[NT / 32];
    const double bpq = block_sum_any<NT>(pq, red, redf);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) part[block_linear()] = bpq;
    if (arrive_last(cnt)) {
        const double PQ = sum_parts_cg<NT>(part, nb, red);
        if (threadIdx.x == 0) {
            scal[PS_ALPHA] = scal[PS_RZ] / PQ;
            *cnt = 0u;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||^2; the last block tests convergence.
__global__ void __launch_bounds__(NTV)
    k_cg_update(double* __restrict__ x, double* __restrict__ r, const double* p0, const double* p1,
                const double* __restrict__ q, long long N, double* part, double* part_s, double* scal, int* ictl,
                unsigned int* cnt, double rtol, int max_iter, cudaGraphConditionalHandle h, int use_graph,
                int vec2) {
    pdl_wait();
    pdl_trigger();
    const int fb = blockIdx.y;
    batch_ctl(fb, &scal, &ictl, &cnt);
    // the system has converged (a batch member, or an iteration captured ahead
    // of the loop): x and the reported scalars stay as they are
    const int it = ictl[PI_IT], done = ictl[PI_DONE];
    const double alpha = scal[PS_ALPHA];
    if (done) return;
    x += fb * N;
    r += fb * N;
    p0 += fb * N;
    p1 += fb * N;
    q += fb * N;
    part += (long long)fb * gridDim.x;
    part_s += (long long)fb * gridDim.x;
    const double* __restrict__ p = (it & 1) ? p1 : p0;
    double rr = 0.0, sr = 0.0;
    if (vec2) {
        // two cells per thread step (16-byte accesses; N even and x 16-byte aligned,
        // the launch is sized by N / 2)
        const long long N2 = N >> 1;
        for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N2; t += (long long)gridDim.x * NTV) {
            const double2 pv = reinterpret_cast<const double2*>(p)[t];
            const double2 qv = reinterpret_cast<const double2*>(q)[t];
            double2 xv = reinterpret_cast<const double2*>(x)[t];
            double2 rv = reinterpret_cast<const double2*>(r)[t];
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            rv.x = fma(-alpha, qv.x, rv.x);
            rv.y = fma(-alpha, qv.y, rv.y);
            reinterpret_cast<double2*>(x)[t] = xv;
            reinterpret_cast<double2*>(r)[t] = rv;
            rr = fma(rv.x, rv.x, rr);
            rr = fma(rv.y, rv.y, rr);
            sr += rv.x + rv.y;
        }
    } else {
        for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N; t += (long long)gridDim.x * NTV) {
            x[t] = fma(alpha, p[t], x[t]);
            const double rv = fma(-alpha, q[t], r[t]);
            r[t] = rv;
            rr = fma(rv, rv, rr);
            sr += rv;
        }
    }
    __shared__ double red[2 * (NTV / 32)];
    block_sum2_t<NTV, double>(rr, sr, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rr;
        part_s[blockIdx.x] = sr;
    }
    if (arrive_last_n(cnt, gridDim.x)) {
        double RR, SR;
        sum_parts2_cg<NTV>(part, part_s, gridDim.x, red, &RR, &SR);
        if (threadIdx.x == 0) {
            const int itn = it + 1;
            ictl[PI_IT] = itn;
            scal[PS_RR] = RR;
            scal[PS_MEANR] = SR / (double)N;
            const double ff = scal[PS_FF];
            const int conv = (RR <= rtol * rtol * ff);
            const int bad = !(RR == RR) || !(RR < 1e300);
            const int done = conv || bad || (itn >= max_iter);
            ictl[PI_DONE] = done;
            if (done && !conv) ictl[PI_NOCONV] = 1;
            scal[PS_ITERS] = (double)itn;
            scal[PS_RELRES] = sqrt(RR / ff);
            if (use_graph) cudaGraphSetConditional(h, done ? 0u : 1u);
            *cnt = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Refinement mode: the CG update of an iteration with a reliable update.
// ---------------------------------------------------------------------------
// The CG update of an iteration in refinement mode, with a reliable update
// every time: the FP32 correction e = alpha p (p the FP32 search direction)
// is folded into the FP64 x, the FP64 residual is updated, r64 -= A e, and
// replaces the FP32 one, r32 = r64; the last block counts the iteration and
// applies the FP64 stopping test to ||r64||^2.  e is formed from p on the fly,
// for each cell and its neighbours, so neither e nor a recursively updated
// FP32 residual is stored.  A e and the residual difference are formed in
// float-float arithmetic from the FP32 e (about 2^-46 relative, far below
// what the stopping test needs) with float <-> double conversions by bit
// operations, so that only three FP64 operations per cell (two additions, the
// squared norm) use the 1/64-rate FP64 pipe.  The FP32 search direction and
// r.z are kept.
// W x-consecutive cells per thread step of the reliable-update CG step.
template <int DIM, int W>
__device__ __forceinline__ void ir_vec(const LvT<double>& L, double* __restrict__ x, double* __restrict__ r64,
                                       const float* __restrict__ p, float* __restrict__ r32, float alpha,
                                       const FF* wd, int i0, int stride, int iend, double& rr, double& sr) {
    constexpr int G = W / 4;   // float4 groups per step
    auto ld1 = [&](int i) -> float { return fmaf(alpha, p[i], 0.0f); };
    auto ldw = [&](int i, float* out) {
#pragma unroll
        for (int g4 = 0; g4 < G; ++g4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i + 4 * g4);
            out[4 * g4 + 0] = fmaf(alpha, v.x, 0.0f);
            out[4 * g4 + 1] = fmaf(alpha, v.y, 0.0f);
            out[4 * g4 + 2] = fmaf(alpha, v.z, 0.0f);
            out[4 * g4 + 3] = fmaf(alpha, v.w, 0.0f);
        }
    };
    const int nx = L.n[0], ny = L.n[1];
    const int NW = L.N / W;
    for (int q = i0; q < min(NW, iend); q += stride) {
        const int t0 = W * q;
        int c[3];
        coords(L, t0, c);
        float ev[W];
        ldw(t0, ev);
        float el = 0.0f, er = 0.0f;
        if (c[0] > 0) el = ld1(t0 - 1);
        else if (L.per[0]) el = ld1(t0 + nx - 1);
        if (c[0] + W < nx) er = ld1(t0 + W);
        else if (L.per[0]) er = ld1(t0 + W - nx);
        float nb[2][2][W];   // [y, z][low, high] neighbour rows
        int clo = 0, p3 = 3;
#pragma unroll
        for (int d = 1; d < DIM; ++d) {
            const int n = L.n[d];
            const int sd = (d == 1) ? nx : nx * ny;
#pragma unroll
            for (int i = 0; i < W; ++i) nb[d - 1][0][i] = nb[d - 1][1][i] = 0.0f;
            if (c[d] > 0) ldw(t0 - sd, nb[d - 1][0]);
            else if (L.per[d]) ldw(t0 + (n - 1) * sd, nb[d - 1][0]);
            if (c[d] < n - 1) ldw(t0 + sd, nb[d - 1][1]);
            else if (L.per[d]) ldw(t0 - (n - 1) * sd, nb[d - 1][1]);
            clo += (L.per[d] ? 2 : (int)(c[d] > 0) + (int)(c[d] < n - 1)) * p3;
            p3 *= 3;
        }
        double rin[W], xin[W];
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            const double2 ra = *reinterpret_cast<const double2*>(r64 + t0 + 2 * h);
            const double2 xa = *reinterpret_cast<const double2*>(x + t0 + 2 * h);
            rin[2 * h] = ra.x;
            rin[2 * h + 1] = ra.y;
            xin[2 * h] = xa.x;
            xin[2 * h + 1] = xa.y;
        }
        double rout[W], xout[W];
        float r32o[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const float a0 = (i == 0) ? el : ev[i - 1];
            const float b0 = (i == W - 1) ? er : ev[i + 1];
            FF off;
            off += wd[0] * (FF(a0, 0.0f) + FF(b0, 0.0f));
#pragma unroll
            for (int d = 1; d < DIM; ++d) off += wd[d] * (FF(nb[d - 1][0][i], 0.0f) + FF(nb[d - 1][1][i], 0.0f));
            const int xg = c[0] + i;
            const int cl = (L.per[0] ? 2 : (int)(xg > 0) + (int)(xg < nx - 1)) + clo;
            const FF Ae = FF(L.diag[cl]) * FF(ev[i], 0.0f) - off;
            const FF rv = FF(rin[i]) - Ae;
            xout[i] = xin[i] + f2d_bits(ev[i]);
            rout[i] = f2d_bits(rv.hi) + f2d_bits(rv.lo);
            r32o[i] = rv.hi;
            rr = fma(rout[i], rout[i], rr);
            sr += rout[i];
        }
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            *reinterpret_cast<double2*>(x + t0 + 2 * h) = make_double2(xout[2 * h], xout[2 * h + 1]);
            *reinterpret_cast<double2*>(r64 + t0 + 2 * h) = make_double2(rout[2 * h], rout[2 * h + 1]);
        }
#pragma unroll
        for (int g4 = 0; g4 < G; ++g4)
            *reinterpret_cast<float4*>(r32 + t0 + 4 * g4) =
                make_float4(r32o[4 * g4], r32o[4 * g4 + 1], r32o[4 * g4 + 2], r32o[4 * g4 + 3]);
    }
}

// The cells of the reliable-update CG step handled by one thread: compact
// indices (groups of vec4 = 4 or 8 x-consecutive cells, else single cells)
// from i0 by stride, below iend; adds ||r||^2 and sum r of the new residual
// to rr, sr.
template <int DIM, int W = 4>
__device__ __forceinline__ void ir_cells(const LvT<double>& L, double* __restrict__ x, double* __restrict__ r64,
                                         const float* __restrict__ p, float* __restrict__ r32, float alpha,
                                         int vec4, int i0, int stride, int iend, double& rr, double& sr) {
    // the correction e = alpha p at compact index i (the product rounded once)
    auto ld1 = [&](int i) -> float { return fmaf(alpha, p[i], 0.0f); };
    FF wd[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) wd[d] = FF(L.w[d]);
    if (vec4) {
        // W x-consecutive cells per thread step (nx % W == 0, x 16-byte
        // aligned; the launch is sized by N / W): one coordinate map, 16-byte
        // loads of p's rows (e = alpha p) and of x, r64; each cell's
        // arithmetic is the scalar path's, in its order
        ir_vec<DIM, W>(L, x, r64, p, r32, alpha, wd, i0, stride, iend, rr, sr);
    }
    for (int t = vec4 ? L.N : i0; t < min(L.N, iend); t += stride) {
        int c[3];
        coords(L, t, c);
        FF off;
        int stride = 1, p3 = 1, cl = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int n = L.n[d];
            float a = 0.0f, b = 0.0f;
            if (c[d] > 0) a = ld1(t - stride);
            else if (L.per[d]) a = ld1(t + (n - 1) * stride);
            if (c[d] < n - 1) b = ld1(t + stride);
            else if (L.per[d]) b = ld1(t - (n - 1) * stride);
            off += wd[d] * (FF(a, 0.0f) + FF(b, 0.0f));
            cl += (L.per[d] ? 2 : (int)(c[d] > 0) + (int)(c[d] < n - 1)) * p3;
            stride *= n;
            p3 *= 3;
        }
        const float ev = ld1(t);
        const FF Ae = FF(L.diag[cl]) * FF(ev, 0.0f) - off;
        const FF rv = FF(r64[t]) - Ae;
        x[t] = x[t] + f2d_bits(ev);
        const double rvd = f2d_bits(rv.hi) + f2d_bits(rv.lo);
        r64[t] = rvd;
        r32[t] = rv.hi;
        rr = fma(rvd, rvd, rr);
        sr += rvd;
    }
}

template <int DIM, int W>
__global__ void __launch_bounds__(NTV)
    k_ir_step(LvT<double> L, double* __restrict__ x, double* __restrict__ r64, const float* p0, const float* p1,
              float* __restrict__ r32, double* part, double* part_s, double* scal, int* ictl, unsigned int* cnt,
              double rtol, int max_iter, cudaGraphConditionalHandle h, int use_graph, int vec4) {
    pdl_wait();
    pdl_trigger();
    const int fb = blockIdx.y;
    batch_ctl(fb, &scal, &ictl, &cnt);
    // the system has converged (a batch member, or an iteration captured
    // ahead of the loop): x, r and the reported scalars stay as they are
    const int done = ictl[PI_DONE], it = ictl[PI_IT];
    const float alpha = (float)scal[PS_ALPHA];
    if (done) return;
    const float* __restrict__ p = ((it & 1) ? p1 : p0) + (long long)fb * L.N;
    x += (long long)fb * L.N;
    r64 += (long long)fb * L.N;
    r32 += (long long)fb * L.N;
    part += (long long)fb * gridDim.x;
    part_s += (long long)fb * gridDim.x;
    double rr = 0.0, sr = 0.0;
    ir_cells<DIM, W>(L, x, r64, p, r32, alpha, vec4, blockIdx.x * NTV + threadIdx.x, gridDim.x * NTV, INT_MAX, rr,
                  sr);
    __shared__ double red[2 * (NTV / 32)];
    block_sum2_t<NTV, double>(rr, sr, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rr;
        part_s[blockIdx.x] = sr;
    }
    if (arrive_last_n(cnt, gridDim.x)) {
        double RR, SR;
        sum_parts2_cg<NTV>(part, part_s, gridDim.x, red, &RR, &SR);
        if (threadIdx.x == 0) {
            scal[PS_MEANR] = SR / (double)L.N;
            const int tot = ictl[PI_TOTAL] + 1;
            ictl[PI_IT] = it + 1;
            ictl[PI_TOTAL] = tot;
            scal[PS_ITERS] = (double)tot;
            const double ff = scal[PS_FF];
            const int conv = (RR <= rtol * rtol * ff);
            const int bad = !(RR == RR) || !(RR < 1e300);
            const int done = conv || bad || (tot >= max_iter);
            scal[PS_RR] = RR;
            scal[PS_RELRES] = sqrt(RR / ff);
            ictl[PI_DONE] = done;
            if (done && !conv) ictl[PI_NOCONV] = 1;
            if (use_graph) cudaGraphSetConditional(h, done ? 0u : 1u);
            *cnt = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Compact-array stencil (tail levels, prologue)
// ---------------------------------------------------------------------------
template <class T, int DIM>
__device__ __forceinline__ T off_compact(const LvT<T>& L, const T* u, int t, const int c[3], int* cls) {
    T off = (T)0;
    int stride = 1, p3 = 1, cl = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int n = L.n[d];
        const T w = L.w[d];
        if (c[d] > 0) off += w * u[t - stride];
        else if (L.per[d]) off += w * u[t + (n - 1) * stride];
        if (c[d] < n - 1) off += w * u[t + stride];
        else if (L.per[d]) off += w * u[t - (n - 1) * stride];
        cl += (L.per[d] ? 2 : (int)(c[d] > 0) + (int)(c[d] < n - 1)) * p3;
        stride *= n;
        p3 *= 3;
    }
    *cls = cl;
    return off;
}

// Sum of b (partials; the last block stores the mean).
__global__ void __launch_bounds__(NTV) k_mean(const double* __restrict__ b, long long N, double* part,
                                              double* scal, int slot, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    const int fb = blockIdx.y;
    scal += (long long)fb * PS_NSCAL;
    cnt += (long long)fb * kNumCounters;
    b += fb * N;
    part += (long long)fb * gridDim.x;
    double v = 0.0;
    for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N; t += (long long)gridDim.x * NTV) v += b[t];
    __shared__ double red[NTV / 32];
    v = block_sum<NTV>(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
    if (arrive_last_n(cnt, gridDim.x)) {
        const double s = sum_parts_cg<NTV>(part, gridDim.x, red);
        if (threadIdx.x == 0) {
            scal[slot] = s / (double)N;
            *cnt = 0u;
        }
    }
}

// r = -(b - mean b) - A x at the compact cells from i0 by stride; adds
// ||f||^2, ||r||^2 and sum r to ff, rr, sr.
template <int DIM>
__device__ __forceinline__ void init_cells(const LvT<double>& L, const double* __restrict__ b,
                                           const double* __restrict__ x, double* __restrict__ r,
                                           float* __restrict__ r32, double mean_b, int i0, int stride, double& ff,
                                           double& rr, double& sr) {
    for (int t = i0; t < L.N; t += stride) {
        int c[3];
        coords(L, t, c);
        int cl;
        const double off = off_compact<double, DIM>(L, x, t, c, &cl);
        const double f = -(b[t] - mean_b);
        const double rv = f - (L.diag[cl] * x[t] - off);
        r[t] = rv;
        if (r32) r32[t] = (float)rv;
        ff = fma(f, f, ff);
        rr = fma(rv, rv, rr);
        sr += rv;
    }
}

// r = -(b - mean b) - A x; ||f||^2, ||r||^2; the last block initialises the
// control words and the while-node conditional.
template <int DIM>
__global__ void __launch_bounds__(NTV)
    k_pcg_init(LvT<double> L, const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
               float* __restrict__ r32, double* pff, double* prr, double* psr, double* scal, int* ictl,
               unsigned int* cnt, double rtol, cudaGraphConditionalHandle h, int use_graph) {
    pdl_wait();
    pdl_trigger();
    const int fb = blockIdx.y;
    batch_ctl(fb, &scal, &ictl, &cnt);
    b += (long long)fb * L.N;
    x += (long long)fb * L.N;
    r += (long long)fb * L.N;
    if (r32) r32 += (long long)fb * L.N;
    pff += (long long)fb * gridDim.x;
    prr += (long long)fb * gridDim.x;
    psr += (long long)fb * gridDim.x;
    const double mean_b = scal[PS_MEANB];
    double ff = 0.0, rr = 0.0, sr = 0.0;
    init_cells<DIM>(L, b, x, r, r32, mean_b, blockIdx.x * NTV + threadIdx.x, gridDim.x * NTV, ff, rr, sr);
    __shared__ double red[2 * (NTV / 32)];
    block_sum2_t<NTV, double>(ff, rr, red);
    sr = block_sum<NTV>(sr, red);
    if (threadIdx.x == 0) {
        pff[blockIdx.x] = ff;
        prr[blockIdx.x] = rr;
        psr[blockIdx.x] = sr;
    }
    if (arrive_last_n(cnt, gridDim.x)) {
        double FF, RR;
        sum_parts2_cg<NTV>(pff, prr, gridDim.x, red, &FF, &RR);
        const double SR = sum_parts_cg<NTV>(psr, gridDim.x, red);
        if (threadIdx.x == 0) {
            scal[PS_FF] = FF;
            scal[PS_RR] = RR;
            scal[PS_MEANR] = SR / (double)L.N;
            scal[PS_RZ] = 0.0;
            scal[PS_BETA] = 0.0;
            scal[PS_ITERS] = 0.0;
            ictl[PI_IT] = 0;
            ictl[PI_TOTAL] = 0;
            ictl[PI_NOCONV] = 0;
            const int zero = !(FF > 0.0);
            ictl[PI_ZERO] = zero;
            int done = zero || (RR <= rtol * rtol * FF);
            scal[PS_RELRES] = zero ? 0.0 : sqrt(RR / FF);
            if (!(RR == RR)) {             // non-finite input
                done = 1;
                ictl[PI_NOCONV] = 1;
            }
            ictl[PI_DONE] = done;
            if (use_graph) cudaGraphSetConditional(h, done ? 0u : 1u);
            *cnt = 0u;
        }
    }
}

// Batches: the solve continues while any system is active (sets the
// while-node condition, and bdone for a host-driven loop).
__global__ void __launch_bounds__(NTV) k_batch_cond(const int* ictl, int nb, int* bdone,
                                                    cudaGraphConditionalHandle h, int use_graph) {
    pdl_wait();
    pdl_trigger();
    int active = 0;
    for (int k = threadIdx.x; k < nb; k += NTV) active |= !ictl[(long long)k * PI_NINT + PI_DONE];
    active = __syncthreads_or(active);
    if (threadIdx.x == 0) {
        *bdone = !active;
        if (use_graph) cudaGraphSetConditional(h, active ? 1u : 0u);
    }
}

// Batches: each system's iteration count and relative residual to rep[k],
// non-convergence into *status[k].
__global__ void __launch_bounds__(NTV) k_batch_report(const double* scal, const int* ictl, int nb,
                                                      double* const* rep, int* const* status, int bit) {
    pdl_wait();
    pdl_trigger();
    for (int k = threadIdx.x; k < nb; k += NTV) {
        if (rep && rep[k]) {
            rep[k][0] = scal[(long long)k * PS_NSCAL + PS_ITERS];
            rep[k][1] = scal[(long long)k * PS_NSCAL + PS_RELRES];
        }
        if (status && status[k] && ictl[(long long)k * PI_NINT + PI_NOCONV]) atomicOr(status[k], bit);
    }
}

// Zero-mean x; report iterations / residual / status.
__global__ void __launch_bounds__(NTV) k_sub_mean(double* __restrict__ x, long long N, const double* scal,
                                                  const int* ictl, double* rep, int* status, int bit) {
    pdl_wait();
    pdl_trigger();
    const int fb = blockIdx.y;
    scal += (long long)fb * PS_NSCAL;
    ictl += (long long)fb * PI_NINT;
    x += fb * N;
    const double mean = scal[PS_MEANX];
    const int zero = ictl[PI_ZERO];
    for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N; t += (long long)gridDim.x * NTV)
        x[t] = zero ? 0.0 : (x[t] - mean);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rep) {
            rep[0] = scal[PS_ITERS];
            rep[1] = scal[PS_RELRES];
        }
        if (status && ictl[PI_NOCONV]) atomicOr(status, bit);
    }
}

// ---------------------------------------------------------------------------
// Tail: levels top .. nlev-1 in the shared memory of one block.
// ---------------------------------------------------------------------------
struct TailArgs {
    int top, nlev, Nc;
    int off_u[kMaxLevels], off_f[kMaxLevels], off_r;
};

template <class T, int DIM>
__device__ void tail_smooth_color(const LvT<T>& L, T* u, const T* f, int color) {
    for (int t = threadIdx.x; t < L.N; t += kTailThreads) {
        int c[3];
        coords(L, t, c);
        if (((c[0] + c[1] + c[2]) & 1) != color) continue;
        int cl;
        const T off = off_compact<T, DIM>(L, u, t, c, &cl);
        u[t] = (f[t] + off) * L.invd[cl];
    }
}

template <class T, int DIM>
__global__ void __launch_bounds__(kTailThreads)
    k_mg_tail(const LvT<T>* __restrict__ levs, TailArgs a, const T* __restrict__ f_top, T* __restrict__ u_top,
              const T* __restrict__ Minv) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int top = a.top, last = a.nlev - 1;
    {
        const LvT<T>& L = levs[top];
        T* f = sm + a.off_f[top];
        for (int t = threadIdx.x; t < L.N; t += kTailThreads) f[t] = f_top[t];
    }
    __syncthreads();
    for (int l = top; l < last; ++l) {
        const LvT<T>& L = levs[l];
        const LvT<T>& C = levs[l + 1];
        T* u = sm + a.off_u[l];
        const T* f = sm + a.off_f[l];
        T* r = sm + a.off_r;
        T* fc = sm + a.off_f[l + 1];
        for (int t = threadIdx.x; t < L.N; t += kTailThreads) {
            int c[3];
            coords(L, t, c);
            int cl = 0, p3 = 1;
            for (int d = 0; d < DIM; ++d) {
                cl += (L.per[d] ? 2 : (int)(c[d] > 0) + (int)(c[d] < L.n[d] - 1)) * p3;
                p3 *= 3;
            }
            u[t] = (((c[0] + c[1] + c[2]) & 1) == 0) ? f[t] * L.invd[cl] : (T)0;
        }
        __syncthreads();
        tail_smooth_color<T, DIM>(L, u, f, 1);
        __syncthreads();
        for (int t = threadIdx.x; t < L.N; t += kTailThreads) {
            int c[3];
            coords(L, t, c);
            int cl;
            const T off = off_compact<T, DIM>(L, u, t, c, &cl);
            r[t] = f[t] - (L.diag[cl] * u[t] - off);
        }
        __syncthreads();
        for (int T_ = threadIdx.x; T_ < C.N; T_ += kTailThreads) {
            int I[3];
            coords(C, T_, I);
            T acc = (T)0;
            const int az_n = (DIM == 3) ? 4 : 1;
            for (int az = 0; az < az_n; ++az) {
                T wz = (T)1;
                int fz = 0;
                if (DIM == 3) {
                    wz = (T)rweight(az, I[2], C.n[2], C.per[2]);
                    if (wz == (T)0) continue;
                    fz = wrapi(2 * I[2] - 1 + az, L.n[2]);
                }
                for (int ay = 0; ay < 4; ++ay) {
                    const T wy = (T)rweight(ay, I[1], C.n[1], C.per[1]);
                    if (wy == (T)0) continue;
                    const int fy = wrapi(2 * I[1] - 1 + ay, L.n[1]);
                    for (int ax = 0; ax < 4; ++ax) {
                        const T wx = (T)rweight(ax, I[0], C.n[0], C.per[0]);
                        if (wx == (T)0) continue;
                        const int fx = wrapi(2 * I[0] - 1 + ax, L.n[0]);
                        acc += wz * wy * wx * r[fx + L.n[0] * (fy + L.n[1] * fz)];
                    }
                }
            }
            fc[T_] = acc * (T)((DIM == 3) ? 0.125 : 0.25);
        }
        __syncthreads();
    }
    {
        // coarsest level: u = Minv f
        const int Nc = a.Nc;
        const T* f = sm + a.off_f[last];
        T* u = sm + a.off_u[last];
        for (int i = threadIdx.x; i < Nc; i += kTailThreads) {
            T acc = (T)0;
            const T* row = Minv + (size_t)i * Nc;
            for (int j = 0; j < Nc; ++j) acc += row[j] * f[j];
            u[i] = acc;
        }
    }
    __syncthreads();
    for (int l = last - 1; l >= top; --l) {
        const LvT<T>& L = levs[l];
        const LvT<T>& C = levs[l + 1];
        T* u = sm + a.off_u[l];
        const T* f = sm + a.off_f[l];
        const T* uc = sm + a.off_u[l + 1];
        for (int t = threadIdx.x; t < L.N; t += kTailThreads) {
            int c[3];
            coords(L, t, c);
            u[t] += prolong_at<T, DIM>(C, uc, c);
        }
        __syncthreads();
        tail_smooth_color<T, DIM>(L, u, f, 1);
        __syncthreads();
        tail_smooth_color<T, DIM>(L, u, f, 0);
        __syncthreads();
    }
    {
        const LvT<T>& L = levs[top];
        const T* u = sm + a.off_u[top];
        for (int t = threadIdx.x; t < L.N; t += kTailThreads) u_top[t] = u[t];
    }
}

// Single-level grid (the fine level is the coarsest): z = Minv r, then the
// r.z / sum z scalars (one block).
template <class T>
__global__ void __launch_bounds__(kTailThreads)
    k_direct(const T* __restrict__ Minv, int Nc, const double* __restrict__ r, T* __restrict__ z, double* scal,
             const int* ictl) {
    pdl_wait();
    pdl_trigger();
    double rz = 0.0, sz = 0.0;
    for (int i = threadIdx.x; i < Nc; i += kTailThreads) {
        T acc = (T)0;
        const T* row = Minv + (size_t)i * Nc;
        for (int j = 0; j < Nc; ++j) acc += row[j] * (T)r[j];
        z[i] = acc;
        rz += r[i] * (double)acc;
        sz += (double)acc;
    }
    __shared__ double red[kTailThreads / 32];
    rz = block_sum<kTailThreads>(rz, red);
    sz = block_sum<kTailThreads>(sz, red);
    if (threadIdx.x == 0) {
        const int it = ictl[PI_IT];
        scal[PS_BETA] = (it == 0) ? 0.0 : rz / scal[PS_RZ];
        scal[PS_RZ] = rz;
        scal[PS_MEANZ] = sz / (double)Nc;
    }
}

// ---------------------------------------------------------------------------
// 2D kernels: a 32-column shared-memory box, one warp per box row (lane =
// column), colour sweeps two rows per warp step (lanes 0-15 and 16-31 take
// alternate rows, so the two half-warps hit even and odd banks).
// ---------------------------------------------------------------------------
namespace k2 {

constexpr int NW = 16;            // warps per block
constexpr int NT = 32 * NW;
constexpr int SY = 32;            // box rows
// NS red-black sweeps per smoothing: down keeps a halo of 2 NS + 1 (fine tile
// 32 - 2 (2 NS + 1)), up a halo of 2 NS (fine tile 32 - 4 NS).
__host__ __device__ constexpr int fd_of(int ns) { return 32 - 2 * (2 * ns + 1); }   // down fine tile (26 / 22)
__host__ __device__ constexpr int cd_of(int ns) { return fd_of(ns) / 2; }           // down coarse tile (13 / 11)
__host__ __device__ constexpr int fu_of(int ns) { return 32 - 4 * ns; }              // up fine tile (28 / 24)
constexpr int FP = 30;            // CG operator: tile (32 = 30 + 2 x 1)

struct Ax {
    int gw;       // wrapped index (valid cells)
    int cls;      // neighbour count along the axis
    bool valid;   // inside the domain or periodic
    bool in;      // inside the domain (unwrapped)
};

// Box coordinates reach at most the halo (< n for every level the 2D kernels
// run on) beyond the domain, so one add or subtract wraps them; the modulo
// stays as the fallback.
__device__ __forceinline__ Ax axis(int g, int n, int per) {
    Ax a;
    a.in = (g >= 0 && g < n);
    const int w = (g >= -n && g < 2 * n) ? (g < 0 ? g + n : g - n) : wrapi(g, n);
    a.gw = a.in ? g : (per ? w : 0);
    a.valid = a.in || per;
    a.cls = per ? 2 : (int)(a.gw > 0) + (int)(a.gw < n - 1);
    return a;
}

template <class T>
__device__ __forceinline__ T off2(const LvT<T>& L, T (*su)[32], int r, int c) {
    return L.w[0] * (su[r][c - 1] + su[r][c + 1]) + L.w[1] * (su[r - 1][c] + su[r + 1][c]);
}

// Per-block axis codes (class | valid << 2) of the two columns a lane can take
// in a colour sweep (2 (lane & 15) and that + 1) and of every row (shared).
__device__ __forceinline__ int axis_code2(int g, int n, int per) {
    const Ax a = axis(g, n, per);
    return a.cls | ((int)a.valid << 2);
}
struct ColCodes {
    int c[2];
};
template <class T>
__device__ __forceinline__ ColCodes box_codes(const LvT<T>& L, int ox, int oy, int* srow) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < SY) srow[threadIdx.x] = axis_code2(oy + (int)threadIdx.x, L.n[1], L.per[1]);
    ColCodes cc;
    cc.c[0] = axis_code2(ox + 2 * (lane & 15), L.n[0], L.per[0]);
    cc.c[1] = axis_code2(ox + 2 * (lane & 15) + 1, L.n[0], L.per[0]);
    return cc;   // srow is read after the caller's next barrier
}

// One colour on rows [r0, r1] x columns [c0, c1] of the box.
template <class T>
__device__ __forceinline__ void color_sweep(const LvT<T>& L, T (*su)[32], T (*sf)[32], int par0, int color, int r0,
                                            int r1, int c0, int c1, const ColCodes& cc, const int* srow) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npairs = (r1 - r0 + 2) / 2;
    for (int rp = warp; rp < npairs; rp += NW) {
        const int r = r0 + 2 * rp + (lane >> 4);
        const int odd = (color - par0 - r) & 1;
        const int c = 2 * (lane & 15) + odd;
        if (r > r1 || c < c0 || c > c1) continue;
        const int cx = cc.c[odd], cy = srow[r];
        if (!((cx & cy) & 4)) continue;
        su[r][c] = (sf[r][c] + off2<T>(L, su, r, c)) * L.invd[(cx & 3) + 3 * (cy & 3)];
    }
}

// down on the tile (bx, by) of a level: load f (minus mr on the fine level)
// and red from zero, then black, red, black, the residual and the
// restriction.  sf, su (SY x 32) and srow (SY) are the caller's shared
// arrays; the leading barrier lets a block run tiles back to back.
template <class T, class TF, int NS>
__device__ __forceinline__ void down_tile(const LvT<T>& L, const LvT<T>& C, const TF* __restrict__ f,
                                          T* __restrict__ upre, T* __restrict__ fc, TF mr, int bx, int by,
                                          T (*sf)[32], T (*su)[32], int* srow) {
    __syncthreads();
    constexpr int H = 2 * NS + 1, FD = fd_of(NS), CD = cd_of(NS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ox = bx * FD - H, oy = by * FD - H;
    const int nx = L.n[0];
    const int par0 = (ox + oy) & 1;
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    const ColCodes cc = box_codes<T>(L, ox, oy, srow);
    Ax ayk[SY / NW];   // this thread's rows (kept for the residual pass)
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        const Ax ay = axis(oy + r, L.n[1], L.per[1]);
        ayk[k] = ay;
        T fv = (T)0, uv = (T)0;
        if (ax.valid && ay.valid) {
            fv = (T)(f[ax.gw + nx * ay.gw] - mr);
            if (((par0 + lane + r) & 1) == 0) uv = fv * L.invd[ax.cls + 3 * ay.cls];
        }
        sf[r][lane] = fv;
        su[r][lane] = uv;
    }
    __syncthreads();
    // pre-smoothing (red from zero above, then black, red, ...): sweep k works on
    // the box minus k layers
#pragma unroll
    for (int k = 1; k < 2 * NS; ++k) {
        color_sweep<T>(L, su, sf, par0, k & 1, k, SY - 1 - k, k, 31 - k, cc, srow);
        __syncthreads();
    }
    // residual on the box minus 2 NS layers (overwrites f); store the tile's u
    constexpr int R0 = 2 * NS, R1 = 31 - 2 * NS;
    const bool colr = (lane >= R0 && lane <= R1);
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        if (r < R0 || r > R1 || !colr) continue;
        const Ax ay = ayk[k];
        if (!(ax.valid && ay.valid)) continue;
        const T u = su[r][lane];
        sf[r][lane] = sf[r][lane] - (L.diag[ax.cls + 3 * ay.cls] * u - off2<T>(L, su, r, lane));
        if (ax.in && ay.in && lane >= H && lane < H + FD && r >= H && r < H + FD) upre[ax.gw + nx * ay.gw] = u;
    }
    __syncthreads();
    // restriction: coarse cell I of the tile reads fine cells 2I-1 .. 2I+2, at
    // box offset 2 c + H - 1 + a
    for (int c = threadIdx.x; c < CD * CD; c += NT) {
        const int cx = c % CD, cy = c / CD;
        const int I = bx * CD + cx, J = by * CD + cy;
        if (I >= C.n[0] || J >= C.n[1]) continue;
        T wx[4];
#pragma unroll
        for (int axx = 0; axx < 4; ++axx) wx[axx] = (T)rweight(axx, I, C.n[0], C.per[0]);
        T acc = (T)0;
#pragma unroll
        for (int ay = 0; ay < 4; ++ay) {
            const T wy = (T)rweight(ay, J, C.n[1], C.per[1]);
            const int r = 2 * cy + H - 1 + ay;
            T row = (T)0;
#pragma unroll
            for (int axx = 0; axx < 4; ++axx) row += wx[axx] * sf[r][2 * cx + H - 1 + axx];
            acc += wy * row;
        }
        fc[I + C.n[0] * J] = acc * (T)0.25;
    }
}

template <class T, class TF, int NS>
__global__ void __launch_bounds__(NT) down(LvT<T> L, LvT<T> C, const TF* __restrict__ f, T* __restrict__ upre,
                                           T* __restrict__ fc, const double* __restrict__ scal_r) {
    pdl_wait();
    pdl_trigger();
    {   // system of a batch
        const long long fb = blockIdx.z;
        f += fb * L.N;
        upre += fb * L.N;
        fc += fb * C.N;
        if (scal_r) scal_r += fb * PS_NSCAL;
    }
    // fine level: the CG residual enters the preconditioner with its mean removed
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    __shared__ T sf[SY][32];
    __shared__ T su[SY][32];
    __shared__ int srow[SY];
    down_tile<T, TF, NS>(L, C, f, upre, fc, mr, blockIdx.x, blockIdx.y, sf, su, srow);
}

// up on the tile (bx, by) of a level: prolongation-add, then black, red,
// black, red; on the fine level the partial sums of r.z and sum z over the
// tile's cells are added to rz, sz.  Shared arrays as for down_tile.
template <class T, class TF, bool FINE, int NS>
__device__ __forceinline__ void up_tile(const LvT<T>& L, const LvT<T>& C, const T* __restrict__ upre,
                                        const TF* __restrict__ f, const T* __restrict__ uc, T* __restrict__ upost,
                                        TF mr, int bx, int by, T (*sf)[32], T (*su)[32], int* srow, TF& rz,
                                        TF& sz) {
    __syncthreads();
    constexpr int H = 2 * NS, FU = fu_of(NS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ox = bx * FU - H, oy = by * FU - H;
    const int nx = L.n[0];
    const int par0 = (ox + oy) & 1;
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    const ColCodes cc = box_codes<T>(L, ox, oy, srow);
    // coarse columns of this lane's fine column (bilinear prolongation)
    int I0 = 0, I1 = 0;
    if (ax.valid) pro_pair(ax.gw, C.n[0], C.per[0], &I0, &I1);
    const T a = (T)0.75, b = (T)0.25;
    Ax ayk[SY / NW];   // this thread's rows (kept for the output pass)
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        const Ax ay = axis(oy + r, L.n[1], L.per[1]);
        ayk[k] = ay;
        T fv = (T)0, uv = (T)0;
        if (ax.valid && ay.valid) {
            const int g = ax.gw + nx * ay.gw;
            fv = (T)(f[g] - mr);
            int J0, J1;
            pro_pair(ay.gw, C.n[1], C.per[1], &J0, &J1);
            const T* c0 = uc + C.n[0] * J0;
            const T* c1 = uc + C.n[0] * J1;
            uv = upre[g] + a * (a * c0[I0] + b * c0[I1]) + b * (a * c1[I0] + b * c1[I1]);
        }
        sf[r][lane] = fv;
        su[r][lane] = uv;
    }
    __syncthreads();
    // post-smoothing black, red, ...: sweep k on the box minus k layers; the
    // last (red) sweep covers exactly the tile
#pragma unroll
    for (int k = 1; k <= 2 * NS; ++k) {
        color_sweep<T>(L, su, sf, par0, k & 1, k, SY - 1 - k, k, 31 - k, cc, srow);
        __syncthreads();
    }
    const bool colo = ax.in && lane >= H && lane < H + FU;
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        if (!colo || r < H || r >= H + FU) continue;
        const Ax ay = ayk[k];
        if (!ay.in) continue;
        const int g = ax.gw + nx * ay.gw;
        const T u = su[r][lane];
        upost[g] = u;
        if (FINE) {
            // f is still in shared memory, exactly, when T and TF agree
            const TF fv = (sizeof(T) == sizeof(TF)) ? (TF)sf[r][lane] : (TF)(f[g] - mr);
            rz = fma(fv, (TF)u, rz);
            sz += (TF)u;
        }
    }
}

template <class T, class TF, bool FINE, int NS>
__global__ void __launch_bounds__(NT)
    up(LvT<T> L, LvT<T> C, const T* __restrict__ upre, const TF* __restrict__ f, const T* __restrict__ uc,
       T* __restrict__ upost, double* part_rz, double* part_sz, double* scal, const int* ictl, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    {   // system of a batch
        const long long fb = blockIdx.z;
        upre += fb * L.N;
        f += fb * L.N;
        uc += fb * C.N;
        upost += fb * L.N;
        if (FINE) {
            part_rz += fb * gridDim.x * gridDim.y;
            part_sz += fb * gridDim.x * gridDim.y;
            scal += fb * PS_NSCAL;
            ictl += fb * PI_NINT;
            cnt += fb * kNumCounters;
        }
    }
    const TF mr = FINE ? (TF)scal[PS_MEANR] : (TF)0;   // fine level: residual mean removed
    __shared__ T sf[SY][32];
    __shared__ T su[SY][32];
    __shared__ int srow[SY];
    TF rz = (TF)0, sz = (TF)0;    // FP64 path: double; refinement mode: FP32
    up_tile<T, TF, FINE, NS>(L, C, upre, f, uc, upost, mr, blockIdx.x, blockIdx.y, sf, su, srow, rz, sz);
    if (FINE) {
        __shared__ double red[2 * (NT / 32)];
        __shared__ float redf[2 * (NT / 32)];
        double brz, bsz;
        block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
        const int nb = gridDim.x * gridDim.y;
        const int bid = blockIdx.x + gridDim.x * blockIdx.y;
        if (threadIdx.x == 0) {
            part_rz[bid] = brz;
            part_sz[bid] = bsz;
        }
        if (arrive_last_n(cnt, gridDim.x * gridDim.y)) {
            double RZ, SZ;
            sum_parts2_cg<NT>(part_rz, part_sz, nb, red, &RZ, &SZ);
            if (threadIdx.x == 0) {
                const int it = ictl[PI_IT];
                scal[PS_BETA] = (it == 0) ? 0.0 : RZ / scal[PS_RZ];
                scal[PS_RZ] = RZ;
                scal[PS_MEANZ] = SZ / (double)L.N;
                *cnt = 0u;
            }
        }
    }
}

// CG direction and operator on the tile (bx, by): p = (z - mz) + beta p_old
// (double-buffered by the iteration parity it), q = A p; p.q over the tile's
// cells is added to acc.  sp (SY x 32) is the caller's shared array.
template <class T, class V>
__device__ __forceinline__ void pq_tile(const LvT<V>& L, const T* __restrict__ z, V* p0, V* p1, V* __restrict__ q,
                                        int it, V beta, V mz, int bx, int by, V (*sp)[32], V& acc) {
    __syncthreads();
    constexpr int H = 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V* pold = (it & 1) ? p0 : p1;
    V* pnew = (it & 1) ? p1 : p0;
    const int ox = bx * FP - H, oy = by * FP - H;
    const int nx = L.n[0];
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    Ax ayk[SY / NW];   // this thread's rows and p values (kept for the second pass)
    V pvk[SY / NW];
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        const Ax ay = axis(oy + r, L.n[1], L.per[1]);
        ayk[k] = ay;
        V pv = (V)0;
        if (ax.valid && ay.valid) {
            const int g = ax.gw + nx * ay.gw;
            pv = (V)z[g] - mz;
            if (it > 0) pv = fma(beta, pold[g], pv);
        }
        sp[r][lane] = pv;
        pvk[k] = pv;
    }
    __syncthreads();
    const bool colo = ax.in && lane >= H && lane < H + FP;
#pragma unroll
    for (int k = 0; k < SY / NW; ++k) {
        const int r = warp + NW * k;
        if (!colo || r < H || r >= H + FP) continue;
        const Ax ay = ayk[k];
        if (!ay.in) continue;
        const int g = ax.gw + nx * ay.gw;
        const V pv = pvk[k];
        const V off = L.w[0] * (sp[r][lane - 1] + sp[r][lane + 1]) + L.w[1] * (sp[r - 1][lane] + sp[r + 1][lane]);
        const V qv = L.diag[ax.cls + 3 * ay.cls] * pv - off;
        pnew[g] = pv;
        q[g] = qv;
        acc = fma(pv, qv, acc);
    }
}

template <class T, class V>
__global__ void __launch_bounds__(NT) pq(LvT<V> L, const T* __restrict__ z, V* p0, V* p1, V* __restrict__ q,
                                         double* part, double* scal, const int* ictl, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    {   // system of a batch
        const long long fb = blockIdx.z;
        z += fb * L.N;
        p0 += fb * L.N;
        p1 += fb * L.N;
        q += fb * L.N;
        part += fb * gridDim.x * gridDim.y;
        scal += fb * PS_NSCAL;
        ictl += fb * PI_NINT;
        cnt += fb * kNumCounters;
    }
    __shared__ V sp[SY][32];
    V acc = (V)0;
    pq_tile<T, V>(L, z, p0, p1, q, ictl[PI_IT], (V)scal[PS_BETA], (V)scal[PS_MEANZ], blockIdx.x, blockIdx.y, sp,
                  acc);
    __shared__ double red[NT / 32];
    __shared__ float redf[NT / 32];
    const double bacc = block_sum_any<NT>(acc, red, redf);
    const int nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) part[blockIdx.x + gridDim.x * blockIdx.y] = bacc;
    if (arrive_last_n(cnt, gridDim.x * gridDim.y)) {
        const double PQ = sum_parts_cg<NT>(part, nb, red);
        if (threadIdx.x == 0) {
            scal[PS_ALPHA] = scal[PS_RZ] / PQ;
            *cnt = 0u;
        }
    }
}

// Coarse levels top .. nlev-1 in one block; warps over rows, lanes over columns.
constexpr int TW = 16;            // warps of the tail block
constexpr int TT = 32 * TW;

template <class T>
__device__ __forceinline__ T off_c(const LvT<T>& L, const T* u, int i, int j, int* cls) {
    const int nx = L.n[0], ny = L.n[1], t = i + nx * j;
    T o = (T)0;
    if (i > 0) o += L.w[0] * u[t - 1];
    else if (L.per[0]) o += L.w[0] * u[t + nx - 1];
    if (i < nx - 1) o += L.w[0] * u[t + 1];
    else if (L.per[0]) o += L.w[0] * u[t - (nx - 1)];
    if (j > 0) o += L.w[1] * u[t - nx];
    else if (L.per[1]) o += L.w[1] * u[t + nx * (ny - 1)];
    if (j < ny - 1) o += L.w[1] * u[t + nx];
    else if (L.per[1]) o += L.w[1] * u[t - nx * (ny - 1)];
    *cls = (L.per[0] ? 2 : (int)(i > 0) + (int)(i < nx - 1)) + 3 * (L.per[1] ? 2 : (int)(j > 0) + (int)(j < ny - 1));
    return o;
}

template <class T>
__device__ __forceinline__ void tail_color(const LvT<T>& L, T* u, const T* f, int color) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = L.n[0], ny = L.n[1];
    for (int j = warp; j < ny; j += TW)
        for (int i = lane; i < nx; i += 32) {
            if (((i + j) & 1) != color) continue;
            int cl;
            const T o = off_c<T>(L, u, i, j, &cl);
            u[i + nx * j] = (f[i + nx * j] + o) * L.invd[cl];
        }
}

template <class T>
__global__ void __launch_bounds__(TT) tail(const LvT<T>* __restrict__ levs, TailArgs a, const T* __restrict__ f_top,
                                           T* __restrict__ u_top, const T* __restrict__ Minv) {
    pdl_wait();
    pdl_trigger();
    {   // system of a batch (one block each)
        const long long fb = blockIdx.x;
        f_top += fb * levs[a.top].N;
        u_top += fb * levs[a.top].N;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ LvT<T> lv[kMaxLevels];
    T* sm = reinterpret_cast<T*>(smraw);
    const int top = a.top, last = a.nlev - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const int words = (int)(sizeof(LvT<T>) / 4) * (last - top + 1);
        const unsigned int* src = reinterpret_cast<const unsigned int*>(levs + top);
        unsigned int* dst = reinterpret_cast<unsigned int*>(lv + top);
        for (int k = threadIdx.x; k < words; k += TT) dst[k] = src[k];
        const int N = levs[top].N;
        T* f = sm + a.off_f[top];
        for (int t = threadIdx.x; t < N; t += TT) f[t] = f_top[t];
    }
    __syncthreads();
    for (int l = top; l < last; ++l) {
        const LvT<T>& L = lv[l];
        const LvT<T>& C = lv[l + 1];
        const int nx = L.n[0], ny = L.n[1];
        T* u = sm + a.off_u[l];
        const T* f = sm + a.off_f[l];
        T* r = sm + a.off_r;
        T* fc = sm + a.off_f[l + 1];
        for (int j = warp; j < ny; j += TW)
            for (int i = lane; i < nx; i += 32) {
                const int cl = (L.per[0] ? 2 : (int)(i > 0) + (int)(i < nx - 1)) +
                               3 * (L.per[1] ? 2 : (int)(j > 0) + (int)(j < ny - 1));
                u[i + nx * j] = (((i + j) & 1) == 0) ? f[i + nx * j] * L.invd[cl] : (T)0;
            }
        __syncthreads();
        tail_color<T>(L, u, f, 1);
        __syncthreads();
        for (int j = warp; j < ny; j += TW)
            for (int i = lane; i < nx; i += 32) {
                int cl;
                const T o = off_c<T>(L, u, i, j, &cl);
                const int t = i + nx * j;
                r[t] = f[t] - (L.diag[cl] * u[t] - o);
            }
        __syncthreads();
        const int cx = C.n[0], cy = C.n[1];
        for (int J = warp; J < cy; J += TW)
            for (int I = lane; I < cx; I += 32) {
                T acc = (T)0;
#pragma unroll
                for (int ay = 0; ay < 4; ++ay) {
                    const T wy = (T)rweight(ay, J, cy, C.per[1]);
                    const int fy = wrapi(2 * J - 1 + ay, ny);
#pragma unroll
                    for (int axx = 0; axx < 4; ++axx) {
                        const T wx = (T)rweight(axx, I, cx, C.per[0]);
                        const int fx = wrapi(2 * I - 1 + axx, nx);
                        acc += wy * wx * ((wx != (T)0 && wy != (T)0) ? r[fx + nx * fy] : (T)0);
                    }
                }
                fc[I + cx * J] = acc * (T)0.25;
            }
        __syncthreads();
    }
    {
        const int Nc = a.Nc;
        const T* f = sm + a.off_f[last];
        T* u = sm + a.off_u[last];
        for (int i = threadIdx.x; i < Nc; i += TT) {
            T acc = (T)0;
            const T* row = Minv + (size_t)i * Nc;
            for (int j = 0; j < Nc; ++j) acc += row[j] * f[j];
            u[i] = acc;
        }
    }
    __syncthreads();
    for (int l = last - 1; l >= top; --l) {
        const LvT<T>& L = lv[l];
        const LvT<T>& C = lv[l + 1];
        const int nx = L.n[0], ny = L.n[1];
        T* u = sm + a.off_u[l];
        const T* f = sm + a.off_f[l];
        const T* uc = sm + a.off_u[l + 1];
        const T pa = (T)0.75, pb = (T)0.25;
        for (int j = warp; j < ny; j += TW) {
            int J0, J1;
            pro_pair(j, C.n[1], C.per[1], &J0, &J1);
            for (int i = lane; i < nx; i += 32) {
                int I0, I1;
                pro_pair(i, C.n[0], C.per[0], &I0, &I1);
                const T* c0 = uc + C.n[0] * J0;
                const T* c1 = uc + C.n[0] * J1;
                u[i + nx * j] += pa * (pa * c0[I0] + pb * c0[I1]) + pb * (pa * c1[I0] + pb * c1[I1]);
            }
        }
        __syncthreads();
        tail_color<T>(L, u, f, 1);
        __syncthreads();
        tail_color<T>(L, u, f, 0);
        __syncthreads();
    }
    {
        const int N = lv[top].N;
        const T* u = sm + a.off_u[top];
        for (int t = threadIdx.x; t < N; t += TT) u_top[t] = u[t];
    }
}

// Exact solve on the top coarse level by fast diagonalisation (Lynch, Rice &
// Thomas): the level operator is A = Ax (x) I + I (x) Ay with 1D second-difference
// matrices Ad = Sd diag(lam_d) Sd^T, so the zero-mean solution of A u = f is
//   u = Sy [ (Sy^T F Sx) .* IL ] Sx^T,   IL[l][k] = 1 / (lam_y,l + lam_x,k) (0 for the null mode),
// four small dense products in shared memory.  F, u: ny rows of nx values.
constexpr int FT = 256;            // threads of the fast-diagonalisation block

// C[M x N] = LT^T R with LT[K x M] (leading dimension ldl) and R[K x N]
// (leading dimension N), row-major; each thread a 2 x 4 tile: per k one float2
// load of LT and one float4 load of R (no bank conflicts: a warp's float2 loads
// fall on at most four consecutive pairs); optionally C .*= S.  The sum over k
// runs in ascending order with one fmaf per term.  N % 4 == 0, M even.
__device__ __forceinline__ void mmT(float* __restrict__ C, const float* __restrict__ LT, int ldl,
                                    const float* __restrict__ R, int M, int N, int K, const float* __restrict__ S,
                                    int nthreads = FT) {
    const int tn = N / 4;
    for (int tile = threadIdx.x; tile < (M / 2) * tn; tile += nthreads) {
        const int m0 = 2 * (tile / tn), n0 = 4 * (tile % tn);
        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
#pragma unroll 8
        for (int k = 0; k < K; ++k) {
            const float2 a = *reinterpret_cast<const float2*>(LT + k * ldl + m0);
            const float4 r = *reinterpret_cast<const float4*>(R + k * N + n0);
            c0.x = fmaf(a.x, r.x, c0.x);
            c0.y = fmaf(a.x, r.y, c0.y);
            c0.z = fmaf(a.x, r.z, c0.z);
            c0.w = fmaf(a.x, r.w, c0.w);
            c1.x = fmaf(a.y, r.x, c1.x);
            c1.y = fmaf(a.y, r.y, c1.y);
            c1.z = fmaf(a.y, r.z, c1.z);
            c1.w = fmaf(a.y, r.w, c1.w);
        }
        if (S) {
            const float4 s0 = *reinterpret_cast<const float4*>(S + m0 * N + n0);
            const float4 s1 = *reinterpret_cast<const float4*>(S + (m0 + 1) * N + n0);
            c0.x *= s0.x; c0.y *= s0.y; c0.z *= s0.z; c0.w *= s0.w;
            c1.x *= s1.x; c1.y *= s1.y; c1.z *= s1.z; c1.w *= s1.w;
        }
        *reinterpret_cast<float4*>(C + m0 * N + n0) = c0;
        *reinterpret_cast<float4*>(C + (m0 + 1) * N + n0) = c1;
    }
}

// Asynchronous global -> shared copies (no registers held while in flight).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__host__ __device__ constexpr int fdm_ldf(int ny) { return ny + 2; }   // row stride of F^T in shared (2-way store conflicts)
__host__ __device__ constexpr long long fdm_smem_floats(long long nx, long long ny) {
    return 2 * nx * nx + 2 * ny * ny + nx * ny + nx * fdm_ldf((int)ny) + nx * ny;
}

// Shared-memory layout (floats): Sx, SxT (nx*nx each), Sy, SyT (ny*ny each),
// IL (ny*nx) -- the global table, copied linearly -- then X (nx rows of
// ny + 2) and Y (nx*ny).  With C = LT^T R the four products are
//   Y = F Sx                   (LT = F^T in X, R = Sx)
//   X = (Sy^T Y) .* IL         (LT = Sy,       R = Y)
//   Y = (Sy X)^T = X^T Sy^T    (LT = X,        R = SyT)
//   u = Y^T Sx^T               (LT = Y,        R = SxT), written straight to global;
// fdm_smem_floats is the total.
// The table does not depend on the previous kernel, so its copy is issued
// before the programmatic-dependency wait.
__global__ void __launch_bounds__(FT) fdm(int nx, int ny, const float* __restrict__ tab, const float* __restrict__ f,
                                          float* __restrict__ u) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* Sx = reinterpret_cast<float*>(smraw);
    float* SxT = Sx + nx * nx;
    float* Sy = SxT + nx * nx;
    float* SyT = Sy + ny * ny;
    float* IL = SyT + ny * ny;
    float* X = IL + nx * ny;
    float* Y = X + nx * fdm_ldf(ny);
    const int ntab = 2 * nx * nx + 2 * ny * ny + nx * ny;     // a multiple of 4 (nx % 4 == 0, ny % 4 == 0)
    for (int i = threadIdx.x; i < ntab / 4; i += FT) cp_async16(Sx + 4 * i, tab + 4 * i);
    pdl_wait();
    pdl_trigger();
    f += (long long)blockIdx.x * nx * ny;   // system of a batch (one block each)
    u += (long long)blockIdx.x * nx * ny;
    const int ldf = fdm_ldf(ny);
    for (int i = threadIdx.x; i < nx * ny; i += FT) {
        const int y = i / nx, x = i - y * nx;
        cp_async4(X + x * ldf + y, f + i);
    }
    cp_async_wait_all();
    __syncthreads();
    mmT(Y, X, ldf, Sx, ny, nx, nx, nullptr);
    __syncthreads();
    mmT(X, Sy, ny, Y, ny, nx, ny, IL);
    __syncthreads();
    mmT(Y, X, nx, SyT, nx, ny, ny, nullptr);
    __syncthreads();
    mmT(u, Y, ny, SxT, ny, nx, nx, nullptr);
}

}  // namespace k2

// ---------------------------------------------------------------------------
// Persistent 2D solve.  A small 2D system (the 256 x 512 flame: about 15 CG
// iterations per step, each a chain of nine short kernels) is bound by launch
// and drain latency, not by its bytes.  Here the whole solve -- the mean of
// b, r = f - A x, then every CG iteration (the V(2,2) cycle's down sweeps,
// the fast-diagonalisation top level, the up sweeps with r.z, the direction
// and operator p, q, and the reliable update of x and r) -- runs in one
// cooperative launch whose blocks are all resident.  Each phase spreads the
// level's tiles (or cells) over the blocks and ends at a grid barrier; a
// phase that ends in a reduction finishes it in the last block to arrive,
// which sums the blocks' partials in index order (deterministic) and writes
// the scalars before releasing the others.  Every wait is bounded: a block
// that waits longer than kSpin polls raises the abort word, which ends every
// block at its next barrier, and the solve reports non-convergence.
// ---------------------------------------------------------------------------
namespace kp {

constexpr int kLev = 6;                  // levels 0 .. top handled
constexpr unsigned kSpin = 1u << 22;     // polls of a waiting block (about a second)
// barrier words in a scratch array of their own, on separate 128-byte lines (the
// arrival counter, the generation the waiting blocks poll, the abort flag)
enum { BAR_COUNT = 0, BAR_GEN = 32, BAR_ABORT = 64, BAR_WORDS = 96 };

struct Args {
    LvT<float> lev[kLev];   // FP32 level descriptors 0 .. top
    LvT<double> L0;          // the fine level in FP64 (residual and reliable update)
    int top;
    int dtx[kLev], dty[kLev];   // down tiles of level l (its coarse tile grid)
    int utx[kLev], uty[kLev];   // up tiles of level l
    int ptx, pty;               // operator tiles of the fine level
    const double* b;
    double* x;
    double* r;
    float* r32;
    float* u0pre;
    float* z;
    float* upre[kLev];
    float* f[kLev];
    float* upost[kLev];
    float* p0;
    float* p1;
    float* q;
    const float* fdm_tab;
    double* part;               // 3 x gridDim.x partial sums
    double* scal;
    int* ictl;
    unsigned* bar;              // barrier words (BAR_*)
    double rtol;
    int max_iter;
    int vec4;
    int mean_ready;
    unsigned arrivals;          // blocks a barrier waits for (gridDim.x)
    unsigned spin;              // polls before a waiting block gives up
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier.  Every block arrives once; the last one runs fin() with all
// its threads (the other blocks' partials are visible to it: their arrivals
// release, its own acquires), then releases the generation word, which the
// waiting blocks acquire.  Returns false once the solve has been aborted.
__device__ __forceinline__ void st_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <class Fin>
__device__ __forceinline__ bool barrier(const Args& a, Fin fin) {
    __shared__ int s_last, s_ok;
    unsigned* cnt = a.bar + BAR_COUNT;
    unsigned* gen = a.bar + BAR_GEN;
    int* abort = reinterpret_cast<int*>(a.bar + BAR_ABORT);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        s_last = 0;
        const unsigned g0 = ld_acquire_u32(gen);
        const unsigned arrived = atomic_add_acq_rel_gpu(cnt, 1u);
        if (arrived == a.arrivals - 1u) {
            s_last = 1;
        } else {
            unsigned n = 0;
            while (ld_relaxed_u32(gen) == g0) {
                if ((++n & 255u) == 0u) {
                    if (ld_relaxed_i32(abort)) {
                        s_ok = 0;
                        break;
                    }
                    if (n > a.spin) {
                        atomicExch(abort, 1);
                        a.ictl[PI_NOCONV] = 1;
                        a.ictl[PI_DONE] = 1;
                        s_ok = 0;
                        break;
                    }
                }
            }
            fence_acq_rel_gpu();   // the released writes are visible from here on
        }
    }
    __syncthreads();
    if (s_last) {
        fin();
        __syncthreads();
        if (threadIdx.x == 0) {
            *cnt = 0u;
            fence_acq_rel_gpu();
            atomicAdd(gen, 1u);
        }
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void no_fin() {}

// Fast-diagonalisation solve of the top level by one block (all its threads):
// the table and f staged in shared memory, then the four products.
__device__ void fdm_block(int nx, int ny, const float* __restrict__ tab, const float* __restrict__ f,
                          float* __restrict__ u, float* sm) {
    float* Sx = sm;
    float* SxT = Sx + nx * nx;
    float* Sy = SxT + nx * nx;
    float* SyT = Sy + ny * ny;
    float* IL = SyT + ny * ny;
    float* X = IL + nx * ny;
    float* Y = X + nx * k2::fdm_ldf(ny);
    const int ntab = 2 * nx * nx + 2 * ny * ny + nx * ny;
    for (int i = threadIdx.x; i < ntab / 4; i += blockDim.x)
        reinterpret_cast<float4*>(Sx)[i] = __ldcg(reinterpret_cast<const float4*>(tab) + i);
    const int ldf = k2::fdm_ldf(ny);
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int y = i / nx, x = i - y * nx;
        X[x * ldf + y] = __ldcg(f + i);
    }
    __syncthreads();
    k2::mmT(Y, X, ldf, Sx, ny, nx, nx, nullptr, blockDim.x);
    __syncthreads();
    k2::mmT(X, Sy, ny, Y, ny, nx, ny, IL, blockDim.x);
    __syncthreads();
    k2::mmT(Y, X, nx, SyT, nx, ny, ny, nullptr, blockDim.x);
    __syncthreads();
    k2::mmT(u, Y, ny, SxT, ny, nx, nx, nullptr, blockDim.x);
}

__global__ void __launch_bounds__(k2::NT, 2) k_solve2(const __grid_constant__ Args a) {
    using namespace k2;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float sf[SY][32];
    __shared__ float su[SY][32];
    __shared__ int srow[SY];
    __shared__ double red[2 * (NT / 32)];
    __shared__ float redf[2 * (NT / 32)];
    const int nb = gridDim.x, bi = blockIdx.x, tid = threadIdx.x;
    double* P0 = a.part;
    double* P1 = a.part + nb;
    double* P2 = a.part + 2 * nb;
    double* scal = a.scal;
    int* ictl = a.ictl;
    const int N = a.L0.N;
    const int c0 = bi * NT + tid, cs = nb * NT;

    // mean of b (unless the right-hand side's kernel left it)
    if (!a.mean_ready) {
        double acc = 0.0;
        for (int t = c0; t < N; t += cs) acc += a.b[t];
        acc = block_sum<NT>(acc, red);
        if (tid == 0) P0[bi] = acc;
        if (!barrier(a, [&] {
                const double S = sum_parts_cg<NT>(P0, nb, red);
                if (tid == 0) scal[PS_MEANB] = S / (double)N;
            }))
            return;
    }
    // r = -(b - mean b) - A x; ||f||^2, ||r||^2, sum r; the control words
    {
        double ff = 0.0, rr = 0.0, sr = 0.0;
        init_cells<2>(a.L0, a.b, a.x, a.r, a.r32, __ldcg(scal + PS_MEANB), c0, cs, ff, rr, sr);
        block_sum2_t<NT, double>(ff, rr, red);
        sr = block_sum<NT>(sr, red);
        if (tid == 0) {
            P0[bi] = ff;
            P1[bi] = rr;
            P2[bi] = sr;
        }
        if (!barrier(a, [&] {
                double FF, RR;
                sum_parts2_cg<NT>(P0, P1, nb, red, &FF, &RR);
                const double SR = sum_parts_cg<NT>(P2, nb, red);
                if (tid == 0) {
                    scal[PS_FF] = FF;
                    scal[PS_RR] = RR;
                    scal[PS_MEANR] = SR / (double)N;
                    scal[PS_RZ] = 0.0;
                    scal[PS_BETA] = 0.0;
                    scal[PS_ITERS] = 0.0;
                    ictl[PI_IT] = 0;
                    ictl[PI_TOTAL] = 0;
                    ictl[PI_NOCONV] = 0;
                    const int zero = !(FF > 0.0);
                    ictl[PI_ZERO] = zero;
                    int done = zero || (RR <= a.rtol * a.rtol * FF);
                    scal[PS_RELRES] = zero ? 0.0 : sqrt(RR / FF);
                    if (!(RR == RR)) {
                        done = 1;
                        ictl[PI_NOCONV] = 1;
                    }
                    ictl[PI_DONE] = done;
                }
            }))
            return;
    }
    for (;;) {
        if (__ldcg(ictl + PI_DONE)) break;
        const int it = __ldcg(ictl + PI_IT);
        const float mr = (float)__ldcg(scal + PS_MEANR);
        // down sweeps of levels 0 .. top-1
        for (int l = 0; l < a.top; ++l) {
            const int nt = a.dtx[l] * a.dty[l];
            for (int t = bi; t < nt; t += nb) {
                const int tx = t % a.dtx[l], ty = t / a.dtx[l];
                if (l == 0)
                    down_tile<float, float, 2>(a.lev[0], a.lev[1], a.r32, a.u0pre, a.f[1], mr, tx, ty, sf, su, srow);
                else
                    down_tile<float, float, 2>(a.lev[l], a.lev[l + 1], a.f[l], a.upre[l], a.f[l + 1], 0.0f, tx, ty,
                                               sf, su, srow);
            }
            if (!barrier(a, no_fin)) return;
        }
        // the top level, exactly
        if (bi == 0)
            fdm_block(a.lev[a.top].n[0], a.lev[a.top].n[1], a.fdm_tab, a.f[a.top], a.upost[a.top],
                      reinterpret_cast<float*>(smraw));
        if (!barrier(a, no_fin)) return;
        // up sweeps of levels top-1 .. 1
        for (int l = a.top - 1; l >= 1; --l) {
            const int nt = a.utx[l] * a.uty[l];
            float rz = 0.0f, sz = 0.0f;
            for (int t = bi; t < nt; t += nb) {
                const int tx = t % a.utx[l], ty = t / a.utx[l];
                up_tile<float, float, false, 2>(a.lev[l], a.lev[l + 1], a.upre[l], a.f[l], a.upost[l + 1],
                                                a.upost[l], 0.0f, tx, ty, sf, su, srow, rz, sz);
            }
            if (!barrier(a, no_fin)) return;
        }
        // the fine level's up sweep with r.z and sum z
        {
            const int nt = a.utx[0] * a.uty[0];
            float rz = 0.0f, sz = 0.0f;
            for (int t = bi; t < nt; t += nb) {
                const int tx = t % a.utx[0], ty = t / a.utx[0];
                up_tile<float, float, true, 2>(a.lev[0], a.lev[1], a.u0pre, a.r32, a.upost[1], a.z, mr, tx, ty, sf,
                                               su, srow, rz, sz);
            }
            double brz, bsz;
            block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
            if (tid == 0) {
                P0[bi] = brz;
                P1[bi] = bsz;
            }
            if (!barrier(a, [&] {
                    double RZ, SZ;
                    sum_parts2_cg<NT>(P0, P1, nb, red, &RZ, &SZ);
                    if (tid == 0) {
                        scal[PS_BETA] = (it == 0) ? 0.0 : RZ / __ldcg(scal + PS_RZ);
                        scal[PS_RZ] = RZ;
                        scal[PS_MEANZ] = SZ / (double)N;
                    }
                }))
                return;
        }
        // p = (z - mean z) + beta p_old, q = A p, p.q
        {
            const float beta = (float)__ldcg(scal + PS_BETA), mz = (float)__ldcg(scal + PS_MEANZ);
            const int nt = a.ptx * a.pty;
            float acc = 0.0f;
            for (int t = bi; t < nt; t += nb) {
                const int tx = t % a.ptx, ty = t / a.ptx;
                pq_tile<float, float>(a.lev[0], a.z, a.p0, a.p1, a.q, it, beta, mz, tx, ty, sf, acc);
            }
            const double bacc = block_sum_any<NT>(acc, red, redf);
            if (tid == 0) P0[bi] = bacc;
            if (!barrier(a, [&] {
                    const double PQ = sum_parts_cg<NT>(P0, nb, red);
                    if (tid == 0) scal[PS_ALPHA] = __ldcg(scal + PS_RZ) / PQ;
                }))
                return;
        }
        // reliable update: x += e, r64 -= A e (e = alpha p), r32 = r64; the stopping test
        {
            const float alpha = (float)__ldcg(scal + PS_ALPHA);
            const float* p = (it & 1) ? a.p1 : a.p0;
            double rr = 0.0, sr = 0.0;
            // each block a contiguous chunk of the cells (quads), so every SM works
            const int nu = a.vec4 ? (N >> 2) : N, chunk = (nu + nb - 1) / nb;
            ir_cells<2>(a.L0, a.x, a.r, p, a.r32, alpha, a.vec4, bi * chunk + tid, NT, (bi + 1) * chunk, rr, sr);
            block_sum2_t<NT, double>(rr, sr, red);
            if (tid == 0) {
                P0[bi] = rr;
                P1[bi] = sr;
            }
            if (!barrier(a, [&] {
                    double RR, SR;
                    sum_parts2_cg<NT>(P0, P1, nb, red, &RR, &SR);
                    if (tid == 0) {
                        scal[PS_MEANR] = SR / (double)N;
                        const int tot = __ldcg(ictl + PI_TOTAL) + 1;
                        ictl[PI_IT] = it + 1;
                        ictl[PI_TOTAL] = tot;
                        scal[PS_ITERS] = (double)tot;
                        const double ff = __ldcg(scal + PS_FF);
                        const int conv = (RR <= a.rtol * a.rtol * ff);
                        const int bad = !(RR == RR) || !(RR < 1e300);
                        const int done = conv || bad || (tot >= a.max_iter);
                        scal[PS_RR] = RR;
                        scal[PS_RELRES] = sqrt(RR / ff);
                        ictl[PI_DONE] = done;
                        if (done && !conv) ictl[PI_NOCONV] = 1;
                    }
                }))
                return;
        }
    }
}

}  // namespace kp

// ---------------------------------------------------------------------------
// 3D kernels, z-marching ("2.5D"): a block owns a 32-column x 32-row box in
// x-y (lane = column, each warp two rows) and marches through a chunk of
// z-planes, keeping rings of 4 planes in shared memory.  The x-y halo is
// recomputed by neighbouring blocks; the z-halo only at the ends of a chunk.
// Per-cell arithmetic as in the tile kernels above (same smoother, residual,
// restriction and prolongation formulas).
// ---------------------------------------------------------------------------
namespace k3 {

using k2::Ax;
// The 3D kernels keep the plain modulo wrap: with the 2D kernels' single-wrap
// form ptxas allocated 40 instead of 49-52 registers to the z-marching up and
// pq, which then ran 2-5% slower.
__device__ __forceinline__ Ax axis(int g, int n, int per) {
    Ax a;
    a.in = (g >= 0 && g < n);
    a.gw = a.in ? g : (per ? wrapi(g, n) : 0);
    a.valid = a.in || per;
    a.cls = per ? 2 : (int)(a.gw > 0) + (int)(a.gw < n - 1);
    return a;
}
constexpr int NW = 16;            // warps per block
constexpr int NT = 32 * NW;
constexpr int SB = 32;            // box rows and columns
constexpr int FD = 26, CD = 13;   // down: fine tile (halo 3), coarse tile
constexpr int FU = 28;            // up: fine tile (halo 2)
constexpr int FP = 30;            // pq: tile (halo 1)
constexpr int KC = 8;             // down: coarse planes per block
constexpr int ZU = 16;            // up, pq: fine planes per block
constexpr int RING = 4;

template <class T>
using Pl = T[SB][SB];

template <class T>
__device__ __forceinline__ T off3(const LvT<T>& L, const Pl<T>* su, int sm, int s0, int sp, int r, int c) {
    T off = L.w[0] * (su[s0][r][c - 1] + su[s0][r][c + 1]) + L.w[1] * (su[s0][r - 1][c] + su[s0][r + 1][c]);
    off += L.w[2] * (su[sm][r][c] + su[sp][r][c]);
    return off;
}

// Per-block axis data of the box: the two columns a lane can take in a colour
// sweep (2 (lane & 15) and that + 1), and every row (shared), each as
// class | valid << 2 (valid: inside the domain or periodic).
struct BoxAxes {
    int col[2];
};
__device__ __forceinline__ int axis_code(int g, int n, int per) {
    const Ax a = axis(g, n, per);
    return a.cls | ((int)a.valid << 2);
}
template <class T>
__device__ __forceinline__ BoxAxes box_axes(const LvT<T>& L, int ox, int oy, int* srow) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < SB) srow[threadIdx.x] = axis_code(oy + (int)threadIdx.x, L.n[1], L.per[1]);
    BoxAxes b;
    b.col[0] = axis_code(ox + 2 * (lane & 15), L.n[0], L.per[0]);
    b.col[1] = axis_code(ox + 2 * (lane & 15) + 1, L.n[0], L.per[0]);
    return b;   // srow is read after the caller's next barrier
}

// One colour on plane z (ring slot z & 3) over rows [r0, r1] x columns [c0, c1].
template <class T>
__device__ __forceinline__ void color_plane(const LvT<T>& L, Pl<T>* su, const Pl<T>* sf, int ox, int oy, int z,
                                            int zcls, int color, int r0, int r1, int c0, int c1, const BoxAxes& ba,
                                            const int* srow) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int par = (ox + oy + z) & 1;
    const int s0 = z & 3, sm = (z - 1) & 3, sp = (z + 1) & 3;
    const int npairs = (r1 - r0 + 2) / 2;
    for (int rp = warp; rp < npairs; rp += NW) {
        const int r = r0 + 2 * rp + (lane >> 4);
        const int odd = (color - par - r) & 1;
        const int c = 2 * (lane & 15) + odd;
        if (r > r1 || c < c0 || c > c1) continue;
        const int cx = ba.col[odd], cy = srow[r];
        if (!((cx & cy) & 4)) continue;
        su[s0][r][c] = (sf[s0][r][c] + off3<T>(L, su, sm, s0, sp, r, c)) * L.invd[(cx & 3) + 3 * (cy & 3) + 9 * zcls];
    }
}

// down: red from zero, black, residual, restriction.  Block (bx, by, bz): the
// coarse tile CD x CD of columns / rows and coarse planes [K0, K1).
template <class T, class TF>
__global__ void __launch_bounds__(NT) down(LvT<T> L, LvT<T> C, const TF* __restrict__ f, T* __restrict__ upre,
                                           T* __restrict__ fc, const double* __restrict__ scal_r) {
    pdl_wait();
    pdl_trigger();
    // fine level: the CG residual enters the preconditioner with its mean removed
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    constexpr int H = 3;
    extern __shared__ __align__(16) unsigned char smraw[];
    Pl<T>* sF = reinterpret_cast<Pl<T>*>(smraw);
    Pl<T>* sU = sF + RING;
    Pl<T>* sR = sU + RING;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ox = blockIdx.x * FD - H, oy = blockIdx.y * FD - H;
    const int K0 = blockIdx.z * KC;
    const int K1 = min(K0 + KC, C.n[2]);
    const int zs = 2 * K0 - 3, ze = 2 * K1 + 2;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const long long nxy = (long long)nx * ny;
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    Ax ay[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) ay[k] = axis(oy + warp + NW * k, ny, L.per[1]);
    const bool colo = ax.in && lane >= H && lane < H + FD;
    __shared__ int srow[SB];
    const BoxAxes ba = box_axes<T>(L, ox, oy, srow);
    // restriction weights of this thread's coarse cell (fixed across planes)
    const int rcx = threadIdx.x % CD, rcy = threadIdx.x / CD;
    const int rI = blockIdx.x * CD + rcx, rJ = blockIdx.y * CD + rcy;
    const bool rown = threadIdx.x < CD * CD && rI < C.n[0] && rJ < C.n[1];
    T wxr[4], wyr[4];
#pragma unroll
    for (int a4 = 0; a4 < 4; ++a4) {
        wxr[a4] = (T)rweight(a4, rI, C.n[0], C.per[0]);
        wyr[a4] = (T)rweight(a4, rJ, C.n[1], C.per[1]);
    }
    // the next plane's f is loaded one step ahead (its DRAM latency overlaps
    // the current plane's sweeps)
    TF fpre[2];
    auto load_f = [&](int qz) {
        const Ax az = axis(qz, nz, L.per[2]);
#pragma unroll
        for (int k = 0; k < 2; ++k)
            fpre[k] = (ax.valid && ay[k].valid && az.valid) ? (TF)(f[ax.gw + (long long)nx * ay[k].gw + nxy * az.gw] - mr)
                                                            : (TF)0;
    };
    load_f(zs);

    for (int q = zs; q <= ze; ++q) {
        // (a) f and the red cells of u (from a zero guess) on plane q
        {
            const Ax az = axis(q, nz, L.per[2]);
            const int sl = q & 3;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + NW * k;
                T fv = (T)0, uv = (T)0;
                if (ax.valid && ay[k].valid && az.valid) {
                    fv = (T)fpre[k];
                    if (((ox + lane + oy + r + q) & 1) == 0) uv = fv * L.invd[ax.cls + 3 * ay[k].cls + 9 * az.cls];
                }
                sF[sl][r][lane] = fv;
                sU[sl][r][lane] = uv;
            }
        }
        if (q < ze) load_f(q + 1);
        __syncthreads();
        // (b) black on plane q-1, box minus one layer
        {
            const int z = q - 1;
            if (z >= zs + 1 && z <= ze - 1) {
                const Ax az = axis(z, nz, L.per[2]);
                if (az.valid) color_plane<T>(L, sU, sF, ox, oy, z, az.cls, 1, 1, SB - 2, 1, SB - 2, ba, srow);
            }
        }
        __syncthreads();
        // (c) residual on plane q-2, box minus two layers; u of the owned cells
        const int pr = q - 2;
        if (pr >= zs + 2 && pr <= ze - 2) {
            const Ax az = axis(pr, nz, L.per[2]);
            const int s0 = pr & 3, sm = (pr - 1) & 3, sp = (pr + 1) & 3;
            const bool zown = az.in && pr >= 2 * K0 && pr < 2 * K1;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + NW * k;
                T rv = (T)0;
                if (r >= 2 && r <= SB - 3 && lane >= 2 && lane <= SB - 3 && ax.valid && ay[k].valid && az.valid) {
                    const T u = sU[s0][r][lane];
                    rv = sF[s0][r][lane] -
                         (L.diag[ax.cls + 3 * ay[k].cls + 9 * az.cls] * u - off3<T>(L, sU, sm, s0, sp, r, lane));
                    if (zown && colo && ay[k].in && r >= H && r < H + FD)
                        upre[ax.gw + (long long)nx * ay[k].gw + nxy * az.gw] = u;
                }
                sR[s0][r][lane] = rv;
            }
        }
        __syncthreads();
        // (d) restriction of coarse plane K = (pr - 2) / 2 once its fine planes
        // 2K-1 .. 2K+2 are in the residual ring
        if (pr >= 2 * K0 + 2 && pr <= 2 * K1 && ((pr & 1) == 0) && rown) {
            const int K = (pr - 2) / 2;
            T acc = (T)0;
#pragma unroll
            for (int az = 0; az < 4; ++az) {
                const T wz = (T)rweight(az, K, C.n[2], C.per[2]);
                const int sl = (2 * K - 1 + az) & 3;
#pragma unroll
                for (int ayy = 0; ayy < 4; ++ayy) {
                    const int r = 2 * rcy + H - 1 + ayy;
                    T row = (T)0;
#pragma unroll
                    for (int axx = 0; axx < 4; ++axx) row += wxr[axx] * sR[sl][r][2 * rcx + H - 1 + axx];
                    acc += wz * wyr[ayy] * row;
                }
            }
            fc[rI + C.n[0] * (rJ + (long long)C.n[1] * K)] = acc * (T)0.125;
        }
    }
}

// up: prolongation-add, black, red; on the fine level also the partial sums
// of r.z and sum z (finished by the last block).  Block (bx, by, bz): the fine
// tile FU x FU and fine planes [z0, z1).
template <class T, class TF, bool FINE>
__global__ void __launch_bounds__(NT)
    up(LvT<T> L, LvT<T> C, const T* __restrict__ upre, const TF* __restrict__ f, const T* __restrict__ uc,
       T* __restrict__ upost, double* part_rz, double* part_sz, double* scal, const int* ictl, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    const TF mr = FINE ? (TF)scal[PS_MEANR] : (TF)0;   // fine level: residual mean removed
    constexpr int H = 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    Pl<T>* sF = reinterpret_cast<Pl<T>*>(smraw);
    Pl<T>* sU = sF + RING;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ox = blockIdx.x * FU - H, oy = blockIdx.y * FU - H;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int z0 = blockIdx.z * ZU, z1 = min(z0 + ZU, nz);
    const long long nxy = (long long)nx * ny;
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    Ax ay[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) ay[k] = axis(oy + warp + NW * k, ny, L.per[1]);
    const bool colo = ax.in && lane >= H && lane < H + FU;
    __shared__ int srow[SB];
    const BoxAxes ba = box_axes<T>(L, ox, oy, srow);
    TF rz = (TF)0, sz = (TF)0;
    // the next plane's f and u_pre are loaded one step ahead
    TF fpre[2];
    T upre_n[2];
    auto load_fu = [&](int qz) {
        const Ax az = axis(qz, nz, L.per[2]);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool v = ax.valid && ay[k].valid && az.valid;
            const long long g = ax.gw + (long long)nx * ay[k].gw + nxy * az.gw;
            fpre[k] = v ? (TF)(f[g] - mr) : (TF)0;
            upre_n[k] = v ? upre[g] : (T)0;
        }
    };
    load_fu(z0 - 2);

    for (int q = z0 - 2; q <= z1 + 1; ++q) {
        // (a) f and u = u_pre + P u_coarse on plane q
        {
            const Ax az = axis(q, nz, L.per[2]);
            const int sl = q & 3;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + NW * k;
                T fv = (T)0, uv = (T)0;
                if (ax.valid && ay[k].valid && az.valid) {
                    fv = (T)fpre[k];
                    const int gw[3] = {ax.gw, ay[k].gw, az.gw};
                    uv = upre_n[k] + prolong_at<T, 3>(C, uc, gw);
                }
                sF[sl][r][lane] = fv;
                sU[sl][r][lane] = uv;
            }
        }
        if (q < z1 + 1) load_fu(q + 1);
        __syncthreads();
        // (b) black on plane q-1, box minus one layer
        {
            const int z = q - 1;
            if (z >= z0 - 1 && z <= z1) {
                const Ax az = axis(z, nz, L.per[2]);
                if (az.valid) color_plane<T>(L, sU, sF, ox, oy, z, az.cls, 1, 1, SB - 2, 1, SB - 2, ba, srow);
            }
        }
        __syncthreads();
        // (c) red on plane q-2 over the tile
        {
            const int z = q - 2;
            if (z >= z0 && z < z1) {
                const Ax az = axis(z, nz, L.per[2]);
                if (az.valid) color_plane<T>(L, sU, sF, ox, oy, z, az.cls, 0, H, SB - 1 - H, H, SB - 1 - H, ba, srow);
            }
        }
        __syncthreads();
        // (d) store the owned cells of plane q-2
        {
            const int z = q - 2;
            if (z >= z0 && z < z1) {
                const int sl = z & 3;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int r = warp + NW * k;
                    if (!colo || !ay[k].in || r < H || r >= H + FU) continue;
                    const long long g = ax.gw + (long long)nx * ay[k].gw + nxy * z;
                    const T u = sU[sl][r][lane];
                    upost[g] = u;
                    if (FINE) {
                        // plane z's f is still in the ring, exactly, when T and TF agree
                        const TF fv = (sizeof(T) == sizeof(TF)) ? (TF)sF[sl][r][lane] : (TF)(f[g] - mr);
                        rz = fma(fv, (TF)u, rz);
                        sz += (TF)u;
                    }
                }
            }
        }
    }
    if (FINE) {
        __shared__ double red[2 * (NT / 32)];
        __shared__ float redf[2 * (NT / 32)];
        double brz, bsz;
        block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (threadIdx.x == 0) {
            part_rz[block_linear()] = brz;
            part_sz[block_linear()] = bsz;
        }
        if (arrive_last(cnt)) {
            double RZ, SZ;
            sum_parts2_cg<NT>(part_rz, part_sz, nb, red, &RZ, &SZ);
            if (threadIdx.x == 0) {
                const int it = ictl[PI_IT];
                scal[PS_BETA] = (it == 0) ? 0.0 : RZ / scal[PS_RZ];
                scal[PS_RZ] = RZ;
                scal[PS_MEANZ] = SZ / (double)L.N;
                *cnt = 0u;
            }
        }
    }
}

// CG: p = (z - mean z) + beta p_old (p_new buffer by parity), q = A p, p.q;
// the last block forms alpha = r.z / p.q.  Tile FP x FP, fine planes [z0, z1).
// One barrier per plane: the plane written at step qq + 1 (slot qq - 3) is not
// read at step qq.
template <class T, class V>
__global__ void __launch_bounds__(NT) pq(LvT<V> L, const T* __restrict__ z, V* p0, V* p1, V* __restrict__ q,
                                         double* part, double* scal, const int* ictl, unsigned int* cnt) {
    pdl_wait();
    pdl_trigger();
    constexpr int H = 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    Pl<V>* sP = reinterpret_cast<Pl<V>*>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int it = ictl[PI_IT];
    const V* pold = (it & 1) ? p0 : p1;
    V* pnew = (it & 1) ? p1 : p0;
    const V beta = (V)scal[PS_BETA], mz = (V)scal[PS_MEANZ];
    const int ox = blockIdx.x * FP - H, oy = blockIdx.y * FP - H;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int z0 = blockIdx.z * ZU, z1 = min(z0 + ZU, nz);
    const long long nxy = (long long)nx * ny;
    const Ax ax = axis(ox + lane, nx, L.per[0]);
    Ax ay[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) ay[k] = axis(oy + warp + NW * k, ny, L.per[1]);
    const bool colo = ax.in && lane >= H && lane < H + FP;
    V acc = (V)0;
    // the next plane's z and p_old are loaded one step ahead
    T zpre[2];
    V ppre[2];
    auto load_zp = [&](int qz) {
        const Ax az = axis(qz, nz, L.per[2]);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool v = ax.valid && ay[k].valid && az.valid;
            const long long g = ax.gw + (long long)nx * ay[k].gw + nxy * az.gw;
            zpre[k] = v ? z[g] : (T)0;
            ppre[k] = (v && it > 0) ? pold[g] : (V)0;
        }
    };
    load_zp(z0 - 1);
    for (int qq = z0 - 1; qq <= z1; ++qq) {
        {
            const Ax az = axis(qq, nz, L.per[2]);
            const int sl = qq & 3;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + NW * k;
                V pv = (V)0;
                if (ax.valid && ay[k].valid && az.valid) {
                    pv = (V)zpre[k] - mz;
                    if (it > 0) pv = fma(beta, ppre[k], pv);
                }
                sP[sl][r][lane] = pv;
            }
        }
        if (qq < z1) load_zp(qq + 1);
        __syncthreads();
        const int zc = qq - 1;
        if (zc >= z0 && zc < z1) {
            const Ax az = axis(zc, nz, L.per[2]);
            const int s0 = zc & 3, sm = (zc - 1) & 3, sp = (zc + 1) & 3;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + NW * k;
                if (!colo || !ay[k].in || r < H || r >= H + FP) continue;
                const long long g = ax.gw + (long long)nx * ay[k].gw + nxy * zc;
                const V pv = sP[s0][r][lane];
                const V qv = L.diag[ax.cls + 3 * ay[k].cls + 9 * az.cls] * pv - off3<V>(L, sP, sm, s0, sp, r, lane);
                pnew[g] = pv;
                q[g] = qv;
                acc = fma(pv, qv, acc);
            }
        }
    }
    __shared__ double red[NT / 32];
    __shared__ float redf[NT / 32];
    const double bacc = block_sum_any<NT>(acc, red, redf);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) part[block_linear()] = bacc;
    if (arrive_last(cnt)) {
        const double PQ = sum_parts_cg<NT>(part, nb, red);
        if (threadIdx.x == 0) {
            scal[PS_ALPHA] = scal[PS_RZ] / PQ;
            *cnt = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Exact solve on the top coarse level in 3D by fast diagonalisation: the level
// operator is Ax (x) I (x) I + I (x) Ay (x) I + I (x) I (x) Az with the 1D
// second-difference matrices Ad = Sd diag(lam_d) Sd^T, so the zero-mean
// solution of A u = f is u = S [(S^T f) .* IL], S = Sz (x) Sy (x) Sx, with
// IL = 1 / (lam_z + lam_y + lam_x) (0 for the null mode).  S^T f and S v are
// three one-axis transforms each, all in the shared memory of one block.
// ---------------------------------------------------------------------------
constexpr int FT3 = 1024;          // threads of the 3D fast-diagonalisation block
constexpr int kFdm3Cells = 4096;   // largest top level given to it (24^3 measured slower: the
                                   // transforms make one SM instruction-bound, 46 us)

__host__ __device__ constexpr long long fdm3_smem_floats(long long nx, long long ny, long long nz) {
    return 2 * (nx * nx + ny * ny + nz * nz) + 3 * nx * ny * nz;
}

// out[z][y][k] = sum_i M[i][k] in[z][y][i] (M: nx x nx), optionally .* S, to a
// shared or global out.  A thread takes one k and four (z, y) lines.
__device__ __forceinline__ void fdm3_x(float* __restrict__ out, const float* __restrict__ in,
                                       const float* __restrict__ M, int nx, int nlines, const float* __restrict__ S) {
    const int items = nx * (nlines / 4);
    for (int t = threadIdx.x; t < items; t += FT3) {
        const int k = t % nx, l0 = 4 * (t / nx);
        const float* i0 = in + (long long)l0 * nx;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
        for (int i = 0; i < nx; ++i) {
            const float m = M[i * nx + k];
            a0 = fmaf(m, i0[i], a0);
            a1 = fmaf(m, i0[nx + i], a1);
            a2 = fmaf(m, i0[2 * nx + i], a2);
            a3 = fmaf(m, i0[3 * nx + i], a3);
        }
        const int o = l0 * nx + k;
        if (S) {
            a0 *= S[o];
            a1 *= S[o + nx];
            a2 *= S[o + 2 * nx];
            a3 *= S[o + 3 * nx];
        }
        out[o] = a0;
        out[o + nx] = a1;
        out[o + 2 * nx] = a2;
        out[o + 3 * nx] = a3;
    }
}

// Along an outer axis of length n and stride st (ny with st = nx, or nz with
// st = nx ny): out[.., k, ..] = sum_j M[j][k] in[.., j, ..], optionally .* S.
// The cells of one axis position form `inner` consecutive floats (nx, or
// nx ny); `outer` such blocks (nz, or 1).  A thread takes one inner position
// and four consecutive k (M rows read as float4).
__device__ __forceinline__ void fdm3_outer(float* __restrict__ out, const float* __restrict__ in,
                                           const float* __restrict__ M, int n, int inner, int outer,
                                           const float* __restrict__ S) {
    const int nq = n / 4;
    const int items = inner * nq * outer;
    const long long blk = (long long)inner * n;
    for (int t = threadIdx.x; t < items; t += FT3) {
        const int x = t % inner, r = t / inner;
        const int kq = r % nq, ob = r / nq;
        const float* ip = in + ob * blk + x;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            const float v = ip[(long long)j * inner];
            const float4 m = *reinterpret_cast<const float4*>(M + j * n + 4 * kq);
            a.x = fmaf(m.x, v, a.x);
            a.y = fmaf(m.y, v, a.y);
            a.z = fmaf(m.z, v, a.z);
            a.w = fmaf(m.w, v, a.w);
        }
        const long long o = ob * blk + (long long)(4 * kq) * inner + x;
        if (S) {
            a.x *= S[o];
            a.y *= S[o + inner];
            a.z *= S[o + 2 * inner];
            a.w *= S[o + 3 * inner];
        }
        out[o] = a.x;
        out[o + inner] = a.y;
        out[o + 2 * inner] = a.z;
        out[o + 3 * inner] = a.w;
    }
}

// Shared memory (floats): Sx, SxT, Sy, SyT, Sz, SzT, IL (the global table,
// copied linearly before the programmatic-dependency wait), then A and B
// (N = nx ny nz each).  nx, ny, nz multiples of 4.
__global__ void __launch_bounds__(FT3) fdm(int nx, int ny, int nz, const float* __restrict__ tab,
                                           const float* __restrict__ f, float* __restrict__ u) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* Sx = reinterpret_cast<float*>(smraw);
    float* SxT = Sx + nx * nx;
    float* Sy = SxT + nx * nx;
    float* SyT = Sy + ny * ny;
    float* Sz = SyT + ny * ny;
    float* SzT = Sz + nz * nz;
    float* IL = SzT + nz * nz;
    const int N = nx * ny * nz;
    float* A = IL + N;
    float* B = A + N;
    const int ntab = 2 * (nx * nx + ny * ny + nz * nz) + N;   // a multiple of 4
    for (int i = threadIdx.x; i < ntab / 4; i += FT3) k2::cp_async16(Sx + 4 * i, tab + 4 * i);
    pdl_wait();
    pdl_trigger();
    for (int i = threadIdx.x; i < N / 4; i += FT3) k2::cp_async16(A + 4 * i, f + 4 * i);
    k2::cp_async_wait_all();
    __syncthreads();
    const int nxy = nx * ny;
    fdm3_x(B, A, Sx, nx, ny * nz, nullptr);           // S_x^T along x
    __syncthreads();
    fdm3_outer(A, B, Sy, ny, nx, nz, nullptr);         // S_y^T along y
    __syncthreads();
    fdm3_outer(B, A, Sz, nz, nxy, 1, IL);              // S_z^T along z, then .* IL
    __syncthreads();
    fdm3_outer(A, B, SzT, nz, nxy, 1, nullptr);        // S_z along z
    __syncthreads();
    fdm3_outer(B, A, SyT, ny, nx, nz, nullptr);        // S_y along y
    __syncthreads();
    fdm3_x(u, B, SxT, nx, ny * nz, nullptr);           // S_x along x, to global
}

}  // namespace k3

// ---------------------------------------------------------------------------
// Colour-sweep kernels of the large 3D levels: the same smoother, residual and
// transfers as the z-marching kernels (red from zero, black, residual,
// restriction; prolongation-add, black, red), one whole-level pass each, so
// that a pass costs its memory traffic instead of a chain of per-plane
// barriers.  A thread owns an x-pair of cells (one of each colour) of a row;
// a block of 32 x 8 pairs (256 threads, x fastest) walks zc consecutive
// planes, so a plane's z-neighbours are the rows it read one step before and
// reads one step after (L1).  Indices are 32-bit: larger levels keep the
// z-marching kernels.
// ---------------------------------------------------------------------------
namespace k3s {

constexpr int BX = 32, BY = 8, NT = BX * BY;
constexpr int kZC = 4;  // consecutive planes per block (default)
constexpr int kZC8 = 2; // ... of the eight-cell passes

// The x coordinate of this thread's cell of colour `color` ((x + y + z) & 1).
__device__ __forceinline__ int pair_x(int y, int z, int color) {
    const int x0 = 2 * (int)(blockIdx.x * BX + (threadIdx.x & (BX - 1)));
    return x0 + ((color + x0 + y + z) & 1);
}
__device__ __forceinline__ int row_y() { return (int)(blockIdx.y * BY + threadIdx.x / BX); }

__device__ __forceinline__ int cls_of(int g, int n, int per) { return per ? 2 : (int)(g > 0) + (int)(g < n - 1); }

// A cell's index, its six neighbours' (-1 outside a non-periodic level) and
// its class index (the diagonal's and the inverse diagonal's).
struct Nb {
    int i, xm, xp, ym, yp, zm, zp, cls;
};
template <class T>
__device__ __forceinline__ Nb nbr(const LvT<T>& L, int x, int y, int z) {
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], sy = nx, sz = nx * ny;
    Nb b;
    b.i = x + sy * y + sz * z;
    if (x > 0 && x < nx - 1 && y > 0 && y < ny - 1 && z > 0 && z < nz - 1) {
        b.xm = b.i - 1;
        b.xp = b.i + 1;
        b.ym = b.i - sy;
        b.yp = b.i + sy;
        b.zm = b.i - sz;
        b.zp = b.i + sz;
        b.cls = 26;
        return b;
    }
    b.xm = (x > 0) ? b.i - 1 : (L.per[0] ? b.i + (nx - 1) : -1);
    b.xp = (x < nx - 1) ? b.i + 1 : (L.per[0] ? b.i - (nx - 1) : -1);
    b.ym = (y > 0) ? b.i - sy : (L.per[1] ? b.i + sy * (ny - 1) : -1);
    b.yp = (y < ny - 1) ? b.i + sy : (L.per[1] ? b.i - sy * (ny - 1) : -1);
    b.zm = (z > 0) ? b.i - sz : (L.per[2] ? b.i + sz * (nz - 1) : -1);
    b.zp = (z < nz - 1) ? b.i + sz : (L.per[2] ? b.i - sz * (nz - 1) : -1);
    b.cls = cls_of(x, nx, L.per[0]) + 3 * cls_of(y, ny, L.per[1]) + 9 * cls_of(z, nz, L.per[2]);
    return b;
}

template <class T>
__device__ __forceinline__ T at(const T* u, int j) {
    return j < 0 ? (T)0 : u[j];
}

// The off-diagonal sum of the z-marching kernels' off3, in its order.
template <class T>
__device__ __forceinline__ T off7(const LvT<T>& L, const Nb& b, const T* u) {
    T off = L.w[0] * (at(u, b.xm) + at(u, b.xp)) + L.w[1] * (at(u, b.ym) + at(u, b.yp));
    off += L.w[2] * (at(u, b.zm) + at(u, b.zp));
    return off;
}

// Red cells from a zero guess: u = f invd.
template <class T, class TF>
__global__ void __launch_bounds__(NT) red0(LvT<T> L, const TF* __restrict__ f, T* __restrict__ u,
                                           const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y >= L.n[1]) return;
    for (int z = blockIdx.z * zc; z < z1; ++z) {
        const int x = pair_x(y, z, 0);
        if (x >= L.n[0]) continue;
        const Nb b = nbr(L, x, y, z);
        u[b.i] = (T)(f[b.i] - mr) * L.invd[b.cls];
    }
}

// One colour of a Gauss-Seidel sweep in place (the other colour is read).
template <class T, class TF>
__global__ void __launch_bounds__(NT) sweep(LvT<T> L, const TF* __restrict__ f, T* u, int color,
                                            const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y >= L.n[1]) return;
    for (int z = blockIdx.z * zc; z < z1; ++z) {
        const int x = pair_x(y, z, color);
        if (x >= L.n[0]) continue;
        const Nb b = nbr(L, x, y, z);
        u[b.i] = ((T)(f[b.i] - mr) + off7<T>(L, b, u)) * L.invd[b.cls];
    }
}

// Residual r = f - A u at every cell.
template <class T, class TF>
__global__ void __launch_bounds__(NT) resid(LvT<T> L, const TF* __restrict__ f, const T* __restrict__ u,
                                            T* __restrict__ r, const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y >= L.n[1]) return;
    for (int z = blockIdx.z * zc; z < z1; ++z) {
#pragma unroll
        for (int color = 0; color < 2; ++color) {
            const int x = pair_x(y, z, color);
            if (x >= L.n[0]) continue;
            const Nb b = nbr(L, x, y, z);
            r[b.i] = (T)(f[b.i] - mr) - (L.diag[b.cls] * u[b.i] - off7<T>(L, b, u));
        }
    }
}

// Restriction fc = R r (R = P^T / 2 per direction, times 1/8 overall),
// separable through shared memory: a block owns a coarse tile of
// RX x RY x RZ cells, stages its fine footprint (2 RX + 2) x (2 RY + 2) x
// (2 RZ + 2) of r (zero outside a non-periodic level), then sums along x, y
// and z with the 1D weights.
constexpr int RX = 32, RY = 4, RZ = 4;
constexpr int FX = 2 * RX + 2, FY = 2 * RY + 2, FZ = 2 * RZ + 2;
constexpr size_t kRestrictSmem = sizeof(float) * (size_t)(FX * FY * FZ + RX * FY * FZ + RX * RY * FZ);

template <class T>
__global__ void __launch_bounds__(NT) restrict3(LvT<T> L, LvT<T> C, const T* __restrict__ r, T* __restrict__ fc) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sr = reinterpret_cast<T*>(smraw);          // [FZ][FY][FX]
    T* sx = sr + FX * FY * FZ;                     // [FZ][FY][RX]
    T* sy = sx + RX * FY * FZ;                     // [FZ][RY][RX]
    __shared__ T wt[(RX + RY + RZ) * 4];           // 1D weights of the tile's coarse indices
    const int I0 = blockIdx.x * RX, J0 = blockIdx.y * RY, K0 = blockIdx.z * RZ;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const int t = threadIdx.x;
        if (t < RX) {
#pragma unroll
            for (int a = 0; a < 4; ++a) wt[4 * t + a] = (T)rweight(a, I0 + t, C.n[0], C.per[0]);
        } else if (t < RX + RY) {
#pragma unroll
            for (int a = 0; a < 4; ++a) wt[4 * t + a] = (T)rweight(a, J0 + t - RX, C.n[1], C.per[1]);
        } else if (t < RX + RY + RZ) {
#pragma unroll
            for (int a = 0; a < 4; ++a) wt[4 * t + a] = (T)rweight(a, K0 + t - RX - RY, C.n[2], C.per[2]);
        }
    }
    // the fine footprint, one row of FX per warp step (lanes over x), zero
    // outside a non-periodic level
    constexpr int MX = (FX + 31) / 32;
    int gx[MX];
    bool okx[MX];
#pragma unroll
    for (int m = 0; m < MX; ++m) {
        int g = 2 * I0 - 1 + lane + 32 * m;
        bool ok = lane + 32 * m < FX;
        if (g < 0 || g >= nx) {
            ok = ok && L.per[0];
            g = g < 0 ? g + nx : g - nx;
        }
        okx[m] = ok && g >= 0 && g < nx;
        gx[m] = g;
    }
#pragma unroll 2
    for (int row = warp; row < FY * FZ; row += NT / 32) {
        const int b = row % FY, c = row / FY;
        int gy = 2 * J0 - 1 + b, gz = 2 * K0 - 1 + c;
        bool ok = true;
        if (gy < 0 || gy >= ny) {
            ok = ok && L.per[1];
            gy = gy < 0 ? gy + ny : gy - ny;
        }
        if (gz < 0 || gz >= nz) {
            ok = ok && L.per[2];
            gz = gz < 0 ? gz + nz : gz - nz;
        }
        ok = ok && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
        const T* src = r + (long long)nx * (gy + (long long)ny * gz);
        T v[MX];
#pragma unroll
        for (int m = 0; m < MX; ++m) v[m] = (ok && okx[m]) ? __ldg(src + gx[m]) : (T)0;
#pragma unroll
        for (int m = 0; m < MX; ++m)
            if (lane + 32 * m < FX) sr[row * FX + lane + 32 * m] = v[m];
    }
    __syncthreads();
    // x: lane = coarse column i (NT and RX are multiples of 32)
    {
        const T w0 = wt[4 * lane], w1 = wt[4 * lane + 1], w2 = wt[4 * lane + 2], w3 = wt[4 * lane + 3];
        for (int q = warp; q < FY * FZ; q += NT / 32) {
            const T* rowp = sr + q * FX + 2 * lane;
            T v = (T)0;
            v += w0 * rowp[0];
            v += w1 * rowp[1];
            v += w2 * rowp[2];
            v += w3 * rowp[3];
            sx[q * RX + lane] = v;
        }
    }
    __syncthreads();
    for (int q = warp; q < RY * FZ; q += NT / 32) {
        const int j = q % RY, c = q / RY;
        const T* wy = wt + 4 * (RX + j);
        T v = (T)0;
#pragma unroll
        for (int b = 0; b < 4; ++b) v += wy[b] * sx[(c * FY + 2 * j + b) * RX + lane];
        sy[q * RX + lane] = v;
    }
    __syncthreads();
    for (int q = warp; q < RY * RZ; q += NT / 32) {
        const int j = q % RY, k = q / RY;
        const int I = I0 + lane, J = J0 + j, K = K0 + k;
        if (I >= C.n[0] || J >= C.n[1] || K >= C.n[2]) continue;
        const T* wz = wt + 4 * (RX + RY + k);
        T v = (T)0;
#pragma unroll
        for (int c = 0; c < 4; ++c) v += wz[c] * sy[((2 * k + c) * RY + j) * RX + lane];
        fc[I + C.n[0] * (J + C.n[1] * K)] = v * (T)0.125;
    }
}

// u += P uc at every cell (in place).
template <class T>
__global__ void __launch_bounds__(NT) prolong_add(LvT<T> L, LvT<T> C, const T* __restrict__ uc, T* u, int zc) {
    pdl_wait();
    pdl_trigger();
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y >= L.n[1]) return;
    for (int z = blockIdx.z * zc; z < z1; ++z) {
#pragma unroll
        for (int color = 0; color < 2; ++color) {
            const int x = pair_x(y, z, color);
            if (x >= L.n[0]) continue;
            const int gw[3] = {x, y, z};
            const int i = x + L.n[0] * (y + L.n[1] * z);
            u[i] = u[i] + prolong_at<T, 3>(C, uc, gw);
        }
    }
}

// The red half of the post-smoothing, reading u_in (black already swept),
// writing every cell of u_out; on the fine level also r.z and sum z, whose
// last block forms beta, r.z and mean z as the z-marching up does.
template <class T, class TF, bool FINE>
__global__ void __launch_bounds__(NT) red_out(LvT<T> L, const TF* __restrict__ f, const T* __restrict__ u_in,
                                              T* __restrict__ u_out, double* part_rz, double* part_sz, double* scal,
                                              const int* ictl, unsigned int* cnt, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = FINE ? (TF)scal[PS_MEANR] : (TF)0;
    TF rz = (TF)0, sz = (TF)0;
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y < L.n[1]) {
        for (int z = blockIdx.z * zc; z < z1; ++z) {
#pragma unroll
            for (int color = 0; color < 2; ++color) {
                const int x = pair_x(y, z, color);
                if (x >= L.n[0]) continue;
                const Nb b = nbr(L, x, y, z);
                const TF fv = f[b.i] - mr;
                const T u = (color == 0) ? ((T)fv + off7<T>(L, b, u_in)) * L.invd[b.cls] : u_in[b.i];
                u_out[b.i] = u;
                if (FINE) {
                    rz = fma(fv, (TF)u, rz);
                    sz += (TF)u;
                }
            }
        }
    }
    if (FINE) {
        __shared__ double red[2 * (NT / 32)];
        __shared__ float redf[2 * (NT / 32)];
        double brz, bsz;
        block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        const int bl = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        if (threadIdx.x == 0) {
            part_rz[bl] = brz;
            part_sz[bl] = bsz;
        }
        if (arrive_last_n(cnt, (unsigned int)nb)) {
            double RZ, SZ;
            sum_parts2_cg<NT>(part_rz, part_sz, nb, red, &RZ, &SZ);
            if (threadIdx.x == 0) {
                const int it = ictl[PI_IT];
                scal[PS_BETA] = (it == 0) ? 0.0 : RZ / scal[PS_RZ];
                scal[PS_RZ] = RZ;
                scal[PS_MEANZ] = SZ / (double)L.N;
                *cnt = 0u;
            }
        }
    }
}

// ---- eight x-consecutive cells per thread (nx % 8 == 0): 16-byte loads of the
// cells' row segment and of the four neighbour rows, scalar loads of the two
// x-neighbours at the ends.  A thread owns segment (x0 .. x0 + 7, y) of the
// planes of its block's z-chunk; threads run along x, then y.
template <class T>
__device__ __forceinline__ void ld8(const T* __restrict__ p, T* o) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 a = *reinterpret_cast<const double2*>(p + 2 * h);
            o[2 * h] = a.x;
            o[2 * h + 1] = a.y;
        }
    }
}
template <class T>
__device__ __forceinline__ void st8(T* __restrict__ p, const T* o) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(p + 4) = make_float4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) *reinterpret_cast<double2*>(p + 2 * h) = make_double2(o[2 * h], o[2 * h + 1]);
    }
}

// Row-uniform data of a thread's segment: its y, the offsets to the y and z
// neighbour rows (0 when outside a non-periodic level), the x-end offsets.
struct Seg {
    int x0, y, valid;
    int dym, dyp, cy;   // y neighbour rows (offsets from the segment) and class
    int dxm, dxp;       // x neighbours of the first / last cell (offsets from the segment's start)
    bool hym, hyp, hxm, hxp;   // whether each neighbour exists (inside or periodic)
};
template <class T>
__device__ __forceinline__ Seg seg_of(const LvT<T>& L) {
    Seg g;
    const int nx = L.n[0], ny = L.n[1], nseg = nx >> 3;
    const int gid = (int)(blockIdx.x * NT + threadIdx.x);
    g.valid = gid < nseg * ny;
    const int sxi = gid % nseg;
    g.y = gid / nseg;
    g.x0 = 8 * sxi;
    g.hym = g.y > 0 || L.per[1];
    g.hyp = g.y < ny - 1 || L.per[1];
    g.dym = (g.y > 0) ? -nx : nx * (ny - 1);
    g.dyp = (g.y < ny - 1) ? nx : -nx * (ny - 1);
    g.cy = cls_of(g.y, ny, L.per[1]);
    g.hxm = g.x0 > 0 || L.per[0];
    g.hxp = g.x0 + 8 < nx || L.per[0];
    g.dxm = (g.x0 > 0) ? -1 : nx - 1;
    g.dxp = (g.x0 + 8 < nx) ? 8 : 8 - nx;
    return g;
}

// The segment's cells and neighbour rows of plane z (zeros outside).
template <class T>
struct Rows8 {
    T c[8], ym[8], yp[8], zm[8], zp[8];
    T xm, xp;
    int cz;
};
template <class T>
__device__ __forceinline__ void rows8(const LvT<T>& L, const Seg& g, const T* __restrict__ u, int z, int base,
                                      Rows8<T>& R) {
    const int nz = L.n[2], sz = L.n[0] * L.n[1];
    const bool hzm = z > 0 || L.per[2], hzp = z < nz - 1 || L.per[2];
    const int dzm = (z > 0) ? -sz : sz * (nz - 1);
    const int dzp = (z < nz - 1) ? sz : -sz * (nz - 1);
    R.cz = cls_of(z, nz, L.per[2]);
    ld8(u + base, R.c);
#pragma unroll
    for (int i = 0; i < 8; ++i) R.ym[i] = R.yp[i] = R.zm[i] = R.zp[i] = (T)0;
    if (g.hym) ld8(u + base + g.dym, R.ym);
    if (g.hyp) ld8(u + base + g.dyp, R.yp);
    if (hzm) ld8(u + base + dzm, R.zm);
    if (hzp) ld8(u + base + dzp, R.zp);
    R.xm = g.hxm ? u[base + g.dxm] : (T)0;
    R.xp = g.hxp ? u[base + g.dxp] : (T)0;
}

// The off-diagonal sum of cell i of the segment, in off7's order.
template <class T>
__device__ __forceinline__ T off8(const LvT<T>& L, const Rows8<T>& R, int i) {
    const T left = (i > 0) ? R.c[i - 1] : R.xm;
    const T right = (i < 7) ? R.c[i + 1] : R.xp;
    T off = L.w[0] * (left + right) + L.w[1] * (R.ym[i] + R.yp[i]);
    off += L.w[2] * (R.zm[i] + R.zp[i]);
    return off;
}

template <class T>
__device__ __forceinline__ int cls8(const LvT<T>& L, const Seg& g, const Rows8<T>& R, int i) {
    return cls_of(g.x0 + i, L.n[0], L.per[0]) + 3 * g.cy + 9 * R.cz;
}

// One colour of a Gauss-Seidel sweep in place, eight cells per thread: the
// segment is written back whole, the other colour's values unchanged (the
// pass reads them only), so a concurrent reader sees the same values.
template <class T, class TF>
__global__ void __launch_bounds__(NT) sweep8(LvT<T> L, const TF* __restrict__ f, T* u, int color,
                                             const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const Seg g = seg_of(L);
    if (!g.valid) return;
    const int z1 = min((int)(blockIdx.y + 1) * zc, L.n[2]);
    for (int z = blockIdx.y * zc; z < z1; ++z) {
        const int base = g.x0 + L.n[0] * (g.y + L.n[1] * z);
        Rows8<T> R;
        rows8(L, g, u, z, base, R);
        TF fv[8];
        ld8(f + base, fv);
        T out[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            out[i] = R.c[i];
            if (((g.x0 + i + g.y + z) & 1) == color)
                out[i] = ((T)(fv[i] - mr) + off8(L, R, i)) * L.invd[cls8(L, g, R, i)];
        }
        st8(u + base, out);
    }
}

// Residual r = f - A u, eight cells per thread.
template <class T, class TF>
__global__ void __launch_bounds__(NT) resid8(LvT<T> L, const TF* __restrict__ f, const T* __restrict__ u,
                                             T* __restrict__ r, const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const Seg g = seg_of(L);
    if (!g.valid) return;
    const int z1 = min((int)(blockIdx.y + 1) * zc, L.n[2]);
    for (int z = blockIdx.y * zc; z < z1; ++z) {
        const int base = g.x0 + L.n[0] * (g.y + L.n[1] * z);
        Rows8<T> R;
        rows8(L, g, u, z, base, R);
        TF fv[8];
        ld8(f + base, fv);
        T out[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            out[i] = (T)(fv[i] - mr) - (L.diag[cls8(L, g, R, i)] * R.c[i] - off8(L, R, i));
        st8(r + base, out);
    }
}

// Red cells from a zero guess, eight cells per thread (the segment's black
// cells get 0: the black sweep that follows writes them before any read).
template <class T, class TF>
__global__ void __launch_bounds__(NT) red0_8(LvT<T> L, const TF* __restrict__ f, T* __restrict__ u,
                                             const double* __restrict__ scal_r, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = scal_r ? (TF)scal_r[PS_MEANR] : (TF)0;
    const Seg g = seg_of(L);
    if (!g.valid) return;
    const int z1 = min((int)(blockIdx.y + 1) * zc, L.n[2]);
    for (int z = blockIdx.y * zc; z < z1; ++z) {
        const int base = g.x0 + L.n[0] * (g.y + L.n[1] * z);
        const int cz = cls_of(z, L.n[2], L.per[2]);
        TF fv[8];
        ld8(f + base, fv);
        T out[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int cls = cls_of(g.x0 + i, L.n[0], L.per[0]) + 3 * g.cy + 9 * cz;
            out[i] = (((g.x0 + i + g.y + z) & 1) == 0) ? (T)(fv[i] - mr) * L.invd[cls] : (T)0;
        }
        st8(u + base, out);
    }
}

// u += P uc, eight cells per thread.
template <class T>
__global__ void __launch_bounds__(NT) prolong_add8(LvT<T> L, LvT<T> C, const T* __restrict__ uc, T* u, int zc) {
    pdl_wait();
    pdl_trigger();
    const Seg g = seg_of(L);
    if (!g.valid) return;
    const int z1 = min((int)(blockIdx.y + 1) * zc, L.n[2]);
    for (int z = blockIdx.y * zc; z < z1; ++z) {
        const int base = g.x0 + L.n[0] * (g.y + L.n[1] * z);
        T v[8];
        ld8(u + base, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gw[3] = {g.x0 + i, g.y, z};
            v[i] = v[i] + prolong_at<T, 3>(C, uc, gw);
        }
        st8(u + base, v);
    }
}

// The red half of the post-smoothing, eight cells per thread (as red_out).
template <class T, class TF, bool FINE>
__global__ void __launch_bounds__(NT) red_out8(LvT<T> L, const TF* __restrict__ f, const T* __restrict__ u_in,
                                               T* __restrict__ u_out, double* part_rz, double* part_sz,
                                               double* scal, const int* ictl, unsigned int* cnt, int zc) {
    pdl_wait();
    pdl_trigger();
    const TF mr = FINE ? (TF)scal[PS_MEANR] : (TF)0;
    TF rz = (TF)0, sz = (TF)0;
    const Seg g = seg_of(L);
    if (g.valid) {
        const int z1 = min((int)(blockIdx.y + 1) * zc, L.n[2]);
        for (int z = blockIdx.y * zc; z < z1; ++z) {
            const int base = g.x0 + L.n[0] * (g.y + L.n[1] * z);
            Rows8<T> R;
            rows8(L, g, u_in, z, base, R);
            TF fv[8];
            ld8(f + base, fv);
            T out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const TF fi = fv[i] - mr;
                out[i] = (((g.x0 + i + g.y + z) & 1) == 0) ? ((T)fi + off8(L, R, i)) * L.invd[cls8(L, g, R, i)]
                                                           : R.c[i];
                if (FINE) {
                    rz = fma(fi, (TF)out[i], rz);
                    sz += (TF)out[i];
                }
            }
            st8(u_out + base, out);
        }
    }
    if (FINE) {
        __shared__ double red[2 * (NT / 32)];
        __shared__ float redf[2 * (NT / 32)];
        double brz, bsz;
        block_sum2_any<NT>(rz, sz, red, redf, &brz, &bsz);
        const int nb = gridDim.x * gridDim.y;
        const int bl = blockIdx.x + gridDim.x * blockIdx.y;
        if (threadIdx.x == 0) {
            part_rz[bl] = brz;
            part_sz[bl] = bsz;
        }
        if (arrive_last_n(cnt, (unsigned int)nb)) {
            double RZ, SZ;
            sum_parts2_cg<NT>(part_rz, part_sz, nb, red, &RZ, &SZ);
            if (threadIdx.x == 0) {
                const int it = ictl[PI_IT];
                scal[PS_BETA] = (it == 0) ? 0.0 : RZ / scal[PS_RZ];
                scal[PS_RZ] = RZ;
                scal[PS_MEANZ] = SZ / (double)L.N;
                *cnt = 0u;
            }
        }
    }
}

inline dim3 grid8(const int n[3], int zc) {
    const long long segs = (long long)(n[0] / 8) * n[1];
    return dim3((unsigned)((segs + NT - 1) / NT), (unsigned)((n[2] + zc - 1) / zc));
}

// CG direction in a whole-level pass: p = (z - mean z) + beta p_old (no
// neighbours), then the operator pass q = A p with the partial sums of p.q,
// whose last block forms alpha = r.z / p.q as the z-marching pq does.
template <class T, class V>
__global__ void __launch_bounds__(NT) pdir(LvT<V> L, const T* __restrict__ z, V* p0, V* p1, const double* scal,
                                           const int* ictl, int zc) {
    pdl_wait();
    pdl_trigger();
    const int it = ictl[PI_IT];
    const V* __restrict__ pold = (it & 1) ? p0 : p1;
    V* __restrict__ pnew = (it & 1) ? p1 : p0;
    const V beta = (V)scal[PS_BETA], mz = (V)scal[PS_MEANZ];
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y >= L.n[1]) return;
    for (int zz = blockIdx.z * zc; zz < z1; ++zz) {
#pragma unroll
        for (int color = 0; color < 2; ++color) {
            const int x = pair_x(y, zz, color);
            if (x >= L.n[0]) continue;
            const int i = x + L.n[0] * (y + L.n[1] * zz);
            V pv = (V)z[i] - mz;
            if (it > 0) pv = fma(beta, pold[i], pv);
            pnew[i] = pv;
        }
    }
}

template <class V>
__global__ void __launch_bounds__(NT) qop(LvT<V> L, const V* p0, const V* p1, V* __restrict__ q, double* part,
                                          double* scal, const int* ictl, unsigned int* cnt, int zc) {
    pdl_wait();
    pdl_trigger();
    const int it = ictl[PI_IT];
    const V* __restrict__ p = (it & 1) ? p1 : p0;
    V acc = (V)0;
    const int y = row_y();
    const int z1 = min((int)(blockIdx.z + 1) * zc, L.n[2]);
    if (y < L.n[1]) {
        for (int zz = blockIdx.z * zc; zz < z1; ++zz) {
#pragma unroll
            for (int color = 0; color < 2; ++color) {
                const int x = pair_x(y, zz, color);
                if (x >= L.n[0]) continue;
                const Nb b = nbr(L, x, y, zz);
                const V pv = p[b.i];
                const V qv = L.diag[b.cls] * pv - off7<V>(L, b, p);
                q[b.i] = qv;
                acc = fma(pv, qv, acc);
            }
        }
    }
    __shared__ double red[NT / 32];
    __shared__ float redf[NT / 32];
    const double bacc = block_sum_any<NT>(acc, red, redf);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = bacc;
    if (arrive_last_n(cnt, (unsigned int)nb)) {
        const double PQ = sum_parts_cg<NT>(part, nb, red);
        if (threadIdx.x == 0) {
            scal[PS_ALPHA] = scal[PS_RZ] / PQ;
            *cnt = 0u;
        }
    }
}

inline dim3 grid_of(const int n[3], int zc = kZC) {
    const int npx = (n[0] + 1) / 2;
    return dim3((unsigned)((npx + BX - 1) / BX), (unsigned)((n[1] + BY - 1) / BY), (unsigned)((n[2] + zc - 1) / zc));
}
inline dim3 restrict_grid(const int nc[3]) {
    return dim3((unsigned)((nc[0] + RX - 1) / RX), (unsigned)((nc[1] + RY - 1) / RY), (unsigned)((nc[2] + RZ - 1) / RZ));
}

}  // namespace k3s

// ------------------------------ host helpers --------------------------------
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Shapes {
    int nlev;
    int n[kMaxLevels][3];
    long long N[kMaxLevels];
};

bool make_shapes(int dim, const int n[3], Shapes* s, const char** err) {
    int cur[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    s->nlev = 0;
    for (;;) {
        const int l = s->nlev;
        if (l >= kMaxLevels) {
            *err = "too many multigrid levels";
            return false;
        }
        s->n[l][0] = cur[0];
        s->n[l][1] = cur[1];
        s->n[l][2] = cur[2];
        s->N[l] = (long long)cur[0] * cur[1] * cur[2];
        s->nlev = l + 1;
        bool can = s->N[l] > kCoarsenAbove;
        for (int d = 0; d < dim; ++d)
            if (cur[d] % 2 != 0 || cur[d] < 2) can = false;
        if (!can) break;
        for (int d = 0; d < dim; ++d) cur[d] /= 2;
    }
    if (s->N[s->nlev - 1] > kMaxCoarse) {
        *err = "grid does not coarsen to <= 1024 cells by halving (use extents with more factors of 2)";
        return false;
    }
    if (s->N[0] >= (1LL << 31)) {
        *err = "grid too large (more than 2^31 cells)";
        return false;
    }
    return true;
}

bool fdm_fits(const Shapes& s, int top, int dim, int mg_fp32);

// Top coarse level of the one-block solve and whether fast diagonalisation
// solves it (*fdm_out).  In 3D the fast-diagonalisation top is taken unless a
// tail size is given explicitly (which selects the shared-memory V-cycle).
int pick_top(const Shapes& s, int dim, int mg_fp32, long long tail_cells, size_t* smem_out, int* fdm_out) {
    *fdm_out = 0;
    if (s.nlev == 1) {
        *smem_out = 0;
        return 0;
    }
    long long thr = mg_fp32 ? kTailCellsF32 : kTailCellsF64;
    bool fixed = false;
    if (tail_cells > 0) {
        thr = tail_cells;
        fixed = true;
    } else if (const char* e = std::getenv("LOWMACH_TAIL_CELLS")) {   // tuning override
        const long long v = std::atoll(e);
        if (v > 0) {
            thr = v;
            fixed = true;
        }
    }
    if (dim == 3 && mg_fp32 && !fixed) {
        // the largest level of at most kFdm3Cells that the 3D fast-diagonalisation
        // block takes replaces the levels below it
        for (int top = 1; top < s.nlev; ++top)
            if (s.N[top] <= k3::kFdm3Cells && fdm_fits(s, top, dim, mg_fp32)) {
                *smem_out = 0;
                *fdm_out = 1;
                return top;
            }
    }
    const size_t w = mg_fp32 ? 4 : 8;
    for (int top = 1; top < s.nlev; ++top) {
        if (s.N[top] > thr && top < s.nlev - 1) continue;
        size_t b = 0;
        for (int l = top; l < s.nlev; ++l) b += 2 * w * (size_t)s.N[l];
        b += w * (size_t)s.N[top];
        if (b > kTailSmemMax && top < s.nlev - 1) continue;
        *smem_out = b;
        *fdm_out = (dim == 2) && fdm_fits(s, top, dim, mg_fp32);
        return top;
    }
    *smem_out = 0;
    *fdm_out = (dim == 2) && fdm_fits(s, s.nlev - 1, dim, mg_fp32);
    return s.nlev - 1;
}

long long k2_blocks(const int n[3]) {
    const int fu = k2::fu_of(2);   // smallest up tile of any sweep count
    const long long up = (long long)((n[0] + fu - 1) / fu) * ((n[1] + fu - 1) / fu);
    const long long pq = (long long)((n[0] + k2::FP - 1) / k2::FP) * ((n[1] + k2::FP - 1) / k2::FP);
    return up > pq ? up : pq;
}

template <int DIM>
long long tile_blocks(const int n_fine[3]) {
    constexpr int FX = 2 * Tile<DIM>::CX, FY = 2 * Tile<DIM>::CY, FZ = (DIM == 3) ? 2 * Tile<DIM>::CZ : 1;
    return (long long)((n_fine[0] + FX - 1) / FX) * ((n_fine[1] + FY - 1) / FY) *
           ((DIM == 3) ? (n_fine[2] + FZ - 1) / FZ : 1);
}

// z-marching 3D grids (k3): down over coarse tiles and chunks of coarse
// planes, up and pq over fine tiles and chunks of fine planes
dim3 k3_down_grid(const int nc[3]) {
    return dim3((nc[0] + k3::CD - 1) / k3::CD, (nc[1] + k3::CD - 1) / k3::CD, (nc[2] + k3::KC - 1) / k3::KC);
}
dim3 k3_tile_grid(const int n[3], int tile) {
    return dim3((n[0] + tile - 1) / tile, (n[1] + tile - 1) / tile, (n[2] + k3::ZU - 1) / k3::ZU);
}
long long k3_blocks(const int n[3]) {
    const dim3 a = k3_tile_grid(n, k3::FU), b = k3_tile_grid(n, k3::FP), c = k3s::grid_of(n, 1);
    const long long na = (long long)a.x * a.y * a.z, nb = (long long)b.x * b.y * b.z,
                    nc = (long long)c.x * c.y * c.z;
    return std::max(na, std::max(nb, nc));
}

template <int DIM>
dim3 tile_grid(const int n_fine[3]) {
    constexpr int FX = 2 * Tile<DIM>::CX, FY = 2 * Tile<DIM>::CY, FZ = (DIM == 3) ? 2 * Tile<DIM>::CZ : 1;
    return dim3((n_fine[0] + FX - 1) / FX, (n_fine[1] + FY - 1) / FY, (DIM == 3) ? (n_fine[2] + FZ - 1) / FZ : 1);
}

// Gauss-Jordan inverse with partial pivoting (host, double).
bool invert(std::vector<double>& A, long long n) {
    std::vector<double> I((size_t)(n * n), 0.0);
    for (long long i = 0; i < n; ++i) I[(size_t)(i * n + i)] = 1.0;
    for (long long c = 0; c < n; ++c) {
        long long piv = c;
        double best = std::fabs(A[(size_t)(c * n + c)]);
        for (long long r = c + 1; r < n; ++r) {
            const double v = std::fabs(A[(size_t)(r * n + c)]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 0.0)) return false;
        if (piv != c) {
            for (long long k = 0; k < n; ++k) {
                std::swap(A[(size_t)(c * n + k)], A[(size_t)(piv * n + k)]);
                std::swap(I[(size_t)(c * n + k)], I[(size_t)(piv * n + k)]);
            }
        }
        const double d = 1.0 / A[(size_t)(c * n + c)];
        for (long long k = 0; k < n; ++k) {
            A[(size_t)(c * n + k)] *= d;
            I[(size_t)(c * n + k)] *= d;
        }
        for (long long r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)(r * n + c)];
            if (f == 0.0) continue;
            for (long long k = 0; k < n; ++k) {
                A[(size_t)(r * n + k)] -= f * A[(size_t)(c * n + k)];
                I[(size_t)(r * n + k)] -= f * I[(size_t)(c * n + k)];
            }
        }
    }
    A.swap(I);
    return true;
}

// Dense (pseudo-)inverse of the coarsest operator: (A_c + c 1 1^T)^-1 with
// c = max diag / N_c, which maps mean-zero right-hand sides to solutions of A_c.
std::vector<double> coarse_inverse(const MgLevel& L, int dim) {
    const long long Nc = L.N;
    std::vector<double> A((size_t)(Nc * Nc), 0.0);
    double dmax = 0.0;
    for (long long t = 0; t < Nc; ++t) {
        int c[3] = {(int)(t % L.n[0]), (int)((t / L.n[0]) % L.n[1]), (int)(t / ((long long)L.n[0] * L.n[1]))};
        double diag = 0.0;
        for (int d = 0; d < dim; ++d) {
            const long long s = d == 0 ? 1 : (d == 1 ? L.n[0] : (long long)L.n[0] * L.n[1]);
            const double w = L.ih2[d];
            if (c[d] > 0) {
                A[(size_t)(t * Nc + t - s)] -= w;
                diag += w;
            } else if (L.periodic[d]) {
                A[(size_t)(t * Nc + t + (long long)(L.n[d] - 1) * s)] -= w;
                diag += w;
            }
            if (c[d] < L.n[d] - 1) {
                A[(size_t)(t * Nc + t + s)] -= w;
                diag += w;
            } else if (L.periodic[d]) {
                A[(size_t)(t * Nc + t - (long long)(L.n[d] - 1) * s)] -= w;
                diag += w;
            }
        }
        A[(size_t)(t * Nc + t)] += diag;
        if (diag > dmax) dmax = diag;
    }
    const double cshift = dmax / (double)Nc;
    for (auto& v : A) v += cshift;
    if (!invert(A, Nc)) A.assign((size_t)(Nc * Nc), 0.0);
    return A;
}

// Orthonormal eigenvectors (columns, S[i * n + k]) and eigenvalues of the 1D
// cell-centred second-difference matrix (diagonal 2, off-diagonals -1) scaled
// by 1/h^2: Neumann ends (diagonal 1 at the ends) -> DCT-II basis
// cos(pi k (i + 1/2) / n), lam = 2 - 2 cos(pi k / n); periodic -> real Fourier
// basis cos / sin(2 pi m i / n), lam = 2 - 2 cos(2 pi m / n).
void eig1d(int n, int periodic, double h, std::vector<double>& S, std::vector<double>& lam) {
    const double pi = 3.14159265358979323846;
    S.assign((size_t)n * n, 0.0);
    lam.assign(n, 0.0);
    const double ih2 = 1.0 / (h * h);
    if (!periodic) {
        for (int k = 0; k < n; ++k) {
            const double ck = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
            for (int i = 0; i < n; ++i) S[(size_t)i * n + k] = ck * std::cos(pi * k * (i + 0.5) / n);
            lam[k] = (2.0 - 2.0 * std::cos(pi * k / n)) * ih2;
        }
        return;
    }
    for (int i = 0; i < n; ++i) S[(size_t)i * n] = std::sqrt(1.0 / n);
    lam[0] = 0.0;
    int col = 1;
    for (int m = 1; 2 * m < n; ++m) {
        const double l = (2.0 - 2.0 * std::cos(2.0 * pi * m / n)) * ih2;
        for (int i = 0; i < n; ++i) {
            S[(size_t)i * n + col] = std::sqrt(2.0 / n) * std::cos(2.0 * pi * m * i / n);
            S[(size_t)i * n + col + 1] = std::sqrt(2.0 / n) * std::sin(2.0 * pi * m * i / n);
        }
        lam[col] = lam[col + 1] = l;
        col += 2;
    }
    if (n % 2 == 0) {
        for (int i = 0; i < n; ++i) S[(size_t)i * n + col] = (i % 2 == 0 ? 1.0 : -1.0) / std::sqrt((double)n);
        lam[col] = 4.0 * ih2;
    }
}

bool fdm_fits(const Shapes& s, int top, int dim, int mg_fp32) {
    if (!mg_fp32 || s.nlev < 2) return false;
    const long long nx = s.n[top][0], ny = s.n[top][1];
    if (dim == 3) {
        const long long nz = s.n[top][2];
        const size_t smem = sizeof(float) * (size_t)k3::fdm3_smem_floats(nx, ny, nz);
        return nx % 4 == 0 && ny % 4 == 0 && nz % 4 == 0 && s.N[top] <= k3::kFdm3Cells && smem <= kTailSmemMax;
    }
    if (dim != 2) return false;
    const size_t smem = sizeof(float) * (size_t)k2::fdm_smem_floats(nx, ny);
    return nx % 4 == 0 && ny % 4 == 0 && nx <= 128 && ny <= 128 && smem <= kTailSmemMax;
}

// Floats of the fast-diagonalisation table of a top level n (2D: S_x, S_x^T,
// S_y, S_y^T, IL; 3D: S_x, S_x^T, S_y, S_y^T, S_z, S_z^T, IL).
long long fdm_table_floats(const int n[3], int dim) {
    const long long nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const long long sq = nx * nx + ny * ny + ((dim == 3) ? nz * nz : 0);
    return 2 * sq + nx * ny * nz;
}

template <class T>
LvT<T> make_lv(const MgLevel& L, int dim) {
    LvT<T> v;
    std::memset(&v, 0, sizeof(v));
    for (int d = 0; d < 3; ++d) {
        v.n[d] = L.n[d];
        v.per[d] = (d < dim) ? L.periodic[d] : 0;
        v.w[d] = (T)((d < dim) ? L.ih2[d] : 0.0);
    }
    v.N = (int)L.N;
    v.dn0 = make_divu32((unsigned)L.n[0]);
    v.dn1 = make_divu32((unsigned)L.n[1]);
    for (int c = 0; c < 27; ++c) {
        const int cnt[3] = {c % 3, (c / 3) % 3, c / 9};
        double diag = 0.0;
        for (int d = 0; d < dim; ++d) diag += cnt[d] * L.ih2[d];
        v.diag[c] = (T)diag;
        v.invd[c] = (T)(diag > 0.0 ? 1.0 / diag : 0.0);
    }
    return v;
}

// Opt-in shared memory of the kernels that may exceed 48 KB (current device).
template <class T>
void set_smem_attrs() {
    cudaFuncSetAttribute(k_mg_down<T, double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * Box<3, 3>::SN * (int)sizeof(T));
    cudaFuncSetAttribute(k_mg_down<T, T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * Box<3, 3>::SN * (int)sizeof(T));
    cudaFuncSetAttribute(k_mg_up<T, double, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * Box<3, 2>::SN * (int)sizeof(T));
    cudaFuncSetAttribute(k_mg_up<T, T, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * Box<3, 2>::SN * (int)sizeof(T));
    cudaFuncSetAttribute(k_mg_tail<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    cudaFuncSetAttribute(k_mg_tail<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    cudaFuncSetAttribute(k_cg_pq<T, 3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Box<3, 1>::SN * (int)sizeof(double));
    cudaFuncSetAttribute(k2::tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    const int pl3 = k3::SB * k3::SB * k3::RING;
    cudaFuncSetAttribute(k3::down<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * pl3 * (int)sizeof(T));
    cudaFuncSetAttribute(k3::down<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * pl3 * (int)sizeof(T));
    cudaFuncSetAttribute(k3::up<T, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * pl3 * (int)sizeof(T));
    cudaFuncSetAttribute(k3::up<T, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * pl3 * (int)sizeof(T));
    cudaFuncSetAttribute(k3::up<T, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pl3 * (int)sizeof(T));
    cudaFuncSetAttribute(k3::pq<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl3 * (int)sizeof(double));
    cudaFuncSetAttribute(k3s::restrict3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(k3s::kRestrictSmem * (sizeof(T) / 4)));
    cudaFuncSetAttribute(k2::fdm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    cudaFuncSetAttribute(k3::fdm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
}

}  // namespace

// ------------------------------ plan ----------------------------------------
size_t poisson_plan_bytes(int dim, const int n[3], const int periodic[3], int mg_fp32, int tail_cells,
                          int* nlev_out, long long* Nc_out, const char** err) {
    return poisson_plan_bytes_batch(dim, n, periodic, mg_fp32, tail_cells, 1, nlev_out, Nc_out, err);
}

size_t poisson_plan_bytes_batch(int dim, const int n[3], const int periodic[3], int mg_fp32, int tail_cells, int nb,
                                int* nlev_out, long long* Nc_out, const char** err) {
    (void)periodic;
    Shapes s;
    if (!make_shapes(dim, n, &s, err)) return 0;
    if (nb < 1 || (nb > 1 && (dim != 2 || s.nlev == 1))) {
        *err = "batched solves need a 2D grid with at least two multigrid levels";
        return 0;
    }
    const size_t B = (size_t)nb;
    size_t tail_smem = 0;
    int use_fdm = 0;
    const int top = pick_top(s, dim, mg_fp32, tail_cells, &tail_smem, &use_fdm);
    const size_t w = mg_fp32 ? 4 : 8;
    const long long N = s.N[0];
    const long long nblk = (dim == 3) ? std::max(tile_blocks<3>(s.n[0]), k3_blocks(s.n[0])) : k2_blocks(s.n[0]);
    const long long npart = nblk > kMaxPartials ? nblk : kMaxPartials;
    size_t b = 0;
    b += 4 * align256(B * sizeof(double) * N);                      // r p0 p1 q
    b += align256(B * sizeof(double) * N) + align256(B * w * N);    // z (double-sized: one-level grids), u0pre
    if (mg_fp32 && s.nlev > 1) b += 4 * align256(B * sizeof(float) * N);   // r32 p32[2] q32
    b += 3 * align256(B * sizeof(double) * npart);                  // partials
    b += align256(B * sizeof(double) * PS_NSCAL) + align256(B * sizeof(int) * PI_NINT) +
         align256(B * sizeof(unsigned int) * kNumCounters) + align256(sizeof(int));
    for (int l = 1; l < s.nlev; ++l) {
        if (l < top) b += 3 * align256(B * w * s.N[l]);          // upre upost f
        else if (l == top) b += 2 * align256(B * w * s.N[l]);    // f (in), upost (out)
    }
    b += align256((mg_fp32 ? sizeof(LvT<float>) : sizeof(LvT<double>)) * s.nlev);
    const long long Nc = s.N[s.nlev - 1];
    b += align256(sizeof(double) * Nc * Nc) + align256(sizeof(float) * Nc * Nc);
    if (use_fdm) b += align256(sizeof(float) * fdm_table_floats(s.n[top], dim));
    if (nlev_out) *nlev_out = s.nlev;
    if (Nc_out) *Nc_out = Nc;
    return b;
}

bool poisson_plan_init(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                       int mg_fp32, int sweeps, int tail_cells, double rtol, int max_iter, void* ws,
                       size_t ws_bytes, std::vector<double>* minv_host, const char** err) {
    return poisson_plan_init_batch(pl, dim, n, h, periodic, mg_fp32, sweeps, tail_cells, rtol, max_iter, 1, ws,
                                   ws_bytes, minv_host, err);
}

bool poisson_plan_init_batch(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                             int mg_fp32, int sweeps, int tail_cells, double rtol, int max_iter, int nb, void* ws,
                             size_t ws_bytes, std::vector<double>* minv_host, const char** err) {
    Shapes s;
    if (!make_shapes(dim, n, &s, err)) return false;
    const size_t need = poisson_plan_bytes_batch(dim, n, periodic, mg_fp32, tail_cells, nb, nullptr, nullptr, err);
    const size_t B = (size_t)nb;
    if (need == 0) return false;
    if (ws_bytes < need) {
        *err = "poisson workspace too small";
        return false;
    }
    if (((uintptr_t)ws & 255) != 0) {
        *err = "workspace must be 256-byte aligned";
        return false;
    }
    std::memset((void*)pl, 0, sizeof(*pl));
    char* cur = (char*)ws;
    auto take = [&](size_t bytes) {
        char* p = cur;
        cur += align256(bytes);
        return p;
    };
    const size_t w = mg_fp32 ? 4 : 8;
    size_t tail_smem = 0;
    pl->dim = dim;
    pl->nlev = s.nlev;
    int use_fdm = 0;
    pl->top = pick_top(s, dim, mg_fp32, tail_cells, &tail_smem, &use_fdm);
    pl->mg_fp32 = mg_fp32;
    pl->N = s.N[0];
    pl->rtol = rtol;
    pl->max_iter = max_iter;
    // CG iterations captured ahead of the while node of a graph solve (one
    // system, multigrid): each saves the loop's per-iteration cost.  An
    // iteration of the V(2,2)-preconditioned CG gains about 1.4 decades of
    // residual (measured: 7 iterations per warm-started solve to 1e-10 in 2D,
    // 11 in 3D), so 0.6 log10(1 / rtol) iterations, rounded down, stay below
    // the count a solve needs; should a solve converge earlier, the remaining
    // captured iterations leave x and the reported scalars untouched (the
    // update kernels test the done flag) and cost only their launches.
    // LOWMACH_CG_PREFIX overrides the count.
    {
        int u = (rtol > 0.0 && rtol < 1.0) ? (int)std::floor(0.6 * std::log10(1.0 / rtol)) : 0;
        if (const char* e = std::getenv("LOWMACH_CG_PREFIX")) u = std::atoi(e);
        u = u < 0 ? 0 : (u > max_iter ? max_iter : u);
        pl->prefix = (nb == 1) ? u : 0;
    }
    // Programmatic dependent launch for the FP32 multigrid: its kernels are
    // short, and the next one's launch overlaps this one's drain.  The FP64
    // multigrid's kernels run several waves, and successors scheduled early
    // hold SM slots while they wait: its 256 x 512 step measured 2.454 ms with
    // PDL against 2.365 ms without.  LOWMACH_NO_PDL=1 / LOWMACH_PDL=1 override.
    pl->pdl = mg_fp32 ? 1 : 0;
    if (const char* e = std::getenv("LOWMACH_NO_PDL"))
        if (e[0] == '1') pl->pdl = 0;
    if (const char* e = std::getenv("LOWMACH_PDL"))
        if (e[0] == '1') pl->pdl = 1;
    pl->tail_smem = tail_smem;
    // red-black sweeps per smoothing (2D kernels): two, V(2,2).  The fused
    // kernels are latency-bound, so the extra shared-memory sweeps cost less
    // than the iterations they save (256x512: 20 -> 14 iterations per step in
    // FP32; in FP64 a small gain together with the 128-cell tail).  Tuning
    // override LOWMACH_SWEEPS = 1 or 2.
    pl->sweeps = 2;
    if (sweeps == 1 || sweeps == 2) {
        pl->sweeps = sweeps;
    } else if (const char* e = std::getenv("LOWMACH_SWEEPS")) {
        const int v = std::atoi(e);
        if (v == 1 || v == 2) pl->sweeps = v;
    }
    const long long nblk = (dim == 3) ? std::max(tile_blocks<3>(s.n[0]), k3_blocks(s.n[0])) : k2_blocks(s.n[0]);
    pl->npart = (int)(nblk > kMaxPartials ? nblk : kMaxPartials);
    {
        // LOWMACH_MG3_TILES=1: the cube-tile 3D kernels instead of the z-marching ones
        const char* e = std::getenv("LOWMACH_MG3_TILES");
        pl->mg3_tiles = (e && e[0] == '1') ? 1 : 0;
        // large levels on whole-level colour-sweep passes (LOWMACH_MG3_SWEEPS=0:
        // the z-marching kernels, which read each array once but serialise a
        // block's planes behind barriers; C3 192^3 mixed 16.77 -> 15.60 ms,
        // FP64 57.6 -> 48.0 ms per step)
        const char* w = std::getenv("LOWMACH_MG3_SWEEPS");
        pl->mg3_sweeps = (w && w[0] == '0') ? 0 : 1;
        // levels below this many cells keep the cube tiles: 2^17 for the
        // colour sweeps (the 96^3 level of a 192^3 grid on them too: mixed
        // 15.06-15.13 -> 14.89 ms, FP64 45.3 -> 44.0 ms), 2^20 for the
        // z-marching kernels (fewer planes per block would leave them too few
        // blocks)
        const char* m = std::getenv("LOWMACH_MG3_MIN_CELLS");
        pl->mg3_min_cells = (m && std::atoll(m) >= 0) ? std::atoll(m)
                                                      : (pl->mg3_sweeps ? kMg3SweepMinCells : kMg3MinCells);
        const char* zc = std::getenv("LOWMACH_K3S_ZC");
        pl->k3s_zc = (zc && std::atoi(zc) >= 1 && std::atoi(zc) <= 64) ? std::atoi(zc) : k3s::kZC;
    }
    pl->nb = nb;
    pl->r = (double*)take(B * sizeof(double) * pl->N);
    pl->p[0] = (double*)take(B * sizeof(double) * pl->N);
    pl->p[1] = (double*)take(B * sizeof(double) * pl->N);
    pl->q = (double*)take(B * sizeof(double) * pl->N);
    pl->z = take(B * sizeof(double) * pl->N);
    pl->u0pre = take(B * w * pl->N);
    // Refinement mode (FP32 CG with reliable updates) is the mixed default; the
    // tuning override LOWMACH_REFINE=0 keeps the FP64 CG around the FP32 multigrid.
    const char* rf = std::getenv("LOWMACH_REFINE");
    const bool refine_mode = mg_fp32 && s.nlev > 1 && !(rf && rf[0] == '0');
    if (refine_mode) {   // refinement mode (a one-level grid is solved exactly in FP64)
        pl->r32 = (float*)take(B * sizeof(float) * pl->N);
        pl->p32[0] = (float*)take(B * sizeof(float) * pl->N);
        pl->p32[1] = (float*)take(B * sizeof(float) * pl->N);
        pl->q32 = (float*)take(B * sizeof(float) * pl->N);
    }
    pl->part0 = (double*)take(B * sizeof(double) * pl->npart);
    pl->part1 = (double*)take(B * sizeof(double) * pl->npart);
    pl->part2 = (double*)take(B * sizeof(double) * pl->npart);
    pl->scal = (double*)take(B * sizeof(double) * PS_NSCAL);
    pl->ictl = (int*)take(B * sizeof(int) * PI_NINT);
    pl->cnt = (unsigned int*)take(B * sizeof(unsigned int) * kNumCounters);
    pl->bdone = (int*)take(sizeof(int));
    for (int l = 0; l < s.nlev; ++l) {
        MgLevel& L = pl->lev[l];
        for (int d = 0; d < 3; ++d) {
            L.n[d] = s.n[l][d];
            L.periodic[d] = (d < dim) ? (periodic[d] != 0) : 0;
            const double scale = (double)(1 << l);
            L.h[d] = (d < dim) ? h[d] * scale : 1.0;
            L.ih2[d] = (d < dim) ? 1.0 / (L.h[d] * L.h[d]) : 0.0;
        }
        L.N = s.N[l];
        if (l >= 1 && l < pl->top) {
            L.upre = take(B * w * L.N);
            L.upost = take(B * w * L.N);
            L.f = take(B * w * L.N);
        } else if (l >= 1 && l == pl->top) {
            L.f = take(B * w * L.N);
            L.upost = take(B * w * L.N);
        }
    }
    const size_t lvsz = mg_fp32 ? sizeof(LvT<float>) : sizeof(LvT<double>);
    pl->levtab = take(lvsz * s.nlev);
    pl->Nc = s.N[s.nlev - 1];
    pl->Minv = (double*)take(sizeof(double) * pl->Nc * pl->Nc);
    pl->Minv_f = (float*)take(sizeof(float) * pl->Nc * pl->Nc);
    pl->fdm = use_fdm;
    if (pl->fdm) {
        // the top level is solved exactly by fast diagonalisation (replaces the tail V-cycle)
        const int nx = s.n[pl->top][0], ny = s.n[pl->top][1], nz = s.n[pl->top][2];
        pl->fdm_tab_floats = (size_t)fdm_table_floats(s.n[pl->top], dim);
        pl->fdm_tab = (float*)take(sizeof(float) * pl->fdm_tab_floats);
        pl->fdm_smem = sizeof(float) * (size_t)((dim == 3) ? k3::fdm3_smem_floats(nx, ny, nz)
                                                             : k2::fdm_smem_floats(nx, ny));
    }
    // persistent solve: one 2D system in refinement mode with the fast-diagonalisation
    // top level, on request (LOWMACH_PERSIST=1).  Measured on GB300 it is slower
    // than the chain of level kernels: a grid barrier costs 1.8 us, 3.7 us with a
    // reduction finished by the last block (the L2 round trips of the release and
    // acquire), against about 1 us per programmatically dependent launch, so the
    // 256 x 512 step took 1.19 ms against 1.03 ms.
    pl->persist = 0;
    pl->persist_grid = 0;
    {
        const char* pe = std::getenv("LOWMACH_PERSIST");
        const bool on = pe && pe[0] == '1';
        if (on && dim == 2 && nb == 1 && refine_mode && pl->fdm && pl->sweeps == 2 && pl->top >= 1 &&
            pl->top < kp::kLev) {
            int dev = 0, nsm = 0, coop = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            cudaFuncSetAttribute(kp::k_solve2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->fdm_smem);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kp::k_solve2, k2::NT, pl->fdm_smem) !=
                cudaSuccess)
                per = 0;
            cudaGetLastError();
            long long g = (long long)per * nsm;
            if (g > 2LL * nsm) g = 2LL * nsm;
            if (const char* e = std::getenv("LOWMACH_PERSIST_GRID")) {
                const long long v = std::atoll(e);
                if (v >= 1 && v < g) g = v;
            }
            if (g > pl->npart / 3) g = pl->npart / 3;
            if (coop && g >= 1) {
                pl->persist = 1;
                pl->persist_grid = (int)g;
            }
        }
    }
    // tail shared-memory offsets (elements of T)
    {
        int off = 0;
        for (int l = pl->top; l < s.nlev && s.nlev > 1; ++l) {
            pl->tail_off_u[l] = off;
            off += (int)s.N[l];
            pl->tail_off_f[l] = off;
            off += (int)s.N[l];
        }
        pl->tail_off_r = off;
    }
    for (int l = 0; l < s.nlev; ++l) {
        if (mg_fp32) {
            LvT<float> v = make_lv<float>(pl->lev[l], dim);
            std::memcpy(pl->levtab_host + l * lvsz, &v, lvsz);
        } else {
            LvT<double> v = make_lv<double>(pl->lev[l], dim);
            std::memcpy(pl->levtab_host + l * lvsz, &v, lvsz);
        }
    }
    pl->levtab_bytes = lvsz * s.nlev;
    *minv_host = coarse_inverse(pl->lev[s.nlev - 1], dim);
    if (pl->fdm) {
        // appended after the coarse inverse: S_d and S_d^T per axis, then IL
        // (z slowest, x fastest)
        const int nx = s.n[pl->top][0], ny = s.n[pl->top][1], nz = (dim == 3) ? s.n[pl->top][2] : 1;
        std::vector<double> Sx, Sy, Sz, lx, ly, lz(1, 0.0);
        eig1d(nx, pl->lev[pl->top].periodic[0], pl->lev[pl->top].h[0], Sx, lx);
        eig1d(ny, pl->lev[pl->top].periodic[1], pl->lev[pl->top].h[1], Sy, ly);
        if (dim == 3) eig1d(nz, pl->lev[pl->top].periodic[2], pl->lev[pl->top].h[2], Sz, lz);
        auto put = [&](const std::vector<double>& M, int n, bool transpose) {
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) minv_host->push_back(transpose ? M[(size_t)k * n + i] : M[(size_t)i * n + k]);
        };
        put(Sx, nx, false);
        put(Sx, nx, true);
        put(Sy, ny, false);
        put(Sy, ny, true);
        if (dim == 3) {
            put(Sz, nz, false);
            put(Sz, nz, true);
        }
        for (int m = 0; m < nz; ++m)
            for (int l = 0; l < ny; ++l)
                for (int k = 0; k < nx; ++k) {
                    const double lam = lz[m] + ly[l] + lx[k];
                    minv_host->push_back(lam > 0.0 ? 1.0 / lam : 0.0);
                }
    }
    if (mg_fp32) set_smem_attrs<float>();
    else set_smem_attrs<double>();
    cudaGetLastError();   // attribute calls must not leave a sticky error behind
    return true;
}

bool poisson_upload_coarse(PoissonPlan* pl, const std::vector<double>& M, cudaStream_t s, const char** err) {
    const size_t nm = (size_t)(pl->Nc * pl->Nc);
    const size_t nf = pl->fdm ? pl->fdm_tab_floats : 0;
    if (M.size() != nm + nf) {
        *err = "coarse inverse not prepared";
        return false;
    }
    std::vector<float> Mf(M.size());
    for (size_t i = 0; i < M.size(); ++i) Mf[i] = (float)M[i];
    cudaError_t e = cudaMemcpyAsync(pl->Minv, M.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->Minv_f, Mf.data(), sizeof(float) * nm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->levtab, pl->levtab_host, pl->levtab_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && pl->fdm)
        e = cudaMemcpyAsync(pl->fdm_tab, Mf.data() + nm, sizeof(float) * pl->fdm_tab_floats, cudaMemcpyHostToDevice,
                            s);
    const size_t nb = (size_t)(pl->nb > 0 ? pl->nb : 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->cnt, 0, nb * sizeof(unsigned int) * kNumCounters, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ictl, 0, nb * sizeof(int) * PI_NINT, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->bdone, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return false;
    }
    return true;
}

// ------------------------------ enqueue -------------------------------------
namespace {

enum { CNT_UP0 = 0, CNT_PQ = 1, CNT_UPD = 2, CNT_MEANB = 3, CNT_INIT = 4, CNT_MEANX = 5, CNT_REF = 6 };

template <class T>
const LvT<T>* lv_dev(PoissonPlan* pl) {
    return reinterpret_cast<const LvT<T>*>(pl->levtab);
}

template <class T>
LvT<T> lv_host(PoissonPlan* pl, int l) {
    LvT<T> v;
    std::memcpy(&v, pl->levtab_host + l * sizeof(LvT<T>), sizeof(LvT<T>));
    return v;
}

// 2D level kernels with NS sweeps per smoothing.
template <class T, int NS>
void enqueue_down2(PoissonPlan* pl, int l, const LvT<T>& L, const LvT<T>& C, T* fc, cudaStream_t s) {
    constexpr int CD = k2::cd_of(NS);
    const dim3 grid((C.n[0] + CD - 1) / CD, (C.n[1] + CD - 1) / CD, pl->nb);
    const double* sr = pl->scal;   // the fine level removes the CG residual's mean
    if (l == 0 && pl->r32) launch(k2::down<T, float, NS>, grid, k2::NT, 0, s, L, C, pl->r32, (T*)pl->u0pre, fc, sr);
    else if (l == 0) launch(k2::down<T, double, NS>, grid, k2::NT, 0, s, L, C, pl->r, (T*)pl->u0pre, fc, sr);
    else launch(k2::down<T, T, NS>, grid, k2::NT, 0, s, L, C, (const T*)pl->lev[l].f, (T*)pl->lev[l].upre, fc,
                (const double*)nullptr);
}

template <class T, int NS>
void enqueue_up2(PoissonPlan* pl, int l, const LvT<T>& L, const LvT<T>& C, const T* uc, cudaStream_t s) {
    constexpr int FU = k2::fu_of(NS);
    const dim3 grid((L.n[0] + FU - 1) / FU, (L.n[1] + FU - 1) / FU, pl->nb);
    if (l == 0 && pl->r32)
        launch(k2::up<T, float, true, NS>, grid, k2::NT, 0, s, L, C, (const T*)pl->u0pre, pl->r32, uc, (T*)pl->z,
               pl->part0, pl->part1, pl->scal, pl->ictl, pl->cnt + CNT_UP0);
    else if (l == 0)
        launch(k2::up<T, double, true, NS>, grid, k2::NT, 0, s, L, C, (const T*)pl->u0pre, pl->r, uc, (T*)pl->z,
               pl->part0, pl->part1, pl->scal, pl->ictl, pl->cnt + CNT_UP0);
    else
        launch(k2::up<T, T, false, NS>, grid, k2::NT, 0, s, L, C, (const T*)pl->lev[l].upre, (const T*)pl->lev[l].f,
               uc, (T*)pl->lev[l].upost, (double*)nullptr, (double*)nullptr, (double*)nullptr, (const int*)nullptr,
               (unsigned int*)nullptr);
}

// Eight cells per thread in the colour sweeps and residual of the large 3D
// levels (nx % 8 == 0): FP32 levels (192^3 mixed 14.89 -> 14.58 ms); the FP64
// levels keep the cell pairs (44.07 against 47.48 ms: 128 registers).
// LOWMACH_K3S_V8=0 / 1 forces either.
bool k3s_v8(const int n[3], bool fp32) {
    if (n[0] % 8 != 0) return false;
    const char* e = std::getenv("LOWMACH_K3S_V8");
    if (e && (e[0] == '0' || e[0] == '1')) return e[0] == '1';
    return fp32;
}

// Right-hand side of the fine multigrid level: the FP64 CG residual, or the
// FP32 inner residual in refinement mode.
template <class T, int DIM>
void enqueue_down(PoissonPlan* pl, int l, cudaStream_t s) {
    const LvT<T> L = lv_host<T>(pl, l), C = lv_host<T>(pl, l + 1);
    T* fc = (T*)pl->lev[l + 1].f;
    const bool ir = pl->r32 != nullptr;
    if (DIM == 2) {
        {
            if (pl->sweeps == 2) {
                enqueue_down2<T, 2>(pl, l, L, C, fc, s);
                pl->launches += 1;
                return;
            }
        }
        enqueue_down2<T, 1>(pl, l, L, C, fc, s);
    } else if (!pl->mg3_tiles && pl->lev[l].N >= pl->mg3_min_cells && pl->mg3_sweeps && pl->nb == 1 &&
               pl->lev[l].N < (1LL << 31)) {
        // colour-sweep passes; the residual goes through z (not live during the
        // down pass: the previous iteration's z was consumed by its pq)
        const int zc = pl->k3s_zc;
        const dim3 grid = k3s::grid_of(L.n, zc);
        T* u = (l == 0) ? (T*)pl->u0pre : (T*)pl->lev[l].upre;
        T* r = (T*)pl->z;
        const double* sr = pl->scal;
        const bool v8 = k3s_v8(L.n, sizeof(T) == 4);
        const dim3 g8 = k3s::grid8(L.n, k3s::kZC8);
        auto down_passes = [&](auto f, const double* srr) {
            using TFp = std::remove_cv_t<std::remove_pointer_t<decltype(f)>>;
            if (v8) launch(k3s::red0_8<T, TFp>, g8, k3s::NT, 0, s, L, f, u, srr, k3s::kZC8);
            else launch(k3s::red0<T, TFp>, grid, k3s::NT, 0, s, L, f, u, srr, zc);
            if (v8) {
                launch(k3s::sweep8<T, TFp>, g8, k3s::NT, 0, s, L, f, u, 1, srr, k3s::kZC8);
                launch(k3s::resid8<T, TFp>, g8, k3s::NT, 0, s, L, f, (const T*)u, r, srr, k3s::kZC8);
            } else {
                launch(k3s::sweep<T, TFp>, grid, k3s::NT, 0, s, L, f, u, 1, srr, zc);
                launch(k3s::resid<T, TFp>, grid, k3s::NT, 0, s, L, f, (const T*)u, r, srr, zc);
            }
        };
        if (l == 0 && ir) down_passes((const float*)pl->r32, sr);
        else if (l == 0) down_passes((const double*)pl->r, sr);
        else down_passes((const T*)pl->lev[l].f, (const double*)nullptr);
        launch(k3s::restrict3<T>, k3s::restrict_grid(C.n), k3s::NT, k3s::kRestrictSmem * (sizeof(T) / 4), s, L, C,
               (const T*)r, fc);
        pl->launches += 3;
    } else if (!pl->mg3_tiles && pl->lev[l].N >= pl->mg3_min_cells) {
        const dim3 grid = k3_down_grid(pl->lev[l + 1].n);
        const size_t smem = 3 * k3::RING * k3::SB * k3::SB * sizeof(T);
        const double* sr = pl->scal;   // the fine level removes the CG residual's mean
        if (l == 0 && ir)
            launch(k3::down<T, float>, grid, k3::NT, smem, s, L, C, pl->r32, (T*)pl->u0pre, fc, sr);
        else if (l == 0)
            launch(k3::down<T, double>, grid, k3::NT, smem, s, L, C, pl->r, (T*)pl->u0pre, fc, sr);
        else
            launch(k3::down<T, T>, grid, k3::NT, smem, s, L, C, (const T*)pl->lev[l].f, (T*)pl->lev[l].upre, fc,
                   (const double*)nullptr);
    } else {
        const dim3 grid = tile_grid<DIM>(pl->lev[l].n);
        const size_t smem = 2 * Box<DIM, 3>::SN * sizeof(T);
        const double* sr = pl->scal;   // the fine level removes the CG residual's mean
        if (l == 0 && ir)
            launch(k_mg_down<T, float, DIM>, grid, Tile<DIM>::NT, smem, s, L, C, pl->r32, (T*)pl->u0pre, fc, sr);
        else if (l == 0)
            launch(k_mg_down<T, double, DIM>, grid, Tile<DIM>::NT, smem, s, L, C, pl->r, (T*)pl->u0pre, fc, sr);
        else
            launch(k_mg_down<T, T, DIM>, grid, Tile<DIM>::NT, smem, s, L, C, (const T*)pl->lev[l].f,
                                                                   (T*)pl->lev[l].upre, fc, (const double*)nullptr);
    }
    pl->launches += 1;
}

template <class T, int DIM>
void enqueue_up(PoissonPlan* pl, int l, cudaStream_t s) {
    const LvT<T> L = lv_host<T>(pl, l), C = lv_host<T>(pl, l + 1);
    const T* uc = (const T*)pl->lev[l + 1].upost;
    const bool ir = pl->r32 != nullptr;
    if (DIM == 2) {
        {
            if (pl->sweeps == 2) {
                enqueue_up2<T, 2>(pl, l, L, C, uc, s);
                pl->launches += 1;
                return;
            }
        }
        enqueue_up2<T, 1>(pl, l, L, C, uc, s);
    } else if (!pl->mg3_tiles && pl->lev[l].N >= pl->mg3_min_cells && pl->mg3_sweeps && pl->nb == 1 &&
               pl->lev[l].N < (1LL << 31)) {
        const int zc = pl->k3s_zc;
        const dim3 grid = k3s::grid_of(L.n, zc);
        T* u = (l == 0) ? (T*)pl->u0pre : (T*)pl->lev[l].upre;
        // the reducing pass keeps the default plane chunk (its last block sums
        // one partial per block)
        const dim3 rgrid = k3s::grid_of(L.n, k3s::kZC);
        const bool v8 = k3s_v8(L.n, sizeof(T) == 4);
        const dim3 g8 = k3s::grid8(L.n, k3s::kZC8);
        if (v8) launch(k3s::prolong_add8<T>, g8, k3s::NT, 0, s, L, C, uc, u, k3s::kZC8);
        else launch(k3s::prolong_add<T>, grid, k3s::NT, 0, s, L, C, uc, u, zc);
        if (l == 0 && ir) {
            if (v8)
                launch(k3s::sweep8<T, float>, g8, k3s::NT, 0, s, L, (const float*)pl->r32, u, 1,
                       (const double*)pl->scal, k3s::kZC8);
            else
                launch(k3s::sweep<T, float>, grid, k3s::NT, 0, s, L, (const float*)pl->r32, u, 1,
                       (const double*)pl->scal, zc);
            if (v8)
                launch(k3s::red_out8<T, float, true>, g8, k3s::NT, 0, s, L, (const float*)pl->r32, (const T*)u,
                       (T*)pl->z, pl->part0, pl->part1, pl->scal, (const int*)pl->ictl, pl->cnt + CNT_UP0,
                       k3s::kZC8);
            else
                launch(k3s::red_out<T, float, true>, rgrid, k3s::NT, 0, s, L, (const float*)pl->r32, (const T*)u,
                       (T*)pl->z, pl->part0, pl->part1, pl->scal, (const int*)pl->ictl, pl->cnt + CNT_UP0,
                       k3s::kZC);
        } else if (l == 0) {
            if (v8)
                launch(k3s::sweep8<T, double>, g8, k3s::NT, 0, s, L, (const double*)pl->r, u, 1,
                       (const double*)pl->scal, k3s::kZC8);
            else
                launch(k3s::sweep<T, double>, grid, k3s::NT, 0, s, L, (const double*)pl->r, u, 1,
                       (const double*)pl->scal, zc);
            launch(k3s::red_out<T, double, true>, rgrid, k3s::NT, 0, s, L, (const double*)pl->r, (const T*)u,
                   (T*)pl->z, pl->part0, pl->part1, pl->scal, (const int*)pl->ictl, pl->cnt + CNT_UP0, k3s::kZC);
        } else {
            const T* f = (const T*)pl->lev[l].f;
            if (v8)
                launch(k3s::sweep8<T, T>, g8, k3s::NT, 0, s, L, f, u, 1, (const double*)nullptr, k3s::kZC8);
            else
                launch(k3s::sweep<T, T>, grid, k3s::NT, 0, s, L, f, u, 1, (const double*)nullptr, zc);
            if (v8)
                launch(k3s::red_out8<T, T, false>, g8, k3s::NT, 0, s, L, f, (const T*)u, (T*)pl->lev[l].upost,
                       (double*)nullptr, (double*)nullptr, (double*)nullptr, (const int*)nullptr,
                       (unsigned int*)nullptr, k3s::kZC8);
            else
                launch(k3s::red_out<T, T, false>, rgrid, k3s::NT, 0, s, L, f, (const T*)u, (T*)pl->lev[l].upost,
                       (double*)nullptr, (double*)nullptr, (double*)nullptr, (const int*)nullptr,
                       (unsigned int*)nullptr, k3s::kZC);
        }
        pl->launches += 2;
    } else if (!pl->mg3_tiles && pl->lev[l].N >= pl->mg3_min_cells) {
        const dim3 grid = k3_tile_grid(pl->lev[l].n, k3::FU);
        const size_t smem = 2 * k3::RING * k3::SB * k3::SB * sizeof(T);
        if (l == 0 && ir)
            launch(k3::up<T, float, true>, grid, k3::NT, smem, s, L, C, (const T*)pl->u0pre, pl->r32, uc, (T*)pl->z,
                   pl->part0, pl->part1, pl->scal, pl->ictl, pl->cnt + CNT_UP0);
        else if (l == 0)
            launch(k3::up<T, double, true>, grid, k3::NT, smem, s, L, C, (const T*)pl->u0pre, pl->r, uc, (T*)pl->z,
                   pl->part0, pl->part1, pl->scal, pl->ictl, pl->cnt + CNT_UP0);
        else
            launch(k3::up<T, T, false>, grid, k3::NT, smem, s, L, C, (const T*)pl->lev[l].upre,
                   (const T*)pl->lev[l].f, uc, (T*)pl->lev[l].upost, (double*)nullptr, (double*)nullptr,
                   (double*)nullptr, (const int*)nullptr, (unsigned int*)nullptr);
    } else {
        const dim3 grid = tile_grid<DIM>(pl->lev[l].n);
        const size_t smem = 2 * Box<DIM, 2>::SN * sizeof(T);
        if (l == 0 && ir)
            launch(k_mg_up<T, float, DIM, true>, grid, Tile<DIM>::NT, smem, s, 
                L, C, (const T*)pl->u0pre, pl->r32, uc, (T*)pl->z, pl->part0, pl->part1, pl->scal, pl->ictl,
                pl->cnt + CNT_UP0);
        else if (l == 0)
            launch(k_mg_up<T, double, DIM, true>, grid, Tile<DIM>::NT, smem, s, 
                L, C, (const T*)pl->u0pre, pl->r, uc, (T*)pl->z, pl->part0, pl->part1, pl->scal, pl->ictl,
                pl->cnt + CNT_UP0);
        else
            launch(k_mg_up<T, T, DIM, false>, grid, Tile<DIM>::NT, smem, s, 
                L, C, (const T*)pl->lev[l].upre, (const T*)pl->lev[l].f, uc, (T*)pl->lev[l].upost, nullptr, nullptr,
                nullptr, nullptr, nullptr);
    }
    pl->launches += 1;
}

template <class T, int DIM>
void enqueue_tail(PoissonPlan* pl, cudaStream_t s) {
    TailArgs a;
    std::memset(&a, 0, sizeof(a));
    a.top = pl->top;
    a.nlev = pl->nlev;
    a.Nc = (int)pl->Nc;
    for (int l = 0; l < kMaxLevels; ++l) {
        a.off_u[l] = pl->tail_off_u[l];
        a.off_f[l] = pl->tail_off_f[l];
    }
    a.off_r = pl->tail_off_r;
    const T* Minv = (sizeof(T) == 4) ? (const T*)pl->Minv_f : (const T*)pl->Minv;
    if (DIM == 2 && pl->fdm) {
        const int nx = pl->lev[pl->top].n[0], ny = pl->lev[pl->top].n[1];
        launch(k2::fdm, pl->nb, k2::FT, pl->fdm_smem, s, nx, ny, pl->fdm_tab, (const float*)pl->lev[pl->top].f,
                                                (float*)pl->lev[pl->top].upost);
    } else if (DIM == 3 && pl->fdm) {
        const int nx = pl->lev[pl->top].n[0], ny = pl->lev[pl->top].n[1], nz = pl->lev[pl->top].n[2];
        launch(k3::fdm, 1, k3::FT3, pl->fdm_smem, s, nx, ny, nz, (const float*)pl->fdm_tab,
               (const float*)pl->lev[pl->top].f, (float*)pl->lev[pl->top].upost);
    } else if (DIM == 2)
        launch(k2::tail<T>, pl->nb, k2::TT, pl->tail_smem, s, lv_dev<T>(pl), a, (const T*)pl->lev[pl->top].f,
                                                     (T*)pl->lev[pl->top].upost, Minv);
    else
        launch(k_mg_tail<T, DIM>, 1, kTailThreads, pl->tail_smem, s, lv_dev<T>(pl), a, (const T*)pl->lev[pl->top].f,
                                                                 (T*)pl->lev[pl->top].upost, Minv);
    pl->launches += 1;
}

// The large 3D fine level's CG direction and operator as two whole-level
// passes (FP64 vectors; 192^3: 46.3-46.4 -> 45.3 ms per step) or the
// z-marching pq, which stages p once per plane (FP32 vectors of the
// refinement mode: 15.04-15.14 against 15.39 ms for the passes).
// LOWMACH_PQ_PASSES=0 / 1 forces either.
bool pq_passes(bool fp32_vectors) {
    const char* e = std::getenv("LOWMACH_PQ_PASSES");
    if (e && (e[0] == '0' || e[0] == '1')) return e[0] == '1';
    return !fp32_vectors;
}

// CG direction update + operator application: FP64 vectors, or the FP32
// inner vectors in refinement mode.
template <class T, int DIM>
void enqueue_pq(PoissonPlan* pl, cudaStream_t s) {
    const bool ir = pl->r32 != nullptr;
    if (DIM == 2) {
        const dim3 grid((pl->lev[0].n[0] + k2::FP - 1) / k2::FP, (pl->lev[0].n[1] + k2::FP - 1) / k2::FP, pl->nb);
        if (ir)
            launch(k2::pq<T, float>, grid, k2::NT, 0, s, make_lv<float>(pl->lev[0], DIM), (const T*)pl->z, pl->p32[0],
                                                     pl->p32[1], pl->q32, pl->part2, pl->scal, pl->ictl,
                                                     pl->cnt + CNT_PQ);
        else
            launch(k2::pq<T, double>, grid, k2::NT, 0, s, make_lv<double>(pl->lev[0], DIM), (const T*)pl->z, pl->p[0],
                                                      pl->p[1], pl->q, pl->part2, pl->scal, pl->ictl,
                                                      pl->cnt + CNT_PQ);
    } else if (!pl->mg3_tiles && pl->lev[0].N >= pl->mg3_min_cells && pl->mg3_sweeps && pl->nb == 1 &&
               pq_passes(ir)) {
        const dim3 grid = k3s::grid_of(pl->lev[0].n, k3s::kZC);
        if (ir) {
            launch(k3s::pdir<T, float>, grid, k3s::NT, 0, s, make_lv<float>(pl->lev[0], DIM), (const T*)pl->z,
                   pl->p32[0], pl->p32[1], (const double*)pl->scal, (const int*)pl->ictl, k3s::kZC);
            launch(k3s::qop<float>, grid, k3s::NT, 0, s, make_lv<float>(pl->lev[0], DIM), (const float*)pl->p32[0],
                   (const float*)pl->p32[1], pl->q32, pl->part2, pl->scal, (const int*)pl->ictl, pl->cnt + CNT_PQ,
                   k3s::kZC);
        } else {
            launch(k3s::pdir<T, double>, grid, k3s::NT, 0, s, make_lv<double>(pl->lev[0], DIM), (const T*)pl->z,
                   pl->p[0], pl->p[1], (const double*)pl->scal, (const int*)pl->ictl, k3s::kZC);
            launch(k3s::qop<double>, grid, k3s::NT, 0, s, make_lv<double>(pl->lev[0], DIM), (const double*)pl->p[0],
                   (const double*)pl->p[1], pl->q, pl->part2, pl->scal, (const int*)pl->ictl, pl->cnt + CNT_PQ,
                   k3s::kZC);
        }
        pl->launches += 1;
    } else if (!pl->mg3_tiles && pl->lev[0].N >= pl->mg3_min_cells) {
        const dim3 grid = k3_tile_grid(pl->lev[0].n, k3::FP);
        const size_t pl3 = (size_t)k3::RING * k3::SB * k3::SB;
        if (ir)
            launch(k3::pq<T, float>, grid, k3::NT, pl3 * sizeof(float), s, make_lv<float>(pl->lev[0], DIM),
                   (const T*)pl->z, pl->p32[0], pl->p32[1], pl->q32, pl->part2, pl->scal, pl->ictl,
                   pl->cnt + CNT_PQ);
        else
            launch(k3::pq<T, double>, grid, k3::NT, pl3 * sizeof(double), s, make_lv<double>(pl->lev[0], DIM),
                   (const T*)pl->z, pl->p[0], pl->p[1], pl->q, pl->part2, pl->scal, pl->ictl, pl->cnt + CNT_PQ);
    } else {
        const dim3 grid = tile_grid<DIM>(pl->lev[0].n);
        if (ir)
            launch(k_cg_pq<T, DIM, float>, grid, Tile<DIM>::NT, Box<DIM, 1>::SN * sizeof(float), s, 
                make_lv<float>(pl->lev[0], DIM), (const T*)pl->z, pl->p32[0], pl->p32[1], pl->q32, pl->part2,
                pl->scal, pl->ictl, pl->cnt + CNT_PQ);
        else
            launch(k_cg_pq<T, DIM, double>, grid, Tile<DIM>::NT, Box<DIM, 1>::SN * sizeof(double), s, 
                make_lv<double>(pl->lev[0], DIM), (const T*)pl->z, pl->p[0], pl->p[1], pl->q, pl->part2, pl->scal,
                pl->ictl, pl->cnt + CNT_PQ);
    }
    pl->launches += 1;
}

template <class T, int DIM>
void body(PoissonPlan* pl, double* x, cudaStream_t s, cudaGraphConditionalHandle h, int use_graph) {
    const bool ir = pl->r32 != nullptr;
    if (pl->nlev == 1) {
        // one-level grid: the preconditioner is the exact coarse solve (FP64)
        launch(k_direct<double>, 1, kTailThreads, 0, s, pl->Minv, (int)pl->Nc, pl->r, (double*)pl->z, pl->scal,
                                                    pl->ictl);
        pl->launches += 1;
        enqueue_pq<double, DIM>(pl, s);
    } else {
        for (int l = 0; l < pl->top; ++l) enqueue_down<T, DIM>(pl, l, s);
        enqueue_tail<T, DIM>(pl, s);
        for (int l = pl->top - 1; l >= 0; --l) enqueue_up<T, DIM>(pl, l, s);
        enqueue_pq<T, DIM>(pl, s);
    }
    const dim3 rb(reduce_blocks(pl->N), pl->nb);
    // a batch sets the while-node condition once, from every system's state
    const int ug = (pl->nb > 1) ? 0 : use_graph;
    if (ir) {
        // four x-consecutive cells per thread step when nx % 4 == 0 and x (the
        // caller's array) is 16-byte aligned
        // (LOWMACH_IR_VEC4=0: one cell per thread step; =8: eight when nx % 8 == 0)
        const char* v4 = std::getenv("LOWMACH_IR_VEC4");
        int vec4 = ((pl->lev[0].n[0] % 4 == 0) && (((uintptr_t)x & 15) == 0) && !(v4 && v4[0] == '0')) ? 4 : 0;
        if (vec4 && v4 && v4[0] == '8' && pl->lev[0].n[0] % 8 == 0) vec4 = 8;
        const dim3 rbr(vec4 ? reduce_blocks(pl->N / vec4) : reduce_blocks(pl->N), pl->nb);
        if (vec4 == 8)
            launch(k_ir_step<DIM, 8>, rbr, NTV, 0, s, make_lv<double>(pl->lev[0], DIM), x, pl->r,
                   (const float*)pl->p32[0], (const float*)pl->p32[1], pl->r32, pl->part1, pl->part2, pl->scal,
                   pl->ictl, pl->cnt + CNT_REF, pl->rtol, pl->max_iter, h, ug, vec4);
        else
            launch(k_ir_step<DIM, 4>, rbr, NTV, 0, s, make_lv<double>(pl->lev[0], DIM), x, pl->r,
                   (const float*)pl->p32[0], (const float*)pl->p32[1], pl->r32, pl->part1, pl->part2, pl->scal,
                   pl->ictl, pl->cnt + CNT_REF, pl->rtol, pl->max_iter, h, ug, vec4);
        pl->launches += 1;
    } else {
        // the update runs two cells per thread step when N is even and x (the
        // caller's array) is 16-byte aligned
        const int vec2 = (pl->N % 2 == 0) && (((uintptr_t)x & 15) == 0);
        const dim3 rbu(vec2 ? reduce_blocks(pl->N / 2) : reduce_blocks(pl->N), pl->nb);
        launch(k_cg_update, rbu, NTV, 0, s, x, pl->r, pl->p[0], pl->p[1], pl->q, pl->N, pl->part0, pl->part2,
               pl->scal, pl->ictl,
                                       pl->cnt + CNT_UPD, pl->rtol, pl->max_iter, h, ug, vec2);
        pl->launches += 1;
    }
    if (pl->nb > 1) {
        launch(k_batch_cond, 1, NTV, 0, s, (const int*)pl->ictl, pl->nb, pl->bdone, h, use_graph);
        pl->launches += 1;
    }
}

template <int DIM>
void prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s, cudaGraphConditionalHandle h,
              int use_graph, int mean_ready) {
    const dim3 rb(reduce_blocks(pl->N), pl->nb);
    if (!mean_ready) {
        launch(k_mean, rb, NTV, 0, s, b, pl->N, pl->part0, pl->scal, PS_MEANB, pl->cnt + CNT_MEANB);
        pl->launches += 1;
    }
    const LvT<double> L = make_lv<double>(pl->lev[0], DIM);
    launch(k_pcg_init<DIM>, rb, NTV, 0, s, L, b, x, pl->r, pl->r32, pl->part1, pl->part2, pl->part0, pl->scal,
           pl->ictl,
                                       pl->cnt + CNT_INIT, pl->rtol, h, (pl->nb > 1) ? 0 : use_graph);
    pl->launches += 1;
    if (pl->nb > 1) {
        launch(k_batch_cond, 1, NTV, 0, s, (const int*)pl->ictl, pl->nb, pl->bdone, h, use_graph);
        pl->launches += 1;
    }
}

}  // namespace

cudaError_t poisson_enqueue_prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s,
                                     unsigned long long graph_handle, int mean_ready) {
    const PdlScope pdl(pl);
    const int use_graph = graph_handle != 0ULL;
    if (pl->dim == 3)
        prologue<3>(pl, b, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph, mean_ready);
    else
        prologue<2>(pl, b, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph, mean_ready);
    return cudaGetLastError();
}

void poisson_meanb_target(PoissonPlan* pl, double** part, unsigned int** cnt, double** out) {
    *part = pl->part0;
    *cnt = pl->cnt + CNT_MEANB;
    *out = pl->scal + PS_MEANB;
}

cudaError_t poisson_enqueue_body(PoissonPlan* pl, double* x, cudaStream_t s, unsigned long long graph_handle) {
    const PdlScope pdl(pl);
    const int use_graph = graph_handle != 0ULL;
    const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)graph_handle;
    if (pl->mg_fp32) {
        if (pl->dim == 3) body<float, 3>(pl, x, s, h, use_graph);
        else body<float, 2>(pl, x, s, h, use_graph);
    } else {
        if (pl->dim == 3) body<double, 3>(pl, x, s, h, use_graph);
        else body<double, 2>(pl, x, s, h, use_graph);
    }
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_epilogue(PoissonPlan* pl, double* x, cudaStream_t s, double* rep, int* status,
                                     int status_bit, int remove_mean) {
    const PdlScope pdl(pl);
    if (!remove_mean) {
        // the report alone (one block, no pass over x); a batch reports separately
        if (pl->nb == 1) {
            launch(k_sub_mean, dim3(1, 1), NTV, 0, s, x, 0LL, (const double*)pl->scal, (const int*)pl->ictl, rep,
                   status, status_bit);
            pl->launches += 1;
        }
        return cudaGetLastError();
    }
    const dim3 rb(reduce_blocks(pl->N), pl->nb);
    launch(k_mean, rb, NTV, 0, s, (const double*)x, pl->N, pl->part0, pl->scal, PS_MEANX, pl->cnt + CNT_MEANX);
    launch(k_sub_mean, rb, NTV, 0, s, x, pl->N, (const double*)pl->scal, (const int*)pl->ictl,
           pl->nb > 1 ? nullptr : rep, pl->nb > 1 ? nullptr : status, status_bit);
    pl->launches += 2;
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_remove_mean(PoissonPlan* pl, double* x, cudaStream_t s) {
    const PdlScope pdl(pl);
    const dim3 rb(reduce_blocks(pl->N), 1);
    launch(k_mean, rb, NTV, 0, s, (const double*)x, pl->N, pl->part0, pl->scal, PS_MEANX, pl->cnt + CNT_MEANX);
    launch(k_sub_mean, rb, NTV, 0, s, x, pl->N, (const double*)pl->scal, (const int*)pl->ictl, (double*)nullptr,
           (int*)nullptr, 0);
    return cudaGetLastError();
}

cudaError_t poisson_launch_single(PoissonPlan* pl, int which, cudaStream_t s) {
    const PdlScope pdl(pl);
    if (pl->nlev == 1) return cudaSuccess;
    const int f32 = pl->mg_fp32, d3 = pl->dim == 3;
    switch (which) {
        case 0:
            if (f32) d3 ? enqueue_down<float, 3>(pl, 0, s) : enqueue_down<float, 2>(pl, 0, s);
            else d3 ? enqueue_down<double, 3>(pl, 0, s) : enqueue_down<double, 2>(pl, 0, s);
            break;
        case 1:
            if (f32) d3 ? enqueue_pq<float, 3>(pl, s) : enqueue_pq<float, 2>(pl, s);
            else d3 ? enqueue_pq<double, 3>(pl, s) : enqueue_pq<double, 2>(pl, s);
            break;
        case 2:
            if (f32) d3 ? enqueue_up<float, 3>(pl, 0, s) : enqueue_up<float, 2>(pl, 0, s);
            else d3 ? enqueue_up<double, 3>(pl, 0, s) : enqueue_up<double, 2>(pl, 0, s);
            break;
        case 3:
            if (f32) d3 ? enqueue_tail<float, 3>(pl, s) : enqueue_tail<float, 2>(pl, s);
            else d3 ? enqueue_tail<double, 3>(pl, s) : enqueue_tail<double, 2>(pl, s);
            break;
        default: break;
    }
    return cudaGetLastError();
}

int poisson_prefix_iters(const PoissonPlan* pl) { return (pl->nb == 1 && pl->nlev > 1) ? pl->prefix : 0; }

double poisson_loop_iters(const PoissonPlan* pl, double iters) {
    const double u = (double)poisson_prefix_iters(pl);
    return iters > u ? iters - u : 0.0;
}

const int* poisson_done_flag(const PoissonPlan* pl) { return pl->nb > 1 ? pl->bdone : pl->ictl + PI_DONE; }

cudaError_t poisson_enqueue_batch_report(PoissonPlan* pl, double* const* rep, int* const* status, int status_bit,
                                         cudaStream_t s) {
    const PdlScope pdl(pl);
    launch(k_batch_report, 1, NTV, 0, s, (const double*)pl->scal, (const int*)pl->ictl, pl->nb, rep, status,
           status_bit);
    pl->launches += 1;
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_persistent(PoissonPlan* pl, const double* b, double* x, cudaStream_t s, int mean_ready) {
    if (!pl->persist) return cudaErrorInvalidValue;
    kp::Args a;
    std::memset(&a, 0, sizeof(a));
    for (int l = 0; l <= pl->top; ++l) a.lev[l] = lv_host<float>(pl, l);
    a.L0 = make_lv<double>(pl->lev[0], 2);
    a.top = pl->top;
    constexpr int CD = k2::cd_of(2), FU = k2::fu_of(2);
    for (int l = 0; l < pl->top; ++l) {
        a.dtx[l] = (pl->lev[l + 1].n[0] + CD - 1) / CD;
        a.dty[l] = (pl->lev[l + 1].n[1] + CD - 1) / CD;
        a.utx[l] = (pl->lev[l].n[0] + FU - 1) / FU;
        a.uty[l] = (pl->lev[l].n[1] + FU - 1) / FU;
        if (l >= 1) {
            a.upre[l] = (float*)pl->lev[l].upre;
            a.f[l] = (float*)pl->lev[l].f;
            a.upost[l] = (float*)pl->lev[l].upost;
        }
    }
    a.f[pl->top] = (float*)pl->lev[pl->top].f;
    a.upost[pl->top] = (float*)pl->lev[pl->top].upost;
    a.ptx = (pl->lev[0].n[0] + k2::FP - 1) / k2::FP;
    a.pty = (pl->lev[0].n[1] + k2::FP - 1) / k2::FP;
    a.b = b;
    a.x = x;
    a.r = pl->r;
    a.r32 = pl->r32;
    a.u0pre = (float*)pl->u0pre;
    a.z = (float*)pl->z;
    a.p0 = pl->p32[0];
    a.p1 = pl->p32[1];
    a.q = pl->q32;
    a.fdm_tab = pl->fdm_tab;
    a.part = pl->part0;
    a.scal = pl->scal;
    a.ictl = pl->ictl;
    a.bar = reinterpret_cast<unsigned*>(pl->part2);   // unused by the persistent solve
    a.rtol = pl->rtol;
    a.max_iter = pl->max_iter;
    a.vec4 = (pl->lev[0].n[0] % 4 == 0) && (((uintptr_t)x & 15) == 0);
    a.mean_ready = mean_ready;
    a.arrivals = (unsigned)pl->persist_grid;
    a.spin = kp::kSpin;
    if (const char* e = std::getenv("LOWMACH_PERSIST_TEST_TIMEOUT")) {
        // failure injection for the tests: a barrier that waits for one block
        // more than the grid has, with a short poll limit
        if (e[0] == '1') {
            a.arrivals = (unsigned)pl->persist_grid + 1u;
            a.spin = 1u << 14;
        }
    }
    cudaError_t e = cudaMemsetAsync(pl->part2, 0, kp::BAR_WORDS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)pl->persist_grid);
    cfg.blockDim = dim3(k2::NT);
    cfg.dynamicSmemBytes = pl->fdm_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kp::k_solve2, a);
    pl->launches += 1;
    return e;
}

cudaError_t poisson_solve_host_loop(PoissonPlan* pl, const double* b, double* x, cudaStream_t s) {
    if (pl->persist) {
        cudaError_t e = poisson_enqueue_persistent(pl, b, x, s, 0);
        if (e != cudaSuccess) return e;
        return poisson_enqueue_epilogue(pl, x, s, nullptr, nullptr, 0, 1);
    }
    const PdlScope pdl(pl);
    cudaError_t e = poisson_enqueue_prologue(pl, b, x, s, 0ULL, 0);
    if (e != cudaSuccess) return e;
    int done = 0;
    e = cudaMemcpyAsync(&done, poisson_done_flag(pl), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int guard = 0; !done && guard <= pl->max_iter; ++guard) {
        e = poisson_enqueue_body(pl, x, s, 0ULL);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(&done, poisson_done_flag(pl), sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
    }
    return poisson_enqueue_epilogue(pl, x, s, nullptr, nullptr, 0, 1);
}

}  // namespace lm
