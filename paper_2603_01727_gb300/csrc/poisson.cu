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

#include <cmath>
#include <cstring>
#include <vector>

#include "poisson.cuh"

namespace lm {

namespace {

constexpr int NTV = kThreads;            // block size of the pointwise kernels
constexpr int kTailThreads = 512;
constexpr long long kTailCellsF32 = 4096;   // largest level handled by the tail (FP32)
constexpr long long kTailCellsF64 = 512;    // (FP64: one SM's FP64 rate is 1/64 of FP32)
constexpr size_t kTailSmemMax = 200 * 1024;

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

// Last block of a grid to arrive (after its partial sums are visible).
__device__ __forceinline__ bool arrive_last(unsigned int* cnt) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        am_last = (atomicAdd(cnt, 1u) == nb - 1u);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last != 0;
}

template <int NT>
__device__ __forceinline__ double sum_parts_cg(const double* part, int np, double* smem) {
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += NT) v += __ldcg(part + i);
    return block_sum<NT>(v, smem);
}

__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ---------------------------------------------------------------------------
// down: red from zero, black, residual, restriction (one level)
// ---------------------------------------------------------------------------
template <class T, class TF, int DIM>
__global__ void __launch_bounds__(Tile<DIM>::NT) k_mg_down(LvT<T> L, LvT<T> C, const TF* __restrict__ f,
                                                           T* __restrict__ upre, T* __restrict__ fc) {
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
            fv = (T)f[gi];
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
            fv = (T)f[gi];
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
    double rz = 0.0, sz = 0.0;
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
                rz += (double)f[gi] * (double)u;
                sz += (double)u;
            }
        }
    }
    if (FINE) {
        __shared__ double red[NT / 32];
        rz = block_sum<NT>(rz, red);
        sz = block_sum<NT>(sz, red);
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (threadIdx.x == 0) {
            part_rz[block_linear()] = rz;
            part_sz[block_linear()] = sz;
        }
        if (arrive_last(cnt)) {
            const double RZ = sum_parts_cg<NT>(part_rz, nb, red);
            const double SZ = sum_parts_cg<NT>(part_sz, nb, red);
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
template <class T, int DIM>
__global__ void __launch_bounds__(Tile<DIM>::NT)
    k_cg_pq(LvT<double> L, const T* __restrict__ z, double* p0, double* p1, double* __restrict__ q,
            double* part, double* scal, const int* ictl, unsigned int* cnt) {
    constexpr int H = 1;
    using B = Box<DIM, H>;
    constexpr int NT = Tile<DIM>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* sp = reinterpret_cast<double*>(smraw);
    const int it = ictl[PI_IT];
    const double* pold = (it & 1) ? p0 : p1;
    double* pnew = (it & 1) ? p1 : p0;
    const double beta = scal[PS_BETA], mz = scal[PS_MEANZ];
    const int o[3] = {(int)blockIdx.x * B::FX - H, (int)blockIdx.y * B::FY - H,
                      (DIM == 3) ? (int)blockIdx.z * B::FZ - H : 0};
    int F[3] = {B::FX, B::FY, B::FZ};
    for (int i = threadIdx.x; i < B::SN; i += NT) {
        const int s[3] = {i % B::SX, (i / B::SX) % B::SY, i / B::S2};
        int gi, cl;
        bool own;
        double pv = 0.0;
        if (cell_info<double, DIM>(L, o, s, H, F, &gi, &cl, &own)) {
            pv = (double)z[gi] - mz;
            if (it > 0) pv = fma(beta, pold[gi], pv);
        }
        sp[i] = pv;
    }
    __syncthreads();
    double pq = 0.0;
    {
        constexpr int W = B::FX, RY = B::FY, RZ = B::FZ;
        for (int k = threadIdx.x; k < W * RY * RZ; k += NT) {
            const int s[3] = {1 + k % W, 1 + (k / W) % RY, (DIM == 3) ? 1 + k / (W * RY) : 0};
            int gi, cl;
            bool own;
            cell_info<double, DIM>(L, o, s, H, F, &gi, &cl, &own);
            if (!own) continue;
            const int i = s[0] + B::S1 * s[1] + B::S2 * s[2];
            const double pv = sp[i];
            const double qv = L.diag[cl] * pv - off_box<double, DIM, B>(L, sp, i);
            pnew[gi] = pv;
            q[gi] = qv;
            pq = fma(pv, qv, pq);
        }
    }
    __shared__ double red[NT / 32];
    pq = block_sum<NT>(pq, red);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) part[block_linear()] = pq;
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
                const double* __restrict__ q, long long N, double* part, double* scal, int* ictl,
                unsigned int* cnt, double rtol, int max_iter, cudaGraphConditionalHandle h, int use_graph) {
    const int it = ictl[PI_IT];
    const double* __restrict__ p = (it & 1) ? p1 : p0;
    const double alpha = scal[PS_ALPHA];
    double rr = 0.0;
    for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N; t += (long long)gridDim.x * NTV) {
        x[t] = fma(alpha, p[t], x[t]);
        const double rv = fma(-alpha, q[t], r[t]);
        r[t] = rv;
        rr = fma(rv, rv, rr);
    }
    __shared__ double red[NTV / 32];
    rr = block_sum<NTV>(rr, red);
    if (threadIdx.x == 0) part[blockIdx.x] = rr;
    if (arrive_last(cnt)) {
        const double RR = sum_parts_cg<NTV>(part, gridDim.x, red);
        if (threadIdx.x == 0) {
            const int itn = it + 1;
            ictl[PI_IT] = itn;
            scal[PS_RR] = RR;
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

__device__ __forceinline__ void coords(const int n[3], int t, int c[3]) {
    c[0] = t % n[0];
    const int r = t / n[0];
    c[1] = r % n[1];
    c[2] = r / n[1];
}

// Sum of b (partials; the last block stores the mean).
__global__ void __launch_bounds__(NTV) k_mean(const double* __restrict__ b, long long N, double* part,
                                              double* scal, int slot, unsigned int* cnt) {
    double v = 0.0;
    for (long long t = (long long)blockIdx.x * NTV + threadIdx.x; t < N; t += (long long)gridDim.x * NTV) v += b[t];
    __shared__ double red[NTV / 32];
    v = block_sum<NTV>(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
    if (arrive_last(cnt)) {
        const double s = sum_parts_cg<NTV>(part, gridDim.x, red);
        if (threadIdx.x == 0) {
            scal[slot] = s / (double)N;
            *cnt = 0u;
        }
    }
}

// r = -(b - mean b) - A x; ||f||^2, ||r||^2; the last block initialises the
// control words and the while-node conditional.
template <int DIM>
__global__ void __launch_bounds__(NTV)
    k_pcg_init(LvT<double> L, const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
               double* pff, double* prr, double* scal, int* ictl, unsigned int* cnt, double rtol,
               cudaGraphConditionalHandle h, int use_graph) {
    const double mean_b = scal[PS_MEANB];
    double ff = 0.0, rr = 0.0;
    for (int t = blockIdx.x * NTV + threadIdx.x; t < L.N; t += gridDim.x * NTV) {
        int c[3];
        coords(L.n, t, c);
        int cl;
        const double off = off_compact<double, DIM>(L, x, t, c, &cl);
        const double f = -(b[t] - mean_b);
        const double rv = f - (L.diag[cl] * x[t] - off);
        r[t] = rv;
        ff = fma(f, f, ff);
        rr = fma(rv, rv, rr);
    }
    __shared__ double red[NTV / 32];
    ff = block_sum<NTV>(ff, red);
    rr = block_sum<NTV>(rr, red);
    if (threadIdx.x == 0) {
        pff[blockIdx.x] = ff;
        prr[blockIdx.x] = rr;
    }
    if (arrive_last(cnt)) {
        const double FF = sum_parts_cg<NTV>(pff, gridDim.x, red);
        const double RR = sum_parts_cg<NTV>(prr, gridDim.x, red);
        if (threadIdx.x == 0) {
            scal[PS_FF] = FF;
            scal[PS_RR] = RR;
            scal[PS_RZ] = 0.0;
            scal[PS_BETA] = 0.0;
            scal[PS_ITERS] = 0.0;
            ictl[PI_IT] = 0;
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

// Zero-mean x; report iterations / residual / status.
__global__ void __launch_bounds__(NTV) k_sub_mean(double* __restrict__ x, long long N, const double* scal,
                                                  const int* ictl, double* rep, int* status, int bit) {
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
        coords(L.n, t, c);
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
            coords(L.n, t, c);
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
            coords(L.n, t, c);
            int cl;
            const T off = off_compact<T, DIM>(L, u, t, c, &cl);
            r[t] = f[t] - (L.diag[cl] * u[t] - off);
        }
        __syncthreads();
        for (int T_ = threadIdx.x; T_ < C.N; T_ += kTailThreads) {
            int I[3];
            coords(C.n, T_, I);
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
            coords(L.n, t, c);
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

int pick_top(const Shapes& s, int mg_fp32, size_t* smem_out) {
    if (s.nlev == 1) {
        *smem_out = 0;
        return 0;
    }
    const long long thr = mg_fp32 ? kTailCellsF32 : kTailCellsF64;
    const size_t w = mg_fp32 ? 4 : 8;
    for (int top = 1; top < s.nlev; ++top) {
        if (s.N[top] > thr && top < s.nlev - 1) continue;
        size_t b = 0;
        for (int l = top; l < s.nlev; ++l) b += 2 * w * (size_t)s.N[l];
        b += w * (size_t)s.N[top];
        if (b > kTailSmemMax && top < s.nlev - 1) continue;
        *smem_out = b;
        return top;
    }
    *smem_out = 0;
    return s.nlev - 1;
}

template <int DIM>
long long tile_blocks(const int n_fine[3]) {
    constexpr int FX = 2 * Tile<DIM>::CX, FY = 2 * Tile<DIM>::CY, FZ = (DIM == 3) ? 2 * Tile<DIM>::CZ : 1;
    return (long long)((n_fine[0] + FX - 1) / FX) * ((n_fine[1] + FY - 1) / FY) *
           ((DIM == 3) ? (n_fine[2] + FZ - 1) / FZ : 1);
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
    cudaFuncSetAttribute(k_cg_pq<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Box<3, 1>::SN * (int)sizeof(double));
}

}  // namespace

// ------------------------------ plan ----------------------------------------
size_t poisson_plan_bytes(int dim, const int n[3], const int periodic[3], int mg_fp32, int* nlev_out,
                          long long* Nc_out, const char** err) {
    (void)periodic;
    Shapes s;
    if (!make_shapes(dim, n, &s, err)) return 0;
    size_t tail_smem = 0;
    const int top = pick_top(s, mg_fp32, &tail_smem);
    const size_t w = mg_fp32 ? 4 : 8;
    const long long N = s.N[0];
    const long long nblk = (dim == 3) ? tile_blocks<3>(s.n[0]) : tile_blocks<2>(s.n[0]);
    const long long npart = nblk > kMaxPartials ? nblk : kMaxPartials;
    size_t b = 0;
    b += 4 * align256(sizeof(double) * N);                  // r p0 p1 q
    b += 2 * align256(w * N);                               // z u0pre
    b += 3 * align256(sizeof(double) * npart);              // partials
    b += align256(sizeof(double) * PS_NSCAL) + align256(sizeof(int) * PI_NINT) +
         align256(sizeof(unsigned int) * kNumCounters);
    for (int l = 1; l < s.nlev; ++l) {
        if (l < top) b += 3 * align256(w * s.N[l]);          // upre upost f
        else if (l == top) b += 2 * align256(w * s.N[l]);    // f (in), upost (out)
    }
    b += align256((mg_fp32 ? sizeof(LvT<float>) : sizeof(LvT<double>)) * s.nlev);
    const long long Nc = s.N[s.nlev - 1];
    b += align256(sizeof(double) * Nc * Nc) + align256(sizeof(float) * Nc * Nc);
    if (nlev_out) *nlev_out = s.nlev;
    if (Nc_out) *Nc_out = Nc;
    return b;
}

bool poisson_plan_init(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                       int mg_fp32, double rtol, int max_iter, void* ws, size_t ws_bytes,
                       std::vector<double>* minv_host, const char** err) {
    Shapes s;
    if (!make_shapes(dim, n, &s, err)) return false;
    const size_t need = poisson_plan_bytes(dim, n, periodic, mg_fp32, nullptr, nullptr, err);
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
    pl->top = pick_top(s, mg_fp32, &tail_smem);
    pl->mg_fp32 = mg_fp32;
    pl->N = s.N[0];
    pl->rtol = rtol;
    pl->max_iter = max_iter;
    pl->tail_smem = tail_smem;
    const long long nblk = (dim == 3) ? tile_blocks<3>(s.n[0]) : tile_blocks<2>(s.n[0]);
    pl->npart = (int)(nblk > kMaxPartials ? nblk : kMaxPartials);
    pl->r = (double*)take(sizeof(double) * pl->N);
    pl->p[0] = (double*)take(sizeof(double) * pl->N);
    pl->p[1] = (double*)take(sizeof(double) * pl->N);
    pl->q = (double*)take(sizeof(double) * pl->N);
    pl->z = take(w * pl->N);
    pl->u0pre = take(w * pl->N);
    pl->part0 = (double*)take(sizeof(double) * pl->npart);
    pl->part1 = (double*)take(sizeof(double) * pl->npart);
    pl->part2 = (double*)take(sizeof(double) * pl->npart);
    pl->scal = (double*)take(sizeof(double) * PS_NSCAL);
    pl->ictl = (int*)take(sizeof(int) * PI_NINT);
    pl->cnt = (unsigned int*)take(sizeof(unsigned int) * kNumCounters);
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
            L.upre = take(w * L.N);
            L.upost = take(w * L.N);
            L.f = take(w * L.N);
        } else if (l >= 1 && l == pl->top) {
            L.f = take(w * L.N);
            L.upost = take(w * L.N);
        }
    }
    const size_t lvsz = mg_fp32 ? sizeof(LvT<float>) : sizeof(LvT<double>);
    pl->levtab = take(lvsz * s.nlev);
    pl->Nc = s.N[s.nlev - 1];
    pl->Minv = (double*)take(sizeof(double) * pl->Nc * pl->Nc);
    pl->Minv_f = (float*)take(sizeof(float) * pl->Nc * pl->Nc);
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
    if (mg_fp32) set_smem_attrs<float>();
    else set_smem_attrs<double>();
    cudaGetLastError();   // attribute calls must not leave a sticky error behind
    return true;
}

bool poisson_upload_coarse(PoissonPlan* pl, const std::vector<double>& M, cudaStream_t s, const char** err) {
    if ((long long)M.size() != pl->Nc * pl->Nc) {
        *err = "coarse inverse not prepared";
        return false;
    }
    std::vector<float> Mf(M.size());
    for (size_t i = 0; i < M.size(); ++i) Mf[i] = (float)M[i];
    cudaError_t e = cudaMemcpyAsync(pl->Minv, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->Minv_f, Mf.data(), sizeof(float) * Mf.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->levtab, pl->levtab_host, pl->levtab_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->cnt, 0, sizeof(unsigned int) * kNumCounters, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ictl, 0, sizeof(int) * PI_NINT, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return false;
    }
    return true;
}

// ------------------------------ enqueue -------------------------------------
namespace {

enum { CNT_UP0 = 0, CNT_PQ = 1, CNT_UPD = 2, CNT_MEANB = 3, CNT_INIT = 4, CNT_MEANX = 5 };

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

template <class T, int DIM>
void enqueue_down(PoissonPlan* pl, int l, cudaStream_t s) {
    const LvT<T> L = lv_host<T>(pl, l), C = lv_host<T>(pl, l + 1);
    const dim3 grid = tile_grid<DIM>(pl->lev[l].n);
    const size_t smem = 2 * Box<DIM, 3>::SN * sizeof(T);
    T* fc = (T*)pl->lev[l + 1].f;
    if (l == 0)
        k_mg_down<T, double, DIM><<<grid, Tile<DIM>::NT, smem, s>>>(L, C, pl->r, (T*)pl->u0pre, fc);
    else
        k_mg_down<T, T, DIM><<<grid, Tile<DIM>::NT, smem, s>>>(L, C, (const T*)pl->lev[l].f, (T*)pl->lev[l].upre,
                                                               fc);
    pl->launches += 1;
}

template <class T, int DIM>
void enqueue_up(PoissonPlan* pl, int l, cudaStream_t s) {
    const LvT<T> L = lv_host<T>(pl, l), C = lv_host<T>(pl, l + 1);
    const dim3 grid = tile_grid<DIM>(pl->lev[l].n);
    const size_t smem = 2 * Box<DIM, 2>::SN * sizeof(T);
    const T* uc = (const T*)pl->lev[l + 1].upost;
    if (l == 0)
        k_mg_up<T, double, DIM, true><<<grid, Tile<DIM>::NT, smem, s>>>(
            L, C, (const T*)pl->u0pre, pl->r, uc, (T*)pl->z, pl->part0, pl->part1, pl->scal, pl->ictl,
            pl->cnt + CNT_UP0);
    else
        k_mg_up<T, T, DIM, false><<<grid, Tile<DIM>::NT, smem, s>>>(
            L, C, (const T*)pl->lev[l].upre, (const T*)pl->lev[l].f, uc, (T*)pl->lev[l].upost, nullptr, nullptr,
            nullptr, nullptr, nullptr);
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
    k_mg_tail<T, DIM><<<1, kTailThreads, pl->tail_smem, s>>>(lv_dev<T>(pl), a, (const T*)pl->lev[pl->top].f,
                                                             (T*)pl->lev[pl->top].upost, Minv);
    pl->launches += 1;
}

template <class T, int DIM>
void enqueue_pq(PoissonPlan* pl, cudaStream_t s) {
    const LvT<double> L = make_lv<double>(pl->lev[0], DIM);
    const dim3 grid = tile_grid<DIM>(pl->lev[0].n);
    k_cg_pq<T, DIM><<<grid, Tile<DIM>::NT, Box<DIM, 1>::SN * sizeof(double), s>>>(
        L, (const T*)pl->z, pl->p[0], pl->p[1], pl->q, pl->part2, pl->scal, pl->ictl, pl->cnt + CNT_PQ);
    pl->launches += 1;
}

template <class T, int DIM>
void body(PoissonPlan* pl, double* x, cudaStream_t s, cudaGraphConditionalHandle h, int use_graph) {
    if (pl->nlev == 1) {
        const T* Minv = (sizeof(T) == 4) ? (const T*)pl->Minv_f : (const T*)pl->Minv;
        k_direct<T><<<1, kTailThreads, 0, s>>>(Minv, (int)pl->Nc, pl->r, (T*)pl->z, pl->scal, pl->ictl);
        pl->launches += 1;
    } else {
        for (int l = 0; l < pl->top; ++l) enqueue_down<T, DIM>(pl, l, s);
        enqueue_tail<T, DIM>(pl, s);
        for (int l = pl->top - 1; l >= 0; --l) enqueue_up<T, DIM>(pl, l, s);
    }
    enqueue_pq<T, DIM>(pl, s);
    const int rb = reduce_blocks(pl->N);
    k_cg_update<<<rb, NTV, 0, s>>>(x, pl->r, pl->p[0], pl->p[1], pl->q, pl->N, pl->part0, pl->scal, pl->ictl,
                                   pl->cnt + CNT_UPD, pl->rtol, pl->max_iter, h, use_graph);
    pl->launches += 1;
}

template <int DIM>
void prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s, cudaGraphConditionalHandle h,
              int use_graph) {
    const int rb = reduce_blocks(pl->N);
    k_mean<<<rb, NTV, 0, s>>>(b, pl->N, pl->part0, pl->scal, PS_MEANB, pl->cnt + CNT_MEANB);
    const LvT<double> L = make_lv<double>(pl->lev[0], DIM);
    k_pcg_init<DIM><<<rb, NTV, 0, s>>>(L, b, x, pl->r, pl->part1, pl->part2, pl->scal, pl->ictl,
                                       pl->cnt + CNT_INIT, pl->rtol, h, use_graph);
    pl->launches += 2;
}

}  // namespace

cudaError_t poisson_enqueue_prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s,
                                     unsigned long long graph_handle) {
    const int use_graph = graph_handle != 0ULL;
    if (pl->dim == 3)
        prologue<3>(pl, b, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph);
    else
        prologue<2>(pl, b, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph);
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_body(PoissonPlan* pl, double* x, cudaStream_t s, unsigned long long graph_handle) {
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
                                     int status_bit) {
    const int rb = reduce_blocks(pl->N);
    k_mean<<<rb, NTV, 0, s>>>(x, pl->N, pl->part0, pl->scal, PS_MEANX, pl->cnt + CNT_MEANX);
    k_sub_mean<<<rb, NTV, 0, s>>>(x, pl->N, pl->scal, pl->ictl, rep, status, status_bit);
    pl->launches += 2;
    return cudaGetLastError();
}

cudaError_t poisson_launch_single(PoissonPlan* pl, int which, cudaStream_t s) {
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

cudaError_t poisson_solve_host_loop(PoissonPlan* pl, const double* b, double* x, cudaStream_t s) {
    cudaError_t e = poisson_enqueue_prologue(pl, b, x, s, 0ULL);
    if (e != cudaSuccess) return e;
    int done = 0;
    e = cudaMemcpyAsync(&done, pl->ictl + PI_DONE, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int guard = 0; !done && guard <= pl->max_iter; ++guard) {
        e = poisson_enqueue_body(pl, x, s, 0ULL);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(&done, pl->ictl + PI_DONE, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
    }
    return poisson_enqueue_epilogue(pl, x, s, nullptr, nullptr, 0);
}

}  // namespace lm
