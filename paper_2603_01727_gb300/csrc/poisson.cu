// Multigrid-preconditioned conjugate gradients for the pressure equation of
// the projection, L P = b - mean(b) with L = sum_d delta_1(delta_1 . / delta_1 x_d)
// / delta_1 x_d (paper Eqs 3.9, 3.17, 3.24; homogeneous Neumann on sides with a
// known boundary mass flux, Sec. 3.3; zero-mean solution selected as by the
// augmented-matrix method).  The paper solves this system with a sparse direct
// solver; here it is solved iteratively on the device:
//
//   A = -L (symmetric positive semi-definite, null space = constants);
//   CG on the mean-zero subspace, preconditioned by one symmetric V-cycle:
//   red-black Gauss-Seidel (pre: red, black; post: black, red), cell-centred
//   bilinear/trilinear prolongation P and restriction R = P^T / 2^dim, the
//   operator re-discretised on every level, and an exact dense solve of the
//   coarsest level (pseudo-inverse through A_c + c 1 1^T).
//
// Every reduction is a fixed-order two-stage sum (block partials, then one
// ordered sum), so a solve is bitwise reproducible run to run.

#include <cmath>
#include <cstring>
#include <vector>

#include "poisson.cuh"

namespace lm {

namespace {

constexpr int NT = kThreads;

__device__ __forceinline__ void lvl_coords(const MgLevel& L, long long t, int c[3]) {
    c[0] = (int)(t % L.n[0]);
    long long r = t / L.n[0];
    c[1] = (int)(r % L.n[1]);
    c[2] = (int)(r / L.n[1]);
}

__device__ __forceinline__ long long lvl_stride(const MgLevel& L, int d) {
    return d == 0 ? 1LL : (d == 1 ? (long long)L.n[0] : (long long)L.n[0] * L.n[1]);
}

// (A u)_t and the diagonal of A at cell t (A = -L, Neumann faces carry nothing).
template <int DIM>
__device__ __forceinline__ void stencil(const MgLevel& L, const double* __restrict__ u, long long t,
                                        const int c[3], double& off_sum, double& diag) {
    off_sum = 0.0;
    diag = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const long long s = lvl_stride(L, d);
        const int n = L.n[d];
        const double w = L.ih2[d];
        if (c[d] > 0) {
            off_sum += w * u[t - s];
            diag += w;
        } else if (L.periodic[d]) {
            off_sum += w * u[t + (long long)(n - 1) * s];
            diag += w;
        }
        if (c[d] < n - 1) {
            off_sum += w * u[t + s];
            diag += w;
        } else if (L.periodic[d]) {
            off_sum += w * u[t - (long long)(n - 1) * s];
            diag += w;
        }
    }
}

// One colour of red-black Gauss-Seidel on A u = f.
template <int DIM>
__global__ void k_smooth(MgLevel L, double* __restrict__ u, const double* __restrict__ f, int color) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.N) return;
    int c[3];
    lvl_coords(L, t, c);
    const int par = (c[0] + c[1] + (DIM == 3 ? c[2] : 0)) & 1;
    if (par != color) return;
    double off, diag;
    stencil<DIM>(L, u, t, c, off, diag);
    u[t] = (f[t] + off) / diag;
}

// Red sweep from u = 0: red cells get f/diag, black cells 0.
template <int DIM>
__global__ void k_zero_init_red(MgLevel L, double* __restrict__ u, const double* __restrict__ f) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.N) return;
    int c[3];
    lvl_coords(L, t, c);
    const int par = (c[0] + c[1] + (DIM == 3 ? c[2] : 0)) & 1;
    double diag = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const double w = L.ih2[d];
        if (c[d] > 0 || L.periodic[d]) diag += w;
        if (c[d] < L.n[d] - 1 || L.periodic[d]) diag += w;
    }
    u[t] = (par == 0) ? f[t] / diag : 0.0;
}

template <int DIM>
__global__ void k_residual(MgLevel L, const double* __restrict__ u, const double* __restrict__ f,
                           double* __restrict__ r) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.N) return;
    int c[3];
    lvl_coords(L, t, c);
    double off, diag;
    stencil<DIM>(L, u, t, c, off, diag);
    r[t] = f[t] - (diag * u[t] - off);
}

// 1D weights of R = P^T / 2 (times 2) for coarse index I and offset a = 0..3
// (fine index 2I-1+a); Neumann ends drop the outside fine cell and give the
// end cell the reflected weight.
__device__ __forceinline__ double rweight(int a, int I, int Nc, int periodic) {
    const double base[4] = {0.25, 0.75, 0.75, 0.25};
    double w = base[a];
    if (!periodic) {
        if (I == 0) {
            if (a == 0) w = 0.0;
            if (a == 1) w = 1.0;
        }
        if (I == Nc - 1) {
            if (a == 3) w = 0.0;
            if (a == 2) w = 1.0;
        }
    }
    return w;
}

template <int DIM>
__global__ void k_restrict(MgLevel F, MgLevel C, const double* __restrict__ rf, double* __restrict__ fc) {
    const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= C.N) return;
    int I[3];
    lvl_coords(C, T, I);
    double acc = 0.0;
    const int az = (DIM == 3) ? 4 : 1;
    for (int cz = 0; cz < az; ++cz) {
        double wz = 1.0;
        int fz = 0;
        if (DIM == 3) {
            wz = rweight(cz, I[2], C.n[2], C.periodic[2]);
            if (wz == 0.0) continue;
            fz = 2 * I[2] - 1 + cz;
            if (fz < 0) fz += F.n[2];
            if (fz >= F.n[2]) fz -= F.n[2];
        }
        for (int cy = 0; cy < 4; ++cy) {
            const double wy = rweight(cy, I[1], C.n[1], C.periodic[1]);
            if (wy == 0.0) continue;
            int fy = 2 * I[1] - 1 + cy;
            if (fy < 0) fy += F.n[1];
            if (fy >= F.n[1]) fy -= F.n[1];
            for (int cx = 0; cx < 4; ++cx) {
                const double wx = rweight(cx, I[0], C.n[0], C.periodic[0]);
                if (wx == 0.0) continue;
                int fx = 2 * I[0] - 1 + cx;
                if (fx < 0) fx += F.n[0];
                if (fx >= F.n[0]) fx -= F.n[0];
                const long long ft = fx + (long long)F.n[0] * (fy + (long long)F.n[1] * fz);
                acc += wx * wy * wz * rf[ft];
            }
        }
    }
    fc[T] = acc * (DIM == 3 ? 0.125 : 0.25);
}

// u_f += P u_c (cell-centred bilinear / trilinear; Neumann ends reflect).
template <int DIM>
__global__ void k_prolong(MgLevel F, MgLevel C, const double* __restrict__ uc, double* __restrict__ uf) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F.N) return;
    int f[3];
    lvl_coords(F, t, f);
    int i0[3], i1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= DIM) {
            i0[d] = i1[d] = 0;
            continue;
        }
        const int I = f[d] >> 1;
        int J = (f[d] & 1) ? I + 1 : I - 1;
        if (J < 0) J = C.periodic[d] ? C.n[d] - 1 : I;
        if (J >= C.n[d]) J = C.periodic[d] ? 0 : I;
        i0[d] = I;
        i1[d] = J;
    }
    double acc = 0.0;
    const int nz = (DIM == 3) ? 2 : 1;
    for (int bz = 0; bz < nz; ++bz) {
        const int kz = (DIM == 3) ? (bz ? i1[2] : i0[2]) : 0;
        const double wz = (DIM == 3) ? (bz ? 0.25 : 0.75) : 1.0;
        for (int by = 0; by < 2; ++by) {
            const int ky = by ? i1[1] : i0[1];
            const double wy = by ? 0.25 : 0.75;
            for (int bx = 0; bx < 2; ++bx) {
                const int kx = bx ? i1[0] : i0[0];
                const double wx = bx ? 0.25 : 0.75;
                acc += wx * wy * wz * uc[kx + (long long)C.n[0] * (ky + (long long)C.n[1] * kz)];
            }
        }
    }
    uf[t] += acc;
}

// Coarsest level: u = Minv f (one block, ordered dot products).
__global__ void k_coarse_solve(const double* __restrict__ M, long long Nc, const double* __restrict__ f,
                               double* __restrict__ u) {
    for (long long i = threadIdx.x; i < Nc; i += blockDim.x) {
        double acc = 0.0;
        for (long long j = 0; j < Nc; ++j) acc += M[i * Nc + j] * f[j];
        u[i] = acc;
    }
}

// ------------------------------- Krylov part --------------------------------
__global__ void k_sum_partial(const double* __restrict__ x, long long N, double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    double v = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT)
        v += x[t];
    v = block_sum<NT>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// r = -(b - mean b) - A x ; partials of ||f||^2 and ||r||^2.
template <int DIM>
__global__ void k_pcg_init(MgLevel L, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ r, const double* __restrict__ pb, int npb,
                           double* __restrict__ pff, double* __restrict__ prr) {
    __shared__ double sm[NT / 32];
    const double mean_b = sum_partials<NT>(pb, npb, sm) / (double)L.N;
    double ff = 0.0, rr = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < L.N; t += (long long)gridDim.x * NT) {
        int c[3];
        lvl_coords(L, t, c);
        double off, diag;
        stencil<DIM>(L, x, t, c, off, diag);
        const double f = -(b[t] - mean_b);
        const double rv = f - (diag * x[t] - off);
        r[t] = rv;
        ff += f * f;
        rr += rv * rv;
    }
    ff = block_sum<NT>(ff, sm);
    rr = block_sum<NT>(rr, sm);
    if (threadIdx.x == 0) {
        pff[blockIdx.x] = ff;
        prr[blockIdx.x] = rr;
    }
}

__global__ void k_ctrl_init(double* scal, int* ictl, const double* pff, const double* prr, int np,
                            double rtol, cudaGraphConditionalHandle h, int use_graph) {
    __shared__ double sm[NT / 32];
    const double ff = sum_partials<NT>(pff, np, sm);
    const double rr = sum_partials<NT>(prr, np, sm);
    if (threadIdx.x == 0) {
        scal[PS_FF] = ff;
        scal[PS_RR] = rr;
        scal[PS_RZ] = 0.0;
        scal[PS_BETA] = 0.0;
        scal[PS_ITERS] = 0.0;
        ictl[PI_IT] = 0;
        ictl[PI_NOCONV] = 0;
        const int zero = !(ff > 0.0);
        ictl[PI_ZERO] = zero;
        const int done = zero || (rr <= rtol * rtol * ff);
        ictl[PI_DONE] = done;
        scal[PS_RELRES] = zero ? 0.0 : sqrt(rr / ff);
        if (!(rr == rr)) {             // non-finite input
            ictl[PI_DONE] = 1;
            ictl[PI_NOCONV] = 1;
        }
        if (use_graph) cudaGraphSetConditional(h, ictl[PI_DONE] ? 0u : 1u);
    }
}

__global__ void k_dot_rz(const double* __restrict__ r, const double* __restrict__ z, long long N,
                         double* __restrict__ prz, double* __restrict__ psz) {
    __shared__ double sm[NT / 32];
    double rz = 0.0, sz = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT) {
        rz += r[t] * z[t];
        sz += z[t];
    }
    rz = block_sum<NT>(rz, sm);
    sz = block_sum<NT>(sz, sm);
    if (threadIdx.x == 0) {
        prz[blockIdx.x] = rz;
        psz[blockIdx.x] = sz;
    }
}

__global__ void k_ctrl_beta(double* scal, const int* ictl, const double* prz, const double* psz, int np,
                            long long N) {
    __shared__ double sm[NT / 32];
    const double rz = sum_partials<NT>(prz, np, sm);
    const double sz = sum_partials<NT>(psz, np, sm);
    if (threadIdx.x == 0) {
        const double beta = (ictl[PI_IT] == 0) ? 0.0 : rz / scal[PS_RZ];
        scal[PS_BETA] = beta;
        scal[PS_RZ] = rz;
        scal[PS_MEANZ] = sz / (double)N;
    }
}

__global__ void k_update_p(const double* __restrict__ z, double* __restrict__ p, const double* scal,
                           const int* ictl, long long N) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    // first iteration: p = z (p holds no previous direction, whatever its bits)
    const double zc = z[t] - scal[PS_MEANZ];
    p[t] = (ictl[PI_IT] == 0) ? zc : zc + scal[PS_BETA] * p[t];
}

template <int DIM>
__global__ void k_matvec_dot(MgLevel L, const double* __restrict__ p, double* __restrict__ q,
                             double* __restrict__ ppq) {
    __shared__ double sm[NT / 32];
    double pq = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < L.N; t += (long long)gridDim.x * NT) {
        int c[3];
        lvl_coords(L, t, c);
        double off, diag;
        stencil<DIM>(L, p, t, c, off, diag);
        const double qv = diag * p[t] - off;
        q[t] = qv;
        pq += p[t] * qv;
    }
    pq = block_sum<NT>(pq, sm);
    if (threadIdx.x == 0) ppq[blockIdx.x] = pq;
}

__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, long long N, const double* scal,
                            const double* ppq, int np, double* __restrict__ prr) {
    __shared__ double sm[NT / 32];
    const double pq = sum_partials<NT>(ppq, np, sm);
    const double alpha = scal[PS_RZ] / pq;
    double rr = 0.0;
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT) {
        x[t] += alpha * p[t];
        const double rv = r[t] - alpha * q[t];
        r[t] = rv;
        rr += rv * rv;
    }
    rr = block_sum<NT>(rr, sm);
    if (threadIdx.x == 0) prr[blockIdx.x] = rr;
}

__global__ void k_ctrl_conv(double* scal, int* ictl, const double* prr, int np, double rtol, int max_iter,
                            cudaGraphConditionalHandle h, int use_graph) {
    __shared__ double sm[NT / 32];
    const double rr = sum_partials<NT>(prr, np, sm);
    if (threadIdx.x == 0) {
        const int it = ictl[PI_IT] + 1;
        ictl[PI_IT] = it;
        scal[PS_RR] = rr;
        const double ff = scal[PS_FF];
        const int conv = (rr <= rtol * rtol * ff);
        const int bad = !(rr == rr) || !(rr < 1e300);
        const int done = conv || bad || (it >= max_iter);
        ictl[PI_DONE] = done;
        if (done && !conv) ictl[PI_NOCONV] = 1;
        scal[PS_ITERS] = (double)it;
        scal[PS_RELRES] = sqrt(rr / ff);
        if (use_graph) cudaGraphSetConditional(h, done ? 0u : 1u);
    }
}

__global__ void k_sub_mean(double* __restrict__ x, long long N, const double* part, int np,
                           const int* ictl) {
    __shared__ double sm[NT / 32];
    const double mean = sum_partials<NT>(part, np, sm) / (double)N;
    const int zero = ictl[PI_ZERO];
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < N; t += (long long)gridDim.x * NT)
        x[t] = zero ? 0.0 : (x[t] - mean);
}

// ------------------------------ host helpers --------------------------------
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Shapes {
    int nlev;
    int n[kMaxLevels][3];
    long long N[kMaxLevels];
};

bool make_shapes(int dim, const int n[3], const int periodic[3], Shapes* s, const char** err) {
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
    (void)periodic;
    if (s->N[s->nlev - 1] > kMaxCoarse) {
        *err = "grid does not coarsen to <= 1024 cells by halving (use extents with more factors of 2)";
        return false;
    }
    return true;
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
std::vector<double> coarse_inverse(const MgLevel& L) {
    const long long Nc = L.N;
    std::vector<double> A((size_t)(Nc * Nc), 0.0);
    double dmax = 0.0;
    for (long long t = 0; t < Nc; ++t) {
        int c[3] = {(int)(t % L.n[0]), (int)((t / L.n[0]) % L.n[1]), (int)(t / ((long long)L.n[0] * L.n[1]))};
        double diag = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (L.n[d] == 1 && d == 2) continue;
            const long long s = d == 0 ? 1 : (d == 1 ? L.n[0] : (long long)L.n[0] * L.n[1]);
            const double w = L.ih2[d];
            if (w == 0.0) continue;
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

}  // namespace

size_t poisson_plan_bytes(int dim, const int n[3], const int periodic[3], int* nlev_out, long long* Nc_out,
                          const char** err) {
    Shapes s;
    if (!make_shapes(dim, n, periodic, &s, err)) return 0;
    size_t b = 0;
    const long long N = s.N[0];
    b += 4 * align256(sizeof(double) * N);                  // r z p q
    b += 3 * align256(sizeof(double) * kMaxPartials);       // partials
    b += align256(sizeof(double) * PS_NSCAL) + align256(sizeof(int) * PI_NINT);
    for (int l = 0; l < s.nlev; ++l) {
        if (l > 0) b += 2 * align256(sizeof(double) * s.N[l]);   // u f
        b += align256(sizeof(double) * s.N[l]);                  // r scratch
    }
    const long long Nc = s.N[s.nlev - 1];
    b += align256(sizeof(double) * Nc * Nc);
    if (nlev_out) *nlev_out = s.nlev;
    if (Nc_out) *Nc_out = Nc;
    return b;
}

bool poisson_plan_init(PoissonPlan* pl, int dim, const int n[3], const double h[3], const int periodic[3],
                       double rtol, int max_iter, void* ws, size_t ws_bytes, std::vector<double>* minv_host,
                       const char** err) {
    Shapes s;
    if (!make_shapes(dim, n, periodic, &s, err)) return false;
    const size_t need = poisson_plan_bytes(dim, n, periodic, nullptr, nullptr, err);
    if (need == 0) return false;
    if (ws_bytes < need) {
        *err = "poisson workspace too small";
        return false;
    }
    if (((uintptr_t)ws & 255) != 0) {
        *err = "workspace must be 256-byte aligned";
        return false;
    }
    std::memset(pl, 0, sizeof(*pl));
    char* cur = (char*)ws;
    auto take = [&](size_t bytes) {
        char* p = cur;
        cur += align256(bytes);
        return p;
    };
    pl->dim = dim;
    pl->nlev = s.nlev;
    pl->N = s.N[0];
    pl->rtol = rtol;
    pl->max_iter = max_iter;
    pl->r = (double*)take(sizeof(double) * pl->N);
    pl->z = (double*)take(sizeof(double) * pl->N);
    pl->p = (double*)take(sizeof(double) * pl->N);
    pl->q = (double*)take(sizeof(double) * pl->N);
    pl->part0 = (double*)take(sizeof(double) * kMaxPartials);
    pl->part1 = (double*)take(sizeof(double) * kMaxPartials);
    pl->part2 = (double*)take(sizeof(double) * kMaxPartials);
    pl->scal = (double*)take(sizeof(double) * PS_NSCAL);
    pl->ictl = (int*)take(sizeof(int) * PI_NINT);
    for (int l = 0; l < s.nlev; ++l) {
        MgLevel& L = pl->lev[l];
        for (int d = 0; d < 3; ++d) {
            L.n[d] = s.n[l][d];
            L.periodic[d] = (d < dim) ? periodic[d] : 0;
            const double scale = (double)(1 << l);
            L.h[d] = (d < dim) ? h[d] * scale : 1.0;
            L.ih2[d] = (d < dim) ? 1.0 / (L.h[d] * L.h[d]) : 0.0;
        }
        L.N = s.N[l];
        if (l > 0) {
            L.u = (double*)take(sizeof(double) * L.N);
            L.f = (double*)take(sizeof(double) * L.N);
        }
        L.r = (double*)take(sizeof(double) * L.N);
    }
    pl->Nc = s.N[s.nlev - 1];
    pl->Minv = (double*)take(sizeof(double) * pl->Nc * pl->Nc);
    *minv_host = coarse_inverse(pl->lev[s.nlev - 1]);
    return true;
}

bool poisson_upload_coarse(PoissonPlan* pl, const std::vector<double>& M, cudaStream_t s, const char** err) {
    if ((long long)M.size() != pl->Nc * pl->Nc) {
        *err = "coarse inverse not prepared";
        return false;
    }
    cudaError_t e = cudaMemcpyAsync(pl->Minv, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return false;
    }
    return true;
}

// ------------------------------ enqueue -------------------------------------
template <int DIM>
static void vcycle(PoissonPlan* pl, cudaStream_t s) {
    const int Lc = pl->nlev - 1;
    for (int l = 0; l < Lc; ++l) {
        MgLevel& L = pl->lev[l];
        double* u = (l == 0) ? pl->z : L.u;
        const double* f = (l == 0) ? pl->r : L.f;
        const int nb = blocks_for(L.N);
        k_zero_init_red<DIM><<<nb, NT, 0, s>>>(L, u, f);
        k_smooth<DIM><<<nb, NT, 0, s>>>(L, u, f, 1);
        k_residual<DIM><<<nb, NT, 0, s>>>(L, u, f, L.r);
        MgLevel& C = pl->lev[l + 1];
        k_restrict<DIM><<<blocks_for(C.N), NT, 0, s>>>(L, C, L.r, C.f);
        pl->launches += 4;
    }
    {
        MgLevel& C = pl->lev[Lc];
        double* u = (Lc == 0) ? pl->z : C.u;
        const double* f = (Lc == 0) ? pl->r : C.f;
        k_coarse_solve<<<1, NT, 0, s>>>(pl->Minv, pl->Nc, f, u);
        pl->launches += 1;
    }
    for (int l = Lc - 1; l >= 0; --l) {
        MgLevel& L = pl->lev[l];
        MgLevel& C = pl->lev[l + 1];
        double* u = (l == 0) ? pl->z : L.u;
        const double* f = (l == 0) ? pl->r : L.f;
        const int nb = blocks_for(L.N);
        k_prolong<DIM><<<nb, NT, 0, s>>>(L, C, C.u, u);
        k_smooth<DIM><<<nb, NT, 0, s>>>(L, u, f, 1);
        k_smooth<DIM><<<nb, NT, 0, s>>>(L, u, f, 0);
        pl->launches += 3;
    }
}

template <int DIM>
static void prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s) {
    const int rb = reduce_blocks(pl->N);
    k_sum_partial<<<rb, NT, 0, s>>>(b, pl->N, pl->part0);
    k_pcg_init<DIM><<<rb, NT, 0, s>>>(pl->lev[0], b, x, pl->r, pl->part0, rb, pl->part1, pl->part2);
    pl->launches += 2;
}

template <int DIM>
static void body(PoissonPlan* pl, double* x, cudaStream_t s, cudaGraphConditionalHandle h, int use_graph) {
    const int rb = reduce_blocks(pl->N);
    const int nb = blocks_for(pl->N);
    vcycle<DIM>(pl, s);
    k_dot_rz<<<rb, NT, 0, s>>>(pl->r, pl->z, pl->N, pl->part0, pl->part1);
    k_ctrl_beta<<<1, NT, 0, s>>>(pl->scal, pl->ictl, pl->part0, pl->part1, rb, pl->N);
    k_update_p<<<nb, NT, 0, s>>>(pl->z, pl->p, pl->scal, pl->ictl, pl->N);
    k_matvec_dot<DIM><<<rb, NT, 0, s>>>(pl->lev[0], pl->p, pl->q, pl->part0);
    k_update_xr<<<rb, NT, 0, s>>>(x, pl->r, pl->p, pl->q, pl->N, pl->scal, pl->part0, rb, pl->part1);
    k_ctrl_conv<<<1, NT, 0, s>>>(pl->scal, pl->ictl, pl->part1, rb, pl->rtol, pl->max_iter, h, use_graph);
    pl->launches += 6;
}

cudaError_t poisson_enqueue_prologue(PoissonPlan* pl, const double* b, double* x, cudaStream_t s) {
    if (pl->dim == 3)
        prologue<3>(pl, b, x, s);
    else
        prologue<2>(pl, b, x, s);
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_ctrl_init(PoissonPlan* pl, cudaStream_t s, cudaGraphConditionalHandle h,
                                      int use_graph) {
    const int rb = reduce_blocks(pl->N);
    k_ctrl_init<<<1, NT, 0, s>>>(pl->scal, pl->ictl, pl->part1, pl->part2, rb, pl->rtol, h, use_graph);
    pl->launches += 1;
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_body(PoissonPlan* pl, double* x, cudaStream_t s, unsigned long long graph_handle) {
    const int use_graph = graph_handle != 0ULL;
    if (pl->dim == 3)
        body<3>(pl, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph);
    else
        body<2>(pl, x, s, (cudaGraphConditionalHandle)graph_handle, use_graph);
    return cudaGetLastError();
}

cudaError_t poisson_enqueue_epilogue(PoissonPlan* pl, double* x, cudaStream_t s) {
    const int rb = reduce_blocks(pl->N);
    k_sum_partial<<<rb, NT, 0, s>>>(x, pl->N, pl->part0);
    k_sub_mean<<<rb, NT, 0, s>>>(x, pl->N, pl->part0, rb, pl->ictl);
    pl->launches += 2;
    return cudaGetLastError();
}

template <int DIM>
static void single(PoissonPlan* pl, int which, cudaStream_t s) {
    MgLevel& L = pl->lev[0];
    const int nb = blocks_for(L.N);
    if (which == 0) {
        k_smooth<DIM><<<nb, NT, 0, s>>>(L, pl->z, pl->r, 1);
    } else if (which == 1) {
        k_matvec_dot<DIM><<<reduce_blocks(L.N), NT, 0, s>>>(L, pl->p, pl->q, pl->part0);
    } else if (pl->nlev > 1) {
        k_residual<DIM><<<nb, NT, 0, s>>>(L, pl->z, pl->r, L.r);
        MgLevel& C = pl->lev[1];
        k_restrict<DIM><<<blocks_for(C.N), NT, 0, s>>>(L, C, L.r, C.f);
    }
}

cudaError_t poisson_launch_single(PoissonPlan* pl, int which, cudaStream_t s) {
    if (pl->dim == 3)
        single<3>(pl, which, s);
    else
        single<2>(pl, which, s);
    return cudaGetLastError();
}

cudaError_t poisson_solve_host_loop(PoissonPlan* pl, const double* b, double* x, cudaStream_t s) {
    cudaError_t e = poisson_enqueue_prologue(pl, b, x, s);
    if (e != cudaSuccess) return e;
    e = poisson_enqueue_ctrl_init(pl, s, 0, 0);
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
    return poisson_enqueue_epilogue(pl, x, s);
}

}  // namespace lm
