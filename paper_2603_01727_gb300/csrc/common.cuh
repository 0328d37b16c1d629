// Shared device-side definitions of the sm_103a path: grid geometry, the
// padded field layout, physical constants of a run and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lm {

constexpr int kMaxDim = 3;

enum BcKind : int { BC_PERIODIC = 0, BC_INFLOW = 1, BC_OUTFLOW = 2, BC_WALL = 3, BC_SLIP = 4, BC_WALL_T = 5 };

// Grid geometry.  Cell fields live in a padded array with one ghost layer on
// each side of every active direction (ghost index 0 and n+1, interior 1..n),
// x fastest.  In 2D the z extent is 1 and has no ghosts.
// Unsigned 32-bit division by an invariant divisor as a multiply-high and two
// shifts (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0)
// where t = mulhi(m, n), exact for every 32-bit n.  Cell indices stay below
// 2^32, so the index maps below need no 64-bit division.
struct DivU32 {
    unsigned m;
    int s1, s2;
};
inline DivU32 make_divu32(unsigned d) {
    int l = 0;
    while ((1ULL << l) < d) ++l;
    DivU32 f;
    f.m = (unsigned)(((1ULL << 32) * ((1ULL << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}
__host__ __device__ __forceinline__ unsigned divu32(unsigned n, const DivU32& f) {
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(f.m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Geom {
    int dim;
    int n[3];        // interior cells (n[2] = 1 in 2D)
    int p[3];        // padded extents
    long long s[3];  // strides of the padded array (s[0] = 1)
    long long npad;  // padded cells
    long long ncell; // interior cells
    double h[3];     // spacing
    double ih[3];    // 1 / h
    double ih2[3];   // 1 / h^2
    double dV;       // cell volume
    int periodic[3];
    DivU32 dn0, dn1; // division by n[0], n[1] (interior index maps)
    DivU32 dp0, dp1; // division by p[0], p[1] (padded index maps)
    int tile_x;      // projection kernel: x extent of a block's cell tile (0: linear)
};

// Interior linear index t (x fastest over the interior) -> padded index.
__host__ __device__ inline void interior_coords(const Geom& g, long long t, int c[3]) {
    const unsigned tt = (unsigned)t;
    const unsigned r = divu32(tt, g.dn0);
    const unsigned k = divu32(r, g.dn1);
    c[0] = (int)(tt - r * (unsigned)g.n[0]);
    c[1] = (int)(r - k * (unsigned)g.n[1]);
    c[2] = (int)k;
}

__host__ __device__ inline long long pad_index(const Geom& g, long long t) {
    int c[3];
    interior_coords(g, t, c);
    const long long kz = (g.dim == 3) ? (c[2] + 1) : 0;
    return (long long)(c[0] + 1) + (long long)(c[1] + 1) * g.s[1] + kz * g.s[2];
}

// Physical constants of a run (paper notation), derived once on the host.
struct Phys {
    double S, Q, k, Pe, PrPe, zeta;   // Eqs 2.34-2.37, 3.34; PrPe = Pr/Pe
    double Le_F, Le_O, N_F, N_O;       // Eqs 3.35a-b
    double sigma, inv_Fr2;
    double Fshift;                     // level translation of F_eps (text after Eq 3.41)
    double kappa_in, rho_in_T;         // inflow transport coefficient, inflow temperature
    double inflow_v[3], inflow_Z, inflow_H;
    double cA, cB, cT;                 // T = cT (cA (|x| + log1p(e^-2|x|)) + cB (Z - 1) + H), Eq 3.42
    double iPe, iLePe;                 // 1/Pe, 1/(Le Pe) (uniform Le)
    int incompressible, closed;        // closed: p0 != 1 (enclosed, Eq 2.40, or semi-enclosed)
    int semi;                          // semi-enclosed: p0 from the ODE of Eq 2.38
    double NpF, NpO;                   // N'_F = -1/S, N'_O = 1 (Eq 2.39)
    double ode_gV, ode_heat;           // gamma / V and Q / ((S + 1) Pe) of Eq 2.38
    int mixed;                         // 1: FP32 stencil arithmetic and multigrid (SIM_MIXED)
    int sigma_is_07;                   // sigma == 0.7 exactly (paper value, Eq 2.50)
    int transport;                     // 0: kappa = T^sigma (Eq 2.50); 1: Sutherland (Eq 4.12)
    double suth_C;                     // Sutherland constant over the reference temperature
    double wall_H[3][2];               // Dirichlet H of isothermal walls, [direction][side]
    double kap_wall[3][2];             // kappa of the isothermal walls' states
};

// Transport coefficient of a temperature, FP64 (Eq 2.50 or Eq 4.12).
__host__ __device__ inline double kappa_of(const Phys& ph, double T) {
    if (ph.transport == 1) return pow(T, 1.5) * (1.0 + ph.suth_C) / (T + ph.suth_C);
    return pow(T, ph.sigma);
}

// ---------------------------------------------------------------------------
// Forward-mode dual number (value, derivative): instantiating a cell function
// with Dual evaluates its exact derivative along one seeded input, which the
// adjoint kernels assemble into transposed Jacobian-vector products.
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    __host__ __device__ Dual() : v(0.0), d(0.0) {}
    __host__ __device__ Dual(double x) : v(x), d(0.0) {}
    __host__ __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
__host__ __device__ inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
__device__ inline double tanh_c(double x) { return tanh(x); }
__device__ inline Dual tanh_c(Dual x) {
    const double t = tanh(x.v);
    return Dual(t, (1.0 - t * t) * x.d);
}

// ---------------------------------------------------------------------------
// Float-float number: an unevaluated sum hi + lo of two FP32 values with
// |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32 pipes
// (GB300 runs FP64 at 1/64 of the FP32 rate).  Error-free transformations:
// Knuth's two-sum, the fast two-sum of Dekker (|a| >= |b|), and the exact
// product error by one fused multiply-add.  Addition is the one-pass
// ("sloppy") form: relative error ~2^-44, or an absolute ~2^-48 max(|a|,|b|)
// under cancellation; multiplication ~2^-46.  Conversions from double keep 48
// bits of the input.
// ---------------------------------------------------------------------------
struct FF {
    float hi, lo;
    __device__ __forceinline__ FF() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ FF(float h, float l) : hi(h), lo(l) {}
    // Split of a double by integer operations on its bits (no FP64 or
    // conversion instructions): hi = x truncated to 24 significant bits, lo =
    // the remaining 29 bits truncated to 24; |x| < 2^-74 (far below every
    // field's scale) keeps hi only, zero and non-normal floats map to zero.
    __device__ __forceinline__ FF(double x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const unsigned int h32 = (unsigned int)(b >> 32), l32 = (unsigned int)b;
        const unsigned int sgn = h32 & 0x80000000u;
        const int e = (int)((h32 >> 20) & 0x7ffu);
        if (e < 897 || e > 1150) {
            hi = 0.f;
            lo = 0.f;
            return;
        }
        hi = __uint_as_float(sgn | ((unsigned int)(e - 896) << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29));
        const unsigned int r = l32 & 0x1fffffffu;
        const int lz = __clz(r);
        const int ef = e - 917 - lz;   // float exponent field of r * 2^(e - 1075)
        lo = (r == 0u || ef < 1) ? 0.f
                                 : __uint_as_float(sgn | ((unsigned int)ef << 23) | ((r << (lz + 1)) >> 9));
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return FF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ FF operator+(FF a, FF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return ff_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF operator-(FF a) { return FF(-a.hi, -a.lo); }
__device__ __forceinline__ FF operator-(FF a, FF b) { return a + (-b); }
__device__ __forceinline__ FF operator*(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF operator/(FF a, FF b) {
    // q1 = a/b in FP32, then one correction from the float-float remainder
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const FF r = a - b * FF(q1, 0.f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}
// Exact float -> double by integer operations on the bits (normal floats;
// zero and subnormal floats give zero, infinities and NaN give NaN), so that
// no conversion instruction is issued.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    if (e == 0xffu) return __longlong_as_double(0x7ff8000000000000LL);
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ FF& operator+=(FF& a, FF b) { return a = a + b; }
__device__ __forceinline__ FF& operator-=(FF& a, FF b) { return a = a - b; }
__device__ inline FF tanh_c(FF x) { return FF(tanh((double)x)); }

// ---------------------------------------------------------------------------
// Deterministic block reduction (fixed tree for a fixed block size).
// ---------------------------------------------------------------------------
template <int NT>
__device__ inline double block_sum(double v, double* smem /* NT/32 doubles */) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? smem[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (l == 0) smem[0] = r;
    }
    __syncthreads();
    r = smem[0];
    __syncthreads();
    return r;
}

// Block maximum of non-negative values (same tree as block_sum).
template <int NT>
__device__ inline double block_max(double v, double* smem /* NT/32 doubles */) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? smem[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (l == 0) smem[0] = r;
    }
    __syncthreads();
    r = smem[0];
    __syncthreads();
    return r;
}

// FP32 variant (for the FP32 inner Krylov loop); same fixed tree.
template <int NT>
__device__ inline float block_sum_f(float v, float* smem /* NT/32 floats */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    float r = 0.0f;
    if (w == 0) {
        r = (l < NT / 32) ? smem[l] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (l == 0) smem[0] = r;
    }
    __syncthreads();
    r = smem[0];
    __syncthreads();
    return r;
}

// Two sums at once, each with the tree of block_sum / block_sum_f (bitwise the
// same values as two separate calls, with half the barriers).
template <int NT, class V>
__device__ inline void block_sum2_t(V& a, V& b, V* smem /* 2 NT/32 */) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        smem[w] = a;
        smem[NT / 32 + w] = b;
    }
    __syncthreads();
    if (w == 0) {
        V ra = (l < NT / 32) ? smem[l] : (V)0;
        V rb = (l < NT / 32) ? smem[NT / 32 + l] : (V)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ra += __shfl_xor_sync(0xffffffffu, ra, o);
            rb += __shfl_xor_sync(0xffffffffu, rb, o);
        }
        if (l == 0) {
            smem[0] = ra;
            smem[1] = rb;
        }
    }
    __syncthreads();
    a = smem[0];
    b = smem[1];
    __syncthreads();
}
template <int NT>
__device__ inline void block_sum2_any(double a, double b, double* smem, float*, double* A, double* B) {
    block_sum2_t<NT, double>(a, b, smem);
    *A = a;
    *B = b;
}
template <int NT>
__device__ inline void block_sum2_any(float a, float b, double*, float* smemf, double* A, double* B) {
    block_sum2_t<NT, float>(a, b, smemf);
    *A = (double)a;
    *B = (double)b;
}

// Block sum in the accumulator's own type, returned as double.
template <int NT>
__device__ inline double block_sum_any(double v, double* smem, float*) { return block_sum<NT>(v, smem); }
template <int NT>
__device__ inline double block_sum_any(float v, double*, float* smemf) { return (double)block_sum_f<NT>(v, smemf); }

// Sum of npart partial sums, every thread of the block gets the same value
// (same order of additions in every block, so the result is bitwise identical).
template <int NT>
__device__ inline double sum_partials(const double* part, int npart, double* smem) {
    double v = 0.0;
    for (int i = threadIdx.x; i < npart; i += NT) v += part[i];
    return block_sum<NT>(v, smem);
}

// Last block of a grid to arrive (nblocks blocks counting on *cnt).  The
// block's partial sums are written by thread 0 before the call; thread 0
// counts in with one acquire-release atomic at GPU scope, which publishes its
// partials (release) and, in the last block, makes every other block's
// published partials visible (acquire) before the block barrier hands them to
// the block's other threads.  The last block resets *cnt.
__device__ __forceinline__ unsigned int atomic_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ bool arrive_last_n(unsigned int* cnt, unsigned int nblocks) {
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomic_add_acq_rel_gpu(cnt, 1u) == nblocks - 1u);
    __syncthreads();
    return am_last != 0;
}

constexpr int kThreads = 256;     // block size of the stencil / vector kernels
constexpr int kMaxPartials = 2048; // capacity of a partial-sum buffer

inline int blocks_for(long long n, int nt = kThreads) {
    long long b = (n + nt - 1) / nt;
    if (b < 1) b = 1;
    return (int)b;
}

// The projection kernel (one thread per interior cell): blocks of the cell
// map, linear (kThreads consecutive cells) or tiled (tile_x x kThreads/tile_x
// cells, x by rows of y and z), and the interior index of a thread (-1 when
// its tile position lies outside the grid).
inline int cell_blocks(const Geom& g) {
    if (g.tile_x <= 0) return blocks_for(g.ncell);
    const long long rows = (long long)g.n[1] * g.n[2];
    const int ty = kThreads / g.tile_x;
    return (int)(((g.n[0] + g.tile_x - 1) / g.tile_x) * ((rows + ty - 1) / ty));
}
__device__ __forceinline__ long long cell_of_block(const Geom& g, int bx) {
    if (g.tile_x <= 0) {
        const long long t = (long long)bx * kThreads + threadIdx.x;
        return t < g.ncell ? t : -1;
    }
    const int tx = g.tile_x, ty = kThreads / tx;
    const int ntx = (g.n[0] + tx - 1) / tx;
    const int i = (bx % ntx) * tx + (int)threadIdx.x % tx;
    const long long row = (long long)(bx / ntx) * ty + (int)threadIdx.x / tx;
    if (i >= g.n[0] || row >= (long long)g.n[1] * g.n[2]) return -1;
    return i + (long long)g.n[0] * row;
}

// Grid-stride launch bounded by the partial-sum capacity.
inline int reduce_blocks(long long n, int nt = kThreads) {
    long long b = (n + nt - 1) / nt;
    if (b > kMaxPartials) b = kMaxPartials;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace lm
