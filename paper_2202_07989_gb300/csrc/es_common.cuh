// Shared device definitions of the ES moving-mesh library (arXiv 2202.07989).
//
// Data layout in HBM: every field is structure of arrays, field-major,
// a[f][i3][i2][i1], interior nodes only (no ghost storage).  Ghost nodes are
// reached through index maps on load (periodic wrap, wall mirror, outflow copy,
// inflow state).  Metrics live in a padded buffer with 3 ghost layers per
// direction, M[(k*(d+1)+c)][i3+3][i2+3][i1+3].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace es {

constexpr int MAXC = 6;    // N + d + 1 <= 6
constexpr int HALO = 3;    // stencil half width of the flux (w = 3) and WENO-MR

enum { BC_PERIODIC = 0, BC_REFLECT = 1, BC_INFLOW = 2, BC_OUTFLOW = 3 };
enum { SIG_RHO = 0, SIG_RHO1 = 1, SIG_RHO2 = 2, SIG_P = 3, SIG_Y2 = 4, SIG_V1 = 5 };
enum { ST_NONPHYSICAL = 1, ST_TIMEOUT = 2 };
enum { MON_GRAD2 = 0, MON_GRAD = 1, MON_LAP = 2 };   // monitor term operators

// alpha_{3,m} of the sixth-order EC flux (Sec. 3.1) and the matching delta weights
// alpha_m of the 2w-order central difference and EC flux (Sec. 3.1: sum_m alpha_m = 1 and
// sum_m alpha_m m^(2s-1) = 0 for s = 2..w), w = 1, 2, 3; zero for m > w
__host__ __device__ constexpr double alpha_w(int w, int m)
{
    return w == 1 ? (m == 1 ? 1.0 : 0.0)
         : w == 2 ? (m == 1 ? 4.0 / 3.0 : (m == 2 ? -1.0 / 6.0 : 0.0))
                  : (m == 1 ? 1.5 : (m == 2 ? -0.3 : 1.0 / 30.0));
}

// one instance of the problem: grid, boundary, physics and scheme parameters
struct Inst {
    int d, N, nc;
    int n[3];                 // nodes per direction (n[2] = 1 in 2D)
    int P[3];                 // padded extents of the metric buffer
    long long ncell, npad;
    double dxi[3], inv_dxi[3], xi_lo[3], L[3];
    int bc[3][2];
    double inflow[3][2][8];
    double gamma[2], cv[2], pinf[2], Rs[2], cvG[2], pinf_tot;
    int es;
    double chi[3], weno_eps, cfl;
    int n_sigma, sigma[4], sigma_op[4];
    double alpha[4];
    int mu, nf;
    int weno;                 // ES_WENO_MR (0) or ES_WENO_JS (1)
    int fixed;                // 1: the mesh never moves
    int ntile_nodes;          // 1D node tiles for node-wise kernels
    int zc;                   // 3D: planes per chunk of the kernels that march along i3
    // binary32 copies of the physical and scheme constants for the FP32 arithmetic of the
    // mixed form (converting the binary64 ones in the kernels would use the FP64 pipe)
    float f_gamma[2], f_cv[2], f_Rs[2], f_cvG[2], f_pinf_tot, f_chi[3], f_eps;
    float f_h2[3];            // 1 / dxi_k^2 (Jacobi weights of the mixed form)
    float f_inv_dxi[3], f_alpha[4];
    float f_ichi3;            // 1 / chi_3 of WENO-MR
    double mc[3][3];          // (1/2) alpha_m / dxi_k: delta_k of a coordinate divided by dxi_k
    int w;                    // EC flux order 2w
    double ecw[3];            // alpha_m of order 2w (zero for m > w): the EC pair sum and delta_k
    double gcw[3];            // the GCL stencil: (1/2) sum_{m >= j+1} alpha_m for node pairs j = 0..2
    float f_ecw[3], f_gcw[3]; // binary32 copies
};

// Programmatic dependent launch: every kernel of a step waits until its predecessor has
// completed and its memory is visible before it touches any data.  A CTA lets the next
// kernel launch when it exits (no explicit trigger: CTAs of the next kernel would otherwise
// sit on the SMs beside the running ones).  A no-op for a kernel that was not launched with
// programmatic stream serialization.
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// the constants of an instance in the compute type R
template <typename R>
struct Cst;
template <>
struct Cst<double> {
    static __device__ __forceinline__ double gamma(const Inst& I, int l) { return I.gamma[l]; }
    static __device__ __forceinline__ double cv(const Inst& I, int l) { return I.cv[l]; }
    static __device__ __forceinline__ double Rs(const Inst& I, int l) { return I.Rs[l]; }
    static __device__ __forceinline__ double cvG(const Inst& I, int l) { return I.cvG[l]; }
    static __device__ __forceinline__ double pinf(const Inst& I) { return I.pinf_tot; }
    static __device__ __forceinline__ double chi(const Inst& I, int q) { return I.chi[q]; }
    static __device__ __forceinline__ double eps(const Inst& I) { return I.weno_eps; }
    static __device__ __forceinline__ double ecw(const Inst& I, int m) { return I.ecw[m]; }
    static __device__ __forceinline__ double gcw(const Inst& I, int j) { return I.gcw[j]; }
};
template <>
struct Cst<float> {
    static __device__ __forceinline__ float gamma(const Inst& I, int l) { return I.f_gamma[l]; }
    static __device__ __forceinline__ float cv(const Inst& I, int l) { return I.f_cv[l]; }
    static __device__ __forceinline__ float Rs(const Inst& I, int l) { return I.f_Rs[l]; }
    static __device__ __forceinline__ float cvG(const Inst& I, int l) { return I.f_cvG[l]; }
    static __device__ __forceinline__ float pinf(const Inst& I) { return I.f_pinf_tot; }
    static __device__ __forceinline__ float chi(const Inst& I, int q) { return I.f_chi[q]; }
    static __device__ __forceinline__ float eps(const Inst& I) { return I.f_eps; }
    static __device__ __forceinline__ float ecw(const Inst& I, int m) { return I.f_ecw[m]; }
    static __device__ __forceinline__ float gcw(const Inst& I, int j) { return I.f_gcw[j]; }
};

// per-call device pointers of one instance: the stage input, the metric target,
// the residual accumulators, the RK base and output, and the step scalars.
// Single-instance calls pass it by value; batched calls use a device table.
struct StagePtrs {
    const double* JU;         // stage input (JU, J, x) and the mesh velocity
    const double* J;
    const double* x;
    const double* xdot;
    double* M;                // padded metrics target
    double* Md;               // 2D: padded metrics of the mesh velocity (stage k: M + s_k dt Md)
    double* accU;             // residual accumulators: n_c fields and J
    double* accJ;
    const double* JU0;        // RK base state q^n
    const double* J0;
    const double* x0;
    double* JUo;              // RK stage output
    double* Jo;
    double* xo;
    const double* dt;         // device scalar: the time step
    double* xdot_out;         // mesh_redistribute outputs
    double* out;              // {Delta t, Delta_tau}, or {P, S} of the entropy diagnostics
    double dt_fixed;          // > 0: use this time step instead of Eq. (cfl)
};

// context-owned scratch of one instance (fixed for the context's lifetime)
struct Scratch {
    double* M;                // padded metrics
    double* Md;               // 2D: padded metrics of the mesh velocity
    double* D3;               // 3D: products delta_b[x_p] x_q on the grid with 6 ghost layers
    double* XE;               // 3D: x on the grid with 9 ghost layers (boundary maps applied once)
    double* M3;               // 3D moving mesh: padded metrics of the third RK stage's mesh
    double* Xm;               // 3D: the positions the spatial rows of M were formed from (NaN before)
    double* accU;
    double* accJ;
    double* red;              // reductions: [0] CFL max, [1..4] monitor maxima, [5] Delta_tau
    double* g;                // monitor gradients, n_sigma fields
    void* th0;                // monitor function ping-pong (compute type)
    void* th1;
    double* xa;               // Jacobi ping-pong (mixed form: binary32 displacements x - x^n)
    double* xb;
    float* dl;                // mixed form: mesh spacings x^n_{i+-e_k} - x^n_i, [k][+-][j][node]
    double* zeros;            // d zero fields (absent mesh velocity)
};

// the per-instance reduction slots at the start of a mesh step (CFL max, monitor maxima,
// Delta_tau = 1, schlieren max), done by block 0 of the first kernel of the step
__device__ __forceinline__ void reset_reductions(const Scratch* scr, int ninst)
{
    if (!scr || blockIdx.x != 0) return;
    for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
        double* r = scr[i].red;
        for (int q = 0; q < 5; ++q) r[q] = 0.0;
        r[5] = 1.0;
        r[6] = 0.0;
        r[7] = 0.0;
    }
}

#define ES_PTRS(P) const StagePtrs P = (table ? table[it.x] : single)

// node-wise kernels run over tiles of NT_X x NT_Y nodes of one (i1, i0) plane
constexpr int NT_X = 32, NT_Y = 8;

// number of node tiles of a grid extended by `pad` ghost layers in every direction of the instance
__host__ __device__ inline int node_tiles(const Inst& I, int pad)
{
    int e0 = I.n[0] + 2 * pad, e1 = I.n[1] + 2 * pad, e2 = I.d == 3 ? I.n[2] + 2 * pad : 1;
    return ((e0 + NT_X - 1) / NT_X) * ((e1 + NT_Y - 1) / NT_Y) * e2;
}

// 3D kernels that march along i3: an item is a 32 x 8 column of the (i1, i2) plane and a
// chunk of zc planes of it
struct Col3 {
    int b0, b1, z0, z1;
};
__host__ __device__ inline int col3_items(const Inst& I)
{
    return ((I.n[0] + NT_X - 1) / NT_X) * ((I.n[1] + NT_Y - 1) / NT_Y) * ((I.n[2] + I.zc - 1) / I.zc);
}
__device__ inline Col3 col3(const Inst& I, int item)
{
    const int ntx = (I.n[0] + NT_X - 1) / NT_X, nc = ntx * ((I.n[1] + NT_Y - 1) / NT_Y);
    const int t = item % nc, ch = item / nc;
    Col3 c;
    c.b0 = (t % ntx) * NT_X;
    c.b1 = (t / ntx) * NT_Y;
    c.z0 = ch * I.zc;
    c.z1 = min(I.n[2], c.z0 + I.zc);
    return c;
}

// the node of this thread in node tile `tile` (ghost layers included); false outside the grid
__device__ inline bool tile_node(const Inst& I, int tile, int pad, int& i0, int& i1, int& i2)
{
    int e0 = I.n[0] + 2 * pad, e1 = I.n[1] + 2 * pad;
    int ntx = (e0 + NT_X - 1) / NT_X, nty = (e1 + NT_Y - 1) / NT_Y;
    int tx = tile % ntx, r = tile / ntx;
    int ty = r % nty, tz = r / nty;
    int lx = (int)threadIdx.x % NT_X, ly = (int)threadIdx.x / NT_X;
    int a = tx * NT_X + lx, b = ty * NT_Y + ly;
    i0 = a - pad;
    i1 = b - pad;
    i2 = I.d == 3 ? tz - pad : 0;
    return a < e0 && b < e1;
}

__host__ __device__ inline long long lin(const Inst& I, int i0, int i1, int i2)
{
    return ((long long)i2 * I.n[1] + i1) * I.n[0] + i0;
}

__host__ __device__ inline long long plin(const Inst& I, int i0, int i1, int i2)
{
    return ((long long)(I.d == 3 ? i2 + 3 : 0) * I.P[1] + (i1 + 3)) * I.P[0] + (i0 + 3);
}

__device__ inline int floordiv_(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// mesh position at any node index: periodic sides wrap and shift x_k by the box
// length, all other sides mirror about the wall (velocity: mirror negates x_k)
template <bool VEL>
__device__ inline void x_at(const Inst& I, const double* __restrict__ x, int i0, int i1, int i2, double* out)
{
    int i[3] = { i0, i1, i2 };
    double shift[3] = { 0, 0, 0 }, wall[3] = { 0, 0, 0 };
    bool flip[3] = { false, false, false };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= I.d) break;
        int n = I.n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        int side = i[k] < 0 ? 0 : 1;
        if (I.bc[k][side] == BC_PERIODIC) {
            int s = floordiv_(i[k], n);
            i[k] -= s * n;
            shift[k] = s * I.L[k];
        } else {
            i[k] = side == 0 ? -1 - i[k] : 2 * n - 1 - i[k];
            flip[k] = true;
            wall[k] = side == 0 ? I.xi_lo[k] : I.xi_lo[k] + I.L[k];
        }
    }
    long long id = lin(I, i[0], i[1], I.d == 3 ? i[2] : 0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= I.d) break;
        double v = x[j * I.ncell + id];
        if (VEL) {
            if (flip[j]) v = -v;
        } else {
            if (flip[j]) v = 2.0 * wall[j] - v;
            v += shift[j];
        }
        out[j] = v;
    }
}

// node index along direction k (g may be a ghost) -> interior index and the
// boundary treatment: 0 none, 1 negate the k-momentum (reflect), 2 inflow state
__device__ inline int map_line(const Inst& I, int k, int g, int& gi, int& side)
{
    int n = I.n[k];
    side = g < 0 ? 0 : 1;
    if (g >= 0 && g < n) { gi = g; return 0; }
    switch (I.bc[k][side]) {
    case BC_PERIODIC: gi = g - floordiv_(g, n) * n; return 0;
    case BC_REFLECT: gi = side == 0 ? -1 - g : 2 * n - 1 - g; if (gi < 0) gi = 0; if (gi >= n) gi = n - 1; return 1;
    case BC_OUTFLOW: gi = side == 0 ? 0 : n - 1; return 0;
    default: gi = side == 0 ? 0 : n - 1; return 2;
    }
}

// VCL metric J xi_k/t = -sum_j xdot_j J xi_k/x_j (Eq. (VCLCoeff)) from one row of the spatial
// metrics, in one fixed evaluation order for every kernel that forms it
template <int D>
__device__ __forceinline__ double vcl_metric(const double* xd, const double* m)
{
    double s = xd[0] * m[0];
#pragma unroll
    for (int j = 1; j < D; ++j) s = fma(xd[j], m[j], s);
    return -s;
}

// 2D metrics of a staged two-component field v at tile position (cy, cx) (3-node halo):
// m[0] = delta_2[v_2] / dxi_2, m[1] = -delta_2[v_1] / dxi_2, m[2] = -delta_1[v_2] / dxi_1,
// m[3] = delta_1[v_1] / dxi_1, with mc = alpha_m / (2 dxi_k).  The operator is linear in v, so
// the metrics of the mesh x + s xdot are M(x) + s M(xdot).
template <int HY, int HX>
__device__ __forceinline__ void metrics2d_at(const Inst& I, const double (*v)[HY][HX], int cy, int cx, double m[4])
{
    double m11 = 0.0, m12 = 0.0, m21 = 0.0, m22 = 0.0;
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
        const double c1 = I.mc[0][a - 1], c2 = I.mc[1][a - 1];
        m11 = fma(c2, v[1][cy + a][cx] - v[1][cy - a][cx], m11);
        m12 = fma(c2, v[0][cy - a][cx] - v[0][cy + a][cx], m12);
        m21 = fma(c1, v[1][cy][cx - a] - v[1][cy][cx + a], m21);
        m22 = fma(c1, v[0][cy][cx + a] - v[0][cy][cx - a], m22);
    }
    m[0] = m11;
    m[1] = m12;
    m[2] = m21;
    m[3] = m22;
}

// the six padded 2D metric rows at p: VCL row, then the spatial rows, for k = 1, 2
__device__ __forceinline__ void store_metrics2d(double* M, long long np, long long p, const double xd[2], const double m[4])
{
    const double r1[2] = { m[0], m[1] }, r2[2] = { m[2], m[3] };
    M[0 * np + p] = vcl_metric<2>(xd, r1);
    M[1 * np + p] = m[0];
    M[2 * np + p] = m[1];
    M[3 * np + p] = vcl_metric<2>(xd, r2);
    M[4 * np + p] = m[2];
    M[5 * np + p] = m[3];
}

// scalar node field with periodic wrap, else copy of the boundary node
__device__ inline long long s_map(const Inst& I, int i0, int i1, int i2)
{
    int i[3] = { i0, i1, i2 };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= I.d) break;
        int n = I.n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        int side = i[k] < 0 ? 0 : 1;
        if (I.bc[k][side] == BC_PERIODIC) i[k] -= floordiv_(i[k], n) * n;
        else i[k] = side == 0 ? 0 : n - 1;
    }
    return lin(I, i[0], i[1], I.d == 3 ? i[2] : 0);
}

// conserved point state at a node reached along one grid line (ghost maps of the
// boundary conditions); returns false for a non-physical state
__device__ inline void load_U(const Inst& I, const double* __restrict__ JU, const double* __restrict__ J,
                              int i0, int i1, int i2, double* U)
{
    int i[3] = { i0, i1, i2 };
    int neg = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= I.d) break;
        if (i[k] >= 0 && i[k] < I.n[k]) continue;
        int gi, side;
        int t = map_line(I, k, i[k], gi, side);
        if (t == 2) {
            for (int q = 0; q < I.nc; ++q) U[q] = I.inflow[k][side][q];
            return;
        }
        if (t == 1) neg = k;
        i[k] = gi;
    }
    long long id = lin(I, i[0], i[1], I.d == 3 ? i[2] : 0);
    double inv = 1.0 / J[id];
    for (int q = 0; q < I.nc; ++q) U[q] = JU[q * I.ncell + id] * inv;
    if (neg >= 0) U[I.N + neg] = -U[I.N + neg];
}

// IEEE 754 binary64 -> binary32 with round-to-nearest-even, done with integer
// instructions only (the hardware conversion issues on the FP64 pipe, which GB300 runs
// at 1/64 of the FP32 rate).  Values below 2^-126 in magnitude become a signed zero;
// |x| >= 2^128 (after rounding) and infinities become infinities; NaN becomes the
// canonical binary32 NaN.
__device__ __forceinline__ float f64_to_f32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hi = (unsigned int)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned int sign = hi & 0x80000000u;
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    if (e < 1023 - 126) return __int_as_float((int)sign);
    if (e > 1023 + 127) return __int_as_float((int)(e == 0x7ff && mant != 0ull ? 0x7fffffffu : (sign | 0x7f800000u)));
    const unsigned int m = (unsigned int)(mant >> 29);
    const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull);
    unsigned int f = sign | ((unsigned int)(e - 1023 + 127) << 23) | m;
    // a carry out of the significand steps the exponent (up to infinity), as rounding must
    f += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __int_as_float((int)f);
}

// IEEE 754 binary32 -> binary64 (exact), with integer instructions only; subnormals are
// normalised, infinities kept, NaN keeps its payload with the quiet bit set
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned int b = (unsigned int)__float_as_int(f);
    const unsigned int e = (b >> 23) & 0xffu;
    const unsigned int mant = b & 0x7fffffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned long long d;
    if (e == 0xffu) {
        d = sign | 0x7ff0000000000000ull | ((unsigned long long)mant << 29) | (mant ? 0x0008000000000000ull : 0ull);
    } else if (e == 0u) {
        if (mant == 0u) {
            d = sign;
        } else {
            // mant * 2^-149 with its leading one at bit 23 - sh
            const int sh = __clz((int)mant) - 8;
            d = sign | ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)((mant << sh) & 0x7fffffu) << 29);
        }
    } else {
        d = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)mant << 29);
    }
    return __longlong_as_double((long long)d);
}

template <typename R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return f64_to_f32(x); }

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return f32_to_f64(x); }

// {a} = a/2 + b/2 of two positive binary32 values as the exact binary64 value, built with
// integer instructions.  For normal a, b (biased exponents >= 2) whose exponents differ by
// at most 7, the sum of the significands aligned to the smaller exponent has at most 32
// bits, so a/2 + b/2 = M 2^(e - 151) exactly; M is placed in the binary64 fields directly.
// Otherwise the value is the binary64 sum of the halves, as the FP64 pipe forms it.
__device__ __forceinline__ double half_sum_exact(float a, float b)
{
    const unsigned int ua = __float_as_uint(a), ub = __float_as_uint(b);
    const int ea = (int)(ua >> 23), eb = (int)(ub >> 23);
    const int e = min(ea, eb), dl = max(ea, eb) - e;
    if (e < 2 || dl > 7 || max(ea, eb) > 254) return f32_to_f64(0.5f * a) + f32_to_f64(0.5f * b);
    const unsigned int ma = (ua & 0x7fffffu) | 0x800000u, mb = (ub & 0x7fffffu) | 0x800000u;
    const unsigned int M = (ma << (ea - e)) + (mb << (eb - e));
    const int k = 31 - __clz((int)M);     // the leading one of M; its bit carries into the exponent
    const unsigned long long bits =
        ((unsigned long long)(k + e + 871) << 52) + ((unsigned long long)M << (52 - k));
    return __longlong_as_double((long long)bits);
}

// binary32 -> binary64 (exact) of a positive normal value: the significand shifted into place
// and the exponent rebiased from 127 to 1023 by one 64-bit add
__device__ __forceinline__ double f32_to_f64_posnormal(float f)
{
    return __longlong_as_double((long long)(((unsigned long long)__float_as_uint(f) << 29) + (896ull << 52)));
}

// binary64 -> binary32, round to nearest even, of a positive value whose binary32 result is a
// normal number or infinity: the exponent rebiased from 1023 to 127 in the shifted bit pattern
__device__ __forceinline__ float f64_to_f32_posnormal(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned int f = (unsigned int)((b >> 29) - (896ull << 23));
    const unsigned int rem = (unsigned int)b & 0x1fffffffu;
    f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

// {a}(1 - del) rounded to binary32, the value of the log-mean small-jump branch (the
// Ismail-Roe series, Sec. 3.3): {a} = a/2 + b/2 exact in binary64, times (1 - del) by one FP64
// fused multiply-add, then rounded.  a, b > 0 and 0 <= del <= 1/2.  When a and b are normal
// (biased exponents >= 2) and at most 7 binades apart and del is zero or normal, {a} is built
// with integer instructions (as in half_sum_exact) and the conversions skip their special
// cases; otherwise the general conversions run.  Both give the same value.
__device__ __forceinline__ float logmean_small(float a, float b, float del)
{
    const unsigned int ua = __float_as_uint(a), ub = __float_as_uint(b);
    const int ea = (int)(ua >> 23), eb = (int)(ub >> 23);
    const int e = min(ea, eb), dl = max(ea, eb) - e;
    const bool del_ok = del == 0.0f || (__float_as_uint(del) >> 23) != 0u;
    if (e >= 2 && dl <= 7 && max(ea, eb) <= 254 && del_ok) {
        const unsigned int ma = (ua & 0x7fffffu) | 0x800000u, mb = (ub & 0x7fffffu) | 0x800000u;
        const unsigned int M = (ma << (ea - e)) + (mb << (eb - e));
        const int k = 31 - __clz((int)M);
        const double hs = __longlong_as_double(
            (long long)(((unsigned long long)(k + e + 871) << 52) + ((unsigned long long)M << (52 - k))));
        const double d = del == 0.0f ? 0.0 : f32_to_f64_posnormal(del);
        return f64_to_f32_posnormal(fma(-hs, d, hs));
    }
    const double hs = f32_to_f64(0.5f * a) + f32_to_f64(0.5f * b);
    return f64_to_f32(fma(-hs, f32_to_f64(del), hs));
}

// bounded reductions of non-negative doubles: the IEEE order of non-negative
// doubles is the order of their bit patterns
__device__ inline void atomic_max_pos(double* a, double v)
{
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

__device__ inline void atomic_min_pos(double* a, double v)
{
    atomicMin(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

}  // namespace es
