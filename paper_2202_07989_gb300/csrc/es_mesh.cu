// Per-step kernels: CFL time step (Eq. (cfl)), monitor function (Eq. (monitor)),
// low-pass filter (remark in Sec. 4), Jacobi sweeps of the discrete mesh
// equation, the movement limiter Delta_tau and the mesh velocity (Sec. 4), and
// the entropy diagnostics.  FP64 positions and reductions; the monitor and the
// filter run in the compute type of the context (FP32 in the mixed form).
#include "es_mesh.cuh"

#include <type_traits>

namespace es {

// reduction slots per instance
//   red[0] max_i sum_k rho_{i,k}/dxi_k,  red[1..4] max |grad sigma_s|,  red[5] Delta_tau

__device__ inline void node_coords(const Inst& I, long long p, int& i0, int& i1, int& i2)
{
    i0 = (int)(p % I.n[0]);
    i1 = (int)((p / I.n[0]) % I.n[1]);
    i2 = (int)(p / ((long long)I.n[0] * I.n[1]));
}

__device__ inline void prim(const Inst& I, const double* U, double* rl, double* v, double& T, double& p, double& rho)
{
    rho = 0.0;
    double cvr = 0.0, rr = 0.0;
    for (int l = 0; l < I.N; ++l) { rl[l] = U[l]; rho += U[l]; cvr += I.cv[l] * U[l]; rr += I.Rs[l] * U[l]; }
    double v2 = 0.0;
    for (int m = 0; m < I.d; ++m) { v[m] = U[I.N + m] / rho; v2 += v[m] * v[m]; }
    T = (U[I.N + I.d] - 0.5 * rho * v2 - I.pinf_tot) / cvr;
    p = rr * T - I.pinf_tot;
}

__device__ inline double sigma_of(const Inst& I, int kind, const double* U)
{
    const double rho = I.N == 2 ? U[0] + U[1] : U[0];
    switch (kind) {
    case SIG_RHO1: return U[0];
    case SIG_RHO2: return I.N == 2 ? U[1] : 0.0;
    case SIG_Y2: return I.N == 2 ? U[1] / rho : 0.0;
    case SIG_V1: return U[I.N] / rho;
    case SIG_P: {
        double rl[2], v[3], T, p, r;
        prim(I, U, rl, v, T, p, r);
        return p;
    }
    default: return rho;
    }
}

// conserved point state at a node in the compute type (ghost maps of load_U)
template <typename R>
__device__ __forceinline__ void load_U_t(const Inst& I, const double* __restrict__ JU, const double* __restrict__ J,
                                         int i0, int i1, int i2, R* U)
{
    if constexpr (std::is_same<R, double>::value) {
        load_U(I, JU, J, i0, i1, i2, U);
    } else {
        int i[3] = { i0, i1, i2 };
        int neg = -1;
        for (int k = 0; k < I.d; ++k) {
            if (i[k] >= 0 && i[k] < I.n[k]) continue;
            int gi, side;
            int t = map_line(I, k, i[k], gi, side);
            if (t == 2) {
                for (int q = 0; q < I.nc; ++q) U[q] = to_r<R>(I.inflow[k][side][q]);
                return;
            }
            if (t == 1) neg = k;
            i[k] = gi;
        }
        long long id = lin(I, i[0], i[1], I.d == 3 ? i[2] : 0);
        R inv = R(1) / to_r<R>(J[id]);
        for (int q = 0; q < I.nc; ++q) U[q] = to_r<R>(JU[q * I.ncell + id]) * inv;
        if (neg >= 0) U[I.N + neg] = -U[I.N + neg];
    }
}

template <typename R>
__device__ __forceinline__ R sigma_t(const Inst& I, int kind, const R* U)
{
    const R rho = I.N == 2 ? U[0] + U[1] : U[0];
    switch (kind) {
    case SIG_RHO1: return U[0];
    case SIG_RHO2: return I.N == 2 ? U[1] : R(0);
    case SIG_Y2: return I.N == 2 ? U[1] / rho : R(0);
    case SIG_V1: return U[I.N] / rho;
    case SIG_P: {
        R cvr = R(0), rr = R(0), v2 = R(0);
        for (int l = 0; l < I.N; ++l) { cvr += to_r<R>(I.cv[l]) * U[l]; rr += to_r<R>(I.Rs[l]) * U[l]; }
        for (int m = 0; m < I.d; ++m) { R v = U[I.N + m] / rho; v2 += v * v; }
        R T = (U[I.N + I.d] - R(0.5) * rho * v2 - to_r<R>(I.pinf_tot)) / cvr;
        return rr * T - to_r<R>(I.pinf_tot);
    }
    default: return rho;
    }
}

// the reciprocal of dxi_k, the weight alpha_q and the monitor gradient storage in the compute
// type (the mixed form keeps binary32 copies, so its node kernels run no FP64 arithmetic)
template <typename R>
__device__ __forceinline__ R inv_dxi_r(const Inst& I, int k)
{
    if constexpr (std::is_same<R, float>::value) return I.f_inv_dxi[k];
    else return I.inv_dxi[k];
}
template <typename R>
__device__ __forceinline__ R alpha_r(const Inst& I, int q)
{
    if constexpr (std::is_same<R, float>::value) return I.f_alpha[q];
    else return I.alpha[q];
}
template <typename R>
__device__ __forceinline__ R* grad_r(const Scratch& S) { return reinterpret_cast<R*>(S.g); }

// one pass over the nodes: the CFL spectral-radius sum of Eq. (cfl) at x^n and the monitor
// terms |grad_xi sigma_s| or |Laplacian_xi sigma_s| (second-order central differences);
// per-instance maxima by atomics on the non-negative bit patterns; the metrics are read from
// M.  Each block evaluates sigma once per node of its 32 x 8 tile and of a 1-node halo in the
// (i1, i2) plane into shared memory; the third direction reads globally.  It serves the FP64
// form of 3D instances (R = double); 2D instances run cfl_grad2d_kernel, and the mixed form of
// 3D instances cfl_sigma3d_kernel and grad3d_kernel, with the same terms.
template <typename R>
__global__ void __launch_bounds__(NODE_TPB) cfl_grad_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                             const StagePtrs* __restrict__ table,
                                                             const int2* __restrict__ work, int nwork,
                                                             const Scratch* __restrict__ scr)
{
    pdl_entry();
    constexpr int TX = NT_X + 2, TY = NT_Y + 2;
    __shared__ R ssig[4][TY][TX];
    __shared__ double sh[32];
    const int lx = (int)threadIdx.x % NT_X, ly = (int)threadIdx.x / NT_X;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const int n0 = I.n[0], n1 = I.n[1], ns = I.n_sigma;
        const int ntx = (n0 + NT_X - 1) / NT_X, nty = (n1 + NT_Y - 1) / NT_Y;
        const int tr = it.y / ntx;
        const int b0 = (it.y % ntx) * NT_X - 1, b1 = (tr % nty) * NT_Y - 1, i2 = I.d == 3 ? tr / nty : 0;
        __syncthreads();    // the previous tile's readers are done
        for (int q = threadIdx.x; q < TX * TY; q += NODE_TPB) {
            const int a = q % TX, b = q / TX;
            const int g0 = b0 + a, g1 = b1 + b;
            const bool corner = (a == 0 || a == TX - 1) && (b == 0 || b == TY - 1);
            if (corner || g0 > n0 || g1 > n1 || ns == 0) continue;
            R Ug[MAXC];
            load_U_t<R>(I, P.JU, P.J, g0, g1, i2, Ug);
            for (int s = 0; s < ns; ++s) ssig[s][b][a] = sigma_t<R>(I, I.sigma[s], Ug);
        }
        __syncthreads();
        const int i[3] = { b0 + 1 + lx, b1 + 1 + ly, i2 };
        const bool valid = i[0] < n0 && i[1] < n1;
        double s = 0.0, g[4] = { 0, 0, 0, 0 };
        if (valid) {
            const long long p = lin(I, i[0], i[1], i[2]);
            R U[MAXC];
            load_U_t<R>(I, P.JU, P.J, i[0], i[1], i[2], U);
            const R rho = U[0] + (I.N == 2 ? U[1] : R(0));
            R v[3], v2 = R(0), cvr = R(0), a = R(0), gm = R(0);
            for (int m = 0; m < I.d; ++m) { v[m] = U[I.N + m] / rho; v2 += v[m] * v[m]; }
            for (int l = 0; l < I.N; ++l) {
                a += Cst<R>::Rs(I, l) * U[l];          // (Gamma_l - 1) c_v,l rho_l
                gm += Cst<R>::cvG(I, l) * U[l];        // Gamma_l c_v,l rho_l
                cvr += Cst<R>::cv(I, l) * U[l];
            }
            const R T = (U[I.N + I.d] - R(0.5) * rho * v2 - Cst<R>::pinf(I)) / cvr;
            const R c = sqrt((a / rho) * (gm / cvr) * T);
            // spatial metrics of x^n, formed by the metrics pass that opens the mesh step
            const long long pid = plin(I, i[0], i[1], i[2]);
            const R Jp = to_r<R>(P.J[p]);
            R sr = R(0);
            for (int k = 0; k < I.d; ++k) {
                R L2 = R(0), vn = R(0);
                for (int j = 0; j < I.d; ++j) {
                    const R mk = to_r<R>(scr[it.x].M[(long long)(k * (I.d + 1) + 1 + j) * I.npad + pid]);
                    L2 += mk * mk;
                    vn += mk * v[j];
                }
                sr += (fabs(vn) + c * sqrt(L2)) / Jp * inv_dxi_r<R>(I, k);
            }
            s = to_d(sr);
            if (!(s >= 0.0)) s = 0.0;
            // per term |grad_xi sigma| (squared sums) or the Laplacian (second differences)
            R gr[4] = { R(0), R(0), R(0), R(0) }, lp[4] = { R(0), R(0), R(0), R(0) };
            for (int k = 0; k < I.d; ++k) {
                R Up[MAXC], Um[MAXC];
                if (k == 2) {
                    load_U_t<R>(I, P.JU, P.J, i[0], i[1], i[2] + 1, Up);
                    load_U_t<R>(I, P.JU, P.J, i[0], i[1], i[2] - 1, Um);
                }
                const R hk = R(0.5) * inv_dxi_r<R>(I, k);
                const R h2 = inv_dxi_r<R>(I, k) * inv_dxi_r<R>(I, k);
                for (int q = 0; q < ns; ++q) {
                    R sp, sm;
                    if (k == 0) { sp = ssig[q][ly + 1][lx + 2]; sm = ssig[q][ly + 1][lx]; }
                    else if (k == 1) { sp = ssig[q][ly + 2][lx + 1]; sm = ssig[q][ly][lx + 1]; }
                    else { sp = sigma_t<R>(I, I.sigma[q], Up); sm = sigma_t<R>(I, I.sigma[q], Um); }
                    const R gk = (sp - sm) * hk;
                    gr[q] += gk * gk;
                    lp[q] += (sp - R(2) * ssig[q][ly + 1][lx + 1] + sm) * h2;
                }
            }
            for (int q = 0; q < ns; ++q) {
                const R gq = I.sigma_op[q] == MON_LAP ? R(fabs(lp[q])) : R(sqrt(gr[q]));
                grad_r<R>(scr[it.x])[(long long)q * I.ncell + p] = gq;
                g[q] = to_d(gq);
                if (!(g[q] >= 0.0)) g[q] = 0.0;
            }
        }
        double mx = block_max<double>(s, sh);
        if (threadIdx.x == 0) atomic_max_pos(&scr[it.x].red[0], mx);
        for (int q = 0; q < 4; ++q) {
            if (q >= ns) break;
            double mq = block_max<double>(g[q], sh);
            if (threadIdx.x == 0) atomic_max_pos(&scr[it.x].red[1 + q], mq);
        }
    }
}

// ordered integer key of a non-negative value (the IEEE order of non-negative floats and
// doubles is the order of their bit patterns), for exact max reductions on the integer ALU
__device__ __forceinline__ unsigned int max_key(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long max_key(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned int shfl_max(unsigned int k, int o) { return max(k, __shfl_xor_sync(0xffffffffu, k, o)); }
__device__ __forceinline__ unsigned long long shfl_max(unsigned long long k, int o)
{
    return max(k, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)k, o));
}
__device__ __forceinline__ double key_value(unsigned int k) { return to_d(__uint_as_float(k)); }
__device__ __forceinline__ double key_value(unsigned long long k) { return __longlong_as_double((long long)k); }

// sigma_t of a D-dimensional instance with NS species (the same arithmetic, with the field
// indices known)
template <typename R, int NS, int D = 2>
__device__ __forceinline__ R sigma2d(const Inst& I, int kind, const R* U)
{
    const R rho = NS == 2 ? U[0] + U[1] : U[0];
    switch (kind) {
    case SIG_RHO1: return U[0];
    case SIG_RHO2: return NS == 2 ? U[1] : R(0);
    case SIG_Y2: return NS == 2 ? U[1] / rho : R(0);
    case SIG_V1: return U[NS] / rho;
    case SIG_P: {
        R cvr = R(0), rr = R(0), v2 = R(0);
#pragma unroll
        for (int l = 0; l < NS; ++l) { cvr += to_r<R>(I.cv[l]) * U[l]; rr += to_r<R>(I.Rs[l]) * U[l]; }
#pragma unroll
        for (int m = 0; m < D; ++m) { R v = U[NS + m] / rho; v2 += v * v; }
        R T = (U[NS + D] - R(0.5) * rho * v2 - to_r<R>(I.pinf_tot)) / cvr;
        return rr * T - to_r<R>(I.pinf_tot);
    }
    default: return rho;
    }
}

// cfl_grad_kernel for 2D instances with NS species: the same terms in the same arithmetic.
// The halo pass loads each node's state once: it stores sigma_s and, at the tile's own
// nodes, forms the CFL spectral-radius sum there.  The gradient pass then reads only shared
// memory, and one block reduction (integer keys of the non-negative maxima) ends the tile.
template <typename R, int NS>
__global__ void __launch_bounds__(NODE_TPB) cfl_grad2d_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                               const StagePtrs* __restrict__ table,
                                                               const int2* __restrict__ work, int nwork,
                                                               const Scratch* __restrict__ scr)
{
    pdl_entry();
    using K = decltype(max_key(R(0)));
    constexpr int NC = NS + 3, TX = NT_X + 2, TY = NT_Y + 2, NW = NODE_TPB / 32;
    __shared__ R ssig[4][TY][TX];
    __shared__ K sred[5][NW];
    const int lane = (int)threadIdx.x & 31, wid = (int)threadIdx.x >> 5;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const Scratch& Sc = scr[it.x];
        const int n0 = I.n[0], n1 = I.n[1], ns = I.n_sigma;
        const int ntx = (n0 + NT_X - 1) / NT_X;
        const int b0 = (it.y % ntx) * NT_X - 1, b1 = (it.y / ntx) * NT_Y - 1;
        K kmax[5] = { 0, 0, 0, 0, 0 };    // CFL sum, then the monitor terms
        __syncthreads();    // the previous tile's readers are done
        // at most two halo slots per thread, in one unrolled body so that the loads of both
        // are issued together
        static_assert(TX * TY <= 2 * NODE_TPB, "two halo slots per thread");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = (int)threadIdx.x + h * NODE_TPB;
            if (q >= TX * TY) continue;
            const int a = q % TX, b = q / TX;
            const int g0 = b0 + a, g1 = b1 + b;
            // a node outside the domain in both directions (a tile corner, or on a ragged tile
            // an edge node beyond the last row or column) is no neighbour of any tile node
            const bool out0 = g0 < 0 || g0 >= n0, out1 = g1 < 0 || g1 >= n1;
            if ((out0 && out1) || g0 > n0 || g1 > n1) continue;
            const bool own = a >= 1 && a <= NT_X && b >= 1 && b <= NT_Y && !out0 && !out1;
            if (ns == 0 && !own) continue;
            // the spatial metrics of x^n at a tile node, loaded ahead of the state arithmetic
            const long long p = lin(I, g0, g1, 0), pid = plin(I, g0, g1, 0);
            double mraw[4] = { 0.0, 0.0, 0.0, 0.0 };
            if (own) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int j = 0; j < 2; ++j) mraw[2 * k + j] = Sc.M[(long long)(k * 3 + 1 + j) * I.npad + pid];
            }
            // the point state with the ghost map of the one direction the node lies outside:
            // the arithmetic of load_U_t, with the field count known
            R U[MAXC];
            {
                int gi0 = g0, gi1 = g1, kk = 0, side = 0, tmap = 0;
                if (out0) tmap = map_line(I, 0, g0, gi0, side);
                else if (out1) { kk = 1; tmap = map_line(I, 1, g1, gi1, side); }
                if (tmap == 2) {
#pragma unroll
                    for (int f = 0; f < NC; ++f) U[f] = to_r<R>(I.inflow[kk][side][f]);
                } else {
                    const long long id = lin(I, gi0, gi1, 0);
                    const R inv = R(1) / to_r<R>(P.J[id]);
#pragma unroll
                    for (int f = 0; f < NC; ++f) U[f] = to_r<R>(P.JU[f * I.ncell + id]) * inv;
                    if (tmap == 1) U[NS + kk] = -U[NS + kk];
                }
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s < ns) ssig[s][b][a] = sigma2d<R, NS>(I, I.sigma[s], U);
            if (!own) continue;
            // Eq. (cfl) at node (g0, g1) with the metrics of x^n
            const R rho = U[0] + (NS == 2 ? U[1] : R(0));
            R v[2], v2 = R(0), cvr = R(0), ar = R(0), gm = R(0);
#pragma unroll
            for (int m = 0; m < 2; ++m) { v[m] = U[NS + m] / rho; v2 += v[m] * v[m]; }
#pragma unroll
            for (int l = 0; l < NS; ++l) {
                ar += Cst<R>::Rs(I, l) * U[l];          // (Gamma_l - 1) c_v,l rho_l
                gm += Cst<R>::cvG(I, l) * U[l];         // Gamma_l c_v,l rho_l
                cvr += Cst<R>::cv(I, l) * U[l];
            }
            const R T = (U[NC - 1] - R(0.5) * rho * v2 - Cst<R>::pinf(I)) / cvr;
            const R c = sqrt((ar / rho) * (gm / cvr) * T);
            const R Jp = to_r<R>(P.J[p]);
            R sr = R(0);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                R L2 = R(0), vn = R(0);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const R mk = to_r<R>(mraw[2 * k + j]);
                    L2 += mk * mk;
                    vn += mk * v[j];
                }
                sr += (fabs(vn) + c * sqrt(L2)) / Jp * inv_dxi_r<R>(I, k);
            }
            if (!(sr >= R(0))) sr = R(0);
            kmax[0] = max(kmax[0], max_key(sr));
        }
        __syncthreads();
        // per term |grad_xi sigma| (squared sums) or the Laplacian (second differences)
        {
            const int lx = (int)threadIdx.x % NT_X, ly = (int)threadIdx.x / NT_X;
            const int i0 = b0 + 1 + lx, i1 = b1 + 1 + ly;
            if (i0 < n0 && i1 < n1) {
                const long long p = lin(I, i0, i1, 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q >= ns) break;
                    R gr = R(0), lp = R(0);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const R hk = R(0.5) * inv_dxi_r<R>(I, k);
                        const R h2 = inv_dxi_r<R>(I, k) * inv_dxi_r<R>(I, k);
                        const R sp = k == 0 ? ssig[q][ly + 1][lx + 2] : ssig[q][ly + 2][lx + 1];
                        const R sm = k == 0 ? ssig[q][ly + 1][lx] : ssig[q][ly][lx + 1];
                        const R gk = (sp - sm) * hk;
                        gr += gk * gk;
                        lp += (sp - R(2) * ssig[q][ly + 1][lx + 1] + sm) * h2;
                    }
                    R gq = I.sigma_op[q] == MON_LAP ? R(fabs(lp)) : R(sqrt(gr));
                    grad_r<R>(Sc)[(long long)q * I.ncell + p] = gq;
                    if (!(gq >= R(0))) gq = R(0);
                    kmax[1 + q] = max(kmax[1 + q], max_key(gq));
                }
            }
        }
        // block maxima of the CFL sum and of each monitor term, then the instance maxima
#pragma unroll
        for (int r = 0; r < 5; ++r)
            for (int o = 16; o > 0; o >>= 1) kmax[r] = shfl_max(kmax[r], o);
        if (lane == 0)
            for (int r = 0; r < 5; ++r) sred[r][wid] = kmax[r];
        __syncthreads();
        if ((int)threadIdx.x <= ns) {
            K m = sred[threadIdx.x][0];
            for (int w = 1; w < NW; ++w) m = max(m, sred[threadIdx.x][w]);
            atomic_max_pos(&Sc.red[threadIdx.x], key_value(m));
        }
    }
}

// cfl_grad_kernel for 3D instances in the mixed form, in two passes with the same terms.
// Pass 1, one node per thread: the CFL spectral-radius sum of Eq. (cfl) with the metrics of
// x^n, and sigma_s of the node state, stored behind the gradients in the gradient buffer.
template <int NS>
__global__ void __launch_bounds__(NODE_TPB, 4) cfl_sigma3d_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                                const StagePtrs* __restrict__ table,
                                                                const int2* __restrict__ work, int nwork,
                                                                const Scratch* __restrict__ scr)
{
    pdl_entry();
    using R = float;
    using K = unsigned int;
    constexpr int NC = NS + 4, NW = NODE_TPB / 32;
    __shared__ K sred[NW];
    const int lane = (int)threadIdx.x & 31, wid = (int)threadIdx.x >> 5;
    // the CFL maximum of a run of items of one instance: one block reduction per run
    K kc = 0;
    int cur = -1;
    auto flush = [&]() {
        for (int o = 16; o > 0; o >>= 1) kc = shfl_max(kc, o);
        __syncthreads();    // the previous run's readers of sred are done
        if (lane == 0) sred[wid] = kc;
        __syncthreads();
        if (threadIdx.x == 0) {
            K mx = sred[0];
            for (int w = 1; w < NW; ++w) mx = max(mx, sred[w]);
            atomic_max_pos(&scr[cur].red[0], key_value(mx));
        }
        kc = 0;
    };
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        if (it.x != cur) {
            if (cur >= 0) flush();
            cur = it.x;
        }
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const Scratch& Sc = scr[it.x];
        int i0, i1, i2;
        if (tile_node(I, it.y, 0, i0, i1, i2)) {
            const long long p = lin(I, i0, i1, i2), pid = plin(I, i0, i1, i2);
            double mraw[9];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j) mraw[3 * k + j] = Sc.M[(long long)(k * 4 + 1 + j) * I.npad + pid];
            R U[NC];
            const R Jp = to_r<R>(P.J[p]);
            const R inv = R(1) / Jp;
#pragma unroll
            for (int f = 0; f < NC; ++f) U[f] = to_r<R>(P.JU[f * I.ncell + p]) * inv;
            float* sg = grad_r<R>(Sc) + (long long)I.n_sigma * I.ncell;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s < I.n_sigma) sg[(long long)s * I.ncell + p] = sigma2d<R, NS, 3>(I, I.sigma[s], U);
            const R rho = U[0] + (NS == 2 ? U[1] : R(0));
            R v[3], v2 = R(0), cvr = R(0), ar = R(0), gm = R(0);
#pragma unroll
            for (int m = 0; m < 3; ++m) { v[m] = U[NS + m] / rho; v2 += v[m] * v[m]; }
#pragma unroll
            for (int l = 0; l < NS; ++l) {
                ar += Cst<R>::Rs(I, l) * U[l];          // (Gamma_l - 1) c_v,l rho_l
                gm += Cst<R>::cvG(I, l) * U[l];         // Gamma_l c_v,l rho_l
                cvr += Cst<R>::cv(I, l) * U[l];
            }
            const R T = (U[NC - 1] - R(0.5) * rho * v2 - Cst<R>::pinf(I)) / cvr;
            const R c = sqrt((ar / rho) * (gm / cvr) * T);
            R sr = R(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                R L2 = R(0), vn = R(0);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const R mk = to_r<R>(mraw[3 * k + j]);
                    L2 += mk * mk;
                    vn += mk * v[j];
                }
                sr += (fabs(vn) + c * sqrt(L2)) / Jp * inv_dxi_r<R>(I, k);
            }
            if (!(sr >= R(0))) sr = R(0);
            kc = max(kc, max_key(sr));
        }
    }
    if (cur >= 0) flush();
}

// sigma_s (s < n_sigma) at position g of a staged plane, at most one node outside the grid in
// one direction: at a ghost node, the value of the mapped node (load_U's maps), with v_1
// negated across a wall normal to i1 (the only monitor variable the reflection changes) and
// the inflow state's values on an inflow side
template <int NS>
__device__ __forceinline__ void grad3d_sigma(const Inst& I, const float* __restrict__ sg, int g0, int g1, int g2,
                                             float v[4])
{
    v[0] = v[1] = v[2] = v[3] = 0.0f;
    const int ns = I.n_sigma;
    int i[3] = { g0, g1, g2 }, kk = -1, out = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (i[k] < -1 || i[k] > I.n[k]) return;
        if (i[k] < 0 || i[k] >= I.n[k]) { kk = k; ++out; }
    }
    if (out > 1) return;
    int tmap = 0, side = 0;
    if (kk >= 0) {
        int gi;
        tmap = map_line(I, kk, kk == 0 ? i[0] : (kk == 1 ? i[1] : i[2]), gi, side);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k == kk) i[k] = gi;     // (unrolled: i stays in registers)
    }
    if (tmap == 2) {
        float U[MAXC];
#pragma unroll
        for (int f = 0; f < NS + 4; ++f) U[f] = to_r<float>(I.inflow[kk][side][f]);
#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (s < ns) v[s] = sigma2d<float, NS, 3>(I, I.sigma[s], U);
        return;
    }
    const long long p = lin(I, i[0], i[1], i[2]);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s >= ns) break;
        v[s] = sg[(long long)s * I.ncell + p];
        if (tmap == 1 && kk == 0 && I.sigma[s] == SIG_V1) v[s] = -v[s];
    }
}

// Pass 2, marching along i3 over the column items of col3: per monitor term |grad_xi sigma|
// or |Laplacian_xi sigma| (second-order central differences) from sigma_s staged plane by
// plane (the column and its one-node halo, in a ring of four planes), the instance maxima by
// one block reduction per item (integer keys of the non-negative maxima).
template <int NS>
__global__ void __launch_bounds__(NODE_TPB) grad3d_kernel(const Inst* __restrict__ insts,
                                                          const int2* __restrict__ work, int nwork,
                                                          const Scratch* __restrict__ scr)
{
    pdl_entry();
    using R = float;
    using K = unsigned int;
    constexpr int NW = NODE_TPB / 32;
    __shared__ R ssig[4][4][M3_PY][M3_PX];
    __shared__ K sred[4][NW];
    const int lx = (int)threadIdx.x % M3_TX, ly = (int)threadIdx.x / M3_TX;
    const int lane = (int)threadIdx.x & 31, wid = (int)threadIdx.x >> 5;
    int ha = -1, hb = -1;
    if ((int)threadIdx.x < M3_NH) m3_halo_slot((int)threadIdx.x, ha, hb);
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& Sc = scr[it.x];
        const Col3 C = col3(I, it.y);
        const int ns = I.n_sigma;
        const float* sg = grad_r<R>(Sc) + (long long)ns * I.ncell;
        const int g0 = C.b0 + lx, g1 = C.b1 + ly, h0 = C.b0 - 1 + ha, h1 = C.b1 - 1 + hb;
        const bool valid = g0 < I.n[0] && g1 < I.n[1];
        K kmax[4] = { 0, 0, 0, 0 };
        float vo[4], vh[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
        auto put = [&](int q) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                ssig[q & 3][s][ly + 1][lx + 1] = vo[s];
                if (ha >= 0) ssig[q & 3][s][hb][ha] = vh[s];
            }
        };
        __syncthreads();    // the previous item's readers are done
        for (int q = C.z0 - 1; q <= C.z0 + 1; ++q) {
            grad3d_sigma<NS>(I, sg, g0, g1, q, vo);
            if (ha >= 0) grad3d_sigma<NS>(I, sg, h0, h1, q, vh);
            put(q);
        }
        for (int z = C.z0; z < C.z1; ++z) {
            __syncthreads();
            // plane z + 2 into registers, into the ring after this plane's terms (its slot last
            // held plane z - 2, read at plane z - 1)
            const bool more = z + 2 <= C.z1;
            if (more) {
                grad3d_sigma<NS>(I, sg, g0, g1, z + 2, vo);
                if (ha >= 0) grad3d_sigma<NS>(I, sg, h0, h1, z + 2, vh);
            }
            if (valid) {
                const long long p = lin(I, g0, g1, z);
                const int c = z & 3, m = (z - 1) & 3, pp = (z + 1) & 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q >= ns) break;
                    const R sc = ssig[c][q][ly + 1][lx + 1];
                    R gr = R(0), lp = R(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const R hk = R(0.5) * inv_dxi_r<R>(I, k);
                        const R h2 = inv_dxi_r<R>(I, k) * inv_dxi_r<R>(I, k);
                        const R sp = k == 0 ? ssig[c][q][ly + 1][lx + 2] : (k == 1 ? ssig[c][q][ly + 2][lx + 1] : ssig[pp][q][ly + 1][lx + 1]);
                        const R sm = k == 0 ? ssig[c][q][ly + 1][lx] : (k == 1 ? ssig[c][q][ly][lx + 1] : ssig[m][q][ly + 1][lx + 1]);
                        const R gk = (sp - sm) * hk;
                        gr += gk * gk;
                        lp += (sp - R(2) * sc + sm) * h2;
                    }
                    R gq = I.sigma_op[q] == MON_LAP ? R(fabs(lp)) : R(sqrt(gr));
                    grad_r<R>(Sc)[(long long)q * I.ncell + p] = gq;
                    if (!(gq >= R(0))) gq = R(0);
                    kmax[q] = max(kmax[q], max_key(gq));
                }
            }
            if (more) put(z + 2);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            for (int o = 16; o > 0; o >>= 1) kmax[r] = shfl_max(kmax[r], o);
        __syncthreads();    // the previous item's readers of sred are done
        if (lane == 0)
            for (int r = 0; r < 4; ++r) sred[r][wid] = kmax[r];
        __syncthreads();
        if ((int)threadIdx.x < ns) {
            K mx = sred[threadIdx.x][0];
            for (int w = 1; w < NW; ++w) mx = max(mx, sred[threadIdx.x][w]);
            atomic_max_pos(&Sc.red[1 + threadIdx.x], key_value(mx));
        }
    }
}

// Eq. (monitor) at node p from the gradients and the reciprocal instance maxima (0 for a zero maximum)
template <typename R>
__device__ __forceinline__ R theta_at(const Inst& I, const Scratch& S, const R* inv, long long p)
{
    R t = R(1);
    for (int q = 0; q < I.n_sigma; ++q) {
        if (inv[q] > R(0)) {
            const R r = grad_r<R>(S)[(long long)q * I.ncell + p] * inv[q];
            // Eq. (monitor) squares the ratio; the vortex monitor's terms are linear
            t += I.sigma_op[q] == MON_GRAD2 ? alpha_r<R>(I, q) * r * r : alpha_r<R>(I, q) * r;
        }
    }
    return sqrt(t);
}

// reciprocal of the instance maximum of monitor term q in the compute type (0 for a zero maximum)
template <typename R>
__device__ __forceinline__ R inv_max(const Scratch& S, int q)
{
    const double m = S.red[1 + q];
    if (!(m > 0.0)) return R(0);
    if constexpr (std::is_same<R, float>::value) return R(1) / f64_to_f32(m);
    else return 1.0 / m;
}

template <typename R>
__global__ void monitor_theta_kernel(const Inst* __restrict__ insts, const int2* __restrict__ work, int nwork,
                                     const Scratch* __restrict__ scr)
{
    pdl_entry();
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& P = scr[it.x];
        int i0, i1, i2;
        if (!tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long p = lin(I, i0, i1, i2);
        R inv[4] = { R(0), R(0), R(0), R(0) };
        for (int q = 0; q < I.n_sigma; ++q) inv[q] = inv_max<R>(P, q);
        reinterpret_cast<R*>(P.th0)[p] = theta_at<R>(I, P, inv, p);
    }
}

// one pass of the low-pass filter, weights (1/2)^(|j|_1 + d) over the 3^d stencil; the first
// pass (FROM_G) forms the monitor function of each stencil node from the gradients directly
template <typename R, bool FROM_G>
__global__ void filter_kernel(const Inst* __restrict__ insts, const int2* __restrict__ work, int nwork,
                              const Scratch* __restrict__ scr, int parity)
{
    pdl_entry();
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& Sc = scr[it.x];
        int i0, i1, i2;
        if (!tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long p = lin(I, i0, i1, i2);
        const R* a = reinterpret_cast<const R*>(parity ? Sc.th1 : Sc.th0);
        R* dst = reinterpret_cast<R*>(parity ? Sc.th0 : Sc.th1);
        R inv[4] = { R(0), R(0), R(0), R(0) };
        if (FROM_G)
            for (int q = 0; q < I.n_sigma; ++q) inv[q] = inv_max<R>(Sc, q);
        auto val = [&](long long q) -> R { return FROM_G ? theta_at<R>(I, Sc, inv, q) : a[q]; };
        R acc = R(0);
        int lo3 = I.d == 3 ? -1 : 0, hi3 = I.d == 3 ? 1 : 0;
        const int n0 = I.n[0], n1 = I.n[1];
        const bool inner = i0 >= 1 && i0 < n0 - 1 && i1 >= 1 && i1 < n1 - 1 && (I.d == 2 || (i2 >= 1 && i2 < I.n[2] - 1));
        for (int j3 = lo3; j3 <= hi3; ++j3)
            for (int j2 = -1; j2 <= 1; ++j2) {
                R row = R(0);
                if (inner) {
                    const long long q = p + (long long)j3 * n0 * n1 + j2 * n0;
                    row = R(0.25) * (val(q - 1) + val(q + 1)) + R(0.5) * val(q);
                } else {
                    for (int j1 = -1; j1 <= 1; ++j1) row += (j1 == 0 ? R(0.5) : R(0.25)) * val(s_map(I, i0 + j1, i1 + j2, i2 + j3));
                }
                acc += (j2 == 0 ? R(0.5) : R(0.25)) * (j3 == 0 ? (I.d == 3 ? R(0.5) : R(1)) : R(0.25)) * row;
            }
        dst[p] = acc;
    }
}

// one Jacobi sweep: x_i = sum_k (T_{k+} x_{i+e_k} + T_{k-} x_{i-e_k}) / dxi_k^2 / sum_k (T_{k+} + T_{k-}) / dxi_k^2;
// the last sweep also forms the limiter bounds of Sec. 4 from x^[mu] - x^n (per-instance minimum)
template <typename R, bool LAST>
__global__ void jacobi_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                              const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr, int sweep,
                              int theta_sel)
{
    pdl_entry();
    __shared__ double sh[32];
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        int i[3];
        const bool valid = tile_node(I, it.y, 0, i[0], i[1], i[2]);
        ES_PTRS(P);
        double bnd = 1.0;
        if (valid) {
            const long long p = lin(I, i[0], i[1], i[2]);
            const Scratch& Sc = scr[it.x];
            const R* th = reinterpret_cast<const R*>(theta_sel ? Sc.th1 : Sc.th0);
            const double* xs = sweep == 0 ? P.x : (sweep % 2 == 1 ? Sc.xa : Sc.xb);
            double* xd_ = sweep % 2 == 0 ? Sc.xa : Sc.xb;
            double tc = to_d(th[p]);
            double num[3] = { 0, 0, 0 }, den = 0.0;
            bool inner = true;
            for (int k = 0; k < I.d; ++k) inner = inner && i[k] >= 1 && i[k] < I.n[k] - 1;
            long long stride = 1;
            for (int k = 0; k < I.d; ++k) {
                double tp, tm, xp[3], xm[3];
                if (inner) {
                    tp = 0.5 * (tc + to_d(th[p + stride]));
                    tm = 0.5 * (tc + to_d(th[p - stride]));
                    for (int j = 0; j < I.d; ++j) {
                        xp[j] = xs[(long long)j * I.ncell + p + stride];
                        xm[j] = xs[(long long)j * I.ncell + p - stride];
                    }
                } else {
                    int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
                    ip[k] += 1;
                    im[k] -= 1;
                    tp = 0.5 * (tc + to_d(th[s_map(I, ip[0], ip[1], ip[2])]));
                    tm = 0.5 * (tc + to_d(th[s_map(I, im[0], im[1], im[2])]));
                    x_at<false>(I, xs, ip[0], ip[1], ip[2], xp);
                    x_at<false>(I, xs, im[0], im[1], im[2], xm);
                }
                stride *= I.n[k];
                double h2 = I.inv_dxi[k] * I.inv_dxi[k];
                for (int j = 0; j < I.d; ++j) num[j] += (tp * xp[j] + tm * xm[j]) * h2;
                den += (tp + tm) * h2;
            }
            double id;
            if constexpr (std::is_same<R, double>::value) {
                id = 1.0 / den;
            } else {
                // FP32 reciprocal refined by one Newton-Raphson step in FP64 (relative error ~1e-14)
                double r0 = f32_to_f64(__frcp_rn(f64_to_f32(den)));
                id = r0 * fma(-den, r0, 2.0);
            }
            double xnew[3];
            for (int j = 0; j < I.d; ++j) {
                xnew[j] = num[j] * id;
                xd_[(long long)j * I.ncell + p] = xnew[j];
            }
            if (LAST) {
                for (int k = 0; k < I.d; ++k) {
                    double xc = P.x[(long long)k * I.ncell + p];
                    double dx = xnew[k] - xc;
                    int nb[3] = { i[0], i[1], i[2] };
                    double xn[3];
                    if (dx < 0.0) {
                        nb[k] -= 1;
                        x_at<false>(I, P.x, nb[0], nb[1], nb[2], xn);
                        bnd = fmin(bnd, -(xc - xn[k]) / (2.0 * dx));
                    } else if (dx > 0.0) {
                        nb[k] += 1;
                        x_at<false>(I, P.x, nb[0], nb[1], nb[2], xn);
                        bnd = fmin(bnd, (xn[k] - xc) / (2.0 * dx));
                    }
                }
                if (!(bnd >= 0.0)) bnd = 0.0;
            }
        }
        if (LAST) {
            double m = block_min_pos(bnd, sh);
            if (threadIdx.x == 0) atomic_min_pos(&scr[it.x].red[5], m);
        }
    }
}

// Mixed form: one Jacobi sweep of the mesh equation on the displacement y = x - x^n in
// binary32.  With the spacings dl_{k+-} = x^n_{i+-e_k} - x^n_i (formed in FP64 by the first
// sweep, stored rounded to binary32) the sweep x_i <- sum T_{k+-} x_{i+-e_k} / dxi_k^2 /
// sum T_{k+-} / dxi_k^2 reads y_i <- sum w_{k+-} (dl_{k+-} + y_{i+-e_k}) / sum w_{k+-}.
// The positions stay FP64 (x^n + y); only the sweep arithmetic is FP32.  The last sweep
// also forms the limiter bounds of Sec. 4, dl_{k,s}[k] / (2 y_k) with s the sign of y_k.
template <int D, bool FIRST, bool LAST>
__global__ void __launch_bounds__(NODE_TPB) jacobi_y_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                             const StagePtrs* __restrict__ table,
                                                             const int2* __restrict__ work, int nwork,
                                                             const Scratch* __restrict__ scr, int sweep, int theta_sel)
{
    pdl_entry();
    __shared__ double sh[32];
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        int i[3];
        const bool valid = tile_node(I, it.y, 0, i[0], i[1], i[2]);
        ES_PTRS(P);
        float bnd = 1.0f;
        if (valid) {
            const Scratch& Sc = scr[it.x];
            const long long n = I.ncell;
            const long long p = lin(I, i[0], i[1], i[2]);
            const float* th = reinterpret_cast<const float*>(theta_sel ? Sc.th1 : Sc.th0);
            const float* ys = reinterpret_cast<const float*>(sweep % 2 == 1 ? Sc.xa : Sc.xb);
            float* yd = reinterpret_cast<float*>(sweep % 2 == 0 ? Sc.xa : Sc.xb);
            float* dl = Sc.dl;
            const float tc = th[p];
            bool inner = true;
#pragma unroll
            for (int k = 0; k < D; ++k) inner = inner && i[k] >= 1 && i[k] < I.n[k] - 1;
            float num[D], den = 0.0f, dk[D][2];
#pragma unroll
            for (int j = 0; j < D; ++j) num[j] = 0.0f;
            if (inner && !FIRST) {
                // interior, after the first sweep: every load up front, no boundary maps
                const long long st[3] = { 1, I.n[0], (long long)I.n[0] * I.n[1] };
                float tn[D][2], dv[D][2][D], yv[D][2][D];
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const long long q = p + (s ? st[k] : -st[k]);
                        tn[k][s] = th[q];
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            dv[k][s][j] = dl[((k * 2 + s) * D + j) * n + p];
                            yv[k][s][j] = ys[j * n + q];
                        }
                    }
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const float w = 0.5f * (tc + tn[k][s]) * I.f_h2[k];
                        dk[k][s] = dv[k][s][k];
#pragma unroll
                        for (int j = 0; j < D; ++j) num[j] = fmaf(w, dv[k][s][j] + yv[k][s][j], num[j]);
                        den += w;
                    }
            } else {
            long long stride = 1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    int nb[3] = { i[0], i[1], i[2] };
                    nb[k] += s ? 1 : -1;
                    const long long q = p + (s ? stride : -stride);
                    const float w = 0.5f * (tc + th[inner ? q : s_map(I, nb[0], nb[1], nb[2])]) * I.f_h2[k];
                    float dv[D], yv[D];
                    if (FIRST) {
                        double xn[3];
                        if (inner) {
#pragma unroll
                            for (int j = 0; j < D; ++j) xn[j] = P.x[j * n + q];
                        } else {
                            x_at<false>(I, P.x, nb[0], nb[1], nb[2], xn);
                        }
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            dv[j] = f64_to_f32(xn[j] - P.x[j * n + p]);
                            dl[((k * 2 + s) * D + j) * n + p] = dv[j];
                            yv[j] = 0.0f;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < D; ++j) dv[j] = dl[((k * 2 + s) * D + j) * n + p];
                        if (inner) {
#pragma unroll
                            for (int j = 0; j < D; ++j) yv[j] = ys[j * n + q];
                        } else {
                            y_at(I, ys, nb[0], nb[1], nb[2], yv);
                        }
                    }
                    dk[k][s] = dv[k];
#pragma unroll
                    for (int j = 0; j < D; ++j) num[j] = fmaf(w, dv[j] + yv[j], num[j]);
                    den += w;
                }
                stride *= I.n[k];
            }
            }
            float ynew[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                ynew[j] = num[j] / den;
                yd[j * n + p] = ynew[j];
            }
            if (LAST) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float dx = ynew[k];
                    if (dx < 0.0f) bnd = fminf(bnd, dk[k][0] / (2.0f * dx));
                    else if (dx > 0.0f) bnd = fminf(bnd, dk[k][1] / (2.0f * dx));
                }
                if (!(bnd >= 0.0f)) bnd = 0.0f;
            }
        }
        if (LAST) {
            const double m = block_min_pos(f32_to_f64(bnd), sh);
            if (threadIdx.x == 0) atomic_min_pos(&scr[it.x].red[5], m);
        }
    }
}

// Slot q = threadIdx.x, threadIdx.x + TPB, ... of a W-wide region (TPB threads per block) and its column and row
// (a, b) = (q % W, q / W), stepped without a division per slot (W is a run-time width)
template <int TPB>
struct SlotIterN {
    int q, a, b, da, db, W;
    __device__ explicit SlotIterN(int W_) : q((int)threadIdx.x), W(W_)
    {
        b = q / W;
        a = q - b * W;
        db = TPB / W;
        da = TPB - db * W;
    }
    __device__ void next()
    {
        q += TPB;
        a += da;
        b += db;
        if (a >= W) { a -= W; ++b; }
    }
};
using SlotIter = SlotIterN<NODE_TPB>;


// Mixed form, 2D: the monitor, its F <= 4 filter passes and all H = mu <= 8 Jacobi sweeps
// of jacobi_y_kernel in one launch (temporal blocking).  A block of TPB threads stages the region
// of its TX x TY node tile plus a halo of H + F nodes in shared memory: Theta (formed from the
// monitor gradients, then filtered F times; the halo shrinks by one node per pass), then on
// the inner region (halo H) the displacements (ping-pong) and the spacings dl_{k+-} (formed in
// FP64 from x^n, rounded to binary32).  Each Jacobi sweep updates every in-domain node of the
// inner region with the arithmetic of jacobi_y_kernel, then re-mirrors the wall ghost nodes
// from their source nodes; each filter pass likewise re-copies the boundary node into its
// ghosts (the maps of s_map).  The valid zone shrinks by one node per pass or sweep, so after
// all of them the tile is exact.  Periodic directions need no care: the region runs over
// unwrapped indices and reads the wrapped node's data.  The last sweep forms the limiter
// bounds of Sec. 4 for the tile.  F < 0: Theta is read from the buffer theta_sel instead.
template <int TX, int TY, int TPB>
__global__ void __launch_bounds__(TPB, 1024 / TPB) jacobi_fused2d_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                                          const StagePtrs* __restrict__ table,
                                                                          const int2* __restrict__ work, int nwork,
                                                                          const Scratch* __restrict__ scr, int H, int F,
                                                                          int theta_sel)
{
    using SI = SlotIterN<TPB>;
    pdl_entry();
    extern __shared__ float jsm[];
    __shared__ double sh[32];
    const int Fp = F > 0 ? F : 0;
    const int RX = TX + 2 * H, RY = TY + 2 * H, NR = RX * RY;
    const int RXo = RX + 2 * Fp, RYo = RY + 2 * Fp, NRo = RXo * RYo;
    float* ya = jsm;              // [2][NR]
    float* yb = ya + 2 * NR;      // [2][NR]
    float* dq = yb + 2 * NR;      // [8][NR]: (k * 2 + s) * 2 + j
    float* ta = dq + 8 * NR;      // [NRo] Theta ping-pong on the outer region
    float* tb = ta + NRo;
    float* wq = tb + NRo;         // [4][NR] sweep weights (k * 2 + s), fixed while Theta is
    float* dn = wq + 4 * NR;      // [NR] their sum; 0 marks a slot no sweep updates
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const Scratch& Sc = scr[it.x];
        const int n0 = I.n[0], n1 = I.n[1];
        const bool per0 = I.bc[0][0] == BC_PERIODIC, per1 = I.bc[1][0] == BC_PERIODIC;
        const int ntx = (n0 + TX - 1) / TX;
        const int r0 = (it.y % ntx) * TX - H, r1 = (it.y / ntx) * TY - H;    // inner region origin
        const int o0 = r0 - Fp, o1 = r1 - Fp;                                     // outer region origin
        const long long n = I.ncell;
        // whether the outer / inner region holds wall ghost nodes (tile-uniform: a region
        // without them skips the ghost passes and their barriers)
        const bool gh_out = (!per0 && (o0 < 0 || o0 + RXo > n0)) || (!per1 && (o1 < 0 || o1 + RYo > n1));
        const bool gh_in = (!per0 && (r0 < 0 || r0 + RX > n0)) || (!per1 && (r1 < 0 || r1 + RY > n1));
        __syncthreads();
        // Theta on the outer region: Eq. (monitor) from the gradients at the mapped node (s_map)
        float inv[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
        if (F >= 0)
            for (int q = 0; q < I.n_sigma; ++q) inv[q] = inv_max<float>(Sc, q);
        const float* th = reinterpret_cast<const float*>(theta_sel ? Sc.th1 : Sc.th0);
        for (SI sl(RXo); sl.q < NRo; sl.next()) {
            const int q = sl.q;
            const long long src = s_map(I, o0 + sl.a, o1 + sl.b, 0);
            ta[q] = F >= 0 ? theta_at<float>(I, Sc, inv, src) : th[src];
        }
        __syncthreads();
        // F filter passes (weights (1/2)^(|j|_1 + 2) over the 3 x 3 stencil)
        float* tc_ = ta;
        float* tn_ = tb;
        for (int f = 0; f < F; ++f) {
            for (SI sl(RXo); sl.q < NRo; sl.next()) {
                const int q = sl.q, a = sl.a, b = sl.b;
                const int g0 = o0 + a, g1 = o1 + b;
                const bool ghost = (!per0 && (g0 < 0 || g0 >= n0)) || (!per1 && (g1 < 0 || g1 >= n1));
                if (ghost || a == 0 || a == RXo - 1 || b == 0 || b == RYo - 1) continue;
                float acc = 0.0f;
#pragma unroll
                for (int j2 = -1; j2 <= 1; ++j2) {
                    const int qr = q + j2 * RXo;
                    const float row = 0.25f * (tc_[qr - 1] + tc_[qr + 1]) + 0.5f * tc_[qr];
                    acc += (j2 == 0 ? 0.5f : 0.25f) * row;
                }
                tn_[q] = acc;
            }
            __syncthreads();
            // wall ghosts: copies of the boundary node
            if (gh_out) {
            for (SI sl(RXo); sl.q < NRo; sl.next()) {
                const int q = sl.q, a = sl.a, b = sl.b;
                const int g0 = o0 + a, g1 = o1 + b;
                const bool x0 = !per0 && (g0 < 0 || g0 >= n0), x1 = !per1 && (g1 < 0 || g1 >= n1);
                if (!x0 && !x1) continue;
                const int sa = (x0 ? (g0 < 0 ? 0 : n0 - 1) : g0) - o0, sb = (x1 ? (g1 < 0 ? 0 : n1 - 1) : g1) - o1;
                tn_[q] = (sa >= 0 && sa < RXo && sb >= 0 && sb < RYo) ? tn_[sb * RXo + sa] : 1.0f;
            }
            __syncthreads();
            }
            float* t = tc_;
            tc_ = tn_;
            tn_ = t;
        }
        const float* tq = tc_ + Fp * RXo + Fp;     // Theta at inner node (a, b): tq[b * RXo + a]
        // stage Theta, y = 0 and the + side spacings x^n_{i+e_k} - x^n_i of the in-domain nodes
        // (a periodic copy takes its wrapped node's, unshifted); the - side of a node whose
        // - neighbour is a wall ghost is formed here too, all others below
        for (SI sl(RX); sl.q < NR; sl.next()) {
            const int q = sl.q, a = sl.a, b = sl.b;
            const int g0 = r0 + a, g1 = r1 + b;
            ya[q] = ya[NR + q] = yb[q] = yb[NR + q] = 0.0f;
            const bool ghost = (!per0 && (g0 < 0 || g0 >= n0)) || (!per1 && (g1 < 0 || g1 >= n1));
            if (ghost) continue;
            const int w0 = per0 ? g0 - floordiv_(g0, n0) * n0 : g0, w1 = per1 ? g1 - floordiv_(g1, n1) * n1 : g1;
            const long long c = lin(I, w0, w1, 0);
            const double xc[2] = { P.x[c], P.x[n + c] };
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int sd = 0; sd < 2; ++sd) {
                    const int nb0 = w0 + (k == 0 ? (sd ? 1 : -1) : 0), nb1 = w1 + (k == 1 ? (sd ? 1 : -1) : 0);
                    const bool inside = nb0 >= 0 && nb0 < n0 && nb1 >= 0 && nb1 < n1;
                    const bool wall = !(k == 0 ? per0 : per1) && !inside;
                    if (sd == 0 && !wall) continue;          // from the neighbour's + side below
                    double xn[3];
                    if (inside) {
                        const long long cn = lin(I, nb0, nb1, 0);
                        xn[0] = P.x[cn];
                        xn[1] = P.x[n + cn];
                    } else {
                        x_at<false>(I, P.x, nb0, nb1, 0, xn);
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) dq[((k * 2 + sd) * 2 + j) * NR + q] = f64_to_f32(xn[j] - xc[j]);
                }
        }
        __syncthreads();
        // the remaining - sides: minus the + side of the - neighbour (the same pair of nodes);
        // and the sweep weights Theta_{k+-1/2} / dxi_k^2 of every slot a sweep updates, with
        // their sum, formed once since Theta stays fixed through the sweeps
        for (SI sl(RX); sl.q < NR; sl.next()) {
            const int q = sl.q, a = sl.a, b = sl.b;
            const int g0 = r0 + a, g1 = r1 + b;
            const bool ghost = (!per0 && (g0 < 0 || g0 >= n0)) || (!per1 && (g1 < 0 || g1 >= n1));
            float den = 0.0f;
            if (!ghost && a != 0 && a != RX - 1 && b != 0 && b != RY - 1) {
                const int qt = b * RXo + a;
                const float tc = tq[qt];
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int sd = 0; sd < 2; ++sd) {
                        const int qtn = qt + (k == 0 ? (sd ? 1 : -1) : (sd ? RXo : -RXo));
                        const float w = 0.5f * (tc + tq[qtn]) * I.f_h2[k];
                        wq[(k * 2 + sd) * NR + q] = w;
                        den += w;
                    }
            }
            dn[q] = den;
            if (ghost) continue;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool wall = k == 0 ? (!per0 && g0 == 0) : (!per1 && g1 == 0);
                if (wall || (k == 0 ? a == 0 : b == 0)) continue;
                const int qn = q - (k == 0 ? 1 : RX);
#pragma unroll
                for (int j = 0; j < 2; ++j) dq[((k * 2 + 0) * 2 + j) * NR + q] = -dq[((k * 2 + 1) * 2 + j) * NR + qn];
            }
        }
        __syncthreads();
        float* yc = ya;
        float* yn = yb;
        for (int sw = 0; sw < H; ++sw) {
            // in-domain nodes: one sweep (neighbours outside the region leave a node invalid);
            // the slots with a zero weight sum (wall ghosts, the region's edge) keep their values
            for (int q = threadIdx.x; q < NR; q += TPB) {
                const float den = dn[q];
                if (den == 0.0f) continue;
                float num[2] = { 0.0f, 0.0f };
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int sd = 0; sd < 2; ++sd) {
                        const int qn = q + (k == 0 ? (sd ? 1 : -1) : (sd ? RX : -RX));
                        const float w = wq[(k * 2 + sd) * NR + q];
#pragma unroll
                        for (int j = 0; j < 2; ++j) num[j] = fmaf(w, dq[((k * 2 + sd) * 2 + j) * NR + q] + yc[j * NR + qn], num[j]);
                    }
#pragma unroll
                for (int j = 0; j < 2; ++j) yn[j * NR + q] = num[j] / den;
            }
            __syncthreads();
            // wall ghosts: the mirror of their source node, the mirrored component negated
            if (gh_in) {
            for (SI sl(RX); sl.q < NR; sl.next()) {
                const int q = sl.q, a = sl.a, b = sl.b;
                const int g0 = r0 + a, g1 = r1 + b;
                const bool o0 = !per0 && (g0 < 0 || g0 >= n0), o1 = !per1 && (g1 < 0 || g1 >= n1);
                if (!o0 && !o1) continue;
                const int m0 = o0 ? (g0 < 0 ? -1 - g0 : 2 * n0 - 1 - g0) : g0;
                const int m1 = o1 ? (g1 < 0 ? -1 - g1 : 2 * n1 - 1 - g1) : g1;
                const int sa = m0 - r0, sb = m1 - r1;
                float v0 = 0.0f, v1 = 0.0f;
                if (sa >= 0 && sa < RX && sb >= 0 && sb < RY) {    // else the ghost is outside the valid zone
                    v0 = yn[sb * RX + sa];
                    v1 = yn[NR + sb * RX + sa];
                }
                yn[q] = o0 ? -v0 : v0;
                yn[NR + q] = o1 ? -v1 : v1;
            }
            __syncthreads();
            }
            float* t = yc;
            yc = yn;
            yn = t;
        }
        // the tile: store y^[mu] and form the limiter bounds
        const int lx = (int)threadIdx.x % TX, ly = (int)threadIdx.x / TX;
        const int i0 = r0 + H + lx, i1 = r1 + H + ly;
        float bnd = 1.0f;
        if ((int)threadIdx.x < TX * TY && i0 < n0 && i1 < n1) {
            const int q = (ly + H) * RX + lx + H;
            const long long p = lin(I, i0, i1, 0);
            float* yd = reinterpret_cast<float*>(I.mu % 2 == 1 ? Sc.xa : Sc.xb);
            yd[p] = yc[q];
            yd[n + p] = yc[NR + q];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float dx = yc[k * NR + q];
                if (dx < 0.0f) bnd = fminf(bnd, dq[((k * 2 + 0) * 2 + k) * NR + q] / (2.0f * dx));
                else if (dx > 0.0f) bnd = fminf(bnd, dq[((k * 2 + 1) * 2 + k) * NR + q] / (2.0f * dx));
            }
            if (!(bnd >= 0.0f)) bnd = 0.0f;
        }
        const double m = block_min_pos(f32_to_f64(bnd), sh);
        if (threadIdx.x == 0) atomic_min_pos(&scr[it.x].red[5], m);
    }
}

size_t jacobi_fused2d_smem(int H, int F, int shape)
{
    const int TX = JF_SHAPES[shape][0], TY = JF_SHAPES[shape][1];
    const size_t nr = (size_t)(TX + 2 * H) * (TY + 2 * H);
    const size_t Fp = F > 0 ? F : 0, nro = (TX + 2 * H + 2 * Fp) * (TY + 2 * H + 2 * Fp);
    return sizeof(float) * (17 * nr + 2 * nro);
}

#define JF_KERNELS(X) X(0, 32, 8, 256) X(1, 32, 16, 512) X(2, 24, 16, 512) X(3, 24, 12, 512)

void prepare_mesh()
{
    prepare_mesh3d();
#define JF_ATTR(S, TX, TY, TPB)                                                                         \
    cudaFuncSetAttribute(jacobi_fused2d_kernel<TX, TY, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)jacobi_fused2d_smem(JACOBI_FUSED_MAX, FILTER_FUSED_MAX, S));
    JF_KERNELS(JF_ATTR)
#undef JF_ATTR
}

void launch_jacobi_fused2d(int shape, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                           const StagePtrs* table, const int2* work, int nwork, const Scratch* scr, int H, int F,
                           int theta_sel)
{
    const size_t sm = jacobi_fused2d_smem(H, F, shape);
#define JF_LAUNCH(S, TX, TY, TPB)                                                                                  \
    if (shape == S)                                                                                                \
        pdl_launch(jacobi_fused2d_kernel<TX, TY, TPB>, grid, TPB, sm, st, insts, single, table, work, nwork, scr, H, F, \
                   theta_sel);
    JF_KERNELS(JF_LAUNCH)
#undef JF_LAUNCH
}

// Delta_tau = min(1, bounds of Sec. 4) per instance
__device__ inline const double* xmu_of(const StagePtrs& P, const Scratch& S, int mu)
{
    return mu == 0 ? P.x : (mu % 2 == 1 ? S.xa : S.xb);
}

__global__ void limiter_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                               const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr)
{
    pdl_entry();
    __shared__ double sh[32];
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const double* xmu = xmu_of(P, scr[it.x], I.mu);
        int i[3];
        const bool valid = tile_node(I, it.y, 0, i[0], i[1], i[2]);
        const long long p = valid ? lin(I, i[0], i[1], i[2]) : 0;
        double b = 1.0;
        if (valid) {
            for (int k = 0; k < I.d; ++k) {
                double xc = P.x[(long long)k * I.ncell + p];
                double dx = xmu[(long long)k * I.ncell + p] - xc;
                int nb[3] = { i[0], i[1], i[2] };
                double xn[3];
                if (dx < 0.0) {
                    nb[k] -= 1;
                    x_at<false>(I, P.x, nb[0], nb[1], nb[2], xn);
                    b = fmin(b, -(xc - xn[k]) / (2.0 * dx));
                } else if (dx > 0.0) {
                    nb[k] += 1;
                    x_at<false>(I, P.x, nb[0], nb[1], nb[2], xn);
                    b = fmin(b, (xn[k] - xc) / (2.0 * dx));
                }
            }
            if (!(b >= 0.0)) b = 0.0;
        }
        double m = block_min_pos(b, sh);
        if (threadIdx.x == 0) atomic_min_pos(&scr[it.x].red[5], m);
    }
}

// Delta t = C / max (or the given step), xdot = Delta_tau (x^[mu] - x^n) / Delta t;
// out = (Delta t, Delta_tau)
template <bool FAST>
__global__ void xdot_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                            const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr)
{
    pdl_entry();
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const double* red = scr[it.x].red;
        const double* xmu = xmu_of(P, scr[it.x], I.mu);
        double dt = P.dt_fixed > 0.0 ? P.dt_fixed : I.cfl / red[0];
        double dtau = red[5];
        if (it.y == 0 && threadIdx.x == 0) {
            P.out[0] = dt;
            P.out[1] = dtau;
        }
        int i0, i1, i2;
        if (!tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long p = lin(I, i0, i1, i2);
        if (FAST) {
            // mixed form: x^[mu] - x^n is the binary32 displacement of the sweeps
            const double sc = dtau / dt;
            const float* y = reinterpret_cast<const float*>(xmu);
            for (int j = 0; j < I.d; ++j) {
                const long long q = (long long)j * I.ncell + p;
                P.xdot_out[q] = I.mu > 0 ? sc * f32_to_f64(y[q]) : 0.0;
            }
        } else {
            for (int j = 0; j < I.d; ++j) {
                const long long q = (long long)j * I.ncell + p;
                P.xdot_out[q] = dtau * (xmu[q] - P.x[q]) / dt;
            }
        }
    }
}

// xdot_kernel over the padded node range of a full time step: interior nodes store the
// mesh velocity, and every node of the padded range stores the VCL metrics of the first
// RK stage from that velocity (ghost nodes through the velocity map) and the spatial
// metrics of x^n that the mesh step left in M, so the first stage forms no metrics.
// The velocity and the VCL metric are evaluated exactly as xdot_kernel and the metrics
// kernels do.
template <int D, bool MIXED>
__global__ void xdot_vcl_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr)
{
    pdl_entry();
    __shared__ double sc3[3];
    int cur = -1;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const double* xmu = xmu_of(P, scr[it.x], I.mu);
        // Delta t, Delta_tau and Delta_tau / Delta t: one thread of the block divides, once per
        // run of items of one instance
        if (it.x != cur) {
            __syncthreads();
            if (threadIdx.x == 0) {
                const double* red = scr[it.x].red;
                const double dt_ = P.dt_fixed > 0.0 ? P.dt_fixed : I.cfl / red[0];
                sc3[0] = dt_;
                sc3[1] = red[5];
                sc3[2] = red[5] / dt_;
            }
            __syncthreads();
            cur = it.x;
        }
        if (threadIdx.x == 0 && it.y == 0) {
            P.out[0] = sc3[0];
            P.out[1] = sc3[1];
        }
        const double dt = sc3[0], dtau = sc3[1];
        int i[3];
        if (!tile_node(I, it.y, 3, i[0], i[1], i[2])) continue;
        bool interior = true;
#pragma unroll
        for (int k = 0; k < D; ++k) interior = interior && i[k] >= 0 && i[k] < I.n[k];
        const long long n = I.ncell;
        const long long c = interior ? lin(I, i[0], i[1], i[2]) : 0;
        double xd[3] = { 0.0, 0.0, 0.0 };
        if (MIXED) {
            if (I.mu > 0) {
                const double sc = sc3[2];
                const float* y = reinterpret_cast<const float*>(xmu);
                float yv[3];
                if (interior) {
#pragma unroll
                    for (int j = 0; j < D; ++j) yv[j] = y[j * n + c];
                } else {
                    y_at(I, y, i[0], i[1], i[2], yv);
                }
#pragma unroll
                for (int j = 0; j < D; ++j) xd[j] = sc * f32_to_f64(yv[j]);
            }
        } else {
            double a[3], b[3];
            if (interior) {
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    a[j] = xmu[j * n + c];
                    b[j] = P.x[j * n + c];
                }
            } else {
                x_at<true>(I, xmu, i[0], i[1], i[2], a);
                x_at<true>(I, P.x, i[0], i[1], i[2], b);
            }
#pragma unroll
            for (int j = 0; j < D; ++j) xd[j] = dtau * (a[j] - b[j]) / dt;
        }
        if (interior) {
#pragma unroll
            for (int j = 0; j < D; ++j) P.xdot_out[j * n + c] = xd[j];
        }
        double* M = scr[it.x].M;
        const long long np = I.npad, p = plin(I, i[0], i[1], i[2]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double m[3];
#pragma unroll
            for (int j = 0; j < D; ++j) m[j] = M[(k * (D + 1) + 1 + j) * np + p];
            M[(k * (D + 1)) * np + p] = vcl_metric<D>(xd, m);
        }
    }
}

// 2D velocity pass of a full time step, over the padded node range: the mesh velocity on a tile
// plus a 3-node halo in shared memory (ghost nodes through the velocity map, values exactly as
// xdot_kernel forms them), then at every padded node the first stage's VCL metrics (from the
// spatial metrics of x^n in M), the metrics of the velocity into Md (the later stages use
// M + s dt Md: the 2D metrics are linear in x) and, at interior nodes, xdot itself.
template <bool MIXED>
__global__ void __launch_bounds__(NODE_TPB) xdot_vel2d_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                               const StagePtrs* __restrict__ table,
                                                               const int2* __restrict__ work, int nwork,
                                                               const Scratch* __restrict__ scr)
{
    pdl_entry();
    constexpr int HX = NT_X + 6, HY = NT_Y + 6;
    __shared__ double sv[2][HY][HX];
    __shared__ double sc3[3];
    const int lx = (int)threadIdx.x % NT_X, ly = (int)threadIdx.x / NT_X;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        const Scratch& Sc = scr[it.x];
        const double* xmu = xmu_of(P, Sc, I.mu);
        __syncthreads();
        if (threadIdx.x == 0) {
            const double dt_ = P.dt_fixed > 0.0 ? P.dt_fixed : I.cfl / Sc.red[0];
            sc3[0] = dt_;
            sc3[1] = Sc.red[5];
            sc3[2] = Sc.red[5] / dt_;
            if (it.y == 0) {
                P.out[0] = dt_;
                P.out[1] = Sc.red[5];
            }
        }
        __syncthreads();
        const double dt = sc3[0], dtau = sc3[1], sc = sc3[2];
        const int n0 = I.n[0], n1 = I.n[1];
        const long long n = I.ncell;
        const int ntx = (n0 + 6 + NT_X - 1) / NT_X;
        const int b0 = (it.y % ntx) * NT_X - 6, b1 = (it.y / ntx) * NT_Y - 6;
        for (int q = threadIdx.x; q < HX * HY; q += NODE_TPB) {
            const int a = q % HX, b = q / HX;
            const int g0 = b0 + a, g1 = b1 + b;
            double w[2] = { 0.0, 0.0 };
            if (g0 >= -6 && g0 < n0 + 6 && g1 >= -6 && g1 < n1 + 6) {
                const bool in = g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1;
                if (MIXED) {
                    if (I.mu > 0) {
                        const float* y = reinterpret_cast<const float*>(xmu);
                        float yv[3];
                        if (in) {
                            yv[0] = y[(long long)g1 * n0 + g0];
                            yv[1] = y[n + (long long)g1 * n0 + g0];
                        } else {
                            y_at(I, y, g0, g1, 0, yv);
                        }
                        w[0] = sc * f32_to_f64(yv[0]);
                        w[1] = sc * f32_to_f64(yv[1]);
                    }
                } else {
                    double ax[3], bx[3];
                    if (in) {
                        const long long c = (long long)g1 * n0 + g0;
                        ax[0] = xmu[c];
                        ax[1] = xmu[n + c];
                        bx[0] = P.x[c];
                        bx[1] = P.x[n + c];
                    } else {
                        x_at<true>(I, xmu, g0, g1, 0, ax);
                        x_at<true>(I, P.x, g0, g1, 0, bx);
                    }
                    w[0] = dtau * (ax[0] - bx[0]) / dt;
                    w[1] = dtau * (ax[1] - bx[1]) / dt;
                }
            }
            sv[0][b][a] = w[0];
            sv[1][b][a] = w[1];
        }
        __syncthreads();
        const int i0 = b0 + 3 + lx, i1 = b1 + 3 + ly;
        if (i0 >= n0 + 3 || i1 >= n1 + 3) continue;
        const int cx = lx + 3, cy = ly + 3;
        const double xd[2] = { sv[0][cy][cx], sv[1][cy][cx] };
        if (i0 >= 0 && i0 < n0 && i1 >= 0 && i1 < n1) {
            const long long c = (long long)i1 * n0 + i0;
            P.xdot_out[c] = xd[0];
            P.xdot_out[n + c] = xd[1];
        }
        const long long np = I.npad, p = plin(I, i0, i1, 0);
        const double m[4] = { Sc.M[1 * np + p], Sc.M[2 * np + p], Sc.M[4 * np + p], Sc.M[5 * np + p] };
        // the spatial rows of M hold m already (the metrics pass of x^n): only the VCL rows change
        const double r1[2] = { m[0], m[1] }, r2[2] = { m[2], m[3] };
        Sc.M[0 * np + p] = vcl_metric<2>(xd, r1);
        Sc.M[3 * np + p] = vcl_metric<2>(xd, r2);
        double md[4];
        metrics2d_at<HY, HX>(I, sv, cy, cx, md);
        store_metrics2d(Sc.Md, np, p, xd, md);
    }
}

// entropy diagnostics: per-block partial sums of V.dJU - phi dJ and J eta
__global__ void entropy_partial_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                       const int2* __restrict__ work, int nwork, double* __restrict__ partial)
{
    pdl_entry();
    __shared__ double sh[2][32];
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(P);
        int i0, i1, i2;
        const bool valid = tile_node(I, it.y, 0, i0, i1, i2);
        const long long p = valid ? lin(I, i0, i1, i2) : 0;
        double a = 0.0, b = 0.0;
        if (valid) {
            const double* JU = P.JU;
            double J = P.J[p], U[MAXC];
            for (int q = 0; q < I.nc; ++q) U[q] = JU[(long long)q * I.ncell + p] / J;
            double rl[2], v[3], T, pr, rho;
            prim(I, U, rl, v, T, pr, rho);
            double v2 = 0.0, eta = 0.0, phi = 0.0;
            for (int m = 0; m < I.d; ++m) v2 += v[m] * v[m];
            double lT = log(T);
            double V[MAXC];
            for (int l = 0; l < I.N; ++l) {
                double S = I.cv[l] * lT - I.Rs[l] * log(rl[l]);
                V[l] = -S - v2 / (2.0 * T) + I.cvG[l];
                eta -= rl[l] * S;
                phi += I.Rs[l] * rl[l] - I.pinf[l] / T;
            }
            for (int m = 0; m < I.d; ++m) V[I.N + m] = v[m] / T;
            V[I.N + I.d] = -1.0 / T;
            if (P.accU && P.accJ) {
                for (int q = 0; q < I.nc; ++q) a += V[q] * P.accU[(long long)q * I.ncell + p];
                a -= phi * P.accJ[p];
            }
            b = J * eta;
        }
        // deterministic block sums (fixed shuffle tree)
        for (int o = 16; o > 0; o >>= 1) { a += __shfl_xor_sync(0xffffffffu, a, o); b += __shfl_xor_sync(0xffffffffu, b, o); }
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sa = 0.0, sb = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += sh[0][q]; sb += sh[1][q]; }
            partial[2 * (long long)wi] = sa;
            partial[2 * (long long)wi + 1] = sb;
        }
    }
}

// one block per instance sums its partials in a fixed order
__global__ void entropy_final_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                     const int* __restrict__ first_work, const double* __restrict__ partial)
{
    pdl_entry();
    __shared__ double sh[2][32];
    int inst = blockIdx.x;
    const Inst& I = insts[inst];
    const StagePtrs P = table ? table[inst] : single;
    int w0 = first_work[inst], w1 = first_work[inst + 1];
    double a = 0.0, b = 0.0;
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) { a += partial[2 * (long long)w]; b += partial[2 * (long long)w + 1]; }
    for (int o = 16; o > 0; o >>= 1) { a += __shfl_xor_sync(0xffffffffu, a, o); b += __shfl_xor_sync(0xffffffffu, b, o); }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += sh[0][q]; sb += sh[1][q]; }
        double vol = 1.0;
        for (int k = 0; k < I.d; ++k) vol *= I.dxi[k];
        P.out[0] = vol * sa;
        P.out[1] = vol * sb;
    }
}

// schlieren function (Example 5.8, Eq. (schlieren)), pass 1: |grad_x rho| = |(1/J) sum_k
// J xi_k/x d rho/d xi_k| with central differences in xi and the metrics in M; per-instance
// maximum into red[6]
__global__ void schlieren_grad_kernel(const Inst* __restrict__ insts, StagePtrs single, const int2* __restrict__ work,
                                      int nwork, const Scratch* __restrict__ scr)
{
    pdl_entry();
    __shared__ double sh[32];
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const StagePtrs& P = single;
        int i[3];
        const bool valid = tile_node(I, it.y, 0, i[0], i[1], i[2]);
        double gmag = 0.0;
        if (valid) {
            const long long p = lin(I, i[0], i[1], i[2]), pid = plin(I, i[0], i[1], i[2]);
            double drho[3] = { 0.0, 0.0, 0.0 };
            for (int k = 0; k < I.d; ++k) {
                int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
                ip[k] += 1;
                im[k] -= 1;
                double Up[MAXC], Um[MAXC];
                load_U(I, P.JU, P.J, ip[0], ip[1], ip[2], Up);
                load_U(I, P.JU, P.J, im[0], im[1], im[2], Um);
                const double rp = Up[0] + (I.N == 2 ? Up[1] : 0.0), rm = Um[0] + (I.N == 2 ? Um[1] : 0.0);
                drho[k] = (rp - rm) * (0.5 * I.inv_dxi[k]);
            }
            double acc = 0.0;
            for (int j = 0; j < I.d; ++j) {
                double gj = 0.0;
                for (int k = 0; k < I.d; ++k) gj += scr[it.x].M[(long long)(k * (I.d + 1) + 1 + j) * I.npad + pid] * drho[k];
                gj /= P.J[p];
                acc += gj * gj;
            }
            gmag = sqrt(acc);
            scr[it.x].g[p] = gmag;
        }
        const double m = block_max<double>(gmag, sh);
        if (threadIdx.x == 0) atomic_max_pos(&scr[it.x].red[6], m);
    }
}

// pass 2: phi = exp(-Psi |grad rho| / max), Psi = (psi1 rho_1 + psi2 rho_2) / rho; 1 for max 0
__global__ void schlieren_phi_kernel(const Inst* __restrict__ insts, StagePtrs single, const int2* __restrict__ work,
                                     int nwork, const Scratch* __restrict__ scr, double psi1, double psi2)
{
    pdl_entry();
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const StagePtrs& P = single;
        int i0, i1, i2;
        if (!tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long p = lin(I, i0, i1, i2);
        const double gmax = scr[it.x].red[6];
        const double r1 = P.JU[p], r2 = I.N == 2 ? P.JU[I.ncell + p] : 0.0;   // J rho_l: J cancels in Psi
        const double psi = (psi1 * r1 + psi2 * r2) / (r1 + r2);
        P.out[p] = gmax > 0.0 ? exp(-psi * scr[it.x].g[p] / gmax) : 1.0;
    }
}

void launch_monitor_theta(bool mixed, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                          const Scratch* scr)
{
    if (mixed) pdl_launch(monitor_theta_kernel<float>, grid, NODE_TPB, 0, st, insts, work, nwork, scr);
    else pdl_launch(monitor_theta_kernel<double>, grid, NODE_TPB, 0, st, insts, work, nwork, scr);
}

void launch_filter(bool mixed, bool from_g, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                   const Scratch* scr, int parity)
{
    if (mixed) {
        if (from_g) pdl_launch(filter_kernel<float, true>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, parity);
        else pdl_launch(filter_kernel<float, false>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, parity);
    } else {
        if (from_g) pdl_launch(filter_kernel<double, true>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, parity);
        else pdl_launch(filter_kernel<double, false>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, parity);
    }
}

void launch_cfl_grad(bool mixed, int d, int N, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                     const StagePtrs* table, const int2* work, int nwork, const Scratch* scr)
{
    if (d == 2) {
        if (mixed) {
            if (N == 1) pdl_launch(cfl_grad2d_kernel<float, 1>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
            else pdl_launch(cfl_grad2d_kernel<float, 2>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
        } else {
            if (N == 1) pdl_launch(cfl_grad2d_kernel<double, 1>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
            else pdl_launch(cfl_grad2d_kernel<double, 2>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
        }
        return;
    }
    // 3D: the FP64 form here; the mixed form runs launch_cfl_grad3d
    (void)mixed;
    pdl_launch(cfl_grad_kernel<double>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
}

void launch_cfl_grad3d(int N, int grid_cell, int grid_col, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                       const StagePtrs* table, const int2* w_cell, int n_cell, const int2* w_col, int n_col,
                       const Scratch* scr, bool monitor)
{
    if (N == 1) pdl_launch(cfl_sigma3d_kernel<1>, grid_cell, NODE_TPB, 0, st, insts, single, table, w_cell, n_cell, scr);
    else pdl_launch(cfl_sigma3d_kernel<2>, grid_cell, NODE_TPB, 0, st, insts, single, table, w_cell, n_cell, scr);
    if (!monitor) return;
    if (N == 1) pdl_launch(grad3d_kernel<1>, grid_col, NODE_TPB, 0, st, insts, w_col, n_col, scr);
    else pdl_launch(grad3d_kernel<2>, grid_col, NODE_TPB, 0, st, insts, w_col, n_col, scr);
}

void launch_xdot_vcl(bool mixed, int d, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                     const StagePtrs* table, const int2* work, int nwork, const Scratch* scr)
{
#define XV(D, MX) pdl_launch(xdot_vcl_kernel<D, MX>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr)
    if (d == 2) { if (mixed) XV(2, true); else XV(2, false); }
    else { if (mixed) XV(3, true); else XV(3, false); }
#undef XV
}

void launch_xdot_vel2d(bool mixed, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                       const StagePtrs* table, const int2* work, int nwork, const Scratch* scr)
{
    if (mixed) pdl_launch(xdot_vel2d_kernel<true>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
    else pdl_launch(xdot_vel2d_kernel<false>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
}

void launch_xdot(bool mixed, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                 const StagePtrs* table, const int2* work, int nwork, const Scratch* scr)
{
    if (mixed) pdl_launch(xdot_kernel<true>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
    else pdl_launch(xdot_kernel<false>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr);
}

void launch_jacobi(bool mixed, int d, bool last, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                   const StagePtrs* table, const int2* work, int nwork, const Scratch* scr, int sweep, int theta_sel)
{
#define JL(R, LS) pdl_launch(jacobi_kernel<R, LS>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr, sweep, theta_sel)
#define JY(D, F, LS) pdl_launch(jacobi_y_kernel<D, F, LS>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, scr, sweep, theta_sel)
    if (mixed) {
        // 2D (beyond the fused kernel's limits); the mixed 3D sweeps run launch_jacobi3d
        (void)d;
        const bool first = sweep == 0;
        if (first) { if (last) JY(2, true, true); else JY(2, true, false); }
        else { if (last) JY(2, false, true); else JY(2, false, false); }
    } else {
        if (last) JL(double, true);
        else JL(double, false);
    }
#undef JY
#undef JL
}

}  // namespace es
