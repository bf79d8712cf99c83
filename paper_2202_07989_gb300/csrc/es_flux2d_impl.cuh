// Fused 2D stage kernel: both directions of the residual of Eqs. (semi_U), (semi_J) for
// one SSP-RK3 stage of a two-dimensional instance in one launch, over TX x TY node tiles.
//
// A tile stages the cross of nodes its stencils reach: TX x TY output nodes, 3 halo
// columns on each side of its rows and 3 halo rows above and below its columns (the
// node array is (TX + 6) x (TY + 6) with its four 3 x 3 corners unused).  A node is
// formed once and serves both directions.  Direction 1 runs over the TY rows and direction
// 2 over the TX columns.  Each runs phases 2 and 3 of the per-direction kernel: distinct
// pairs, then interfaces.  The direction-1 divergence waits in shared memory (FP64) until
// direction 2 adds its own and applies the stage update.  The arithmetic is the
// per-direction kernel's, shared through es_flux_core.cuh, and so is the order of every
// sum (r_1 + r_2 in FP64).  The stage results are therefore bitwise those of the two
// per-direction launches.
#pragma once

#include "es_flux_core.cuh"

namespace es {

template <int TX, int TY>
struct Tile2 {
    static constexpr int RW = TX + 6;                          // row width of the node array
    static constexpr int NN = (TX + 6) * (TY + 6);             // node slots
    static constexpr int NO = TX * TY;                         // output nodes
    static constexpr int NPL0 = 3 * TX + 6, NPL1 = 3 * TY + 6; // distinct pairs per row / per column
    static constexpr int NP0 = NPL0 * TY, NP1 = NPL1 * TX;
    static constexpr int NP = NP0 > NP1 ? NP0 : NP1;
    static constexpr int NI0 = (TX + 1) * TY, NI1 = (TY + 1) * TX;
    static constexpr int NI = NI0 > NI1 ? NI0 : NI1;
    static constexpr int NM0 = (TX + 6) * TY, NM1 = TX * (TY + 6);   // FP64 J xi_k/t on the rows / columns
};

template <int NS, typename R, int TX, int TY>
__host__ __device__ constexpr size_t smem_flux2d()
{
    using Y = Lay<2, NS>;
    using T = Tile2<TX, TY>;
    return sizeof(double) * ((Y::NC + 1) * T::NO + T::NI + T::NM0 + T::NM1) +
           sizeof(R) * ((Y::NF + 3) * T::NN + Y::NC * T::NP + (NS + 1) * T::NI + Y::NC * T::NI);
}

// Phases 2 (distinct pairs) and 3 (interfaces) of direction K (0: along the rows, 1: along
// the columns).  Row pairs and interfaces are numbered line by line; column pairs and
// interfaces position by position across the TX columns, so that consecutive threads read
// consecutive nodes in both directions.  The kernel inlines both directions (constant K);
// a single copy looping over a run-time K measured no faster.
template <int NS, typename R, int TX, int TY, int WK>
__device__ __forceinline__ void flux2d_pairs(const int K, const Inst& I, int i0, int j0, const R* nr, R* pf, R* cm)
{
    using Y = Lay<2, NS>;
    using T = Tile2<TX, TY>;
    constexpr int NN = T::NN, NP = T::NP, NI = T::NI, RW = T::RW;
    const int S = K ? TY : TX, NPK = K ? T::NP1 : T::NP0, MR = K ? Y::NF : Y::MR;
    const int nk = I.n[K], na = I.n[1 - K], s0 = K ? j0 : i0, a0 = K ? i0 : j0;
    for (int t = threadIdx.x; t < NPK; t += blockDim.x) {
        const int w = K ? t % TX : t / T::NPL0, r_ = K ? t / TX : t % T::NPL0;
        int m, Ln;
        if (r_ < S + 1) { m = 1; Ln = r_ + 2; }
        else if (r_ < 2 * S + 3) { m = 2; Ln = r_ - (S + 1) + 1; }
        else { m = 3; Ln = r_ - (2 * S + 3); }
        if (a0 + w >= na || s0 - 3 + Ln + m > nk + 2) continue;
        const int l = K ? Ln * RW + (w + 3) : (w + 3) * RW + Ln;
        const int ci = m == 1 ? (K ? (Ln - 2) * TX + w : w * (S + 1) + (Ln - 2)) : -1;
        pair_flux<2, NS, R>(I, nr, NN, MR, l, l + m * (K ? RW : 1), pf, NP, t, cm, NI, ci);
    }
}

template <int NS, typename R, int TX, int TY, int WK>
__device__ __forceinline__ void flux2d_ifaces(const int K, const Inst& I, int i0, int j0, const R* nr, const double* mtk,
                                              const R* pf, const R* cm, R* fl, double* gt)
{
    using Y = Lay<2, NS>;
    using T = Tile2<TX, TY>;
    constexpr int NN = T::NN, NP = T::NP, NI = T::NI, RW = T::RW;
    const int S = K ? TY : TX, NIK = K ? T::NI1 : T::NI0, MR = K ? Y::NF : Y::MR;
    const int nk = I.n[K], na = I.n[1 - K], s0 = K ? j0 : i0, a0 = K ? i0 : j0;
    // strides: nodes along the line, J xi_k/t along the line, pairs of one kind along the line
    const int ns = K ? RW : 1, ms = K ? TX : 1, ps = K ? TX : 1;
    for (int f = threadIdx.x; f < NIK; f += blockDim.x) {
        const int w = K ? f % TX : f / (TX + 1), s = K ? f / TX : f % (TX + 1);
        const int gi = s0 - 1 + s;     // interface gi + 1/2
        if (a0 + w >= na || gi > nk - 1) continue;
        const int base = K ? s * RW + (w + 3) : (w + 3) * RW + s;    // node gi - 2 of line w
        const int mb = K ? s * TX + w : w * RW + s;
        const int p = K ? s * TX + w : w * T::NPL0 + s;
        iface_flux<2, NS, R, WK>(I, nr + base, NN, ns, MR, mtk + mb, ms, pf, NP, p, p + (S + 1) * ps, p + (2 * S + 3) * ps,
                                 ps, cm, NI, f, fl, gt);
    }
}

// divergence of direction 1 at the tile's output nodes into acc (FP64)
template <int NS, typename R, int TX, int TY>
__device__ __forceinline__ void flux2d_div1(const Inst& I, int i0, int j0, const R* fl, const double* gt, double* acc)
{
    constexpr int NC = NS + 3, NI = Tile2<TX, TY>::NI, NO = TX * TY;
    for (int t = threadIdx.x; t < NO; t += blockDim.x) {
        const int il = t % TX, jl = t / TX;
        if (i0 + il >= I.n[0] || j0 + jl >= I.n[1]) continue;
        const int fr = jl * (TX + 1) + il + 1;
        double r[NC + 1];
        node_div<NC, R>(I, fl, NI, gt, fr, fr - 1, I.inv_dxi[0], r);
#pragma unroll
        for (int q = 0; q <= NC; ++q) acc[q * NO + t] = r[q];
    }
}

// FP32 tiles: 3 CTAs per SM (<= 85 registers); FP64 tiles: 1 (FP64-pipe bound).  Modes:
// MODE_RK (the stage update) and MODE_WRITE (the residual r_1 + r_2 into accU, accJ).
template <int NS, typename R, int TX, int TY, int WK>
__global__ void __launch_bounds__(FLUX_TPB, (sizeof(R) == 4 ? 3 : 1)) flux2d_kernel(FluxLaunch L)
{
    pdl_entry();
    using Y = Lay<2, NS>;
    using T = Tile2<TX, TY>;
    constexpr int NC = Y::NC, NN = T::NN, NI = T::NI, NP = T::NP, NO = T::NO, RW = T::RW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* acc = reinterpret_cast<double*>(smem_raw);      // [NC + 1][NO] divergence of direction 1
    double* gt = acc + (NC + 1) * NO;                       // [NI] GCL flux of J xi_k/t
    double* mt0 = gt + NI;                                  // [TY][TX + 6] J xi_1/t on the rows
    double* mt1 = mt0 + T::NM0;                             // [TY + 6][TX] J xi_2/t on the columns
    R* nr = reinterpret_cast<R*>(mt1 + T::NM1);             // [NF + 3][NN] node data, both metric rows
    R* pf = nr + (Y::NF + 3) * NN;                          // [NC][NP] pair fluxes
    R* cm = pf + NC * NP;                                   // [NS + 1][NI] centre-pair means
    R* fl = cm + (NS + 1) * NI;                             // [NC][NI] interface fluxes

    for (int wi = blockIdx.x; wi < L.nwork; wi += gridDim.x) {
        const int2 it = L.work[wi];
        const Inst& I = L.insts[it.x];
        const StagePtrs P = L.ptrs ? L.ptrs[it.x] : L.single;
        const int n0 = I.n[0], n1 = I.n[1];
        const int ntx = (n0 + TX - 1) / TX;
        const int i0 = (it.y % ntx) * TX, j0 = (it.y / ntx) * TY;
        const long long ncell = I.ncell;
        // stage metrics M + s Md with s = mcoef dt (the stage mesh is x^n + s xdot)
        const double sM = L.mcoef != 0.0 ? L.mcoef * *P.dt : 0.0;

        // ---------------- phase 1: node states, entropy variables, both metric rows ----------------
        for (int t = threadIdx.x; t < NN; t += blockDim.x) {
            const int ii = t % RW, jj = t / RW;
            const int i = i0 - 3 + ii, j = j0 - 3 + jj;
            // row nodes serve direction 1, column nodes direction 2; a node neither reads is
            // never read (the corners, and nodes past the last ghost layer or output line)
            const bool use0 = jj >= 3 && jj < TY + 3 && j < n1 && i <= n0 + 2;
            const bool use1 = ii >= 3 && ii < TX + 3 && i < n0 && j <= n1 + 2;
            if (!use0 && !use1) continue;
            // a used node lies outside the domain in one direction at most: the boundary map of
            // that direction (x for a node left or right of it, else y, the identity inside)
            const int k = (i < 0 || i >= n0) ? 0 : 1;
            R U[MAXC];
            {
                int gi, side;
                const int tmap = map_line(I, k, k == 0 ? i : j, gi, side);
                if (tmap == 2) {
                    for (int q = 0; q < NC; ++q) U[q] = to_r<R>(I.inflow[k][side][q]);
                } else {
                    const long long id = k == 0 ? lin(I, gi, j, 0) : lin(I, i, gi, 0);
                    const R inv = Ar<R>::rcp(to_r<R>(P.J[id]));
#pragma unroll
                    for (int q = 0; q < NC; ++q) U[q] = to_r<R>(P.JU[q * ncell + id]) * inv;
                    if (tmap == 1) U[NS + k] = -U[NS + k];
                }
            }
            node_fields<2, NS, R>(I, U, nr, NN, t, L.status);
            // the stage update of x at an output node needs no residual: it runs here, where
            // the FP64 pipe is idle, instead of in the FP64-bound epilogue.  With xdot constant
            // over the step the Shu-Osher combination of the mesh is x^n + xc dt xdot
            if (L.mode == MODE_RK && P.xo && use0 && use1) {
                const long long id = lin(I, i, j, 0);
                const double cdt = L.xc * *P.dt;
#pragma unroll
                for (int c = 0; c < 2; ++c) P.xo[c * ncell + id] = fma(cdt, P.xdot[c * ncell + id], P.x0[c * ncell + id]);
            }
            const long long pid = plin(I, i, j, 0);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                if (!(kk == 0 ? use0 : use1)) continue;
                const long long mrow = (long long)(kk * 3) * I.npad + pid;
                double mv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) mv[c] = P.M[mrow + c * I.npad];
                if (sM != 0.0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) mv[c] = fma(sM, P.Md[mrow + c * I.npad], mv[c]);
                }
                if (kk == 0) mt0[(jj - 3) * RW + ii] = mv[0];
                else mt1[jj * TX + (ii - 3)] = mv[0];
                const int mr = kk == 0 ? Y::MR : Y::NF;
#pragma unroll
                for (int c = 0; c < 3; ++c) nr[(mr + c) * NN + t] = to_r<R>(mv[c]);
            }
        }
        __syncthreads();

        // ---------------- direction 1: pairs, interfaces ----------------
        flux2d_pairs<NS, R, TX, TY, WK>(0, I, i0, j0, nr, pf, cm);
        __syncthreads();
        flux2d_ifaces<NS, R, TX, TY, WK>(0, I, i0, j0, nr, mt0, pf, cm, fl, gt);
        __syncthreads();

        // ---------------- divergence of direction 1; direction 2: pairs, interfaces ----------------
        flux2d_div1<NS, R, TX, TY>(I, i0, j0, fl, gt, acc);
        flux2d_pairs<NS, R, TX, TY, WK>(1, I, i0, j0, nr, pf, cm);
        __syncthreads();
        flux2d_ifaces<NS, R, TX, TY, WK>(1, I, i0, j0, nr, mt1, pf, cm, fl, gt);
        __syncthreads();

        // ---------------- divergence of direction 2 and output ----------------
        const double dt = L.mode == MODE_RK ? *P.dt : 0.0;
        for (int t = threadIdx.x; t < NO; t += blockDim.x) {
            const int il = t % TX, jl = t / TX;
            if (i0 + il >= n0 || j0 + jl >= n1) continue;
            const long long id = lin(I, i0 + il, j0 + jl, 0);
            double r[NC + 1];
            node_div<NC, R>(I, fl, NI, gt, t + TX, t, I.inv_dxi[1], r);
            if (L.mode == MODE_RK) {
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    P.JUo[q * ncell + id] = rk_stage(L, P.JU[q * ncell + id], P.JU0 + q * ncell + id, dt, acc[q * NO + t] + r[q]);
                P.Jo[id] = rk_stage(L, P.J[id], P.J0 + id, dt, acc[NC * NO + t] + r[NC]);
            } else {
#pragma unroll
                for (int q = 0; q < NC; ++q) P.accU[q * ncell + id] = acc[q * NO + t] + r[q];
                P.accJ[id] = acc[NC * NO + t] + r[NC];
            }
        }
        __syncthreads();
    }
}

// one case per fused tile shape of the table in es_kernels.cuh
#define ES_FLUX2D_SHAPES(X) X(0) X(1) X(2) X(3) X(4)
static_assert(NFSHAPE == 5, "ES_FLUX2D_SHAPES lists every fused tile shape");

template <int NS, typename R, int WK>
void prepare_flux2d()
{
#define ES_PREP2(SH)                                                                                        \
    cudaFuncSetAttribute(flux2d_kernel<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH], WK>,                             \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_flux2d<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH]>());
    ES_FLUX2D_SHAPES(ES_PREP2)
#undef ES_PREP2
}

template <int NS, typename R, int WK>
int flux2d_blocks_per_sm(int shape)
{
    int nb = 0;
#define ES_OCC2(SH)                                                                                            \
    if (shape == SH)                                                                                           \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flux2d_kernel<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH], WK>, \
                                                      FLUX_TPB, smem_flux2d<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH]>());
    ES_FLUX2D_SHAPES(ES_OCC2)
#undef ES_OCC2
    return nb > 0 ? nb : 1;
}

template <int NS, typename R, int WK>
void launch_flux2d(const FluxLaunch& L, int shape, int grid, cudaStream_t st)
{
#define ES_LAUNCH2(SH)                                                                                        \
    if (shape == SH)                                                                                          \
        pdl_launch(flux2d_kernel<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH], WK>, grid, FLUX_TPB,                    \
                   smem_flux2d<NS, R, FSHAPE_TX[SH], FSHAPE_TY[SH]>(), st, L);
    ES_FLUX2D_SHAPES(ES_LAUNCH2)
#undef ES_LAUNCH2
}

// explicit instantiation of one (species, reconstruction) case in both compute types
#define ES_FLUX2D_INSTANTIATE(NS, WK)                                                      \
    template void prepare_flux2d<NS, double, WK>();                                        \
    template void prepare_flux2d<NS, float, WK>();                                         \
    template int flux2d_blocks_per_sm<NS, double, WK>(int);                                \
    template int flux2d_blocks_per_sm<NS, float, WK>(int);                                 \
    template void launch_flux2d<NS, double, WK>(const FluxLaunch&, int, int, cudaStream_t); \
    template void launch_flux2d<NS, float, WK>(const FluxLaunch&, int, int, cudaStream_t);

}  // namespace es
