// Flux + divergence kernel of the semi-discrete scheme, one launch per direction k
// (Eqs. (semi_U), (semi_J)), with the SSP-RK3 stage update fused into the last
// direction; the per-node, per-pair and per-interface arithmetic is in es_flux_core.cuh.
//
// Tile: (S + 6) x WT nodes staged in shared memory (3 halo nodes per side along
// k), one thread per interface ((S + 1) x WT = 256), one thread per node in the
// load and store phases (coalesced along the contiguous dimension).
#pragma once

#include "es_flux_core.cuh"

namespace es {

template <int S, int WT>
struct Tile {
    static constexpr int NN = (S + 6) * WT;   // staged nodes (3 halo nodes per side)
    static constexpr int NI = (S + 1) * WT;   // interfaces
    static constexpr int NPL = 3 * S + 6;     // distinct node pairs (j, j+m), m = 1..3, per line
    static constexpr int NP = NPL * WT;
};

// rows of the staging buffer: JU (n_c), J and the metric row of direction k (d + 1); a 2D
// stage's Md rows (metrics M + s dt Md) are read directly in phase 1 (staging them too cost
// the RK launch of the batched form a quarter of its speed)
template <int D, int NS>
__host__ __device__ constexpr int stage_rows() { return NS + 2 * D + 3; }

// whether tiles of this case stage the next tile's inputs (not in 3D, whose tiles run 4 CTAs per SM)
template <int D, int NS>
__host__ __device__ constexpr bool stages_inputs() { return D != 3; }

// byte offset of the staging buffer behind the compute-type arrays of a flux tile (16-byte aligned)
template <int D, int NS, typename R, int S, int WT>
__host__ __device__ constexpr size_t stage_offset()
{
    using Y = Lay<D, NS>;
    using TL = Tile<S, WT>;
    return (sizeof(double) * (TL::NI + TL::NN) +
            sizeof(R) * (Y::NF * TL::NN + Y::NC * TL::NP + (NS + 1) * TL::NI + Y::NC * TL::NI) + 15) / 16 * 16;
}

// asynchronous 8-byte global -> shared copies (cp.async), one group per tile
__device__ __forceinline__ void cp_async8(double* smem, const double* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Issue the raw FP64 node inputs of tile `wi` into the staging buffer stg[stage_rows][NN]:
// JU and J of the node the boundary map of direction k reaches (nothing for an inflow
// ghost, whose state is a constant) and the metric row of direction k at the node.
template <int D, int NS, int S, int WT>
__device__ __forceinline__ void flux_stage(const FluxLaunch& L, int k, int wi, double* stg)
{
    using TL = Tile<S, WT>;
    constexpr int NC = NS + D + 1, NN = TL::NN;
    const int adim = k == 0 ? 1 : 0, bdim = k == 2 ? 1 : 2;
    const int2 it = L.work[wi];
    const Inst& I = L.insts[it.x];
    const double* JU = L.ptrs ? L.ptrs[it.x].JU : L.single.JU;
    const double* J = L.ptrs ? L.ptrs[it.x].J : L.single.J;
    const double* M = L.ptrs ? L.ptrs[it.x].M : L.single.M;
    const int nk = I.n[k], na = I.n[adim];
    const int ns = (nk + S - 1) / S, nat = (na + WT - 1) / WT;
    const int s0 = (it.y % ns) * S, a0 = ((it.y / ns) % nat) * WT, tb = it.y / (ns * nat);
    const long long ncell = I.ncell, np = I.npad;
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
        int s, w;
        if (k == 0) { s = t % (S + 6); w = t / (S + 6); }
        else { w = t % WT; s = t / WT; }
        const int node = w * (S + 6) + s;
        const int g = s0 - 3 + s, a = a0 + w;
        if (a >= na || g > nk + 2) continue;
        int idx[3] = { 0, 0, 0 };
        idx[k] = g;
        idx[adim] = a;
        if (bdim < D) idx[bdim] = tb;
        int gi, side;
        if (map_line(I, k, g, gi, side) != 2) {
            int src[3] = { idx[0], idx[1], idx[2] };
            src[k] = gi;
            const long long id = lin(I, src[0], src[1], src[2]);
#pragma unroll
            for (int q = 0; q < NC; ++q) cp_async8(stg + q * NN + node, JU + q * ncell + id);
            cp_async8(stg + NC * NN + node, J + id);
        }
        const long long pid = plin(I, idx[0], idx[1], idx[2]);
#pragma unroll
        for (int c = 0; c <= D; ++c) cp_async8(stg + (NC + 1 + c) * NN + node, M + (long long)(k * (D + 1) + c) * np + pid);
    }
    cp_async_commit();
}

// Phases of one tile: (1) node states, entropy variables and metrics into shared memory;
// (2) every distinct two-point flux F(U_j, U_{j+m}) (m = 1, 2, 3) of the tile, once; (3)
// per interface the 2w-order EC flux as sum_m alpha_m sum_s of the stored pairs, the GCL
// flux of J xi_k/t and the ES dissipation; (4) divergence and output / RK stage.
// FP32 tiles: 3 CTAs per SM in 2D (<= 85 registers), 4 in 3D (<= 64 registers: the compact 3D
// node layout and no staging buffer leave room for 4, measured 3-10% faster than 3 with the
// staging buffer, spills included); FP64 tiles: 1 (FP64-pipe bound)
template <int D, int NS, typename R, int S, int WT, int WK>
__global__ void __launch_bounds__(FLUX_TPB, (sizeof(R) == 4 ? (D == 3 ? 4 : 3) : 1)) flux_kernel(FluxLaunch L)
{
    pdl_entry();
    using Y = Lay<D, NS>;
    using TL = Tile<S, WT>;
    constexpr int NC = Y::NC, NN = TL::NN, NI = TL::NI, NF = Y::NF, NPL = TL::NPL, NP = TL::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* gt = reinterpret_cast<double*>(smem_raw);           // [NI] GCL flux of J xi_k/t
    double* mt64 = gt + NI;                                      // [NN] J xi_k/t at the nodes
    R* nr = reinterpret_cast<R*>(mt64 + NN);                     // [NF][NN] node data
    R* pf = nr + NF * NN;                                        // [NC][NP] pair fluxes
    R* cm = pf + NC * NP;                                        // [NS + 1][NI] centre-pair means
    R* fl = cm + (NS + 1) * NI;                                  // [NC][NI] interface fluxes
    double* stg = reinterpret_cast<double*>(smem_raw + stage_offset<D, NS, R, S, WT>());   // [NC + D + 2][NN]
    const int k = L.k;
    const int adim = k == 0 ? 1 : 0, bdim = k == 2 ? 1 : 2;

    // When a CTA has several tiles, their node inputs go through the staging buffer: the
    // first tile's now, each later tile's once the previous tile's phase 1 has consumed the
    // buffer, so their loads overlap phases 2-4.  With one tile per CTA there is nothing to
    // overlap, and phase 1 loads directly.
    const bool staged = stages_inputs<D, NS>() && L.nwork > (int)gridDim.x;
    if (staged && blockIdx.x < L.nwork) flux_stage<D, NS, S, WT>(L, k, blockIdx.x, stg);
    for (int wi = blockIdx.x; wi < L.nwork; wi += gridDim.x) {
        const int2 it = L.work[wi];
        const Inst& I = L.insts[it.x];
        const StagePtrs P = L.ptrs ? L.ptrs[it.x] : L.single;
        const int nk = I.n[k], na = I.n[adim];
        const int ns = (nk + S - 1) / S, nat = (na + WT - 1) / WT;
        const int ts = it.y % ns, ta = (it.y / ns) % nat, tb = it.y / (ns * nat);
        const int s0 = ts * S, a0 = ta * WT;
        const long long ncell = I.ncell;
        const double inv_dx = I.inv_dxi[k];
        // 2D stage metrics M + s Md with s = mcoef dt (the stage mesh is x^n + s xdot)
        const double sM = (D == 2 && L.mcoef != 0.0) ? L.mcoef * *P.dt : 0.0;

        // ---------------- phase 1: node states, entropy variables, metrics ----------------
        if (staged) {
            cp_async_wait_all();
            __syncthreads();
        }
        for (int t = threadIdx.x; t < NN; t += blockDim.x) {
            int s, w;
            if (k == 0) { s = t % (S + 6); w = t / (S + 6); }
            else { w = t % WT; s = t / WT; }
            const int node = w * (S + 6) + s;
            const int g = s0 - 3 + s, a = a0 + w;
            if (a >= na || g > nk + 2) {
                for (int f = 0; f < NF; ++f) nr[f * NN + node] = R(1);
                mt64[node] = 0.0;
                continue;
            }
            int idx[3] = { 0, 0, 0 };
            idx[k] = g;
            idx[adim] = a;
            if (bdim < D) idx[bdim] = tb;
            // the conserved point state from the staged JU, J; the boundary map of direction k
            // negates the normal momentum (reflect) or gives the fixed state (inflow)
            R U[MAXC];
            const long long pid = plin(I, idx[0], idx[1], idx[2]);
            {
                int gi, side;
                const int tmap = map_line(I, k, g, gi, side);
                if (tmap == 2) {
                    for (int q = 0; q < NC; ++q) U[q] = to_r<R>(I.inflow[k][side][q]);
                } else {
                    int src[3] = { idx[0], idx[1], idx[2] };
                    src[k] = gi;
                    const long long id = staged ? 0 : lin(I, src[0], src[1], src[2]);
                    const R inv = Ar<R>::rcp(to_r<R>(staged ? stg[NC * NN + node] : P.J[id]));
#pragma unroll
                    for (int q = 0; q < NC; ++q) U[q] = to_r<R>(staged ? stg[q * NN + node] : P.JU[q * ncell + id]) * inv;
                    if (tmap == 1) U[NS + k] = -U[NS + k];
                }
            }
            node_fields<D, NS, R>(I, U, nr, NN, node, L.status);
            // metrics of direction k at this node from the metrics kernel (padded buffer covering
            // g in [-3, n + 3))
            {
                const long long mrow = (long long)(k * (D + 1)) * I.npad + pid;
                double mv[D + 1];
#pragma unroll
                for (int c = 0; c <= D; ++c) mv[c] = staged ? stg[(NC + 1 + c) * NN + node] : P.M[mrow + c * I.npad];
                if (D == 2 && sM != 0.0) {
#pragma unroll
                    for (int c = 0; c <= D; ++c)
                        mv[c] = fma(sM, P.Md[mrow + c * I.npad], mv[c]);
                }
                mt64[node] = mv[0];
                nr[Y::MR * NN + node] = to_r<R>(mv[0]);
#pragma unroll
                for (int j = 0; j < D; ++j) nr[(Y::MR + 1 + j) * NN + node] = to_r<R>(mv[1 + j]);
            }
        }
        __syncthreads();
        if (staged && wi + (int)gridDim.x < L.nwork) flux_stage<D, NS, S, WT>(L, k, wi + (int)gridDim.x, stg);

        // ---------------- phase 2: distinct two-point EC fluxes ----------------
        for (int t = threadIdx.x; t < NP; t += blockDim.x) {
            const int w = t / NPL, r_ = t % NPL;
            int m, Ln;
            if (r_ < S + 1) { m = 1; Ln = r_ + 2; }
            else if (r_ < 2 * S + 3) { m = 2; Ln = r_ - (S + 1) + 1; }
            else { m = 3; Ln = r_ - (2 * S + 3); }
            if (a0 + w >= na || s0 - 3 + Ln + m > nk + 2) continue;
            const int l = w * (S + 6) + Ln;
            pair_flux<D, NS, R>(I, nr, NN, Y::MR, l, l + m, pf, NP, t, cm, NI, m == 1 ? w * (S + 1) + (Ln - 2) : -1);
        }
        __syncthreads();

        // ---------------- phase 3: interface fluxes ----------------
        for (int f = threadIdx.x; f < NI; f += blockDim.x) {
            const int s = f % (S + 1), w = f / (S + 1);
            const int gi = s0 - 1 + s;     // interface gi + 1/2
            if (a0 + w >= na || gi > nk - 1) continue;
            const int base = w * (S + 6) + s;   // node gi - 2
            const int p1 = w * NPL + s, p2 = w * NPL + (S + 1) + s, p3 = w * NPL + (2 * S + 3) + s;
            iface_flux<D, NS, R, WK>(I, nr + base, NN, 1, Y::MR, mt64 + base, 1, pf, NP, p1, p2, p3, 1, cm, NI, f, fl, gt);
        }
        __syncthreads();

        // ---------------- phase 4: divergence and output ----------------
        const double dt = L.mode == MODE_RK ? *P.dt : 0.0;
        for (int t = threadIdx.x; t < S * WT; t += blockDim.x) {
            int s, w;
            if (k == 0) { s = t % S; w = t / S; }
            else { w = t % WT; s = t / WT; }
            const int g = s0 + s, a = a0 + w;
            if (g >= nk || a >= na) continue;
            int idx[3] = { 0, 0, 0 };
            idx[k] = g;
            idx[adim] = a;
            if (bdim < D) idx[bdim] = tb;
            const long long id = lin(I, idx[0], idx[1], idx[2]);
            const int fr = w * (S + 1) + s + 1, fL = fr - 1;
            double r[NC + 1];
            node_div<NC, R>(I, fl, NI, gt, fr, fL, inv_dx, r);
            if (L.mode == MODE_WRITE) {
#pragma unroll
                for (int q = 0; q < NC; ++q) P.accU[q * ncell + id] = r[q];
                P.accJ[id] = r[NC];
            } else if (L.mode == MODE_ACC) {
#pragma unroll
                for (int q = 0; q < NC; ++q) P.accU[q * ncell + id] += r[q];
                P.accJ[id] += r[NC];
            } else {
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    P.JUo[q * ncell + id] = rk_stage(L, P.JU[q * ncell + id], P.JU0 + q * ncell + id, dt, P.accU[q * ncell + id] + r[q]);
                P.Jo[id] = rk_stage(L, P.J[id], P.J0 + id, dt, P.accJ[id] + r[NC]);
                if (P.xo) {    // null on a fixed mesh; xdot is constant over the step: x^n + xc dt xdot
                    const double cdt = L.xc * dt;
#pragma unroll
                    for (int j = 0; j < D; ++j) P.xo[j * ncell + id] = fma(cdt, P.xdot[j * ncell + id], P.x0[j * ncell + id]);
                }
            }
        }
        __syncthreads();
    }
}

template <int D, int NS, typename R, int S, int WT>
static size_t smem_of()
{
    return stage_offset<D, NS, R, S, WT>() + (stages_inputs<D, NS>() ? sizeof(double) * stage_rows<D, NS>() * Tile<S, WT>::NN : 0);
}

// one case per tile shape of the table in es_kernels.cuh
#define ES_FLUX_SHAPES(X) X(0) X(1) X(2) X(3) X(4) X(5)
static_assert(NSHAPE == 6, "ES_FLUX_SHAPES lists every tile shape");

template <int D, int NS, typename R, int WK>
void prepare_flux()
{
#define ES_PREP(SH)                                                                                       \
    cudaFuncSetAttribute(flux_kernel<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH], WK>,                             \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH]>());
    ES_FLUX_SHAPES(ES_PREP)
#undef ES_PREP
}

template <int D, int NS, typename R, int WK>
int flux_blocks_per_sm(int shape)
{
    int nb = 0;
#define ES_OCC(SH)                                                                                           \
    if (shape == SH)                                                                                         \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flux_kernel<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH], WK>, \
                                                      FLUX_TPB, smem_of<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH]>());
    ES_FLUX_SHAPES(ES_OCC)
#undef ES_OCC
    return nb > 0 ? nb : 1;
}

template <int D, int NS, typename R, int WK>
void launch_flux(const FluxLaunch& L, int shape, int grid, cudaStream_t st)
{
    // the staging buffer only when a CTA has several tiles (the kernel's own test)
    const bool staged = stages_inputs<D, NS>() && L.nwork > grid;
#define ES_LAUNCH(SH)                                                                                        \
    if (shape == SH)                                                                                         \
        pdl_launch(flux_kernel<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH], WK>, grid, FLUX_TPB,                       \
                   staged ? smem_of<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH]>() : stage_offset<D, NS, R, SHAPE_S[SH], SHAPE_WT[SH]>(), \
                   st, L);
    ES_FLUX_SHAPES(ES_LAUNCH)
#undef ES_LAUNCH
}

// explicit instantiation of one (dimension, species, reconstruction) case in both compute types
#define ES_FLUX_INSTANTIATE(D, NS, WK)                                                        \
    template void prepare_flux<D, NS, double, WK>();                                          \
    template void prepare_flux<D, NS, float, WK>();                                           \
    template int flux_blocks_per_sm<D, NS, double, WK>(int);                                  \
    template int flux_blocks_per_sm<D, NS, float, WK>(int);                                   \
    template void launch_flux<D, NS, double, WK>(const FluxLaunch&, int, int, cudaStream_t);  \
    template void launch_flux<D, NS, float, WK>(const FluxLaunch&, int, int, cudaStream_t);

}  // namespace es
