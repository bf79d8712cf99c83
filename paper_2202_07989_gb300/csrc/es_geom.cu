// Geometry kernels: SCL-consistent metrics (Sec. 3.2, Eq. (SCLCoeff) and its
// cyclic permutations; the 2D degenerate case), the VCL metric
// J xi_k/t = -sum_j xdot_j J xi_k/x_j (Eq. (VCLCoeff)) and the initial
// Jacobian J^0 = det(delta_k[x_j] / dxi_k).  All FP64.
#include "es_kernels.cuh"

namespace es {

// delta_k[a] = (1/2) sum_m alpha_m (a_{+m} - a_{-m}) of the mesh coordinate p
__device__ inline double delta_x(const Inst& I, const double* __restrict__ x, int i0, int i1, int i2, int k, int p)
{
    double acc = 0.0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        double a[3], b[3];
        int ip[3] = { i0, i1, i2 }, im[3] = { i0, i1, i2 };
        ip[k] += m;
        im[k] -= m;
        x_at<false>(I, x, ip[0], ip[1], ip[2], a);
        x_at<false>(I, x, im[0], im[1], im[2], b);
        acc += I.ecw[m - 1] * (a[p] - b[p]);
    }
    return 0.5 * acc;
}

// 2D: J xi_1/x = (delta_2[x_2], -delta_2[x_1]) / dxi_2, J xi_2/x = (-delta_1[x_2], delta_1[x_1]) / dxi_1
// over the padded node range (3 ghost layers); with DOT also the metrics of the mesh velocity
// xdot into Md (the 2D metrics are linear in x); with `reset`, block 0 also resets the reduction
// slots of the ninst instances (the first kernel of a mesh step); vcl = false leaves the VCL
// rows of M alone (a moving-mesh step, whose velocity pass writes them).  Each block stages x on its tile and on a
// halo of 3 nodes in shared memory (ghost nodes through the boundary maps, once per node),
// then forms both derivatives from shared memory; the coefficients mc = alpha_m / (2 dxi_k)
// fold the scaling into the stencil.
template <bool DOT>
__global__ void __launch_bounds__(NODE_TPB) metrics2d_kernel(const Inst* __restrict__ insts, StagePtrs single,
                                                              const StagePtrs* __restrict__ table,
                                                              const int2* __restrict__ work, int nwork,
                                                              const Scratch* __restrict__ reset, int ninst, bool vcl)
{
    pdl_entry();
    reset_reductions(reset, ninst);
    constexpr int HX = NT_X + 6, HY = NT_Y + 6;
    __shared__ double sx[2][HY][HX];
    __shared__ double sv[DOT ? 2 : 1][DOT ? HY : 1][DOT ? HX : 1];
    const int lx = (int)threadIdx.x % NT_X, ly = (int)threadIdx.x / NT_X;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        const int n0 = I.n[0], n1 = I.n[1];
        const int ntx = (n0 + 6 + NT_X - 1) / NT_X;
        // node of the halo box's first entry: tile origin (pad 3) minus the halo of 3
        const int b0 = (it.y % ntx) * NT_X - 6, b1 = (it.y / ntx) * NT_Y - 6;
        const bool inner = b0 >= 0 && b0 + HX <= n0 && b1 >= 0 && b1 + HY <= n1;
        __syncthreads();
        // at most three halo slots per thread, in one unrolled body so that their loads are
        // issued together
        static_assert(HX * HY <= 3 * NODE_TPB, "three halo slots per thread");
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const int q = (int)threadIdx.x + h * NODE_TPB;
            if (q >= HX * HY) continue;
            const int a = q % HX, b = q / HX;
            const int g0 = b0 + a, g1 = b1 + b;
            double v[2] = { 0.0, 0.0 }, w[2] = { 0.0, 0.0 };
            if (inner) {
                const int c = g1 * n0 + g0;
                v[0] = S.x[c];
                v[1] = S.x[I.ncell + c];
                if (DOT) {
                    w[0] = S.xdot[c];
                    w[1] = S.xdot[I.ncell + c];
                }
            } else if (g0 >= -6 && g0 < n0 + 6 && g1 >= -6 && g1 < n1 + 6) {
                // entries beyond 6 ghost layers feed only nodes outside the padded range
                x_at<false>(I, S.x, g0, g1, 0, v);
                if (DOT) x_at<true>(I, S.xdot, g0, g1, 0, w);
            }
            sx[0][b][a] = v[0];
            sx[1][b][a] = v[1];
            if (DOT) {
                sv[0][b][a] = w[0];
                sv[1][b][a] = w[1];
            }
        }
        __syncthreads();
        const int i0 = b0 + 3 + lx, i1 = b1 + 3 + ly;
        if (i0 >= n0 + 3 || i1 >= n1 + 3) continue;
        const int cx = lx + 3, cy = ly + 3;
        double m[4];
        metrics2d_at<HY, HX>(I, sx, cy, cx, m);
        double xd[2] = { 0.0, 0.0 };
        if (DOT) {
            xd[0] = sv[0][cy][cx];
            xd[1] = sv[1][cy][cx];
        } else if (!S.xdot) {
        } else if (i0 >= 0 && i0 < n0 && i1 >= 0 && i1 < n1) {
            const int c = i1 * n0 + i0;
            xd[0] = S.xdot[c];
            xd[1] = S.xdot[I.ncell + c];
        } else {
            x_at<true>(I, S.xdot, i0, i1, 0, xd);
        }
        const long long np = I.npad, p = plin(I, i0, i1, 0);
        if (vcl) {
            store_metrics2d(S.M, np, p, xd, m);
        } else {
            S.M[1 * np + p] = m[0];
            S.M[2 * np + p] = m[1];
            S.M[4 * np + p] = m[2];
            S.M[5 * np + p] = m[3];
        }
        if (DOT) {
            // metrics of the mesh velocity: the stages of an RK step use M + s dt Md
            double md[4];
            metrics2d_at<DOT ? HY : 1, DOT ? HX : 1>(I, sv, cy, cx, md);
            store_metrics2d(S.Md, np, p, xd, md);
        }
    }
}

void launch_metrics2d(bool dot, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                      const StagePtrs* table, const int2* work, int nwork, const Scratch* reset, int ninst, bool vcl)
{
    if (dot) pdl_launch(metrics2d_kernel<true>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, reset, ninst, true);
    else pdl_launch(metrics2d_kernel<false>, grid, NODE_TPB, 0, st, insts, single, table, work, nwork, reset, ninst, vcl);
}

// Reuse test of the spatial metrics, before the pass that opens a mesh step: they are reused
// when every instance's mesh equals, bit for bit, the positions its metrics buffer M was formed
// from (Xm) and the pass writes M.  After an SSP-RK3 step the new mesh x^n + dt xdot is exactly
// the second stage's mesh, whose metrics the second stage left in M; a fixed mesh never changes.
// The context's flag words: [0] collects mismatches (bit 0) and passes with a nonzero mesh
// velocity (bit 1), [1] counts finished blocks, [2] the outcome (spatial rows kept), [3] set by
// metrics3d_kernel: the VCL rows in M were formed with a zero mesh velocity, [4] the outcome that
// the VCL rows are kept too (kept spatial rows, a zero velocity now and then).  The last block
// stores [2] and [4] and clears [0] and [1] for the next test.
__global__ void metrics_reuse_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                     const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr, int* flag)
{
    pdl_entry();
    int bad = 0, moving = 0;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        const Scratch& Sc = scr[it.x];
        if (S.M != Sc.M || !Sc.Xm) bad = 1;
        if (S.xdot && S.xdot != Sc.zeros) moving = 1;
        int i0, i1, i2;
        if (bad || !tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long c = lin(I, i0, i1, i2);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (!(S.x[q * I.ncell + c] == Sc.Xm[q * I.ncell + c])) bad = 1;
    }
    bad = __syncthreads_or(bad);
    moving = __syncthreads_or(moving);
    if (threadIdx.x == 0) {
        if (bad || moving) atomicOr(&flag[0], (bad ? 1 : 0) | (moving ? 2 : 0));
        __threadfence();
        if (atomicAdd(&flag[1], 1) == (int)gridDim.x - 1) {
            const int v = atomicOr(&flag[0], 0);
            flag[2] = (v & 1) == 0 ? 1 : 0;
            flag[4] = (v == 0 && flag[3] == 1) ? 1 : 0;
            flag[0] = 0;
            flag[1] = 0;
            __threadfence();
        }
    }
}

// 3D pass 0: x on the grid with 9 ghost layers (extent n + 18), filled within `pad` of them (6
// when the nested operators run at the interior nodes only, 9 when they also run on the 3 ghost
// layers of the metrics buffer), every ghost node mapped once (periodic shift, wall mirror), so
// the passes below read positions without branches.  When the pass writes the context's metrics buffer M, the
// interior positions also go to Xm (the positions M's spatial rows are formed from).
__global__ void xe_fill_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                               const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr, int reset_n,
                               const int* reuse, int pad)
{
    pdl_entry();
    reset_reductions(reset_n > 0 ? scr : nullptr, reset_n);
    // kept metrics of a fixed mesh: nothing reads these positions (no sweeps, no new metrics)
    const bool keep = reuse && *reuse;
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        if (keep && I.fixed) continue;
        ES_PTRS(S);
        int i0, i1, i2;
        if (!tile_node(I, it.y, pad, i0, i1, i2)) continue;
        const long long X0 = I.n[0] + 18, X1 = I.n[1] + 18, nx = X0 * X1 * (I.n[2] + 18);
        const long long e = ((long long)(i2 + 9) * X1 + (i1 + 9)) * X0 + (i0 + 9);
        double v[3];
        if (i0 >= 0 && i0 < I.n[0] && i1 >= 0 && i1 < I.n[1] && i2 >= 0 && i2 < I.n[2]) {
            const long long c = lin(I, i0, i1, i2);
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] = S.x[q * I.ncell + c];
            double* Xm = scr[it.x].Xm;
            if (Xm && S.M == scr[it.x].M) {
#pragma unroll
                for (int q = 0; q < 3; ++q) Xm[q * I.ncell + c] = v[q];
            }
        } else {
            x_at<false>(I, S.x, i0, i1, i2, v);
        }
        double* XE = scr[it.x].XE;
#pragma unroll
        for (int q = 0; q < 3; ++q) XE[q * nx + e] = v[q];
    }
}

// 3D pass 1: at the nodes within `pad` ghost layers (3 or 6; stored on the grid with 6 ghost
// layers, extent n + 12), from the ghost-extended positions, the products P[b][j] = delta_b[x_p] x_q for
// (p, q) = (2,3), (3,1), (1,2) (j = 1, 2, 3): every delta_b[x_p] enters Eq. (SCLCoeff) only
// multiplied by x_q at the same node
__global__ void dx3d_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                            const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr, const int* reuse,
                            int pad)
{
    pdl_entry();
    if (reuse && *reuse) return;      // the spatial metrics in M are those of this mesh
    const int PQ[3][2] = { { 1, 2 }, { 2, 0 }, { 0, 1 } };
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        long long E0 = I.n[0] + 12, E1 = I.n[1] + 12, E2 = I.n[2] + 12, ne = E0 * E1 * E2;
        int i0, i1, i2;
        if (!tile_node(I, it.y, pad, i0, i1, i2)) continue;
        const long long p = ((long long)(i2 + 6) * E1 + (i1 + 6)) * E0 + (i0 + 6);
        const long long X0 = I.n[0] + 18, X1 = I.n[1] + 18, nx = X0 * X1 * (I.n[2] + 18);
        const long long xc = ((long long)(i2 + 9) * X1 + (i1 + 9)) * X0 + (i0 + 9);
        const long long xst[3] = { 1, X0, X0 * X1 };
        const double* XE = scr[it.x].XE;
        double* D = scr[it.x].D3;
        // delta_b[x_q] = (1/2) sum_m alpha_m (x_q(+m) - x_q(-m)): the 1/2 folded into the weights
        double acc[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[b][q] = 0.0;
#pragma unroll
        for (int m = 1; m <= 3; ++m) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    acc[b][q] += (0.5 * I.ecw[m - 1]) * (XE[q * nx + xc + m * xst[b]] - XE[q * nx + xc - m * xst[b]]);
            }
        }
        double xq[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) xq[q] = XE[q * nx + xc];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int j = 0; j < 3; ++j) D[(b * 3 + j) * ne + p] = acc[b][PQ[j][0]] * xq[PQ[j][1]];
    }
}

// 3D pass 2: J xi_k/x_j = (delta_a[P_b] - delta_b[P_a]) / (dxi_a dxi_b), P_b = delta_b[x_p] x_q
// with (a, b) = (3,2), (1,3), (2,1) for k = 1, 2, 3 and (p, q) = (2,3), (3,1), (1,2)
// for j = 1, 2, 3 (cyclic permutation of Eq. (SCLCoeff)), at the nodes within `pad` ghost layers
// (0: the ghost layers follow by metrics3d_ghost_kernel; 3: the whole padded buffer).  Every
// ordered pair (a, b), a != b, belongs to
// exactly one k, with sign +1 when (a, b) is k's pair and -1 when reversed; the kernel walks
// the outer direction a and offset m once and adds each product term to its k.
__global__ void metrics3d_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                 const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr, int* flag,
                                 int consult, int vcl, int pad)
{
    pdl_entry();
    const bool keep = consult && flag[2];   // spatial rows of M already formed: the VCL rows only,
    if (keep && (!vcl || flag[4])) return;  // unless the velocity pass writes them or they are kept
    if (blockIdx.x == 0 && threadIdx.x == 0 && nwork > 0) {
        // whether the VCL rows this pass forms in the context's M come from a zero mesh velocity
        const int2 it = work[0];
        ES_PTRS(S);
        if (S.M == scr[it.x].M) flag[3] = (!S.xdot || S.xdot == scr[it.x].zeros) ? 1 : 0;
    }
    // the ordered pair (a, b) belongs to metric row k = 3 - a - b, with sign +1 when b follows a
    // cyclically by two, -1 by one (compile-time constants once the loops unroll)
    const int AB[3][2] = { { 2, 1 }, { 0, 2 }, { 1, 0 } };
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        int i0, i1, i2;
        if (!tile_node(I, it.y, pad, i0, i1, i2)) continue;
        const long long p = plin(I, i0, i1, i2);
        double* M = S.M;
        const long long np = I.npad;
        double xd[3] = { 0, 0, 0 };
        if (S.xdot) x_at<true>(I, S.xdot, i0, i1, i2, xd);
        if (keep) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double m[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) m[j] = M[(k * 4 + 1 + j) * np + p];
                M[(k * 4 + 0) * np + p] = vcl_metric<3>(xd, m);
            }
            continue;
        }
        const double* D = scr[it.x].D3;
        const long long E0 = I.n[0] + 12, E1 = I.n[1] + 12, ne = E0 * E1 * (I.n[2] + 12);
        const long long e_c = ((long long)(i2 + 6) * E1 + (i1 + 6)) * E0 + (i0 + 6);
        const long long est[3] = { 1, E0, E0 * E1 };
        double t[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) t[k][j] = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int mm = 1; mm <= 3; ++mm) {
                const long long ep = e_c + mm * est[a], em = e_c - mm * est[a];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (b == a) continue;
                    const int k = 3 - a - b;
                    const double sg = (b == (a + 2) % 3 ? 1.0 : -1.0) * I.ecw[mm - 1];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const double* Pbj = D + (long long)(b * 3 + j) * ne;   // delta_b[x_p] x_q
                        t[k][j] += sg * (Pbj[ep] - Pbj[em]);
                    }
                }
            }
        }
        double m[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double ck = 0.5 * I.inv_dxi[AB[k][0]] * I.inv_dxi[AB[k][1]];
#pragma unroll
            for (int j = 0; j < 3; ++j) m[k][j] = t[k][j] * ck;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M[(k * 4 + 0) * np + p] = vcl_metric<3>(xd, m[k]);
#pragma unroll
            for (int j = 0; j < 3; ++j) M[(k * 4 + 1 + j) * np + p] = m[k][j];
        }
    }
}

// 3D pass 3: the metrics at the 3 ghost layers of the padded buffer from those of the interior
// node the ghost maps to.  A periodic ghost is the wrapped node shifted by the box length, so
// its metrics are the wrapped node's.  A wall ghost (every non-periodic side) is the half-cell
// mirror of an interior node with the normal coordinate mirrored, x_d -> 2a - x_d: the
// reflections of xi_d and x_d flip the sign of J xi_k/x_j when exactly one of k, j is d, and of
// J xi_k/t (with xdot_d negated) when k is d; a node outside in several directions takes the
// product of the flips.  The values equal the nested operators evaluated at the ghost node from
// the mapped positions, up to the rounding of the shifted or mirrored coordinates.
__global__ void metrics3d_ghost_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                       const int2* __restrict__ work, int nwork, const int* flag, int consult, int vcl)
{
    pdl_entry();
    if (consult && flag[2] && (!vcl || flag[4])) return;    // ghost metrics kept with the interior ones
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        int i[3];
        if (!tile_node(I, it.y, 3, i[0], i[1], i[2])) continue;
        int src[3] = { i[0], i[1], i[2] };
        bool mir[3] = { false, false, false }, ghost = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int n = I.n[d];
            if (i[d] >= 0 && i[d] < n) continue;
            ghost = true;
            const int side = i[d] < 0 ? 0 : 1;
            if (I.bc[d][side] == BC_PERIODIC) {
                src[d] = i[d] - floordiv_(i[d], n) * n;
            } else {
                src[d] = side == 0 ? -1 - i[d] : 2 * n - 1 - i[d];
                mir[d] = true;
            }
        }
        if (!ghost) continue;
        double* M = S.M;
        const long long np = I.npad, p = plin(I, i[0], i[1], i[2]), q = plin(I, src[0], src[1], src[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                bool neg = false;
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (mir[d] && ((k == d) != (c > 0 && c - 1 == d))) neg = !neg;
                const double v = M[(k * 4 + c) * np + q];
                M[(k * 4 + c) * np + p] = neg ? -v : v;
            }
        }
    }
}

// J^0 = det(delta_k[x_j] / dxi_k) at the interior nodes
__global__ void init_J_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                              const int2* __restrict__ work, int nwork)
{
    pdl_entry();
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        int i0, i1, i2;
        if (!tile_node(I, it.y, 0, i0, i1, i2)) continue;
        const long long p = lin(I, i0, i1, i2);
        double A[3][3];
        for (int j = 0; j < I.d; ++j)
            for (int k = 0; k < I.d; ++k) A[j][k] = delta_x(I, S.x, i0, i1, i2, k, j) * I.inv_dxi[k];
        double det;
        if (I.d == 2) det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        else
            det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        S.Jo[p] = det;
    }
}

__global__ void conversion_check_kernel(const double* __restrict__ in, int n, float* __restrict__ o32,
                                        double* __restrict__ o64)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f = f64_to_f32(in[i]);
    o32[i] = f;
    o64[i] = f32_to_f64(f);
}

__global__ void half_sum_check_kernel(const float* __restrict__ a, const float* __restrict__ b, int n,
                                      double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = half_sum_exact(a[i], b[i]);
}

// logmean_small beside the same value by the general conversions and an FP64 add for {a}
__global__ void logmean_small_check_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                           const float* __restrict__ del, int n, float* __restrict__ fast,
                                           float* __restrict__ general)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    fast[i] = logmean_small(a[i], b[i], del[i]);
    const double hs = f32_to_f64(0.5f * a[i]) + f32_to_f64(0.5f * b[i]);
    general[i] = f64_to_f32(fma(-hs, f32_to_f64(del[i]), hs));
}

}  // namespace es
