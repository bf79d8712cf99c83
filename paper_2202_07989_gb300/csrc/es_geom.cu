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
        acc += alpha3(m) * (a[p] - b[p]);
    }
    return 0.5 * acc;
}

// 2D: J xi_1/x = (delta_2[x_2], -delta_2[x_1]) / dxi_2, J xi_2/x = (-delta_1[x_2], delta_1[x_1]) / dxi_1
__global__ void metrics2d_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                 const int2* __restrict__ work, int nwork)
{
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        int i0, i1, i2;
        if (!tile_node(I, it.y, 3, i0, i1, i2)) continue;
        const long long p = plin(I, i0, i1, 0);
        // delta_1 and delta_2 of both coordinates
        double d1[2] = { 0, 0 }, d2[2] = { 0, 0 };
        const int n0 = I.n[0], n1 = I.n[1];
        if (i0 >= 3 && i0 < n0 - 3 && i1 >= 3 && i1 < n1 - 3) {
            // interior: no ghost node in the stencil
            const double* X0 = S.x;
            const double* X1 = S.x + I.ncell;
            const int c = i1 * n0 + i0;
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                d1[0] += alpha3(m) * (X0[c + m] - X0[c - m]);
                d1[1] += alpha3(m) * (X1[c + m] - X1[c - m]);
                d2[0] += alpha3(m) * (X0[c + m * n0] - X0[c - m * n0]);
                d2[1] += alpha3(m) * (X1[c + m * n0] - X1[c - m * n0]);
            }
        } else {
            double a[2], b[2], cc[2], e[2];
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                x_at<false>(I, S.x, i0 + m, i1, 0, a);
                x_at<false>(I, S.x, i0 - m, i1, 0, b);
                x_at<false>(I, S.x, i0, i1 + m, 0, cc);
                x_at<false>(I, S.x, i0, i1 - m, 0, e);
                d1[0] += alpha3(m) * (a[0] - b[0]);
                d1[1] += alpha3(m) * (a[1] - b[1]);
                d2[0] += alpha3(m) * (cc[0] - e[0]);
                d2[1] += alpha3(m) * (cc[1] - e[1]);
            }
        }
        double m11 = 0.5 * d2[1] * I.inv_dxi[1], m12 = -0.5 * d2[0] * I.inv_dxi[1];
        double m21 = -0.5 * d1[1] * I.inv_dxi[0], m22 = 0.5 * d1[0] * I.inv_dxi[0];
        double xd[2] = { 0, 0 };
        if (S.xdot) x_at<true>(I, S.xdot, i0, i1, 0, xd);
        double* M = S.M;
        long long np = I.npad;
        M[0 * np + p] = -(xd[0] * m11 + xd[1] * m12);
        M[1 * np + p] = m11;
        M[2 * np + p] = m12;
        M[3 * np + p] = -(xd[0] * m21 + xd[1] * m22);
        M[4 * np + p] = m21;
        M[5 * np + p] = m22;
    }
}

// 3D pass 1: D[b][p] = delta_b[x_p] at nodes with 6 ghost layers (extent n + 12)
__global__ void dx3d_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                            const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr)
{
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        long long E0 = I.n[0] + 12, E1 = I.n[1] + 12, E2 = I.n[2] + 12, ne = E0 * E1 * E2;
        int i0, i1, i2;
        if (!tile_node(I, it.y, 6, i0, i1, i2)) continue;
        const long long p = ((long long)(i2 + 6) * E1 + (i1 + 6)) * E0 + (i0 + 6);
        double* D = scr[it.x].D3;
        double acc[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[b][q] = 0.0;
        const bool inner = i0 >= 3 && i0 < I.n[0] - 3 && i1 >= 3 && i1 < I.n[1] - 3 && i2 >= 3 && i2 < I.n[2] - 3;
        const long long ci = inner ? lin(I, i0, i1, i2) : 0;
        const long long st[3] = { 1, I.n[0], (long long)I.n[0] * I.n[1] };
#pragma unroll
        for (int m = 1; m <= 3; ++m) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double u[3], v[3];
                if (inner) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        u[q] = S.x[q * I.ncell + ci + m * st[b]];
                        v[q] = S.x[q * I.ncell + ci - m * st[b]];
                    }
                } else {
                    int ip[3] = { i0, i1, i2 }, im[3] = { i0, i1, i2 };
                    ip[b] += m;
                    im[b] -= m;
                    x_at<false>(I, S.x, ip[0], ip[1], ip[2], u);
                    x_at<false>(I, S.x, im[0], im[1], im[2], v);
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[b][q] += alpha3(m) * (u[q] - v[q]);
            }
        }
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) D[(b * 3 + q) * ne + p] = 0.5 * acc[b][q];
    }
}

// 3D pass 2: J xi_k/x_j = (delta_a[D_b[x_p] x_q] - delta_b[D_a[x_p] x_q]) / (dxi_a dxi_b)
// with (a, b) = (3,2), (1,3), (2,1) for k = 1, 2, 3 and (p, q) = (2,3), (3,1), (1,2)
// for j = 1, 2, 3 (cyclic permutation of Eq. (SCLCoeff)).  Every ordered pair (a, b), a != b,
// belongs to exactly one k, with sign +1 when (a, b) is k's pair and -1 when reversed; the
// kernel walks the outer direction a and offset m once and adds each product term to its k.
__global__ void metrics3d_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                                 const int2* __restrict__ work, int nwork, const Scratch* __restrict__ scr)
{
    // KOF[a][b]: metric row k of the ordered pair (a, b); SGN[a][b]: its sign
    const int KOF[3][3] = { { -1, 2, 1 }, { 2, -1, 0 }, { 1, 0, -1 } };
    const double SGN[3][3] = { { 0.0, -1.0, 1.0 }, { 1.0, 0.0, -1.0 }, { -1.0, 1.0, 0.0 } };
    const int AB[3][2] = { { 2, 1 }, { 0, 2 }, { 1, 0 } };
    const int PQ[3][2] = { { 1, 2 }, { 2, 0 }, { 0, 1 } };
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        int2 it = work[wi];
        const Inst& I = insts[it.x];
        ES_PTRS(S);
        int i0, i1, i2;
        if (!tile_node(I, it.y, 3, i0, i1, i2)) continue;
        const long long p = plin(I, i0, i1, i2);
        const double* D = scr[it.x].D3;
        const long long E0 = I.n[0] + 12, E1 = I.n[1] + 12, ne = E0 * E1 * (I.n[2] + 12);
        const long long e_c = ((long long)(i2 + 6) * E1 + (i1 + 6)) * E0 + (i0 + 6);
        const long long est[3] = { 1, E0, E0 * E1 };
        const bool inner = i0 >= 3 && i0 < I.n[0] - 3 && i1 >= 3 && i1 < I.n[1] - 3 && i2 >= 3 && i2 < I.n[2] - 3;
        const long long ci = inner ? lin(I, i0, i1, i2) : 0;
        const long long st[3] = { 1, I.n[0], (long long)I.n[0] * I.n[1] };
        double t[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) t[k][j] = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int mm = 1; mm <= 3; ++mm) {
                double xp[3], xm[3];
                if (inner) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        xp[q] = S.x[q * I.ncell + ci + mm * st[a]];
                        xm[q] = S.x[q * I.ncell + ci - mm * st[a]];
                    }
                } else {
                    int ip[3] = { i0, i1, i2 }, im[3] = { i0, i1, i2 };
                    ip[a] += mm;
                    im[a] -= mm;
                    x_at<false>(I, S.x, ip[0], ip[1], ip[2], xp);
                    x_at<false>(I, S.x, im[0], im[1], im[2], xm);
                }
                const long long ep = e_c + mm * est[a], em = e_c - mm * est[a];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (b == a) continue;
                    const int k = KOF[a][b];
                    const double sg = SGN[a][b] * alpha3(mm);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int pp = PQ[j][0], q = PQ[j][1];
                        const double* Dbp = D + (long long)(b * 3 + pp) * ne;
                        t[k][j] += sg * (Dbp[ep] * xp[q] - Dbp[em] * xm[q]);
                    }
                }
            }
        }
        double m[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) m[k][j] = 0.5 * t[k][j] * I.inv_dxi[AB[k][0]] * I.inv_dxi[AB[k][1]];
        double xd[3] = { 0, 0, 0 };
        if (S.xdot) x_at<true>(I, S.xdot, i0, i1, i2, xd);
        double* M = S.M;
        long long np = I.npad;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M[(k * 4 + 0) * np + p] = -(xd[0] * m[k][0] + xd[1] * m[k][1] + xd[2] * m[k][2]);
#pragma unroll
            for (int j = 0; j < 3; ++j) M[(k * 4 + 1 + j) * np + p] = m[k][j];
        }
    }
}

// J^0 = det(delta_k[x_j] / dxi_k) at the interior nodes
__global__ void init_J_kernel(const Inst* __restrict__ insts, StagePtrs single, const StagePtrs* __restrict__ table,
                              const int2* __restrict__ work, int nwork)
{
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

}  // namespace es
