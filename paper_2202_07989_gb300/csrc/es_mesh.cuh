// Declarations of the per-step kernels (es_mesh.cu).
#pragma once

#include "es_kernels.cuh"

namespace es {

// kernels marching along i3 (3D): a block owns a 32 x 8 column of the (i1, i2) plane and stages
// planes of it with a one-node halo
constexpr int M3_TX = NT_X, M3_TY = NT_Y;               // 32 x 8 node columns
constexpr int M3_PX = M3_TX + 2, M3_PY = M3_TY + 2;     // a staged plane: the column and its halo
constexpr int M3_NH = 2 * M3_TX + 2 * M3_TY;            // halo slots of a plane (no corners)
static_assert(M3_TX == 32 && M3_TX * M3_TY == NODE_TPB, "one warp per row of a column");
static_assert(M3_NH <= NODE_TPB, "one halo slot per thread at most");

// The binary32 edge spacings E_k of the mixed 3D Jacobi sweeps (9 components) live on the grid
// extended by one node below in every direction. Rows have a pitch of a multiple of 4 floats
// and node i1 = 0 sits at column 4, so the row segment of a 32 x 8 column starts on a 16-byte
// boundary (16-byte cp.async copies); the buffer carries E3_PAD floats of slack for the
// copies of a ragged column's last row.
constexpr int E3_PAD = 32;
__host__ __device__ inline int e3_pitch(int n0) { return (n0 + 4 + 3) & ~3; }
__host__ __device__ inline long long e3_size(int n0, int n1, int n2)
{
    return 9LL * e3_pitch(n0) * (n1 + 1) * (n2 + 1) + E3_PAD;
}

// the halo slot h of a staged plane (slot coordinates a in [0, M3_PX), b in [0, M3_PY))
__device__ __forceinline__ void m3_halo_slot(int h, int& a, int& b)
{
    if (h < M3_TX) { a = h + 1; b = 0; }
    else if (h < 2 * M3_TX) { a = h - M3_TX + 1; b = M3_PY - 1; }
    else if (h < 2 * M3_TX + M3_TY) { a = 0; b = h - 2 * M3_TX + 1; }
    else { a = M3_PX - 1; b = h - 2 * M3_TX - M3_TY + 1; }
}

template <typename T>
__device__ inline T block_max(T v, T* sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

__device__ inline double block_min_pos(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 1.0;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// binary32 displacement y = x - x^n at a node reached along grid lines: periodic wrap
// (the shift cancels), wall mirror negates the mirrored component
__device__ inline void y_at(const Inst& I, const float* __restrict__ y, int i0, int i1, int i2, float* out)
{
    int i[3] = { i0, i1, i2 };
    bool flip[3] = { false, false, false };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= I.d) break;
        const int n = I.n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        const int side = i[k] < 0 ? 0 : 1;
        if (I.bc[k][side] == BC_PERIODIC) {
            i[k] -= floordiv_(i[k], n) * n;
        } else {
            i[k] = side == 0 ? -1 - i[k] : 2 * n - 1 - i[k];
            flip[k] = true;
        }
    }
    const long long id = lin(I, i[0], i[1], I.d == 3 ? i[2] : 0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= I.d) break;
        const float v = y[j * I.ncell + id];
        out[j] = flip[j] ? -v : v;
    }
}

void launch_cfl_grad(bool mixed, int d, int N, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                     const StagePtrs* table, const int2* work, int nwork, const Scratch* scr);
// mixed form, 3D: Eq. (cfl) and sigma_s one node per thread (work list w_cell), then with monitor
// terms (n_sigma > 0) the monitor gradients marching along i3 (the column items w_col of col3)
void launch_cfl_grad3d(int N, int grid_cell, int grid_col, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                       const StagePtrs* table, const int2* w_cell, int n_cell, const int2* w_col, int n_col,
                       const Scratch* scr, bool monitor);
void launch_xdot(bool mixed, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                 const StagePtrs* table, const int2* work, int nwork, const Scratch* scr);
void launch_xdot_vcl(bool mixed, int d, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                     const StagePtrs* table, const int2* work, int nwork, const Scratch* scr);
void launch_xdot_vel2d(bool mixed, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                       const StagePtrs* table, const int2* work, int nwork, const Scratch* scr);
void launch_monitor_theta(bool mixed, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                          const Scratch* scr);
void launch_filter(bool mixed, bool from_g, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                   const Scratch* scr, int parity);
// mixed form, 2D: the monitor, up to FILTER_FUSED_MAX filter passes and up to JACOBI_FUSED_MAX
// sweeps in one launch (F < 0: Theta read from the buffer theta_sel), over node tiles of one of
// the shapes JF_SHAPES (TX, TY, threads per block) and a work list of those tiles
constexpr int JACOBI_FUSED_MAX = 8, FILTER_FUSED_MAX = 4;
constexpr int NJF_SHAPE = 4;
constexpr int JF_SHAPES[NJF_SHAPE][3] = { { 32, 8, 256 }, { 32, 16, 512 }, { 24, 16, 512 }, { 24, 12, 512 } };
constexpr int JF_SHAPE_DEFAULT = 0;
void prepare_mesh();    // kernel attributes, once per context
void prepare_mesh3d();  // those of es_mesh3d.cu
size_t jacobi_fused2d_smem(int H, int F, int shape);
void launch_jacobi_fused2d(int shape, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                           const StagePtrs* table, const int2* work, int nwork, const Scratch* scr, int H, int F,
                           int theta_sel);
// mixed form, 3D: one filter pass marching along i3 over the column items of col3 (es_mesh3d.cu)
void launch_filter3d(int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork, const Scratch* scr,
                     int parity);
// mixed form, 3D: one Jacobi sweep marching along i3 over the column items of col3 (es_mesh3d.cu)
void launch_jacobi3d(bool first, bool last, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                     const Scratch* scr, int sweep, int theta_sel);
void launch_jacobi(bool mixed, int d, bool last, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                   const StagePtrs* table, const int2* work, int nwork, const Scratch* scr, int sweep, int theta_sel);
__global__ void limiter_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                               const Scratch* scr);
__global__ void schlieren_grad_kernel(const Inst* insts, StagePtrs single, const int2* work, int nwork,
                                      const Scratch* scr);
__global__ void schlieren_phi_kernel(const Inst* insts, StagePtrs single, const int2* work, int nwork,
                                     const Scratch* scr, double psi1, double psi2);
__global__ void entropy_partial_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work,
                                       int nwork, double* partial);
__global__ void entropy_final_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int* first_work,
                                     const double* partial);

}  // namespace es
