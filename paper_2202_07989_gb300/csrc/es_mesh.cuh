// Declarations of the per-step kernels (es_mesh.cu).
#pragma once

#include "es_kernels.cuh"

namespace es {

void launch_cfl_grad(bool mixed, int d, int N, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                     const StagePtrs* table, const int2* work, int nwork, const Scratch* scr);
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
// sweeps in one launch (F < 0: Theta read from the buffer theta_sel)
constexpr int JACOBI_FUSED_MAX = 8, FILTER_FUSED_MAX = 4;
void prepare_mesh();    // kernel attributes, once per context
void launch_jacobi_fused2d(int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                           const StagePtrs* table, const int2* work, int nwork, const Scratch* scr, int H, int F,
                           int theta_sel);
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
