// Kernel declarations and launch shapes shared by the library's translation units.
#pragma once

#include "es_common.cuh"

namespace es {

// flux tiles of S nodes along the line x WT lines: (3S + 6) WT = 768 distinct node pairs
// (three per thread) and (S + 1) WT <= 256 interfaces
constexpr int FLUX_TPB = 256;
constexpr int S_K0 = 62, WT_K0 = 4;    // direction 1: 62 nodes along the line x 4 lines
constexpr int S_KN = 30, WT_KN = 8;    // directions 2, 3: 30 nodes x 8 neighbouring lines (coalesced)
constexpr int NODE_TPB = 256;

enum { MODE_WRITE = 0, MODE_ACC = 1, MODE_RK = 2 };

struct FluxLaunch {
    const Inst* insts;
    StagePtrs single;         // pointers of a single-instance call
    const StagePtrs* ptrs;    // per-instance table of a batched call (or null)
    const int2* work;
    int nwork;
    int k;             // direction
    int mode;          // MODE_*
    double a, b;       // Shu-Osher coefficients of the stage (MODE_RK)
    int* status;
};

__global__ void metrics2d_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork);
__global__ void dx3d_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                            const Scratch* scr);
__global__ void metrics3d_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                                 const Scratch* scr);
__global__ void conversion_check_kernel(const double* in, int n, float* o32, double* o64);
__global__ void init_J_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork);

// flux + divergence (+ RK stage) for one direction; D dims, NS species, R compute type
template <int D, int NS, typename R>
void launch_flux(const FluxLaunch& L, int grid, cudaStream_t st);
template <int D, int NS, typename R>
void prepare_flux();
template <int D, int NS, typename R>
int flux_blocks_per_sm(int k);

size_t flux_smem_bytes(int D, int NS, bool mixed, int k);

}  // namespace es
