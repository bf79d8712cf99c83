// Kernel declarations and launch shapes shared by the library's translation units.
#pragma once

#include "es_common.cuh"

namespace es {

// flux tile shapes: S nodes along the line x WT neighbouring lines, (S + 1) WT <= 256
// interfaces (one thread each), (S + 6) WT staged nodes and (3S + 6) WT distinct node pairs.
// The autotuner picks one shape (and a persistent grid size) per direction.
constexpr int FLUX_TPB = 256;
constexpr int NSHAPE = 6;
constexpr int SHAPE_S[NSHAPE] = { 62, 58, 122, 30, 26, 14 };
constexpr int SHAPE_WT[NSHAPE] = { 4, 4, 2, 8, 8, 16 };
constexpr int SHAPE_DEFAULT_K0 = 0;    // direction 1: 62 nodes along the line x 4 lines
constexpr int SHAPE_DEFAULT_KN = 3;    // directions 2, 3: 30 nodes x 8 neighbouring lines (coalesced)
// fused 2D stage tiles (both directions in one launch): TX x TY output nodes, at most 256
// interfaces per direction; the autotuner picks one shape, or the per-direction launches
constexpr int NFSHAPE = 5;
constexpr int FSHAPE_TX[NFSHAPE] = { 16, 12, 14, 24, 20 };
constexpr int FSHAPE_TY[NFSHAPE] = { 12, 16, 14, 8, 10 };
constexpr int NODE_TPB = 256;

// launch with programmatic stream serialization (the kernel must begin with pdl_entry())
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

enum { MODE_WRITE = 0, MODE_ACC = 1, MODE_RK = 2 };

struct FluxLaunch {
    const Inst* insts;
    StagePtrs single;         // pointers of a single-instance call
    const StagePtrs* ptrs;    // per-instance table of a batched call (or null)
    const int2* work;
    int nwork;
    int k;             // direction (per-direction kernel)
    int mode;          // MODE_*
    double a, b;       // Shu-Osher coefficients of the stage (MODE_RK)
    double mcoef;      // 2D: the stage metrics are M + mcoef dt Md (0: M alone)
    double xc;         // MODE_RK: the stage's output mesh is x^n + xc dt xdot (xdot constant over the step)
    int* status;
};

// 2D metrics; dot = true also forms the metrics of the mesh velocity into Md; vcl = false
// stores the spatial rows only
void launch_metrics2d(bool dot, int grid, cudaStream_t st, const Inst* insts, const StagePtrs& single,
                      const StagePtrs* table, const int2* work, int nwork, const Scratch* reset, int ninst,
                      bool vcl = true);
__global__ void metrics_reuse_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work,
                                     int nwork, const Scratch* scr, int* flag);
__global__ void xe_fill_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                               const Scratch* scr, int reset_n, const int* reuse, int pad);
__global__ void dx3d_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                            const Scratch* scr, const int* reuse, int pad);
__global__ void metrics3d_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork,
                                 const Scratch* scr, int* flag, int consult, int vcl, int pad);
__global__ void metrics3d_ghost_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work,
                                       int nwork, const int* flag, int consult, int vcl);
__global__ void conversion_check_kernel(const double* in, int n, float* o32, double* o64);
__global__ void half_sum_check_kernel(const float* a, const float* b, int n, double* out);
__global__ void logmean_small_check_kernel(const float* a, const float* b, const float* del, int n, float* fast,
                                           float* general);
__global__ void init_J_kernel(const Inst* insts, StagePtrs single, const StagePtrs* table, const int2* work, int nwork);

// flux + divergence (+ RK stage) for one direction; D dims, NS species, R compute type,
// WK the reconstruction of the dissipation (0 WENO-MR, 1 WENO-JS), tile shape index `shape`
template <int D, int NS, typename R, int WK>
void launch_flux(const FluxLaunch& L, int shape, int grid, cudaStream_t st);
template <int D, int NS, typename R, int WK>
void prepare_flux();
template <int D, int NS, typename R, int WK>
int flux_blocks_per_sm(int shape);

// fused 2D stage (both directions, MODE_RK or MODE_WRITE), fused tile shape index `shape`
template <int NS, typename R, int WK>
void launch_flux2d(const FluxLaunch& L, int shape, int grid, cudaStream_t st);
template <int NS, typename R, int WK>
void prepare_flux2d();
template <int NS, typename R, int WK>
int flux2d_blocks_per_sm(int shape);

}  // namespace es
