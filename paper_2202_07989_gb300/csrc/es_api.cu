// C ABI of the library (include/es.h): contexts, argument checks, work lists and
// the launch sequences of every entry point.  Single-instance calls pass their
// pointers to the kernels by value; batched calls use per-instance tables
// uploaded by es_bind_batch.  Nothing here allocates after creation.
#include "../../include/es.h"
#include "es_mesh.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace es;

struct es_ctx {
    int n_inst = 0, d = 2, N = 1, nc = 4;
    bool mixed = false;
    int weno = 0;             // reconstruction of the dissipation: 0 WENO-MR, 1 WENO-JS
    std::vector<Inst> hI;
    Inst* dI = nullptr;
    std::vector<Scratch> hS;
    Scratch* dS = nullptr;
    std::vector<void*> allocs;
    unsigned long long bytes = 0;
    // work lists (inst, tile)
    int2* w_pad = nullptr;  int n_pad = 0;
    int2* w_ext = nullptr;  int n_ext = 0;
    int2* w_xe = nullptr;   int n_xe = 0;      // 3D FP64 form: nodes within 9 ghost layers
    int2* w_cell = nullptr; int n_cell = 0;
    int2* w_col = nullptr;  int n_col = 0;     // 3D: column chunks of the kernels marching along i3
    int2* w_flux[3][NSHAPE] = {};          // flux work list per direction and tile shape
    int n_flux[3][NSHAPE] = {};
    int2* w_fused[NFSHAPE] = {};           // fused 2D stage work list per fused tile shape
    int n_fused[NFSHAPE] = {};
    int2* w_jf[NJF_SHAPE] = {};            // mixed 2D: fused mesh-step tiles per shape (JF_SHAPES)
    int n_jf[NJF_SHAPE] = {};
    int jf_shape = JF_SHAPE_DEFAULT;
    float jf_ms = 0.f;
    int* d_first_cell = nullptr;
    double* partial = nullptr;
    int* status = nullptr;
    int* mflag = nullptr;     // 3D: reuse test of the metrics (5 words, see metrics_reuse_kernel)
    // stage buffers (per instance): (JU | J | x) for the two intermediate stages
    std::vector<double*> stA, stB;
    // batched tables
    StagePtrs* tab_mesh = nullptr;
    StagePtrs* tab_stage[3] = { nullptr, nullptr, nullptr };
    bool bound = false;
    // device buffers of es_run_host, and its CUDA graph of one step on them (captured on a
    // private stream; rebuilt after a change of tuning or of dt_fixed)
    double *hJU = nullptr, *hJ = nullptr, *hx = nullptr, *hxd = nullptr, *hdt = nullptr, *htacc = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t run_exec = nullptr;
    double run_dtf = 0.0;
    double* tacc_pinned = nullptr;     // mapped pinned host word for the elapsed time (htacc: its device address)
    int sms = 152;
    // flux launch configuration per direction (defaults, or the autotuner's choice)
    int flux_shape[3] = { SHAPE_DEFAULT_K0, SHAPE_DEFAULT_KN, SHAPE_DEFAULT_KN };
    int flux_grid[3] = { 0, 0, 0 };
    float flux_ms[3] = { 0.f, 0.f, 0.f };
    // fused 2D stage launch (-1: one launch per direction)
    int fused_shape = -1;
    int fused_grid = 0;
    float fused_ms = 0.f;
    std::string err;
    // kernel timing (es_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_class;
    size_t ev_used = 0;
    double prof_ms[8] = { 0 };
    long long prof_n[8] = { 0 };
};

namespace {

es_status fail(es_ctx* c, es_status s, const std::string& m)
{
    if (c) c->err = m;
    return s;
}

bool dalloc(es_ctx* c, void** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    c->allocs.push_back(*p);
    c->bytes += bytes;
    return true;
}

es_status cuda_check(es_ctx* c, const char* where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, ES_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return ES_OK;
}

// the step graph of es_run_host bakes in the launch configuration: drop it when that changes
void drop_run_graph(es_ctx* c)
{
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    c->run_exec = nullptr;
}

std::string check_cfg(const es_config& g)
{
    if (g.d != 2 && g.d != 3) return "d must be 2 or 3";
    if (g.N != 1 && g.N != 2) return "N must be 1 or 2";
    if (g.precision != ES_FP64 && g.precision != ES_MIXED) return "precision must be ES_FP64 or ES_MIXED";
    for (int k = 0; k < 3; ++k) {
        if (k < g.d) {
            if (g.n[k] < 10) return "n[k] must be >= 10";
            if (!(g.dxi[k] > 0.0)) return "dxi[k] must be > 0";
            for (int s = 0; s < 2; ++s)
                if (g.bc[k][s] < 0 || g.bc[k][s] > 3) return "bad boundary code";
            if ((g.bc[k][0] == ES_BC_PERIODIC) != (g.bc[k][1] == ES_BC_PERIODIC))
                return "a periodic direction must be periodic on both sides";
        } else if (g.n[k] != 1) {
            return "n[2] must be 1 when d = 2";
        }
    }
    if ((double)g.n[0] * g.n[1] * g.n[2] > 2.0e9) return "grid too large (over 2^31 nodes)";
    for (int l = 0; l < g.N; ++l) {
        if (!(g.gamma[l] > 1.0)) return "gamma must be > 1";
        if (!(g.cv[l] > 0.0)) return "cv must be > 0";
        if (!(g.pinf[l] >= 0.0)) return "pinf must be >= 0";
    }
    if (!(g.chi[0] > 0 && g.chi[1] > 0 && g.chi[2] > 0)) return "chi must be positive";
    if (!(g.weno_eps > 0)) return "weno_eps must be > 0";
    if (!(g.cfl > 0)) return "cfl must be > 0";
    if (g.n_sigma < 0 || g.n_sigma > 4) return "n_sigma must be in 0..4";
    for (int s = 0; s < g.n_sigma; ++s) {
        if (g.sigma[s] < 0 || g.sigma[s] > 5) return "bad monitor variable";
        if (!(g.alpha[s] >= 0)) return "alpha must be >= 0";
        if (g.sigma_op[s] < ES_MON_GRAD2 || g.sigma_op[s] > ES_MON_LAP) return "bad monitor term operator";
    }
    if (g.mu < 0 || g.nf < 0) return "mu and nf must be >= 0";
    if (g.weno != ES_WENO_MR && g.weno != ES_WENO_JS) return "weno must be ES_WENO_MR or ES_WENO_JS";
    if (g.fixed_mesh != 0 && g.fixed_mesh != 1) return "fixed_mesh must be 0 or 1";
    if (g.w < 0 || g.w > 3) return "w must be 1, 2 or 3 (0: 3)";
    if (g.march_planes != 0 && (g.d != 3 || g.march_planes < 4 || g.march_planes > g.n[2]))
        return "march_planes must be 0, or 4..n[2] on a 3D instance";
    return "";
}

Inst make_inst(const es_config& g)
{
    Inst I;
    memset(&I, 0, sizeof(I));
    I.d = g.d;
    I.N = g.N;
    I.nc = g.N + g.d + 1;
    for (int k = 0; k < 3; ++k) {
        I.n[k] = k < g.d ? g.n[k] : 1;
        I.P[k] = k < g.d ? g.n[k] + 6 : 1;
        I.dxi[k] = k < g.d ? g.dxi[k] : 1.0;
        I.inv_dxi[k] = 1.0 / I.dxi[k];
        I.xi_lo[k] = g.xi_lo[k];
        I.L[k] = I.n[k] * I.dxi[k];
        for (int s = 0; s < 2; ++s) {
            I.bc[k][s] = g.bc[k][s];
            for (int q = 0; q < 8; ++q) I.inflow[k][s][q] = g.inflow[k][s][q];
        }
    }
    I.ncell = (long long)I.n[0] * I.n[1] * I.n[2];
    I.npad = (long long)I.P[0] * I.P[1] * I.P[2];
    I.pinf_tot = 0.0;
    for (int l = 0; l < 2; ++l) {
        I.gamma[l] = g.gamma[l];
        I.cv[l] = g.cv[l];
        I.pinf[l] = l < g.N ? g.pinf[l] : 0.0;
        I.Rs[l] = g.cv[l] * (g.gamma[l] - 1.0);
        I.cvG[l] = g.cv[l] * g.gamma[l];
        if (l < g.N) I.pinf_tot += g.pinf[l];
    }
    I.es = g.es;
    for (int q = 0; q < 3; ++q) I.chi[q] = g.chi[q];
    I.weno_eps = g.weno_eps;
    I.cfl = g.cfl;
    I.n_sigma = g.n_sigma;
    for (int s = 0; s < 4; ++s) { I.sigma[s] = g.sigma[s]; I.alpha[s] = g.alpha[s]; I.sigma_op[s] = g.sigma_op[s]; }
    I.mu = g.mu;
    I.nf = g.nf;
    I.weno = g.weno;
    I.fixed = g.fixed_mesh;
    I.w = g.w == 0 ? 3 : g.w;
    if (I.fixed) {
        // no monitor, no sweeps: the mesh step reduces to the CFL time step
        I.n_sigma = 0;
        I.mu = 0;
        I.nf = 0;
    }
    I.ntile_nodes = node_tiles(I, 0);
    for (int l = 0; l < 2; ++l) {
        I.f_gamma[l] = (float)I.gamma[l];
        I.f_cv[l] = (float)I.cv[l];
        I.f_Rs[l] = (float)I.Rs[l];
        I.f_cvG[l] = (float)I.cvG[l];
    }
    I.f_pinf_tot = (float)I.pinf_tot;
    for (int q = 0; q < 3; ++q) I.f_chi[q] = (float)I.chi[q];
    I.f_eps = (float)I.weno_eps;
    for (int q = 0; q < 4; ++q) I.f_alpha[q] = (float)I.alpha[q];
    I.f_ichi3 = (float)(1.0 / I.chi[2]);
    for (int k = 0; k < 3; ++k) {
        I.f_h2[k] = (float)(I.inv_dxi[k] * I.inv_dxi[k]);
        I.f_inv_dxi[k] = (float)I.inv_dxi[k];
        for (int m = 1; m <= 3; ++m) I.mc[k][m - 1] = 0.5 * alpha_w(I.w, m) * I.inv_dxi[k];
    }
    for (int m = 0; m < 3; ++m) {
        I.ecw[m] = alpha_w(I.w, m + 1);
        I.f_ecw[m] = (float)I.ecw[m];
    }
    // GCL stencil weights of node pairs (i-j, i+1+j): (1/2) sum over the pair distances m >= j + 1
    I.gcw[0] = 0.5 * (I.ecw[0] + I.ecw[1] + I.ecw[2]);
    I.gcw[1] = 0.5 * (I.ecw[1] + I.ecw[2]);
    I.gcw[2] = 0.5 * I.ecw[2];
    for (int j = 0; j < 3; ++j) I.f_gcw[j] = (float)I.gcw[j];
    return I;
}

template <typename F>
int2* build_work(es_ctx* c, F count, int& n)
{
    std::vector<int2> w;
    for (int i = 0; i < c->n_inst; ++i) {
        long long t = count(c->hI[i]);
        for (long long j = 0; j < t; ++j) w.push_back(make_int2(i, (int)j));
    }
    n = (int)w.size();
    int2* d = nullptr;
    if (!dalloc(c, (void**)&d, sizeof(int2) * (w.empty() ? 1 : w.size()))) return nullptr;
    if (!w.empty()) cudaMemcpy(d, w.data(), sizeof(int2) * w.size(), cudaMemcpyHostToDevice);
    return d;
}

template <int D, int NS>
void prepare_all(int weno)
{
    if (weno) {
        prepare_flux<D, NS, double, 1>();
        prepare_flux<D, NS, float, 1>();
    } else {
        prepare_flux<D, NS, double, 0>();
        prepare_flux<D, NS, float, 0>();
    }
    if constexpr (D == 2) {
        if (weno) {
            prepare_flux2d<NS, double, 1>();
            prepare_flux2d<NS, float, 1>();
        } else {
            prepare_flux2d<NS, double, 0>();
            prepare_flux2d<NS, float, 0>();
        }
    }
}

// one flux launch in the given tile shape and grid
void flux_launch(es_ctx* c, const FluxLaunch& L, int shape, int grid, cudaStream_t st)
{
    if (grid > L.nwork) grid = L.nwork;
    if (grid <= 0) return;
#define FD(d, n)                                                                                      \
    do {                                                                                              \
        if (c->weno) { if (c->mixed) launch_flux<d, n, float, 1>(L, shape, grid, st); else launch_flux<d, n, double, 1>(L, shape, grid, st); } \
        else { if (c->mixed) launch_flux<d, n, float, 0>(L, shape, grid, st); else launch_flux<d, n, double, 0>(L, shape, grid, st); }        \
    } while (0)
    if (c->d == 2 && c->N == 1) FD(2, 1);
    else if (c->d == 2 && c->N == 2) FD(2, 2);
    else if (c->d == 3 && c->N == 1) FD(3, 1);
    else FD(3, 2);
#undef FD
}

// one fused 2D stage launch in the given fused tile shape and grid
void flux2d_launch(es_ctx* c, const FluxLaunch& L, int shape, int grid, cudaStream_t st)
{
    if (grid > L.nwork) grid = L.nwork;
    if (grid <= 0) return;
#define F2(n)                                                                                         \
    do {                                                                                              \
        if (c->weno) { if (c->mixed) launch_flux2d<n, float, 1>(L, shape, grid, st); else launch_flux2d<n, double, 1>(L, shape, grid, st); } \
        else { if (c->mixed) launch_flux2d<n, float, 0>(L, shape, grid, st); else launch_flux2d<n, double, 0>(L, shape, grid, st); }        \
    } while (0)
    if (c->N == 1) F2(1);
    else F2(2);
#undef F2
}

int flux2d_occ(es_ctx* c, int shape)
{
#define FO2(n)                                                                                                \
    do {                                                                                                      \
        if (c->weno) return c->mixed ? flux2d_blocks_per_sm<n, float, 1>(shape) : flux2d_blocks_per_sm<n, double, 1>(shape); \
        return c->mixed ? flux2d_blocks_per_sm<n, float, 0>(shape) : flux2d_blocks_per_sm<n, double, 0>(shape);            \
    } while (0)
    if (c->N == 1) FO2(1);
    FO2(2);
#undef FO2
}

// fused 2D stage tiles of instance I in fused tile shape `shape`
long long fused_tiles(const Inst& I, int shape)
{
    return (long long)((I.n[0] + FSHAPE_TX[shape] - 1) / FSHAPE_TX[shape]) * ((I.n[1] + FSHAPE_TY[shape] - 1) / FSHAPE_TY[shape]);
}

// flux tiles of instance I along direction k in tile shape `shape`
long long flux_tiles(const Inst& I, int k, int shape)
{
    const int S = SHAPE_S[shape], WT = SHAPE_WT[shape];
    const int adim = k == 0 ? 1 : 0, bdim = k == 2 ? 1 : 2;
    const long long nb = bdim < I.d ? I.n[bdim] : 1;
    return (long long)((I.n[k] + S - 1) / S) * ((I.n[adim] + WT - 1) / WT) * nb;
}

int flux_occ(es_ctx* c, int shape)
{
#define FO(d, n)                                                                                             \
    do {                                                                                                     \
        if (c->weno) return c->mixed ? flux_blocks_per_sm<d, n, float, 1>(shape) : flux_blocks_per_sm<d, n, double, 1>(shape); \
        return c->mixed ? flux_blocks_per_sm<d, n, float, 0>(shape) : flux_blocks_per_sm<d, n, double, 0>(shape);            \
    } while (0)
    if (c->d == 2 && c->N == 1) FO(2, 1);
    if (c->d == 2 && c->N == 2) FO(2, 2);
    if (c->d == 3 && c->N == 1) FO(3, 1);
    FO(3, 2);
#undef FO
}

// planes per chunk of the 3D kernels that march along i3: chunks enough for about four
// waves of 3 CTAs per SM over the instance's columns, at least 4 planes a chunk
int march_zc(const Inst& I, int sms)
{
    const long long cols = (long long)((I.n[0] + NT_X - 1) / NT_X) * ((I.n[1] + NT_Y - 1) / NT_Y);
    long long chunks = (12LL * sms + cols - 1) / cols;
    if (chunks > I.n[2]) chunks = I.n[2];
    const int zc = (int)((I.n[2] + chunks - 1) / chunks);
    return zc >= 4 ? zc : (I.n[2] < 4 ? I.n[2] : 4);
}

int node_grid(es_ctx* c, int nwork)
{
    int cap = c->sms * 8;
    return nwork < cap ? nwork : cap;
}

constexpr int PC_FLUX = 0, PC_METRICS = 3, PC_MESH = 4, PC_ENTROPY = 5, PC_FLUX2D = 6;

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

// event pair around one launch: prof_begin returns the pair index or -1
int prof_begin(es_ctx* c, int cls, cudaStream_t st)
{
    if (!c->prof || c->ev_used + 2 > c->ev.size() || capturing(st)) return -1;
    int i = (int)c->ev_used;
    c->ev_used += 2;
    c->ev_class[i / 2] = cls;
    cudaEventRecord(c->ev[i], st);
    return i;
}

void prof_end(es_ctx* c, int i, cudaStream_t st)
{
    if (i >= 0) cudaEventRecord(c->ev[i + 1], st);
}

struct ProfScope {
    es_ctx* c;
    int i;
    cudaStream_t st;
    ProfScope(es_ctx* c_, int cls, cudaStream_t s) : c(c_), i(prof_begin(c_, cls, s)), st(s) {}
    ~ProfScope() { prof_end(c, i, st); }
};

// metrics of the stage mesh P.x / P.xdot into P.M; reset = true also resets the reduction
// slots (the first kernel of a mesh step); dot = true (2D) also forms the metrics of the mesh
// velocity into P.Md, so the later stages of an RK step need no metrics pass; reuse = true (3D)
// keeps the spatial rows of M when they were formed from this very mesh (the VCL rows are
// formed again when vcl = true, and left to the velocity pass otherwise)
void launch_metrics(es_ctx* c, const StagePtrs& P, const StagePtrs* tab, cudaStream_t st, bool reset = false,
                    bool dot = false, bool vcl = true, bool reuse = false)
{
    ProfScope ps(c, PC_METRICS, st);
    if (c->d == 2) {
        launch_metrics2d(dot, node_grid(c, c->n_pad), st, c->dI, P, tab, c->w_pad, c->n_pad, reset ? c->dS : nullptr,
                         c->n_inst, vcl);
    } else {
        // mixed form: positions within 6 ghost layers, products within 3, the nested operators at
        // the interior nodes, then the metrics of the 3 ghost layers from those of the nodes they
        // map to.  FP64 form: the nested operators at every node of the padded buffer as well
        // (positions within 9 ghost layers, products within 6), the oracle's evaluation order
        // at the ghost nodes too.
        const int* ru = reuse ? c->mflag + 2 : nullptr;
        const bool sym = c->mixed;
        if (reuse)
            pdl_launch(metrics_reuse_kernel, node_grid(c, c->n_cell), NODE_TPB, 0, st, c->dI, P, tab, c->w_cell, c->n_cell,
                       c->dS, c->mflag);
        if (sym) {
            pdl_launch(xe_fill_kernel, node_grid(c, c->n_ext), NODE_TPB, 0, st, c->dI, P, tab, c->w_ext, c->n_ext, c->dS,
                       reset ? c->n_inst : 0, ru, 6);
            pdl_launch(dx3d_kernel, node_grid(c, c->n_pad), NODE_TPB, 0, st, c->dI, P, tab, c->w_pad, c->n_pad, c->dS, ru, 3);
            pdl_launch(metrics3d_kernel, node_grid(c, c->n_cell), NODE_TPB, 0, st, c->dI, P, tab, c->w_cell, c->n_cell,
                       c->dS, c->mflag, reuse ? 1 : 0, vcl ? 1 : 0, 0);
            // kept metrics keep their ghost layers unless the VCL rows are formed again
            pdl_launch(metrics3d_ghost_kernel, node_grid(c, c->n_pad), NODE_TPB, 0, st, c->dI, P, tab, c->w_pad, c->n_pad,
                       c->mflag, reuse ? 1 : 0, vcl ? 1 : 0);
        } else {
            pdl_launch(xe_fill_kernel, node_grid(c, c->n_xe), NODE_TPB, 0, st, c->dI, P, tab, c->w_xe, c->n_xe, c->dS,
                       reset ? c->n_inst : 0, ru, 9);
            pdl_launch(dx3d_kernel, node_grid(c, c->n_ext), NODE_TPB, 0, st, c->dI, P, tab, c->w_ext, c->n_ext, c->dS, ru, 6);
            pdl_launch(metrics3d_kernel, node_grid(c, c->n_pad), NODE_TPB, 0, st, c->dI, P, tab, c->w_pad, c->n_pad,
                       c->dS, c->mflag, reuse ? 1 : 0, vcl ? 1 : 0, 3);
        }
    }
}

// residual of one stage: metrics, then one flux launch per direction (or, in 2D, the
// fused stage launch when the context uses it).  With rk = true the last direction applies
// the Shu-Osher stage (a, b); metrics = false when M already holds the metrics of the stage;
// mcoef != 0 (2D) makes the stage metrics M + mcoef dt Md, the metrics of x^n + mcoef dt
// xdot; dot = true (2D) forms Md with M.
void launch_residual(es_ctx* c, const StagePtrs& P, const StagePtrs* tab, bool rk, double a, double b, cudaStream_t st,
                     bool metrics = true, double mcoef = 0.0, bool dot = false, double xc = 0.0)
{
    if (metrics) launch_metrics(c, P, tab, st, false, dot);
    if (c->d == 2 && c->fused_shape >= 0) {
        FluxLaunch L;
        L.insts = c->dI;
        L.single = P;
        L.ptrs = tab;
        L.work = c->w_fused[c->fused_shape];
        L.nwork = c->n_fused[c->fused_shape];
        L.k = 0;
        L.mode = rk ? MODE_RK : MODE_WRITE;
        L.a = a;
        L.b = b;
        L.mcoef = mcoef;
        L.xc = xc;
        L.status = c->status;
        ProfScope ps(c, PC_FLUX2D, st);
        flux2d_launch(c, L, c->fused_shape, c->fused_grid, st);
        return;
    }
    for (int k = 0; k < c->d; ++k) {
        FluxLaunch L;
        L.insts = c->dI;
        L.single = P;
        L.ptrs = tab;
        const int sh = c->flux_shape[k];
        L.work = c->w_flux[k][sh];
        L.nwork = c->n_flux[k][sh];
        L.k = k;
        L.mode = k == 0 ? MODE_WRITE : MODE_ACC;
        if (rk && k == c->d - 1) L.mode = MODE_RK;
        L.a = a;
        L.b = b;
        L.mcoef = mcoef;
        L.xc = xc;
        L.status = c->status;
        ProfScope ps(c, PC_FLUX + k, st);
        flux_launch(c, L, sh, c->flux_grid[k], st);
    }
}

// the stage pointer sets of one SSP-RK3 step on (JU, J, x)
void stage_ptrs(es_ctx* c, int i, double* JU, double* J, double* x, const double* xdot, const double* dt, StagePtrs out[3])
{
    const Inst& I = c->hI[i];
    const Scratch& S = c->hS[i];
    long long n = I.ncell;
    double* A = c->stA[i];
    double* B = c->stB[i];
    double* Au = A;
    double* Aj = A + I.nc * n;
    double* Ax = Aj + n;
    double* Bu = B;
    double* Bj = B + I.nc * n;
    double* Bx = Bj + n;
    const double* in_u[3] = { JU, Au, Bu };
    const double* in_j[3] = { J, Aj, Bj };
    const bool fixed = I.fixed != 0;
    const double* in_x[3] = { x, fixed ? x : Ax, fixed ? x : Bx };
    double* out_u[3] = { Au, Bu, JU };
    double* out_j[3] = { Aj, Bj, J };
    // a fixed mesh is never rewritten (no x update in the RK stages)
    double* out_x[3] = { fixed ? nullptr : Ax, fixed ? nullptr : Bx, fixed ? nullptr : x };
    for (int s = 0; s < 3; ++s) {
        StagePtrs P;
        memset(&P, 0, sizeof(P));
        P.JU = in_u[s];
        P.J = in_j[s];
        P.x = in_x[s];
        P.xdot = (xdot && !fixed) ? xdot : S.zeros;
        // a 3D moving mesh keeps the second stage's metrics (those of x^n + dt xdot, the next
        // step's mesh) in M and forms the third stage's in M3
        P.M = (s == 2 && S.M3) ? S.M3 : S.M;
        P.Md = S.Md;
        P.accU = S.accU;
        P.accJ = S.accJ;
        P.JU0 = JU;
        P.J0 = J;
        P.x0 = x;
        P.JUo = out_u[s];
        P.Jo = out_j[s];
        P.xo = out_x[s];
        P.dt = dt;
        out[s] = P;
    }
}

const double RK_A[3] = { 0.0, 0.75, 1.0 / 3.0 };
const double RK_B[3] = { 1.0, 0.25, 2.0 / 3.0 };
// the stage meshes of SSP-RK3 with xdot constant: x^n, x^n + dt xdot, x^n + dt xdot / 2 (the
// input of stage s), and the stage outputs x^n + dt xdot, x^n + dt xdot / 2, x^n + dt xdot
const double MCOEF[3] = { 0.0, 1.0, 0.5 };
const double XCOEF[3] = { 1.0, 0.5, 1.0 };

// 2D moving meshes form the stage metrics as M(x^n) + s dt M(xdot) (the metrics are linear in x)
bool linear_stage_metrics(const es_ctx* c) { return c->d == 2 && !c->hI[0].fixed; }

// whether the mesh step runs the fused 2D launch (monitor, filter passes and sweeps)
bool fused_mesh2d(const es_ctx* c)
{
    const Inst& I = c->hI[0];
    return c->mixed && c->d == 2 && !I.fixed && I.mu >= 1 && I.mu <= JACOBI_FUSED_MAX && I.nf <= FILTER_FUSED_MAX;
}

// mesh redistribution (Sec. 4): the metrics of x^n (Eq. (cfl) and the monitor need them),
// Delta t and the monitor gradients, the filter passes, the Jacobi sweeps with the limiter,
// and the mesh velocity.  With step = true (a full time step follows) the velocity pass
// also stores the VCL metrics of the first RK stage in M.
void launch_mesh(es_ctx* c, const StagePtrs& P, const StagePtrs* tab, cudaStream_t st, bool step = false)
{
    StagePtrs Q = P;
    Q.xdot = nullptr;
    Q.M = c->hS[0].M;
    // also resets the reduction slots; the VCL rows (xdot = 0 here) matter only on a fixed mesh,
    // whose stages use these metrics: a moving-mesh step's velocity pass writes them
    launch_metrics(c, Q, tab, st, true, false, c->hI[0].fixed != 0, true);
    ProfScope ps(c, PC_MESH, st);
    int gc = node_grid(c, c->n_cell);
    if (c->mixed && c->d == 3)
        launch_cfl_grad3d(c->N, gc, node_grid(c, c->n_col), st, c->dI, P, tab, c->w_cell, c->n_cell, c->w_col, c->n_col,
                          c->dS, c->hI[0].n_sigma > 0 || c->n_inst > 1);
    else launch_cfl_grad(c->mixed, c->d, c->N, gc, st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS);
    if (c->hI[0].fixed) {
        // fixed mesh: Delta t only; xdot = 0 (the metrics above carry no VCL part)
        launch_xdot(c->mixed, gc, st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS);
        return;
    }
    int nf = c->hI[0].nf, mu = c->hI[0].mu;
    int th_sel = nf % 2;
    if (fused_mesh2d(c)) {
        // monitor, filter passes and sweeps in one launch
        const int js = c->jf_shape;
        launch_jacobi_fused2d(js, node_grid(c, c->n_jf[js]), st, c->dI, P, tab, c->w_jf[js], c->n_jf[js], c->dS, mu, nf,
                              th_sel);
    } else {
        // Theta once per node, then plain filter passes (forming it inside the first pass costs
        // 3^d evaluations per node)
        launch_monitor_theta(c->mixed, gc, st, c->dI, c->w_cell, c->n_cell, c->dS);
        for (int f = 0; f < nf; ++f) {
            if (c->mixed && c->d == 3) launch_filter3d(node_grid(c, c->n_col), st, c->dI, c->w_col, c->n_col, c->dS, f % 2);
            else launch_filter(c->mixed, false, gc, st, c->dI, c->w_cell, c->n_cell, c->dS, f % 2);
        }
        for (int s = 0; s < mu; ++s) {
            if (c->mixed && c->d == 3)
                launch_jacobi3d(s == 0, s == mu - 1, node_grid(c, c->n_col), st, c->dI, c->w_col, c->n_col, c->dS, s,
                                th_sel);
            else
                launch_jacobi(c->mixed, c->d, s == mu - 1, gc, st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS, s, th_sel);
        }
    }
    if (mu == 0) pdl_launch(limiter_kernel, gc, NODE_TPB, 0, st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS);
    if (step && c->d == 2) launch_xdot_vel2d(c->mixed, node_grid(c, c->n_pad), st, c->dI, P, tab, c->w_pad, c->n_pad, c->dS);
    else if (step) launch_xdot_vcl(c->mixed, c->d, node_grid(c, c->n_pad), st, c->dI, P, tab, c->w_pad, c->n_pad, c->dS);
    else launch_xdot(c->mixed, gc, st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS);
}

// one full time step: mesh redistribution, then the three SSP-RK3 stages; the first
// stage reuses the metrics the mesh step formed
void launch_step(es_ctx* c, const StagePtrs& mesh, const StagePtrs* tab_mesh, const StagePtrs stage[3],
                 StagePtrs* const tab_stage[3], cudaStream_t st)
{
    launch_mesh(c, mesh, tab_mesh, st, true);
    // the first stage reuses the metrics of x^n; on a fixed mesh every stage does; in 2D the
    // velocity pass also formed M(xdot), so no stage forms metrics
    const bool fixed = c->hI[0].fixed != 0, lin = linear_stage_metrics(c);
    for (int s = 0; s < 3; ++s)
        launch_residual(c, stage[s], tab_stage[s], true, RK_A[s], RK_B[s], st, s > 0 && !fixed && !lin,
                        lin ? MCOEF[s] : 0.0, false, XCOEF[s]);
}

__global__ void time_acc_kernel(double* t, const double* dt_dtau) { *t += dt_dtau[0]; }

// copies of (JU, J, x) between the caller's host buffers and the context's device buffers,
// which are consecutive in one allocation: one transfer each way when the host buffers are
// consecutive too, else one per buffer (one SM-driven copy kernel over mapped pinned memory
// measured no faster than these)
void copy_state(es_ctx* c, double* JU, double* J, double* x, bool to_device, cudaStream_t st)
{
    const Inst& I = c->hI[0];
    const long long n = I.ncell;
    if (J == JU + I.nc * n && x == J + n) {
        const size_t bytes = sizeof(double) * (I.nc + 1 + I.d) * n;
        cudaMemcpyAsync(to_device ? c->hJU : JU, to_device ? JU : c->hJU, bytes,
                        to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
        return;
    }
    double* host[3] = { JU, J, x };
    double* dev[3] = { c->hJU, c->hJ, c->hx };
    const long long cnt[3] = { I.nc * n, n, I.d * n };
    for (int k = 0; k < 3; ++k)
        cudaMemcpyAsync(to_device ? dev[k] : host[k], to_device ? host[k] : dev[k], sizeof(double) * cnt[k],
                        to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
}

}  // namespace

extern "C" {

es_status es_create_batch(const es_config* cfgs, int n_inst, es_ctx** out)
{
    if (!out) return ES_ERR_ARG;
    *out = nullptr;
    if (!cfgs || n_inst <= 0) return ES_ERR_ARG;
    for (int i = 0; i < n_inst; ++i) {
        std::string m = check_cfg(cfgs[i]);
        if (!m.empty()) {
            fprintf(stderr, "es_create: instance %d: %s\n", i, m.c_str());
            return ES_ERR_ARG;
        }
        if (cfgs[i].d != cfgs[0].d || cfgs[i].N != cfgs[0].N || cfgs[i].precision != cfgs[0].precision ||
            cfgs[i].mu != cfgs[0].mu || cfgs[i].nf != cfgs[0].nf || cfgs[i].fixed_mesh != cfgs[0].fixed_mesh ||
            cfgs[i].weno != cfgs[0].weno) {
            fprintf(stderr, "es_create: instances of a batch must share d, N, precision, mu, nf, fixed_mesh and weno\n");
            return ES_ERR_UNSUPPORTED;
        }
    }
    es_ctx* c = new es_ctx();
    c->n_inst = n_inst;
    c->d = cfgs[0].d;
    c->N = cfgs[0].N;
    c->nc = c->N + c->d + 1;
    c->mixed = cfgs[0].precision == ES_MIXED;
    c->weno = cfgs[0].weno;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < n_inst; ++i) c->hI.push_back(make_inst(cfgs[i]));
    for (int i = 0; i < n_inst; ++i) {
        Inst& I = c->hI[i];
        I.zc = I.d == 3 ? (cfgs[i].march_planes > 0 ? cfgs[i].march_planes : march_zc(I, c->sms)) : 1;
    }
    bool ok = true;
    ok = ok && dalloc(c, (void**)&c->dI, sizeof(Inst) * n_inst);
    size_t rsz = c->mixed ? sizeof(float) : sizeof(double);
    for (int i = 0; i < n_inst && ok; ++i) {
        const Inst& I = c->hI[i];
        Scratch S;
        memset(&S, 0, sizeof(S));
        long long n = I.ncell;
        ok = ok && dalloc(c, (void**)&S.M, sizeof(double) * I.d * (I.d + 1) * I.npad);
        if (I.d == 2) ok = ok && dalloc(c, (void**)&S.Md, sizeof(double) * 6 * I.npad);
        if (I.d == 3) {
            long long ne = (long long)(I.n[0] + 12) * (I.n[1] + 12) * (I.n[2] + 12);
            ok = ok && dalloc(c, (void**)&S.D3, sizeof(double) * 9 * ne);
            const long long nx = (long long)(I.n[0] + 18) * (I.n[1] + 18) * (I.n[2] + 18);
            ok = ok && dalloc(c, (void**)&S.XE, sizeof(double) * 3 * nx);
            if (!I.fixed) ok = ok && dalloc(c, (void**)&S.M3, sizeof(double) * 12 * I.npad);
            ok = ok && dalloc(c, (void**)&S.Xm, sizeof(double) * 3 * n);
            if (ok) cudaMemset(S.Xm, 0xff, sizeof(double) * 3 * n);     // NaN: equal to no position
        }
        ok = ok && dalloc(c, (void**)&S.accU, sizeof(double) * I.nc * n);
        ok = ok && dalloc(c, (void**)&S.accJ, sizeof(double) * n);
        ok = ok && dalloc(c, (void**)&S.red, sizeof(double) * 8);
        ok = ok && dalloc(c, (void**)&S.g, sizeof(double) * (I.n_sigma > 0 ? I.n_sigma : 1) * n);
        ok = ok && dalloc(c, &S.th0, rsz * n);
        ok = ok && dalloc(c, &S.th1, rsz * n);
        ok = ok && dalloc(c, (void**)&S.xa, sizeof(double) * I.d * n);
        ok = ok && dalloc(c, (void**)&S.xb, sizeof(double) * I.d * n);
        if (c->mixed) {
            // 2D: dl_{k+-} per node; 3D: the edge spacings E_k on the grid extended by one node below
            // (es_mesh3d.cu)
            long long nd = 2LL * I.d * I.d * n;
            if (I.d == 3) nd = e3_size(I.n[0], I.n[1], I.n[2]);
            ok = ok && dalloc(c, (void**)&S.dl, sizeof(float) * nd);
        }
        ok = ok && dalloc(c, (void**)&S.zeros, sizeof(double) * I.d * n);
        if (ok) cudaMemset(S.zeros, 0, sizeof(double) * I.d * n);
        double *A = nullptr, *B = nullptr;
        ok = ok && dalloc(c, (void**)&A, sizeof(double) * (I.nc + 1 + I.d) * n);
        ok = ok && dalloc(c, (void**)&B, sizeof(double) * (I.nc + 1 + I.d) * n);
        c->stA.push_back(A);
        c->stB.push_back(B);
        c->hS.push_back(S);
    }
    ok = ok && dalloc(c, (void**)&c->dS, sizeof(Scratch) * n_inst);
    ok = ok && dalloc(c, (void**)&c->status, sizeof(int));
    ok = ok && dalloc(c, (void**)&c->mflag, sizeof(int) * 5);
    if (!ok) {
        es_destroy(c);
        fprintf(stderr, "es_create: device allocation failed\n");
        return ES_ERR_CUDA;
    }
    cudaMemcpy(c->dI, c->hI.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice);
    cudaMemcpy(c->dS, c->hS.data(), sizeof(Scratch) * n_inst, cudaMemcpyHostToDevice);
    cudaMemset(c->status, 0, sizeof(int));
    cudaMemset(c->mflag, 0, sizeof(int) * 5);
    c->w_pad = build_work(c, [](const Inst& I) { return (long long)node_tiles(I, 3); }, c->n_pad);
    c->w_cell = build_work(c, [](const Inst& I) { return (long long)node_tiles(I, 0); }, c->n_cell);
    if (c->d == 3) c->w_ext = build_work(c, [](const Inst& I) { return (long long)node_tiles(I, 6); }, c->n_ext);
    if (c->d == 3) c->w_col = build_work(c, [](const Inst& I) { return (long long)col3_items(I); }, c->n_col);
    if (c->d == 3 && !c->mixed) c->w_xe = build_work(c, [](const Inst& I) { return (long long)node_tiles(I, 9); }, c->n_xe);
    for (int k = 0; k < c->d; ++k)
        for (int sh = 0; sh < NSHAPE; ++sh) {
            c->w_flux[k][sh] = build_work(c, [k, sh](const Inst& I) { return flux_tiles(I, k, sh); }, c->n_flux[k][sh]);
            ok = ok && c->w_flux[k][sh];
        }
    if (c->d == 2)
        for (int sh = 0; sh < NFSHAPE; ++sh) {
            c->w_fused[sh] = build_work(c, [sh](const Inst& I) { return fused_tiles(I, sh); }, c->n_fused[sh]);
            ok = ok && c->w_fused[sh];
        }
    if (c->d == 2 && c->mixed)
        for (int sh = 0; sh < NJF_SHAPE; ++sh) {
            c->w_jf[sh] = build_work(c, [sh](const Inst& I) {
                return (long long)((I.n[0] + JF_SHAPES[sh][0] - 1) / JF_SHAPES[sh][0]) *
                       ((I.n[1] + JF_SHAPES[sh][1] - 1) / JF_SHAPES[sh][1]);
            }, c->n_jf[sh]);
            ok = ok && c->w_jf[sh];
        }
    // per-instance ranges of the cell work list (entropy reduction)
    std::vector<int> first(n_inst + 1, 0);
    for (int i = 0; i < n_inst; ++i) first[i + 1] = first[i] + c->hI[i].ntile_nodes;
    ok = ok && dalloc(c, (void**)&c->d_first_cell, sizeof(int) * (n_inst + 1)) &&
         dalloc(c, (void**)&c->partial, sizeof(double) * 2 * (first[n_inst] > 0 ? first[n_inst] : 1));
    if (ok) cudaMemcpy(c->d_first_cell, first.data(), sizeof(int) * (n_inst + 1), cudaMemcpyHostToDevice);
    if (c->d == 2 && c->N == 1) prepare_all<2, 1>(c->weno);
    else if (c->d == 2 && c->N == 2) prepare_all<2, 2>(c->weno);
    else if (c->d == 3 && c->N == 1) prepare_all<3, 1>(c->weno);
    else prepare_all<3, 2>(c->weno);
    prepare_mesh();
    for (int k = 0; k < c->d; ++k) c->flux_grid[k] = c->sms * flux_occ(c, c->flux_shape[k]);
    // 2D contexts start with the fused stage launch in fused shape 0 (es_autotune may change it)
    if (c->d == 2) {
        c->fused_shape = 0;
        c->fused_grid = c->sms * flux2d_occ(c, 0);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (!ok || e != cudaSuccess || !c->w_pad || !c->w_cell || (c->d == 3 && (!c->w_ext || !c->w_col || (!c->mixed && !c->w_xe)))) {
        fprintf(stderr, "es_create: setup failed: %s\n", cudaGetErrorString(e));
        es_destroy(c);
        return ES_ERR_CUDA;
    }
    *out = c;
    return ES_OK;
}

es_status es_create(const es_config* cfg, es_ctx** out) { return es_create_batch(cfg, 1, out); }

void es_destroy(es_ctx* c)
{
    if (!c) return;
    drop_run_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->tacc_pinned) cudaFreeHost(c->tacc_pinned);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

const char* es_last_error(const es_ctx* c) { return c ? c->err.c_str() : "null context"; }

int es_num_instances(const es_ctx* c) { return c ? c->n_inst : 0; }

unsigned long long es_scratch_bytes(const es_ctx* c) { return c ? c->bytes : 0ull; }

es_status es_init_mesh(es_ctx* c, const double* x, double* J, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!x || !J) return fail(c, ES_ERR_ARG, "es_init_mesh: null pointer");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.x = x;
    P.Jo = J;
    int n = c->hI[0].ntile_nodes;
    // instance 0 only: its cell tiles are the first n entries of the cell work list
    pdl_launch(init_J_kernel, node_grid(c, n), NODE_TPB, 0, (cudaStream_t)stream, c->dI, P, nullptr, c->w_cell, n);
    return cuda_check(c, "es_init_mesh");
}

es_status es_metrics(es_ctx* c, const double* x, const double* xdot, double* metrics, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!x || !metrics) return fail(c, ES_ERR_ARG, "es_metrics: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_metrics: single-instance context required");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.x = x;
    P.xdot = xdot;
    P.M = metrics;
    launch_metrics(c, P, nullptr, (cudaStream_t)stream);
    return cuda_check(c, "es_metrics");
}

es_status es_rhs(es_ctx* c, const double* JU, const double* J, const double* x, const double* xdot, double* dJU,
                 double* dJ, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !dJU || !dJ) return fail(c, ES_ERR_ARG, "es_rhs: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_rhs: single-instance context required");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.JU = JU;
    P.J = J;
    P.x = x;
    P.xdot = xdot ? xdot : c->hS[0].zeros;
    P.M = c->hS[0].M;
    P.accU = dJU;
    P.accJ = dJ;
    launch_residual(c, P, nullptr, false, 0.0, 1.0, (cudaStream_t)stream);
    return cuda_check(c, "es_rhs");
}

es_status es_rk_step(es_ctx* c, double* JU, double* J, double* x, const double* xdot, const double* dt, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !dt) return fail(c, ES_ERR_ARG, "es_rk_step: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_rk_step: single-instance context required");
    StagePtrs P[3];
    stage_ptrs(c, 0, JU, J, x, xdot, dt, P);
    // on a fixed mesh the stage meshes equal x, so the metrics of the first stage serve all three;
    // in 2D the first stage also forms M(xdot) and the others use M + s dt M(xdot)
    const bool fixed = c->hI[0].fixed != 0, lin = linear_stage_metrics(c);
    for (int s = 0; s < 3; ++s)
        launch_residual(c, P[s], nullptr, true, RK_A[s], RK_B[s], (cudaStream_t)stream, s == 0 || (!fixed && !lin),
                        lin ? MCOEF[s] : 0.0, lin && s == 0, XCOEF[s]);
    return cuda_check(c, "es_rk_step");
}

es_status mesh_redistribute(es_ctx* c, const double* JU, const double* J, const double* x, double dt_fixed,
                            double* xdot, double* dt_dtau, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !xdot || !dt_dtau) return fail(c, ES_ERR_ARG, "mesh_redistribute: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "mesh_redistribute: single-instance context required");
    if (!(dt_fixed >= 0.0)) return fail(c, ES_ERR_ARG, "mesh_redistribute: dt_fixed must be >= 0");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.JU = JU;
    P.J = J;
    P.x = x;
    P.xdot_out = xdot;
    P.out = dt_dtau;
    P.dt_fixed = dt_fixed;
    launch_mesh(c, P, nullptr, (cudaStream_t)stream);
    return cuda_check(c, "mesh_redistribute");
}

es_status es_step(es_ctx* c, double* JU, double* J, double* x, double dt_fixed, double* xdot, double* dt_dtau,
                  void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !xdot || !dt_dtau) return fail(c, ES_ERR_ARG, "es_step: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_step: single-instance context required");
    if (!(dt_fixed >= 0.0)) return fail(c, ES_ERR_ARG, "es_step: dt_fixed must be >= 0");
    StagePtrs M;
    memset(&M, 0, sizeof(M));
    M.JU = JU;
    M.J = J;
    M.x = x;
    M.xdot_out = xdot;
    M.out = dt_dtau;
    M.dt_fixed = dt_fixed;
    StagePtrs P[3];
    stage_ptrs(c, 0, JU, J, x, xdot, dt_dtau, P);
    StagePtrs* const none[3] = { nullptr, nullptr, nullptr };
    launch_step(c, M, nullptr, P, none, (cudaStream_t)stream);
    return cuda_check(c, "es_step");
}

es_status es_schlieren(es_ctx* c, const double* JU, const double* J, const double* x, double psi1, double psi2,
                       double* phi, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !phi) return fail(c, ES_ERR_ARG, "es_schlieren: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_schlieren: single-instance context required");
    cudaStream_t st = (cudaStream_t)stream;
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.JU = JU;
    P.J = J;
    P.x = x;
    P.M = c->hS[0].M;
    P.out = phi;
    launch_metrics(c, P, nullptr, st, true);     // metrics of x (no VCL part); reduction slots reset
    const int gc = node_grid(c, c->n_cell);
    pdl_launch(schlieren_grad_kernel, gc, NODE_TPB, 0, st, c->dI, P, c->w_cell, c->n_cell, c->dS);
    pdl_launch(schlieren_phi_kernel, gc, NODE_TPB, 0, st, c->dI, P, c->w_cell, c->n_cell, c->dS, psi1, psi2);
    return cuda_check(c, "es_schlieren");
}

es_status entropy_production(es_ctx* c, const double* JU, const double* J, const double* dJU, const double* dJ,
                             double* out2, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !out2) return fail(c, ES_ERR_ARG, "entropy_production: null pointer");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "entropy_production: single-instance context required");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    P.JU = JU;
    P.J = J;
    P.accU = const_cast<double*>(dJU);
    P.accJ = const_cast<double*>(dJ);
    P.out = out2;
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps(c, PC_ENTROPY, st);
    pdl_launch(entropy_partial_kernel, node_grid(c, c->n_cell), NODE_TPB, 0, st, c->dI, P, nullptr, c->w_cell, c->n_cell, c->partial);
    pdl_launch(entropy_final_kernel, 1, 256, 0, st, c->dI, P, nullptr, c->d_first_cell, c->partial);
    return cuda_check(c, "entropy_production");
}

es_status es_bind_batch(es_ctx* c, double* const* JU, double* const* J, double* const* x, double* const* xdot,
                        double* const* dt_dtau)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || !xdot || !dt_dtau) return fail(c, ES_ERR_ARG, "es_bind_batch: null table");
    for (int i = 0; i < c->n_inst; ++i)
        if (!JU[i] || !J[i] || !x[i] || !xdot[i] || !dt_dtau[i]) return fail(c, ES_ERR_ARG, "es_bind_batch: null pointer");
    std::vector<StagePtrs> mesh(c->n_inst), st[3];
    for (int s = 0; s < 3; ++s) st[s].resize(c->n_inst);
    for (int i = 0; i < c->n_inst; ++i) {
        StagePtrs P;
        memset(&P, 0, sizeof(P));
        P.JU = JU[i];
        P.J = J[i];
        P.x = x[i];
        P.M = c->hS[i].M;
        P.xdot_out = xdot[i];
        P.out = dt_dtau[i];
        mesh[i] = P;
        StagePtrs S3[3];
        stage_ptrs(c, i, JU[i], J[i], x[i], xdot[i], dt_dtau[i], S3);
        for (int s = 0; s < 3; ++s) st[s][i] = S3[s];
    }
    if (!c->tab_mesh) {
        bool ok = dalloc(c, (void**)&c->tab_mesh, sizeof(StagePtrs) * c->n_inst);
        for (int s = 0; s < 3; ++s) ok = ok && dalloc(c, (void**)&c->tab_stage[s], sizeof(StagePtrs) * c->n_inst);
        if (!ok) return fail(c, ES_ERR_CUDA, "es_bind_batch: table allocation failed");
    }
    cudaMemcpy(c->tab_mesh, mesh.data(), sizeof(StagePtrs) * c->n_inst, cudaMemcpyHostToDevice);
    for (int s = 0; s < 3; ++s) cudaMemcpy(c->tab_stage[s], st[s].data(), sizeof(StagePtrs) * c->n_inst, cudaMemcpyHostToDevice);
    c->bound = true;
    return cuda_check(c, "es_bind_batch");
}

es_status es_step_batch(es_ctx* c, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!c->bound) return fail(c, ES_ERR_ARG, "es_step_batch: call es_bind_batch first");
    cudaStream_t st = (cudaStream_t)stream;
    StagePtrs none;
    memset(&none, 0, sizeof(none));
    const StagePtrs stage[3] = { none, none, none };
    launch_step(c, none, c->tab_mesh, stage, c->tab_stage, st);
    return cuda_check(c, "es_step_batch");
}

es_status es_run_host(es_ctx* c, double* JU, double* J, double* x, int steps, double dt_fixed, double* t, void* stream)
{
    if (!c) return ES_ERR_ARG;
    if (!JU || !J || !x || steps < 0) return fail(c, ES_ERR_ARG, "es_run_host: bad argument");
    if (c->n_inst != 1) return fail(c, ES_ERR_UNSUPPORTED, "es_run_host: single-instance context required");
    const Inst& I = c->hI[0];
    long long n = I.ncell;
    if (!c->hJU) {
        // JU, J and x consecutive in one block (see copy_state)
        bool ok = dalloc(c, (void**)&c->hJU, sizeof(double) * (I.nc + 1 + I.d) * n) &&
                  dalloc(c, (void**)&c->hxd, sizeof(double) * I.d * n) &&
                  dalloc(c, (void**)&c->hdt, sizeof(double) * 2) &&
                  cudaHostAlloc((void**)&c->tacc_pinned, sizeof(double), cudaHostAllocMapped) == cudaSuccess;
        // the elapsed time accumulates in a mapped pinned host word: the host zeroes it and
        // reads it, no copy or memset on the stream
        ok = ok && cudaHostGetDevicePointer((void**)&c->htacc, c->tacc_pinned, 0) == cudaSuccess;
        if (!ok) return fail(c, ES_ERR_CUDA, "es_run_host: allocation failed");
        c->hJ = c->hJU + I.nc * n;
        c->hx = c->hJ + n;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (capturing(st)) return fail(c, ES_ERR_ARG, "es_run_host: not allowed during stream capture");
    // one step (es_step + the time accumulation) as a CUDA graph, replayed per step; with
    // es_profile on, the launches stay eager so that each is timed
    const bool graph = !c->prof;
    if (graph && (!c->run_exec || c->run_dtf != dt_fixed)) {
        drop_run_graph(c);
        if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, ES_ERR_CUDA, "es_run_host: stream creation failed");
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(c, ES_ERR_CUDA, "es_run_host: graph capture failed");
        es_status r = es_step(c, c->hJU, c->hJ, c->hx, dt_fixed, c->hxd, c->hdt, c->cap_stream);
        if (r == ES_OK) time_acc_kernel<<<1, 1, 0, c->cap_stream>>>(c->htacc, c->hdt);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (r != ES_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->run_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->run_exec = nullptr;
            return fail(c, ES_ERR_CUDA, std::string("es_run_host: step graph: ") + cudaGetErrorString(e));
        }
        c->run_dtf = dt_fixed;
    }
    *c->tacc_pinned = 0.0;    // the previous call synchronised: no kernel writes it now
    copy_state(c, JU, J, x, true, st);
    for (int s = 0; s < steps; ++s) {
        if (graph) {
            if (cudaGraphLaunch(c->run_exec, st) != cudaSuccess) return fail(c, ES_ERR_CUDA, "es_run_host: graph launch failed");
            continue;
        }
        es_status r = es_step(c, c->hJU, c->hJ, c->hx, dt_fixed, c->hxd, c->hdt, stream);
        if (r != ES_OK) return r;
        time_acc_kernel<<<1, 1, 0, st>>>(c->htacc, c->hdt);
    }
    copy_state(c, JU, J, x, false, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(c, ES_ERR_CUDA, std::string("es_run_host: ") + cudaGetErrorString(e));
    if (t) *t += *c->tacc_pinned;
    return cuda_check(c, "es_run_host");
}

es_status es_autotune(es_ctx* c, const double* JU, const double* J, const double* x, const double* xdot, int reps,
                      void* stream)
{
    if (!c) return ES_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (capturing(st)) return fail(c, ES_ERR_ARG, "es_autotune: not allowed during stream capture");
    StagePtrs P;
    memset(&P, 0, sizeof(P));
    const StagePtrs* tab = nullptr;
    if (c->n_inst == 1 && JU) {
        if (!J || !x) return fail(c, ES_ERR_ARG, "es_autotune: null pointer");
        StagePtrs S3[3];
        stage_ptrs(c, 0, const_cast<double*>(JU), const_cast<double*>(J), const_cast<double*>(x), xdot, nullptr, S3);
        P = S3[0];
    } else if (c->bound) {
        tab = c->tab_stage[0];
    } else {
        return fail(c, ES_ERR_ARG, "es_autotune: pass the state of a single-instance context or bind a batch first");
    }
    if (reps <= 0) reps = 5;
    // the metrics of the state into the context's scratch; the timed flux launches write
    // only the scratch accumulators (MODE_WRITE), so no caller buffer changes
    launch_metrics(c, P, tab, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < c->d; ++k) {
        float best = 3.0e38f;
        for (int sh = 0; sh < NSHAPE; ++sh) {
            const int occ = flux_occ(c, sh);
            for (int o = occ; o >= 1 && o >= occ - 1; --o) {
                FluxLaunch L;
                L.insts = c->dI;
                L.single = P;
                L.ptrs = tab;
                L.work = c->w_flux[k][sh];
                L.nwork = c->n_flux[k][sh];
                L.k = k;
                L.mode = MODE_WRITE;
                L.a = 0.0;
                L.b = 1.0;
                L.mcoef = 0.0;
                L.xc = 0.0;
                L.status = c->status;
                const int grid = c->sms * o;
                flux_launch(c, L, sh, grid, st);
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps; ++r) flux_launch(c, L, sh, grid, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (ms < best) {
                    best = ms;
                    c->flux_shape[k] = sh;
                    c->flux_grid[k] = grid;
                }
            }
        }
        c->flux_ms[k] = best;
    }
    // 2D: the fused stage launch in each fused shape against the sum of the best
    // per-direction launches (both in MODE_WRITE); the faster form is kept
    c->fused_shape = -1;
    c->fused_ms = 0.f;
    drop_run_graph(c);
    if (c->d == 2) {
        float best = 3.0e38f;
        for (int sh = 0; sh < NFSHAPE; ++sh) {
            const int occ = flux2d_occ(c, sh);
            for (int o = occ; o >= 1 && o >= occ - 1; --o) {
                FluxLaunch L;
                L.insts = c->dI;
                L.single = P;
                L.ptrs = tab;
                L.work = c->w_fused[sh];
                L.nwork = c->n_fused[sh];
                L.k = 0;
                L.mode = MODE_WRITE;
                L.a = 0.0;
                L.b = 1.0;
                L.mcoef = 0.0;
                L.xc = 0.0;
                L.status = c->status;
                const int grid = c->sms * o;
                flux2d_launch(c, L, sh, grid, st);
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps; ++r) flux2d_launch(c, L, sh, grid, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (ms < best) {
                    best = ms;
                    c->fused_ms = ms;
                    if (ms < c->flux_ms[0] + c->flux_ms[1]) {
                        c->fused_shape = sh;
                        c->fused_grid = grid;
                    }
                }
            }
        }
    }
    // mixed 2D: the fused mesh-step launch in each tile shape, after the passes it reads
    // (metrics, CFL and monitor gradients) on the same state; it writes only scratch
    c->jf_ms = 0.f;
    if (fused_mesh2d(c)) {
        StagePtrs Q = P;
        Q.xdot = nullptr;
        const int mu = c->hI[0].mu, nf = c->hI[0].nf;
        launch_metrics(c, Q, tab, st, true, false, false);
        launch_cfl_grad(c->mixed, c->d, c->N, node_grid(c, c->n_cell), st, c->dI, P, tab, c->w_cell, c->n_cell, c->dS);
        float best = 3.0e38f;
        for (int sh = 0; sh < NJF_SHAPE; ++sh) {
            const int grid = node_grid(c, c->n_jf[sh]);
            launch_jacobi_fused2d(sh, grid, st, c->dI, P, tab, c->w_jf[sh], c->n_jf[sh], c->dS, mu, nf, nf % 2);
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r)
                launch_jacobi_fused2d(sh, grid, st, c->dI, P, tab, c->w_jf[sh], c->n_jf[sh], c->dS, mu, nf, nf % 2);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < best) {
                best = ms;
                c->jf_ms = ms;
                c->jf_shape = sh;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_check(c, "es_autotune");
}

es_status es_get_mesh_tiles(const es_ctx* c, int* shape, int* TX, int* TY, int* threads, float* ms)
{
    if (!c || !shape || !TX || !TY || !threads || !ms) return ES_ERR_ARG;
    const bool on = fused_mesh2d(c);
    *shape = on ? c->jf_shape : -1;
    *TX = on ? JF_SHAPES[c->jf_shape][0] : 0;
    *TY = on ? JF_SHAPES[c->jf_shape][1] : 0;
    *threads = on ? JF_SHAPES[c->jf_shape][2] : 0;
    *ms = on ? c->jf_ms : 0.f;
    return ES_OK;
}

es_status es_set_mesh_tiles(es_ctx* c, int shape)
{
    if (!c) return ES_ERR_ARG;
    if (!c->mixed || c->d != 2 || shape < 0 || shape >= NJF_SHAPE)
        return fail(c, ES_ERR_ARG, "es_set_mesh_tiles: shape out of range or not a mixed-form 2D context");
    c->jf_shape = shape;
    c->jf_ms = 0.f;
    drop_run_graph(c);
    return ES_OK;
}

es_status es_get_tuning(const es_ctx* c, int* shape, int* S, int* WT, int* grid, float* ms)
{
    if (!c || !shape || !S || !WT || !grid || !ms) return ES_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        const bool on = k < c->d;
        shape[k] = on ? c->flux_shape[k] : 0;
        S[k] = on ? SHAPE_S[c->flux_shape[k]] : 0;
        WT[k] = on ? SHAPE_WT[c->flux_shape[k]] : 0;
        grid[k] = on ? c->flux_grid[k] : 0;
        ms[k] = on ? c->flux_ms[k] : 0.f;
    }
    return ES_OK;
}

es_status es_set_tuning(es_ctx* c, int k, int shape, int grid)
{
    if (!c) return ES_ERR_ARG;
    if (k < 0 || k >= c->d || shape < 0 || shape >= NSHAPE || grid < 0)
        return fail(c, ES_ERR_ARG, "es_set_tuning: direction, shape or grid out of range");
    c->flux_shape[k] = shape;
    c->flux_grid[k] = grid > 0 ? grid : c->sms * flux_occ(c, shape);
    c->flux_ms[k] = 0.f;
    drop_run_graph(c);
    return ES_OK;
}

es_status es_get_fusion(const es_ctx* c, int* shape, int* TX, int* TY, int* grid, float* ms)
{
    if (!c || !shape || !TX || !TY || !grid || !ms) return ES_ERR_ARG;
    const int sh = c->fused_shape;
    *shape = sh;
    *TX = sh >= 0 ? FSHAPE_TX[sh] : 0;
    *TY = sh >= 0 ? FSHAPE_TY[sh] : 0;
    *grid = sh >= 0 ? c->fused_grid : 0;
    *ms = c->fused_ms;
    return ES_OK;
}

es_status es_set_fusion(es_ctx* c, int shape, int grid)
{
    if (!c) return ES_ERR_ARG;
    if (shape < -1 || shape >= NFSHAPE || grid < 0 || (shape >= 0 && c->d != 2))
        return fail(c, ES_ERR_ARG, "es_set_fusion: shape out of range, negative grid or not a 2D context");
    c->fused_shape = shape;
    c->fused_grid = shape >= 0 ? (grid > 0 ? grid : c->sms * flux2d_occ(c, shape)) : 0;
    c->fused_ms = 0.f;
    drop_run_graph(c);
    return ES_OK;
}

es_status es_check_conversions(const double* in, int n, float* out32, double* out64, void* stream)
{
    if (!in || !out32 || !out64 || n < 0) return ES_ERR_ARG;
    if (n == 0) return ES_OK;
    conversion_check_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(in, n, out32, out64);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

es_status es_check_half_sums(const float* a, const float* b, int n, double* out, void* stream)
{
    if (!a || !b || !out || n < 0) return ES_ERR_ARG;
    if (n == 0) return ES_OK;
    half_sum_check_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(a, b, n, out);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

es_status es_check_logmean_small(const float* a, const float* b, const float* del, int n, float* fast, float* general,
                                 void* stream)
{
    if (!a || !b || !del || !fast || !general || n < 0) return ES_ERR_ARG;
    if (n == 0) return ES_OK;
    logmean_small_check_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(a, b, del, n, fast, general);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

es_status es_profile(es_ctx* c, int enable)
{
    if (!c) return ES_ERR_ARG;
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->ev_class.clear();
    c->ev_used = 0;
    for (int q = 0; q < 8; ++q) { c->prof_ms[q] = 0.0; c->prof_n[q] = 0; }
    c->prof = enable != 0;
    if (c->prof) {
        const int pairs = 8192;
        c->ev.resize(2 * pairs);
        c->ev_class.resize(pairs);
        for (auto& e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { c->prof = false; return fail(c, ES_ERR_CUDA, "es_profile: event creation failed"); }
    }
    return ES_OK;
}

es_status es_profile_read(es_ctx* c, double* ms, long long* launches, int n_classes)
{
    if (!c || n_classes < 0 || n_classes > 8) return ES_ERR_ARG;
    if (c->ev_used > 0) {
        cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1]);
        if (e != cudaSuccess) return fail(c, ES_ERR_CUDA, std::string("es_profile_read: ") + cudaGetErrorString(e));
    }
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float t = 0.f;
        cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]);
        int cls = c->ev_class[i / 2];
        c->prof_ms[cls] += t;
        c->prof_n[cls] += 1;
    }
    c->ev_used = 0;
    for (int q = 0; q < n_classes; ++q) {
        if (ms) ms[q] = c->prof_ms[q];
        if (launches) launches[q] = c->prof_n[q];
        c->prof_ms[q] = 0.0;
        c->prof_n[q] = 0;
    }
    return ES_OK;
}

es_status es_poll_status(es_ctx* c, int* flags, void* stream)
{
    if (!c || !flags) return ES_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemsetAsync(c->status, 0, sizeof(int), st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(c, ES_ERR_CUDA, std::string("es_poll_status: ") + cudaGetErrorString(e));
    *flags = h;
    if (h & ST_NONPHYSICAL) return fail(c, ES_ERR_NONPHYSICAL, "non-physical state (rho_l <= 0, T <= 0 or NaN)");
    return ES_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entropy diagnostics (es_entropy_production_noalloc).
//
// For callers that may not allocate device memory: runtimes that hand out every
// byte of device memory from their own pool, and real-time loops where an
// allocation may synchronise the device.  The per-tile partial sums that
// entropy_production keeps in context scratch live here in one file-scope device
// array of fixed size instead; no context is created.
// ---------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr int NOALLOC_TPB = 256;
constexpr int NOALLOC_MAX_TILES = 4096;      // tiles of 256 nodes: at most 1,048,576 nodes
constexpr int NOALLOC_MAX_DEVICES = 64;

// two doubles per tile: 64 KiB, held by every GPU that loads the library until exit
static __device__ __align__(256) double g_noalloc_partial[2 * NOALLOC_MAX_TILES];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// device address of g_noalloc_partial on the current device, looked up once per device
es_status noalloc_scratch(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return ES_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "es_entropy_production_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return ES_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return ES_OK;
}

// one tile of 256 consecutive nodes per block: V.dJU - phi dJ and J eta summed in a
// deterministic, fixed order (warp shuffles, then the warps in order).  The order differs
// from the context's entropy reduction, which sums over 2D node tiles, so the two calls
// agree to round-off, not bit for bit
__global__ void noalloc_entropy_partial_kernel(Inst I, const double* __restrict__ JU, const double* __restrict__ J,
                                               const double* __restrict__ dJU, const double* __restrict__ dJ,
                                               double* __restrict__ partial)
{
    __shared__ double sh[2][32];
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (p < I.ncell) {
        double Jp = J[p], U[MAXC];
        for (int q = 0; q < I.nc; ++q) U[q] = JU[(long long)q * I.ncell + p] / Jp;
        double rho = 0.0, cvr = 0.0, rr = 0.0;
        for (int l = 0; l < I.N; ++l) { rho += U[l]; cvr += I.cv[l] * U[l]; rr += I.Rs[l] * U[l]; }
        double v[3], v2 = 0.0;
        for (int m = 0; m < I.d; ++m) { v[m] = U[I.N + m] / rho; v2 += v[m] * v[m]; }
        double T = (U[I.N + I.d] - 0.5 * rho * v2 - I.pinf_tot) / cvr;
        double eta = 0.0, phi = 0.0, lT = log(T), V[MAXC];
        for (int l = 0; l < I.N; ++l) {
            double S = I.cv[l] * lT - I.Rs[l] * log(U[l]);
            V[l] = -S - v2 / (2.0 * T) + I.cvG[l];
            eta -= U[l] * S;
            phi += I.Rs[l] * U[l] - I.pinf[l] / T;
        }
        for (int m = 0; m < I.d; ++m) V[I.N + m] = v[m] / T;
        V[I.N + I.d] = -1.0 / T;
        if (dJU && dJ) {
            for (int q = 0; q < I.nc; ++q) a += V[q] * dJU[(long long)q * I.ncell + p];
            a -= phi * dJ[p];
        }
        b = Jp * eta;
    }
    for (int o = 16; o > 0; o >>= 1) { a += __shfl_xor_sync(0xffffffffu, a, o); b += __shfl_xor_sync(0xffffffffu, b, o); }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += sh[0][q]; sb += sh[1][q]; }
        partial[2 * (long long)blockIdx.x] = sa;
        partial[2 * (long long)blockIdx.x + 1] = sb;
    }
}

__global__ void noalloc_entropy_final_kernel(Inst I, int ntiles, const double* __restrict__ partial,
                                             double* __restrict__ out)
{
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int w = threadIdx.x; w < ntiles; w += blockDim.x) { a += partial[2 * w]; b += partial[2 * w + 1]; }
    for (int o = 16; o > 0; o >>= 1) { a += __shfl_xor_sync(0xffffffffu, a, o); b += __shfl_xor_sync(0xffffffffu, b, o); }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += sh[0][q]; sb += sh[1][q]; }
        double vol = 1.0;
        for (int k = 0; k < I.d; ++k) vol *= I.dxi[k];
        out[0] = vol * sa;
        out[1] = vol * sb;
    }
}

}  // namespace

extern "C" es_status es_entropy_production_noalloc(const es_config* cfg, const double* JU, const double* J,
                                                   const double* dJU, const double* dJ, double* out2, void* stream)
{
    if (!cfg || !JU || !J || !out2) {
        fprintf(stderr, "es_entropy_production_noalloc: null pointer\n");
        return ES_ERR_ARG;
    }
    std::string m = check_cfg(*cfg);
    if (!m.empty()) {
        fprintf(stderr, "es_entropy_production_noalloc: %s\n", m.c_str());
        return ES_ERR_ARG;
    }
    Inst I = make_inst(*cfg);
    long long ntiles = (I.ncell + NOALLOC_TPB - 1) / NOALLOC_TPB;
    if (ntiles > NOALLOC_MAX_TILES) {
        fprintf(stderr, "es_entropy_production_noalloc: %lld nodes exceed the limit of %d nodes of the "
                        "allocation-free call (use entropy_production with a context)\n",
                I.ncell, NOALLOC_MAX_TILES * NOALLOC_TPB);
        return ES_ERR_ARG;
    }
    double* partial = nullptr;
    es_status s = noalloc_scratch(&partial);
    if (s != ES_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    noalloc_entropy_partial_kernel<<<(int)ntiles, NOALLOC_TPB, 0, st>>>(I, JU, J, dJU, dJ, partial);
    noalloc_entropy_final_kernel<<<1, NOALLOC_TPB, 0, st>>>(I, (int)ntiles, partial, out2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "es_entropy_production_noalloc: %s\n", cudaGetErrorString(e));
        return ES_ERR_CUDA;
    }
    return ES_OK;
}
