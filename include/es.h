/*
 * es.h -- C ABI of the GB300 library for the entropy-stable adaptive
 * moving-mesh finite-difference method of arXiv 2202.07989 (Duan & Tang,
 * "High-order accurate entropy stable adaptive moving mesh finite difference
 * schemes for (multi-component) compressible Euler equations with the
 * stiffened equation of state").
 *
 * Problem (Sec. 1, Eq. (1.1)): U = (rho_1..rho_N, rho v_1..rho v_d, E),
 * N in {1, 2} species, d in {2, 3}, stiffened mixture EOS (Eq. (1.2)).
 * The state advanced in time is (JU, J, x) on a fixed computational grid
 * (Sec. 2, Eq. (2.2)): the Jacobian-weighted conserved variables, the
 * Jacobian and the physical node positions.
 *
 * Data layout (all calls): every array is a contiguous structure of arrays,
 * field-major, a[f][i3][i2][i1] with i1 fastest, interior nodes only, FP64.
 * n_c = N + d + 1 conserved fields; x and xdot have d fields; J has 1.  In 2D
 * n[2] = 1.  Nodes sit at the cell centres xi_{k,i} = xi_lo[k] + (i + 1/2) dxi[k].
 *
 * Ownership: the caller owns every state, input and output buffer; pointers
 * are DEVICE pointers unless a call says HOST.  A context owns only scratch it
 * allocates in es_create / es_create_batch and frees in es_destroy; no call
 * after creation allocates device memory, except es_run_host (its buffers on
 * the first call; its step graph on the first call after a tuning change) and
 * es_profile(ctx, 1) on a context.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls are asynchronous on that stream unless they say otherwise;
 * scalar results are written to device memory so whole steps can be captured
 * in a CUDA graph (es_rk_step, mesh_redistribute, es_step, entropy_production).
 *
 * Errors: every call returns an es_status.  Argument errors are detected on
 * the host before any launch (ES_ERR_ARG, ES_ERR_UNSUPPORTED).  Launch errors
 * return ES_ERR_CUDA.  Non-physical states met by a kernel (rho_l <= 0,
 * T <= 0, NaN) set a sticky device status word and the kernel carries on with
 * placeholder values; es_poll_status reads it (synchronising the stream) and
 * reports ES_ERR_NONPHYSICAL.  No kernel traps or asserts.  es_last_error
 * returns a message for the last failing call on a context.
 */
#ifndef ES_H
#define ES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum es_status {
    ES_OK = 0,
    ES_ERR_ARG = 1,          /* bad argument (null pointer, size, parameter range) */
    ES_ERR_UNSUPPORTED = 2,  /* configuration outside what this build implements */
    ES_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
    ES_ERR_NONPHYSICAL = 4,  /* a kernel met rho_l <= 0, T <= 0 or NaN */
    ES_ERR_TIMEOUT = 5       /* reserved for bounded device waits */
} es_status;

enum { ES_BC_PERIODIC = 0, ES_BC_REFLECT = 1, ES_BC_INFLOW = 2, ES_BC_OUTFLOW = 3 };
enum { ES_FP64 = 0, ES_MIXED = 1 };
enum { ES_WENO_MR = 0, ES_WENO_JS = 1 };
enum { ES_MON_GRAD2 = 0, ES_MON_GRAD = 1, ES_MON_LAP = 2 };
enum { ES_SIG_RHO = 0, ES_SIG_RHO1 = 1, ES_SIG_RHO2 = 2, ES_SIG_P = 3, ES_SIG_Y2 = 4, ES_SIG_V1 = 5 };

/* One instance.  Physics: Gamma_l, c_{v,l}, p_{inf,l} (Sec. 1, Eq. (1.2)).
 * Scheme: sixth-order EC flux (w = 3, Sec. 3.1), WENO-MR dissipation with
 * linear weights chi and epsilon (Appendix A) when es = 1, SSP-RK3, CFL number
 * cfl (Eq. (cfl)).  Mesh: monitor Eq. (monitor) on the variables sigma[] with
 * weights alpha[], nf filter passes and mu Jacobi sweeps (Sec. 4).
 * precision: ES_FP64 runs everything in FP64; ES_MIXED runs the EC pairs, the
 * WENO-MR dissipation and the monitor/filter in FP32 and keeps metrics, the
 * GCL flux of J, the small-jump logarithmic-mean branch, divergence and RK
 * accumulation and the entropy diagnostics in FP64. */
typedef struct es_config {
    int d;                   /* 2 or 3 */
    int N;                   /* 1 or 2 species */
    int n[3];                /* nodes per direction; n[2] = 1 when d = 2; n[k] >= 10 */
    double xi_lo[3];         /* lower corner of the computational box */
    double dxi[3];           /* node spacing (box length / n) */
    int bc[3][2];            /* ES_BC_* per direction and side (periodic on both or neither) */
    double inflow[3][2][8];  /* conserved state on ES_BC_INFLOW sides */
    double gamma[2], cv[2], pinf[2];
    int es;                  /* 1: entropy stable (EC + dissipation); 0: entropy conservative */
    int precision;           /* ES_FP64 or ES_MIXED */
    double chi[3];           /* WENO-MR linear weights, positive, summing to 1 */
    double weno_eps;         /* WENO-MR epsilon (1e-10 in the paper) */
    double cfl;              /* CFL number (0.4 in 2D, 0.3 in 3D in the paper) */
    int n_sigma;             /* 0..4 monitor variables */
    int sigma[4];            /* ES_SIG_* */
    double alpha[4];         /* monitor weights alpha_k >= 0 */
    int mu;                  /* Jacobi sweeps per step (>= 0) */
    int nf;                  /* filter passes per step (>= 0) */
    int weno;                /* ES_WENO_MR (Appendix A; the paper's scheme) or ES_WENO_JS */
    int fixed_mesh;          /* 1: the mesh never moves (the paper's uniform-mesh runs): xdot = 0,
                                no monitor or sweeps, metrics formed once per step and x never
                                rewritten; sigma, alpha, mu and nf are ignored */
    int sigma_op[4];         /* per monitor term: ES_MON_GRAD2 (alpha (|grad_xi sigma|/max)^2, Eq.
                                (monitor); 0 = default), ES_MON_GRAD (alpha |grad_xi sigma|/max) or
                                ES_MON_LAP (alpha |Laplacian_xi sigma|/max), the linear terms of
                                Example 5.1's vortex monitor; second-order central differences */
    int w;                   /* EC flux order 2w (Sec. 3.1): 1, 2 or 3; 0 means 3, the order of the
                                paper's examples.  The metric operator delta_k and the GCL flux
                                take the same order; the dissipation (5th-order WENO) does not */
    int march_planes;        /* 3D mixed form: planes per chunk of the mesh-step kernels that march
                                along i3 (a schedule, not part of the method; it changes no result).
                                0 = automatic (about four waves of CTAs); otherwise 4 <= value <= n[2] */
} es_config;

typedef struct es_ctx es_ctx;

/* Create a context for one instance (es_create) or for n_inst independent
 * instances advanced together (es_create_batch; cfgs is a HOST array).  All
 * instances of a batch share d, N and precision.  Allocates the scratch of
 * every later call on the current CUDA device.  On failure *out is NULL. */
es_status es_create(const es_config* cfg, es_ctx** out);
es_status es_create_batch(const es_config* cfgs, int n_inst, es_ctx** out);
void es_destroy(es_ctx* ctx);
const char* es_last_error(const es_ctx* ctx);
int es_num_instances(const es_ctx* ctx);

/* Bytes of device scratch the context holds. */
unsigned long long es_scratch_bytes(const es_ctx* ctx);

/* J^0 = det(delta_k[x_j] / dxi_k) at the nodes from caller-filled positions x
 * (the initial Jacobian; Sec. 3.2 operators).  x: d fields (read), J: 1 field
 * (written).  Instance 0 of the context. */
es_status es_init_mesh(es_ctx* ctx, const double* x, double* J, void* stream);

/* Metrics of Sec. 3.2: J xi_k/x_j by Eq. (SCLCoeff) (3D; the 2D degenerate
 * case otherwise) and J xi_k/t = -sum_j xdot_j J xi_k/x_j (Eq. (VCLCoeff)).
 * x, xdot: d fields each (xdot may be NULL = 0).  metrics (written):
 * d*(d+1) fields on the padded grid with 3 ghost layers per direction,
 * metrics[(k*(d+1) + c)][i3+3][i2+3][i1+3], c = 0 for J xi_k/t and 1 + j for
 * J xi_k/x_j; padded extents n[k] + 6 (1 for the absent third direction in 2D). */
es_status es_metrics(es_ctx* ctx, const double* x, const double* xdot, double* metrics, void* stream);

/* Semi-discrete residual, Eqs. (semi_U) and (semi_J): dJU = d(JU)/dt (n_c
 * fields) and dJ = dJ/dt (1 field) from the state (JU, J, x) and the mesh
 * velocity xdot (NULL = 0).  EC flux Eq. (ECFlux_curv_2p) with the two-point
 * flux Eq. (ECfluxMM); ES flux Eq. (HOstable) when cfg.es = 1.  Instance 0. */
es_status es_rhs(es_ctx* ctx, const double* JU, const double* J, const double* x, const double* xdot,
                 double* dJU, double* dJ, void* stream);

/* One SSP-RK3 step (Shu-Osher form, Sec. 5) of (JU, J, x) IN PLACE with the
 * mesh velocity xdot held constant over the step (xdot may be NULL = 0).
 * dt: DEVICE pointer to the time step (e.g. the first output of
 * mesh_redistribute).  Three residual evaluations; no host synchronisation. */
es_status es_rk_step(es_ctx* ctx, double* JU, double* J, double* x, const double* xdot, const double* dt,
                     void* stream);

/* Mesh redistribution of Sec. 4 for the next step: Delta t by Eq. (cfl) on
 * x (or dt_fixed when dt_fixed > 0, HOST value), the monitor Eq. (monitor)
 * smoothed nf times, mu Jacobi sweeps of the discrete mesh equations, the
 * limiter Delta_tau and xdot = Delta_tau (x^[mu] - x) / Delta t.
 * xdot (written): d fields.  dt_dtau (written, DEVICE): {Delta t, Delta_tau}. */
es_status mesh_redistribute(es_ctx* ctx, const double* JU, const double* J, const double* x, double dt_fixed,
                            double* xdot, double* dt_dtau, void* stream);

/* One full time step on one instance: mesh_redistribute on (JU, J, x), then
 * es_rk_step with the mesh velocity and time step just formed -- the same
 * results, bit for bit, as those two calls in sequence.  The first RK stage
 * reuses the spatial metrics of x that the mesh step forms, so the step forms
 * metrics three times instead of four.  JU, J, x: updated IN PLACE.
 * dt_fixed: HOST value as in mesh_redistribute.  xdot (written): d fields.
 * dt_dtau (written, DEVICE): {Delta t, Delta_tau}.  ES_ERR_UNSUPPORTED on a
 * batch context (use es_step_batch); no host synchronisation. */
es_status es_step(es_ctx* ctx, double* JU, double* J, double* x, double dt_fixed, double* xdot, double* dt_dtau,
                  void* stream);

/* Autotuner of the flux launches (tile shapes and schedules; the paper has no
 * counterpart -- it is part of the batched form).  For every direction it times
 * each flux tile shape (S nodes along the line x WT lines; es_get_tuning lists
 * the one chosen) at one and at full persistent occupancy on the given state,
 * and keeps the fastest for all later calls on the context.  Tile shape and grid
 * change no result: every interface flux and node divergence is formed by the
 * same arithmetic in any tile.  Single-instance context: JU, J, x (and xdot, may
 * be NULL) give the state, read only.  Batch context: pass NULLs after
 * es_bind_batch; the bound state is read only.  The timed launches write only
 * context scratch.  reps <= 0 means 5 timed launches per candidate.  Host
 * synchronisation; ES_ERR_ARG during stream capture. */
es_status es_autotune(es_ctx* ctx, const double* JU, const double* J, const double* x, const double* xdot, int reps,
                      void* stream);

/* The flux launch configuration per direction k = 0..2 (zeros for directions
 * the problem lacks): shape index, S, WT, persistent grid size (CTAs) and the
 * time per launch the last es_autotune measured (0 if none).  Each argument
 * points to 3 values (HOST). */
es_status es_get_tuning(const es_ctx* ctx, int* shape, int* S, int* WT, int* grid, float* ms);

/* Fix the flux launch of direction k to tile shape `shape` (0..5) and `grid`
 * CTAs (0 = SM count x occupancy of that shape).  ES_ERR_ARG when out of range. */
es_status es_set_tuning(es_ctx* ctx, int k, int shape, int grid);

/* Fused 2D stage launch (the paper has no counterpart; a launch schedule): both
 * directions of the residual of Eqs. (semi_U), (semi_J), and the stage update,
 * in one launch over TX x TY node tiles (5 fused shapes).  Every interface flux
 * and node divergence is formed by the arithmetic of the per-direction launches,
 * and the two directions' divergences are summed in the same FP64 order, so
 * results are bitwise those of the per-direction launches.  es_autotune on a 2D
 * context also times each fused shape and keeps the fused launch when it beats
 * the sum of the best per-direction launches.  A new 2D context starts with the
 * fused launch in shape 0 (16 x 12 tiles, full occupancy).
 * es_get_fusion: fused shape index (-1: per-direction launches), TX, TY, grid
 * (CTAs) and the best fused time per launch the last es_autotune measured (0 if
 * none; set even when the per-direction launches won).  All pointers HOST, one
 * value each. */
es_status es_get_fusion(const es_ctx* ctx, int* shape, int* TX, int* TY, int* grid, float* ms);

/* Fix the fused 2D stage launch: shape -1 (per-direction launches) or 0..4, and
 * `grid` CTAs (0 = SM count x occupancy of that shape).  ES_ERR_ARG when out of
 * range or when shape >= 0 on a 3D context. */
es_status es_set_fusion(es_ctx* ctx, int shape, int grid);

/* Tiles of the mixed-form 2D mesh step (the paper has no counterpart; a launch
 * schedule).  The monitor, the filter passes and the Jacobi sweeps of Sec. 4 run
 * in one launch over TX x TY node tiles, each staged in shared memory with a halo
 * of mu + n_f nodes (temporal blocking), in one of 4 shapes: 0: 32 x 8 tiles with
 * 256 threads per block; 1: 32 x 16, 2: 24 x 16, 3: 24 x 12, each with 512.
 * Every node's displacement is formed by the same arithmetic in any tile, so the
 * shape changes no result.  es_autotune on such a context also times every shape
 * on one mesh step of the given state and keeps the fastest.  A new context
 * starts in shape 0.
 * es_get_mesh_tiles: shape index, TX, TY, threads per block and the best time per
 * launch the last es_autotune measured (0 if none).  All pointers HOST, one value
 * each; on contexts without the fused mesh step, shape -1 and zeros.
 * es_set_mesh_tiles: shape 0..3; ES_ERR_ARG when out of range or when the context
 * is not a mixed-form 2D context. */
es_status es_get_mesh_tiles(const es_ctx* ctx, int* shape, int* TX, int* TY, int* threads, float* ms);
es_status es_set_mesh_tiles(es_ctx* ctx, int shape);

/* Schlieren function of Example 5.8, Eq. (schlieren), on one instance:
 * phi = exp(-Psi |grad rho| / max |grad rho|), Psi = (psi1 rho_1 + psi2 rho_2) / rho
 * (the paper uses psi1 = 30, psi2 = 150), grad the physical gradient
 * (1/J) sum_k J xi_k/x d rho/d xi_k with second-order central differences in xi and
 * the metrics of x; phi = 1 everywhere when max |grad rho| = 0.  JU, J, x: state
 * (read).  phi (written, DEVICE): 1 field.  FP64 in both precisions; no host
 * synchronisation.  Uses the context's scratch (not concurrently with other calls
 * on the same context). */
es_status es_schlieren(es_ctx* ctx, const double* JU, const double* J, const double* x, double psi1, double psi2,
                       double* phi, void* stream);

/* Entropy diagnostics (Sec. 1 definitions, Sec. 5 total entropy):
 * out2[0] = P = sum_i dxi^d (V_i . dJU_i - phi_i dJ_i)  (= d/dt of the total
 * entropy; 0 for the EC scheme on periodic data, <= 0 for the ES scheme) and
 * out2[1] = sum_i J_i eta(U_i) dxi^d.  dJU, dJ may be NULL (then P = 0).
 * out2: DEVICE, 2 doubles.  Deterministic (fixed reduction order). */
es_status entropy_production(es_ctx* ctx, const double* JU, const double* J, const double* dJU, const double* dJ,
                             double* out2, void* stream);

/* Allocation-free entropy diagnostics: the same two sums as entropy_production
 * for one instance described by cfg, without a context.  The paper has no
 * counterpart; this call exists for callers that may not allocate device
 * memory -- runtimes that hand out all device memory from their own pool, and
 * real-time loops where an allocation may synchronise the device.  It calls no
 * cudaMalloc, cudaFree or allocating library routine; the caller passes the
 * inputs and the output (out2: DEVICE, 2 doubles).
 * Its per-tile partial sums live in one library-wide device array of 64 KiB
 * (4096 tiles of 256 nodes), which every GPU that loads the library holds
 * until the process exits; grids over 4096 * 256 = 1,048,576 nodes are
 * rejected with ES_ERR_ARG and a message on stderr.  The first call on a
 * device looks up the array's device address for that device.  All calls
 * share the array: every slot a call reads is written by the same call first,
 * but calls that overlap on the GPU (concurrent streams, several host threads)
 * race on it. */
es_status es_entropy_production_noalloc(const es_config* cfg, const double* JU, const double* J,
                                        const double* dJU, const double* dJ, double* out2, void* stream);

/* Batched forms: arrays of n_inst DEVICE pointers passed as HOST arrays; one
 * launch per kernel covers every instance.  es_bind_batch uploads the
 * pointer tables (synchronous; call it again when buffers change) and
 * es_step_batch then runs, for every instance, mesh_redistribute followed by
 * es_rk_step with the instance's own Delta t, Delta_tau and xdot, writing
 * {Delta t, Delta_tau} to dt_dtau[i].  es_step_batch does not synchronise and
 * can be captured in a CUDA graph. */
es_status es_bind_batch(es_ctx* ctx, double* const* JU, double* const* J, double* const* x, double* const* xdot,
                        double* const* dt_dtau);
es_status es_step_batch(es_ctx* ctx, void* stream);

/* Full steps on HOST buffers (instance 0): copies (JU, J, x) to the device,
 * runs `steps` times mesh_redistribute (CFL Delta t, or dt_fixed > 0) + an
 * SSP-RK3 step, copies (JU, J, x) back and adds the elapsed time to *t.
 * Synchronous.  Uses device buffers owned by the context, allocated by the
 * first call (JU, J and x consecutive in one block, with one pinned host word
 * for the elapsed time).  Copies: one cudaMemcpyAsync each way when the host
 * buffers are consecutive in one allocation (J = JU + n_c * cells,
 * x = J + cells), else one per buffer and direction (asynchronous when the host
 * memory is pinned).  Each step replays a CUDA graph of es_step on the device
 * buffers, captured on a private stream by the first call and again after
 * es_autotune, es_set_tuning, es_set_fusion, es_set_mesh_tiles or a new
 * dt_fixed; with es_profile on, the steps are launched one kernel at a time
 * instead.  ES_ERR_ARG during stream capture. */
es_status es_run_host(es_ctx* ctx, double* JU, double* J, double* x, int steps, double dt_fixed, double* t,
                      void* stream);

/* Kernel timing.  es_profile(ctx, 1) preallocates CUDA events; while enabled,
 * calls that are not being captured into a CUDA graph record an event pair
 * around every kernel launch on the call's stream.  es_profile_read
 * synchronises, returns per class the summed milliseconds and the launch
 * count since the last read, then resets them.  Classes (n_classes <= 8):
 * 0..2 flux + divergence (+ RK stage) for directions 1..3 (per-direction
 * launches), 3 metrics, 4 mesh redistribution (CFL, monitor, filter, Jacobi,
 * limiter, xdot), 5 entropy diagnostics, 6 the fused 2D stage launch (both
 * directions, + RK stage).  es_profile(ctx, 0) frees the events. */
es_status es_profile(es_ctx* ctx, int enable);
es_status es_profile_read(es_ctx* ctx, double* ms, long long* launches, int n_classes);

/* Self-check of the IEEE 754 binary64 <-> binary32 conversions the mixed form
 * does with integer instructions (GB300 issues the hardware conversions on its
 * FP64 pipe): out32[i] = round-to-nearest-even binary32 of in[i] (values below
 * 2^-126 in magnitude become a signed zero) and out64[i] = out32[i] widened
 * exactly.  in, out32, out64: DEVICE arrays of n elements. */
es_status es_check_conversions(const double* in, int n, float* out32, double* out64, void* stream);

/* Self-check of the exact mean {a} = a/2 + b/2 that the mixed form's log-mean
 * small-jump branch (Sec. 3.3, the Ismail-Roe series) assembles with integer
 * instructions: out[i] = a[i]/2 + b[i]/2 as a binary64 value.  Exact for
 * positive normal a, b whose binary32 exponents differ by at most 7 (the branch
 * has |b - a| < (a + b)/10); otherwise the binary64 sum of the binary32 halves.
 * a, b: DEVICE arrays of n binary32 values; out: DEVICE array of n doubles. */
es_status es_check_half_sums(const float* a, const float* b, int n, double* out, void* stream);

/* Self-check of the mixed form's log-mean small-jump value {a}(1 - del) rounded to
 * binary32 (Sec. 3.3): fast[i] as the flux kernels form it (integer-built {a},
 * conversions without special cases where their preconditions hold) and
 * general[i] by the general conversions with an FP64 add for {a}; both through
 * one FP64 fused multiply-add.  a, b > 0, 0 <= del <= 1/2.  a, b, del, fast,
 * general: DEVICE arrays of n binary32 values. */
es_status es_check_logmean_small(const float* a, const float* b, const float* del, int n, float* fast, float* general,
                                 void* stream);

/* ALU throughput microbenchmark: the measured denominators of the flux kernels'
 * roofline (the paper has no counterpart; its method is bound by the plain FP32 and
 * FP64 pipes, not by HBM or tensor cores).  Launches `grid` CTAs of 256 threads; every
 * thread runs `iters` rounds of 16 independent fused multiply-add chains of kind
 * 0 = binary32 (FFMA), 1 = paired binary32 (FFMA2: two lanes per instruction) or
 * 2 = binary64 (DFMA).  The caller times the launch on `stream` (CUDA events).
 * sink (written, DEVICE): grid * 256 doubles, each thread's chain sum, which keeps
 * every operation live.  es_alu_peak_flops returns the flops of such a launch
 * (2 per multiply-add lane), 0 for bad arguments.  ES_ERR_ARG for a bad kind, a
 * non-positive grid or iters, or a null sink. */
es_status es_alu_peak(int kind, int grid, int iters, double* sink, void* stream);
long long es_alu_peak_flops(int kind, int grid, int iters);

/* Reads and clears the sticky device status (synchronises the stream):
 * *flags = bit 0 non-physical state, bit 1 timeout. */
es_status es_poll_status(es_ctx* ctx, int* flags, void* stream);

#ifdef __cplusplus
}
#endif
#endif
