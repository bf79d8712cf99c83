/*
 * FP64 CPU oracle for the entropy-stable adaptive moving-mesh finite-difference
 * method (arXiv 2202.07989).  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the benchmark's CPU-baseline leg call it; the product library never
 * does, and this code shares nothing with it.
 *
 * Plain, slow, obviously-correct C99, compiled with -O2 -ffp-contract=off.
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or garbled the reading taken is stated beside the code.
 *
 * Grid: d in {2,3} computational directions, n[k] nodes per direction at the
 * cell centres xi_{k,i} = xi_lo[k] + (i + 1/2) dxi[k].  Fields are stored as
 * structure of arrays, field-major: a[f][i3][i2][i1], interior nodes only.
 * Conserved state U = (rho_1..rho_N, rho v_1..rho v_d, E), n_c = N + d + 1.
 */
#ifndef ES_ORACLE_H
#define ES_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_PERIODIC = 0, OR_BC_REFLECT = 1, OR_BC_INFLOW = 2, OR_BC_OUTFLOW = 3 };
enum { OR_SIG_RHO = 0, OR_SIG_RHO1 = 1, OR_SIG_RHO2 = 2, OR_SIG_P = 3, OR_SIG_Y2 = 4, OR_SIG_V1 = 5 };

typedef struct or_config {
    int d;                   /* 2 or 3 */
    int N;                   /* species, 1 or 2 */
    int n[3];                /* nodes per direction; n[2] = 1 when d = 2 */
    int w;                   /* EC flux order 2w, w in {1,2,3} */
    int es;                  /* 1: add the WENO-MR dissipation, 0: pure EC */
    double xi_lo[3];         /* lower corner of the computational box */
    double dxi[3];           /* node spacing; box length is n[k]*dxi[k] */
    int bc[3][2];            /* OR_BC_* per direction and side */
    double inflow[3][2][8];  /* conserved state on inflow sides */
    double gamma[2], cv[2], pinf[2];
    double chi[3];           /* WENO-MR linear weights */
    double weno_eps;         /* WENO-MR epsilon */
    double cfl;              /* CFL number */
    int n_sigma;             /* monitor variables, <= 4 */
    int sigma[4];            /* OR_SIG_* */
    double alpha[4];         /* monitor weights */
    int mu;                  /* Jacobi sweeps per step */
    int nf;                  /* low-pass filter passes per step */
    double y_band;           /* sign band of [[W_m]] in Y relative to its round-off scale; 0 = 1e-12 */
    int weno;                /* 0: WENO-MR (Appendix A), 1: classical fifth-order WENO-JS */
    int sigma_op[4];         /* per monitor term: OR_MON_GRAD2 (Eq. (monitor)), OR_MON_GRAD, OR_MON_LAP */
} or_config;

/* monitor terms: alpha (|grad_xi sigma| / max)^2 as in Eq. (monitor); alpha |grad_xi sigma| / max
   and alpha |Laplacian_xi sigma| / max as in the vortex monitor of Example 5.1 */
enum { OR_MON_GRAD2 = 0, OR_MON_GRAD = 1, OR_MON_LAP = 2 };

int    or_nc(const or_config* c);

/* schlieren function of Example 5.8, Eq. (schlieren): Phi = exp(-Psi |grad rho| / max |grad rho|),
   Psi = (psi1 rho_1 + psi2 rho_2) / rho, grad the physical gradient (1/J) sum_k J xi_k/x
   d rho/d xi_k with second-order central differences in xi; Phi = 1 where max |grad rho| = 0 */
void   or_schlieren(const or_config* c, const double* JU, const double* J, const double* x, double psi1, double psi2,
                    double* phi);
long   or_ncell(const or_config* c);
long   or_npad(const or_config* c);

/* alpha_{w,m}, m = 1..w (Sec. 3.1, the linear conditions below Eq. (ECFlux_curv_2p)) */
void   or_alpha(int w, double* alpha);

/* physics of one node state U (Sec. 1, Eq. (StiffenedEOS); Sec. 3.3) */
void   or_primitives(const or_config* c, const double* U, double* rho_l, double* v, double* T, double* p);
void   or_entropy_vars(const or_config* c, const double* U, double* V);
double or_eta(const or_config* c, const double* U);
double or_phi(const or_config* c, const double* U);
void   or_phys_flux(const or_config* c, int j, const double* U, double* F);
void   or_prim_to_cons(const or_config* c, const double* rho_l, const double* v, double p, double* U);

/* two-point entropy-conservative flux (Sec. 3.3) */
double or_logmean(double a, double b);
void   or_Utilde(const or_config* c, const double* Ul, const double* Ur, double* out);
void   or_Ftilde(const or_config* c, int j, const double* Ul, const double* Ur, double* out);
void   or_ec_pair(const or_config* c, const double* Ul, const double* Ur,
                  const double* Ml, const double* Mr, double* out);

/* scaled eigenvectors at a point state in the frame of direction 1 (Sec. 3.4) */
void   or_eigvec_point(const or_config* c, const double* U, double* R);
/* the same built from the averaged values at an interface (Sec. 3.4) */
void   or_eigvec_avg(const or_config* c, const double* Ul, const double* Ur, double* R, double* cbar);

/* fifth-order multi-resolution WENO value at x_{j+1/2} from W_{j-2..j+2} (Appendix A) */
double or_weno_mr(const double* w5, const double* chi, double eps);
/* classical fifth-order WENO (Jiang and Shu, cited in Sec. 3.4 and Sec. 5 for the
   MM-WENOJS comparison) at x_{j+1/2} from W_{j-2..j+2}, with the same epsilon */
double or_weno_js(const double* w5, double eps);

/* geometry (Sec. 3.2) */
void   or_metrics(const or_config* c, const double* x, const double* xdot, double* M);
void   or_init_J(const or_config* c, const double* x, double* J);

/* semi-discrete residual, Eqs. (semi_U), (semi_J) */
void   or_rhs(const or_config* c, const double* JU, const double* J, const double* x,
              const double* xdot, double* dJU, double* dJ);
/* the residual and, per node, the smallest distance (in decades) of a Y decision from the
 * round-off band |[[W_m]]| = 1e-12 ||r_m|| (||V_i|| + ||V_i+1||) over its interfaces; near 0
 * means that rounding can decide Y */
void   or_rhs_margins(const or_config* c, const double* JU, const double* J, const double* x,
                      const double* xdot, double* dJU, double* dJ, double* node_margin);
/* one SSP-RK3 step on (JU, J, x) with a constant mesh velocity */
void   or_rk_step(const or_config* c, double* JU, double* J, double* x, const double* xdot, double dt);

/* time step (Eq. (cfl)) and mesh redistribution (Sec. 4) */
double or_cfl_dt(const or_config* c, const double* JU, const double* J, const double* x);
void   or_monitor(const or_config* c, const double* JU, const double* J, double* theta);
void   or_filter(const or_config* c, double* theta);
void   or_jacobi(const or_config* c, const double* x, const double* theta, double* xmu);
double or_limiter(const or_config* c, const double* x, const double* xmu);
void   or_mesh_redistribute(const or_config* c, const double* JU, const double* J, const double* x,
                            double dt_in, double* xdot, double* dt_dtau);

/* total-entropy diagnostics: out[0] = P = sum dxi^d (V.dJU - phi dJ), out[1] = sum J eta dxi^d */
void   or_entropy(const or_config* c, const double* JU, const double* J,
                  const double* dJU, const double* dJ, double* out);

#ifdef __cplusplus
}
#endif
#endif
