/*
 * FP64 CPU oracle for the entropy-stable adaptive moving-mesh finite-difference
 * method of arXiv 2202.07989.  TEST INFRASTRUCTURE: only the tests, the smoke
 * check and the benchmark's CPU-baseline leg use it.  It shares no code with
 * the CUDA library.  See es_oracle.h for the data layout.
 *
 * Readings of points the paper leaves open:
 *  - nodes sit at cell centres, dxi = box length / n (Sec. 3 puts nodes on both
 *    ends; the workloads count cells);
 *  - ghost nodes: periodic sides wrap (x shifted by the box length), all other
 *    sides mirror x about the wall; U is wrapped (periodic), mirrored with the
 *    wall-normal momentum negated (reflect), copied from the boundary node
 *    (outflow) or set to a fixed state (inflow);
 *  - logarithmic mean: the paper's [[a]]/[[ln a]] (Sec. 3.3), with the
 *    Ismail-Roe series when u = ((b-a)/(b+a))^2 < 1e-4;
 *  - the dissipation uses the 2w-order GCL flux values as interface metrics;
 *  - the rotation is built from the unit normal directly;
 *  - W_j = R^T T V_j with R and T frozen at the interface;
 *  - WENO-MR acts on point values; beta_2, beta_3 are the closed forms of
 *    Appendix A (they equal the integrals over the central cell);
 *  - mesh velocity is constant over a time step; the stage meshes come from
 *    the same SSP-RK3 combination as (JU, J);
 *  - CFL spectral radius (|n.v| + c) L / J at x^n, mesh velocity excluded;
 *  - sign matrix Y: a jump [[W_m]] within 1e-12 of its round-off scale
 *    ||r_m|| (||V_i|| + ||V_i+1||) has no sign (Y = 0), as an exactly zero jump;
 *  - initial Jacobian: determinant of the delta-derivative matrix.
 */
#include "es_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXC 8   /* max conserved components (N + d + 1 <= 6) */
#define OR_Y_ROUNDOFF (c->y_band > 0.0 ? c->y_band : 1.0e-12)   /* sign band of [[W_m]] in Y */

/* ------------------------------------------------------------------------ */
/* sizes and indexing                                                        */
/* ------------------------------------------------------------------------ */

int or_nc(const or_config* c) { return c->N + c->d + 1; }

long or_ncell(const or_config* c) { return (long)c->n[0] * c->n[1] * (c->d == 3 ? c->n[2] : 1); }

static int pad_of(const or_config* c, int k) { return k < c->d ? 3 : 0; }

long or_npad(const or_config* c)
{
    long p = 1;
    for (int k = 0; k < 3; ++k) p *= (k < c->d ? c->n[k] + 6 : 1);
    return p;
}

static long idx_of(const or_config* c, const int* i)
{
    int n3 = c->d == 3 ? i[2] : 0;
    return ((long)n3 * c->n[1] + i[1]) * c->n[0] + i[0];
}

static long pidx_of(const or_config* c, const int* i)
{
    long P0 = c->n[0] + 6, P1 = c->n[1] + 6;
    long i2 = c->d == 3 ? i[2] + 3 : 0;
    return (i2 * P1 + (i[1] + 3)) * P0 + (i[0] + 3);
}

static double box_len(const or_config* c, int k) { return c->n[k] * c->dxi[k]; }

static int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

/* ------------------------------------------------------------------------ */
/* alpha_{w,m}: sum_m m alpha = 1, sum_m m^{2s-1} alpha = 0 (s = 2..w),       */
/* Sec. 3.1.  Solved by Gaussian elimination with partial pivoting.          */
/* ------------------------------------------------------------------------ */

void or_alpha(int w, double* alpha)
{
    double A[3][4];
    for (int s = 1; s <= w; ++s) {
        for (int m = 1; m <= w; ++m) A[s - 1][m - 1] = pow((double)m, 2.0 * s - 1.0);
        A[s - 1][w] = (s == 1) ? 1.0 : 0.0;
    }
    for (int col = 0; col < w; ++col) {
        int piv = col;
        for (int r = col + 1; r < w; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int q = 0; q <= w; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int r = 0; r < w; ++r) {
            if (r == col) continue;
            double f = A[r][col] / A[col][col];
            for (int q = col; q <= w; ++q) A[r][q] -= f * A[col][q];
        }
    }
    for (int m = 0; m < w; ++m) alpha[m] = A[m][w] / A[m][m];
}

/* ------------------------------------------------------------------------ */
/* physics: stiffened-gas mixture, Sec. 1 Eq. (StiffenedEOS)                 */
/* ------------------------------------------------------------------------ */

static double Rsp(const or_config* c, int l) { return c->cv[l] * (c->gamma[l] - 1.0); }

static double pinf_tot(const or_config* c)
{
    double s = 0.0;
    for (int l = 0; l < c->N; ++l) s += c->pinf[l];
    return s;
}

void or_primitives(const or_config* c, const double* U, double* rho_l, double* v, double* T, double* p)
{
    int N = c->N, d = c->d;
    double rho = 0.0, cvr = 0.0, rr = 0.0;
    for (int l = 0; l < N; ++l) {
        rho_l[l] = U[l];
        rho += U[l];
        cvr += c->cv[l] * U[l];
        rr += Rsp(c, l) * U[l];
    }
    double v2 = 0.0;
    for (int m = 0; m < d; ++m) { v[m] = U[N + m] / rho; v2 += v[m] * v[m]; }
    double rhoe = U[N + d] - 0.5 * rho * v2;
    *T = (rhoe - pinf_tot(c)) / cvr;
    *p = rr * (*T) - pinf_tot(c);
}

void or_prim_to_cons(const or_config* c, const double* rho_l, const double* v, double p, double* U)
{
    int N = c->N, d = c->d;
    double rho = 0.0, cvr = 0.0, rr = 0.0, v2 = 0.0;
    for (int l = 0; l < N; ++l) { rho += rho_l[l]; cvr += c->cv[l] * rho_l[l]; rr += Rsp(c, l) * rho_l[l]; U[l] = rho_l[l]; }
    double T = (p + pinf_tot(c)) / rr;
    for (int m = 0; m < d; ++m) { U[N + m] = rho * v[m]; v2 += v[m] * v[m]; }
    U[N + d] = cvr * T + pinf_tot(c) + 0.5 * rho * v2;
}

/* entropy variables V = eta'(U): Sec. 3.3.1 (N = 1) and Sec. 3.3.2 (N = 2) */
void or_entropy_vars(const or_config* c, const double* U, double* V)
{
    int N = c->N, d = c->d;
    double rl[2], v[3], T, p;
    or_primitives(c, U, rl, v, &T, &p);
    double v2 = 0.0;
    for (int m = 0; m < d; ++m) v2 += v[m] * v[m];
    for (int l = 0; l < N; ++l) {
        double S = c->cv[l] * log(T) - Rsp(c, l) * log(rl[l]);
        V[l] = -S - v2 / (2.0 * T) + c->cv[l] * c->gamma[l];
    }
    for (int m = 0; m < d; ++m) V[N + m] = v[m] / T;
    V[N + d] = -1.0 / T;
}

/* eta = -sum_l rho_l S_l, S_l = c_{v,l} ln T - R_l ln rho_l (Eqs. (entropypair-1D), (entropypair)) */
double or_eta(const or_config* c, const double* U)
{
    double rl[2], v[3], T, p, e = 0.0;
    or_primitives(c, U, rl, v, &T, &p);
    for (int l = 0; l < c->N; ++l) e -= rl[l] * (c->cv[l] * log(T) - Rsp(c, l) * log(rl[l]));
    return e;
}

/* phi = sum_l (R_l rho_l - p_{inf,l}/T), Eqs. (potentialN1), (potentialN2) */
double or_phi(const or_config* c, const double* U)
{
    double rl[2], v[3], T, p, s = 0.0;
    or_primitives(c, U, rl, v, &T, &p);
    for (int l = 0; l < c->N; ++l) s += Rsp(c, l) * rl[l] - c->pinf[l] / T;
    return s;
}

/* physical flux F_j of Eq. (ConserLaw) */
void or_phys_flux(const or_config* c, int j, const double* U, double* F)
{
    int N = c->N, d = c->d;
    double rl[2], v[3], T, p, rho = 0.0;
    or_primitives(c, U, rl, v, &T, &p);
    for (int l = 0; l < N; ++l) { F[l] = rl[l] * v[j]; rho += rl[l]; }
    for (int m = 0; m < d; ++m) F[N + m] = rho * v[m] * v[j] + (m == j ? p : 0.0);
    F[N + d] = (U[N + d] + p) * v[j];
}

/* ------------------------------------------------------------------------ */
/* two-point EC flux, Sec. 3.3                                                */
/* ------------------------------------------------------------------------ */

/* {a}^ln = [[a]] / [[ln a]] (Sec. 3.3.1); for small jumps the Ismail-Roe
 * series in u = f^2, f = (b - a)/(b + a):  {a}^ln = {a} / (1 + u/3 + u^2/5 + u^3/7). */
double or_logmean(double a, double b)
{
    double f = (b - a) / (b + a);
    double u = f * f;
    if (u < 1.0e-4) return 0.5 * (a + b) / (1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0);
    return (b - a) / (log(b) - log(a));
}

/* the means of the parameter vector z = (rho_1..rho_N, v, 1/T) used by
 * U-tilde and F-tilde */
typedef struct {
    double lnrho[2], arho[2];  /* log and arithmetic means of rho_l */
    double vm[3], v2m[3];      /* {v_m}, {v_m^2} */
    double lnb, ab;            /* log and arithmetic means of beta = 1/T */
} or_means;

static void z_means(const or_config* c, const double* Ul, const double* Ur, or_means* M)
{
    double rl[2], vl[3], Tl, pl, rr_[2], vr[3], Tr, pr;
    or_primitives(c, Ul, rl, vl, &Tl, &pl);
    or_primitives(c, Ur, rr_, vr, &Tr, &pr);
    for (int l = 0; l < c->N; ++l) {
        M->lnrho[l] = or_logmean(rl[l], rr_[l]);
        M->arho[l] = 0.5 * (rl[l] + rr_[l]);
    }
    for (int m = 0; m < c->d; ++m) {
        M->vm[m] = 0.5 * (vl[m] + vr[m]);
        M->v2m[m] = 0.5 * (vl[m] * vl[m] + vr[m] * vr[m]);
    }
    M->lnb = or_logmean(1.0 / Tl, 1.0 / Tr);
    M->ab = 0.5 * (1.0 / Tl + 1.0 / Tr);
}

/* U-tilde: the closed forms of Sec. 3.3.1 (N = 1) and 3.3.2 (N = 2) */
void or_Utilde(const or_config* c, const double* Ul, const double* Ur, double* out)
{
    int N = c->N, d = c->d;
    or_means M;
    z_means(c, Ul, Ur, &M);
    double sumr = 0.0, hv2 = 0.0, vv = 0.0, e = 0.0;
    for (int l = 0; l < N; ++l) sumr += M.lnrho[l];
    for (int m = 0; m < d; ++m) { hv2 += 0.5 * M.v2m[m]; vv += M.vm[m] * M.vm[m]; }
    for (int l = 0; l < N; ++l) out[l] = M.lnrho[l];
    for (int m = 0; m < d; ++m) out[N + m] = M.vm[m] * sumr;
    for (int l = 0; l < N; ++l) e += M.lnrho[l] * (c->cv[l] / M.lnb - hv2);
    out[N + d] = e + sumr * vv + pinf_tot(c);
}

/* F-tilde_j: the closed forms of F-tilde_1 with the roles of v_1 and v_j
 * exchanged, which is the rotation of Eq. (rotation) by (phi, theta) =
 * (0, pi/2) for j = 2 and (pi/2, 0) for j = 3. */
void or_Ftilde(const or_config* c, int j, const double* Ul, const double* Ur, double* out)
{
    int N = c->N, d = c->d;
    or_means M;
    z_means(c, Ul, Ur, &M);
    double sumF = 0.0, hv2 = 0.0, Rr = 0.0, e = 0.0;
    for (int l = 0; l < N; ++l) { out[l] = M.lnrho[l] * M.vm[j]; sumF += out[l]; Rr += Rsp(c, l) * M.arho[l]; }
    for (int m = 0; m < d; ++m) hv2 += 0.5 * M.v2m[m];
    for (int m = 0; m < d; ++m) out[N + m] = M.vm[m] * sumF + (m == j ? Rr / M.ab - pinf_tot(c) : 0.0);
    for (int l = 0; l < N; ++l) e += out[l] * (c->cv[l] / M.lnb - hv2);
    for (int m = 0; m < d; ++m) e += M.vm[m] * out[N + m];
    out[N + d] = e + pinf_tot(c) * M.vm[j];
}

/* curvilinear two-point flux, Eq. (ECfluxMM); M = (J xi_t, J xi_x1..xd) */
void or_ec_pair(const or_config* c, const double* Ul, const double* Ur,
                const double* Ml, const double* Mr, double* out)
{
    int nc = or_nc(c);
    double Ut[MAXC], Ft[MAXC];
    or_Utilde(c, Ul, Ur, Ut);
    double mt = 0.5 * (Ml[0] + Mr[0]);
    for (int q = 0; q < nc; ++q) out[q] = mt * Ut[q];
    for (int j = 0; j < c->d; ++j) {
        or_Ftilde(c, j, Ul, Ur, Ft);
        double mj = 0.5 * (Ml[1 + j] + Mr[1 + j]);
        for (int q = 0; q < nc; ++q) out[q] += mj * Ft[q];
    }
}

/* ------------------------------------------------------------------------ */
/* scaled eigenvectors, Sec. 3.4                                              */
/* ------------------------------------------------------------------------ */

/* thermodynamic inputs of R: density(ies), velocity, temperature and the
 * mixture quantities built from them */
typedef struct {
    double rho, rl[2], v[3], T;
    double Rmix, Gmix;       /* R = sum (G_l - 1) cv_l rho_l / rho, Gamma of Sec. 1 */
    double H;                /* total enthalpy */
    double Y[2];
} or_eig_in;

/* R = R-tilde * diag(scales) for N = 1; R = R-tilde * D for N = 2 (Sec. 3.4).
 * Columns: acoustic(-), species/entropy, shear for m = 2..d, acoustic(+). */
static void build_R(const or_config* c, const or_eig_in* s, double* R)
{
    int N = c->N, d = c->d, nc = N + d + 1;
    double v2 = 0.0;
    for (int m = 0; m < d; ++m) v2 += s->v[m] * s->v[m];
    double cs = sqrt(s->Rmix * s->Gmix * s->T);
    double Rt[MAXC][MAXC];
    memset(Rt, 0, sizeof(Rt));
    int cm = 0, cp = nc - 1;
    /* acoustic columns */
    for (int l = 0; l < N; ++l) { Rt[l][cm] = (N == 1) ? 1.0 : s->Y[l]; Rt[l][cp] = (N == 1) ? 1.0 : s->Y[l]; }
    for (int m = 0; m < d; ++m) { Rt[N + m][cm] = s->v[m]; Rt[N + m][cp] = s->v[m]; }
    Rt[N][cm] -= cs;
    Rt[N][cp] += cs;
    Rt[N + d][cm] = s->H - cs * s->v[0];
    Rt[N + d][cp] = s->H + cs * s->v[0];
    /* species / entropy columns 1..N */
    for (int l = 0; l < N; ++l) {
        int col = 1 + l;
        for (int q = 0; q < N; ++q) Rt[q][col] = (q == l) ? 1.0 : 0.0;
        for (int m = 0; m < d; ++m) Rt[N + m][col] = s->v[m];
        if (N == 1) {
            Rt[N + d][col] = 0.5 * v2;
        } else {
            double hl = (c->cv[l] + Rsp(c, l)) * s->T;
            double dl = hl - s->Gmix * c->cv[l] * s->T;
            Rt[N + d][col] = 0.5 * v2 - dl / (s->Gmix - 1.0);
        }
    }
    /* shear columns for velocity components 2..d */
    for (int m = 1; m < d; ++m) {
        int col = N + m;
        double sc = (N == 1) ? 1.0 : cs;
        Rt[N + m][col] = sc;
        Rt[N + d][col] = sc * s->v[m];
    }
    /* scaling */
    double Dm[MAXC][MAXC];
    memset(Dm, 0, sizeof(Dm));
    if (N == 1) {
        double G = c->gamma[0], Rg = Rsp(c, 0), cv = c->cv[0];
        double ac = sqrt(s->rho / (2.0 * G * Rg));
        Dm[cm][cm] = ac;
        Dm[cp][cp] = ac;
        Dm[1][1] = sqrt(s->rho / (cv * G));
        for (int m = 1; m < d; ++m) Dm[N + m][N + m] = sqrt(s->rho * s->T);
    } else {
        double G = s->Gmix, pre = sqrt(s->rho / (s->Gmix * s->Rmix));
        double R1 = Rsp(c, 0), R2 = Rsp(c, 1), Y1 = s->Y[0], Y2 = s->Y[1];
        Dm[cm][cm] = pre / sqrt(2.0);
        Dm[cp][cp] = pre / sqrt(2.0);
        Dm[1][1] = -pre * sqrt(Y1 * Y2) * sqrt(G * R2 / R1);
        Dm[1][2] = pre * Y1 * sqrt(G - 1.0);
        Dm[2][1] = pre * sqrt(Y1 * Y2) * sqrt(G * R1 / R2);
        Dm[2][2] = pre * Y2 * sqrt(G - 1.0);
        for (int m = 1; m < d; ++m) Dm[N + m][N + m] = pre;
    }
    for (int r = 0; r < nc; ++r)
        for (int q = 0; q < nc; ++q) {
            double acc = 0.0;
            for (int t = 0; t < nc; ++t) acc += Rt[r][t] * Dm[t][q];
            R[r * nc + q] = acc;
        }
}

static void mixture(const or_config* c, const double* rl, double* Rmix, double* Gmix)
{
    double rho = 0.0, a = 0.0, g = 0.0, cvr = 0.0;
    for (int l = 0; l < c->N; ++l) {
        rho += rl[l];
        a += (c->gamma[l] - 1.0) * c->cv[l] * rl[l];
        g += c->gamma[l] * c->cv[l] * rl[l];
        cvr += c->cv[l] * rl[l];
    }
    *Rmix = a / rho;
    *Gmix = g / cvr;
}

void or_eigvec_point(const or_config* c, const double* U, double* R)
{
    or_eig_in s;
    double p;
    or_primitives(c, U, s.rl, s.v, &s.T, &p);
    s.rho = 0.0;
    for (int l = 0; l < c->N; ++l) s.rho += s.rl[l];
    for (int l = 0; l < c->N; ++l) s.Y[l] = s.rl[l] / s.rho;
    mixture(c, s.rl, &s.Rmix, &s.Gmix);
    s.H = (U[c->N + c->d] + p) / s.rho;
    build_R(c, &s, R);
}

/* interface averages of Sec. 3.4: N = 1 uses {rho}^ln, {v} and
 * p + p_inf = {rho}^ln / {rho/(p + p_inf)}^ln; N = 2 uses {rho_l}^ln,
 * {rho}^ln, {v}, T = 1/{1/T}^ln, {R}, {Gamma} and
 * sum rho_l h_l = sum (cv_l rho_l T + p_inf_l) + {p}; Y_l = rho_l/rho. */
void or_eigvec_avg(const or_config* c, const double* Ul, const double* Ur, double* R, double* cbar)
{
    int N = c->N, d = c->d;
    double rl[2], vl[3], Tl, pl, rr_[2], vr[3], Tr, pr;
    or_primitives(c, Ul, rl, vl, &Tl, &pl);
    or_primitives(c, Ur, rr_, vr, &Tr, &pr);
    or_eig_in s;
    double v2 = 0.0;
    for (int m = 0; m < d; ++m) { s.v[m] = 0.5 * (vl[m] + vr[m]); v2 += s.v[m] * s.v[m]; }
    if (N == 1) {
        double pi = c->pinf[0], Rg = Rsp(c, 0);
        s.rho = or_logmean(rl[0], rr_[0]);
        s.rl[0] = s.rho;
        double ppi = s.rho / or_logmean(rl[0] / (pl + pi), rr_[0] / (pr + pi));
        s.T = ppi / (Rg * s.rho);
        s.Rmix = Rg;
        s.Gmix = c->gamma[0];
        s.Y[0] = 1.0;
        s.H = c->gamma[0] * c->cv[0] * s.T + 0.5 * v2;
    } else {
        double rhol = rl[0] + rl[1], rhor = rr_[0] + rr_[1];
        for (int l = 0; l < 2; ++l) s.rl[l] = or_logmean(rl[l], rr_[l]);
        s.rho = or_logmean(rhol, rhor);
        s.T = 1.0 / or_logmean(1.0 / Tl, 1.0 / Tr);
        double Rl_, Gl_, Rr_, Gr_;
        mixture(c, rl, &Rl_, &Gl_);
        mixture(c, rr_, &Rr_, &Gr_);
        s.Rmix = 0.5 * (Rl_ + Rr_);
        s.Gmix = 0.5 * (Gl_ + Gr_);
        double rh = 0.5 * (pl + pr);
        for (int l = 0; l < 2; ++l) rh += c->cv[l] * s.rl[l] * s.T + c->pinf[l];
        for (int l = 0; l < 2; ++l) s.Y[l] = s.rl[l] / s.rho;
        s.H = rh / s.rho + 0.5 * v2;
    }
    build_R(c, &s, R);
    if (cbar) *cbar = sqrt(s.Rmix * s.Gmix * s.T);
}

/* ------------------------------------------------------------------------ */
/* fifth-order multi-resolution WENO, Appendix A                              */
/* ------------------------------------------------------------------------ */

/* Classical fifth-order WENO at x_{j+1/2}.  Three quadratic reconstructions on the
 * cells {j-2,j-1,j}, {j-1,j,j+1}, {j,j+1,j+2} give the candidate values q_k; the
 * smoothness indicator of each is the sum over the first two derivatives of the
 * squared derivative integrated over cell j (scaled by the cell width); the linear
 * weights 1/10, 6/10, 3/10 make the combination the five-cell value; the nonlinear
 * weights are d_k / (eps + beta_k)^2, normalised. */
double or_weno_js(const double* w5, double eps)
{
    double Wm2 = w5[0], Wm1 = w5[1], W0 = w5[2], Wp1 = w5[3], Wp2 = w5[4];
    double q[3], beta[3], a[3];
    const double d[3] = { 0.1, 0.6, 0.3 };
    q[0] = (2.0 * Wm2 - 7.0 * Wm1 + 11.0 * W0) / 6.0;
    q[1] = (-Wm1 + 5.0 * W0 + 2.0 * Wp1) / 6.0;
    q[2] = (2.0 * W0 + 5.0 * Wp1 - Wp2) / 6.0;
    beta[0] = 13.0 / 12.0 * (Wm2 - 2.0 * Wm1 + W0) * (Wm2 - 2.0 * Wm1 + W0)
            + 0.25 * (Wm2 - 4.0 * Wm1 + 3.0 * W0) * (Wm2 - 4.0 * Wm1 + 3.0 * W0);
    beta[1] = 13.0 / 12.0 * (Wm1 - 2.0 * W0 + Wp1) * (Wm1 - 2.0 * W0 + Wp1)
            + 0.25 * (Wm1 - Wp1) * (Wm1 - Wp1);
    beta[2] = 13.0 / 12.0 * (W0 - 2.0 * Wp1 + Wp2) * (W0 - 2.0 * Wp1 + Wp2)
            + 0.25 * (3.0 * W0 - 4.0 * Wp1 + Wp2) * (3.0 * W0 - 4.0 * Wp1 + Wp2);
    double as = 0.0, num = 0.0;
    for (int k = 0; k < 3; ++k) {
        a[k] = d[k] / ((eps + beta[k]) * (eps + beta[k]));
        as += a[k];
        num += a[k] * q[k];
    }
    return num / as;
}

double or_weno_mr(const double* w5, const double* chi, double eps)
{
    double Wm2 = w5[0], Wm1 = w5[1], W0 = w5[2], Wp1 = w5[3], Wp2 = w5[4];
    /* Legendre coefficients of h_2 and h_3 (step 1) */
    double a2 = 0.5 * (Wp1 - Wm1);
    double a3 = 0.5 * (Wm1 - 2.0 * W0 + Wp1);
    double b2 = (11.0 * Wm2 - 82.0 * Wm1 + 82.0 * Wp1 - 11.0 * Wp2) / 120.0;
    double b3 = (-3.0 * Wm2 + 40.0 * Wm1 - 74.0 * W0 + 40.0 * Wp1 - 3.0 * Wp2) / 56.0;
    double b4 = (-Wm2 + 2.0 * Wm1 - 2.0 * Wp1 + Wp2) / 12.0;
    double b5 = (Wm2 - 4.0 * Wm1 + 6.0 * W0 - 4.0 * Wp1 + Wp2) / 24.0;
    /* smoothness indicators (step 2) */
    double d0 = (W0 - Wm1) * (W0 - Wm1), d1 = (Wp1 - W0) * (Wp1 - W0);
    double beta1 = d0 < d1 ? d0 : d1;
    double beta2 = a2 * a2 + 13.0 / 3.0 * a3 * a3;
    double t1 = b2 + b4 / 10.0, t2 = b3 + 123.0 / 455.0 * b5;
    double beta3 = t1 * t1 + 13.0 / 3.0 * t2 * t2 + 781.0 / 20.0 * b4 * b4 + 1421461.0 / 2275.0 * b5 * b5;
    /* nonlinear weights (step 3) */
    double tau = 0.5 * (fabs(beta3 - beta1) + fabs(beta3 - beta2));
    tau = tau * tau;
    double wb1 = chi[0] * (1.0 + tau / (eps + beta1));
    double wb2 = chi[1] * (1.0 + tau / (eps + beta2));
    double wb3 = chi[2] * (1.0 + tau / (eps + beta3));
    double ws = wb1 + wb2 + wb3;
    double om1 = wb1 / ws, om2 = wb2 / ws, om3 = wb3 / ws;
    /* h_m at x_{j+1/2}: Legendre basis values 1, 1/2, 1/6, 1/20, 1/70 (step 4) */
    double h1 = W0;
    double h2 = W0 + a2 / 2.0 + a3 / 6.0;
    double h3 = W0 + b2 / 2.0 + b3 / 6.0 + b4 / 20.0 + b5 / 70.0;
    return om1 * h1 + om2 * h2 + om3 * (h3 / chi[2] - chi[0] / chi[2] * h1 - chi[1] / chi[2] * h2);
}

/* ------------------------------------------------------------------------ */
/* ghost-node mappings                                                       */
/* ------------------------------------------------------------------------ */

/* mesh position (and velocity) at any node index: periodic sides wrap and
 * shift x_k by the box length, all other sides mirror about the wall. */
static void x_at(const or_config* c, const double* x, const int* i_in, double* out, int is_velocity)
{
    int d = c->d, i[3] = { i_in[0], i_in[1], d == 3 ? i_in[2] : 0 };
    double shift[3] = { 0, 0, 0 };
    int flip[3] = { 0, 0, 0 };
    double wall[3] = { 0, 0, 0 };
    for (int k = 0; k < d; ++k) {
        int n = c->n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        int side = i[k] < 0 ? 0 : 1;
        if (c->bc[k][side] == OR_BC_PERIODIC) {
            int s = floordiv(i[k], n);
            i[k] -= s * n;
            shift[k] = s * box_len(c, k);
        } else {
            i[k] = side == 0 ? -1 - i[k] : 2 * n - 1 - i[k];
            flip[k] = 1;
            wall[k] = side == 0 ? c->xi_lo[k] : c->xi_lo[k] + box_len(c, k);
        }
    }
    long id = idx_of(c, i), nn = or_ncell(c);
    for (int j = 0; j < d; ++j) out[j] = x[j * nn + id];
    for (int k = 0; k < d; ++k) {
        if (is_velocity) {
            if (flip[k]) out[k] = -out[k];
        } else {
            if (flip[k]) out[k] = 2.0 * wall[k] - out[k];
            out[k] += shift[k];
        }
    }
}

/* conserved point state U = JU/J at any node reached along the grid lines */
static void U_at(const or_config* c, const double* JU, const double* J, const int* i_in, double* U)
{
    int N = c->N, d = c->d, nc = or_nc(c);
    int i[3] = { i_in[0], i_in[1], d == 3 ? i_in[2] : 0 };
    int neg[3] = { 0, 0, 0 };
    for (int k = 0; k < d; ++k) {
        int n = c->n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        int side = i[k] < 0 ? 0 : 1;
        switch (c->bc[k][side]) {
        case OR_BC_PERIODIC: i[k] -= floordiv(i[k], n) * n; break;
        case OR_BC_REFLECT: i[k] = side == 0 ? -1 - i[k] : 2 * n - 1 - i[k]; neg[k] = 1; break;
        case OR_BC_OUTFLOW: i[k] = side == 0 ? 0 : n - 1; break;
        default: /* inflow: fixed state */
            for (int q = 0; q < nc; ++q) U[q] = c->inflow[k][side][q];
            return;
        }
    }
    long id = idx_of(c, i), nn = or_ncell(c);
    for (int q = 0; q < nc; ++q) U[q] = JU[q * nn + id] / J[id];
    for (int k = 0; k < d; ++k)
        if (neg[k]) U[N + k] = -U[N + k];
}

/* scalar node field with periodic wrap, else copy of the boundary node */
static double s_at(const or_config* c, const double* a, const int* i_in)
{
    int i[3] = { i_in[0], i_in[1], c->d == 3 ? i_in[2] : 0 };
    for (int k = 0; k < c->d; ++k) {
        int n = c->n[k];
        if (i[k] >= 0 && i[k] < n) continue;
        int side = i[k] < 0 ? 0 : 1;
        if (c->bc[k][side] == OR_BC_PERIODIC) i[k] -= floordiv(i[k], n) * n;
        else i[k] = side == 0 ? 0 : n - 1;
    }
    return a[idx_of(c, i)];
}

/* ------------------------------------------------------------------------ */
/* metrics, Sec. 3.2: Eq. (SCLCoeff) and its cyclic permutations, Eq. (VCLCoeff) */
/* ------------------------------------------------------------------------ */

/* delta_k[x_p] at node i: (1/2) sum_m alpha_m (x_p(i + m e_k) - x_p(i - m e_k)) */
static double delta_x(const or_config* c, const double* x, const double* alpha, const int* i, int k, int p)
{
    double acc = 0.0, a[3], b[3];
    for (int m = 1; m <= c->w; ++m) {
        int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
        ip[k] += m;
        im[k] -= m;
        x_at(c, x, ip, a, 0);
        x_at(c, x, im, b, 0);
        acc += alpha[m - 1] * (a[p] - b[p]);
    }
    return 0.5 * acc;
}

/* delta_a[ delta_b[x_p] x_q ] at node i */
static double delta_nested(const or_config* c, const double* x, const double* alpha, const int* i,
                           int a, int b, int p, int q)
{
    double acc = 0.0, xa[3], xb[3];
    for (int m = 1; m <= c->w; ++m) {
        int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
        ip[a] += m;
        im[a] -= m;
        x_at(c, x, ip, xa, 0);
        x_at(c, x, im, xb, 0);
        acc += alpha[m - 1] * (delta_x(c, x, alpha, ip, b, p) * xa[q] - delta_x(c, x, alpha, im, b, p) * xb[q]);
    }
    return 0.5 * acc;
}

/* node metrics at node i: m[k][0] = J xi_k/t, m[k][1 + j] = J xi_k/x_j */
static void node_metrics(const or_config* c, const double* x, const double* xdot, const double* alpha,
                         const int* i, double m[3][4])
{
    int d = c->d;
    if (d == 2) {
        double d1x1 = delta_x(c, x, alpha, i, 0, 0), d1x2 = delta_x(c, x, alpha, i, 0, 1);
        double d2x1 = delta_x(c, x, alpha, i, 1, 0), d2x2 = delta_x(c, x, alpha, i, 1, 1);
        m[0][1] = d2x2 / c->dxi[1];
        m[0][2] = -d2x1 / c->dxi[1];
        m[1][1] = -d1x2 / c->dxi[0];
        m[1][2] = d1x1 / c->dxi[0];
    } else {
        /* J xi_k/x_j = (delta_a[delta_b[x_p] x_q] - delta_b[delta_a[x_p] x_q]) / (dxi_a dxi_b)
         * with (a, b) = (3,2), (1,3), (2,1) for k = 1, 2, 3 and
         * (p, q) = (2,3), (3,1), (1,2) for j = 1, 2, 3 (0-based below). */
        static const int ab[3][2] = { { 2, 1 }, { 0, 2 }, { 1, 0 } };
        static const int pq[3][2] = { { 1, 2 }, { 2, 0 }, { 0, 1 } };
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) {
                int a = ab[k][0], b = ab[k][1], p = pq[j][0], q = pq[j][1];
                double t = delta_nested(c, x, alpha, i, a, b, p, q) - delta_nested(c, x, alpha, i, b, a, p, q);
                m[k][1 + j] = t / (c->dxi[a] * c->dxi[b]);
            }
    }
    double xd[3] = { 0, 0, 0 };
    if (xdot) x_at(c, xdot, i, xd, 1);
    for (int k = 0; k < d; ++k) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s -= xd[j] * m[k][1 + j];
        m[k][0] = s;
    }
}

/* metrics at all nodes with up to 3 ghost layers per direction.  Output layout:
 * M[(k*(d+1) + c)][padded node], c = 0 for J xi_k/t and 1 + j for J xi_k/x_j. */
void or_metrics(const or_config* c, const double* x, const double* xdot, double* M)
{
    int d = c->d;
    double alpha[3];
    or_alpha(c->w, alpha);
    long np = or_npad(c);
    int lo2 = -pad_of(c, 2), hi2 = d == 3 ? c->n[2] + 3 : 1;
    int i[3];
    for (i[2] = lo2; i[2] < hi2; ++i[2])
        for (i[1] = -3; i[1] < c->n[1] + 3; ++i[1])
            for (i[0] = -3; i[0] < c->n[0] + 3; ++i[0]) {
                double m[3][4];
                node_metrics(c, x, xdot, alpha, i, m);
                long pid = pidx_of(c, i);
                for (int k = 0; k < d; ++k)
                    for (int q = 0; q <= d; ++q) M[(long)(k * (d + 1) + q) * np + pid] = m[k][q];
            }
}

/* J^0 = det(delta_k[x_j] / dxi_k) at the nodes */
void or_init_J(const or_config* c, const double* x, double* J)
{
    int d = c->d;
    double alpha[3];
    or_alpha(c->w, alpha);
    int i[3] = { 0, 0, 0 };
    int n2 = d == 3 ? c->n[2] : 1;
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                double A[3][3];
                for (int j = 0; j < d; ++j)
                    for (int k = 0; k < d; ++k) A[j][k] = delta_x(c, x, alpha, i, k, j) / c->dxi[k];
                double det;
                if (d == 2) det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
                else
                    det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                        - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                        + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
                J[idx_of(c, i)] = det;
            }
}

/* ------------------------------------------------------------------------ */
/* residual, Eqs. (semi_U), (semi_J), (ECFlux_curv_2p), (GCL_flux), (HOstable) */
/* ------------------------------------------------------------------------ */

/* expanded rotation T of Eq. (rotamatrix) acting on the velocity block, built
 * from the unit normal n: first row n, cos(theta) = n1/r, sin(theta) = n2/r,
 * cos(phi) = r, sin(phi) = n3 with r = sqrt(n1^2 + n2^2). */
static void rotation(int d, const double* n, double Tv[3][3])
{
    if (d == 2) {
        Tv[0][0] = n[0]; Tv[0][1] = n[1];
        Tv[1][0] = -n[1]; Tv[1][1] = n[0];
        return;
    }
    double r = sqrt(n[0] * n[0] + n[1] * n[1]);
    double ct = r > 0.0 ? n[0] / r : 1.0, st = r > 0.0 ? n[1] / r : 0.0;
    double cp = r, sp = n[2];
    Tv[0][0] = cp * ct;  Tv[0][1] = cp * st;  Tv[0][2] = sp;
    Tv[1][0] = -st;      Tv[1][1] = ct;       Tv[1][2] = 0.0;
    Tv[2][0] = -sp * ct; Tv[2][1] = -sp * st; Tv[2][2] = cp;
}

static void rotate(const or_config* c, double Tv[3][3], const double* a, double* out, int transpose)
{
    int N = c->N, d = c->d, nc = or_nc(c);
    for (int q = 0; q < nc; ++q) out[q] = a[q];
    for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s += (transpose ? Tv[j][m] : Tv[m][j]) * a[N + j];
        out[N + m] = s;
    }
}

/* dissipation term of Eq. (HOstable) at the interface between u6[2] and u6[3];
 * G = (J xi_t, J xi_x1..xd) from the GCL flux at that interface. */
static void dissipation(const or_config* c, double u6[6][MAXC], const double* G, double* D, double* margin)
{
    int d = c->d, N = c->N, nc = or_nc(c);
    double L = 0.0, n[3];
    for (int j = 0; j < d; ++j) L += G[1 + j] * G[1 + j];
    L = sqrt(L);
    for (int j = 0; j < d; ++j) n[j] = G[1 + j] / L;
    double Tv[3][3];
    rotation(d, n, Tv);
    double Ul[MAXC], Ur[MAXC], R[MAXC * MAXC], cbar;
    rotate(c, Tv, u6[2], Ul, 0);
    rotate(c, Tv, u6[3], Ur, 0);
    or_eigvec_avg(c, Ul, Ur, R, &cbar);
    double vhat1 = 0.5 * (Ul[N] / (Ul[0] + (N == 2 ? Ul[1] : 0.0)) + Ur[N] / (Ur[0] + (N == 2 ? Ur[1] : 0.0)));
    double lam = fabs(G[0] + L * vhat1) + L * cbar;
    /* scaled entropy variables W_j = R^T T V_j, j = i-2..i+3 */
    double W[6][MAXC];
    for (int j = 0; j < 6; ++j) {
        double V[MAXC], TV[MAXC];
        or_entropy_vars(c, u6[j], V);
        rotate(c, Tv, V, TV, 0);
        for (int m = 0; m < nc; ++m) {
            double s = 0.0;
            for (int q = 0; q < nc; ++q) s += R[q * nc + m] * TV[q];
            W[j][m] = s;
        }
    }
    /* round-off scale of [[W_m]]: ||r_m|| (||V_i|| + ||V_i+1||) (rotation invariant) */
    double nv = 0.0;
    {
        double Vi[MAXC], Vr[MAXC], a = 0.0, b = 0.0;
        or_entropy_vars(c, u6[2], Vi);
        or_entropy_vars(c, u6[3], Vr);
        for (int q = 0; q < nc; ++q) { a += Vi[q] * Vi[q]; b += Vr[q] * Vr[q]; }
        nv = sqrt(a) + sqrt(b);
    }
    double coef[MAXC];
    for (int m = 0; m < nc; ++m) {
        double wl[5] = { W[0][m], W[1][m], W[2][m], W[3][m], W[4][m] };
        double wr[5] = { W[5][m], W[4][m], W[3][m], W[2][m], W[1][m] };
        double Wminus = c->weno ? or_weno_js(wl, c->weno_eps) : or_weno_mr(wl, c->chi, c->weno_eps);
        double Wplus = c->weno ? or_weno_js(wr, c->weno_eps) : or_weno_mr(wr, c->chi, c->weno_eps);
        double jw = Wplus - Wminus, jump = W[3][m] - W[2][m];
        int sjw = (jw > 0) - (jw < 0), sj = (jump > 0) - (jump < 0);
        /* Y of Sec. 3.4: 1 when sign([[W_m]]^WENOMR) sign([[W_m]]) > 0.  A jump no larger
         * than OR_Y_ROUNDOFF times its round-off scale has no reliable sign and counts as 0
         * (zero jumps give Y = 0). */
        double rn = 0.0;
        for (int q = 0; q < nc; ++q) rn += R[q * nc + m] * R[q * nc + m];
        double scale = sqrt(rn) * nv;
        int sig = fabs(jump) > OR_Y_ROUNDOFF * scale;
        double Y = (sig && sjw * sj > 0) ? 1.0 : 0.0;
        coef[m] = lam * Y * jw;
        if (margin && scale > 0.0) {
            /* distance of the decision from the round-off band, in decades */
            double mg = fabs(log10(fabs(jump) / (OR_Y_ROUNDOFF * scale) + 1e-300));
            if (mg < *margin) *margin = mg;
        }
    }
    double Dh[MAXC];
    for (int q = 0; q < nc; ++q) {
        double s = 0.0;
        for (int m = 0; m < nc; ++m) s += R[q * nc + m] * coef[m];
        Dh[q] = s;
    }
    double Dr[MAXC];
    rotate(c, Tv, Dh, Dr, 1);
    for (int q = 0; q < nc; ++q) D[q] = -0.5 * Dr[q];
}

static void rhs_impl(const or_config* c, const double* JU, const double* J, const double* x,
                     const double* xdot, double* dJU, double* dJ, double* node_margin);

void or_rhs(const or_config* c, const double* JU, const double* J, const double* x,
            const double* xdot, double* dJU, double* dJ)
{
    rhs_impl(c, JU, J, x, xdot, dJU, dJ, NULL);
}

/* the residual plus, per node, the smallest relative magnitude |[[W_m]]| / (|W_m,i| + |W_m,i+1|)
 * over the interfaces around the node: where it is at round-off level the sign matrix Y
 * of Sec. 3.4 is decided by rounding (test diagnostics) */
void or_rhs_margins(const or_config* c, const double* JU, const double* J, const double* x,
                    const double* xdot, double* dJU, double* dJ, double* node_margin)
{
    rhs_impl(c, JU, J, x, xdot, dJU, dJ, node_margin);
}

static void rhs_impl(const or_config* c, const double* JU, const double* J, const double* x,
                     const double* xdot, double* dJU, double* dJ, double* node_margin)
{
    int d = c->d, nc = or_nc(c), w = c->w;
    long nn = or_ncell(c), np = or_npad(c);
    double alpha[3];
    or_alpha(w, alpha);
    double* M = (double*)malloc(sizeof(double) * (size_t)(d * (d + 1)) * (size_t)np);
    or_metrics(c, x, xdot, M);
    memset(dJU, 0, sizeof(double) * (size_t)nc * (size_t)nn);
    memset(dJ, 0, sizeof(double) * (size_t)nn);
    int n2 = d == 3 ? c->n[2] : 1;
    int nmax = c->n[0] > c->n[1] ? c->n[0] : c->n[1];
    if (n2 > nmax) nmax = n2;
    double* F = (double*)malloc(sizeof(double) * (size_t)(nmax + 1) * nc);
    double* G = (double*)malloc(sizeof(double) * (size_t)(nmax + 1));
    double* Mg = (double*)malloc(sizeof(double) * (size_t)(nmax + 1));
    if (node_margin)
        for (long q = 0; q < nn; ++q) node_margin[q] = 1.0e300;
    for (int k = 0; k < d; ++k) {
        int nk = c->n[k];
        int lim[3] = { c->n[0], c->n[1], n2 };
        lim[k] = 1;
        int o[3];
        for (o[2] = 0; o[2] < lim[2]; ++o[2])
            for (o[1] = 0; o[1] < lim[1]; ++o[1])
                for (o[0] = 0; o[0] < lim[0]; ++o[0]) {
                    for (int i = -1; i < nk; ++i) {
                        /* nodes i-2..i+3 along direction k */
                        double u6[6][MAXC], m6[6][4];
                        for (int t = 0; t < 6; ++t) {
                            int id[3] = { o[0], o[1], o[2] };
                            id[k] = i - 2 + t;
                            U_at(c, JU, J, id, u6[t]);
                            long pid = pidx_of(c, id);
                            for (int q = 0; q <= d; ++q) m6[t][q] = M[(long)(k * (d + 1) + q) * np + pid];
                        }
                        double f[MAXC], g[4], pair[MAXC];
                        for (int q = 0; q < nc; ++q) f[q] = 0.0;
                        for (int q = 0; q <= d; ++q) g[q] = 0.0;
                        for (int m = 1; m <= w; ++m)
                            for (int s = 0; s <= m - 1; ++s) {
                                int l = 2 - s, r = 2 - s + m;
                                or_ec_pair(c, u6[l], u6[r], m6[l], m6[r], pair);
                                for (int q = 0; q < nc; ++q) f[q] += alpha[m - 1] * pair[q];
                                for (int q = 0; q <= d; ++q) g[q] += alpha[m - 1] * 0.5 * (m6[l][q] + m6[r][q]);
                            }
                        Mg[i + 1] = 1.0e300;
                        if (c->es) {
                            double D[MAXC];
                            dissipation(c, u6, g, D, node_margin ? &Mg[i + 1] : NULL);
                            for (int q = 0; q < nc; ++q) f[q] += D[q];
                        }
                        for (int q = 0; q < nc; ++q) F[(i + 1) * nc + q] = f[q];
                        G[i + 1] = g[0];
                    }
                    for (int i = 0; i < nk; ++i) {
                        int id[3] = { o[0], o[1], o[2] };
                        id[k] = i;
                        long li = idx_of(c, id);
                        for (int q = 0; q < nc; ++q)
                            dJU[q * nn + li] -= (F[(i + 1) * nc + q] - F[i * nc + q]) / c->dxi[k];
                        dJ[li] -= (G[i + 1] - G[i]) / c->dxi[k];
                        if (node_margin) {
                            double mm = Mg[i + 1] < Mg[i] ? Mg[i + 1] : Mg[i];
                            if (mm < node_margin[li]) node_margin[li] = mm;
                        }
                    }
                }
    }
    free(F);
    free(G);
    free(Mg);
    free(M);
}

/* SSP-RK3 (Shu-Osher form) on q = (JU, J, x) with dx/dt = xdot, Sec. 5 */
void or_rk_step(const or_config* c, double* JU, double* J, double* x, const double* xdot, double dt)
{
    int d = c->d, nc = or_nc(c);
    long nn = or_ncell(c);
    size_t nu = (size_t)nc * nn, nx = (size_t)d * nn;
    double* JU1 = (double*)malloc(sizeof(double) * nu);
    double* J1 = (double*)malloc(sizeof(double) * nn);
    double* x1 = (double*)malloc(sizeof(double) * nx);
    double* dU = (double*)malloc(sizeof(double) * nu);
    double* dJ = (double*)malloc(sizeof(double) * nn);
    static const double A[3] = { 0.0, 0.75, 1.0 / 3.0 }, B[3] = { 1.0, 0.25, 2.0 / 3.0 };
    memcpy(JU1, JU, sizeof(double) * nu);
    memcpy(J1, J, sizeof(double) * nn);
    memcpy(x1, x, sizeof(double) * nx);
    for (int st = 0; st < 3; ++st) {
        or_rhs(c, JU1, J1, x1, xdot, dU, dJ);
        for (size_t q = 0; q < nu; ++q) JU1[q] = A[st] * JU[q] + B[st] * (JU1[q] + dt * dU[q]);
        for (long q = 0; q < nn; ++q) J1[q] = A[st] * J[q] + B[st] * (J1[q] + dt * dJ[q]);
        for (size_t q = 0; q < nx; ++q) x1[q] = A[st] * x[q] + B[st] * (x1[q] + dt * xdot[q]);
    }
    memcpy(JU, JU1, sizeof(double) * nu);
    memcpy(J, J1, sizeof(double) * nn);
    memcpy(x, x1, sizeof(double) * nx);
    free(JU1); free(J1); free(x1); free(dU); free(dJ);
}

/* ------------------------------------------------------------------------ */
/* time step, Eq. (cfl)                                                      */
/* ------------------------------------------------------------------------ */

static double sound_speed(const or_config* c, const double* rl, double T)
{
    double Rm, Gm;
    mixture(c, rl, &Rm, &Gm);
    return sqrt(Rm * Gm * T);
}

double or_cfl_dt(const or_config* c, const double* JU, const double* J, const double* x)
{
    int d = c->d;
    double alpha[3];
    or_alpha(c->w, alpha);
    int n2 = d == 3 ? c->n[2] : 1;
    double mx = 0.0;
    int i[3] = { 0, 0, 0 };
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                double m[3][4], U[MAXC], rl[2], v[3], T, p;
                node_metrics(c, x, NULL, alpha, i, m);
                U_at(c, JU, J, i, U);
                or_primitives(c, U, rl, v, &T, &p);
                double cs = sound_speed(c, rl, T), Jn = J[idx_of(c, i)], s = 0.0;
                for (int k = 0; k < d; ++k) {
                    double L = 0.0, vn = 0.0;
                    for (int j = 0; j < d; ++j) { L += m[k][1 + j] * m[k][1 + j]; vn += m[k][1 + j] * v[j]; }
                    L = sqrt(L);
                    s += (fabs(vn) + cs * L) / Jn / c->dxi[k];
                }
                if (s > mx) mx = s;
            }
    return c->cfl / mx;
}

/* ------------------------------------------------------------------------ */
/* adaptive moving mesh, Sec. 4                                              */
/* ------------------------------------------------------------------------ */

static double sigma_of(const or_config* c, int kind, const double* U)
{
    double rl[2], v[3], T, p, rho = 0.0;
    or_primitives(c, U, rl, v, &T, &p);
    for (int l = 0; l < c->N; ++l) rho += rl[l];
    switch (kind) {
    case OR_SIG_RHO1: return rl[0];
    case OR_SIG_RHO2: return c->N == 2 ? rl[1] : 0.0;
    case OR_SIG_P: return p;
    case OR_SIG_Y2: return c->N == 2 ? rl[1] / rho : 0.0;
    case OR_SIG_V1: return v[0];
    default: return rho;
    }
}

/* Eq. (monitor) with second-order central xi-gradients, followed by the
 * low-pass filter of the remark in Sec. 4 applied nf times */
void or_monitor(const or_config* c, const double* JU, const double* J, double* theta)
{
    int d = c->d;
    long nn = or_ncell(c);
    int n2 = d == 3 ? c->n[2] : 1;
    double* g = (double*)malloc(sizeof(double) * (size_t)nn * (c->n_sigma > 0 ? c->n_sigma : 1));
    double gmax[4] = { 0, 0, 0, 0 };
    int i[3] = { 0, 0, 0 };
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                long id = idx_of(c, i);
                double Uc[MAXC];
                U_at(c, JU, J, i, Uc);
                for (int s = 0; s < c->n_sigma; ++s) {
                    /* |grad_xi sigma| by central differences, or the Laplacian's magnitude */
                    double acc = 0.0, lap = 0.0;
                    for (int k = 0; k < d; ++k) {
                        int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
                        ip[k] += 1;
                        im[k] -= 1;
                        double Up[MAXC], Um[MAXC];
                        U_at(c, JU, J, ip, Up);
                        U_at(c, JU, J, im, Um);
                        double sp = sigma_of(c, c->sigma[s], Up), sm = sigma_of(c, c->sigma[s], Um);
                        double gk = (sp - sm) / (2.0 * c->dxi[k]);
                        acc += gk * gk;
                        lap += (sp - 2.0 * sigma_of(c, c->sigma[s], Uc) + sm) / (c->dxi[k] * c->dxi[k]);
                    }
                    g[s * nn + id] = c->sigma_op[s] == OR_MON_LAP ? fabs(lap) : sqrt(acc);
                    if (g[s * nn + id] > gmax[s]) gmax[s] = g[s * nn + id];
                }
            }
    for (long id = 0; id < nn; ++id) {
        double t = 1.0;
        for (int s = 0; s < c->n_sigma; ++s)
            if (gmax[s] > 0.0) {
                double r = g[s * nn + id] / gmax[s];
                t += c->sigma_op[s] == OR_MON_GRAD2 ? c->alpha[s] * r * r : c->alpha[s] * r;
            }
        theta[id] = sqrt(t);
    }
    free(g);
    for (int f = 0; f < c->nf; ++f) or_filter(c, theta);
}

void or_schlieren(const or_config* c, const double* JU, const double* J, const double* x, double psi1, double psi2,
                  double* phi)
{
    int d = c->d;
    long nn = or_ncell(c), np = or_npad(c);
    int n2 = d == 3 ? c->n[2] : 1;
    double* M = (double*)malloc(sizeof(double) * (size_t)np * d * (d + 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)nn);
    or_metrics(c, x, NULL, M);
    double gmax = 0.0;
    int i[3] = { 0, 0, 0 };
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                long id = idx_of(c, i);
                double drho[3] = { 0, 0, 0 };
                for (int k = 0; k < d; ++k) {
                    int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
                    ip[k] += 1;
                    im[k] -= 1;
                    double Up[MAXC], Um[MAXC];
                    U_at(c, JU, J, ip, Up);
                    U_at(c, JU, J, im, Um);
                    drho[k] = (sigma_of(c, OR_SIG_RHO, Up) - sigma_of(c, OR_SIG_RHO, Um)) / (2.0 * c->dxi[k]);
                }
                double acc = 0.0;
                for (int j = 0; j < d; ++j) {
                    double gj = 0.0;
                    for (int k = 0; k < d; ++k) gj += M[(long)(k * (d + 1) + 1 + j) * np + pidx_of(c, i)] * drho[k];
                    gj /= J[id];
                    acc += gj * gj;
                }
                g[id] = sqrt(acc);
                if (g[id] > gmax) gmax = g[id];
            }
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                long id = idx_of(c, i);
                double U[MAXC];
                U_at(c, JU, J, i, U);
                double rho = sigma_of(c, OR_SIG_RHO, U);
                double psi = (psi1 * U[0] + (c->N == 2 ? psi2 * U[1] : 0.0)) / rho;
                phi[id] = gmax > 0.0 ? exp(-psi * g[id] / gmax) : 1.0;
            }
    free(M);
    free(g);
}

/* one pass of the low-pass filter: weights (1/2)^(|j1|+..+|jd| + d) */
void or_filter(const or_config* c, double* theta)
{
    int d = c->d;
    long nn = or_ncell(c);
    int n2 = d == 3 ? c->n[2] : 1;
    double* out = (double*)malloc(sizeof(double) * (size_t)nn);
    int i[3] = { 0, 0, 0 };
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                double s = 0.0;
                int j3lo = d == 3 ? -1 : 0, j3hi = d == 3 ? 1 : 0;
                for (int j3 = j3lo; j3 <= j3hi; ++j3)
                    for (int j2 = -1; j2 <= 1; ++j2)
                        for (int j1 = -1; j1 <= 1; ++j1) {
                            int nb[3] = { i[0] + j1, i[1] + j2, i[2] + j3 };
                            int e = abs(j1) + abs(j2) + abs(j3) + d;
                            s += pow(0.5, e) * s_at(c, theta, nb);
                        }
                out[idx_of(c, i)] = s;
            }
    memcpy(theta, out, sizeof(double) * (size_t)nn);
    free(out);
}

/* mu Jacobi sweeps of the discrete mesh equation, Sec. 4 */
void or_jacobi(const or_config* c, const double* x, const double* theta, double* xmu)
{
    int d = c->d;
    long nn = or_ncell(c);
    int n2 = d == 3 ? c->n[2] : 1;
    double* cur = (double*)malloc(sizeof(double) * (size_t)d * nn);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)d * nn);
    memcpy(cur, x, sizeof(double) * (size_t)d * nn);
    for (int nu = 0; nu < c->mu; ++nu) {
        int i[3] = { 0, 0, 0 };
        for (i[2] = 0; i[2] < n2; ++i[2])
            for (i[1] = 0; i[1] < c->n[1]; ++i[1])
                for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                    long id = idx_of(c, i);
                    double num[3] = { 0, 0, 0 }, den = 0.0, th = theta[id];
                    for (int k = 0; k < d; ++k) {
                        int ip[3] = { i[0], i[1], i[2] }, im[3] = { i[0], i[1], i[2] };
                        ip[k] += 1;
                        im[k] -= 1;
                        double tp = 0.5 * (th + s_at(c, theta, ip)), tm = 0.5 * (th + s_at(c, theta, im));
                        double xp[3], xm[3];
                        x_at(c, cur, ip, xp, 0);
                        x_at(c, cur, im, xm, 0);
                        double h2 = c->dxi[k] * c->dxi[k];
                        for (int j = 0; j < d; ++j) num[j] += (tp * xp[j] + tm * xm[j]) / h2;
                        den += (tp + tm) / h2;
                    }
                    for (int j = 0; j < d; ++j) nxt[j * nn + id] = num[j] / den;
                }
        double* t = cur; cur = nxt; nxt = t;
    }
    memcpy(xmu, cur, sizeof(double) * (size_t)d * nn);
    free(cur);
    free(nxt);
}

/* Delta_tau = min(1, the bounds of Sec. 4 over all nodes and directions) */
double or_limiter(const or_config* c, const double* x, const double* xmu)
{
    int d = c->d;
    long nn = or_ncell(c);
    int n2 = d == 3 ? c->n[2] : 1;
    double dtau = 1.0;
    int i[3] = { 0, 0, 0 };
    for (i[2] = 0; i[2] < n2; ++i[2])
        for (i[1] = 0; i[1] < c->n[1]; ++i[1])
            for (i[0] = 0; i[0] < c->n[0]; ++i[0]) {
                long id = idx_of(c, i);
                for (int k = 0; k < d; ++k) {
                    double dx = xmu[k * nn + id] - x[k * nn + id];
                    int nb[3] = { i[0], i[1], i[2] };
                    double xn[3];
                    if (dx < 0.0) {
                        nb[k] -= 1;
                        x_at(c, x, nb, xn, 0);
                        double b = -(x[k * nn + id] - xn[k]) / (2.0 * dx);
                        if (b < dtau) dtau = b;
                    } else if (dx > 0.0) {
                        nb[k] += 1;
                        x_at(c, x, nb, xn, 0);
                        double b = (xn[k] - x[k * nn + id]) / (2.0 * dx);
                        if (b < dtau) dtau = b;
                    }
                }
            }
    return dtau;
}

/* one mesh redistribution: Delta t (Eq. (cfl)) unless given, monitor + filter,
 * Jacobi sweeps, limiter and the mesh velocity xdot = Delta_tau delta_tau x / Delta t */
void or_mesh_redistribute(const or_config* c, const double* JU, const double* J, const double* x,
                          double dt_in, double* xdot, double* dt_dtau)
{
    int d = c->d;
    long nn = or_ncell(c);
    double dt = dt_in > 0.0 ? dt_in : or_cfl_dt(c, JU, J, x);
    double* th = (double*)malloc(sizeof(double) * (size_t)nn);
    double* xmu = (double*)malloc(sizeof(double) * (size_t)d * nn);
    or_monitor(c, JU, J, th);
    or_jacobi(c, x, th, xmu);
    double dtau = or_limiter(c, x, xmu);
    for (long q = 0; q < (long)d * nn; ++q) xdot[q] = dtau * (xmu[q] - x[q]) / dt;
    dt_dtau[0] = dt;
    dt_dtau[1] = dtau;
    free(th);
    free(xmu);
}

/* ------------------------------------------------------------------------ */
/* entropy diagnostics: d(J eta)/dt = V^T d(JU)/dt - phi dJ/dt (Sec. 1, phi = V^T U - eta) */
/* ------------------------------------------------------------------------ */

void or_entropy(const or_config* c, const double* JU, const double* J,
                const double* dJU, const double* dJ, double* out)
{
    int d = c->d, nc = or_nc(c);
    long nn = or_ncell(c);
    double vol = 1.0;
    for (int k = 0; k < d; ++k) vol *= c->dxi[k];
    double P = 0.0, S = 0.0;
    for (long id = 0; id < nn; ++id) {
        double U[MAXC], V[MAXC];
        for (int q = 0; q < nc; ++q) U[q] = JU[q * nn + id] / J[id];
        or_entropy_vars(c, U, V);
        double s = 0.0;
        if (dJU && dJ) {
            for (int q = 0; q < nc; ++q) s += V[q] * dJU[q * nn + id];
            s -= or_phi(c, U) * dJ[id];
        }
        P += vol * s;
        S += vol * J[id] * or_eta(c, U);
    }
    out[0] = P;
    out[1] = S;
}
