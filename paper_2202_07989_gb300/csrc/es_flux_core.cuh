// Arithmetic of the flux kernels shared by the per-direction kernel and the fused
// 2D stage kernel: the compute-type helpers, the WENO reconstructions, the node
// field layout and the per-node, per-pair and per-interface steps of Eqs. (semi_U),
// (semi_J): the sixth-order EC flux as sum_m alpha_m sum_s F(U_{i-s}, U_{i-s+m})
// with the two-point flux of Eq. (ECfluxMM) (Sec. 3.3), the GCL flux of J xi_k/t
// (Eq. (GCL_flux)) and the ES dissipation -1/2 T^T R |Lambda| Y [[W]]^WENOMR of
// Eq. (HOstable) with the scaled eigenvectors of Sec. 3.4 and the WENO-MR of Appendix A.
//
// Contracted two-point flux.  With means over the pair, u~ = Mt + sum_j Mx_j {v_j},
// rho~ = sum_l {rho_l}^ln, P' = sum_l R_l {rho_l} / {beta} (= P~ + p_inf) and
// E' = sum_l {rho_l}^ln c_{v,l} / {beta}^ln - rho~ sum_m {v_m^2}/2 + rho~ sum_m {v_m}^2
// (= U~_E - p_inf), the flux of Eq. (ECfluxMM) is
//   F_l = u~ {rho_l}^ln,  F_m = u~ rho~ {v_m} + Mx_m (P' - p_inf),
//   F_E = u~ E' + (u~ - Mt) P' + p_inf Mt.
// Summed over the pairs, the p_inf Mx_m terms give p_inf times the GCL flux of
// J xi_k/x_m, whose divergence vanishes by the discrete SCL (Eq. (SCL_dis)), and
// the p_inf Mt terms give p_inf times the GCL flux of J xi_k/t.  The kernel drops
// the first and adds the second in FP64, which keeps the large p_inf of stiffened
// gases out of the low-precision pair arithmetic.
#pragma once

#include "es_kernels.cuh"

#include <type_traits>

namespace es {

template <typename R>
struct Ar;

template <>
struct Ar<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
    static __device__ __forceinline__ double ab(double x) { return fabs(x); }
    // {a}^ln: [[a]]/[[ln a]], Ismail-Roe series when ((b-a)/(b+a))^2 < 1e-4
    static __device__ __forceinline__ double lmean(double a, double b, double la, double lb)
    {
        double s = a + b, dd = b - a;
        if (fabs(dd) < 0.01 * s) {
            double f = dd / s, u = f * f;
            return 0.5 * s * (1.0 - u * (1.0 / 3.0 + u * (4.0 / 45.0 + u * (44.0 / 945.0))));
        }
        return dd / (lb - la);
    }
    // 1/{a}^ln given is = 1/(a + b)
    static __device__ __forceinline__ double inv_lmean(double a, double b, double la, double lb, double is)
    {
        double dd = b - a;
        if (fabs(dd) < 0.01 * (a + b)) {
            double f = dd * is, u = f * f;
            return 2.0 * is * (1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0))));
        }
        return (lb - la) / dd;
    }
    // the same with the logarithms formed only in their branch
    static __device__ __forceinline__ double lmean(double a, double b)
    {
        double s = a + b, dd = b - a;
        if (fabs(dd) < 0.01 * s) return lmean(a, b, 0.0, 0.0);
        return dd / (lg(b) - lg(a));
    }
    static __device__ __forceinline__ double inv_lmean(double a, double b, double is)
    {
        double dd = b - a;
        if (fabs(dd) < 0.01 * (a + b)) return inv_lmean(a, b, 0.0, 0.0, is);
        return (lg(b) - lg(a)) / dd;
    }
};

template <>
struct Ar<float> {
    static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
    static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float lg(float x) { return logf(x); }
    static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float ab(float x) { return fabsf(x); }
    // small jumps ((b-a)/(b+a))^2 < 1e-2: {a}^ln = {a} (1 - delta(u)), the mean {a}
    // and the correction formed in FP64 (logmean_small: {a} exact in binary64, built with
    // integer instructions, and one FP64 fused multiply-add); delta is the series of
    // 1 - f/artanh(f).  Here a, b > 0: |b - a| < (a + b)/10
    static __device__ __forceinline__ float small_branch(float a, float b, float u)
    {
        float del = u * (1.f / 3.f + u * (4.f / 45.f + u * (44.f / 945.f + u * (428.f / 14175.f))));
        return logmean_small(a, b, del);
    }
    static __device__ __forceinline__ float lmean(float a, float b, float la, float lb)
    {
        float s = a + b, dd = b - a;
        if (fabsf(dd) < 0.1f * s) {
            float f = __fdividef(dd, s);
            return small_branch(a, b, f * f);
        }
        return __fdividef(dd, lb - la);
    }
    static __device__ __forceinline__ float inv_lmean(float a, float b, float la, float lb, float is)
    {
        float dd = b - a;
        if (fabsf(dd) < 0.1f * (a + b)) {
            float f = dd * is;
            return __frcp_rn(small_branch(a, b, f * f));
        }
        return __fdividef(lb - la, dd);
    }
    // the same with the logarithms formed only in their branch
    static __device__ __forceinline__ float lmean(float a, float b)
    {
        float s = a + b, dd = b - a;
        if (fabsf(dd) < 0.1f * s) return lmean(a, b, 0.0f, 0.0f);
        return __fdividef(dd, lg(b) - lg(a));
    }
    static __device__ __forceinline__ float inv_lmean(float a, float b, float is)
    {
        float dd = b - a;
        if (fabsf(dd) < 0.1f * (a + b)) return inv_lmean(a, b, 0.0f, 0.0f, is);
        return __fdividef(lg(b) - lg(a), dd);
    }
};

// Sign band of the sign matrix Y (Sec. 3.4): a jump [[W_m]] no larger than delta times
// its round-off scale ||r_m|| (||V_i|| + ||V_i+1||) has no reliable sign and counts as
// zero, like an exactly zero jump (Y = 0 keeps the ES sign property).
template <typename R>
struct YBand;
template <>
struct YBand<double> { static constexpr double value = 1.0e-12; };
template <>
struct YBand<float> { static constexpr double value = 3.0e-7; };

// fifth-order multi-resolution WENO value at x_{j+1/2} from W_{j-2..j+2} (Appendix A);
// beta_2, beta_3 are the closed forms printed there.
template <typename R>
__device__ __forceinline__ R weno_mr(R w0, R w1, R w2, R w3, R w4, R c1, R c2, R c3, R eps)
{
    R a2 = R(0.5) * (w3 - w1);
    R a3 = R(0.5) * (w1 + w3) - w2;
    R b2 = (R(11) * (w0 - w4) + R(82) * (w3 - w1)) * R(1.0 / 120.0);
    R b3 = (R(-3) * (w0 + w4) + R(40) * (w1 + w3) - R(74) * w2) * R(1.0 / 56.0);
    R b4 = (w4 - w0 + R(2) * (w1 - w3)) * R(1.0 / 12.0);
    R b5 = (w0 + w4 - R(4) * (w1 + w3) + R(6) * w2) * R(1.0 / 24.0);
    R d0 = (w2 - w1) * (w2 - w1), d1 = (w3 - w2) * (w3 - w2);
    R be1 = d0 < d1 ? d0 : d1;
    R be2 = a2 * a2 + R(13.0 / 3.0) * a3 * a3;
    R t1 = b2 + R(0.1) * b4, t2 = b3 + R(123.0 / 455.0) * b5;
    R be3 = t1 * t1 + R(13.0 / 3.0) * t2 * t2 + R(781.0 / 20.0) * b4 * b4 + R(1421461.0 / 2275.0) * b5 * b5;
    R tau = R(0.5) * (Ar<R>::ab(be3 - be1) + Ar<R>::ab(be3 - be2));
    tau = tau * tau;
    R h1 = w2;
    R h2 = w2 + R(0.5) * a2 + R(1.0 / 6.0) * a3;
    R h3 = w2 + R(0.5) * b2 + R(1.0 / 6.0) * b3 + R(0.05) * b4 + R(1.0 / 70.0) * b5;
    R h3c = (h3 - c1 * h1 - c2 * h2) * Ar<R>::rcp(c3);
    R e1 = eps + be1, e2 = eps + be2, e3 = eps + be3;
    if constexpr (std::is_same<R, double>::value) {
        // common denominator e1 e2 e3: one division
        R o1 = c1 * (e1 + tau) * e2 * e3, o2 = c2 * (e2 + tau) * e1 * e3, o3 = c3 * (e3 + tau) * e1 * e2;
        return (o1 * h1 + o2 * h2 + o3 * h3c) / (o1 + o2 + o3);
    } else {
        R o1 = c1 * (R(1) + Ar<R>::dv(tau, e1)), o2 = c2 * (R(1) + Ar<R>::dv(tau, e2)), o3 = c3 * (R(1) + Ar<R>::dv(tau, e3));
        return Ar<R>::dv(o1 * h1 + o2 * h2 + o3 * h3c, o1 + o2 + o3);
    }
}

// binary32 pairs: two independent evaluations in the two lanes of Blackwell's paired FP32
// instructions (FADD2 / FMUL2 / FFMA2, IEEE round-to-nearest in each lane)
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }   // a - b, one rounding

// weno_mr<float> for W^- (lane x, from W_{j-2..j+2}) and W^+ (lane y, the mirrored stencil)
// at once: the same closed forms, evaluated lane by lane; divisions and min/abs per lane
__device__ __forceinline__ float2 weno_mr_pair(float2 w0, float2 w1, float2 w2, float2 w3, float2 w4, float c1, float c2,
                                               float c3, float ic3, float eps)
{
    const float2 s13 = add2(w1, w3), d31 = sub2(w3, w1), s04 = add2(w0, w4), d04 = sub2(w0, w4);
    const float2 a2 = mul2(f2(0.5f), d31);
    const float2 a3 = sub2(mul2(f2(0.5f), s13), w2);
    const float2 b2 = mul2(fma2(f2(11.0f), d04, mul2(f2(82.0f), d31)), f2(1.0f / 120.0f));
    const float2 b3 = mul2(fma2(f2(-3.0f), s04, fma2(f2(40.0f), s13, mul2(f2(-74.0f), w2))), f2(1.0f / 56.0f));
    const float2 b4 = mul2(fma2(f2(2.0f), d31, d04), f2(-1.0f / 12.0f));
    const float2 b5 = mul2(fma2(f2(-4.0f), s13, fma2(f2(6.0f), w2, s04)), f2(1.0f / 24.0f));
    const float2 d21 = sub2(w2, w1), d32 = sub2(w3, w2);
    const float2 q0 = mul2(d21, d21), q1 = mul2(d32, d32);
    const float2 be1 = make_float2(fminf(q0.x, q1.x), fminf(q0.y, q1.y));
    const float2 be2 = fma2(f2(13.0f / 3.0f), mul2(a3, a3), mul2(a2, a2));
    const float2 t1 = fma2(f2(0.1f), b4, b2), t2 = fma2(f2(123.0f / 455.0f), b5, b3);
    const float2 be3 = fma2(t1, t1, fma2(f2(13.0f / 3.0f), mul2(t2, t2),
                                         fma2(f2(781.0f / 20.0f), mul2(b4, b4), mul2(f2(1421461.0f / 2275.0f), mul2(b5, b5)))));
    const float2 u1 = sub2(be3, be1), u2 = sub2(be3, be2);
    const float tx = 0.5f * (fabsf(u1.x) + fabsf(u2.x)), ty = 0.5f * (fabsf(u1.y) + fabsf(u2.y));
    const float2 tau = make_float2(tx * tx, ty * ty);
    const float2 h2 = fma2(f2(1.0f / 6.0f), a3, fma2(f2(0.5f), a2, w2));
    const float2 h3 = fma2(f2(1.0f / 70.0f), b5, fma2(f2(0.05f), b4, fma2(f2(1.0f / 6.0f), b3, fma2(f2(0.5f), b2, w2))));
    const float2 h3c = mul2(fma2(f2(-c2), h2, fma2(f2(-c1), w2, h3)), f2(ic3));
    const float2 e1 = add2(f2(eps), be1), e2 = add2(f2(eps), be2), e3 = add2(f2(eps), be3);
    const float2 o1 = fma2(f2(c1), make_float2(__fdividef(tau.x, e1.x), __fdividef(tau.y, e1.y)), f2(c1));
    const float2 o2 = fma2(f2(c2), make_float2(__fdividef(tau.x, e2.x), __fdividef(tau.y, e2.y)), f2(c2));
    const float2 o3 = fma2(f2(c3), make_float2(__fdividef(tau.x, e3.x), __fdividef(tau.y, e3.y)), f2(c3));
    const float2 num = fma2(o3, h3c, fma2(o2, h2, mul2(o1, w2)));
    const float2 den = add2(o1, add2(o2, o3));
    return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

// classical fifth-order WENO (Jiang and Shu; the MM-WENOJS comparison of Sec. 5) at
// x_{j+1/2} from W_{j-2..j+2}: candidate values of the three quadratic reconstructions,
// their smoothness indicators, linear weights 1/10, 6/10, 3/10 and weights d_k/(eps+beta_k)^2
template <typename R>
__device__ __forceinline__ R weno_js(R w0, R w1, R w2, R w3, R w4, R eps)
{
    const R s0 = w0 - R(2) * w1 + w2, t0 = w0 - R(4) * w1 + R(3) * w2;
    const R s1 = w1 - R(2) * w2 + w3, t1 = w1 - w3;
    const R s2 = w2 - R(2) * w3 + w4, t2 = R(3) * w2 - R(4) * w3 + w4;
    const R e0 = eps + (R(13.0 / 12.0) * s0 * s0 + R(0.25) * t0 * t0);
    const R e1 = eps + (R(13.0 / 12.0) * s1 * s1 + R(0.25) * t1 * t1);
    const R e2 = eps + (R(13.0 / 12.0) * s2 * s2 + R(0.25) * t2 * t2);
    const R q0 = (R(2) * w0 - R(7) * w1 + R(11) * w2) * R(1.0 / 6.0);
    const R q1 = (-w1 + R(5) * w2 + R(2) * w3) * R(1.0 / 6.0);
    const R q2 = (R(2) * w2 + R(5) * w3 - w4) * R(1.0 / 6.0);
    if constexpr (std::is_same<R, double>::value) {
        // common denominator (e0 e1 e2)^2: one division
        const R f0 = e0 * e0, f1 = e1 * e1, f2 = e2 * e2;
        const R a0 = R(0.1) * f1 * f2, a1 = R(0.6) * f0 * f2, a2 = R(0.3) * f0 * f1;
        return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
    } else {
        // products of the squared terms could leave the binary32 range: one division each
        const R a0 = Ar<R>::dv(R(0.1), e0 * e0), a1 = Ar<R>::dv(R(0.6), e1 * e1), a2 = Ar<R>::dv(R(0.3), e2 * e2);
        return Ar<R>::dv(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
    }
}

// the reconstruction of the dissipation: WK = 0 WENO-MR (Appendix A), 1 WENO-JS
template <typename R, int WK>
__device__ __forceinline__ R weno_val(R w0, R w1, R w2, R w3, R w4, R c1, R c2, R c3, R eps)
{
    if constexpr (WK == 0) return weno_mr<R>(w0, w1, w2, w3, w4, c1, c2, c3, eps);
    else return weno_js<R>(w0, w1, w2, w3, w4, eps);
}

// Node fields in shared memory.  2D tiles keep species densities and their logs, velocity,
// beta and ln beta, the mixture quantities (two species), the entropy variables, ||V|| and the
// metrics.  3D tiles are compact: species densities, velocity, entropy variables (the last
// component is -beta) and metrics; the logs are formed in the branch of a log mean that needs
// them, the mixture quantities and ||V|| at the interface.  The compact tiles fit 4 CTAs per SM
// (measured 3-10% faster in 3D); in the fused 2D stage kernel the recomputation cost more than
// the smaller tile gained.
template <int D, int NS>
struct Lay {
    static constexpr bool COMPACT = D == 3;
    static constexpr int NC = NS + D + 1;
    static constexpr int RHO = 0;
    static constexpr int LRHO = COMPACT ? -1 : NS;
    static constexpr int V = COMPACT ? NS : 2 * NS;
    static constexpr int B = COMPACT ? -1 : V + D;
    static constexpr int LB = COMPACT ? -1 : B + 1;
    static constexpr int X = COMPACT ? -1 : LB + 1;
    static constexpr int NX = (!COMPACT && NS == 2) ? 5 : 0;   // p, rho, ln rho, R_mix, Gamma_mix
    static constexpr int VV = COMPACT ? V + D : X + NX;        // entropy variables
    static constexpr int VN = COMPACT ? -1 : VV + NC;          // ||V||_2
    static constexpr int MR = COMPACT ? VV + NC : VN + 1;      // metrics J xi_k/t, J xi_k/x_j (compute type)
    static constexpr int NF = MR + 1 + D;
};

// ||V||_2 of the node at nb (field stride NN)
template <int NC, int VV, typename R>
__device__ __forceinline__ R vnorm(const R* nb, int NN)
{
    R vn = R(0);
#pragma unroll
    for (int q = 0; q < NC; ++q) vn += nb[(VV + q) * NN] * nb[(VV + q) * NN];
    return Ar<R>::sq(vn);
}

// Phase 1 of one node: from its conserved point state U, the fields of Lay<D, NS> up to
// ||V|| (species densities and their logs, velocity, beta and ln beta, the mixture
// quantities, the entropy variables and their norm) at `node` of the field-major node
// array nr (field stride NN).  A non-physical state sets ST_NONPHYSICAL.
template <int D, int NS, typename R>
__device__ __forceinline__ void node_fields(const Inst& I, const R* U, R* nr, int NN, int node, int* status)
{
    using Y = Lay<D, NS>;
    constexpr int NC = Y::NC;
    R rho = U[0] + (NS == 2 ? U[1] : R(0));
    R irho = Ar<R>::rcp(rho);
    R v[D], v2 = R(0);
#pragma unroll
    for (int m = 0; m < D; ++m) { v[m] = U[NS + m] * irho; v2 += v[m] * v[m]; }
    R cvr = Cst<R>::cv(I, 0) * U[0] + (NS == 2 ? Cst<R>::cv(I, 1) * U[1] : R(0));
    R rhoe_p = U[NS + D] - R(0.5) * rho * v2 - Cst<R>::pinf(I);
    R beta = cvr * Ar<R>::rcp(rhoe_p);
    bool bad = !(rhoe_p > R(0)) || !(U[0] > R(0)) || (NS == 2 && !(U[1] > R(0)));
    if (bad) {
        atomicOr(status, ST_NONPHYSICAL);
        beta = R(1);
    }
    R lb = Ar<R>::lg(beta);
    R lr0 = Ar<R>::lg(bad ? R(1) : U[0]);
    R lr1 = NS == 2 ? Ar<R>::lg(bad ? R(1) : U[1]) : R(0);
#pragma unroll
    for (int m = 0; m < D; ++m) nr[(Y::V + m) * NN + node] = v[m];
    if constexpr (Y::COMPACT) {
        // a non-physical node keeps positive densities (its log means stay finite)
        nr[Y::RHO * NN + node] = bad ? R(1) : U[0];
        if (NS == 2) nr[(Y::RHO + 1) * NN + node] = bad ? R(1) : U[1];
    } else {
    nr[Y::RHO * NN + node] = U[0];
    nr[Y::LRHO * NN + node] = lr0;
    if (NS == 2) { nr[(Y::RHO + 1) * NN + node] = U[1]; nr[(Y::LRHO + 1) * NN + node] = lr1; }
    nr[Y::B * NN + node] = beta;
    nr[Y::LB * NN + node] = lb;
    if (NS == 2) {
        R T = Ar<R>::rcp(beta);
        R rr = Cst<R>::Rs(I, 0) * U[0] + Cst<R>::Rs(I, 1) * U[1];
        nr[(Y::X + 0) * NN + node] = rr * T - Cst<R>::pinf(I);                 // p
        nr[(Y::X + 1) * NN + node] = rho;                                    // rho
        nr[(Y::X + 2) * NN + node] = Ar<R>::lg(bad ? R(1) : rho);           // ln rho
        nr[(Y::X + 3) * NN + node] = rr * irho;                              // R_mix
        nr[(Y::X + 4) * NN + node] = (Cst<R>::cvG(I, 0) * U[0] + Cst<R>::cvG(I, 1) * U[1]) * Ar<R>::rcp(cvr);  // Gamma_mix
    }
    }
    // entropy variables V_l = c_{v,l} ln beta + R_l ln rho_l - |v|^2 beta/2 + c_{v,l} Gamma_l
    R hv = R(0.5) * v2 * beta;
    R Vn[NC];
    Vn[0] = Cst<R>::cv(I, 0) * lb + Cst<R>::Rs(I, 0) * lr0 - hv + Cst<R>::cvG(I, 0);
    if (NS == 2) Vn[1] = Cst<R>::cv(I, 1) * lb + Cst<R>::Rs(I, 1) * lr1 - hv + Cst<R>::cvG(I, 1);
#pragma unroll
    for (int m = 0; m < D; ++m) Vn[NS + m] = v[m] * beta;
    Vn[NS + D] = -beta;
    R vn = R(0);
#pragma unroll
    for (int q = 0; q < NC; ++q) { nr[(Y::VV + q) * NN + node] = Vn[q]; vn += Vn[q] * Vn[q]; }
    if constexpr (!Y::COMPACT) nr[Y::VN * NN + node] = Ar<R>::sq(vn);
}

// Phase 2 of one pair (l, r) of nodes: the contracted two-point flux of every field into
// pf at t (field stride NP).  mr is the first metric field (J xi_k/t, then J xi_k/x_j) of
// the direction.  ci >= 0 marks the centre pair (i, i+1) of interface ci, whose log means
// {rho_l}^ln and 1/{beta}^ln go to cm (field stride NI) for the dissipation.
template <int D, int NS, typename R>
__device__ __forceinline__ void pair_flux(const Inst& I, const R* nr, int NN, int mr, int l, int rr, R* pf, int NP,
                                          int t, R* cm, int NI, int ci)
{
    using Y = Lay<D, NS>;
    constexpr int NC = Y::NC;
    R mt = R(0.5) * (nr[mr * NN + l] + nr[mr * NN + rr]);
    R mx[D], vb[D];
    R ut = mt, v2b = R(0), vbsq = R(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        mx[j] = R(0.5) * (nr[(mr + 1 + j) * NN + l] + nr[(mr + 1 + j) * NN + rr]);
        R vl = nr[(Y::V + j) * NN + l], vr = nr[(Y::V + j) * NN + rr];
        vb[j] = R(0.5) * (vl + vr);
        v2b += R(0.5) * (vl * vl + vr * vr);
        vbsq += vb[j] * vb[j];
        ut += mx[j] * vb[j];
    }
    R lr[NS], rt = R(0), rra = R(0);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        R al = nr[(Y::RHO + q) * NN + l], ar = nr[(Y::RHO + q) * NN + rr];
        if constexpr (Y::COMPACT) lr[q] = Ar<R>::lmean(al, ar);
        else lr[q] = Ar<R>::lmean(al, ar, nr[(Y::LRHO + q) * NN + l], nr[(Y::LRHO + q) * NN + rr]);
        rt += lr[q];
        rra += Cst<R>::Rs(I, q) * (al + ar);
    }
    R bl, br, ilb;
    R is;
    if constexpr (Y::COMPACT) {
        bl = -nr[(Y::VV + NC - 1) * NN + l];
        br = -nr[(Y::VV + NC - 1) * NN + rr];
        is = Ar<R>::rcp(bl + br);
        ilb = Ar<R>::inv_lmean(bl, br, is);
    } else {
        bl = nr[Y::B * NN + l];
        br = nr[Y::B * NN + rr];
        is = Ar<R>::rcp(bl + br);
        ilb = Ar<R>::inv_lmean(bl, br, nr[Y::LB * NN + l], nr[Y::LB * NN + rr], is);
    }
    R Pp = rra * is;                                   // sum R_l {rho_l} / {beta}
    R Ep = -R(0.5) * rt * v2b + rt * vbsq;
#pragma unroll
    for (int q = 0; q < NS; ++q) Ep += lr[q] * Cst<R>::cv(I, q) * ilb;
#pragma unroll
    for (int q = 0; q < NS; ++q) pf[q * NP + t] = ut * lr[q];
#pragma unroll
    for (int j = 0; j < D; ++j) pf[(NS + j) * NP + t] = ut * rt * vb[j] + mx[j] * Pp;
    pf[(NS + D) * NP + t] = ut * Ep + (ut - mt) * Pp;
    if (ci >= 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) cm[q * NI + ci] = lr[q];
        cm[NS * NI + ci] = ilb;
    }
}

// Phase 3 of one interface i+1/2 of a line.  nb points at field 0 of node i-2 of the
// field-major node array (field stride NN, node stride ns along the line), mr is the
// first metric field of the direction and m64 points at the FP64 J xi_k/t of node i-2
// (stride ms).  The distinct pair fluxes (field stride NP) of (i, i+1) sit at p1, of
// (i-1, i+1) and (i, i+2) at p2 and p2 + ps, of (i-2, i+1), (i-1, i+2) and (i, i+3) at
// p3, p3 + ps and p3 + 2 ps; the centre-pair means cm (field stride NI) and the outputs,
// the interface flux fl (field stride NI) and the FP64 GCL flux gt, at f.  Each output is
// stored as soon as it is formed, which keeps registers free through the dissipation.
template <int D, int NS, typename R, int WK>
__device__ __forceinline__ void iface_flux(const Inst& I, const R* nb, int NN, int ns, int mr, const double* m64, int ms,
                                           const R* pf, int NP, int p1, int p2, int p3, int ps, const R* cm, int NI, int f,
                                           R* fl, double* gt)
{
    using Y = Lay<D, NS>;
    constexpr int NC = Y::NC;
#define NR(fld, j) nb[(fld) * NN + (j) * ns]
    const R a1 = Cst<R>::ecw(I, 0), a2 = Cst<R>::ecw(I, 1), a3 = Cst<R>::ecw(I, 2);
    // the EC flux goes to its output slot at once; the dissipation is subtracted there at the end
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const R* pq = pf + q * NP;
        fl[q * NI + f] = a1 * pq[p1] + a2 * (pq[p2] + pq[p2 + ps]) + a3 * (pq[p3] + pq[p3 + ps] + pq[p3 + 2 * ps]);
    }
    // GCL flux of (J xi_k/t, J xi_k/x_j): stencil (1, -8, 37, 37, -8, 1)/60 for w = 3
    const double c0 = I.gcw[0], c1 = I.gcw[1], c2 = I.gcw[2];
    const double Gt = c0 * (m64[2 * ms] + m64[3 * ms]) + c1 * (m64[ms] + m64[4 * ms]) + c2 * (m64[0] + m64[5 * ms]);
    gt[f] = Gt;
    if (I.es) {
        R Gx[D], L2 = R(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int fj = mr + 1 + j;
            Gx[j] = Cst<R>::gcw(I, 0) * (NR(fj, 2) + NR(fj, 3)) + Cst<R>::gcw(I, 1) * (NR(fj, 1) + NR(fj, 4)) +
                    Cst<R>::gcw(I, 2) * (NR(fj, 0) + NR(fj, 5));
            L2 += Gx[j] * Gx[j];
        }
        R Ln = Ar<R>::sq(L2), iL = Ar<R>::rcp(Ln);
        R n[D];
#pragma unroll
        for (int j = 0; j < D; ++j) n[j] = Gx[j] * iL;
        // rotation rows t0 = n, t1, t2 (Eq. (rotamatrix) built from the unit normal)
        R T[D][D];
        if constexpr (D == 2) {
            T[0][0] = n[0]; T[0][1] = n[1];
            T[1][0] = -n[1]; T[1][1] = n[0];
        } else {
            R rr2 = n[0] * n[0] + n[1] * n[1];
            R rq = Ar<R>::sq(rr2);
            R ct = R(1), st = R(0);
            if (rq > R(0)) { R irq = Ar<R>::rcp(rq); ct = n[0] * irq; st = n[1] * irq; }
            R cp = rq, sp = n[D - 1];
            T[0][0] = n[0]; T[0][1] = n[1]; T[0][D - 1] = n[D - 1];
            T[1][0] = -st; T[1][1] = ct; T[1][D - 1] = R(0);
            T[D - 1][0] = -sp * ct; T[D - 1][1] = -sp * st; T[D - 1][D - 1] = cp;
        }
        // interface averages (Sec. 3.4); the log means of the centre pair come from phase 2
        R lr_c[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) lr_c[q] = cm[q * NI + f];
        const R Tb = cm[NS * NI + f];       // T-bar = 1 / {beta}^ln
        R vb[D], vh[D], vv = R(0);
#pragma unroll
        for (int j = 0; j < D; ++j) { vb[j] = R(0.5) * (NR(Y::V + j, 2) + NR(Y::V + j, 3)); vv += vb[j] * vb[j]; }
#pragma unroll
        for (int m = 0; m < D; ++m) {
            R s_ = R(0);
#pragma unroll
            for (int j = 0; j < D; ++j) s_ += T[m][j] * vb[j];
            vh[m] = s_;
        }
        R cb, H, sa, se = R(0), ssh, Y1 = R(1), Y2 = R(0), D11 = R(0), D12 = R(0), D21 = R(0), D22 = R(0), e1 = R(0), e2 = R(0);
        if constexpr (NS == 1) {
            const R G = Cst<R>::gamma(I, 0), Rg = Cst<R>::Rs(I, 0), cv = Cst<R>::cv(I, 0);
            const R rb = lr_c[0];
            cb = Ar<R>::sq(Rg * G * Tb);
            H = G * cv * Tb + R(0.5) * vv;
            sa = Ar<R>::sq(rb * Ar<R>::rcp(R(2) * G * Rg));
            se = Ar<R>::sq(rb * Ar<R>::rcp(cv * G));
            ssh = Ar<R>::sq(rb * Tb);
        } else {
            // the mixture quantities rho, R_mix, Gamma_mix and p of the two centre nodes
            R xr[2], xR[2], xG[2], xp[2], xl[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if constexpr (Y::COMPACT) {
                    const R u0 = NR(Y::RHO, 2 + c), u1 = NR(Y::RHO + 1, 2 + c), beta = -NR(Y::VV + NC - 1, 2 + c);
                    const R rr = Cst<R>::Rs(I, 0) * u0 + Cst<R>::Rs(I, 1) * u1;
                    const R cvr = Cst<R>::cv(I, 0) * u0 + Cst<R>::cv(I, 1) * u1;
                    xr[c] = u0 + u1;
                    xR[c] = rr * Ar<R>::rcp(xr[c]);
                    xG[c] = (Cst<R>::cvG(I, 0) * u0 + Cst<R>::cvG(I, 1) * u1) * Ar<R>::rcp(cvr);
                    xp[c] = rr * Ar<R>::rcp(beta) - Cst<R>::pinf(I);
                } else {
                    xp[c] = NR(Y::X + 0, 2 + c);
                    xr[c] = NR(Y::X + 1, 2 + c);
                    xl[c] = NR(Y::X + 2, 2 + c);
                    xR[c] = NR(Y::X + 3, 2 + c);
                    xG[c] = NR(Y::X + 4, 2 + c);
                }
            }
            R rb;
            if constexpr (Y::COMPACT) rb = Ar<R>::lmean(xr[0], xr[1]);
            else rb = Ar<R>::lmean(xr[0], xr[1], xl[0], xl[1]);
            const R Rb = R(0.5) * (xR[0] + xR[1]);
            const R Gb = R(0.5) * (xG[0] + xG[1]);
            const R pb = R(0.5) * (xp[0] + xp[1]);
            R rh = pb + Cst<R>::pinf(I) + (Cst<R>::cv(I, 0) * lr_c[0] + Cst<R>::cv(I, 1) * lr_c[1]) * Tb;
            R irb = Ar<R>::rcp(rb);
            Y1 = lr_c[0] * irb;
            Y2 = lr_c[1] * irb;
            H = rh * irb + R(0.5) * vv;
            cb = Ar<R>::sq(Rb * Gb * Tb);
            const R pre = Ar<R>::sq(rb * Ar<R>::rcp(Gb * Rb));
            sa = pre * R(0.70710678118654752440);
            ssh = Ar<R>::sq(rb * Tb);
            const R R1 = Cst<R>::Rs(I, 0), R2 = Cst<R>::Rs(I, 1);
            R sy = Ar<R>::sq(Y1 * Y2), sg = Ar<R>::sq(Gb - R(1));
            D11 = -pre * sy * Ar<R>::sq(Gb * R2 * Ar<R>::rcp(R1));
            D21 = pre * sy * Ar<R>::sq(Gb * R1 * Ar<R>::rcp(R2));
            D12 = pre * Y1 * sg;
            D22 = pre * Y2 * sg;
            R igm = Ar<R>::rcp(Gb - R(1));
            e1 = R(0.5) * vv - (Cst<R>::cv(I, 0) + R1 - Gb * Cst<R>::cv(I, 0)) * Tb * igm;
            e2 = R(0.5) * vv - (Cst<R>::cv(I, 1) + R2 - Gb * Cst<R>::cv(I, 1)) * Tb * igm;
        }
        const R lam = Ar<R>::ab(to_r<R>(Gt) + Ln * vh[0]) + Ln * cb;
        // round-off band of [[W_m]]: delta ||r_m|| (||V_i|| + ||V_i+1||)
        R nvb;
        if constexpr (Y::COMPACT) nvb = vnorm<NC, Y::VV, R>(nb + 2 * ns, NN) + vnorm<NC, Y::VV, R>(nb + 3 * ns, NN);
        else nvb = NR(Y::VN, 2) + NR(Y::VN, 3);
        const R band2 = R(YBand<R>::value * YBand<R>::value) * nvb * nvb;
        const R ch1 = Cst<R>::chi(I, 0), ch2 = Cst<R>::chi(I, 1), ch3 = Cst<R>::chi(I, 2), eps = Cst<R>::eps(I);
        R Fd[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) Fd[q] = R(0);
        // the two acoustic columns first, so that their averages are dead for the others.  The
        // 3D two-species tiles keep the loop rolled: unrolled it spills at the 64 registers of 4
        // blocks per SM (800 bytes of spill loads against 212), and rolled it ran the Example 5.11
        // flux launches 11% faster; elsewhere the unrolled loop is the faster one.
#pragma unroll((D == 3 && NS == 2) ? 1 : NC)
        for (int ci = 0; ci < NC; ++ci) {
            const int col = ci == 0 ? 0 : (ci == 1 ? NC - 1 : ci - 1);
            // column col of R in the rotated frame
            R rc[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) rc[q] = R(0);
            if (col == 0 || col == NC - 1) {
                const R sg = col == 0 ? R(-1) : R(1);
                if (NS == 1) rc[0] = R(1);
                else { rc[0] = Y1; rc[1] = Y2; }
#pragma unroll
                for (int j = 0; j < D; ++j) rc[NS + j] = vh[j];
                rc[NS] += sg * cb;
                rc[NS + D] = H + sg * cb * vh[0];
#pragma unroll
                for (int q = 0; q < NC; ++q) rc[q] *= sa;
            } else if (col <= NS) {
                if constexpr (NS == 1) {
#pragma unroll
                    for (int j = 0; j < D; ++j) rc[1 + j] = se * vh[j];
                    rc[0] = se;
                    rc[1 + D] = se * R(0.5) * vv;
                } else {
                    const R da = col == 1 ? D11 : D12, db = col == 1 ? D21 : D22;
                    rc[0] = da;
                    rc[1] = db;
#pragma unroll
                    for (int j = 0; j < D; ++j) rc[2 + j] = (da + db) * vh[j];
                    rc[2 + D] = da * e1 + db * e2;
                }
            } else {
                const int mm = col - NS;      // shear: rotated velocity component mm (1..D-1)
#pragma unroll
                for (int j = 1; j < D; ++j)   // a constant register index also when the loop is rolled
                    if (j == mm) {
                        rc[NS + j] = ssh;
                        rc[NS + D] = ssh * vh[j];
                    }
            }
            // back to the unrotated frame: T^T on the velocity block
            R ru[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                R s_ = R(0);
#pragma unroll
                for (int m = 0; m < D; ++m) s_ += T[m][j] * rc[NS + m];
                ru[j] = s_;
            }
#pragma unroll
            for (int j = 0; j < D; ++j) rc[NS + j] = ru[j];
            // scaled entropy variables W_j = r_col . V_j at the six nodes, then W^- and W^+
            R Wm, Wp, jp;
            if constexpr (std::is_same<R, float>::value && WK == 0) {
                // binary32 WENO-MR: the node pairs (0,5), (1,4), (2,3) of the two stencils in paired lanes
                float2 p05 = f2(0.0f), p14 = f2(0.0f), p23 = f2(0.0f);
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const float2 rq = f2(rc[q]);
                    p05 = fma2(rq, make_float2(NR(Y::VV + q, 0), NR(Y::VV + q, 5)), p05);
                    p14 = fma2(rq, make_float2(NR(Y::VV + q, 1), NR(Y::VV + q, 4)), p14);
                    p23 = fma2(rq, make_float2(NR(Y::VV + q, 2), NR(Y::VV + q, 3)), p23);
                }
                const float2 r = weno_mr_pair(p05, p14, p23, make_float2(p23.y, p23.x), make_float2(p14.y, p14.x),
                                              ch1, ch2, ch3, I.f_ichi3, eps);
                Wm = r.x;
                Wp = r.y;
                jp = p23.y - p23.x;
            } else {
                R wv[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    R s_ = R(0);
#pragma unroll
                    for (int q = 0; q < NC; ++q) s_ += rc[q] * NR(Y::VV + q, j);
                    wv[j] = s_;
                }
                Wm = weno_val<R, WK>(wv[0], wv[1], wv[2], wv[3], wv[4], ch1, ch2, ch3, eps);
                Wp = weno_val<R, WK>(wv[5], wv[4], wv[3], wv[2], wv[1], ch1, ch2, ch3, eps);
                jp = wv[3] - wv[2];
            }
            R jw = Wp - Wm;
            R rn = R(0);
#pragma unroll
            for (int q = 0; q < NC; ++q) rn += rc[q] * rc[q];
            const bool sig = jp * jp > band2 * rn;
            if (sig && ((jw > R(0) && jp > R(0)) || (jw < R(0) && jp < R(0)))) {
                R cf = lam * jw;
#pragma unroll
                for (int q = 0; q < NC; ++q) Fd[q] += rc[q] * cf;
            }
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) fl[q * NI + f] = fl[q * NI + f] - R(0.5) * Fd[q];
    }
#undef NR
}

// Shu-Osher stage of one FP64 field (SSP-RK3, Sec. 5): a q^n + b (q + dt r).  The first stage
// (a = 0, b = 1) is q + dt r, one fused multiply-add; the others b (q + dt r) + a q^n with the
// outer product fused.  q0 points at q^n (read only when a != 0).
__device__ __forceinline__ double rk_stage(const FluxLaunch& L, double q, const double* q0, double dt, double r)
{
    const double s = fma(dt, r, q);
    return (L.a == 0.0 && L.b == 1.0) ? s : fma(L.b, s, L.a * *q0);
}

// Phase 4 of one node along direction k: r[0..NC) = -(F_{i+1/2} - F_{i-1/2}) / dxi_k from
// the interface fluxes at fr and fL (field stride NI), r[NC] the same of the FP64 GCL flux
// (the J equation), and the p_inf J xi_k/t part of the energy flux added in FP64
template <int NC, typename R>
__device__ __forceinline__ void node_div(const Inst& I, const R* fl, int NI, const double* gt, int fr, int fL,
                                         double inv_dx, double* r)
{
    const R rdx = to_r<R>(inv_dx);
    r[NC] = -(gt[fr] - gt[fL]) * inv_dx;
#pragma unroll
    for (int q = 0; q < NC; ++q) r[q] = to_d(-(fl[q * NI + fr] - fl[q * NI + fL]) * rdx);
    r[NC - 1] += I.pinf_tot * r[NC];
}

}  // namespace es
