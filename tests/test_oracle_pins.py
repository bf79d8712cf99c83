"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, an identity the paper states (consistency, Tadmor's EC condition,
the rotation identity, dU/dV = R R^T), a closed form, an independent symbolic
derivation, or an invariant of the scheme (discrete SCL / free-stream, zero
entropy production of the EC scheme, design order).  No GPU is needed.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2202_07989_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))

CASES = [(2, 1), (2, 2), (3, 1), (3, 2)]


def _random_state(pb, rng, pinf_scale=1.0):
    rl = rng.uniform(0.3, 2.0, size=pb.N)
    v = rng.uniform(-1.0, 1.0, size=pb.d)
    p = rng.uniform(0.3, 2.0)
    return W.cons_state(pb, rl, v, p)[: pb.nc]


def _pb(d, N, pinf=0.0, **kw):
    pb = W.random_problem(d, N, (12,) * d, pinf=pinf, **kw)
    if N == 2 and pinf:
        pb = pb.with_(pinf=(pinf, 0.5 * pinf))
    return pb


# ---------------------------------------------------------------------------
# coefficients
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("w", [1, 2, 3])
def test_alpha_matches_paper_conditions(w):
    """alpha_{w,m} of Sec. 3.1 equal the exact rational solutions."""
    o = Oracle(_pb(2, 1))
    want = [float(Fraction(a, b)) for a, b in GOLD["alpha"]["w%d" % w]]
    np.testing.assert_allclose(o.alpha(w), want, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# pointwise physics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("pinf", [0.0, 2.5])
def test_entropy_variables_are_gradient_of_eta(d, N, pinf):
    """V = eta'(U)^T (Definition of the entropy pair, Sec. 1) by central differences of eta."""
    pb = _pb(d, N, pinf)
    o = Oracle(pb)
    rng = np.random.default_rng(11)
    for _ in range(5):
        U = _random_state(pb, rng)
        V = o.entropy_vars(U)
        g = np.zeros(pb.nc)
        for q in range(pb.nc):
            h = 1e-6 * max(1.0, abs(U[q]))
            up, um = U.copy(), U.copy()
            up[q] += h
            um[q] -= h
            g[q] = (o.eta(up) - o.eta(um)) / (2 * h)
        np.testing.assert_allclose(V, g, rtol=2e-7, atol=2e-7)


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("pinf", [0.0, 2.5])
def test_potentials(d, N, pinf):
    """phi = V^T U - eta and psi_k = V^T F_k - q_k = phi v_k with q_k = eta v_k (Sec. 1, Sec. 3.3)."""
    pb = _pb(d, N, pinf)
    o = Oracle(pb)
    rng = np.random.default_rng(12)
    for _ in range(5):
        U = _random_state(pb, rng)
        V, eta, phi = o.entropy_vars(U), o.eta(U), o.phi(U)
        _, v, _, _ = o.primitives(U)
        assert abs(V @ U - eta - phi) <= 1e-13 * (abs(V) @ abs(U) + abs(eta))
        for k in range(d):
            F = o.phys_flux(k, U)
            lhs = V @ F - eta * v[k]
            assert abs(lhs - phi * v[k]) <= 1e-13 * (abs(V) @ abs(F) + abs(eta * v[k]))


def test_logmean_against_high_precision():
    """{a}^ln = [[a]]/[[ln a]] (Sec. 3.3.1) to 1e-15 across both branches (mpmath reference)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    o = Oracle(_pb(2, 1))
    rng = np.random.default_rng(13)
    for rel in [0.0, 1e-14, 1e-9, 1e-5, 1e-3, 0.019, 0.021, 0.1, 1.0, 10.0]:
        for _ in range(20):
            a = rng.uniform(0.1, 10.0)
            b = a * (1.0 + rel * rng.uniform(-1, 1)) if rel < 1 else a * rng.uniform(1.0, 1.0 + rel)
            got = o.logmean(a, b)
            A, B = mpmath.mpf(a), mpmath.mpf(b)
            want = A if A == B else (B - A) / (mpmath.log(B) - mpmath.log(A))
            f = (b - a) / (b + a)
            # series branch: a few ulps; [[a]]/[[ln a]] branch: cancellation in [[ln a]]
            # costs about 5e-16 / |[[ln a]]|, at most ~3e-14 above the branch threshold
            tol = 2e-15 if f * f < 1e-4 else 1e-13
            assert abs(got - float(want)) <= tol * float(want), (a, b, got, float(want))
            assert got == o.logmean(b, a)


# ---------------------------------------------------------------------------
# two-point EC flux (Sec. 3.3)
# ---------------------------------------------------------------------------

def _random_metrics(d, rng):
    return rng.uniform(-1.0, 1.0, size=d + 1) + np.r_[0.0, np.ones(d)]


def _pair(pb, rng, kind):
    Ul = _random_state(pb, rng)
    if kind == "near":
        rl, v, T, p = Oracle(pb).primitives(Ul)
        rl2 = rl * (1 + 1e-4 * rng.uniform(-1, 1, size=pb.N))
        v2 = v + 1e-4 * rng.uniform(-1, 1, size=pb.d)
        p2 = p * (1 + 1e-4 * rng.uniform(-1, 1))
        Ur = W.cons_state(pb, rl2, v2, p2)[: pb.nc]
    else:
        Ur = _random_state(pb, rng)
    return Ul, Ur


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("pinf", [0.0, 2.5])
def test_ec_pair_consistency(d, N, pinf):
    """F(U, U, M, M) = J xi_t U + sum_j J xi_x_j F_j(U) (Proposition 3.1)."""
    pb = _pb(d, N, pinf)
    o = Oracle(pb)
    rng = np.random.default_rng(14)
    for _ in range(10):
        U = _random_state(pb, rng)
        M = _random_metrics(d, rng)
        got = o.ec_pair(U, U, M, M)
        want = M[0] * U + sum(M[1 + j] * o.phys_flux(j, U) for j in range(d))
        scale = abs(M[0]) * abs(U) + sum(abs(M[1 + j]) * abs(o.phys_flux(j, U)) for j in range(d))
        assert np.all(np.abs(got - want) <= 1e-13 * scale)


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("pinf", [0.0, 2.5])
@pytest.mark.parametrize("kind", ["far", "near"])
def test_ec_condition_and_symmetry(d, N, pinf, kind):
    """Tadmor's condition Eq. (ECCondition_curv) to 1e-13 relative; symmetry F(l,r) = F(r,l)."""
    pb = _pb(d, N, pinf)
    o = Oracle(pb)
    rng = np.random.default_rng(15)
    for _ in range(20):
        Ul, Ur = _pair(pb, rng, kind)
        Ml, Mr = _random_metrics(d, rng), _random_metrics(d, rng)
        F = o.ec_pair(Ul, Ur, Ml, Mr)
        assert np.array_equal(F, o.ec_pair(Ur, Ul, Mr, Ml))
        dV = o.entropy_vars(Ur) - o.entropy_vars(Ul)
        _, vl, _, _ = o.primitives(Ul)
        _, vr, _, _ = o.primitives(Ur)
        pl, pr = o.phi(Ul), o.phi(Ur)
        rhs = 0.5 * (Ml[0] + Mr[0]) * (pr - pl)
        scale = abs(0.5 * (Ml[0] + Mr[0])) * (abs(pr) + abs(pl))
        for j in range(d):
            mj = 0.5 * (Ml[1 + j] + Mr[1 + j])
            rhs += mj * (pr * vr[j] - pl * vl[j])
            scale += abs(mj) * (abs(pr * vr[j]) + abs(pl * vl[j]))
        lhs = dV @ F
        scale += np.abs(o.entropy_vars(Ur)) @ np.abs(F) + np.abs(o.entropy_vars(Ul)) @ np.abs(F)
        assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("N", [1, 2])
def test_rotation_identity(N):
    """F~_{phi,theta} = T^{-1} F~_1(T U_l, T U_r) (Eq. (rotation)) gives F~_2, F~_3 at the two
    stated angle pairs and the normal combination sum_j n_j F~_j for any angles."""
    pb = _pb(3, N, 1.5)
    o = Oracle(pb)
    rng = np.random.default_rng(16)

    def Tmat(ph, th):
        T = np.eye(pb.nc)
        cp, sp, ct, st = math.cos(ph), math.sin(ph), math.cos(th), math.sin(th)
        T[N:N + 3, N:N + 3] = [[cp * ct, cp * st, sp], [-st, ct, 0], [-sp * ct, -sp * st, cp]]
        return T

    for _ in range(10):
        Ul, Ur = _pair(pb, rng, "far")
        for (ph, th), j in [((0.0, math.pi / 2), 1), ((math.pi / 2, 0.0), 2)]:
            T = Tmat(ph, th)
            got = np.linalg.solve(T, o.Ftilde(0, T @ Ul, T @ Ur))
            np.testing.assert_allclose(got, o.Ftilde(j, Ul, Ur), rtol=1e-13, atol=1e-13)
        ph, th = rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi)
        T = Tmat(ph, th)
        n = T[N, N:N + 3]
        got = np.linalg.solve(T, o.Ftilde(0, T @ Ul, T @ Ur))
        want = sum(n[j] * o.Ftilde(j, Ul, Ur) for j in range(3))
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# scaled eigenvectors (Sec. 3.4, Eq. (eigen))
# ---------------------------------------------------------------------------

def _jac(f, U, n):
    Jm = np.zeros((n, len(U)))
    for q in range(len(U)):
        h = 1e-6 * max(1.0, abs(U[q]))
        up, um = U.copy(), U.copy()
        up[q] += h
        um[q] -= h
        Jm[:, q] = (f(up) - f(um)) / (2 * h)
    return Jm


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("pinf", [0.0, 2.5])
def test_scaled_eigenvectors(d, N, pinf):
    """dU/dV = R R^T and dF_1/dU R = R Lambda with Lambda = diag(v1-c, v1, .., v1, v1+c)."""
    pb = _pb(d, N, pinf)
    o = Oracle(pb)
    rng = np.random.default_rng(17)
    for _ in range(4):
        U = _random_state(pb, rng)
        R = o.eigvec_point(U)
        dVdU = _jac(o.entropy_vars, U, pb.nc)
        np.testing.assert_allclose(R @ R.T @ dVdU, np.eye(pb.nc), atol=2e-6)
        rl, v, T, p = o.primitives(U)
        rho = rl.sum()
        Rm = sum((pb.gamma[l] - 1) * pb.cv[l] * rl[l] for l in range(N)) / rho
        Gm = sum(pb.gamma[l] * pb.cv[l] * rl[l] for l in range(N)) / sum(pb.cv[l] * rl[l] for l in range(N))
        c = math.sqrt(Rm * Gm * T)
        lam = np.array([v[0] - c] + [v[0]] * (pb.nc - 2) + [v[0] + c])
        A = _jac(lambda u: o.phys_flux(0, u), U, pb.nc)
        np.testing.assert_allclose(A @ R, R * lam[None, :], atol=2e-6 * max(1.0, np.abs(A @ R).max()))


@pytest.mark.parametrize("d,N", CASES)
def test_interface_eigenvectors_reduce_to_point(d, N):
    """With U_l = U_r the averaged R of Sec. 3.4 equals the point-state R."""
    pb = _pb(d, N, 1.0)
    o = Oracle(pb)
    rng = np.random.default_rng(18)
    U = _random_state(pb, rng)
    R, _ = o.eigvec_avg(U, U)
    np.testing.assert_allclose(R, o.eigvec_point(U), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d,N", CASES)
def test_interface_averages_are_symmetric_and_between(d, N):
    """The interface averages of Sec. 3.4 are means of the two states: swapping the states
    leaves the averaged R and c-bar unchanged, and c-bar^2 = R-bar Gamma-bar T-bar lies between
    the smallest and largest products of the two states' R_mix, Gamma_mix and T (T-bar is a
    mean of T, R-bar and Gamma-bar are means of the mixture values).  A one-sided value (the
    left state's in place of a mean) or a wrong average (a sum, rho-bar in place of T-bar)
    fails one of them."""
    pb = _pb(d, N, 1.0)
    o = Oracle(pb)
    rng = np.random.default_rng(19 + 10 * d + N)

    def mix(U):
        rho_l = U[:N]
        rho = rho_l.sum()
        v2 = sum((U[N + m] / rho) ** 2 for m in range(d))
        cvr = sum(pb.cv[l] * rho_l[l] for l in range(N))
        rr = sum(pb.R(l) * rho_l[l] for l in range(N))
        T = (U[N + d] - 0.5 * rho * v2 - sum(pb.pinf[:N])) / cvr
        gmix = sum(pb.gamma[l] * pb.cv[l] * rho_l[l] for l in range(N)) / cvr
        return rr / rho, gmix, T

    for _ in range(20):
        Ul, Ur = _random_state(pb, rng), _random_state(pb, rng)
        R1, c1 = o.eigvec_avg(Ul, Ur)
        R2, c2 = o.eigvec_avg(Ur, Ul)
        np.testing.assert_allclose(R1, R2, rtol=1e-13, atol=1e-13 * np.abs(R1).max())
        assert abs(c1 - c2) <= 1e-13 * c1
        (Rl, Gl, Tl), (Rr, Gr, Tr) = mix(Ul), mix(Ur)
        lo = min(Rl, Rr) * min(Gl, Gr) * min(Tl, Tr)
        hi = max(Rl, Rr) * max(Gl, Gr) * max(Tl, Tr)
        assert lo * (1 - 1e-12) <= c1 * c1 <= hi * (1 + 1e-12), (lo, c1 * c1, hi)


# ---------------------------------------------------------------------------
# WENO-MR (Appendix A)
# ---------------------------------------------------------------------------

def test_weno_linear_limit_is_five_point_stencil():
    """With linear weights (eps -> infinity) the value is h_3(x_{j+1/2}) = (2,-13,47,27,-3)/60."""
    o = Oracle(_pb(2, 1))
    rng = np.random.default_rng(19)
    st = np.array(GOLD["weno_mr"]["linear_stencil_60ths"]) / 60.0
    for _ in range(20):
        w5 = rng.uniform(-2, 2, size=5)
        got = o.weno_mr(w5, eps=1e30)
        assert abs(got - st @ w5) <= 1e-14 * (np.abs(st) @ np.abs(w5))


def test_weno_weights_from_symbolic_indicators():
    """beta_1..beta_3, tau and the nonlinear weights rebuilt from the definitions of
    Appendix A with sympy (beta_2, beta_3 integrated over the central cell), then
    compared with the oracle's WENO-MR value."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    Ws = sp.symbols("w0:5")
    L = [sp.Integer(1), x, x ** 2 - sp.Rational(1, 12), x ** 3 - sp.Rational(3, 20) * x,
         x ** 4 - sp.Rational(3, 14) * x ** 2 + sp.Rational(3, 560)]

    def recon(deg, cells):
        cs = sp.symbols("c0:%d" % (deg + 1))
        h = sum(ci * Li for ci, Li in zip(cs, L))
        eqs = [sp.integrate(h, (x, l - sp.Rational(1, 2), l + sp.Rational(1, 2))) - Ws[l + 2] for l in cells]
        return sp.expand(h.subs(sp.solve(eqs, cs)))

    h2 = recon(2, [-1, 0, 1])
    h3 = recon(4, [-2, -1, 0, 1, 2])
    half = sp.Rational(1, 2)

    def beta(h, deg):
        return sum(sp.integrate(sp.diff(h, x, a) ** 2, (x, -half, half)) for a in range(1, deg + 1))

    b2f = sp.lambdify(Ws, beta(h2, 2))
    b3f = sp.lambdify(Ws, beta(h3, 4))
    h2f = sp.lambdify(Ws, h2.subs(x, half))
    h3f = sp.lambdify(Ws, h3.subs(x, half))
    o = Oracle(_pb(2, 1))
    chi = np.array([float(Fraction(a, b)) for a, b in GOLD["weno_mr"]["chi"]])
    eps = GOLD["weno_mr"]["eps"]
    rng = np.random.default_rng(20)
    samples = [rng.uniform(-1, 1, size=5) for _ in range(30)]
    samples += [np.array([0, 0, 0, 0, 1.0]), np.array([0, 0, 1.0, 1, 1]), np.array([1.0, 1, 1, 0, 0])]
    for w in samples:
        b1 = min((w[2] - w[1]) ** 2, (w[3] - w[2]) ** 2)
        b2, b3 = b2f(*w), b3f(*w)
        tau = (0.5 * (abs(b3 - b1) + abs(b3 - b2))) ** 2
        wb = chi * (1 + tau / (eps + np.array([b1, b2, b3])))
        om = wb / wb.sum()
        hv = np.array([w[2], h2f(*w), h3f(*w)])
        want = om[0] * hv[0] + om[1] * hv[1] + om[2] * (hv[2] / chi[2] - chi[0] / chi[2] * hv[0] - chi[1] / chi[2] * hv[1])
        got = o.weno_mr(w)
        assert abs(got - want) <= 1e-12 * max(1.0, np.abs(w).max()), (w, got, want)


def test_weno_jump_is_fifth_order():
    """[[W]]^WENOMR = W^+ - W^- at x_{j+1/2} vanishes at fifth order on smooth data."""
    o = Oracle(_pb(2, 1))
    errs = []
    for n in [20, 40, 80]:
        h = 2 * math.pi / n
        xs = 0.3 + h * np.arange(-2, 4)
        f = np.sin(xs)
        wm = o.weno_mr(f[0:5])
        wp = o.weno_mr(f[5:0:-1])
        errs.append(abs(wp - wm))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 4.5, (errs, orders)


# ---------------------------------------------------------------------------
# classical WENO-JS (the MM-WENOJS comparison of Sec. 5)
# ---------------------------------------------------------------------------

def test_weno_js_linear_limit_is_five_point_stencil():
    """With linear weights (eps -> infinity) WENO-JS also gives (2,-13,47,27,-3)/60."""
    o = Oracle(_pb(2, 1))
    rng = np.random.default_rng(31)
    st = np.array(GOLD["weno_mr"]["linear_stencil_60ths"]) / 60.0
    for _ in range(20):
        w5 = rng.uniform(-2, 2, size=5)
        got = o.weno_js(w5, eps=1e30)
        assert abs(got - st @ w5) <= 1e-14 * (np.abs(st) @ np.abs(w5))


def test_weno_js_from_symbolic_definitions():
    """Candidate values, smoothness indicators and linear weights rebuilt with sympy from
    their definitions (quadratic reconstructions of three cell averages; beta_k = sum over
    the first two derivatives of the squared derivative integrated over the central cell;
    linear weights that reproduce the five-cell reconstruction), then compared with the
    oracle's WENO-JS value."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    Ws = sp.symbols("w0:5")
    half = sp.Rational(1, 2)

    def recon(deg, cells):
        cs = sp.symbols("c0:%d" % (deg + 1))
        h = sum(ci * x ** i for i, ci in enumerate(cs))
        eqs = [sp.integrate(h, (x, l - half, l + half)) - Ws[l + 2] for l in cells]
        return sp.expand(h.subs(sp.solve(eqs, cs)))

    p = [recon(2, [-2, -1, 0]), recon(2, [-1, 0, 1]), recon(2, [0, 1, 2])]
    p5 = recon(4, [-2, -1, 0, 1, 2])
    dk = sp.symbols("d0:3")
    lin = sp.expand(sum(dk[k] * p[k].subs(x, half) for k in range(3)) - p5.subs(x, half))
    dsol = sp.solve([lin.coeff(w) for w in Ws], dk)
    d = np.array([float(dsol[dk[k]]) for k in range(3)])
    assert np.allclose(d, [0.1, 0.6, 0.3], rtol=0, atol=1e-15)
    beta = [sp.lambdify(Ws, sum(sp.integrate(sp.diff(pk, x, a) ** 2, (x, -half, half)) for a in (1, 2))) for pk in p]
    qv = [sp.lambdify(Ws, pk.subs(x, half)) for pk in p]
    o = Oracle(_pb(2, 1))
    eps = GOLD["weno_mr"]["eps"]
    rng = np.random.default_rng(32)
    samples = [rng.uniform(-1, 1, size=5) for _ in range(30)]
    samples += [np.array([0, 0, 0, 0, 1.0]), np.array([0, 0, 1.0, 1, 1]), np.array([1.0, 1, 1, 0, 0])]
    for w in samples:
        b = np.array([f(*w) for f in beta])
        q = np.array([f(*w) for f in qv])
        a = d / (eps + b) ** 2
        want = (a @ q) / a.sum()
        got = o.weno_js(w)
        assert abs(got - want) <= 1e-13 * max(1.0, np.abs(w).max()), (w, got, want)


def test_weno_js_jump_is_fifth_order_and_eno_at_a_step():
    """[[W]]^WENOJS vanishes at fifth order on smooth data away from extrema, and at a step
    the reconstruction comes from the smooth side."""
    o = Oracle(_pb(2, 1))
    errs = []
    for n in [20, 40, 80]:
        h = 2 * math.pi / n
        xs = 0.3 + h * np.arange(-2, 4)
        f = np.sin(xs)
        errs.append(abs(o.weno_js(f[5:0:-1]) - o.weno_js(f[0:5])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 4.5, (errs, orders)
    assert abs(o.weno_js(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))) < 1e-6
    assert abs(o.weno_js(np.array([0.0, 0.0, 1.0, 1.0, 1.0])) - 1.0) < 1e-6


# ---------------------------------------------------------------------------
# metrics (Sec. 3.2)
# ---------------------------------------------------------------------------

def _interior(pb, M, depth):
    sl = [slice(None)]
    for k in (2, 1, 0):
        if k < pb.d:
            sl.append(slice(3 + depth, 3 + pb.n[k] - depth))
        else:
            sl.append(slice(None))
    return M[tuple(sl)]


@pytest.mark.parametrize("d,w", [(2, 1), (2, 2), (2, 3), (3, 3)])
def test_metrics_exact_for_polynomial_maps(d, w):
    """J xi_k/x_j of Eq. (SCLCoeff) (and the 2D degenerate case) equal the cofactors of
    dx/dxi for polynomial maps the 2w-order central differences differentiate exactly
    (degree 2w in 2D)."""
    n = 20 if d == 2 else 16
    pb = W.random_problem(d, 1, (n,) * d, bc="reflect").with_(w=w)
    o = Oracle(pb)
    rng = np.random.default_rng(21)
    xi = W.xi_nodes(pb)
    deg = 2 * w if d == 2 else 2
    coef = rng.uniform(-0.05, 0.05, size=(d, d, deg + 1))

    def comp(j, xs):
        out = xs[j].copy()
        for k in range(d):
            for e in range(1, deg + 1):
                out = out + coef[j, k, e] * xs[k] ** e
        return out

    def dcomp(j, k, xs):
        return (1.0 if j == k else 0.0) + sum(e * coef[j, k, e] * xs[k] ** (e - 1) for e in range(1, deg + 1))

    x = np.stack([comp(j, xi) for j in range(d)])
    M = o.metrics(x)
    depth = 3 if d == 2 else 6
    A = np.zeros((d, d) + pb.shape)
    for j in range(d):
        for k in range(d):
            A[j, k] = dcomp(j, k, xi)
    # cofactor C[k][j] = det(A) (A^{-1})[k][j]
    Am = np.moveaxis(A, (0, 1), (-2, -1))
    cof = np.linalg.det(Am)[..., None, None] * np.linalg.inv(Am)
    for k in range(d):
        for j in range(d):
            got = _interior(pb, M[k * (d + 1) + 1 + j][None], depth)[0]
            sl = tuple(slice(depth, pb.shape[a] - depth) if (2 - a) < d else slice(None) for a in range(3))
            np.testing.assert_allclose(got, cof[..., k, j][sl], rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,w", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
@pytest.mark.parametrize("bc", ["periodic", "mixed"])
def test_discrete_scl(d, w, bc):
    """Discrete SCL Eq. (SCL_dis): sum_k delta_k[J xi_k/x_j]/dxi_k = 0 at every node
    (the GCL-flux difference telescopes to delta_k), random smooth moving meshes, each order 2w."""
    n = 12 if d == 2 else 10
    pb = W.random_problem(d, 1, (n,) * d, bc=bc).with_(w=w)
    o = Oracle(pb)
    rng = np.random.default_rng(22)
    x = W.smooth_mesh(pb, rng)
    M = o.metrics(x)
    al = list(o.alpha(w)) + [0.0] * (3 - w)
    for j in range(d):
        tot = 0.0
        for k in range(d):
            f = M[k * (d + 1) + 1 + j]
            ax = 2 - k
            dk = sum(0.5 * al[m - 1] * (np.roll(f, -m, axis=ax) - np.roll(f, m, axis=ax)) for m in (1, 2, 3))
            tot = tot + dk / pb.dxi[k]
        inner = _interior(pb, np.asarray(tot)[None], 0)[0]
        assert np.abs(inner).max() <= 1e-11 * np.abs(M).max()


# ---------------------------------------------------------------------------
# whole residual
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("es", [False, True])
@pytest.mark.parametrize("w", [1, 2, 3])
def test_free_stream_preservation(d, N, es, w):
    """A constant state on a randomly perturbed moving mesh stays constant: d(JU)/dt = U dJ/dt
    for the residual and U is unchanged to round-off after SSP-RK3 steps (remark in Sec. 3.2),
    for each order 2w."""
    n = 12 if d == 2 else 10
    pb = W.random_problem(d, N, (n,) * d, pinf=1.0 if N == 1 else 0.0, es=es).with_(w=w)
    o = Oracle(pb)
    rng = np.random.default_rng(23)
    x = W.smooth_mesh(pb, rng)
    xdot = 0.3 * W.smooth_mesh(pb, rng) - 0.3 * np.stack(W.xi_nodes(pb))
    U0 = _random_state(pb, rng)
    J = o.init_J(x)
    U = np.broadcast_to(U0.reshape((-1,) + (1,) * 3), (pb.nc,) + pb.shape).copy()
    JU = U * J
    dJU, dJ = o.rhs(JU, J, x, xdot)
    scale = np.abs(U).max() * max(np.abs(dJ).max(), 1.0) / min(pb.dxi[: d])
    assert np.abs(dJU - U * dJ).max() <= 1e-12 * scale
    dt = 0.2 * min(pb.dxi[:d])
    for _ in range(2):
        JU, J, x = o.rk_step(JU, J, x, xdot, dt)
    np.testing.assert_allclose(JU / J, U, rtol=1e-12, atol=1e-12 * np.abs(U).max())


@pytest.mark.parametrize("d,N", CASES)
def test_ec_entropy_production_zero(d, N):
    """The EC scheme on periodic data satisfies the semi-discrete entropy identity
    Eq. (NumEntropyID): P = sum (V^T dJU - phi dJ) dxi^d = 0 (telescoping)."""
    n = 12 if d == 2 else 8
    pb = W.random_problem(d, N, (n,) * d, es=False, pinf=0.5 if N == 1 else 0.0)
    o = Oracle(pb)
    rng = np.random.default_rng(24)
    x = W.smooth_mesh(pb, rng)
    xdot = 0.3 * (W.smooth_mesh(pb, rng) - np.stack(W.xi_nodes(pb)))
    U = W.smooth_state(pb, x, rng, amp=0.3)
    J = o.init_J(x)
    JU = U * J
    dJU, dJ = o.rhs(JU, J, x, xdot)
    P, _ = o.entropy(JU, J, dJU, dJ)
    V = np.stack([o.entropy_vars(U[(slice(None),) + idx]) for idx in np.ndindex(pb.shape)], axis=1)
    scale = (np.abs(V) * np.abs(dJU.reshape(pb.nc, -1))).sum() * np.prod(pb.dxi[:d])
    assert abs(P) <= 1e-12 * scale, (P, scale)


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("weno", [0, 1])
def test_es_entropy_production_nonpositive(d, N, weno):
    """The ES scheme dissipates entropy: P <= 0 (Sec. 3.4, the sign property of Y, which holds
    for any reconstruction of [[W]], so for WENO-MR and WENO-JS), on smooth and on
    discontinuous periodic data."""
    n = 12 if d == 2 else 8
    pb = W.random_problem(d, N, (n,) * d, es=True).with_(weno=weno)
    o = Oracle(pb)
    rng = np.random.default_rng(25)
    x = W.smooth_mesh(pb, rng)
    xdot = 0.3 * (W.smooth_mesh(pb, rng) - np.stack(W.xi_nodes(pb)))
    J = o.init_J(x)
    for kind in ["smooth", "jump"]:
        U = W.smooth_state(pb, x, rng, amp=0.3)
        if kind == "jump":
            mask = (x[0] > 0.5)
            U = np.where(mask[None], U * 2.0, U)
        JU = U * J
        dJU, dJ = o.rhs(JU, J, x, xdot)
        pb_ec = pb.with_(es=False)
        dJU0, dJ0 = Oracle(pb_ec).rhs(JU, J, x, xdot)
        P, _ = o.entropy(JU, J, dJU, dJ)
        P0, _ = o.entropy(JU, J, dJU0, dJ0)
        scale = np.abs(dJU0).sum() * np.prod(pb.dxi[:d])
        assert abs(P0) <= 1e-11 * scale
        assert P <= 1e-12 * scale, (kind, P)


def test_3d_residual_on_extruded_data_equals_2d():
    """A xi_3-independent state with v_3 = 0 on the extruded mesh x_3 = xi_3 gives the 2D
    residual in the (rho, m_1, m_2, E) rows and zero in the m_3 row (Sec. 3: 2D is the
    degenerate case of the 3D scheme)."""
    rng = np.random.default_rng(26)
    pb2 = W.random_problem(2, 1, (12, 12), es=True)
    pb3 = W.random_problem(3, 1, (12, 12, 8), es=True)
    o2, o3 = Oracle(pb2), Oracle(pb3)
    x2 = W.smooth_mesh(pb2, rng)
    xd2 = 0.2 * (W.smooth_mesh(pb2, rng) - np.stack(W.xi_nodes(pb2)))
    U2 = W.smooth_state(pb2, x2, rng)
    n3 = pb3.n[2]
    x3 = np.stack([np.repeat(x2[0], n3, axis=0), np.repeat(x2[1], n3, axis=0), np.stack(W.xi_nodes(pb3))[2]])
    xd3 = np.stack([np.repeat(xd2[0], n3, axis=0), np.repeat(xd2[1], n3, axis=0), np.zeros(pb3.shape)])
    U3 = np.zeros((5,) + pb3.shape)
    U3[[0, 1, 2, 4]] = np.repeat(U2, n3, axis=1)
    J2, J3 = o2.init_J(x2), o3.init_J(x3)
    np.testing.assert_allclose(J3, np.repeat(J2, n3, axis=0), rtol=1e-13)
    r2 = o2.rhs(U2 * J2, J2, x2, xd2)
    r3 = o3.rhs(U3 * J3, J3, x3, xd3)
    want = np.repeat(r2[0], n3, axis=1)
    got = r3[0][[0, 1, 2, 4]]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())
    assert np.abs(r3[0][3]).max() <= 1e-11 * np.abs(want).max()
    np.testing.assert_allclose(r3[1], np.repeat(r2[1], n3, axis=0), atol=1e-12)


def test_two_species_reduce_to_one():
    """N = 2 with identical species and a uniform mass fraction gives the N = 1 EC residual
    (summed species): the log mean is homogeneous, so sum_l {Y rho}^ln = {rho}^ln."""
    rng = np.random.default_rng(27)
    pb1 = W.random_problem(2, 1, (12, 12), es=False)
    pb2 = W.random_problem(2, 2, (12, 12), es=False).with_(gamma=(1.4, 1.4), cv=(1.0, 1.0))
    x = W.smooth_mesh(pb1, rng)
    xd = 0.2 * (W.smooth_mesh(pb1, rng) - np.stack(W.xi_nodes(pb1)))
    U1 = W.smooth_state(pb1, x, rng)
    Y = 0.3
    U2 = np.concatenate([Y * U1[:1], (1 - Y) * U1[:1], U1[1:]])
    o1, o2 = Oracle(pb1), Oracle(pb2)
    J = o1.init_J(x)
    a = o1.rhs(U1 * J, J, x, xd)[0]
    b = o2.rhs(U2 * J, J, x, xd)[0]
    np.testing.assert_allclose(b[0] + b[1], a[0], atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(b[2:], a[1:], atol=1e-12 * np.abs(a).max())


@pytest.mark.slow
def test_design_order_density_wave():
    """Fifth-order accuracy (Sec. 5, Example 5.1) on a smooth density wave advected through
    the periodic unit box on the moving sinusoidal mesh, Delta t = C (min dxi)^{5/3}."""
    errs = []
    ns = [20, 40]
    for n in ns:
        pb = W.random_problem(2, 1, (n, n), es=True)
        o = Oracle(pb)
        xi = W.xi_nodes(pb)
        bump = 0.02 * np.sin(2 * math.pi * xi[0]) * np.sin(2 * math.pi * xi[1])
        x = np.stack([xi[0] + bump, xi[1] + bump])
        xdot = np.stack([bump, bump])

        def exact(xx, t):
            rho = 1.0 + 0.2 * np.sin(2 * math.pi * (xx[0] + xx[1] - 2 * t))
            return W.prim_to_cons(pb, [rho], [np.ones_like(rho), np.ones_like(rho)], np.ones_like(rho))

        J = o.init_J(x)
        JU = exact(x, 0.0) * J
        tend = 0.05
        dt0 = 0.4 * (1.0 / n) ** (5.0 / 3.0)
        nsteps = int(math.ceil(tend / dt0))
        dt = tend / nsteps
        for _ in range(nsteps):
            JU, J, x = o.rk_step(JU, J, x, xdot, dt)
        err = np.abs(JU[0] / J - exact(x, tend)[0]).mean()
        errs.append(err)
    order = math.log2(errs[0] / errs[1])
    assert order > 4.5, (errs, order)


# ---------------------------------------------------------------------------
# time step and mesh (Sec. 4, Eq. (cfl))
# ---------------------------------------------------------------------------

def test_cfl_uniform_mesh_closed_form():
    """On the uniform mesh with a constant state, Eq. (cfl) reads
    Delta t = C / sum_k (|v_k| + c)/dxi_k."""
    pb = W.random_problem(2, 1, (16, 8), es=True).with_(length=(1.0, 0.5, 1.0))
    o = Oracle(pb)
    x = np.stack(W.xi_nodes(pb))
    U0 = W.cons_state(pb, [1.3], [0.4, -0.7], 0.9)[: pb.nc]
    U = np.broadcast_to(U0.reshape(-1, 1, 1, 1), (pb.nc,) + pb.shape).copy()
    J = o.init_J(x)
    np.testing.assert_allclose(J, 1.0, rtol=1e-14)
    c = math.sqrt(1.4 * 0.9 / 1.3)
    want = pb.cfl / ((0.4 + c) / pb.dxi[0] + (0.7 + c) / pb.dxi[1])
    assert abs(o.cfl_dt(U * J, J, x) - want) <= 1e-14 * want


def test_filter_preserves_constants_and_weights():
    """The low-pass filter of Sec. 4 keeps constants and spreads a unit spike with the
    weights (1/2)^(|j|+d)."""
    pb = W.random_problem(3, 1, (8, 8, 8))
    o = Oracle(pb)
    th = np.full(pb.shape, 2.5)
    np.testing.assert_allclose(o.filter(th), 2.5, rtol=1e-15)
    sp = np.zeros(pb.shape)
    sp[4, 4, 4] = 1.0
    f = o.filter(sp)
    g = GOLD["filter_weights"]
    assert f[4, 4, 4] == float(Fraction(*g["centre_3d"]))
    assert f[4, 4, 5] == float(Fraction(*g["face_3d"]))
    assert f[4, 5, 5] == float(Fraction(*g["edge_3d"]))
    assert f[5, 5, 5] == float(Fraction(*g["corner_3d"]))


@pytest.mark.parametrize("bc", ["periodic", "mixed"])
def test_uniform_mesh_is_fixed_point(bc):
    """Theta = const: the uniform mesh solves the discrete mesh equation, so the Jacobi
    sweeps leave it in place and the limiter gives Delta_tau = 1 with zero motion."""
    pb = W.random_problem(2, 1, (16, 12), bc=bc).with_(mu=10)
    o = Oracle(pb)
    x = np.stack(W.xi_nodes(pb))
    xmu = o.jacobi(x, np.full(pb.shape, 1.7))
    np.testing.assert_allclose(xmu, x, rtol=0, atol=1e-14)
    assert o.limiter(x, xmu) == 1.0


def test_monitor_closed_form():
    """Eq. (monitor) with central xi-gradients for sigma = rho = 1 + 0.3 sin(2 pi xi_1)."""
    pb = W.random_problem(2, 1, (16, 8)).with_(alpha=(50.0,), nf=0)
    o = Oracle(pb)
    xi = W.xi_nodes(pb)
    rho = 1.0 + 0.3 * np.sin(2 * math.pi * xi[0])
    U = W.prim_to_cons(pb, [rho], [np.zeros_like(rho)] * 2, np.ones_like(rho))
    J = np.ones(pb.shape)
    h = pb.dxi[0]
    g = np.abs(0.3 * (np.sin(2 * math.pi * (xi[0] + h)) - np.sin(2 * math.pi * (xi[0] - h))) / (2 * h))
    want = np.sqrt(1 + 50.0 * (g / g.max()) ** 2)
    np.testing.assert_allclose(o.monitor(U, J), want, rtol=1e-14)


def test_vortex_monitor_closed_form():
    """Example 5.1's monitor Theta = (1 + 20 |grad_xi rho| / max + 10 |Laplacian_xi rho| / max)^(1/2)
    (linear terms) for rho = 1 + a sin(2 pi xi_1) + b cos(2 pi xi_2) on a periodic grid.  The
    central first and second differences of the trigonometric terms are written with the
    identities sin(t+h) - sin(t-h) = 2 cos t sin h and sin(t+h) - 2 sin t + sin(t-h) =
    -2 sin t (1 - cos h)."""
    pb = W.random_problem(2, 1, (16, 12)).with_(sigma=(W.SIG_RHO, W.SIG_RHO), alpha=(20.0, 10.0),
                                                sigma_op=(W.MON_GRAD, W.MON_LAP), nf=0)
    o = Oracle(pb)
    xi = W.xi_nodes(pb)
    a, b = 0.3, 0.2
    rho = 1.0 + a * np.sin(2 * math.pi * xi[0]) + b * np.cos(2 * math.pi * xi[1])
    U = W.prim_to_cons(pb, [rho], [np.zeros_like(rho)] * 2, np.ones_like(rho))
    J = np.ones(pb.shape)
    h1, h2 = pb.dxi[0], pb.dxi[1]
    t1, t2 = 2 * math.pi * xi[0], 2 * math.pi * xi[1]
    g1 = a * np.cos(t1) * math.sin(2 * math.pi * h1) / h1
    g2 = -b * np.sin(t2) * math.sin(2 * math.pi * h2) / h2
    lap = -2 * a * np.sin(t1) * (1 - math.cos(2 * math.pi * h1)) / h1 ** 2 \
          - 2 * b * np.cos(t2) * (1 - math.cos(2 * math.pi * h2)) / h2 ** 2
    g = np.sqrt(g1 ** 2 + g2 ** 2)
    want = np.sqrt(1 + 20.0 * g / g.max() + 10.0 * np.abs(lap) / np.abs(lap).max())
    np.testing.assert_allclose(o.monitor(U, J), want, rtol=1e-12)


@pytest.mark.parametrize("N", [1, 2])
def test_schlieren_exact_on_a_linear_density(N):
    """Eq. (schlieren) on the identity mesh with rho = 1 + 0.5 xi_1 between reflecting walls:
    |grad rho| = 0.5 at interior nodes (central differences are exact) and 0.25 at the wall
    nodes (the mirrored ghost equals the node), so Phi = exp(-Psi) inside and exp(-Psi/2) on
    the walls; Psi = (30 rho_1 + 150 rho_2) / rho (constant here).  Uniform rho gives Phi = 1."""
    pb = W.random_problem(2, N, (12, 10), bc="reflect")
    o = Oracle(pb)
    xi = W.xi_nodes(pb)
    x = np.stack(xi)
    rho = 1.0 + 0.5 * xi[0]
    frac = [1.0] if N == 1 else [0.6, 0.4]
    U = W.prim_to_cons(pb, [f * rho for f in frac], [np.zeros_like(rho)] * 2, np.ones_like(rho))
    J = np.ones(pb.shape)
    psi = 30.0 if N == 1 else 30.0 * 0.6 + 150.0 * 0.4
    want = np.full(pb.shape, math.exp(-psi))
    want[..., 0] = want[..., -1] = math.exp(-psi / 2)
    np.testing.assert_allclose(o.schlieren(U, J, x), want, rtol=1e-12)
    U1 = W.prim_to_cons(pb, [f * np.ones_like(rho) for f in frac], [np.zeros_like(rho)] * 2, np.ones_like(rho))
    assert np.all(o.schlieren(U1, J, x) == 1.0)


def test_schlieren_gradient_converges_on_curvilinear_mesh():
    """The physical gradient (1/J) sum_k J xi_k/x (d rho/d xi_k) of the schlieren function
    converges at second order to the exact |grad_x rho| on a perturbed periodic mesh
    (a transposed metric contraction would leave an O(1) error)."""
    errs = []
    for n in (16, 32, 64):
        pb = W.random_problem(2, 1, (n, n))
        o = Oracle(pb)
        rng = np.random.default_rng(33)
        x = W.smooth_mesh(pb, rng, amp=0.05)
        J = o.init_J(x)
        k = 2 * math.pi
        rho = 1.0 + 0.2 * np.sin(k * x[0]) * np.cos(k * x[1])
        gx = 0.2 * k * np.cos(k * x[0]) * np.cos(k * x[1])
        gy = -0.2 * k * np.sin(k * x[0]) * np.sin(k * x[1])
        g = np.sqrt(gx ** 2 + gy ** 2)
        U = W.prim_to_cons(pb, [rho], [np.zeros_like(rho)] * 2, np.ones_like(rho))
        phi = o.schlieren(U * J, J, x)
        got = -np.log(phi) / 30.0          # |grad rho| / max |grad rho|
        errs.append(np.abs(got - g / g.max()).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.7, (errs, orders)


def test_limiter_keeps_node_order_and_mesh_velocity():
    """x^{n+1} = x^n + Delta_tau delta_tau x keeps every grid line monotone (the bounds of
    Sec. 4 allow at most half the neighbour spacing) and xdot = Delta_tau delta_tau x / Delta t."""
    pb, U, x = W.shock_bubble_2d(48, 24)
    o = Oracle(pb.with_(mu=10))
    J = o.init_J(x)
    JU = U * J
    xdot, dt, dtau = o.mesh_redistribute(JU, J, x)
    assert 0 < dtau <= 1 and dt > 0
    xn = x + dt * xdot
    assert np.all(np.diff(xn[0], axis=2) > 0)
    assert np.all(np.diff(xn[1], axis=1) > 0)
    th = o.monitor(JU, J)
    xmu = o.jacobi(x, th)
    np.testing.assert_allclose(xdot, dtau * (xmu - x) / dt, rtol=1e-13, atol=1e-15)
    assert abs(o.limiter(x, xmu) - dtau) == 0.0


# ---------------------------------------------------------------------------
# Jacobi sweeps: the converged discrete mesh equation with a varying monitor
# ---------------------------------------------------------------------------

def _jacobi_equilibrium(theta_line, a, b, periodic):
    """Node positions along one line at the fixed point of the discrete mesh equation of
    Sec. 4 when Theta varies along that line only: Theta_{i+1/2} (x_{i+1} - x_i) = C with
    Theta_{i+1/2} = (Theta_i + Theta_{i+1}) / 2.  Wall sides: the ghost node is the mirror
    image 2a - x_0 and carries Theta_0, so the half cell at the wall gives Theta_0 2 (x_0 - a)
    = C (likewise at b); the spacings fill [a, b].  Periodic sides: the line closes with
    x_n = x_0 + (b - a) and Theta_n = Theta_0; only the spacings are fixed."""
    th = np.asarray(theta_line, dtype=np.float64)
    n = th.size
    if periodic:
        half = 0.5 * (th + np.roll(th, -1))                 # Theta_{i+1/2}, i = 0..n-1
        C = (b - a) / np.sum(1.0 / half)
        return C / half                                     # the n spacings x_{i+1} - x_i
    half = 0.5 * (th[:-1] + th[1:])
    C = (b - a) / (1.0 / (2.0 * th[0]) + np.sum(1.0 / half) + 1.0 / (2.0 * th[-1]))
    x = np.empty(n)
    x[0] = a + C / (2.0 * th[0])
    x[1:] = x[0] + np.cumsum(C / half)
    return x


@pytest.mark.parametrize("bc", ["reflect", "periodic"])
@pytest.mark.parametrize("d", [2, 3])
def test_jacobi_converges_to_the_discrete_equilibrium(bc, d):
    """Theta varying along xi_1 only (by a factor of about 3): after enough Jacobi sweeps the
    x_1 positions on every xi_1 line reach the equilibrium of the discrete mesh equation
    with the half-sum weights (Theta_i + Theta_{i+1})/2, wall half cells included; the other
    coordinates stay uniform.  Weights Theta_i or Theta_{i+1} alone, swapped half weights, or
    a ghost Theta other than the boundary node's give a different equilibrium."""
    n = (13, 10, 10)[:d]
    pb = W.random_problem(d, 1, n, bc=bc).with_(mu=12000)
    o = Oracle(pb)
    xi = np.stack(W.xi_nodes(pb))
    rng = np.random.default_rng(5)
    th1 = 1.0 + 2.0 * rng.uniform(0.0, 1.0, size=n[0])
    theta = np.broadcast_to(th1.reshape((1,) * (3 - 1) + (n[0],)), pb.shape).copy()
    xmu = o.jacobi(xi, theta)
    a, b = pb.xi_lo[0], pb.xi_lo[0] + pb.length[0]
    want = _jacobi_equilibrium(th1, a, b, bc == "periodic")
    for line in xmu[0].reshape(-1, n[0]):
        if bc == "periodic":
            got = np.diff(np.concatenate([line, [line[0] + (b - a)]]))
            np.testing.assert_allclose(got, want, rtol=1e-12)
        else:
            np.testing.assert_allclose(line, want, rtol=0, atol=1e-12 * (b - a))
    for j in range(1, d):
        np.testing.assert_allclose(xmu[j], xi[j], rtol=0, atol=1e-13)
    # the equilibrium is not the uniform mesh: the monitor moves nodes by a sizable fraction
    assert np.abs(xmu[0] - xi[0]).max() > 0.05 * pb.dxi[0]


# ---------------------------------------------------------------------------
# the size of the ES dissipation at a small step
# ---------------------------------------------------------------------------

def _step_state(pb, rng, eps):
    """U_L and U_R = U_L + O(eps) (species densities, velocity and pressure moved along a
    random direction), so every characteristic field jumps."""
    rl = rng.uniform(0.5, 1.5, size=pb.N)
    v = rng.uniform(-0.6, 0.6, size=pb.d)
    p = rng.uniform(0.8, 1.5)
    dr, dv, dp = rng.uniform(0.5, 1.0, size=pb.N), rng.uniform(-1.0, 1.0, size=pb.d), rng.uniform(0.5, 1.0)
    UL = W.cons_state(pb, rl, v, p)[: pb.nc]
    UR = W.cons_state(pb, rl * (1.0 + eps * dr), v + eps * dv, p * (1.0 + eps * dp))[: pb.nc]
    return UL, UR


def _sound_speed(pb, U):
    """c^2 = Gamma_mix (p + p_inf) / rho of the stiffened mixture (Sec. 1)."""
    N, d = pb.N, pb.d
    rho = U[:N].sum()
    v2 = sum((U[N + m] / rho) ** 2 for m in range(d))
    cvr = sum(pb.cv[l] * U[l] for l in range(N))
    pinf = sum(pb.pinf[:N])
    T = (U[N + d] - 0.5 * rho * v2 - pinf) / cvr
    rr = sum(pb.R(l) * U[l] for l in range(N))
    gam = sum(pb.gamma[l] * pb.cv[l] * U[l] for l in range(N)) / cvr
    p = rr * T - pinf
    return math.sqrt(gam * (p + pinf) / rho)


@pytest.mark.parametrize("d,N,pinf", [(2, 1, 0.0), (2, 2, 1.5), (3, 1, 0.8), (3, 2, 1.5)])
def test_dissipation_magnitude_at_a_small_step(d, N, pinf):
    """Eq. (HOstable) between two constant states U_L, U_R = U_L + O(eps) on an affine,
    translating mesh whose xi_1 normal is rotated off the x axes: only the interface at the
    step has [[W]] != 0, there [[W]]^WENO = [[W]] up to the WENO epsilon, so Y = I and, by
    dU/dV = R R^T, the dissipation is D = -1/2 |Lambda| T^T R R^T T [[V]] = -1/2 |Lambda| [[U]]
    + O(eps^2), with |Lambda| = |J xi_t + L n.v| + L c (a scalar, Sec. 3.4).  (dJU_ES - dJU_EC)
    at the node left of the step is -D / dxi_1.  The test forms |Lambda| itself from the affine
    metrics, the mesh velocity and the arithmetic mean state, and checks the error against
    -1/2 |Lambda| [[U]] falls like eps^2.  A dropped 1/2, a dropped J xi_t, a mixed-up T / T^T
    or a wrong eigenvector scaling fail it."""
    n = (24, 14, 14)[:d]
    pb = W.random_problem(d, N, n, bc="reflect", pinf=pinf)
    if N == 2 and pinf:
        pb = pb.with_(pinf=(pinf, 0.5 * pinf))
    # the WENO epsilon is set far below jump^4 so that the WENO-MR weights pick the one-sided
    # constant candidate at the step exactly (with the paper's 1e-10 they would blend in the
    # higher-order candidates for jumps below about 1e-2)
    pb = pb.with_(bc=((W.OUTFLOW, W.OUTFLOW),) * 3, inflow=None, weno_eps=1e-40)
    A = np.eye(d) + np.array([[0.0, 0.35, -0.2], [-0.25, 0.1, 0.3], [0.15, -0.3, 0.05]])[:d, :d]
    Jdet = np.linalg.det(A)
    xi = np.stack(W.xi_nodes(pb))
    x = np.einsum("jk,k...->j...", A, xi)
    bvel = np.array([0.3, -0.2, 0.25])[:d]
    xdot = np.broadcast_to(bvel.reshape((d,) + (1,) * 3), (d,) + pb.shape).copy()
    # J xi_1 / x_j: the first row of the cofactor matrix of A (J = det A); J xi_1 / t
    Mx = np.linalg.inv(A)[0] * Jdet
    Mt = -float(bvel @ Mx)
    L = float(np.linalg.norm(Mx))
    nrm = Mx / L
    i_step = n[0] // 2
    mid = tuple(k // 2 for k in n[1:][::-1])          # a node far from the xi_2, xi_3 sides
    errs = []
    for eps in (0.04, 0.02, 0.01):
        rng = np.random.default_rng(100 + 10 * d + N)
        UL, UR = _step_state(pb, rng, eps)
        right = (np.arange(n[0]) >= i_step).reshape((1,) * 2 + (n[0],))
        U = np.where(right[None], UR.reshape(-1, 1, 1, 1), UL.reshape(-1, 1, 1, 1))
        J = np.full(pb.shape, Jdet)
        JU = U * J
        dES, _ = Oracle(pb).rhs(JU, J, x, xdot)
        dEC, _ = Oracle(pb.with_(es=False)).rhs(JU, J, x, xdot)
        idx = (slice(None),) + ((mid[0],) if d == 3 else (0,)) + (mid[-1], i_step - 1)
        D = -(dES - dEC)[idx] * pb.dxi[0]
        Ubar = 0.5 * (UL + UR)
        rho = Ubar[:N].sum()
        vbar = Ubar[N:N + d] / rho
        lam = abs(Mt + L * float(nrm @ vbar)) + L * _sound_speed(pb, Ubar)
        want = -0.5 * lam * (UR - UL)
        errs.append(np.abs(D - want).max() / np.abs(want).max())
        # the node right of the step sees the same flux with the other sign
        idx_r = idx[:-1] + (i_step,)
        np.testing.assert_allclose(-(dES - dEC)[idx_r] * pb.dxi[0], -D, rtol=1e-9, atol=1e-12 * np.abs(D).max())
    # relative error O(eps): halving eps halves it (absolute error O(eps^2))
    assert errs[-1] < 0.02, errs
    assert errs[1] / errs[2] > 1.6 and errs[0] / errs[1] > 1.6, errs


@pytest.mark.parametrize("d,N", CASES)
@pytest.mark.parametrize("band,below,above", [(1e-12, 4e-16, 1e-9), (3e-7, 2e-9, 1e-5)])
def test_y_band_separates_round_off_from_jumps(d, N, band, below, above):
    """The sign band of Y (Sec. 3.4; a jump [[W_m]] within band x ||r_m|| (||V_i|| + ||V_i+1||)
    counts as zero) sits between round-off and real jumps: for a step whose relative size is a
    few units of the arithmetic's last place (binary64 band 1e-12: 4e-16; binary32 band 3e-7:
    2e-9) every jump falls inside the band and the ES flux equals the EC flux exactly; for a
    step well above the band (1e-9, 1e-5) the dissipation acts at the step."""
    n = (16, 12, 12)[:d]
    pb = W.random_problem(d, N, n, bc="periodic")
    rng = np.random.default_rng(7 + d + N)
    UL = _random_state(pb, rng)
    x = np.stack(W.xi_nodes(pb))
    xdot = np.zeros_like(x)
    J = np.ones(pb.shape)
    right = (np.arange(n[0]) >= n[0] // 2).reshape((1,) * 2 + (n[0],))
    for size, zero in ((below, True), (above, False)):
        UR = UL * (1.0 + size * rng.uniform(0.5, 1.0, size=pb.nc))
        U = np.where(right[None], UR.reshape(-1, 1, 1, 1), UL.reshape(-1, 1, 1, 1))
        es_o = Oracle(pb)
        es_o.cfg.y_band = band
        ec_o = Oracle(pb.with_(es=False))
        dES, _ = es_o.rhs(U * J, J, x, xdot)
        dEC, _ = ec_o.rhs(U * J, J, x, xdot)
        diss = np.abs(dES - dEC).max()
        if zero:
            assert diss == 0.0, (size, diss)
        else:
            assert diss > 0.0, size


# ---------------------------------------------------------------------------
# metrics at ghost nodes: the symmetry of the boundary maps


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("bc", ["periodic", "mixed", "reflect"])
def test_metric_ghosts_follow_the_boundary_maps(d, bc):
    """The positions of a ghost node are those of the interior node it maps to, shifted by the
    box length (periodic side) or mirrored about the wall, x_d -> 2a - x_d, with xdot_d negated
    (every other side; the ghost of node i is node -1-i, a half-cell mirror).  The metrics of
    Eq. (SCLCoeff) and Eq. (VCLCoeff) evaluated there are then the mapped node's: unchanged
    across a periodic side; across a wall the reflections of xi_d and x_d flip the sign of
    J xi_k/x_j when exactly one of k, j is d, and of J xi_k/t when k is d, and flips compose at
    edges and corners.  A mirror about the wrong node or a dropped sign fails this."""
    n = (12, 11, 10)[:d]
    pb = W.random_problem(d, 1, n, bc=bc)
    rng = np.random.default_rng(7 + d)
    x = W.smooth_mesh(pb, rng, amp=0.05)
    xdot = 0.3 * (W.smooth_mesh(pb, rng, amp=0.05) - np.stack(W.xi_nodes(pb)))
    M = Oracle(pb).metrics(x, xdot)
    nf = d * (d + 1)
    P = M.shape[1:][::-1]                       # padded extents (P0, P1[, P2])
    scale = [np.abs(M[f]).max() for f in range(nf)]
    checked = 0
    worst = 0.0
    for idx in np.ndindex(*[P[k] for k in range(d)][::-1]):
        g = [idx[::-1][k] - 3 for k in range(d)]
        if all(0 <= g[k] < n[k] for k in range(d)):
            continue
        src, mir = list(g), [False] * d
        for k in range(d):
            if 0 <= g[k] < n[k]:
                continue
            side = 0 if g[k] < 0 else 1
            if pb.bc[k][side] == W.PERIODIC:
                src[k] = g[k] % n[k]
            else:
                src[k] = -1 - g[k] if side == 0 else 2 * n[k] - 1 - g[k]
                mir[k] = True
        gi = tuple(v + 3 for v in g[::-1])
        si = tuple(v + 3 for v in src[::-1])
        if d == 2:
            gi, si = (0,) + gi, (0,) + si
        for k in range(d):
            for c in range(d + 1):
                neg = False
                for m in range(d):
                    if mir[m] and ((k == m) != (c > 0 and c - 1 == m)):
                        neg = not neg
                f = k * (d + 1) + c
                want = -M[(f,) + si] if neg else M[(f,) + si]
                worst = max(worst, abs(M[(f,) + gi] - want) / scale[f])
        checked += 1
    assert checked > 0
    assert worst <= 1e-12, worst
