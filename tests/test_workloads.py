"""The seeded workload generators against physics they must satisfy (CPU only): the post-shock
state of the shock-bubble inputs against the Rankine-Hugoniot jump conditions of the stiffened
gas (Sec. 1), and the generated shock-bubble fields against their stated primitives, read back
through the oracle's primitive-variable routine."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2202_07989_gb300 import workloads as W


@pytest.mark.parametrize("pinf", [0.0, 0.5, 3.0])
@pytest.mark.parametrize("Ms", [1.05, 1.22, 2.0, 3.5])
def test_post_shock_satisfies_jump_conditions(Ms, pinf):
    """Mass, momentum and energy fluxes through a shock of Mach Ms moving into gas at rest are
    continuous in the shock frame; the gas is a stiffened gas with rho e = (p + Gamma p_inf) /
    (Gamma - 1), so h = Gamma (p + p_inf) / ((Gamma - 1) rho)."""
    pb = W.random_problem(2, 1, (10, 10), pinf=pinf)
    g = pb.gamma[0]
    rho1, p1 = 1.0, 1.0
    rho2, u2, p2 = W._post_shock(pb, Ms, rho1, p1)
    s = Ms * math.sqrt(g * (p1 + pinf) / rho1)       # shock speed: Ms times the sound speed ahead
    w1, w2 = -s, u2 - s                               # velocities relative to the shock
    h = lambda rho, p: g * (p + pinf) / ((g - 1.0) * rho)
    mass = (rho1 * w1, rho2 * w2)
    mom = (rho1 * w1 * w1 + p1, rho2 * w2 * w2 + p2)
    ener = (rho1 * w1 * (h(rho1, p1) + 0.5 * w1 * w1), rho2 * w2 * (h(rho2, p2) + 0.5 * w2 * w2))
    for a, b in (mass, mom, ener):
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b)), (a, b)
    # a compressive shock: denser, higher pressure, gas set in motion along the shock's path
    assert rho2 > rho1 and p2 > p1 and 0.0 < u2 < s


def test_prim_to_cons_is_the_stiffened_gas_energy():
    """E = sum_l rho_l c_v,l T + |m|^2 / (2 rho) + p_inf with p = sum_l rho_l R_l T - p_inf, i.e.
    for one gas E = (p + Gamma p_inf) / (Gamma - 1) + rho |v|^2 / 2."""
    pb = W.random_problem(2, 1, (10, 10), pinf=0.7)
    g = pb.gamma[0]
    rho, v1, v2, p = np.array([1.3]), np.array([0.4]), np.array([-0.2]), np.array([2.1])
    U = W.prim_to_cons(pb, [rho], [v1, v2], p)
    E = (p + g * 0.7) / (g - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    np.testing.assert_allclose(U[-1], E, rtol=1e-14)
    np.testing.assert_allclose(U[1], rho * v1, rtol=1e-15)


def test_shock_bubble_fields():
    """The 2D shock-bubble input: gas at rest with rho = p = 1 ahead of the shock, the
    Rankine-Hugoniot state moving left behind it, and a bubble at the ambient pressure whose
    gas-2 density is rho_ratio times the ambient density (the pure gases' equal-p, equal-T
    ratio, R_2 = R_1 / rho_ratio); each region carries the trace eps of the absent species,
    which shifts the mixture temperatures (T = (p + p_inf) / sum_l rho_l R_l) apart."""
    Ms, ratio, eps = 1.22, 0.138, 0.03
    pb, U, x = W.shock_bubble_2d(80, 40, Ms=Ms, rho_ratio=ratio, eps=eps)
    o = Oracle(pb)
    pts = U.reshape(pb.nc, -1).T
    prim = [o.primitives(u) for u in pts]           # the oracle's point routine, node by node
    shape = U.shape[1:]
    rho_l = [np.array([q[0][l] for q in prim]).reshape(shape) for l in range(2)]
    v = [np.array([q[1][m] for q in prim]).reshape(shape) for m in range(2)]
    T = np.array([q[2] for q in prim]).reshape(shape)
    p = np.array([q[3] for q in prim]).reshape(shape)
    rho = rho_l[0] + rho_l[1]
    post = x[0] > 1.4
    bubble = ((x[0] - 1.0) ** 2 + (x[1] - 0.5) ** 2 < 0.04) & ~post
    ambient = ~post & ~bubble
    rs, us, ps = W._post_shock(pb, Ms, 1.0, 1.0)
    np.testing.assert_allclose(rho[ambient], 1.0, rtol=1e-14)
    np.testing.assert_allclose(p[ambient], 1.0, rtol=1e-13)
    np.testing.assert_allclose(v[0][ambient], 0.0, atol=0.0)
    np.testing.assert_allclose(rho[post], rs, rtol=1e-14)
    np.testing.assert_allclose(p[post], ps, rtol=1e-13)
    np.testing.assert_allclose(v[0][post], -us, rtol=1e-14)
    np.testing.assert_allclose(p[bubble], 1.0, rtol=1e-13)
    R = [pb.cv[l] * (pb.gamma[l] - 1.0) for l in range(2)]
    np.testing.assert_allclose(R[1], R[0] / ratio, rtol=1e-14)
    for region in (ambient, bubble, post):
        np.testing.assert_allclose(T[region], (p[region] + sum(pb.pinf)) / (rho_l[0][region] * R[0] + rho_l[1][region] * R[1]),
                                   rtol=1e-13)
    # the bubble's gas 2 density is rho_ratio times the ambient gas 1 density at equal p and T
    np.testing.assert_allclose(rho_l[1][bubble] + eps, ratio * (1.0 + 0.0), rtol=1e-12)
    np.testing.assert_allclose(rho_l[1][ambient], eps, rtol=1e-14)
    np.testing.assert_allclose(rho_l[0][bubble], eps, rtol=1e-14)
