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


def test_stiffened_3d_shock_bubble_fields():
    """Example 5.11's input: at Mach 10 the post-shock state of the stiffened gas (Gamma 3,
    p_inf 100) ahead of which rho = 1, p = 100 is the one the paper prints (1.980198,
    -121.2497, 29800); the bubble of ideal gas (rho_2 = 5 - eps) and the surroundings sit at
    p = 100; the inflow side carries the post-shock state.  The sharp form has the pure states
    on both sides of x_1 = 275; the default spreads the shock over about one cell, every node
    a state between the two (monotone in x_1), the bubble untouched."""
    pb, U, x = W.shock_bubble_3d_stiffened(8, shock_cells=0.0)
    assert pb.n == (40, 8, 8) and pb.N == 2 and pb.d == 3 and pb.pinf == (100.0, 0.0)
    rs, us, ps = W._post_shock(pb, 10.0, 1.0, 100.0)
    assert abs(rs - 1.980198) < 1e-6 and abs(us - 121.2497) < 1e-4 and abs(ps - 29800.0) < 1e-9
    o = Oracle(pb)

    def prims(U_):
        prim = [o.primitives(u) for u in U_.reshape(pb.nc, -1).T]
        shape = U_.shape[1:]
        rho_l = [np.array([q[0][l] for q in prim]).reshape(shape) for l in range(2)]
        v1 = np.array([q[1][0] for q in prim]).reshape(shape)
        p = np.array([q[3] for q in prim]).reshape(shape)
        return rho_l, v1, p

    rho_l, v1, p = prims(U)
    eps = 0.05
    behind = x[0] > 275.0
    bubble = (x[0] - 225.0) ** 2 + x[1] ** 2 + x[2] ** 2 < 25.0 ** 2
    assert bubble.any() and behind.any() and not (bubble & behind).any()
    np.testing.assert_allclose(p[~behind], 100.0, rtol=1e-12)
    np.testing.assert_allclose(rho_l[1][bubble], 5.0 - eps, rtol=1e-14)
    np.testing.assert_allclose(rho_l[0][~behind & ~bubble], 1.0 - eps, rtol=1e-14)
    np.testing.assert_allclose(p[behind], ps, rtol=1e-12)
    np.testing.assert_allclose(v1[behind], -us, rtol=1e-12)
    np.testing.assert_allclose(rho_l[0][behind], rs - eps, rtol=1e-14)
    infl = o.primitives(pb.inflow[0, 1][: pb.nc])
    assert abs(infl[3] - ps) <= 1e-9 * ps and abs(infl[1][0] + us) <= 1e-12 * us
    # the spread shock: pressure and velocity between the two states, monotone along x_1
    pb1, U1, x1 = W.shock_bubble_3d_stiffened(8)
    rho_l1, v11, p1 = prims(U1)
    assert (p1 >= 100.0 - 1e-9).all() and (p1 <= ps * (1 + 1e-12)).all()
    assert (np.diff(p1, axis=2) >= -1e-9).all() and (np.diff(v11, axis=2) <= 1e-12).all()
    np.testing.assert_allclose(rho_l1[1][bubble], 5.0 - eps, rtol=1e-14)
    mid = np.abs(x1[0] - 275.0) < 0.5 * pb1.dxi[0] + 1e-9
    assert mid.any() and (p1[mid] > 100.0 + 0.1 * (ps - 100.0)).all() and (p1[mid] < ps - 0.1 * (ps - 100.0)).all()


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batch_shard_partitions_the_instances(world):
    """The per-rank shares of the batched workload are disjoint, cover every instance, and no
    rank carries more than the mean share plus the largest instance (largest first to the
    least loaded rank)."""
    sizes = [p["n"] ** 2 for p in W.batched_params(64)]
    shares = [W.shard(sizes, world, r) for r in range(world)]
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(64))
    loads = [sum(sizes[i] for i in s) for s in shares]
    assert max(loads) <= sum(sizes) / world + max(sizes)
    assert W.shard(sizes, world, 0) == shares[0]          # deterministic
