"""Seeded synthetic inputs shaped like the paper's test problems (arXiv 2202.07989, Sec. 5).

This module only *describes* problems and builds initial data: the grid, the
physical parameters, the boundary conditions, the initial mesh and the initial
point values of the conserved variables U.  It holds none of the numerical
scheme (no fluxes, metrics, WENO, time stepping or mesh equations), so both the
CUDA path and the CPU oracle can take their inputs from it.

Conserved variables follow Eq. (1.1): U = (rho_1..rho_N, rho v_1..rho v_d, E),
with the stiffened mixture EOS of Eq. (1.2):
    rho e = sum_l c_{v,l} rho_l T + sum_l p_{inf,l},  p = sum_l rho_l R_l T - sum_l p_{inf,l},
    R_l = c_{v,l} (Gamma_l - 1).
Arrays are field-major structure of arrays, shape (fields, n3, n2, n1) with n3 = 1 in 2D.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

PERIODIC, REFLECT, INFLOW, OUTFLOW = 0, 1, 2, 3
SIG_RHO, SIG_RHO1, SIG_RHO2, SIG_P, SIG_Y2, SIG_V1 = 0, 1, 2, 3, 4, 5
# monitor terms: alpha (|grad sigma|/max)^2 of Eq. (monitor); the linear gradient and Laplacian
# terms of Example 5.1's vortex monitor
MON_GRAD2, MON_GRAD, MON_LAP = 0, 1, 2

SEED = 2202


@dataclasses.dataclass
class Problem:
    """Grid, physics and scheme parameters of one instance."""

    d: int
    N: int
    n: Tuple[int, int, int]
    xi_lo: Tuple[float, float, float]
    length: Tuple[float, float, float]
    bc: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]]
    gamma: Tuple[float, float] = (1.4, 1.4)
    cv: Tuple[float, float] = (1.0, 1.0)
    pinf: Tuple[float, float] = (0.0, 0.0)
    inflow: Optional[np.ndarray] = None      # (3, 2, 8) conserved states on inflow sides
    w: int = 3                                # EC flux order 2w
    es: bool = True                           # add the WENO-MR dissipation
    chi: Tuple[float, float, float] = (1.0 / 111.0, 10.0 / 111.0, 100.0 / 111.0)
    weno_eps: float = 1.0e-10
    cfl: float = 0.4
    sigma: Tuple[int, ...] = (SIG_RHO,)
    alpha: Tuple[float, ...] = (100.0,)
    mu: int = 10
    nf: int = 3
    weno: int = 0                             # 0: WENO-MR (Appendix A), 1: WENO-JS
    sigma_op: Tuple[int, ...] = ()            # per monitor term: MON_GRAD2 (default), MON_GRAD, MON_LAP
    fixed_mesh: bool = False                  # the mesh never moves (uniform-mesh runs)

    @property
    def nc(self) -> int:
        return self.N + self.d + 1

    @property
    def dxi(self) -> Tuple[float, float, float]:
        return tuple(self.length[k] / self.n[k] if k < self.d else 1.0 for k in range(3))

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * (self.n[2] if self.d == 3 else 1)

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.n[2] if self.d == 3 else 1, self.n[1], self.n[0])

    def R(self, l: int) -> float:
        return self.cv[l] * (self.gamma[l] - 1.0)

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# grid helpers
# --------------------------------------------------------------------------

def xi_nodes(pb: Problem) -> List[np.ndarray]:
    """Cell-centred computational nodes xi_{k,i} = xi_lo + (i + 1/2) dxi, broadcast to (n3, n2, n1)."""
    out = []
    for k in range(pb.d):
        c = pb.xi_lo[k] + (np.arange(pb.n[k]) + 0.5) * pb.dxi[k]
        shp = [1, 1, 1]
        shp[2 - k] = pb.n[k]
        out.append(np.broadcast_to(c.reshape(shp), pb.shape).copy())
    return out


def prim_to_cons(pb: Problem, rho_l: Sequence[np.ndarray], v: Sequence[np.ndarray], p: np.ndarray) -> np.ndarray:
    """Point values of U from (rho_l, v, p) through the stiffened mixture EOS (Eq. (1.2))."""
    rho = sum(rho_l)
    rr = sum(r * pb.R(l) for l, r in enumerate(rho_l))
    cvr = sum(r * pb.cv[l] for l, r in enumerate(rho_l))
    pinf = sum(pb.pinf[: pb.N])
    T = (p + pinf) / rr
    v2 = sum(vm * vm for vm in v)
    E = cvr * T + pinf + 0.5 * rho * v2
    return np.stack(list(rho_l) + [rho * vm for vm in v] + [E]).astype(np.float64)


def cons_state(pb: Problem, rho_l, v, p) -> np.ndarray:
    """One conserved state vector (padded to 8 entries) from scalar primitives."""
    U = prim_to_cons(pb, [np.array(r, dtype=np.float64) for r in rho_l],
                     [np.array(x, dtype=np.float64) for x in v], np.array(p, dtype=np.float64))
    out = np.zeros(8)
    out[: pb.nc] = U.reshape(pb.nc)
    return out


def smooth_mesh(pb: Problem, rng: np.random.Generator, amp: float = 0.05) -> np.ndarray:
    """Randomly perturbed smooth mesh: x_k = xi_k + amp * dxi-scaled sum of sine modes.

    The modes are periodic over the box, so the perturbed mesh is compatible
    with periodic sides; they vanish at the walls of non-periodic sides."""
    xi = xi_nodes(pb)
    x = []
    for j in range(pb.d):
        pert = np.zeros(pb.shape)
        for _ in range(3):
            term = np.full(pb.shape, rng.uniform(-1, 1))
            for k in range(pb.d):
                kk = rng.integers(1, 3)
                s = (xi[k] - pb.xi_lo[k]) / pb.length[k]
                term = term * np.sin(2 * math.pi * kk * s + (0.0 if pb.bc[k][0] != PERIODIC else rng.uniform(0, 2 * math.pi)))
            pert += term
        x.append(xi[j] + amp * pb.length[j] / max(pb.n[: pb.d]) * 4.0 * pert)
    return np.stack(x)


def smooth_state(pb: Problem, x: np.ndarray, rng: np.random.Generator, amp: float = 0.2,
                 rho0: float = 1.0, p0: float = 1.0, vel: float = 0.5) -> np.ndarray:
    """Smooth random point values of U on the physical nodes x (periodic in the box)."""
    def field(base, a):
        f = np.full(pb.shape, base, dtype=np.float64)
        for _ in range(3):
            term = np.full(pb.shape, a * rng.uniform(-1, 1))
            for k in range(pb.d):
                kk = rng.integers(1, 3)
                term = term * np.cos(2 * math.pi * kk * (x[k] - pb.xi_lo[k]) / pb.length[k] + rng.uniform(0, 2 * math.pi))
            f += term
        return f
    if pb.N == 1:
        rho_l = [field(rho0, amp * rho0)]
    else:
        r1 = field(0.6 * rho0, 0.3 * amp * rho0)
        r2 = field(0.4 * rho0, 0.3 * amp * rho0)
        rho_l = [r1, r2]
    v = [field(0.0, vel) for _ in range(pb.d)]
    p = field(p0, amp * p0)
    return prim_to_cons(pb, rho_l, v, p)


def random_problem(d: int, N: int, n: Sequence[int], bc: str = "periodic", pinf: float = 0.0,
                   es: bool = True, **kw) -> Problem:
    """A test instance on the unit box with the given sides."""
    n3 = tuple(list(n) + [1] * (3 - len(n)))
    if bc == "periodic":
        sides = ((PERIODIC, PERIODIC),) * 3
    elif bc == "mixed":
        sides = ((OUTFLOW, INFLOW), (REFLECT, REFLECT), (PERIODIC, PERIODIC) if d == 2 else (REFLECT, REFLECT))
    elif bc == "reflect":
        sides = ((REFLECT, REFLECT),) * 3
    else:
        raise ValueError(bc)
    gam = (1.4, 1.648) if N == 2 else (1.4, 1.4)
    cv = (1.0, 2.5) if N == 2 else (1.0, 1.0)
    pb = Problem(d=d, N=N, n=n3, xi_lo=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0), bc=sides,
                 gamma=gam, cv=cv, pinf=(pinf, 0.0 if N == 2 else 0.0), es=es, **kw)
    if bc == "mixed":
        inflow = np.zeros((3, 2, 8))
        rl = [1.2] if N == 1 else [0.7, 0.5]
        inflow[0, 1] = cons_state(pb, rl, [-0.3] + [0.0] * (d - 1), 1.3)
        pb = pb.with_(inflow=inflow)
    return pb


# --------------------------------------------------------------------------
# the paper-shaped workloads
# --------------------------------------------------------------------------

def vortex_2d(n: int = 64, t: float = 0.0, es: bool = True) -> Tuple[Problem, np.ndarray, np.ndarray, np.ndarray]:
    """Isentropic vortex of Example 5.1 re-centred at (5, 5) in the periodic box [0, 10]^2.

    Mesh x = xi + 0.1 sin(pi xi_1/5) sin(pi xi_2/5) (1 + sin t) in both
    components, moving with xdot = 0.1 sin(pi xi_1/5) sin(pi xi_2/5) cos t.
    Returns (problem, U point values, x, xdot)."""
    pb = Problem(d=2, N=1, n=(n, n, 1), xi_lo=(0.0, 0.0, 0.0), length=(10.0, 10.0, 1.0),
                 bc=((PERIODIC, PERIODIC),) * 3, gamma=(1.4, 1.4), cv=(1.0, 1.0), es=es, cfl=0.4,
                 sigma=(SIG_RHO,), alpha=(100.0,), mu=10, nf=3)
    xi = xi_nodes(pb)
    bump = 0.1 * np.sin(math.pi * xi[0] / 5.0) * np.sin(math.pi * xi[1] / 5.0)
    x = np.stack([xi[0] + bump * (1 + math.sin(t)), xi[1] + bump * (1 + math.sin(t))])
    xdot = np.stack([bump * math.cos(t), bump * math.cos(t)])
    U = vortex_state(pb, x, t)
    return pb, U, x, xdot


def vortex_state(pb: Problem, x: np.ndarray, t: float, eps: float = 5.0) -> np.ndarray:
    """Exact vortex solution at time t (translation with the mean velocity (1, 1), periodic)."""
    G = pb.gamma[0]
    L = pb.length[0]
    dx = np.mod(x[0] - t - 5.0 + L / 2, L) - L / 2
    dy = np.mod(x[1] - t - 5.0 + L / 2, L) - L / 2
    r2 = dx * dx + dy * dy
    dv = eps / (2 * math.pi) * np.exp(0.5 * (1 - r2))
    v1 = 1.0 + dv * dy
    v2 = 1.0 - dv * dx
    T = 1.0 - eps * eps / (8 * G * math.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1.0 / (G - 1.0))
    p = rho * pb.R(0) * T
    return prim_to_cons(pb, [rho], [v1, v2], p)


def _post_shock(pb: Problem, Ms: float, rho1: float, p1: float, l: int = 0) -> Tuple[float, float, float]:
    """Rankine-Hugoniot state behind a shock of Mach Ms moving into gas l at rest (ideal part of gas l)."""
    g = pb.gamma[l]
    pi_ = sum(pb.pinf[: pb.N])   # the mixture's p_inf is the sum over species (Sec. 1)
    c1 = math.sqrt(g * (p1 + pi_) / rho1)
    rho2 = rho1 * (g + 1) * Ms * Ms / ((g - 1) * Ms * Ms + 2)
    p2 = p1 + (p1 + pi_) * 2 * g / (g + 1) * (Ms * Ms - 1)
    u2 = Ms * c1 * (1 - rho1 / rho2)
    return rho2, u2, p2


def shock_bubble_2d(nx: int = 400, ny: int = 200, Ms: float = 1.22, radius: float = 0.2,
                    gamma2: float = 1.648, pinf2: float = 0.0, rho_ratio: float = 0.138,
                    length=(2.0, 1.0), shock_x: float = 1.4, centre=(1.0, 0.5), eps: float = 0.03,
                    mu: int = 5) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """Two-component shock-bubble interaction shaped like Example 5.8.

    Gas 1 (Gamma 1.4, p_inf 0, c_v 1) at rest with rho = p = 1; a Mach Ms shock at
    x_1 = shock_x moves left into it; a circular bubble of gas 2 at the same pressure, with
    R_2 = R_1 / rho_ratio and density rho_ratio (the pure gases are then at equal p and T).
    Pure regions carry a trace eps = 0.03 of the other species, the value of Example 5.8
    (the scheme is not positivity preserving, and a trace of 1e-5 goes negative at the
    material interface in the first stage); the traces shift the mixture temperatures of
    the bubble and its surroundings apart.  Reflecting top and bottom, inflow on the right,
    outflow on the left.  Returns (problem, U point values, x)."""
    cv1 = 1.0
    R1 = cv1 * 0.4
    R2 = R1 / rho_ratio
    cv2 = R2 / (gamma2 - 1.0)
    pb = Problem(d=2, N=2, n=(nx, ny, 1), xi_lo=(0.0, 0.0, 0.0), length=(length[0], length[1], 1.0),
                 bc=((OUTFLOW, INFLOW), (REFLECT, REFLECT), (PERIODIC, PERIODIC)),
                 gamma=(1.4, gamma2), cv=(cv1, cv2), pinf=(0.0, pinf2), es=True, cfl=0.4,
                 sigma=(SIG_RHO,), alpha=(100.0,), mu=mu, nf=3)
    rho_s, u_s, p_s = _post_shock(pb, Ms, 1.0, 1.0)
    xi = xi_nodes(pb)
    x = np.stack(xi)
    r2 = (x[0] - centre[0]) ** 2 + (x[1] - centre[1]) ** 2
    inside = r2 < radius * radius
    post = x[0] > shock_x
    # bubble at the same p, T as the ambient gas: rho_2 = rho_1 R_1 / R_2 (pinf2 folded into p)
    T_amb = (1.0 + sum(pb.pinf)) / (1.0 * R1)
    rb = (1.0 + sum(pb.pinf)) / (R2 * T_amb)
    r1 = np.where(post, rho_s - eps, np.where(inside, eps, 1.0 - eps))
    r2_ = np.where(post, eps, np.where(inside, rb - eps, eps))
    v1 = np.where(post, -u_s, 0.0)
    v2 = np.zeros_like(v1)
    p = np.where(post, p_s, 1.0)
    U = prim_to_cons(pb, [r1, r2_], [v1, v2], p)
    inflow = np.zeros((3, 2, 8))
    inflow[0, 1] = cons_state(pb, [rho_s - eps, eps], [-u_s, 0.0], p_s)
    pb = pb.with_(inflow=inflow)
    return pb, U, x


def riemann_3d(n: int = 128, seed: int = SEED, mu: int = 10) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """3D single-component octant Riemann problem on [0, 1]^3: 8 octant states with
    rho ~ U(0.1, 2), p ~ U(0.1, 1.5), v = 0, Gamma 1.4, outflow sides, CFL 0.3,
    monitor on rho with alpha 500 (shaped like Example 5.6)."""
    rng = np.random.default_rng(seed)
    pb = Problem(d=3, N=1, n=(n, n, n), xi_lo=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0),
                 bc=((OUTFLOW, OUTFLOW),) * 3, gamma=(1.4, 1.4), cv=(1.0, 1.0), es=True, cfl=0.3,
                 sigma=(SIG_RHO,), alpha=(500.0,), mu=mu, nf=3)
    rho_o = rng.uniform(0.1, 2.0, size=8)
    p_o = rng.uniform(0.1, 1.5, size=8)
    x = np.stack(xi_nodes(pb))
    octant = (x[0] > 0.5).astype(int) + 2 * (x[1] > 0.5).astype(int) + 4 * (x[2] > 0.5).astype(int)
    rho = rho_o[octant]
    p = p_o[octant]
    z = np.zeros_like(rho)
    U = prim_to_cons(pb, [rho], [z, z, z], p)
    return pb, U, x


def shock_bubble_3d(n: int = 128, Ms: float = 1.22, radius: float = 0.2, gamma2: float = 1.648,
                    rho_ratio: float = 0.138, eps: float = 0.03, mu: int = 10) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """3D two-component shock-bubble shaped like Example 5.10: (2n, n, n) cells on [0, 2] x [0, 1]^2,
    gas 1 (Gamma 1.4) at rest with rho = p = 1, a Mach Ms shock at x_1 = 1.4 moving left, a
    spherical bubble of radius 0.2 at (1, 0.5, 0.5) of gas 2 (density ratio rho_ratio, the pure
    gases' ratio at equal p and T), trace eps of the absent species (which shifts the mixture
    temperatures apart at equal pressure); reflecting side walls, inflow right, outflow left."""
    cv1 = 1.0
    R1 = cv1 * 0.4
    R2 = R1 / rho_ratio
    cv2 = R2 / (gamma2 - 1.0)
    pb = Problem(d=3, N=2, n=(2 * n, n, n), xi_lo=(0.0, 0.0, 0.0), length=(2.0, 1.0, 1.0),
                 bc=((OUTFLOW, INFLOW), (REFLECT, REFLECT), (REFLECT, REFLECT)),
                 gamma=(1.4, gamma2), cv=(cv1, cv2), pinf=(0.0, 0.0), es=True, cfl=0.3,
                 sigma=(SIG_RHO,), alpha=(100.0,), mu=mu, nf=3)
    rho_s, u_s, p_s = _post_shock(pb, Ms, 1.0, 1.0)
    x = np.stack(xi_nodes(pb))
    r2 = (x[0] - 1.0) ** 2 + (x[1] - 0.5) ** 2 + (x[2] - 0.5) ** 2
    inside = r2 < radius * radius
    post = x[0] > 1.4
    rb = rho_ratio
    r1 = np.where(post, rho_s - eps, np.where(inside, eps, 1.0 - eps))
    r2_ = np.where(post, eps, np.where(inside, rb - eps, eps))
    v1 = np.where(post, -u_s, 0.0)
    z = np.zeros_like(v1)
    p = np.where(post, p_s, 1.0)
    U = prim_to_cons(pb, [r1, r2_], [v1, z, z], p)
    inflow = np.zeros((3, 2, 8))
    inflow[0, 1] = cons_state(pb, [rho_s - eps, eps], [-u_s, 0.0, 0.0], p_s)
    return pb.with_(inflow=inflow), U, x


def water_air_3d(n: int = 256, mu: int = 10, eps: float = 1e-5) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """3D water/air shock-bubble shaped like Example 5.11: water (Gamma 4.4, p_inf 6000,
    rho 1) with an air bubble of radius 0.25 at the centre (Gamma 1.4, p_inf 0,
    rho 0.001); planar pressure jump at x_1 = 0.2 (p = 1e4 left, 1 right); outflow
    sides; monitor on (rho, Y_2) with alpha (500, 500)."""
    pb = Problem(d=3, N=2, n=(n, n, n), xi_lo=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0),
                 bc=((OUTFLOW, OUTFLOW),) * 3, gamma=(4.4, 1.4), cv=(1.0, 1.0), pinf=(6000.0, 0.0),
                 es=True, cfl=0.3, sigma=(SIG_RHO, SIG_Y2), alpha=(500.0, 500.0), mu=mu, nf=3)
    x = np.stack(xi_nodes(pb))
    r2 = (x[0] - 0.5) ** 2 + (x[1] - 0.5) ** 2 + (x[2] - 0.5) ** 2
    inside = r2 < 0.25 ** 2
    r1 = np.where(inside, eps, 1.0 - eps)
    r2_ = np.where(inside, 0.001 - eps * 1e-3, eps * 1e-3)
    p = np.where(x[0] < 0.2, 1.0e4, 1.0)
    z = np.zeros_like(p)
    U = prim_to_cons(pb, [r1, r2_], [z, z, z], p)
    return pb, U, x


def batched_params(count: int = 64, nmin: int = 96, nmax: int = 512, seed: int = SEED) -> List[dict]:
    """The seeded draws of the batched workload, one dict per instance: grid n ~ U{nmin..nmax}
    (square), shock Mach Ms ~ U(1.1, 3), bubble radius r ~ U(0.1, 0.3), gas-2 Gamma g2 ~
    U(1.1, 4.4) and p_inf,2 pi2 ~ U(0, 10)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        Ms = float(rng.uniform(1.1, 3.0))
        r = float(rng.uniform(0.1, 0.3))
        g2 = float(rng.uniform(1.1, 4.4))
        pi2 = float(rng.uniform(0.0, 10.0))
        out.append(dict(n=n, Ms=Ms, r=r, g2=g2, pi2=pi2))
    return out


def batched_instance(prm: dict, n: Optional[int] = None, mu: int = 5) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """One instance of the batched workload from its draws (batched_params), on its own grid or
    on an n x n grid: a two-component stiffened-gas shock-bubble on [0, 1]^2, shock at x_1 = 0.8
    moving left, bubble at the centre."""
    n = prm["n"] if n is None else n
    return shock_bubble_2d(n, n, Ms=prm["Ms"], radius=prm["r"], gamma2=prm["g2"], pinf2=prm["pi2"],
                           length=(1.0, 1.0), shock_x=0.8, centre=(0.5, 0.5), mu=mu)


def batched_2d(count: int = 64, nmin: int = 96, nmax: int = 512, seed: int = SEED,
               mu: int = 5) -> List[Tuple[Problem, np.ndarray, np.ndarray]]:
    """Independent two-component stiffened-gas shock-bubble instances on [0, 1]^2 with
    n ~ U{nmin..nmax} (square grids), shock Mach ~ U(1.1, 3), bubble radius ~ U(0.1, 0.3),
    gas-2 Gamma ~ U(1.1, 4.4) and p_inf,2 ~ U(0, 10); shock at x_1 = 0.8 moving left."""
    return [batched_instance(prm, mu=mu) for prm in batched_params(count, nmin, nmax, seed)]


def shard(sizes: Sequence[int], world: int, rank: int) -> List[int]:
    """The instances rank `rank` of `world` advances when independent instances of the given
    sizes (cells) are split across ranks: largest first, each to the rank with the fewest
    cells so far (ties to the lower rank).  Every instance goes to exactly one rank."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def shock_bubble_3d_stiffened(n: int = 80, eps: float = 0.05, Ms: float = 10.0, mu: int = 10, nf: int = 3,
                              shock_cells: float = 1.0,
                              fixed_mesh: bool = True) -> Tuple[Problem, np.ndarray, np.ndarray]:
    """3D shock-bubble interaction II of Example 5.11: on [0, 445] x [-44.5, 44.5]^2 with
    (5n, n, n) cells, a bubble of ideal gas (species 2: Gamma 1.4, p_inf 0) of radius 25 at
    (225, 0, 0) in a stiffened gas (species 1: Gamma 3, p_inf 100), c_v = 1 for both; a Mach Ms
    shock at x_1 = 275 moving left.  States (rho_1, rho_2, v, p): surroundings ahead of the
    shock (1 - eps, eps, 0, 100), behind it the Rankine-Hugoniot state of the stiffened gas
    (at Mach 10: 1.980198 - eps, eps, (-121.2497, 0, 0), 29800), bubble (eps, 5 - eps, 0, 100),
    eps = 0.05.  Monitor on (rho_1, p) with alpha (500, 500), WENO-MR linear weights
    (0.95, 0.045, 0.005) as in Example 5.10, CFL 0.3.  Sides as in the 2D shock-bubble
    (Example 5.8) extended to 3D: reflecting walls in x_2 and x_3, outflow on the left, inflow
    of the post-shock state on the right.

    The shock is spread over about `shock_cells` cells (a tanh profile in x_1 between the two
    states; 0 = the sharp step): a sharp Mach 10 step drives the trace rho_2 negative behind it
    in the first stage.  fixed_mesh = True is the paper's uniform-mesh form of the example
    (UM-WENOMR); from a uniform start mesh the moving-mesh form's first mesh step moves the
    nodes at the bubble half a cell per step and drives the traces negative there."""
    pb = Problem(d=3, N=2, n=(5 * n, n, n), xi_lo=(0.0, -44.5, -44.5), length=(445.0, 89.0, 89.0),
                 bc=((OUTFLOW, INFLOW), (REFLECT, REFLECT), (REFLECT, REFLECT)),
                 gamma=(3.0, 1.4), cv=(1.0, 1.0), pinf=(100.0, 0.0), es=True, cfl=0.3,
                 chi=(0.95, 0.045, 0.005), sigma=(SIG_RHO1, SIG_P), alpha=(500.0, 500.0), mu=mu, nf=nf,
                 fixed_mesh=fixed_mesh)
    x = np.stack(xi_nodes(pb))
    inside = (x[0] - 225.0) ** 2 + x[1] ** 2 + x[2] ** 2 < 25.0 ** 2
    rho_s, u_s, p_s = _post_shock(pb, Ms, 1.0, 100.0)     # (1.980198, 121.2497, 29800) at Mach 10
    if shock_cells > 0:
        s = 0.5 * (1.0 + np.tanh((x[0] - 275.0) / (shock_cells * pb.dxi[0])))
    else:
        s = (x[0] > 275.0).astype(np.float64)
    r1 = np.where(inside, eps, (1.0 - eps) * (1.0 - s) + (rho_s - eps) * s)
    r2 = np.where(inside, 5.0 - eps, eps)
    v1 = -u_s * s
    z = np.zeros_like(v1)
    p = 100.0 * (1.0 - s) + p_s * s
    U = prim_to_cons(pb, [r1, r2], [v1, z, z], p)
    inflow = np.zeros((3, 2, 8))
    inflow[0, 1] = cons_state(pb, [rho_s - eps, eps], [-u_s, 0.0, 0.0], p_s)
    return pb.with_(inflow=inflow), U, x
