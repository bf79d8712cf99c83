"""Shared helpers of the GPU parity tests: seeded inputs, oracle runs, comparisons."""
import numpy as np
import pytest

from paper_2202_07989_gb300 import workloads as W

# FP64 GPU path vs the FP64 oracle: relative max-norm per field (spec bound)
TOL_FP64 = 1e-12


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07989_gb300 import build as B
    B.build()
    return torch


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_max_err(got, want, floor=0.0):
    """max |got - want| / max |want| over the whole array (per-field callers slice)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(np.abs(want).max(), floor)
    if scale == 0.0:
        return np.abs(got).max()
    return np.abs(got - want).max() / scale


def field_scales(want, N=None, d=None, floor=0.0):
    """Per-field max-norm scales; with (N, d) given, the momentum components share the
    max-norm of the momentum vector."""
    sc = [max(np.abs(w).max(), floor) for w in want]
    if N is not None and d is not None:
        m = max(sc[N:N + d])
        for q in range(N, N + d):
            sc[q] = m
    return sc


def fieldwise(got, want, floor=0.0, N=None, d=None):
    sc = field_scales(want, N, d, floor)
    out = []
    for g, w, s in zip(got, want, sc):
        diff = np.abs(np.asarray(g) - np.asarray(w)).max()
        out.append(diff / s if s > 0 else diff)
    return out


def case(d, N, n, bc, es=True, seed=0, pinf=0.0, amp_mesh=0.05, jump=False):
    """(problem, JU, J, x, xdot) of a smooth random state on a perturbed moving mesh;
    J comes from the oracle's initial-Jacobian routine (any positive J is valid input)."""
    from oracle.oracle import Oracle
    pb = W.random_problem(d, N, n, bc=bc, es=es, pinf=pinf)
    if N == 2 and pinf:
        pb = pb.with_(pinf=(pinf, 0.5 * pinf))
    rng = np.random.default_rng(seed)
    x = W.smooth_mesh(pb, rng, amp=amp_mesh)
    xdot = 0.3 * (W.smooth_mesh(pb, rng, amp=amp_mesh) - np.stack(W.xi_nodes(pb)))
    U = W.smooth_state(pb, x, rng, amp=0.25)
    if jump:
        U = np.where((x[0] > 0.45)[None], U * np.array([2.0] * pb.N + [1.0] * pb.d + [2.5]).reshape(-1, 1, 1, 1), U)
    J = Oracle(pb).init_J(x)
    return pb, U * J, J, x, xdot


# Y decisions closer than this (in decades) to the round-off band may be decided by
# rounding differently on the two sides; such nodes are left out of element-wise parity
MARGIN_DECADES = 0.01


def masked_fieldwise(got, want, margin, N, d, floor=0.0):
    """Relative max-norm error per field (momentum components share one scale) over the
    nodes whose Y decisions are robust, and the number of nodes left out."""
    keep = margin >= MARGIN_DECADES
    errs = []
    for g, w, s in zip(got, want, field_scales(want, N, d, floor)):
        diff = np.abs(np.asarray(g) - np.asarray(w))[keep]
        errs.append((diff.max() / s if s > 0 else diff.max()) if diff.size else 0.0)
    return errs, int((~keep).sum())
