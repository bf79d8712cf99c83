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


def fieldwise(got, want, floor=0.0):
    return [rel_max_err(g, w, floor) for g, w in zip(got, want)]


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


def masked_fieldwise(got, want, margin, floor=0.0):
    """Relative max-norm error per field over the nodes whose Y decisions are robust, and the
    number of nodes left out."""
    keep = margin >= MARGIN_DECADES
    errs = []
    for g, w in zip(got, want):
        scale = max(np.abs(w).max(), floor)
        d = np.abs(np.asarray(g) - np.asarray(w))[keep]
        errs.append(d.max() / scale if d.size else 0.0)
    return errs, int((~keep).sum())
