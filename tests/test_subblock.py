"""CPU check of the block reduction the full-size GPU parity tests rely on: the oracle's residual
on a 13-node block around a node, sides that are not grid sides treated as outflow, equals the
oracle's residual of the whole grid at that node, bit for bit, at corners, edges, faces and inside,
on a moving curvilinear mesh with reflecting, inflow and outflow sides."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2202_07989_gb300 import workloads as W

from .helpers import case
from .test_gpu_fullsize import _oracle_at, _samples


@pytest.mark.parametrize("d,N", [(2, 2), (3, 1), (3, 2)])
def test_block_residual_equals_whole_grid_residual(d, N):
    n = (30, 26) if d == 2 else (20, 18, 16)
    pb, JU, J, x, xdot = case(d, N, n, "mixed", es=True, seed=90 + d + N, pinf=0.5, jump=True)
    if d == 2:
        pb = pb.with_(bc=((W.OUTFLOW, W.INFLOW), (W.REFLECT, W.REFLECT), (W.PERIODIC, W.PERIODIC)))
    dJU, dJ = Oracle(pb).rhs(JU, J, x, xdot)
    for c in _samples(pb, np.random.default_rng(3), 6):
        b_dJU, b_dJ, _ = _oracle_at(pb, JU, J, x, xdot, c, 1e-12)
        idx = tuple(c[k] if k < d else 0 for k in (2, 1, 0))
        assert np.array_equal(b_dJU, dJU[(slice(None),) + idx]) and b_dJ == dJ[idx], c
