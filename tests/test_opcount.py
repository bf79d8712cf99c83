"""The operation-counting build of the oracle (CPU only): it computes the plain oracle's
results bit for bit, and the stored counts (tests/golden/op_counts.json, written by
python -m oracle.opcount) are what it counts now."""
import json

import numpy as np
import pytest

from oracle.oracle import Oracle
from oracle.opcount import GOLDEN, CountingOracle, count_case
from paper_2202_07989_gb300 import workloads as W

from .helpers import case


@pytest.mark.parametrize("d,N", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_counting_build_equals_plain_oracle(d, N):
    pb, JU, J, x, xdot = case(d, N, (12,) * d, "mixed", es=True, seed=3, pinf=0.5, jump=True)
    pb = pb.with_(mu=3, nf=2)
    a, b = Oracle(pb), CountingOracle(pb)
    for f in ("rhs", "metrics"):
        ra = getattr(a, f)(JU, J, x, xdot) if f == "rhs" else a.metrics(x, xdot)
        rb = getattr(b, f)(JU, J, x, xdot) if f == "rhs" else b.metrics(x, xdot)
        for u, v in zip(ra if isinstance(ra, tuple) else (ra,), rb if isinstance(rb, tuple) else (rb,)):
            assert np.array_equal(u, v)
    ma, mb = a.mesh_redistribute(JU, J, x), b.mesh_redistribute(JU, J, x)
    assert np.array_equal(ma[0], mb[0]) and ma[1:] == mb[1:]
    b.reset()
    b.rhs(JU, J, x, xdot)
    cnt = b.read()
    assert cnt["add"] > 0 and cnt["mul"] > 0 and cnt["div"] > 0 and cnt["log"] > 0 and cnt["sqrt"] > 0


def test_stored_counts_are_current():
    stored = json.load(open(GOLDEN))
    for key, v in stored["cases"].items():
        d, N = int(key[0]), int(key[2])
        fresh = count_case(d, N)
        for part in ("per_interface_flux", "per_padded_node_metrics", "per_cell_rk_step", "per_cell_mesh_redistribute"):
            assert fresh[part] == pytest.approx(v[part], rel=1e-12), (key, part)
