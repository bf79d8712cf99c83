"""Floating-point operation counts of the FP64 oracle per interface, per node and per step.

TEST AND MEASUREMENT INFRASTRUCTURE.  The operation-counting build of the oracle
(opcount.cpp: es_oracle.c with a binary64 type that counts every operation) runs the
residual, the metrics, the SSP-RK3 step and the mesh redistribution once on a 16^d grid
(periodic, smooth random state on a perturbed moving mesh, seed 2202), and the counts are
divided by the interfaces or nodes processed.  They are the algorithmic work of the method
as the paper writes it: every pair of every interface formed from scratch (Eq. (ECfluxMM)
with the logarithmic means of Sec. 3.3), the GCL flux (Eq. (GCL_flux)), the dissipation of
Eq. (HOstable) with the eigenvector matrices of Sec. 3.4 written out and WENO-MR
(Appendix A), the metrics of Sec. 3.2, the SSP-RK3 update and the mesh step of Sec. 4.

    python -m oracle.opcount        # writes tests/golden/op_counts.json

Classes: add (and subtract), mul, div, sqrt, log, exp (and pow), cmp (comparisons and
absolute values, no arithmetic result).  flops = add + mul + div + sqrt + log + exp.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import sys

import numpy as np

from . import build as _build
from .oracle import Oracle, bind

CLASSES = ("add", "mul", "div", "sqrt", "log", "exp", "cmp")
FLOP_CLASSES = ("add", "mul", "div", "sqrt", "log", "exp")
GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                      "op_counts.json")

_clib = None


def counting_lib():
    global _clib
    if _clib is None:
        L = bind(C.CDLL(_build.build_opcount()))
        L.or_op_reset.restype = None
        L.or_op_reset.argtypes = []
        L.or_op_read.restype = None
        L.or_op_read.argtypes = [C.POINTER(C.c_longlong)]
        _clib = L
    return _clib


class CountingOracle(Oracle):
    """The oracle on the operation-counting build: the same results, bit for bit."""

    def __init__(self, pb):
        super().__init__(pb)
        self.L = counting_lib()

    def reset(self):
        self.L.or_op_reset()

    def read(self) -> dict:
        out = (C.c_longlong * 7)()
        self.L.or_op_read(out)
        d = {k: int(out[i]) for i, k in enumerate(CLASSES)}
        d["flops"] = sum(d[k] for k in FLOP_CLASSES)
        return d


def _per(counts: dict, units: float) -> dict:
    return {k: v / units for k, v in counts.items()}


def _minus(a: dict, b: dict) -> dict:
    return {k: a[k] - b[k] for k in a}


def count_case(d: int, N: int, n: int = 16, seed: int = 2202) -> dict:
    """Counts of one (d, N) case: the inputs are those of the parity tests' random smooth
    periodic case (workloads.random_problem / smooth_mesh / smooth_state)."""
    from paper_2202_07989_gb300 import workloads as W
    pb = W.random_problem(d, N, (n,) * d, bc="periodic", pinf=0.5)
    if N == 2:
        pb = pb.with_(pinf=(0.5, 0.25))
    rng = np.random.default_rng(seed)
    x = W.smooth_mesh(pb, rng, amp=0.05)
    xdot = 0.3 * (W.smooth_mesh(pb, rng, amp=0.05) - np.stack(W.xi_nodes(pb)))
    U = W.smooth_state(pb, x, rng, amp=0.25)
    o = CountingOracle(pb)
    J = o.init_J(x)
    JU = U * J
    ncell = pb.ncell
    ifaces = d * (n + 1) * n ** (d - 1)
    npad = (n + 6) ** d
    o.reset()
    o.metrics(x, xdot)
    met = o.read()
    o.reset()
    o.rhs(JU, J, x, xdot)
    rhs = o.read()
    flux = _minus(rhs, met)                  # the residual without its metrics pass
    o.reset()
    o.rk_step(JU, J, x, xdot, 1e-4)
    rk = o.read()
    o.reset()
    o.mesh_redistribute(JU, J, x)
    mesh = o.read()
    ec = CountingOracle(pb.with_(es=False))
    ec.reset()
    ec.rhs(JU, J, x, xdot)
    ec_only = _minus(ec.read(), met)
    return {
        "grid": [n] * d, "interfaces": ifaces, "nodes": ncell, "padded_nodes": npad,
        "per_interface_flux": _per(flux, ifaces),
        "per_interface_ec_gcl_only": _per(ec_only, ifaces),
        "per_padded_node_metrics": _per(met, npad),
        "per_cell_rk_step": _per(rk, ncell),
        "per_cell_mesh_redistribute": _per(mesh, ncell),
    }


def count_all() -> dict:
    out = {"what": "floating-point operations of the FP64 oracle (es_oracle.c) counted by its counting "
                   "build (opcount.cpp) on a 16^d periodic smooth random case, seed 2202; flops = add + mul "
                   "+ div + sqrt + log + exp",
           "classes": list(CLASSES), "cases": {}}
    for d, N in ((2, 1), (2, 2), (3, 1), (3, 2)):
        out["cases"]["%dd%d" % (d, N)] = count_case(d, N)
    return out


def main(argv=None):
    res = count_all()
    with open(GOLDEN, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")
    for k, v in res["cases"].items():
        print(k, "flux flops/interface %.1f" % v["per_interface_flux"]["flops"],
              "metrics flops/node %.1f" % v["per_padded_node_metrics"]["flops"])


if __name__ == "__main__":
    main(sys.argv[1:])
