"""EC flux orders 2w = 2 and 4 (es_config.w = 1, 2) on the GPU against the FP64 oracle: the
metric operator delta_k, the initial Jacobian, the residual and full steps take the weights
alpha(w) of Sec. 3.1; the dissipation keeps its fifth-order WENO reconstruction."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2202_07989_gb300 import workloads as W

from .helpers import TOL_FP64, case, fieldwise, masked_fieldwise, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

GRIDS = {2: (70, 37), 3: (22, 12, 11)}


def _ctx(pb, precision=0):
    from paper_2202_07989_gb300 import es
    return es.Context(pb, precision)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("w", [1, 2])
def test_metrics_and_init_J_order(d, w):
    torch = need_gpu()
    pb, JU, J, x, xdot = case(d, 1, GRIDS[d], "mixed")
    pb = pb.with_(w=w)
    o = Oracle(pb)
    ctx = _ctx(pb)
    Jg = ctx.es_init_mesh(to_dev(x, torch)).cpu().numpy()
    assert rel_max_err(Jg, o.init_J(x)) <= TOL_FP64
    Mg = ctx.es_metrics(to_dev(x, torch), to_dev(xdot, torch)).cpu().numpy()
    errs = fieldwise(Mg, o.metrics(x, xdot), floor=1e-3)
    assert max(errs) <= TOL_FP64, errs


@pytest.mark.parametrize("d,N", [(2, 1), (2, 2), (3, 1), (3, 2)])
@pytest.mark.parametrize("w", [1, 2])
def test_rhs_order_fp64(d, N, w):
    """FP64 residual (2D: the fused stage launch; 3D: per-direction launches) at 1e-12."""
    torch = need_gpu()
    pb, JU, J, x, xdot = case(d, N, GRIDS[d], "mixed", es=True, seed=60 + 10 * w + d + N, jump=True)
    pb = pb.with_(w=w)       # (JU, J) of the case are a valid state at any order
    dJU_o, dJ_o, mg = Oracle(pb).rhs_margins(JU, J, x, xdot)
    ctx = _ctx(pb)
    dJU, dJ = ctx.es_rhs(to_dev(JU, torch), to_dev(J, torch), to_dev(x, torch), to_dev(xdot, torch))
    e, skipped = masked_fieldwise(dJU.cpu().numpy(), dJU_o, mg, pb.N, pb.d)
    e.append(rel_max_err(dJ.cpu().numpy(), dJ_o))
    assert max(e) <= TOL_FP64, e
    assert skipped <= 0.01 * pb.ncell, skipped


@pytest.mark.parametrize("w", [1, 2])
def test_fused_split_bitwise_order(w):
    """At order 2w the fused 2D stage launch still equals the per-direction launches bit for bit."""
    torch = need_gpu()
    pb, JU, J, x, xdot = case(2, 2, (41, 29), "mixed", es=True, seed=70 + w, jump=True)
    pb = pb.with_(w=w)
    for form in (0, 1):
        ctx = _ctx(pb, form)
        G = [to_dev(t, torch) for t in (JU, J, x, xdot)]
        ctx.es_set_fusion(-1)
        ref = ctx.es_rhs(*G)
        ctx.es_set_fusion(0)
        got = ctx.es_rhs(*G)
        assert all(bool((a == b).all()) for a, b in zip(got, ref))


@pytest.mark.parametrize("d,N", [(2, 2), (3, 1)])
@pytest.mark.parametrize("form", [0, 1])
def test_full_step_order(d, N, form):
    """One full step (mesh redistribution + SSP-RK3) at order 4 (w = 2): FP64 at 1e-12 per
    field, mixed at FP32 level."""
    torch = need_gpu()
    pb, JU, J, x, xdot = case(d, N, GRIDS[d], "mixed", es=True, seed=80 + d)
    pb = pb.with_(w=2, mu=3, nf=2, sigma=(W.SIG_RHO, W.SIG_P), alpha=(50.0, 20.0))
    o = Oracle(pb)
    J = o.init_J(x)
    xd_o, dt_o, dtau_o = o.mesh_redistribute(JU, J, x)
    JUo, Jo, xo = o.rk_step(JU, J, x, xd_o, dt_o)
    ctx = _ctx(pb, form)
    JUg, Jg, xg = to_dev(JU, torch), to_dev(J, torch), to_dev(x, torch)
    xd, dd = ctx.es_step(JUg, Jg, xg)
    e = fieldwise(JUg.cpu().numpy(), JUo, N=pb.N, d=pb.d) + [rel_max_err(Jg.cpu().numpy(), Jo),
                                                             rel_max_err(xg.cpu().numpy(), xo)]
    print("order-4 full step", d, N, form, e)
    assert max(e) <= (TOL_FP64 if form == 0 else 2e-4), e
    assert ctx.es_poll_status() == 0
