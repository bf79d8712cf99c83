"""The fused 2D stage launch (both directions of a stage's residual and the stage update in
one launch over TX x TY node tiles) against the per-direction launches, bit for bit, and
against the FP64 oracle.

Grids: 70 x 37 leaves ragged tiles in both directions for every fused shape (16x12, 12x16,
14x14, 24x8, 20x10); 10 x 11 is smaller than one tile in both directions.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2202_07989_gb300 import workloads as W

from .helpers import TOL_FP64, case, fieldwise, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

NFSHAPE = 5
NJF_SHAPE = 4


def _ctx(pb, precision=0):
    from paper_2202_07989_gb300 import es
    return es.Context(pb, precision)


def _same(a, b):
    return all(bool((u == v).all()) for u, v in zip(a, b))


@pytest.mark.parametrize("N", [1, 2])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("bc", ["periodic", "mixed", "reflect"])
def test_fused_stage_bitwise(N, form, bc):
    """Every fused shape, at one CTA per SM and at full occupancy, gives the residual and the
    RK step (stage metrics M + s dt Md) of the per-direction launches bit for bit: with and
    without the dissipation, WENO-MR and WENO-JS, ragged and sub-tile grids."""
    torch = need_gpu()
    variants = (((70, 37), True, 0, 11), ((10, 11), True, 0, 12), ((70, 37), False, 0, 13), ((41, 29), True, 1, 14))
    for n, es_, weno, seed in variants:
        pb, JU, J, x, xdot = case(2, N, n, bc, es=es_, seed=seed + N, jump=True, pinf=0.6 if N == 1 else 0.0)
        pb = pb.with_(weno=weno)
        ctx = _ctx(pb, form)
        G = [to_dev(t, torch) for t in (JU, J, x, xdot)]
        dt = torch.tensor([0.3 * Oracle(pb).cfl_dt(JU, J, x)], dtype=torch.float64, device="cuda")
        assert ctx.es_get_fusion()[:3] == (0, 16, 12)
        ctx.es_set_fusion(-1)
        ref = ctx.es_rhs(*G)
        A = [t.clone() for t in G[:3]]
        ctx.es_rk_step(*A, G[3], dt)
        for shape in range(NFSHAPE):
            for grid in (0, 152):
                ctx.es_set_fusion(shape, grid)
                got = ctx.es_rhs(*G)
                assert _same(got, ref), (n, es_, weno, shape, grid)
                B = [t.clone() for t in G[:3]]
                ctx.es_rk_step(*B, G[3], dt)
                assert _same(A, B), (n, es_, weno, shape, grid)
        ctx.es_set_fusion(-1)
        assert ctx.es_poll_status() == 0


@pytest.mark.parametrize("form", [0, 1])
def test_fused_step_and_batch_bitwise(form):
    """Full steps (mesh redistribution + SSP-RK3) with the fused stage launch equal those with
    the per-direction launches bit for bit, for a single shock-bubble instance and for a
    batch of uneven instances."""
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, U, x = W.shock_bubble_2d(96, 64)
    J = Oracle(pb).init_J(x)
    st0 = [to_dev(t, torch) for t in (U * J, J, x)]
    runs = []
    for shape in (-1, 0, 3):
        ctx = _ctx(pb, form)
        ctx.es_set_fusion(shape)
        S = [t.clone() for t in st0]
        for _ in range(2):
            xd, dd = ctx.es_step(*S)
        runs.append(S + [xd, dd])
    assert _same(runs[0], runs[1]) and _same(runs[0], runs[2])

    insts = W.batched_2d(count=3, nmin=40, nmax=90, mu=3)
    probs = [p for p, _, _ in insts]
    st = []
    for p, U, x in insts:
        J = Oracle(p).init_J(x)
        st.append((U * J, J, x))
    outs = []
    for shape in (-1, 1, 4):
        b = es.Context(probs, form)
        b.es_set_fusion(shape)
        JU = [to_dev(s[0], torch) for s in st]
        Jd = [to_dev(s[1], torch) for s in st]
        X = [to_dev(s[2], torch) for s in st]
        XD = [torch.zeros_like(t) for t in X]
        DD = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in st]
        b.es_bind_batch(JU, Jd, X, XD, DD)
        for _ in range(2):
            b.es_step_batch()
        outs.append(JU + Jd + X)
    assert _same(outs[0], outs[1]) and _same(outs[0], outs[2])


@pytest.mark.parametrize("N", [1, 2])
def test_fused_rk_step_vs_oracle(N):
    """With the fused stage launch, one FP64 RK step from the oracle's state matches the
    oracle's step to 1e-12 per field (ragged tiles, outflow/inflow and reflecting sides)."""
    torch = need_gpu()
    pb, JU, J, x, xdot = case(2, N, (70, 37), "mixed", es=True, seed=5 + N)
    o = Oracle(pb)
    dt = 0.3 * o.cfl_dt(JU, J, x)
    ctx = _ctx(pb)
    ctx.es_set_fusion(0)
    JUg, Jg, xg = to_dev(JU, torch), to_dev(J, torch), to_dev(x, torch)
    ctx.es_rk_step(JUg, Jg, xg, to_dev(xdot, torch), torch.tensor([dt], dtype=torch.float64, device="cuda"))
    JUo, Jo, xo = o.rk_step(JU, J, x, xdot, dt)
    e = fieldwise(JUg.cpu().numpy(), JUo, N=N, d=2) + [rel_max_err(Jg.cpu().numpy(), Jo), rel_max_err(xg.cpu().numpy(), xo)]
    assert max(e) <= TOL_FP64, e


def test_fused_autotune_and_errors():
    """es_autotune on a 2D context also times the fused launch and reports a valid choice;
    results after tuning are unchanged; a fused shape on a 3D context or out of range is
    refused with ES_ERR_ARG."""
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, JU, J, x, xdot = case(2, 2, (70, 37), "mixed", es=True, seed=41, jump=True)
    ctx = _ctx(pb, 1)
    G = [to_dev(t, torch) for t in (JU, J, x, xdot)]
    ref = ctx.es_rhs(*G)
    ctx.es_autotune(*G, reps=2)
    sh, TX, TY, grid, ms = ctx.es_get_fusion()
    assert -1 <= sh < NFSHAPE and ms > 0
    if sh >= 0:
        assert (TX + 1) * TY <= 256 and (TY + 1) * TX <= 256 and grid > 0
    assert _same(ctx.es_rhs(*G), ref)
    for bad in (-2, NFSHAPE):
        with pytest.raises(es.EsError):
            ctx.es_set_fusion(bad)
    pb3, *_ = case(3, 1, (12, 11, 10), "periodic", seed=1)
    c3 = _ctx(pb3, 1)
    with pytest.raises(es.EsError):
        c3.es_set_fusion(0)
    c3.es_set_fusion(-1)
    assert c3.es_get_fusion()[0] == -1
    assert np.isfinite(ref[0].cpu().numpy()).all()


@pytest.mark.parametrize("form", [0, 1])
def test_run_host_equals_device_steps(form):
    """es_run_host (host buffers; one captured CUDA graph of a step replayed per step) leaves
    the same state, bit for bit, as es_step on device buffers and reports the summed Delta t:
    with the default launch configuration, with the state in one host block (one transfer each
    way), after a tuning change (the graph is rebuilt), with a fixed Delta t, and with
    es_profile on (launches one at a time, each timed)."""
    torch = need_gpu()
    pb, U, x = W.shock_bubble_2d(96, 64)
    J = Oracle(pb).init_J(x)
    host0 = [np.ascontiguousarray(t) for t in (U * J, J, x)]

    def device_run(ctx, steps, dt_fixed=0.0):
        D = [to_dev(t, torch) for t in host0]
        total = 0.0
        for _ in range(steps):
            xd, dd = ctx.es_step(*D, dt_fixed)
            total += float(dd[0])
        return [t.cpu() for t in D], total

    def host_run(ctx, steps, dt_fixed=0.0):
        H = [torch.from_numpy(t.copy()).pin_memory() for t in host0]
        total = ctx.es_run_host(*H, steps, dt_fixed)
        return H, total

    ctx = _ctx(pb, form)
    ref, tref = device_run(ctx, 3)
    got, tgot = host_run(ctx, 3)
    assert _same(got, ref) and tgot == tref
    got, tgot = host_run(ctx, 3)                     # the graph replayed again
    assert _same(got, ref) and tgot == tref
    # the state in one pinned block (JU, J, x consecutive): one transfer each way
    sizes = [t.size for t in host0]
    blk = torch.from_numpy(np.concatenate([t.reshape(-1) for t in host0])).pin_memory()
    H = list(torch.split(blk, sizes))
    tblk = ctx.es_run_host(*H, 3)
    assert _same([h.reshape(t.shape) for h, t in zip(H, ref)], ref) and tblk == tref
    ctx.es_set_fusion(-1)                            # per-direction launches: graph rebuilt
    got, _ = host_run(ctx, 3)
    assert _same(got, ref)
    dtf = 0.5 * tref / 3
    ref_f, tf = device_run(ctx, 2, dtf)
    got_f, tgf = host_run(ctx, 2, dtf)
    assert _same(got_f, ref_f) and tgf == tf == 2 * dtf
    ctx.es_profile(True)
    got, _ = host_run(ctx, 3)
    prof = ctx.es_profile_read()
    ctx.es_profile(False)
    assert _same(got, ref) and prof["flux_k1"][1] == 9 and prof["mesh"][1] == 3


@pytest.mark.parametrize("bc", ["periodic", "mixed", "reflect"])
def test_mesh_tiles_bitwise(bc):
    """The fused mixed 2D mesh step (monitor, filter passes and Jacobi sweeps in one launch) in
    every tile shape gives the mesh velocity and Delta t / Delta tau of shape 0 bit for bit:
    ragged and sub-tile grids, the largest fused halo (mu = 8, n_f = 4) and the smallest (one
    sweep, no filter pass), and a batch of uneven instances; es_autotune keeps one of the shapes
    and changes no result."""
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    for n, mu, nf, seed in (((70, 37), 5, 3, 21), ((10, 11), 4, 2, 22), ((53, 41), 8, 4, 23), ((33, 17), 1, 0, 24)):
        pb, JU, J, x, _ = case(2, 2, n, bc, es=True, seed=seed, jump=True)
        pb = pb.with_(mu=mu, nf=nf, sigma=(W.SIG_RHO1, W.SIG_P), alpha=(60.0, 25.0))
        ctx = _ctx(pb, 1)
        ju, jj, xx = to_dev(JU, torch), to_dev(J, torch), to_dev(x, torch)
        out = []
        for sh in range(NJF_SHAPE):
            ctx.es_set_mesh_tiles(sh)
            assert ctx.es_get_mesh_tiles()[0] == sh
            out.append(ctx.mesh_redistribute(ju, jj, xx))
        assert ctx.es_poll_status() == 0
        for o in out[1:]:
            assert _same(o, out[0]), (n, bc)
        ctx.es_autotune(ju, jj, xx, None, reps=2)
        assert 0 <= ctx.es_get_mesh_tiles()[0] < NJF_SHAPE and ctx.es_get_mesh_tiles()[4] > 0
        assert _same(ctx.mesh_redistribute(ju, jj, xx), out[0])
    # a batch of uneven instances, every shape against shape 0
    insts = []
    for n, seed in (((40, 23), 31), ((17, 52), 32), ((64, 12), 33)):
        pb, JU, J, x, _ = case(2, 2, n, bc, es=True, seed=seed, jump=True)
        insts.append((pb.with_(mu=5, nf=3, sigma=(W.SIG_RHO1, W.SIG_P), alpha=(60.0, 25.0)), JU, J, x))
    res = []
    for sh in range(NJF_SHAPE):
        b = es.Context([i[0] for i in insts], 1)
        b.es_set_mesh_tiles(sh)
        JUs = [to_dev(i[1], torch) for i in insts]
        Js = [to_dev(i[2], torch) for i in insts]
        Xs = [to_dev(i[3], torch) for i in insts]
        XD = [torch.zeros_like(t) for t in Xs]
        DD = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in insts]
        b.es_bind_batch(JUs, Js, Xs, XD, DD)
        b.es_step_batch()
        assert b.es_poll_status() == 0
        res.append(JUs + Js + Xs + XD + DD)
    for r in res[1:]:
        assert _same(r, res[0]), bc


def test_mesh_tiles_refused():
    """es_set_mesh_tiles refuses shapes out of range and contexts without the fused mixed 2D
    mesh step; es_get_mesh_tiles reports -1 there."""
    need_gpu()
    from paper_2202_07989_gb300 import es
    pb, *_ = case(2, 1, (20, 20), "periodic")
    pb = pb.with_(mu=5, nf=3)
    ctx = _ctx(pb, 1)
    for sh in (-1, NJF_SHAPE):
        with pytest.raises(RuntimeError):
            ctx.es_set_mesh_tiles(sh)
    f = _ctx(pb, 0)
    assert f.es_get_mesh_tiles()[0] == -1
    with pytest.raises(RuntimeError):
        f.es_set_mesh_tiles(0)
