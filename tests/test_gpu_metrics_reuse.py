"""Reuse of the 3D spatial metrics across time steps.

The pass that opens a 3D mesh step keeps the spatial metrics in the context's metrics buffer
when they were formed from the very same positions: the second SSP-RK3 stage's mesh
x^n + dt xdot is, bit for bit, the next step's mesh, and a fixed mesh never changes.  Otherwise
it forms them again.  Kept and re-formed metrics agree bit for bit, so a run that reuses must
equal a run whose reuse is defeated between steps, and a mesh changed between steps must give
what a fresh context gives on the changed state.
"""
import pytest

from paper_2202_07989_gb300 import workloads as W

from .helpers import case, need_gpu, to_dev

pytestmark = pytest.mark.gpu

CASES = [((20, 14, 12), "periodic", 1, 1), ((13, 22, 15), "reflect", 2, 2), ((24, 12, 11), "mixed", 3, 2)]


def _problem(n, bc, seed, N, fixed):
    pb, JU, J, x, _ = case(3, N, n, bc, es=True, seed=seed, pinf=0.7)
    sigma = (W.SIG_RHO, W.SIG_P) if N == 1 else (W.SIG_RHO1, W.SIG_P)
    pb = pb.with_(mu=4, nf=2, sigma=sigma, alpha=(50.0, 20.0), fixed_mesh=fixed)
    return pb, JU, J, x


@pytest.mark.parametrize("fixed", [False, True])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,bc,seed,N", CASES)
def test_reused_metrics_equal_reformed(n, bc, seed, N, form, fixed):
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, JU0, J0, x0 = _problem(n, bc, seed, N, fixed)
    out = []
    for spoil in (None, "mesh", "velocity"):
        c = es.Context(pb, form)
        ju, jj, xx = (to_dev(a, torch) for a in (JU0, J0, x0))
        for s in range(3):
            if spoil == "mesh" and s > 0:
                # metrics of another mesh into the context's buffer: the mesh step must form
                # those of xx again
                c.es_rhs(ju, jj, (xx * 1.01).contiguous())
            if spoil == "velocity" and s > 0:
                # the same mesh with a nonzero mesh velocity: the spatial rows may be kept, the
                # VCL rows (zero on a fixed mesh) must be formed again
                c.es_rhs(ju, jj, xx, (0.01 * xx).contiguous())
            c.es_step(ju, jj, xx)
        assert c.es_poll_status() == 0
        out.append((ju, jj, xx))
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert torch.equal(a, b)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,bc,seed,N", CASES)
def test_changed_mesh_is_not_reused(n, bc, seed, N, form):
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, JU0, J0, x0 = _problem(n, bc, seed, N, False)
    c = es.Context(pb, form)
    ju, jj, xx = (to_dev(a, torch) for a in (JU0, J0, x0))
    c.es_step(ju, jj, xx)
    # move one interior node by a small fraction of the spacing between the steps
    k = (n[2] // 2, n[1] // 2, n[0] // 2)
    for j in range(3):
        xx[(j,) + k] += 1e-4 * pb.dxi[j]
    ref = [t.clone() for t in (ju, jj, xx)]
    c.es_step(ju, jj, xx)
    assert c.es_poll_status() == 0
    f = es.Context(pb, form)
    f.es_step(*ref)
    assert f.es_poll_status() == 0
    for a, b in zip((ju, jj, xx), ref):
        assert torch.equal(a, b)


@pytest.mark.parametrize("fixed", [False, True])
def test_run_host_reuses_across_calls(fixed):
    """es_run_host replays one CUDA graph of a step; the reuse test runs on the device inside it.
    Five steps as 3 + 2 steps of es_run_host on host buffers (the second call copies in the state
    the first left, whose metrics the context still holds) equal five es_step calls on device
    buffers in a fresh context, bit for bit."""
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, JU0, J0, x0 = _problem((20, 14, 12), "mixed", 5, 2, fixed)
    c = es.Context(pb, 1)
    H = [torch.from_numpy(a.copy()).pin_memory() for a in (JU0, J0, x0)]
    t = c.es_run_host(*H, 3)
    t += c.es_run_host(*H, 2)
    assert c.es_poll_status() == 0
    d = es.Context(pb, 1)
    D = [to_dev(a, torch) for a in (JU0, J0, x0)]
    td = 0.0
    for _ in range(5):
        _, dd = d.es_step(*D)
        td += float(dd[0])
    assert d.es_poll_status() == 0
    for a, b in zip(H, D):
        assert torch.equal(a, b.cpu())
    assert t == pytest.approx(td, rel=1e-14)
