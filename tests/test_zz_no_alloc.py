"""The allocation-free entropy diagnostics call, es_entropy_production_noalloc.

Some callers may not allocate device memory (a runtime that owns every byte of device
memory, a real-time loop).  For them the library offers one call that keeps its scratch
in a fixed library-wide device array instead of a context.  This test calls it through the C ABI twice in a row, on different inputs,
and checks each result against entropy_production of a context, within the tolerance
of the other parity tests; it also checks that grids over the limit are refused and that a
call leaves the device's free memory unchanged.
It lives in a file that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

from .helpers import case, need_gpu, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _ref_and_inputs(torch, d, N, n, seed):
    from paper_2202_07989_gb300 import es
    pb, JU, J, x, xdot = case(d, N, n, "periodic", es=True, seed=seed)
    ctx = es.Context(pb)
    JUg, Jg = to_dev(JU, torch), to_dev(J, torch)
    dJU, dJ = ctx.es_rhs(JUg, Jg, to_dev(x, torch), to_dev(xdot, torch))
    ref = ctx.entropy_production(JUg, Jg, dJU, dJ).cpu().numpy()
    scale = np.abs(dJU.cpu().numpy()).sum() * np.prod(pb.dxi[:d])
    return pb, JUg, Jg, dJU, dJ, ref, scale


def test_noalloc_matches_context_call_twice():
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    first = _ref_and_inputs(torch, 2, 2, (70, 37), 31)
    second = _ref_and_inputs(torch, 3, 1, (22, 12, 11), 32)
    # outputs are allocated by the caller before the calls
    outs = [torch.full((2,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    for (pb, JU, J, dJU, dJ, ref, scale), out in zip((first, second), outs):
        st = es.es_entropy_production_noalloc(pb, JU, J, dJU, dJ, out)
        assert st == 0
    torch.cuda.synchronize()
    for (pb, JU, J, dJU, dJ, ref, scale), out in zip((first, second), outs):
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= TOL * scale, (got, ref)
        assert abs(got[1] - ref[1]) <= TOL * abs(ref[1]), (got, ref)


def test_noalloc_leaves_free_device_memory_unchanged():
    torch = need_gpu()
    from paper_2202_07989_gb300 import es
    pb, JU, J, dJU, dJ, ref, scale = _ref_and_inputs(torch, 2, 2, (70, 37), 33)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert es.es_entropy_production_noalloc(pb, JU, J, dJU, dJ, out) == 0   # loads the kernels
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert es.es_entropy_production_noalloc(pb, JU, J, dJU, dJ, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = out.cpu().numpy()
    assert abs(got[0] - ref[0]) <= TOL * scale and abs(got[1] - ref[1]) <= TOL * abs(ref[1])


def test_noalloc_rejects_grids_over_the_limit():
    torch = need_gpu()
    from paper_2202_07989_gb300 import es, workloads as W
    pb = W.random_problem(2, 1, (1025, 1024))
    cfg = es.make_config(pb)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    fake = C.c_void_p(out.data_ptr())
    st = es.lib().es_entropy_production_noalloc(C.byref(cfg), fake, fake, None, None, fake, None)
    assert st == 1
