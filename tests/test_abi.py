"""CPU checks of the C ABI: the library loads, exports every function include/es.h
declares, and rejects bad configurations on the host before touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "es.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:es_status|void|const char\*|int|unsigned long long|long long)\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_07989_gb300 import build as B
    B.build()
    from paper_2202_07989_gb300 import es
    return es.lib()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ["es_init_mesh", "es_metrics", "es_rhs", "es_rk_step", "mesh_redistribute", "entropy_production"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_bad_configs_rejected_on_host(lib):
    from paper_2202_07989_gb300 import es, workloads as W
    good = W.random_problem(2, 1, (16, 16))
    bad = [good.with_(n=(8, 16, 1)), good.with_(d=4), good.with_(N=3),
           good.with_(bc=((0, 1), (0, 0), (0, 0))), good.with_(gamma=(0.9, 1.4)),
           good.with_(chi=(0.0, 0.5, 0.5)), good.with_(mu=-1), good.with_(sigma=(9,), alpha=(1.0,)),
           good.with_(w=4), good.with_(sigma=(0,), alpha=(1.0,), sigma_op=(7,))]
    for pb in bad:
        cfg = es.make_config(pb)
        h = C.c_void_p()
        st = lib.es_create(C.byref(cfg), C.byref(h))
        assert st == 1 and not h.value, (pb, st)
    cfg = es.make_config(good, precision=7)
    h = C.c_void_p()
    assert lib.es_create(C.byref(cfg), C.byref(h)) == 1
    cfg = es.make_config(good)
    cfg.n_sigma = 5                     # at most 4 monitor terms
    assert lib.es_create(C.byref(cfg), C.byref(h)) == 1 and not h.value


def test_batch_members_must_share_the_step_structure(lib):
    """A batch's instances may differ in size, boundaries and physics, but not in d, N, the
    precision, mu, n_f, the fixed-mesh flag or the dissipation variant (one launch sequence
    serves all of them): es_create_batch refuses with ES_ERR_UNSUPPORTED, on the host."""
    from paper_2202_07989_gb300 import es, workloads as W
    a = W.random_problem(2, 1, (16, 16))
    for b in (a.with_(mu=a.mu + 1), a.with_(nf=a.nf + 1), a.with_(weno=1), a.with_(fixed_mesh=True)):
        cfgs = (es.EsConfig * 2)(es.make_config(a), es.make_config(b))
        h = C.c_void_p()
        assert lib.es_create_batch(cfgs, 2, C.byref(h)) == 2 and not h.value, b
    h = C.c_void_p()
    assert lib.es_create_batch(None, 2, C.byref(h)) == 1 and not h.value


def test_null_context_calls(lib):
    assert lib.es_rhs(None, None, None, None, None, None, None, None) == 1
    assert lib.es_num_instances(None) == 0
    assert lib.es_last_error(None) == b"null context"
