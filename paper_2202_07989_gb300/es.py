"""Thin Python binding of libes.so (include/es.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module turns
a ``workloads.Problem`` into the C ``es_config``, checks tensor shapes, dtypes and
devices, and passes raw device pointers and the current CUDA stream.  There is
no CPU fallback: if the extension or a GPU is missing, the calls raise.

Function names follow the C ABI (es_create, es_init_mesh, es_metrics, es_rhs,
es_rk_step, mesh_redistribute, entropy_production, ...).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import torch

from .workloads import Problem

FP64, MIXED = 0, 1
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libes.so")
_lib = None

ES_STATUS = {0: "ES_OK", 1: "ES_ERR_ARG", 2: "ES_ERR_UNSUPPORTED", 3: "ES_ERR_CUDA",
             4: "ES_ERR_NONPHYSICAL", 5: "ES_ERR_TIMEOUT"}


class EsError(RuntimeError):
    pass


class EsConfig(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("N", C.c_int), ("n", C.c_int * 3),
        ("xi_lo", C.c_double * 3), ("dxi", C.c_double * 3), ("bc", (C.c_int * 2) * 3),
        ("inflow", ((C.c_double * 8) * 2) * 3),
        ("gamma", C.c_double * 2), ("cv", C.c_double * 2), ("pinf", C.c_double * 2),
        ("es", C.c_int), ("precision", C.c_int),
        ("chi", C.c_double * 3), ("weno_eps", C.c_double), ("cfl", C.c_double),
        ("n_sigma", C.c_int), ("sigma", C.c_int * 4), ("alpha", C.c_double * 4),
        ("mu", C.c_int), ("nf", C.c_int), ("weno", C.c_int), ("fixed_mesh", C.c_int),
        ("sigma_op", C.c_int * 4), ("w", C.c_int), ("march_planes", C.c_int),
    ]


def lib():
    """Load libes.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise EsError("libes.so is not built: run paper_2202_07989_gb300/build.py (or __graft_entry__.build())")
        L = C.CDLL(_LIB_PATH)
        vp, dp, ip = C.c_void_p, C.c_void_p, C.POINTER(C.c_int)
        sig = {
            "es_create": (C.c_int, [C.POINTER(EsConfig), C.POINTER(vp)]),
            "es_create_batch": (C.c_int, [C.POINTER(EsConfig), C.c_int, C.POINTER(vp)]),
            "es_destroy": (None, [vp]),
            "es_last_error": (C.c_char_p, [vp]),
            "es_num_instances": (C.c_int, [vp]),
            "es_scratch_bytes": (C.c_ulonglong, [vp]),
            "es_init_mesh": (C.c_int, [vp, dp, dp, vp]),
            "es_metrics": (C.c_int, [vp, dp, dp, dp, vp]),
            "es_rhs": (C.c_int, [vp, dp, dp, dp, dp, dp, dp, vp]),
            "es_rk_step": (C.c_int, [vp, dp, dp, dp, dp, dp, vp]),
            "mesh_redistribute": (C.c_int, [vp, dp, dp, dp, C.c_double, dp, dp, vp]),
            "es_step": (C.c_int, [vp, dp, dp, dp, C.c_double, dp, dp, vp]),
            "es_schlieren": (C.c_int, [vp, dp, dp, dp, C.c_double, C.c_double, dp, vp]),
            "es_autotune": (C.c_int, [vp, dp, dp, dp, dp, C.c_int, vp]),
            "es_get_tuning": (C.c_int, [vp, ip, ip, ip, ip, C.POINTER(C.c_float)]),
            "es_set_tuning": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
            "es_get_fusion": (C.c_int, [vp, ip, ip, ip, ip, C.POINTER(C.c_float)]),
            "es_set_fusion": (C.c_int, [vp, C.c_int, C.c_int]),
            "es_get_mesh_tiles": (C.c_int, [vp, ip, ip, ip, ip, C.POINTER(C.c_float)]),
            "es_set_mesh_tiles": (C.c_int, [vp, C.c_int]),
            "entropy_production": (C.c_int, [vp, dp, dp, dp, dp, dp, vp]),
            "es_bind_batch": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
            "es_step_batch": (C.c_int, [vp, vp]),
            "es_run_host": (C.c_int, [vp, dp, dp, dp, C.c_int, C.c_double, C.POINTER(C.c_double), vp]),
            "es_poll_status": (C.c_int, [vp, ip, vp]),
            "es_profile": (C.c_int, [vp, C.c_int]),
            "es_check_conversions": (C.c_int, [dp, C.c_int, dp, dp, vp]),
            "es_check_half_sums": (C.c_int, [dp, dp, C.c_int, dp, vp]),
            "es_check_logmean_small": (C.c_int, [dp, dp, dp, C.c_int, dp, dp, vp]),
            "es_entropy_production_noalloc": (C.c_int, [C.POINTER(EsConfig), dp, dp, dp, dp, dp, vp]),
            "es_profile_read": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]),
            "es_alu_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, vp]),
            "es_alu_peak_flops": (C.c_longlong, [C.c_int, C.c_int, C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def make_config(pb: Problem, precision: int = FP64, march_planes: int = 0) -> EsConfig:
    """The C es_config of a problem; march_planes fixes the plane chunk of the 3D mixed
    mesh-step kernels (0 = automatic), a schedule choice that changes no result."""
    c = EsConfig()
    c.march_planes = int(march_planes)
    c.d, c.N = pb.d, pb.N
    for k in range(3):
        c.n[k] = pb.n[k] if k < pb.d else 1
        c.xi_lo[k] = pb.xi_lo[k]
        c.dxi[k] = pb.dxi[k]
        for s in range(2):
            c.bc[k][s] = pb.bc[k][s]
            if pb.inflow is not None:
                for q in range(8):
                    c.inflow[k][s][q] = float(pb.inflow[k, s, q])
    for l in range(2):
        c.gamma[l], c.cv[l], c.pinf[l] = pb.gamma[l], pb.cv[l], pb.pinf[l]
    c.es = int(pb.es)
    c.precision = int(precision)
    for q in range(3):
        c.chi[q] = pb.chi[q]
    c.weno_eps, c.cfl = pb.weno_eps, pb.cfl
    c.n_sigma = len(pb.sigma)
    for q, (s, a) in enumerate(zip(pb.sigma, pb.alpha)):
        c.sigma[q], c.alpha[q] = s, a
    c.mu, c.nf = pb.mu, pb.nf
    c.weno, c.fixed_mesh = int(pb.weno), int(pb.fixed_mesh)
    for q, op in enumerate(pb.sigma_op):
        c.sigma_op[q] = int(op)
    c.w = int(pb.w)
    return c


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor], fields: int, pb: Problem, name: str) -> Optional[C.c_void_p]:
    if t is None:
        return None
    if not t.is_cuda:
        raise EsError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise EsError("%s must be float64" % name)
    if not t.is_contiguous():
        raise EsError("%s must be contiguous" % name)
    if t.numel() != fields * pb.ncell:
        raise EsError("%s has %d elements, expected %d" % (name, t.numel(), fields * pb.ncell))
    return C.c_void_p(t.data_ptr())


class Context:
    """An es_ctx for one instance (or a batch of instances sharing d, N, precision, mu, nf)."""

    def __init__(self, problems, precision: int = FP64, march_planes: int = 0):
        if isinstance(problems, Problem):
            problems = [problems]
        self.problems = list(problems)
        self.pb = self.problems[0]
        self.precision = precision
        self.L = lib()
        cfgs = (EsConfig * len(self.problems))(*[make_config(p, precision, march_planes) for p in self.problems])
        h = C.c_void_p()
        if len(self.problems) == 1:
            st = self.L.es_create(cfgs, C.byref(h))
        else:
            st = self.L.es_create_batch(cfgs, len(self.problems), C.byref(h))
        if st != 0 or not h.value:
            raise EsError("es_create failed: %s" % ES_STATUS.get(st, st))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                self.L.es_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _chk(self, st: int, what: str):
        if st != 0:
            msg = self.L.es_last_error(self.h)
            raise EsError("%s: %s (%s)" % (what, ES_STATUS.get(st, st), msg.decode() if msg else ""))

    @property
    def scratch_bytes(self) -> int:
        return int(self.L.es_scratch_bytes(self.h))

    def padded_shape(self):
        pb = self.pb
        return (pb.n[2] + 6 if pb.d == 3 else 1, pb.n[1] + 6, pb.n[0] + 6)

    # ---- the C calls ----------------------------------------------------------
    def es_init_mesh(self, x: torch.Tensor, J: Optional[torch.Tensor] = None) -> torch.Tensor:
        pb = self.pb
        if J is None:
            J = torch.empty(pb.shape, dtype=torch.float64, device=x.device)
        self._chk(self.L.es_init_mesh(self.h, _ptr(x, pb.d, pb, "x"), _ptr(J, 1, pb, "J"), _stream()), "es_init_mesh")
        return J

    def es_metrics(self, x: torch.Tensor, xdot: Optional[torch.Tensor] = None) -> torch.Tensor:
        pb = self.pb
        M = torch.empty((pb.d * (pb.d + 1),) + self.padded_shape(), dtype=torch.float64, device=x.device)
        self._chk(self.L.es_metrics(self.h, _ptr(x, pb.d, pb, "x"), _ptr(xdot, pb.d, pb, "xdot"),
                                    C.c_void_p(M.data_ptr()), _stream()), "es_metrics")
        return M

    def es_rhs(self, JU, J, x, xdot=None, dJU=None, dJ=None):
        pb = self.pb
        if dJU is None:
            dJU = torch.empty((pb.nc,) + pb.shape, dtype=torch.float64, device=JU.device)
        if dJ is None:
            dJ = torch.empty(pb.shape, dtype=torch.float64, device=JU.device)
        self._chk(self.L.es_rhs(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"), _ptr(x, pb.d, pb, "x"),
                                _ptr(xdot, pb.d, pb, "xdot"), _ptr(dJU, pb.nc, pb, "dJU"), _ptr(dJ, 1, pb, "dJ"),
                                _stream()), "es_rhs")
        return dJU, dJ

    def es_rk_step(self, JU, J, x, xdot, dt: torch.Tensor):
        pb = self.pb
        if not (dt.is_cuda and dt.dtype == torch.float64):
            raise EsError("dt must be a float64 CUDA tensor")
        self._chk(self.L.es_rk_step(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"), _ptr(x, pb.d, pb, "x"),
                                    _ptr(xdot, pb.d, pb, "xdot"), C.c_void_p(dt.data_ptr()), _stream()), "es_rk_step")

    def mesh_redistribute(self, JU, J, x, dt_fixed: float = 0.0, xdot=None, dt_dtau=None):
        pb = self.pb
        if xdot is None:
            xdot = torch.empty((pb.d,) + pb.shape, dtype=torch.float64, device=JU.device)
        if dt_dtau is None:
            dt_dtau = torch.empty(2, dtype=torch.float64, device=JU.device)
        self._chk(self.L.mesh_redistribute(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"),
                                           _ptr(x, pb.d, pb, "x"), float(dt_fixed), _ptr(xdot, pb.d, pb, "xdot"),
                                           C.c_void_p(dt_dtau.data_ptr()), _stream()), "mesh_redistribute")
        return xdot, dt_dtau

    def es_step(self, JU, J, x, dt_fixed: float = 0.0, xdot=None, dt_dtau=None):
        """One full time step (mesh redistribution, then SSP-RK3) of (JU, J, x) in place."""
        pb = self.pb
        if xdot is None:
            xdot = torch.empty((pb.d,) + pb.shape, dtype=torch.float64, device=JU.device)
        if dt_dtau is None:
            dt_dtau = torch.empty(2, dtype=torch.float64, device=JU.device)
        self._chk(self.L.es_step(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"), _ptr(x, pb.d, pb, "x"),
                                 float(dt_fixed), _ptr(xdot, pb.d, pb, "xdot"), C.c_void_p(dt_dtau.data_ptr()),
                                 _stream()), "es_step")
        return xdot, dt_dtau

    def es_autotune(self, JU=None, J=None, x=None, xdot=None, reps: int = 5):
        """Pick the flux tile shape and grid per direction by timing them on the given state
        (single instance) or on the bound batch (no arguments); returns es_get_tuning()."""
        pb = self.pb
        if JU is None:
            args = (None, None, None, None)
        else:
            args = (_ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"), _ptr(x, pb.d, pb, "x"), _ptr(xdot, pb.d, pb, "xdot"))
        self._chk(self.L.es_autotune(self.h, *args, int(reps), _stream()), "es_autotune")
        return self.es_get_tuning()

    def es_get_tuning(self):
        """[(shape, S, WT, grid, ms per launch)] for the directions of the problem."""
        a = [(C.c_int * 3)() for _ in range(4)]
        ms = (C.c_float * 3)()
        self._chk(self.L.es_get_tuning(self.h, a[0], a[1], a[2], a[3], ms), "es_get_tuning")
        return [(a[0][k], a[1][k], a[2][k], a[3][k], ms[k]) for k in range(self.pb.d)]

    def es_set_tuning(self, k: int, shape: int, grid: int = 0):
        self._chk(self.L.es_set_tuning(self.h, int(k), int(shape), int(grid)), "es_set_tuning")

    def es_get_fusion(self):
        """(fused shape or -1, TX, TY, grid, best fused ms per launch) of the 2D stage launch."""
        a = [C.c_int() for _ in range(4)]
        ms = C.c_float()
        self._chk(self.L.es_get_fusion(self.h, *[C.byref(v) for v in a], C.byref(ms)), "es_get_fusion")
        return tuple(v.value for v in a) + (ms.value,)

    def es_set_fusion(self, shape: int, grid: int = 0):
        """Fused 2D stage launch in fused shape `shape` (0..4), or -1 for one launch per direction."""
        self._chk(self.L.es_set_fusion(self.h, int(shape), int(grid)), "es_set_fusion")

    def es_get_mesh_tiles(self):
        """(shape or -1, TX, TY, threads, best ms per launch) of the fused mixed 2D mesh-step launch."""
        a = [C.c_int() for _ in range(4)]
        ms = C.c_float()
        self._chk(self.L.es_get_mesh_tiles(self.h, *[C.byref(v) for v in a], C.byref(ms)), "es_get_mesh_tiles")
        return tuple(v.value for v in a) + (ms.value,)

    def es_set_mesh_tiles(self, shape: int):
        """Fused mixed 2D mesh-step launch in tile shape `shape` (0..3)."""
        self._chk(self.L.es_set_mesh_tiles(self.h, int(shape)), "es_set_mesh_tiles")

    def es_schlieren(self, JU, J, x, psi1: float = 30.0, psi2: float = 150.0, phi=None):
        """Schlieren function of Eq. (schlieren) at the nodes."""
        pb = self.pb
        if phi is None:
            phi = torch.empty(pb.shape, dtype=torch.float64, device=JU.device)
        self._chk(self.L.es_schlieren(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"), _ptr(x, pb.d, pb, "x"),
                                      float(psi1), float(psi2), _ptr(phi, 1, pb, "phi"), _stream()), "es_schlieren")
        return phi

    def entropy_production(self, JU, J, dJU=None, dJ=None, out=None):
        pb = self.pb
        if out is None:
            out = torch.empty(2, dtype=torch.float64, device=JU.device)
        self._chk(self.L.entropy_production(self.h, _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"),
                                            _ptr(dJU, pb.nc, pb, "dJU"), _ptr(dJ, 1, pb, "dJ"),
                                            C.c_void_p(out.data_ptr()), _stream()), "entropy_production")
        return out

    def es_bind_batch(self, JU: Sequence[torch.Tensor], J, x, xdot, dt_dtau):
        n = len(self.problems)

        def tab(ts, fields, name, scalar=False):
            arr = (C.c_void_p * n)()
            for i, t in enumerate(ts):
                if scalar:
                    if not (t.is_cuda and t.dtype == torch.float64 and t.numel() >= 2):
                        raise EsError("%s[%d] must be a float64 CUDA tensor of 2 entries" % (name, i))
                    arr[i] = t.data_ptr()
                else:
                    arr[i] = _ptr(ts[i], fields(self.problems[i]), self.problems[i], "%s[%d]" % (name, i)).value
            return arr

        self._keep = (JU, J, x, xdot, dt_dtau)
        self._chk(self.L.es_bind_batch(self.h, tab(JU, lambda p: p.nc, "JU"), tab(J, lambda p: 1, "J"),
                                       tab(x, lambda p: p.d, "x"), tab(xdot, lambda p: p.d, "xdot"),
                                       tab(dt_dtau, None, "dt_dtau", scalar=True)), "es_bind_batch")

    def es_step_batch(self):
        self._chk(self.L.es_step_batch(self.h, _stream()), "es_step_batch")

    def es_run_host(self, JU: torch.Tensor, J: torch.Tensor, x: torch.Tensor, steps: int, dt_fixed: float = 0.0) -> float:
        """Full steps on HOST tensors (float64, contiguous; pinned for asynchronous copies)."""
        pb = self.pb
        for t, f, nm in ((JU, pb.nc, "JU"), (J, 1, "J"), (x, pb.d, "x")):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != f * pb.ncell:
                raise EsError("%s must be a contiguous float64 host tensor of %d elements" % (nm, f * pb.ncell))
        tt = C.c_double(0.0)
        self._chk(self.L.es_run_host(self.h, C.c_void_p(JU.data_ptr()), C.c_void_p(J.data_ptr()),
                                     C.c_void_p(x.data_ptr()), int(steps), float(dt_fixed), C.byref(tt), _stream()),
                  "es_run_host")
        return tt.value

    PROFILE_CLASSES = ("flux_k1", "flux_k2", "flux_k3", "metrics", "mesh", "entropy", "flux_2d")

    def es_profile(self, enable: bool = True):
        self._chk(self.L.es_profile(self.h, int(enable)), "es_profile")

    def es_profile_read(self):
        """{class: (milliseconds, launches)} since the last read (synchronises)."""
        n = len(self.PROFILE_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        self._chk(self.L.es_profile_read(self.h, ms, cnt, n), "es_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.PROFILE_CLASSES)}

    def es_poll_status(self) -> int:
        f = C.c_int(0)
        st = self.L.es_poll_status(self.h, C.byref(f), _stream())
        if st not in (0, 4):
            self._chk(st, "es_poll_status")
        return f.value


def es_check_conversions(x: torch.Tensor):
    """(binary32, widened binary64) of a float64 CUDA tensor through the library's integer-pipe
    conversions."""
    if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise EsError("x must be a contiguous float64 CUDA tensor")
    o32 = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    o64 = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    st = lib().es_check_conversions(C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(o32.data_ptr()),
                                    C.c_void_p(o64.data_ptr()), _stream())
    if st != 0:
        raise EsError("es_check_conversions: %s" % ES_STATUS.get(st, st))
    return o32, o64


def es_check_half_sums(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """a/2 + b/2 in binary64 of two float32 CUDA tensors through the library's integer-built
    exact mean (the log-mean small-jump branch of the mixed form)."""
    for t, nm in ((a, "a"), (b, "b")):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise EsError("%s must be a contiguous float32 CUDA tensor" % nm)
    if a.shape != b.shape:
        raise EsError("a and b must have the same shape")
    out = torch.empty(a.shape, dtype=torch.float64, device=a.device)
    st = lib().es_check_half_sums(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), a.numel(),
                                  C.c_void_p(out.data_ptr()), _stream())
    if st != 0:
        raise EsError("es_check_half_sums: %s" % ES_STATUS.get(st, st))
    return out


def es_check_logmean_small(a: torch.Tensor, b: torch.Tensor, d: torch.Tensor):
    """(fast, general) binary32 values of the log-mean small-jump branch {a}(1 - d) for float32
    CUDA tensors a, b > 0 and 0 <= d <= 1/2."""
    for t, nm in ((a, "a"), (b, "b"), (d, "d")):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise EsError("%s must be a contiguous float32 CUDA tensor" % nm)
    if not (a.shape == b.shape == d.shape):
        raise EsError("a, b and d must have the same shape")
    fast = torch.empty_like(a)
    general = torch.empty_like(a)
    st = lib().es_check_logmean_small(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(d.data_ptr()),
                                      a.numel(), C.c_void_p(fast.data_ptr()), C.c_void_p(general.data_ptr()), _stream())
    if st != 0:
        raise EsError("es_check_logmean_small: %s" % ES_STATUS.get(st, st))
    return fast, general


# module-level aliases with the C names
def es_create(pb: Problem, precision: int = FP64) -> Context:
    return Context(pb, precision)


def es_create_batch(problems: Sequence[Problem], precision: int = FP64) -> Context:
    return Context(list(problems), precision)


def es_entropy_production_noalloc(pb: Problem, JU, J, dJU, dJ, out2, precision: int = FP64) -> int:
    """Allocation-free entropy diagnostics (no context, no device allocation): for callers
    that may not allocate device memory, e.g. while capturing a CUDA graph or inside a
    runtime that owns all device memory.  out2 (2 float64 on the device) is filled with
    {P, S}; returns the es_status code (0 on success).  Grids over 1,048,576 nodes are
    rejected (ES_ERR_ARG)."""
    if not (out2.is_cuda and out2.dtype == torch.float64 and out2.numel() >= 2 and out2.is_contiguous()):
        raise EsError("out2 must be a contiguous float64 CUDA tensor of 2 entries")
    cfg = make_config(pb, precision)
    return lib().es_entropy_production_noalloc(C.byref(cfg), _ptr(JU, pb.nc, pb, "JU"), _ptr(J, 1, pb, "J"),
                                                _ptr(dJU, pb.nc, pb, "dJU"), _ptr(dJ, 1, pb, "dJ"),
                                                C.c_void_p(out2.data_ptr()), _stream())


ALU_KINDS = ("fp32_ffma", "fp32_ffma2", "fp64_dfma")


def es_alu_peak(kind: int, grid: int, iters: int, sink: torch.Tensor) -> int:
    """Launch the ALU throughput microbenchmark (kind 0 FFMA, 1 FFMA2, 2 DFMA) on the current
    stream; sink is a float64 CUDA tensor of at least grid * 256 entries.  Returns the flops of
    the launch; the caller times it."""
    if not (sink.is_cuda and sink.dtype == torch.float64 and sink.is_contiguous() and sink.numel() >= grid * 256):
        raise EsError("sink must be a contiguous float64 CUDA tensor of grid * 256 entries")
    st = lib().es_alu_peak(int(kind), int(grid), int(iters), C.c_void_p(sink.data_ptr()), _stream())
    if st != 0:
        raise EsError("es_alu_peak: %s" % ES_STATUS.get(st, st))
    return int(lib().es_alu_peak_flops(int(kind), int(grid), int(iters)))
