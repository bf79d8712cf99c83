"""ctypes front end of the FP64 CPU oracle (arXiv 2202.07989).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg import it; the product library never does.  It converts a
``workloads.Problem`` into the oracle's own configuration struct and passes
numpy float64 arrays (field-major, (fields, n3, n2, n1)) to the C functions in
es_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrConfig(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("N", C.c_int), ("n", C.c_int * 3), ("w", C.c_int), ("es", C.c_int),
        ("xi_lo", C.c_double * 3), ("dxi", C.c_double * 3), ("bc", (C.c_int * 2) * 3),
        ("inflow", ((C.c_double * 8) * 2) * 3),
        ("gamma", C.c_double * 2), ("cv", C.c_double * 2), ("pinf", C.c_double * 2),
        ("chi", C.c_double * 3), ("weno_eps", C.c_double), ("cfl", C.c_double),
        ("n_sigma", C.c_int), ("sigma", C.c_int * 4), ("alpha", C.c_double * 4),
        ("mu", C.c_int), ("nf", C.c_int), ("y_band", C.c_double), ("weno", C.c_int),
        ("sigma_op", C.c_int * 4),
    ]


def bind(L):
    """Set the C signatures of the oracle's entry points on a loaded library (the plain build
    or the operation-counting build, which export the same functions)."""
    dp = C.POINTER(C.c_double)
    cp = C.POINTER(OrConfig)
    sig = {
        "or_alpha": (None, [C.c_int, dp]),
        "or_primitives": (None, [cp, dp, dp, dp, dp, dp]),
        "or_entropy_vars": (None, [cp, dp, dp]),
        "or_eta": (C.c_double, [cp, dp]),
        "or_phi": (C.c_double, [cp, dp]),
        "or_phys_flux": (None, [cp, C.c_int, dp, dp]),
        "or_logmean": (C.c_double, [C.c_double, C.c_double]),
        "or_Utilde": (None, [cp, dp, dp, dp]),
        "or_Ftilde": (None, [cp, C.c_int, dp, dp, dp]),
        "or_ec_pair": (None, [cp, dp, dp, dp, dp, dp]),
        "or_eigvec_point": (None, [cp, dp, dp]),
        "or_eigvec_avg": (None, [cp, dp, dp, dp, dp]),
        "or_weno_mr": (C.c_double, [dp, dp, C.c_double]),
        "or_weno_js": (C.c_double, [dp, C.c_double]),
        "or_metrics": (None, [cp, dp, dp, dp]),
        "or_init_J": (None, [cp, dp, dp]),
        "or_rhs": (None, [cp, dp, dp, dp, dp, dp, dp]),
        "or_rk_step": (None, [cp, dp, dp, dp, dp, C.c_double]),
        "or_rhs_margins": (None, [cp, dp, dp, dp, dp, dp, dp, dp]),
        "or_cfl_dt": (C.c_double, [cp, dp, dp, dp]),
        "or_monitor": (None, [cp, dp, dp, dp]),
        "or_schlieren": (None, [cp, dp, dp, dp, C.c_double, C.c_double, dp]),
        "or_filter": (None, [cp, dp]),
        "or_jacobi": (None, [cp, dp, dp, dp]),
        "or_limiter": (C.c_double, [cp, dp, dp]),
        "or_mesh_redistribute": (None, [cp, dp, dp, dp, C.c_double, dp, dp]),
        "or_entropy": (None, [cp, dp, dp, dp, dp, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = bind(C.CDLL(_build.build()))
    return _lib


def config(pb) -> OrConfig:
    c = OrConfig()
    c.d, c.N, c.w, c.es = pb.d, pb.N, pb.w, int(pb.es)
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
    for q in range(3):
        c.chi[q] = pb.chi[q]
    c.weno_eps, c.cfl = pb.weno_eps, pb.cfl
    c.n_sigma = len(pb.sigma)
    for q, (s, a) in enumerate(zip(pb.sigma, pb.alpha)):
        c.sigma[q], c.alpha[q] = s, a
    c.mu, c.nf = pb.mu, pb.nf
    c.y_band = 0.0
    c.weno = int(getattr(pb, "weno", 0))
    for q, op in enumerate(getattr(pb, "sigma_op", ())):
        c.sigma_op[q] = int(op)
    return c


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle wants contiguous float64"
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """The oracle bound to one problem description."""

    def __init__(self, pb):
        self.pb = pb
        self.cfg = config(pb)
        self.L = lib()
        self.nc = pb.nc

    # ---- pointwise physics -------------------------------------------------
    def alpha(self, w=None):
        out = np.zeros(3)
        self.L.or_alpha(w or self.pb.w, _p(out))
        return out[: (w or self.pb.w)]

    def primitives(self, U):
        U = _f64(U)
        rl, v, T, p = np.zeros(2), np.zeros(3), np.zeros(1), np.zeros(1)
        self.L.or_primitives(C.byref(self.cfg), _p(U), _p(rl), _p(v), _p(T), _p(p))
        return rl[: self.pb.N], v[: self.pb.d], T[0], p[0]

    def entropy_vars(self, U):
        V = np.zeros(self.nc)
        self.L.or_entropy_vars(C.byref(self.cfg), _p(_f64(U)), _p(V))
        return V

    def eta(self, U):
        return self.L.or_eta(C.byref(self.cfg), _p(_f64(U)))

    def phi(self, U):
        return self.L.or_phi(C.byref(self.cfg), _p(_f64(U)))

    def phys_flux(self, j, U):
        F = np.zeros(self.nc)
        self.L.or_phys_flux(C.byref(self.cfg), j, _p(_f64(U)), _p(F))
        return F

    def logmean(self, a, b):
        return self.L.or_logmean(float(a), float(b))

    def Utilde(self, Ul, Ur):
        out = np.zeros(self.nc)
        self.L.or_Utilde(C.byref(self.cfg), _p(_f64(Ul)), _p(_f64(Ur)), _p(out))
        return out

    def Ftilde(self, j, Ul, Ur):
        out = np.zeros(self.nc)
        self.L.or_Ftilde(C.byref(self.cfg), j, _p(_f64(Ul)), _p(_f64(Ur)), _p(out))
        return out

    def ec_pair(self, Ul, Ur, Ml, Mr):
        out = np.zeros(self.nc)
        self.L.or_ec_pair(C.byref(self.cfg), _p(_f64(Ul)), _p(_f64(Ur)), _p(_f64(Ml)), _p(_f64(Mr)), _p(out))
        return out

    def eigvec_point(self, U):
        R = np.zeros(self.nc * self.nc)
        self.L.or_eigvec_point(C.byref(self.cfg), _p(_f64(U)), _p(R))
        return R.reshape(self.nc, self.nc)

    def eigvec_avg(self, Ul, Ur):
        R = np.zeros(self.nc * self.nc)
        cb = np.zeros(1)
        self.L.or_eigvec_avg(C.byref(self.cfg), _p(_f64(Ul)), _p(_f64(Ur)), _p(R), _p(cb))
        return R.reshape(self.nc, self.nc), cb[0]

    def weno_mr(self, w5, chi=None, eps=None):
        chi = _f64(chi if chi is not None else self.pb.chi)
        return self.L.or_weno_mr(_p(_f64(w5)), _p(chi), float(self.pb.weno_eps if eps is None else eps))

    def weno_js(self, w5, eps=None):
        return self.L.or_weno_js(_p(_f64(w5)), float(self.pb.weno_eps if eps is None else eps))

    # ---- grid operators ----------------------------------------------------
    def _grid(self, a, fields):
        a = _f64(a)
        assert a.size == fields * self.pb.ncell, (a.shape, fields)
        return a

    def padded_shape(self):
        pb = self.pb
        return (pb.n[2] + 6 if pb.d == 3 else 1, pb.n[1] + 6, pb.n[0] + 6)

    def metrics(self, x, xdot=None):
        pb = self.pb
        x = self._grid(x, pb.d)
        xd = self._grid(xdot, pb.d) if xdot is not None else None
        M = np.zeros((pb.d * (pb.d + 1),) + self.padded_shape())
        self.L.or_metrics(C.byref(self.cfg), _p(x), _p(xd) if xd is not None else None, _p(M))
        return M

    def init_J(self, x):
        J = np.zeros(self.pb.shape)
        self.L.or_init_J(C.byref(self.cfg), _p(self._grid(x, self.pb.d)), _p(J))
        return J

    def rhs(self, JU, J, x, xdot):
        pb = self.pb
        dJU = np.zeros((pb.nc,) + pb.shape)
        dJ = np.zeros(pb.shape)
        self.L.or_rhs(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)),
                      _p(self._grid(x, pb.d)), _p(self._grid(xdot, pb.d)), _p(dJU), _p(dJ))
        return dJU, dJ

    def rhs_margins(self, JU, J, x, xdot):
        """Residual plus the per-node Y-decision margin in decades (see es_oracle.h)."""
        pb = self.pb
        dJU = np.zeros((pb.nc,) + pb.shape)
        dJ = np.zeros(pb.shape)
        mg = np.zeros(pb.shape)
        self.L.or_rhs_margins(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)),
                              _p(self._grid(x, pb.d)), _p(self._grid(xdot, pb.d)), _p(dJU), _p(dJ), _p(mg))
        return dJU, dJ, mg

    def rk_step(self, JU, J, x, xdot, dt):
        pb = self.pb
        JU = self._grid(JU, pb.nc).copy()
        J = self._grid(J, 1).copy()
        x = self._grid(x, pb.d).copy()
        self.L.or_rk_step(C.byref(self.cfg), _p(JU), _p(J), _p(x), _p(self._grid(xdot, pb.d)), float(dt))
        return JU, J, x

    def cfl_dt(self, JU, J, x):
        pb = self.pb
        return self.L.or_cfl_dt(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)),
                                _p(self._grid(x, pb.d)))

    def monitor(self, JU, J):
        pb = self.pb
        th = np.zeros(pb.shape)
        self.L.or_monitor(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)), _p(th))
        return th

    def schlieren(self, JU, J, x, psi1=30.0, psi2=150.0):
        pb = self.pb
        phi = np.zeros(pb.shape)
        self.L.or_schlieren(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)), _p(self._grid(x, pb.d)),
                            float(psi1), float(psi2), _p(phi))
        return phi

    def filter(self, theta):
        th = self._grid(theta, 1).copy()
        self.L.or_filter(C.byref(self.cfg), _p(th))
        return th

    def jacobi(self, x, theta):
        pb = self.pb
        out = np.zeros((pb.d,) + pb.shape)
        self.L.or_jacobi(C.byref(self.cfg), _p(self._grid(x, pb.d)), _p(self._grid(theta, 1)), _p(out))
        return out

    def limiter(self, x, xmu):
        pb = self.pb
        return self.L.or_limiter(C.byref(self.cfg), _p(self._grid(x, pb.d)), _p(self._grid(xmu, pb.d)))

    def mesh_redistribute(self, JU, J, x, dt_in=0.0):
        pb = self.pb
        xdot = np.zeros((pb.d,) + pb.shape)
        out = np.zeros(2)
        self.L.or_mesh_redistribute(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)),
                                    _p(self._grid(x, pb.d)), float(dt_in), _p(xdot), _p(out))
        return xdot, out[0], out[1]

    def entropy(self, JU, J, dJU=None, dJ=None):
        pb = self.pb
        out = np.zeros(2)
        self.L.or_entropy(C.byref(self.cfg), _p(self._grid(JU, pb.nc)), _p(self._grid(J, 1)),
                          _p(self._grid(dJU, pb.nc)) if dJU is not None else None,
                          _p(self._grid(dJ, 1)) if dJ is not None else None, _p(out))
        return out[0], out[1]
