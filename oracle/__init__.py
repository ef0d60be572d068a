"""Python view of the plain FP64 CPU oracle (``oracle/oracle.c``).

Test infrastructure only: the test suite, the smoke check and the CPU
baseline leg of ``bench.py`` load this module; the GPU library never does.
Every function here marshals numpy arrays into the C oracle and back; the
arithmetic lives in ``oracle.c`` and follows the paper (arXiv 2503.07526):
Sec. 2.2 Eq. (cor) and Appendix D Algorithms 1-2 for the correlator,
Sec. 2.3 for the stress tensor, heat flux and Green-Kubo integrals.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NOBS = 12  # U, K, T, sigma[6] (xx yy zz xy xz yz), q[3]


def build(force: bool = False) -> str:
    """Compiles ``oracle.c`` with gcc (OpenMP, no FMA contraction, so x86
    and Arm give the same rounding) into ``oracle/liboracle.so``."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, dp, ip = C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int64)
            L.orc_lj_brute.argtypes = [i64, dp, C.c_double, C.c_int, C.c_double, C.c_double,
                                       C.c_double, C.c_int, dp, dp, dp]
            L.orc_lj_cells.argtypes = [i64, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_int, dp, dp, dp]
            L.orc_lj_near_cutoff.argtypes = [i64, dp, C.c_double, C.c_double, C.c_double,
                                             C.POINTER(C.c_int32)]
            L.orc_observables.argtypes = [i64, C.c_double, dp, dp, dp, dp, dp]
            L.orc_observables.restype = None
            L.orc_corr_new.argtypes = [C.c_int, C.c_int, C.c_int, i64, i64, C.c_int]
            L.orc_corr_new.restype = C.c_void_p
            L.orc_corr_free.argtypes = [C.c_void_p]
            L.orc_corr_free.restype = None
            L.orc_corr_push.argtypes = [C.c_void_p, dp, dp]
            L.orc_corr_read.argtypes = [C.c_void_p, i64, dp, dp, i64]
            L.orc_corr_read.restype = i64
            L.orc_corr_raw.argtypes = [C.c_void_p, dp, ip, C.POINTER(C.c_int)]
            L.orc_corr_raw.restype = None
            L.orc_direct_corr.argtypes = [i64, dp, dp, i64, dp]
            L.orc_gk_trapz.argtypes = [i64, dp, dp, C.c_double, C.c_double, dp, dp]
            L.orc_md_new.argtypes = [i64, C.c_double, dp, dp, C.POINTER(C.c_int32), C.c_int, dp,
                                     C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int]
            L.orc_md_new.restype = C.c_void_p
            L.orc_md_free.argtypes = [C.c_void_p]
            L.orc_md_free.restype = None
            L.orc_md_step.argtypes = [C.c_void_p, i64, C.c_void_p, i64, C.c_void_p, i64, dp]
            L.orc_md_get.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp]
            L.orc_md_get.restype = None
            L.orc_md_scale_velocities.argtypes = [C.c_void_p, C.c_double]
            L.orc_md_scale_velocities.restype = None
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls (for timing)."""
    lib().orc_set_threads(int(n))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def lj_forces(r, L, *, rc=2.5, eps=1.0, sig=1.0, shift=True, method="cells", periodic=True):
    """Forces [3,n], per-particle potential energy [n] and virial [6,n]
    (xx yy zz xy xz yz) for positions r [3,n] (Sec. 2.3; readings R8-R10 of
    oracle.c)."""
    r = _f64(r)
    n = r.shape[1]
    F = np.zeros((3, n))
    e = np.zeros(n)
    W = np.zeros((6, n))
    if method == "brute":
        rc_ = lib().orc_lj_brute(n, _d(r), L, 1 if periodic else 0, eps, sig, rc, int(shift),
                                 _d(F), _d(e), _d(W))
    elif method == "cells":
        if not periodic:
            raise ValueError("link cells need a periodic box")
        rc_ = lib().orc_lj_cells(n, _d(r), L, eps, sig, rc, int(shift), _d(F), _d(e), _d(W))
    else:
        raise ValueError(method)
    if rc_ != 0:
        raise ValueError(f"oracle force call failed ({rc_})")
    return F, e, W


def near_cutoff_pairs(r, L, rc=2.5, band=1e-5):
    """Per atom, neighbours whose distance is within band of rc (test helper
    for reduced-precision forces: the truncated force jumps there)."""
    r = _f64(r)
    out = np.zeros(r.shape[1], dtype=np.int32)
    if lib().orc_lj_near_cutoff(r.shape[1], _d(r), L, rc, band, out.ctypes.data_as(C.POINTER(C.c_int32))) != 0:
        raise ValueError("near-cutoff count failed")
    return out


def observables(V, mass_of, v, epot, W):
    """[U, K, T, sigma(6), q(3)] of Sec. 2.3 from per-particle data."""
    out = np.zeros(NOBS)
    mass_of, v, epot, W = _f64(mass_of), _f64(v), _f64(epot), _f64(W)
    lib().orc_observables(v.shape[1], V, _d(mass_of), _d(v), _d(epot), _d(W), _d(out))
    return out


class Corr:
    """Multiple-tau correlator over ``ns`` series in groups of ``gs``
    (Appendix D, Algorithm 1 update / Algorithm 2 readout)."""

    def __init__(self, b, p, m, ns, gs=1, cross=False):
        self.b, self.p, self.m, self.ns, self.gs, self.cross = b, p, m, ns, gs, cross
        self.ng = ns // gs
        self._h = lib().orc_corr_new(b, p, m, ns, gs, int(cross))
        if not self._h:
            raise ValueError("invalid correlator parameters")

    def push(self, x, y=None):
        x = _f64(x).ravel()
        if x.size != self.ns:
            raise ValueError("x has the wrong number of series")
        if self.cross:
            y = _f64(y).ravel()
            rc = lib().orc_corr_push(self._h, _d(x), _d(y))
        else:
            rc = lib().orc_corr_push(self._h, _d(x), None)
        if rc != 0:
            raise ValueError("push failed")

    def read(self, g=0):
        cap = self.b * self.p
        t = np.zeros(cap)
        v = np.zeros(cap)
        n = lib().orc_corr_read(self._h, g, _d(t), _d(v), cap)
        return t[:n].copy(), v[:n].copy()

    def raw(self):
        vals = np.zeros((self.ng, self.b, self.p))
        cnt = np.zeros((self.b, self.p), dtype=np.int64)
        bu = C.c_int(0)
        lib().orc_corr_raw(self._h, _d(vals), cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(bu))
        return vals, cnt, bu.value

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.orc_corr_free(h)


def direct_corr(x, y, L):
    """Eq. (cor) of Sec. 2.2 at lags 0..L-1."""
    x, y = _f64(x).ravel(), _f64(y).ravel()
    out = np.zeros(L)
    if lib().orc_direct_corr(x.size, _d(x), _d(y), L, _d(out)) != 0:
        raise ValueError("L > S")
    return out


def gk_trapz(t, c, t_cut=np.inf, prefactor=1.0):
    """Trapezoid Green-Kubo integral of Sec. 2.3 up to t_cut; returns
    (integral, running integral at every t)."""
    t, c = _f64(t).ravel(), _f64(c).ravel()
    run = np.zeros(t.size)
    out = C.c_double(0.0)
    if lib().orc_gk_trapz(t.size, _d(t), _d(c), float(t_cut), float(prefactor), C.byref(out), _d(run)) != 0:
        raise ValueError("times must increase")
    return out.value, run


class MD:
    """Velocity-Verlet NVE run of a shifted-LJ system on a periodic cubic box
    (Sec. 1 integrator, Sec. 2.3 observables), pushing into oracle
    correlators after every step."""

    def __init__(self, r, v, L, *, types=None, masses=(1.0,), eps=1.0, sig=1.0, rc=2.5,
                 shift=True, dt=0.005, cells=True):
        r, v = _f64(r), _f64(v)
        self.n = r.shape[1]
        self.L = float(L)
        masses = _f64(masses).ravel()
        t = None
        if types is not None:
            self._types = np.ascontiguousarray(types, dtype=np.int32)
            t = self._types.ctypes.data_as(C.POINTER(C.c_int32))
        self._h = lib().orc_md_new(self.n, L, _d(r), _d(v), t, masses.size, _d(masses),
                                   eps, sig, rc, int(shift), dt, int(cells))
        if not self._h:
            raise ValueError("oracle md_new failed")

    def step(self, nsteps, cs=None, us=1, cv=None, uv=1, record=False):
        out = np.zeros((nsteps, NOBS)) if record else None
        rc = lib().orc_md_step(self._h, nsteps, cs._h if cs else None, us,
                               cv._h if cv else None, uv, _d(out) if record else None)
        if rc != 0:
            raise ValueError(f"oracle md_step failed ({rc})")
        return out

    def get(self):
        n = self.n
        r, v, F = np.zeros((3, n)), np.zeros((3, n)), np.zeros((3, n))
        e, W, obs = np.zeros(n), np.zeros((6, n)), np.zeros(NOBS)
        lib().orc_md_get(self._h, _d(r), _d(v), _d(F), _d(e), _d(W), _d(obs))
        return dict(r=r, v=v, F=F, epot=e, W=W, obs=obs)

    def scale_velocities(self, lam):
        lib().orc_md_scale_velocities(self._h, float(lam))

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.orc_md_free(h)
