"""ctypes binding of ``include/otf_md.h`` (argument marshalling only).

Every computation runs in ``libotfmd.so``.  If the library is missing the
import fails loudly: there is no CPU fallback.  Arrays may be numpy arrays
(host memory) or CUDA torch tensors (device memory); streams are torch
streams or raw ``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_lib

MD_OK, MD_EINVAL, MD_ENOMEM, MD_ECUDA, MD_ESTATE, MD_ETIMEOUT, MD_ECAP = 0, -1, -2, -3, -4, -5, -6
MD_PREC_FP64, MD_PREC_MIXED = 0, 1
MD_MEM_HOST, MD_MEM_DEVICE = 0, 1
MD_CORR_STRESS, MD_CORR_HEATFLUX, MD_CORR_VACF, MD_CORR_MASSFLUX = 0, 1, 2, 3
MD_PAIR_VERLET, MD_PAIR_CELLS, MD_PAIR_TILES = 0, 1, 2
MD_POT_LJ, MD_POT_BUCK_EWALD = 0, 1
MD_K_NAMES = ("integrate", "rebuild", "pair", "reduce", "vacf", "spme")
MD_NKCLASS = 6
KE_EV_ANGSTROM = 14.399645478425668  # e^2 / (4 pi eps0) in eV Angstrom

_ERRNAMES = {MD_EINVAL: "MD_EINVAL", MD_ENOMEM: "MD_ENOMEM", MD_ECUDA: "MD_ECUDA", MD_ESTATE: "MD_ESTATE",
             MD_ETIMEOUT: "MD_ETIMEOUT", MD_ECAP: "MD_ECAP"}


class MdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class corr_spec(C.Structure):
    _fields_ = [("b", C.c_int32), ("p", C.c_int32), ("m", C.c_int32), ("u", C.c_int32)]


class md_params(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double), ("eps", C.c_double), ("sigma", C.c_double),
                ("rc", C.c_double), ("shift", C.c_int32), ("ntypes", C.c_int32), ("mass", C.c_double * 8),
                ("dt", C.c_double), ("precision", C.c_int32), ("pair_mode", C.c_int32), ("skin", C.c_double),
                ("max_neighbors", C.c_int32), ("use_graph", C.c_int32), ("autotune", C.c_int32), ("stress", corr_spec),
                ("heatflux", corr_spec), ("vacf", corr_spec), ("list_build", C.c_int32),
                ("potential", C.c_int32), ("charge", C.c_double * 8), ("buck_A", C.c_double), ("buck_rho", C.c_double),
                ("buck_C", C.c_double), ("coulomb", C.c_double), ("ewald_alpha", C.c_double), ("mesh", C.c_int32),
                ("order", C.c_int32), ("flux_species", C.c_int32), ("massflux", corr_spec),
                ("window_slots", C.c_int32)]


class md_system(C.Structure):
    _fields_ = [("r", C.c_void_p), ("v", C.c_void_p), ("type", C.c_void_p), ("mem", C.c_int32)]


class md_replica(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double), ("r", C.c_void_p), ("v", C.c_void_p), ("type", C.c_void_p)]


class md_config(C.Structure):
    _fields_ = [("replicas", C.c_int32), ("pair_threads", C.c_int32), ("build_warps", C.c_int32),
                ("max_neighbors", C.c_int32), ("atoms", C.c_int64), ("cells", C.c_int64),
                ("build_kind", C.c_int32), ("vacf_input_bytes", C.c_int64), ("tiles", C.c_int64),
                ("window_capacity", C.c_int32), ("tile_threads", C.c_int32), ("tile_extent", C.c_int32 * 3)]


class gk_tail_rule(C.Structure):
    _fields_ = [("T_min", C.c_double), ("T_max", C.c_double), ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("net_error", C.c_double * 2), ("short_coeff", C.c_double * 2)]


class md_obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("U", C.c_double), ("K", C.c_double), ("T", C.c_double),
                ("sigma", C.c_double * 6), ("q", C.c_double * 3), ("T_mean", C.c_double),
                ("rebuilds", C.c_int64), ("j", C.c_double * 3)]


class corr_params(C.Structure):
    _fields_ = [("b", C.c_int32), ("p", C.c_int32), ("m", C.c_int32), ("cross", C.c_int32),
                ("nseries", C.c_int64), ("group_size", C.c_int64), ("precision", C.c_int32),
                ("dt_unit", C.c_double)]


class mlp_params(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("width", C.c_int32), ("depth", C.c_int32), ("n_out", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("weight_decay", C.c_float), ("seed", C.c_uint64)]


_lib = None


def lib(build: bool = False):
    """The loaded ``libotfmd.so`` (built first when ``build`` is set)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_lib.build() if build else build_lib.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() or "
                          "python -m paper_2503_07526_gb300.build_lib")
    L = C.CDLL(path)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
    sig = {
        "md_init": [C.POINTER(md_params), C.POINTER(md_system), vp, C.POINTER(vp)],
        "md_init_replicas": [C.POINTER(md_params), C.POINTER(md_replica), i32, i32, vp, C.POINTER(vp)],
        "md_replica_observables": [vp, i32, C.POINTER(md_obs)],
        "md_replica_observables_all": [vp, vp, i32],
        "md_replica_scale_velocities": [vp, dp],
        "md_get_config": [vp, C.POINTER(md_config)],
        "md_step": [vp, i64],
        "md_observables": [vp, C.POINTER(md_obs)],
        "md_get_particles": [vp, vp, vp, vp, vp, vp, i32],
        "md_scale_velocities": [vp, C.c_double],
        "md_reset_correlators": [vp],
        "md_corr": [vp, i32, C.POINTER(vp)],
        "md_set_timing": [vp, i32],
        "md_kernel_times": [vp, dp, C.POINTER(C.c_int64)],
        "corr_create": [C.POINTER(corr_params), vp, C.POINTER(vp)],
        "corr_push": [vp, vp, vp, i64, i32],
        "corr_read": [vp, i64, dp, dp, i64, C.POINTER(C.c_int64)],
        "corr_raw": [vp, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)],
        "corr_pushes": [vp, C.POINTER(C.c_int64)],
        "corr_reset": [vp],
        "gk_integrate": [dp, dp, i64, C.c_double, C.c_double, dp, dp],
        "md_observables_noalloc": [i64, C.c_double, vp, vp, vp, vp, vp, vp],
        "md_fp32_peak": [i32, i64, i32, vp, dp, dp, C.POINTER(C.c_int32)],
        "mlp_set_wait_limit": [vp, i64],
        "gk_tail_box": [dp, dp, i64, C.POINTER(gk_tail_rule)],
        "gk_tail_rms_rel": [dp, dp, dp, i64, dp],
        "gk_tail_choose": [C.POINTER(gk_tail_rule), dp, dp, dp, dp, dp, i64, dp, vp],
        "mlp_create": [C.POINTER(mlp_params), vp, C.POINTER(vp)],
        "mlp_param_count": [vp, C.POINTER(C.c_int64)],
        "mlp_get_params": [vp, vp, i64, i32],
        "mlp_set_params": [vp, vp, i64, i32],
        "mlp_set_scaler": [vp, vp, vp, vp, vp],
        "mlp_fit_scaler": [vp, vp, vp, i64],
        "mlp_forward": [vp, vp, i64, vp, i32],
        "mlp_loss_grad": [vp, vp, vp, i64, dp, vp, i32],
        "mlp_adam_step": [vp, vp, i32],
        "mlp_train": [vp, vp, vp, i64, i32, vp, C.c_uint64, dp, i32],
        "gk_tail_features": [dp, dp, i64, i64, dp, dp, dp, vp],
        "corr_read_rows": [vp, i64, i64, i64, dp, dp, i64, C.POINTER(C.c_int64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.md_free.argtypes = [vp]
    L.md_free.restype = None
    L.corr_free.argtypes = [vp]
    L.corr_free.restype = None
    L.mlp_free.argtypes = [vp]
    L.mlp_free.restype = None
    L.md_last_error.argtypes = []
    L.md_last_error.restype = C.c_char_p
    _lib = L
    return L


EXPORTS = ("md_init", "md_step", "md_observables", "md_get_particles", "md_scale_velocities", "md_reset_correlators",
           "md_corr", "md_set_timing", "md_kernel_times", "md_free", "corr_create", "corr_push", "corr_read",
           "corr_raw", "corr_pushes", "corr_reset", "corr_free", "gk_integrate", "md_last_error",
           "md_observables_noalloc", "md_init_replicas", "md_replica_observables", "md_replica_scale_velocities",
           "md_get_config", "md_replica_observables_all", "mlp_create", "mlp_param_count", "mlp_get_params",
           "mlp_set_params", "mlp_set_scaler", "mlp_fit_scaler", "mlp_forward", "mlp_loss_grad", "mlp_adam_step",
           "mlp_train", "mlp_free", "gk_tail_features", "corr_read_rows", "md_fp32_peak", "mlp_set_wait_limit", "gk_tail_box", "gk_tail_rms_rel",
           "gk_tail_choose")


def _check(rc):
    if rc != MD_OK:
        raise MdError(rc, lib().md_last_error().decode(errors="replace"))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a, dtype, mem_hint=None):
    """(pointer, mem flag, keep-alive) of a numpy array or CUDA torch tensor."""
    try:
        import torch

        if isinstance(a, torch.Tensor):
            if a.dtype != dtype["torch"]:
                raise TypeError(f"expected {dtype['torch']}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), (MD_MEM_DEVICE if a.is_cuda else MD_MEM_HOST), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype["np"])
    return arr.ctypes.data, MD_MEM_HOST, arr


F64 = {"np": np.float64, "torch": None}
F32 = {"np": np.float32, "torch": None}
I32 = {"np": np.int32, "torch": None}


def _init_dtypes():
    try:
        import torch

        F64["torch"] = torch.float64
        F32["torch"] = torch.float32
        I32["torch"] = torch.int32
    except ImportError:
        pass


_init_dtypes()


def make_params(n, box, *, eps=1.0, sigma=1.0, rc=2.5, shift=True, masses=(1.0,), dt=0.005,
                precision=MD_PREC_FP64, pair_mode=MD_PAIR_VERLET, skin=0.3, max_neighbors=0, use_graph=True,
                autotune=False, stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=(8, 16, 2, 1), list_build=0,
                potential=MD_POT_LJ, charges=(), buckingham=(0.0, 1.0, 0.0), coulomb=KE_EV_ANGSTROM, ewald_alpha=0.0,
                mesh=0, order=8, flux_species=0, massflux=None, window_slots=0):
    p = md_params()
    p.n, p.box, p.eps, p.sigma, p.rc, p.shift = int(n), float(box), eps, sigma, rc, int(bool(shift))
    p.ntypes = len(masses)
    for t, m in enumerate(masses):
        p.mass[t] = float(m)
    p.dt, p.precision, p.pair_mode, p.skin = dt, int(precision), int(pair_mode), float(skin)
    p.max_neighbors, p.use_graph, p.autotune = int(max_neighbors), int(bool(use_graph)), int(bool(autotune))
    p.list_build = int(list_build)
    p.potential = int(potential)
    for t, q in enumerate(charges):
        p.charge[t] = float(q)
    p.buck_A, p.buck_rho, p.buck_C = (float(x) for x in buckingham)
    p.coulomb, p.ewald_alpha, p.mesh, p.order = float(coulomb), float(ewald_alpha), int(mesh), int(order)
    p.flux_species = int(flux_species)
    p.window_slots = int(window_slots)
    for name, spec in (("stress", stress), ("heatflux", heatflux), ("vacf", vacf), ("massflux", massflux)):
        cs = getattr(p, name)
        cs.b, cs.p, cs.m, cs.u = spec if spec is not None else (1, 2, 1, 0)
    return p


class Corr:
    """A correlator handle (free-standing or borrowed from a System)."""

    def __init__(self, handle, owned, nseries, ngroups, cross, b, p, keep=None):
        self._h, self._owned, self.nseries, self.ngroups, self.cross = handle, owned, nseries, ngroups, cross
        self.b, self.p = b, p
        self._keep = keep

    @classmethod
    def create(cls, b, p, m, nseries, group_size=1, cross=False, precision=MD_PREC_FP64, dt_unit=1.0,
               stream=None):
        cp = corr_params(b, p, m, int(bool(cross)), nseries, group_size, precision, dt_unit)
        h = C.c_void_p()
        _check(lib().corr_create(C.byref(cp), _stream_ptr(stream), C.byref(h)))
        return cls(h, True, nseries, nseries // group_size, bool(cross), b, p)

    def push(self, x, y=None):
        px, mem, kx = _ptr(x, F64)
        py, ky = None, None
        if self.cross:
            py, memy, ky = _ptr(y, F64)
            if memy != mem:
                raise ValueError("x and y must live in the same memory")
        _check(lib().corr_push(self._h, px, py, self.nseries, mem))

    def read(self, group=-1):
        cap = self.b * self.p
        t = np.zeros(cap)
        v = np.zeros(cap)
        n = C.c_int64(0)
        dp = C.POINTER(C.c_double)
        _check(lib().corr_read(self._h, group, t.ctypes.data_as(dp), v.ctypes.data_as(dp), cap, C.byref(n)))
        return t[: n.value].copy(), v[: n.value].copy()

    def read_rows(self, g0, rows, avg=1):
        """(times [n], values [rows, n]): row i is the mean of groups
        g0 + i*avg ... g0 + i*avg + avg - 1 on the readout grid."""
        cap = self.b * self.p
        t = np.zeros(cap)
        v = np.zeros((rows, cap))
        n = C.c_int64(0)
        dp = C.POINTER(C.c_double)
        _check(lib().corr_read_rows(self._h, int(g0), int(rows), int(avg), t.ctypes.data_as(dp),
                                    v.ctypes.data_as(dp), cap, C.byref(n)))
        return t[: n.value].copy(), v[:, : n.value].copy()

    def raw(self):
        vals = np.zeros((self.ngroups, self.b, self.p))
        cnt = np.zeros((self.b, self.p), dtype=np.int64)
        used = C.c_int32(0)
        _check(lib().corr_raw(self._h, vals.ctypes.data_as(C.POINTER(C.c_double)),
                              cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(used)))
        return vals, cnt, used.value

    def pushes(self):
        n = C.c_int64(0)
        _check(lib().corr_pushes(self._h, C.byref(n)))
        return n.value

    def reset(self):
        _check(lib().corr_reset(self._h))

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h and self._owned and _lib is not None:
            _lib.corr_free(h)

    __del__ = close


class System:
    """An MD system on the GPU behind md_init / md_step / md_free."""

    def __init__(self, params: md_params, r=None, v=None, types=None, stream=None, replicas=None):
        self.params = params
        if replicas is not None:
            self._init_replicas(params, replicas, stream)
            return
        self.n = params.n
        self.nrep = 1
        pr, mem, kr = _ptr(r, F64)
        pv, memv, kv = _ptr(v, F64)
        pt, kt = None, None
        if types is not None:
            pt, memt, kt = _ptr(types, I32)
            if memt != mem:
                raise ValueError("r, v and types must live in the same memory")
        if memv != mem:
            raise ValueError("r and v must live in the same memory")
        sysd = md_system(pr, pv, pt, mem)
        h = C.c_void_p()
        self.stream = _stream_ptr(stream)
        _check(lib().md_init(C.byref(params), C.byref(sysd), self.stream, C.byref(h)))
        self._h = h

    def _init_replicas(self, params, replicas, stream):
        """replicas: list of dicts with r [3,n], v [3,n], box and optional types
        (numpy arrays or CUDA tensors, all in the same memory)."""
        arr = (md_replica * len(replicas))()
        keep, mems = [], set()
        for k, rp in enumerate(replicas):
            pr, mem, kr = _ptr(rp["r"], F64)
            pv, memv, kv = _ptr(rp["v"], F64)
            pt, kt = None, None
            if rp.get("types") is not None:
                pt, memt, kt = _ptr(rp["types"], I32)
                mems.add(memt)
            mems |= {mem, memv}
            keep += [kr, kv, kt]
            n = int(np.asarray(rp["r"].shape)[1]) if hasattr(rp["r"], "shape") else len(rp["r"][0])
            arr[k] = md_replica(n, float(rp["box"]), pr, pv, pt)
        if len(mems) != 1:
            raise ValueError("all replica arrays must live in the same memory")
        h = C.c_void_p()
        self.stream = _stream_ptr(stream)
        _check(lib().md_init_replicas(C.byref(params), arr, len(replicas), mems.pop(), self.stream, C.byref(h)))
        self._h = h
        self.nrep = len(replicas)
        self.n = sum(arr[k].n for k in range(self.nrep))

    def replica_observables(self, r):
        o = md_obs()
        _check(lib().md_replica_observables(self._h, int(r), C.byref(o)))
        return dict(step=o.step, U=o.U, K=o.K, T=o.T, sigma=np.array(o.sigma[:]), q=np.array(o.q[:]),
                    T_mean=o.T_mean, rebuilds=o.rebuilds, j=np.array(o.j[:]))

    def replica_observables_all(self):
        """Every replica's observables in one device read: dict of arrays
        (step and rebuilds are scalars)."""
        arr = (md_obs * self.nrep)()
        _check(lib().md_replica_observables_all(self._h, arr, self.nrep))
        return dict(step=arr[0].step, rebuilds=arr[0].rebuilds,
                    U=np.array([o.U for o in arr]), K=np.array([o.K for o in arr]), T=np.array([o.T for o in arr]),
                    sigma=np.array([o.sigma[:] for o in arr]), q=np.array([o.q[:] for o in arr]),
                    T_mean=np.array([o.T_mean for o in arr]), j=np.array([o.j[:] for o in arr]))

    def replica_scale_velocities(self, lams):
        lam = np.ascontiguousarray(lams, dtype=np.float64)
        _check(lib().md_replica_scale_velocities(self._h, lam.ctypes.data_as(C.POINTER(C.c_double))))

    def config(self):
        c = md_config()
        _check(lib().md_get_config(self._h, C.byref(c)))
        return dict(replicas=c.replicas, pair_threads=c.pair_threads, build_warps=c.build_warps,
                    build_kind=c.build_kind,
                    max_neighbors=c.max_neighbors, atoms=c.atoms, cells=c.cells,
                    vacf_input_bytes=c.vacf_input_bytes, tiles=c.tiles, window_capacity=c.window_capacity,
                    tile_threads=c.tile_threads, tile_extent=tuple(c.tile_extent))

    def step(self, nsteps):
        _check(lib().md_step(self._h, int(nsteps)))

    def observables(self):
        o = md_obs()
        _check(lib().md_observables(self._h, C.byref(o)))
        return dict(step=o.step, U=o.U, K=o.K, T=o.T, sigma=np.array(o.sigma[:]), q=np.array(o.q[:]),
                    T_mean=o.T_mean, rebuilds=o.rebuilds, j=np.array(o.j[:]))

    def particles(self):
        n = self.n
        r, v, F = np.zeros((3, n)), np.zeros((3, n)), np.zeros((3, n))
        e, W = np.zeros(n), np.zeros((6, n))
        _check(lib().md_get_particles(self._h, r.ctypes.data, v.ctypes.data, F.ctypes.data, e.ctypes.data,
                                      W.ctypes.data, MD_MEM_HOST))
        return dict(r=r, v=v, F=F, epot=e, W=W)

    def particles_device(self, r=None, v=None, F=None, epot=None, W=None):
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(lib().md_get_particles(self._h, ptr(r), ptr(v), ptr(F), ptr(epot), ptr(W), MD_MEM_DEVICE))

    def scale_velocities(self, lam):
        _check(lib().md_scale_velocities(self._h, float(lam)))

    def reset_correlators(self):
        _check(lib().md_reset_correlators(self._h))

    def corr(self, which):
        h = C.c_void_p()
        _check(lib().md_corr(self._h, int(which), C.byref(h)))
        spec = (self.params.stress, self.params.heatflux, self.params.vacf, self.params.massflux)[which]
        if which == MD_CORR_VACF:
            ns, ng = 3 * self.n, 3
        elif which == MD_CORR_MASSFLUX:
            ns, ng = 6 * self.nrep, 6 * self.nrep
        else:
            ns, ng = 3 * self.nrep, 3 * self.nrep
        return Corr(h, False, ns, ng, which == MD_CORR_MASSFLUX, spec.b, spec.p, keep=self)

    def set_timing(self, on=True):
        _check(lib().md_set_timing(self._h, int(bool(on))))

    def kernel_times(self):
        ms = np.zeros(MD_NKCLASS)
        nl = np.zeros(MD_NKCLASS, dtype=np.int64)
        _check(lib().md_kernel_times(self._h, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                     nl.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(MD_K_NAMES)}

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.md_free(h)

    __del__ = close


def gk_integrate(t, c, t_cut=float("inf"), prefactor=1.0):
    """(integral, running integral) by the library's trapezoid rule."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    run = np.zeros(t.size)
    out = C.c_double(0.0)
    dp = C.POINTER(C.c_double)
    _check(lib().gk_integrate(t.ctypes.data_as(dp), c.ctypes.data_as(dp), t.size, float(t_cut), float(prefactor),
                              C.byref(out), run.ctypes.data_as(dp)))
    return out.value, run


def fp32_peak(paired=False, iters=2048, reps=5, stream=None):
    """md_fp32_peak: (flops per launch, device ms per launch, SM count) of
    the FMA-chain kernel (scalar or paired f32x2 FMAs)."""
    fl, ms, sms = C.c_double(0.0), C.c_double(0.0), C.c_int32(0)
    _check(lib().md_fp32_peak(int(bool(paired)), int(iters), int(reps), _stream_ptr(stream), C.byref(fl),
                              C.byref(ms), C.byref(sms)))
    return fl.value, ms.value, sms.value


def observables_noalloc(volume, v, epot, W, mass_of, obs, stream=None):
    """md_observables_noalloc on CUDA tensors (float64): v [3,n], epot [n],
    W [6,n], mass_of [n] in, obs [12] out; enqueued on the stream."""
    n = v.shape[1]
    _check(lib().md_observables_noalloc(n, float(volume), v.data_ptr(), epot.data_ptr(), W.data_ptr(),
                                        mass_of.data_ptr(), obs.data_ptr(), _stream_ptr(stream)))


class MLP:
    """The learned-tail network behind mlp_create / mlp_free (tensor-core
    bfloat16 products, FP32 master weights, Adam)."""

    def __init__(self, n_in, n_out=2, *, width=128, depth=3, batch=256, lr=1e-3, beta1=0.9, beta2=0.999,
                 eps=1e-8, weight_decay=0.0, seed=1, stream=None):
        self.p = mlp_params(n_in, width, depth, n_out, batch, lr, beta1, beta2, eps, weight_decay, seed)
        self.n_in, self.n_out, self.batch = n_in, n_out, batch
        h = C.c_void_p()
        _check(lib().mlp_create(C.byref(self.p), _stream_ptr(stream), C.byref(h)))
        self._h = h
        n = C.c_int64(0)
        _check(lib().mlp_param_count(self._h, C.byref(n)))
        self.nparams = n.value
        self.dims = (n_in,) + (width,) * depth + (n_out,)

    # flat parameter order: per layer W [out, in] then b [out]
    def get_flat(self):
        f = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().mlp_get_params(self._h, f.ctypes.data, self.nparams, MD_MEM_HOST))
        return f

    def set_flat(self, flat):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        if f.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {f.size}")
        _check(lib().mlp_set_params(self._h, f.ctypes.data, self.nparams, MD_MEM_HOST))

    def unflatten(self, flat):
        out, k = [], 0
        for fi, fo in zip(self.dims[:-1], self.dims[1:]):
            W = np.asarray(flat[k:k + fo * fi], dtype=np.float64).reshape(fo, fi)
            k += fo * fi
            b = np.asarray(flat[k:k + fo], dtype=np.float64)
            k += fo
            out.append((W, b))
        return out

    @staticmethod
    def flatten(params):
        return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)

    def get_params(self):
        return self.unflatten(self.get_flat())

    def set_params(self, params):
        self.set_flat(self.flatten(params))

    def set_scaler(self, x_mean, x_std, y_mean, y_std):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (x_mean, x_std, y_mean, y_std)]
        _check(lib().mlp_set_scaler(self._h, *[v.ctypes.data for v in a]))

    def fit_scaler(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        _check(lib().mlp_fit_scaler(self._h, X.ctypes.data, T.ctypes.data, X.shape[0]))

    def forward(self, X):
        px, mem, kx = _ptr(X, F32)
        rows = X.shape[0]
        if mem == MD_MEM_HOST:
            Y = np.zeros((rows, self.n_out), dtype=np.float32)
            py = Y.ctypes.data
        else:
            import torch

            Y = torch.zeros((rows, self.n_out), dtype=torch.float32, device=X.device)
            py = Y.data_ptr()
        _check(lib().mlp_forward(self._h, px, rows, py, mem))
        return Y

    def set_wait_limit(self, ns):
        _check(lib().mlp_set_wait_limit(self._h, int(ns)))

    def loss_grad(self, X, T):
        px, mem, kx = _ptr(X, F32)
        pt, memt, kt = _ptr(T, F32)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = C.c_double(0.0)
        if mem != MD_MEM_HOST:
            raise ValueError("loss_grad takes host arrays")
        _check(lib().mlp_loss_grad(self._h, px, pt, X.shape[0], C.byref(loss), g.ctypes.data, mem))
        return loss.value, g

    def adam_step(self, grad=None):
        if grad is None:
            _check(lib().mlp_adam_step(self._h, None, MD_MEM_HOST))
        else:
            g = np.ascontiguousarray(grad, dtype=np.float32)
            _check(lib().mlp_adam_step(self._h, g.ctypes.data, MD_MEM_HOST))

    def train(self, X, T, epochs, order=None, shuffle_seed=1):
        px, mem, kx = _ptr(X, F32)
        pt, memt, kt = _ptr(T, F32)
        if mem != memt:
            raise ValueError("X and T must live in the same memory")
        rows = X.shape[0]
        po, ko = None, None
        if order is not None:
            ko = np.ascontiguousarray(order, dtype=np.int64)
            if ko.shape != (epochs, rows):
                raise ValueError("order must be [epochs, rows]")
            po = ko.ctypes.data
        hist = np.zeros(max(epochs, 1))
        _check(lib().mlp_train(self._h, px, pt, rows, int(epochs), po, int(shuffle_seed),
                               hist.ctypes.data_as(C.POINTER(C.c_double)), mem))
        return hist[:epochs]

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.mlp_free(h)

    __del__ = close


def _f64c(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if n is None else np.ascontiguousarray(np.broadcast_to(a, (n,)))


def gk_tail_box(temperature, density):
    """The temperature-density box of training runs (a gk_tail_rule with
    only the box set)."""
    T, rho = _f64c(temperature), _f64c(density)
    rule = gk_tail_rule()
    dp = C.POINTER(C.c_double)
    _check(lib().gk_tail_box(T.ctypes.data_as(dp), rho.ctypes.data_as(dp), T.size, C.byref(rule)))
    return rule


def gk_tail_rms_rel(a, b, w=None):
    """sqrt(mean(((a - b) / b)^2 w)) (w = None: weights 1)."""
    a, b = _f64c(a).ravel(), _f64c(b).ravel()
    dp = C.POINTER(C.c_double)
    wp = None if w is None else _f64c(w).ravel()
    out = C.c_double(0.0)
    _check(lib().gk_tail_rms_rel(a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                                 None if wp is None else wp.ctypes.data_as(dp), a.size, C.byref(out)))
    return out.value


def gk_tail_choose(rule, temperature, density, steps, net, own):
    """(out [nruns, 2], used [nruns, 2] bool): the network's (eta, kappa)
    or the runs' own integrals, per the rule."""
    net, own = _f64c(net).reshape(-1, 2), _f64c(own).reshape(-1, 2)
    nr = net.shape[0]
    T, rho, st = _f64c(temperature, nr), _f64c(density, nr), _f64c(steps, nr)
    out = np.zeros((nr, 2))
    used = np.zeros((nr, 2), dtype=np.int32)
    dp = C.POINTER(C.c_double)
    _check(lib().gk_tail_choose(C.byref(rule), T.ctypes.data_as(dp), rho.ctypes.data_as(dp), st.ctypes.data_as(dp),
                                net.ctypes.data_as(dp), own.ctypes.data_as(dp), nr, out.ctypes.data_as(dp),
                                used.ctypes.data))
    return out, used.astype(bool)


def gk_tail_features(c_sigma, c_q, volume, temperature, density):
    """Features [nruns, 132] of the learned tail from per-run readouts
    c_sigma, c_q [nruns, >= 64] (float32)."""
    cs = np.ascontiguousarray(np.atleast_2d(c_sigma), dtype=np.float64)
    cq = np.ascontiguousarray(np.atleast_2d(c_q), dtype=np.float64)
    if cs.shape != cq.shape:
        raise ValueError("c_sigma and c_q must have the same shape")
    nr = cs.shape[0]
    V, T, rho = (np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (nr,)))
                 for a in (volume, temperature, density))
    out = np.zeros((nr, 132), dtype=np.float32)
    dp = C.POINTER(C.c_double)
    _check(lib().gk_tail_features(cs.ctypes.data_as(dp), cq.ctypes.data_as(dp), cs.shape[1], nr,
                                  V.ctypes.data_as(dp), T.ctypes.data_as(dp), rho.ctypes.data_as(dp), out.ctypes.data))
    return out
