"""ctypes binding of the C ABI in include/stdg.h (argument marshalling only).

Every function of the header is exposed under its own name; ``Solver`` is a thin
object wrapper that owns one context.  All arithmetic runs in libstdg.so: if the
library is missing this module raises instead of falling back to anything else.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libstdg.so")

STDG_OK, STDG_EINVAL, STDG_EMESH, STDG_ENOMEM, STDG_ECUDA, STDG_ENOTCONV, STDG_ESTATE = 0, -1, -2, -3, -4, -5, -6
STDG_ENONFINITE = -7
STDG_EENERGY = -8
SCHEME = {"cn": 0, "stdg": 1}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_fp32": 1}


class stdg_options(C.Structure):
    _fields_ = [("p", C.c_int), ("p_gamma", C.c_int), ("scheme", C.c_int), ("precision", C.c_int),
                ("rel_tol", C.c_double), ("max_iters", C.c_int), ("gmres_restart", C.c_int),
                ("inner_tol", C.c_double), ("use_graph", C.c_int), ("preconditioner", C.c_int)]


class stdg_stats(C.Structure):
    _fields_ = [("iters_total", C.c_int), ("iters_max", C.c_int), ("refinements", C.c_int),
                ("final_rel_res", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stdg_tuning(C.Structure):
    _fields_ = [("face_warps_per_block", C.c_int), ("face_blocks_per_sm", C.c_int), ("face_register_cap", C.c_int),
                ("pre2_warps_per_block", C.c_int),
                ("mma_ctas_per_sm", C.c_int), ("face_ms", C.c_double), ("pre2_ms", C.c_double), ("candidates", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)

SIGNATURES = {
    "stdg_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(stdg_options), _P]),
    "stdg_destroy": (None, [_P]),
    "stdg_last_error": (C.c_char_p, [_P]),
    "stdg_set_mesh": (C.c_int, [_P, C.c_int64, _D, C.c_int64, _I32, _D]),
    "stdg_set_material": (C.c_int, [_P, _D, _D, _D]),
    "stdg_set_shots": (C.c_int, [_P, C.c_int]),
    "stdg_set_state": (C.c_int, [_P, C.c_int, _D, _D]),
    "stdg_get_state": (C.c_int, [_P, C.c_int, _D, _D]),
    "stdg_set_plane_wave": (C.c_int, [_P, C.c_int, C.c_int, _D, _D, C.c_double, C.c_double]),
    "stdg_set_sources": (C.c_int, [_P, C.c_int, _D, _D, C.c_double, C.c_double, C.c_double]),
    "stdg_set_point_sources": (C.c_int, [_P, C.c_int, C.c_int, _D, _D, C.c_double, C.c_double, C.c_double]),
    "stdg_set_receivers": (C.c_int, [_P, C.c_int, _D]),
    "stdg_step": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(stdg_stats)]),
    "stdg_get_time": (C.c_int, [_P, _D]),
    "stdg_set_time": (C.c_int, [_P, C.c_double]),
    "stdg_energy": (C.c_int, [_P, _D]),
    "stdg_set_energy_check": (C.c_int, [_P, C.c_int, C.c_double]),
    "stdg_set_time_scale": (C.c_int, [_P, _D]),
    "stdg_set_pre2_storage": (C.c_int, [_P, C.c_int]),
    "stdg_read_receivers": (C.c_int, [_P, _D, C.c_int64]),
    "stdg_apply_operator": (C.c_int, [_P, C.c_double, _D, _D]),
    "stdg_apply_operator_device": (C.c_int, [_P, C.c_double, _P, _P, C.c_int]),
    "stdg_query": (C.c_int, [_P, C.c_int, _I64]),
    "stdg_get_faces": (C.c_int, [_P, _I32, _I32]),
    "stdg_mesh_faces": (C.c_int, [C.c_int, C.c_int64, _D, C.c_int64, _I32, _D, _I64, _I32, _I32]),
    "stdg_locate_points": (C.c_int, [C.c_int, C.c_int64, _D, C.c_int64, _I32, _D, C.c_int64, _D, _I64]),
    "stdg_reference_tables": (C.c_int, [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, _D, _D]),
    "stdg_time_operator": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, _D]),
    "stdg_time_kernel": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, C.c_int, _D]),
    "stdg_misfit_grad": (C.c_int, [_P, C.c_double, C.c_int, _D, C.c_int, _D, _D, _D, _D, _D, C.POINTER(stdg_stats)]),
    "stdg_apply_preconditioner": (C.c_int, [_P, C.c_double, _D, _D]),
    "stdg_residual_noalloc": (C.c_int, [_P, C.c_double, _P, _P, _P, _P]),
    "stdg_inject_wait_error": (C.c_int, [_P]),
    "stdg_apply_preconditioner_device": (C.c_int, [_P, C.c_double, _P, _P, C.c_int]),
    "stdg_measure_fma_peak": (C.c_int, [C.c_int, _D]),
    "stdg_autotune": (C.c_int, [_P, C.c_double, C.POINTER(stdg_tuning)]),
}

_lib = None


def load(path=None):
    """Load libstdg.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libstdg.so not found at %s: run paper_1802_04516_gb300.build.build()" % p)
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def exported_symbols():
    return list(SIGNATURES)


class StdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("stdg error %d: %s" % (code, msg))
        self.code = code


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _need(a, n, name):
    """The library reads (or writes) exactly n values through the pointer: check first."""
    if a.size != n:
        raise ValueError("%s has %d values, the context needs %d" % (name, a.size, n))
    return a


def _out(a, n, name):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("%s must be a C-contiguous float64 array" % name)
    return _need(a, n, name)


def mesh_faces(xyz, elem_vert, period=None):
    """Face table (l(j), r(j), r = -1 on the boundary) of a mesh, built on the host by the
    library's mesh code with no context and no GPU.  Raises StdgError on a bad mesh."""
    lib = load()
    xyz = _f64(xyz)
    ev = np.ascontiguousarray(elem_vert, dtype=np.int32)
    dim = ev.shape[1] - 1
    per = None if period is None else _f64(period)
    per_p = None if per is None else _d(per)
    n = C.c_int64(0)
    args = (dim, xyz.shape[0], _d(xyz), ev.shape[0], ev.ctypes.data_as(_I32), per_p)
    rc = lib.stdg_mesh_faces(*args, C.byref(n), None, None)
    if rc != 0:
        raise StdgError(rc, "stdg_mesh_faces")
    fl = np.zeros(n.value, dtype=np.int32)
    fr = np.zeros(n.value, dtype=np.int32)
    rc = lib.stdg_mesh_faces(*args, C.byref(n), fl.ctypes.data_as(_I32), fr.ctypes.data_as(_I32))
    if rc != 0:
        raise StdgError(rc, "stdg_mesh_faces")
    return fl, fr


def locate_points(xyz, elem_vert, points, period=None):
    """Element of each point (-1 outside), located on the host by the library's code for
    sources and receivers, with no context and no GPU.  Raises StdgError on a bad mesh."""
    lib = load()
    xyz = _f64(xyz)
    ev = np.ascontiguousarray(elem_vert, dtype=np.int32)
    dim = ev.shape[1] - 1
    pts = _need(_f64(np.atleast_2d(points)), np.atleast_2d(points).shape[0] * dim, "points")
    per = None if period is None else _need(_f64(period), dim, "period")
    out = np.zeros(pts.shape[0], dtype=np.int64)
    rc = lib.stdg_locate_points(dim, xyz.shape[0], _d(xyz), ev.shape[0], ev.ctypes.data_as(_I32),
                                None if per is None else _d(per), pts.shape[0], _d(pts), out.ctypes.data_as(_I64))
    if rc != 0:
        raise StdgError(rc, "stdg_locate_points")
    return out


def measure_fma_peak(fp64=True):
    """FP64 (or FP32) FMA rate of this GPU in TFLOP/s, from the library's probe kernel."""
    v = C.c_double(0.0)
    rc = load().stdg_measure_fma_peak(1 if fp64 else 0, C.byref(v))
    if rc != 0:
        raise StdgError(rc, "stdg_measure_fma_peak failed")
    return v.value


def reference_tables(dim, p, p_gamma):
    """The library's reference tables (dict: Mref, W, T, S, kappa, u), computed on the host."""
    from math import comb
    n, g = comb(p + dim, dim), p_gamma + 1
    out = dict(Mref=np.zeros((n, n)), W=np.zeros(g), T=np.zeros((g, g)), S=np.zeros((g, g)), u=np.zeros(g))
    kappa = C.c_double(0.0)
    rc = load().stdg_reference_tables(dim, p, p_gamma, _d(out["Mref"]), _d(out["W"]), _d(out["T"]), _d(out["S"]),
                                      C.byref(kappa), _d(out["u"]))
    if rc != 0:
        raise StdgError(rc, "stdg_reference_tables")
    out["kappa"] = kappa.value
    return out


class Solver:
    """One library context: a mesh, a medium, shots, and the stepping state."""

    def __init__(self, dim, p, p_gamma, scheme="stdg", precision="fp64", rel_tol=1e-8, max_iters=5000,
                 gmres_restart=30, inner_tol=1e-4, use_graph=True, stream=None, preconditioner=1):
        self.lib = load()
        self.dim = dim
        opt = stdg_options(p, p_gamma, SCHEME[scheme], PRECISION[precision], rel_tol, max_iters, gmres_restart,
                           inner_tol, 1 if use_graph else 0, int(preconditioner))
        h = _P()
        rc = self.lib.stdg_create(C.byref(h), dim, C.byref(opt), _P(stream or 0))
        if rc != 0:
            raise StdgError(rc, "stdg_create rejected the options")
        self.h = h
        self.last_stats = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.stdg_destroy(self.h)
            self.h = None

    __del__ = close

    def _chk(self, rc, allow=()):
        if rc < 0 and rc not in allow:
            raise StdgError(rc, self.lib.stdg_last_error(self.h).decode())
        return rc

    def query(self, what):
        v = C.c_int64()
        self._chk(self.lib.stdg_query(self.h, what, C.byref(v)))
        return v.value

    n_elem = property(lambda s: s.query(0))
    n_face = property(lambda s: s.query(1))
    Nphi = property(lambda s: s.query(2))
    Npsi = property(lambda s: s.query(3))
    Ng = property(lambda s: s.query(4))
    n_sig = property(lambda s: s.query(5))
    n_shots = property(lambda s: s.query(6))
    nvel = property(lambda s: s.query(7))

    def set_mesh(self, xyz, elem_vert, period=None):
        xyz = _f64(xyz)
        ev = np.ascontiguousarray(elem_vert, dtype=np.int32)
        per = None if period is None else _f64(period)
        self._chk(self.lib.stdg_set_mesh(self.h, xyz.shape[0], _d(xyz), ev.shape[0], ev.ctypes.data_as(_I32),
                                         None if per is None else _d(per)))

    def set_material(self, lam, mu, rho):
        ne = self.n_elem
        lam, mu, rho = (_need(_f64(a), ne, k) for a, k in ((lam, "lambda"), (mu, "mu"), (rho, "rho")))
        self._chk(self.lib.stdg_set_material(self.h, _d(lam), _d(mu), _d(rho)))

    def set_shots(self, n):
        self._chk(self.lib.stdg_set_shots(self.h, n))

    def set_state(self, v_tr, sig_tr, shot=0):
        v = _need(_f64(v_tr), self.n_elem * self.dim * self.Nphi, "v_tr")
        s = _need(_f64(sig_tr), self.n_face * self.n_sig * self.Npsi, "sig_tr")
        self._chk(self.lib.stdg_set_state(self.h, shot, _d(v), _d(s)))

    def get_state(self, shot=0, out=None):
        """(v_tr, sig_tr); ``out`` = (v, sig) preallocated float64 arrays (e.g. pinned host memory)."""
        if out is None:
            v = np.zeros((self.n_elem, self.dim, self.Nphi))
            s = np.zeros((self.n_face, self.n_sig, self.Npsi))
        else:
            v = _out(out[0], self.n_elem * self.dim * self.Nphi, "out[0]")
            s = _out(out[1], self.n_face * self.n_sig * self.Npsi, "out[1]")
        self._chk(self.lib.stdg_get_state(self.h, shot, _d(v), _d(s)))
        return v, s

    def set_plane_wave(self, kind, n, pol=None, amp=1.0, t=0.0, shot=0):
        n = _need(_f64(n), self.dim, "n")
        pol = None if pol is None else _need(_f64(pol), self.dim, "pol")
        self._chk(self.lib.stdg_set_plane_wave(self.h, shot, kind, _d(n), None if pol is None else _d(pol), amp, t))

    def set_sources(self, xs, direction, f0, t_delay, a1):
        xs, dr = _f64(np.atleast_2d(xs)), _f64(np.atleast_2d(direction))
        _need(xs, xs.shape[0] * self.dim, "xs")
        _need(dr, xs.shape[0] * self.dim, "direction")
        self._chk(self.lib.stdg_set_sources(self.h, xs.shape[0], _d(xs), _d(dr), f0, t_delay, a1))
        self.src_per_shot = 1

    def set_point_sources(self, xs, direction, f0, t_delay, a1, n_shots=1):
        """Several point sources per shot: xs, direction of shape (n_shots * per_shot, dim)."""
        xs, dr = _f64(np.atleast_2d(xs)), _f64(np.atleast_2d(direction))
        if n_shots < 1 or xs.shape[0] % n_shots:
            raise ValueError("%d sources do not split into %d shots" % (xs.shape[0], n_shots))
        _need(xs, xs.shape[0] * self.dim, "xs")
        _need(dr, xs.shape[0] * self.dim, "direction")
        per = xs.shape[0] // n_shots
        self._chk(self.lib.stdg_set_point_sources(self.h, n_shots, per, _d(xs), _d(dr), f0, t_delay, a1))
        self.src_per_shot = per

    def set_receivers(self, xr):
        xr = _f64(np.atleast_2d(xr))
        _need(xr, xr.shape[0] * self.dim, "xr")
        self.n_rec = xr.shape[0]
        self._chk(self.lib.stdg_set_receivers(self.h, xr.shape[0], _d(xr)))

    def step(self, dt, n_steps=1, allow_notconv=False, allow=()):
        st = stdg_stats()
        rc = self.lib.stdg_step(self.h, dt, n_steps, C.byref(st))
        self.last_stats = st.as_dict()
        self.last_rc = rc
        self._chk(rc, allow=tuple(allow) + ((STDG_ENOTCONV,) if allow_notconv else ()))
        return self.last_stats

    def set_time_scale(self, alpha=None):
        """Per-element time scale: step(dt) advances element i by alpha[i] dt (one value per
        disconnected part; None resets to 1)."""
        if alpha is None:
            self._chk(self.lib.stdg_set_time_scale(self.h, None))
            return
        a = _need(_f64(alpha), self.n_elem, "alpha")
        self._chk(self.lib.stdg_set_time_scale(self.h, _d(a)))

    def set_pre2_storage(self, bits):
        """Stencil-preconditioner blocks of the single-shot FP32 inner solve: 16 (balanced FP16,
        default) or 32 bits."""
        self._chk(self.lib.stdg_set_pre2_storage(self.h, int(bits)))

    pre2_bits = property(lambda s: s.query(12))

    def set_energy_check(self, enable=True, rel_tol=0.0):
        """Energy-growth sentinel around step (Theorem 4): STDG_EENERGY when a shot's energy
        grows by more than rel_tol over a source-free step (negative rel_tol: demands a decrease)."""
        self._chk(self.lib.stdg_set_energy_check(self.h, 1 if enable else 0, float(rel_tol)))

    @property
    def time(self):
        t = C.c_double()
        self._chk(self.lib.stdg_get_time(self.h, C.byref(t)))
        return t.value

    @time.setter
    def time(self, t):
        self._chk(self.lib.stdg_set_time(self.h, t))

    def energy(self):
        out = np.zeros(self.n_shots)
        self._chk(self.lib.stdg_energy(self.h, _d(out)))
        return out

    def read_receivers(self, max_steps=100000):
        n_rec = getattr(self, "n_rec", 0)
        if n_rec == 0:
            return np.zeros((self.n_shots, 0, 0, self.dim))
        cap = self.n_shots * max_steps * n_rec * self.dim
        buf = np.zeros(cap)
        k = self._chk(self.lib.stdg_read_receivers(self.h, _d(buf), cap))
        return buf[: self.n_shots * k * n_rec * self.dim].reshape(self.n_shots, k, n_rec, self.dim)

    def apply_operator(self, dt, x):
        x = _need(_f64(x).ravel(), self.nvel, "x")
        y = np.zeros_like(x)
        self._chk(self.lib.stdg_apply_operator(self.h, dt, _d(x), _d(y)))
        return y

    def apply_operator_device(self, dt, x_ptr, y_ptr, fp32=False):
        self._chk(self.lib.stdg_apply_operator_device(self.h, dt, _P(x_ptr), _P(y_ptr), 1 if fp32 else 0))

    def apply_preconditioner(self, dt, r):
        r = _need(_f64(r).ravel(), self.nvel, "r")
        z = np.zeros_like(r)
        self._chk(self.lib.stdg_apply_preconditioner(self.h, dt, _d(r), _d(z)))
        return z

    def apply_preconditioner_device(self, dt, r_ptr, z_ptr, fp32=False):
        """z = P^{-1} r for all shots (stacked) on device buffers; synchronises the stream."""
        self._chk(self.lib.stdg_apply_preconditioner_device(self.h, dt, _P(r_ptr), _P(z_ptr), 1 if fp32 else 0))

    def get_faces(self):
        fl = np.zeros(self.n_face, dtype=np.int32)
        fr = np.zeros(self.n_face, dtype=np.int32)
        self._chk(self.lib.stdg_get_faces(self.h, fl.ctypes.data_as(_I32), fr.ctypes.data_as(_I32)))
        return fl, fr

    def misfit_grad(self, dt, n_steps, data, checkpoint_every=20, grad=True, source_grad=False):
        """(loss, g_lambda, g_mu, g_rho, stats) of n_steps slabs from the current states;
        data: (n_shots, n_steps, n_rec, dim).  grad=False: the loss only (forward run).
        source_grad=True: (loss, g_lambda, g_mu, g_rho, g_src, stats) with g_src of shape
        (n_sources, 1 + 2 dim): d/d amplitude, d/d force direction, d/d position per source."""
        data = _need(_f64(data), self.n_shots * n_steps * getattr(self, "n_rec", 0) * self.dim, "data")
        loss = C.c_double(0.0)
        g = [np.zeros(self.n_elem) for _ in range(3)] if grad else [None, None, None]
        n_src = self.n_shots * getattr(self, "src_per_shot", 1)
        gs = np.zeros((n_src, 1 + 2 * self.dim)) if source_grad else None
        st = stdg_stats()

        def ptr(a):
            return _d(a) if a is not None else None

        self._chk(self.lib.stdg_misfit_grad(self.h, dt, n_steps, _d(data), checkpoint_every, C.byref(loss),
                                            ptr(g[0]), ptr(g[1]), ptr(g[2]), ptr(gs), C.byref(st)))
        if source_grad:
            return loss.value, g[0], g[1], g[2], gs, st.as_dict()
        return loss.value, g[0], g[1], g[2], st.as_dict()

    def time_kernel(self, dt, which, fp32=False, n=20):
        """Average ms of one launch: which 0 face term, 1 block Jacobi, 2 stencil local step, 3 operator."""
        ms = C.c_double(0.0)
        self._chk(self.lib.stdg_time_kernel(self.h, dt, int(which), 1 if fp32 else 0, n, C.byref(ms)))
        return ms.value

    def autotune(self, dt):
        """Time the candidate launch shapes of the hot kernels on this context and keep the fastest."""
        t = stdg_tuning()
        self._chk(self.lib.stdg_autotune(self.h, dt, C.byref(t)))
        return t.as_dict()

    def inject_wait_error(self):
        """Set the device error word as a timed-out bulk-copy wait would (failure-path tests)."""
        self._chk(self.lib.stdg_inject_wait_error(self.h))

    def time_operator(self, dt, fp32=False, n=20):
        ms = C.c_double()
        self._chk(self.lib.stdg_time_operator(self.h, dt, 1 if fp32 else 0, n, C.byref(ms)))
        return ms.value


def solver_from_workload(w, precision="fp64", rel_tol=1e-8, max_iters=5000, gmres_restart=30, inner_tol=1e-4,
                         use_graph=True, stream=None, with_sources=True, with_receivers=True, preconditioner=1):
    """Build a Solver for a ``synth.Workload`` (mesh, media, plane wave or sources, receivers)."""
    s = Solver(w.dim, w.p, w.p_gamma, w.scheme, precision, rel_tol, max_iters, gmres_restart, inner_tol, use_graph,
               stream, preconditioner)
    s.set_mesh(w.xyz, w.elem_vert, w.period)
    s.set_material(w.lam, w.mu, w.rho)
    if with_sources and w.shots_xs is not None:
        s.set_sources(w.shots_xs, w.shots_dir, w.f0, w.t_delay, w.a1)
    elif with_sources and "part_sources" in w.extra:     # ragged batch: one source per mesh part, one shot
        xs = w.extra["part_sources"]
        s.set_point_sources(xs, np.tile(np.eye(w.dim)[-1], (xs.shape[0], 1)), w.f0, w.t_delay, w.a1)
    if w.plane_wave is not None:
        pw = w.plane_wave
        s.set_plane_wave(pw["kind"], pw["n"], pw.get("pol"), pw["amp"])
    if with_receivers and w.receivers is not None:
        s.set_receivers(w.receivers)
    return s


def misfit(solver, lam, mu, rho, dt, n_steps, data, reset=None, checkpoint_every=20, sources=None):
    """Receiver misfit as a differentiable torch function of the per-element lambda, mu, rho and,
    optionally, of the point sources.

    Sets the material from the three tensors.  Without ``sources``, calls ``reset()`` to put the
    initial states back (for instance ``lambda: solver.set_sources(...)``).  With ``sources`` =
    dict(xs=tensor (n_src, dim), force=tensor (n_src, dim), f0=..., t_delay=..., n_shots=...),
    sets the point sources from the tensors (force = amplitude times direction, Ricker wavelet of
    unit amplitude; this also resets the states) and differentiates with respect to xs and force
    too.  Then runs stdg_misfit_grad: the forward value is the misfit of ``n_steps`` slabs against
    ``data`` (n_shots, n_steps, n_rec, dim); backward returns the adjoint gradients scaled by the
    incoming gradient.
    """
    import torch

    d = solver.dim
    src = sources or {}

    class _Misfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, lam_t, mu_t, rho_t, xs_t, force_t):
            solver.set_material(lam_t.detach().cpu().double().numpy(), mu_t.detach().cpu().double().numpy(),
                                rho_t.detach().cpu().double().numpy())
            if xs_t is not None:
                solver.set_point_sources(xs_t.detach().cpu().double().numpy(), force_t.detach().cpu().double().numpy(),
                                         src["f0"], src["t_delay"], 1.0, n_shots=src.get("n_shots", 1))
            else:
                reset()
            out = solver.misfit_grad(dt, n_steps, data, checkpoint_every=checkpoint_every,
                                     source_grad=xs_t is not None)
            like = dict(dtype=lam_t.dtype, device=lam_t.device)
            grads = [torch.as_tensor(g, **like) for g in out[1:4]]
            if xs_t is not None:
                gs = out[4]
                grads += [torch.as_tensor(gs[:, 1 + d:], **like), torch.as_tensor(gs[:, 1:1 + d], **like)]
            ctx.save_for_backward(*grads)
            ctx.has_src = xs_t is not None
            return torch.tensor(out[0], **like)

        @staticmethod
        def backward(ctx, g_out):
            g = [g_out * t for t in ctx.saved_tensors]
            if not ctx.has_src:
                g += [None, None]
            return tuple(g)

    return _Misfit.apply(lam, mu, rho, src.get("xs"), src.get("force"))
