"""Python binding of the C ABI in include/ewos.h (argument marshalling only).

Every step of the toolbox build and of the solves runs in the CUDA library libewos.so built
in-tree by ``paper_2608_07017_b300/build.py``; there is no CPU fallback: loading fails loudly
when the library is missing.  Host arrays are numpy float64; device arrays may be passed as
torch tensors (their data pointers are handed to the library).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libewos.so")
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONV, ETIMEOUT, ESTEPCAP, EIO = range(9)
SDF = {"ball": 0, "box": 1, "polygon": 2}
ARR = {"G": 0, "gradG": 1, "H": 2, "gradH": 3, "Hc": 4, "lambda": 5, "walk_exit": 6, "walk_steps": 7,
       "walk_mass": 8, "walk_vhash": 9, "walk_xexit": 10}
NL = {"linear": 0, "semilinear": 1, "quasilinear": 2}
MODE = {"fp64": 0, "mixed": 1}
ASSEMBLY = {"fp16": 0, "tf32": 1}


class EwosError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Domain(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("params", ctypes.c_void_p), ("nparams", ctypes.c_int64)]


class BuildOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_steps", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("cell_weights", ctypes.c_void_p), ("cell_samples", ctypes.c_int64),
                ("threads_per_block", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("hash_in_smem", ctypes.c_int),
                ("record_walks", ctypes.c_int), ("instance", ctypes.c_uint32), ("inputs_on_device", ctypes.c_int),
                ("lookup_grid_scale", ctypes.c_double), ("v_nodes", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("walk_kernel", ctypes.c_int)]


class BuildReport(ctypes.Structure):
    _fields_ = [("walks", ctypes.c_int64), ("steps", ctypes.c_int64), ("capped", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_walk", ctypes.c_double), ("ms_lookup", ctypes.c_double),
                ("ms_cells", ctypes.c_double), ("threads_per_block", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("grid", ctypes.c_int), ("hash_in_smem", ctypes.c_int), ("smem_bytes", ctypes.c_int64),
                ("lookup_grid_scale", ctypes.c_double), ("lookup_candidates", ctypes.c_int), ("walk_kernel", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("g", ctypes.c_void_p), ("nrhs", ctypes.c_int64), ("nl_kind", ctypes.c_int),
                ("nl_coef", ctypes.c_void_p), ("nl_ncoef", ctypes.c_int), ("mode", ctypes.c_int),
                ("rcond", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inputs_on_device", ctypes.c_int), ("stream", ctypes.c_void_p), ("pivoting", ctypes.c_int),
                ("batched", ctypes.c_int), ("newton_refactor", ctypes.c_int), ("assembly", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("alpha", ctypes.c_double), ("residual", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_assemble", ctypes.c_double), ("ms_factor", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("factorizations", ctypes.c_int), ("pivoted_factorizations", ctypes.c_int),
                ("dev_ms_gemm", ctypes.c_double), ("gemm_flop", ctypes.c_double), ("dev_ms_lu", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdamOpts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_iter", ctypes.c_int64), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int)]


class AdamReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("grad_norm", ctypes.c_double), ("converged", ctypes.c_int),
                ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("memory_fraction", ctypes.c_double), ("reserve_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("queued", ctypes.c_int), ("active", ctypes.c_int), ("peak_active", ctypes.c_int), ("slots", ctypes.c_int),
                ("budget_bytes", ctypes.c_int64), ("charged_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestTiming(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("slot", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load libewos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libewos.so not built at {LIB_PATH}: run paper_2608_07017_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.ewos_status_string.argtypes = [I]
        L.ewos_status_string.restype = ctypes.c_char_p
        L.ewos_last_error.restype = ctypes.c_char_p
        L.ewos_launch_count.restype = ctypes.c_ulonglong
        L.ewos_toolbox_build.argtypes = [ctypes.POINTER(_Domain), P, I64, P, I64, I64, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.POINTER(BuildOpts), ctypes.POINTER(P)]
        L.ewos_toolbox_from_host.argtypes = [I, I64, I64, P, P, P, P, P, P, P, I, P, ctypes.POINTER(P)]
        L.ewos_toolbox_get.argtypes = [P, I, P, ctypes.c_size_t, I]
        L.ewos_toolbox_report.argtypes = [P, ctypes.POINTER(BuildReport)]
        L.ewos_toolbox_shape.argtypes = [P, P, P, P, P, P]
        L.ewos_toolbox_free.argtypes = [P]
        L.ewos_toolbox_free.restype = None
        L.ewos_solve.argtypes = [P, ctypes.POINTER(_Problem), P, P, I, ctypes.POINTER(SolveReport)]
        L.ewos_toolbox_build_noalloc.argtypes = [ctypes.POINTER(_Domain), P, I64, P, I64, I64, ctypes.c_double,
                                                 ctypes.c_uint64, I64, P, P, P, P, ctypes.POINTER(BuildReport)]
        L.ewos_debug_philox.argtypes = [P, P, P, I64]
        L.ewos_debug_green_radius.argtypes = [P, P, I64, I]
        L.ewos_debug_tc_gemm.argtypes = [P, P, P, I, I, I, I]
        L.ewos_debug_tc_assemble.argtypes = [P, P, I, I, I, P, I, I]
        L.ewos_debug_tc_update.argtypes = [P, P, P, I, I, I, I]
        L.ewos_debug_set_flow_wait_limit.argtypes = [I64]
        L.ewos_debug_fail_allocations.argtypes = [I64]
        L.ewos_debug_fail_allocations.restype = None
        L.ewos_toolbox_build_batch.argtypes = [I, P, P, P, P, P, I64, ctypes.c_double, ctypes.c_uint64,
                                               ctypes.POINTER(BuildOpts), P, ctypes.POINTER(BuildReport)]
        L.ewos_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
        L.ewos_server_submit.argtypes = [P, P, ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_uint64)]
        L.ewos_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, P, P, ctypes.POINTER(SolveReport),
                                       ctypes.POINTER(RequestTiming)]
        L.ewos_server_query.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.ewos_server_destroy.argtypes = [P]
        L.ewos_server_destroy.restype = None
        L.ewos_toolbox_save.argtypes = [P, ctypes.c_char_p]
        L.ewos_toolbox_load.argtypes = [ctypes.c_char_p, P, ctypes.POINTER(P)]
        L.ewos_gradient.argtypes = [P, ctypes.POINTER(_Problem), P, P]
        L.ewos_operators.argtypes = [P, ctypes.POINTER(_Problem), P, P, I, ctypes.POINTER(SolveReport)]
        L.ewos_minimize_adam.argtypes = [P, ctypes.POINTER(_Problem), ctypes.POINTER(AdamOpts), P, P,
                                         ctypes.POINTER(AdamReport)]
        for fn in ("ewos_toolbox_build", "ewos_toolbox_build_noalloc", "ewos_toolbox_from_host", "ewos_toolbox_get", "ewos_toolbox_report",
                   "ewos_toolbox_shape", "ewos_solve", "ewos_debug_philox", "ewos_debug_green_radius",
                   "ewos_debug_tc_gemm", "ewos_debug_tc_assemble", "ewos_debug_tc_update", "ewos_server_create", "ewos_server_submit", "ewos_server_wait",
                   "ewos_server_query", "ewos_toolbox_build_batch", "ewos_toolbox_save", "ewos_toolbox_load",
                   "ewos_gradient", "ewos_minimize_adam", "ewos_operators"):
            getattr(L, fn).restype = I
        _lib = L
    return _lib


def _check(status, what, allow=(OK,)):
    if status not in allow:
        raise EwosError(status, f"{what}: {lib().ewos_status_string(status).decode()}: "
                                f"{lib().ewos_last_error().decode()}")
    return status


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Toolbox:
    """Device-resident toolbox (G, gradG, H, gradH, exit counts, cell weights)."""

    def __init__(self, handle, keep=()):
        self._h = ctypes.c_void_p(handle)
        self._keep = keep
        d, n, m, p, prec = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().ewos_toolbox_shape(self._h, ctypes.byref(d), ctypes.byref(n), ctypes.byref(m),
                                        ctypes.byref(p), ctypes.byref(prec)), "shape")
        self.dim, self.n, self.m, self.p, self.precision = d.value, n.value, m.value, p.value, prec.value
        self.status = OK

    def close(self):
        if self._h:
            lib().ewos_toolbox_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def report(self):
        r = BuildReport()
        _check(lib().ewos_toolbox_report(self._h, ctypes.byref(r)), "report")
        return r.as_dict()

    def save(self, path):
        """Write this toolbox to a file (see save_toolbox)."""
        save_toolbox(self, path)

    def get(self, which, walks=None):
        d, n, m, p = self.dim, self.n, self.m, self.p
        shapes = {"G": (n, m), "gradG": (d, n, m), "H": (n, p), "gradH": (d, n, p), "Hc": (n, p), "lambda": (n,)}
        dtypes = {"Hc": np.uint32, "walk_exit": np.int32, "walk_steps": np.int32, "walk_vhash": np.uint32}
        shape = shapes.get(which, (n, walks, d) if which == "walk_xexit" else (n, walks))
        out = np.zeros(shape, dtype=dtypes.get(which, np.float64))
        _check(lib().ewos_toolbox_get(self._h, ARR[which], out.ctypes.data, out.nbytes, 0), f"get {which}")
        return out

    def get_device(self, which, out):
        """Copy into a device buffer (a torch tensor of the right size and dtype)."""
        _check(lib().ewos_toolbox_get(self._h, ARR[which], out.data_ptr(), out.numel() * out.element_size(), 1),
               f"get {which}")
        return out

    def matrices(self):
        return dict(G=self.get("G"), gradG=self.get("gradG"), H=self.get("H"), gradH=self.get("gradH"))

    def solve(self, A, f, g, b=None, c=None, kind="linear", coef=None, mode="fp64", rcond=-1.0, tol=0.0,
              max_iter=0, want_s=False, on_device=False, out=None, stream=None, pivoting=0, batched=False,
              newton_refactor=False, assembly="fp16"):
        """Solve the problem of include/ewos.h; returns (u [nrhs][n] or [n], s or None, report).
        pivoting=1 forces row interchanges in the mixed-mode LU; batched=True refines all
        right-hand sides together (mixed mode; chord iteration for semilinear problems);
        assembly="tf32" assembles Lambda from TF32 parts instead of scaled FP16 halves."""
        if on_device:
            Ad, fd, gd, bd, cd = A, f, g, b, c
            nrhs = f.shape[0] if f.dim() == 2 else 1
        else:
            Ad, fd, gd, bd, cd = _f64(A), _f64(f), _f64(g), _f64(b), _f64(c)
            nrhs = fd.shape[0] if fd.ndim == 2 else 1
        cf = _f64(coef) if coef is not None else None
        pb = _Problem(_ptr(Ad), _ptr(bd), _ptr(cd), _ptr(fd), _ptr(gd), nrhs, NL[kind], _ptr(cf),
                      0 if cf is None else cf.size, MODE[mode], float(rcond), float(tol), int(max_iter),
                      1 if on_device else 0, stream, int(pivoting), 1 if batched else 0, 1 if newton_refactor else 0,
                      ASSEMBLY[assembly])
        if out is not None:
            u = out
            optr = out.data_ptr()
        else:
            u = np.zeros((nrhs, self.n))
            optr = u.ctypes.data
        s = np.zeros((nrhs, self.m)) if want_s else None
        rep = SolveReport()
        st = lib().ewos_solve(self._h, ctypes.byref(pb), optr, _ptr(s), 1 if out is not None else 0, ctypes.byref(rep))
        _check(st, "solve", allow=(OK, ENOCONV))
        r = rep.as_dict()
        r["status"] = st
        if out is None and (fd.ndim if not on_device else f.dim()) == 1:
            u = u[0]
            s = None if s is None else s[0]
        return u, s, r


    def _problem1(self, A, f, g, b, c, kind, coef):
        arrs = [_f64(a) for a in (A, b, c, f, g)]
        cf = _f64(coef) if coef is not None else None
        pb = _Problem(*[_ptr(a) for a in arrs], 1, NL[kind], _ptr(cf), 0 if cf is None else cf.size, MODE["fp64"],
                      0.0, 0.0, 0, 0, None, 0, 0)
        return pb, (arrs, cf)

    def gradient(self, s, A, f, g, b=None, c=None, kind="linear", coef=None):
        """grad J(s) = R(s) of the Euler-Lagrange route (ewos_gradient); host arrays."""
        pb, keep = self._problem1(A, f, g, b, c, kind, coef)
        ss = _f64(s)
        out = np.zeros(self.m)
        _check(lib().ewos_gradient(self._h, ctypes.byref(pb), ss.ctypes.data, out.ctypes.data), "gradient")
        return out

    def operators(self, A, b=None, c=None, mode="fp64", rcond=-1.0, pivoting=0, want=("GL", "HL")):
        """Green-operator and elliptic-measure estimates (ewos_operators): (GL [n][n], HL [n][p],
        report); an output not in `want` is not computed into (returned as None)."""
        arrs = [_f64(a) for a in (A, b, c)]
        pb = _Problem(_ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), None, None, 0, NL["linear"], None, 0, MODE[mode],
                      float(rcond), 0.0, 0, 0, None, int(pivoting), 0)
        GL = np.zeros((self.n, self.n)) if "GL" in want else None
        HL = np.zeros((self.n, self.p)) if "HL" in want else None
        rep = SolveReport()
        _check(lib().ewos_operators(self._h, ctypes.byref(pb), _ptr(GL), _ptr(HL), 0, ctypes.byref(rep)), "operators")
        return GL, HL, rep.as_dict()

    def minimize_adam(self, A, f, g, b=None, c=None, kind="linear", coef=None, s0=None, alpha=1e-3, beta1=0.9,
                      beta2=0.999, eps=1e-10, max_iter=1000, tol=0.0, check_every=0):
        """Adam on J (ewos_minimize_adam); returns (s, u, report)."""
        pb, keep = self._problem1(A, f, g, b, c, kind, coef)
        s = np.zeros(self.m) if s0 is None else _f64(s0).copy()
        u = np.zeros(self.n)
        o = AdamOpts(float(alpha), float(beta1), float(beta2), float(eps), int(max_iter), float(tol), int(check_every))
        rep = AdamReport()
        _check(lib().ewos_minimize_adam(self._h, ctypes.byref(pb), ctypes.byref(o), s.ctypes.data, u.ctypes.data,
                                        ctypes.byref(rep)), "minimize_adam")
        return s, u, rep.as_dict()


def build_toolbox(domain_kind, dim, params, x, z, walks, eps, seed=0, precision=32, max_steps=0, cell_weights=None,
                  cell_samples=0, threads_per_block=0, ctas_per_sm=0, hash_in_smem=-1, record_walks=False,
                  instance=0, stream=None, on_device=False, lookup_grid_scale=0.0, y=None, walk_kernel=0):
    """y: optional V-centres [m][d] of a separate source partition (columns of G, grad G)."""
    prm = _f64(params)
    dom = _Domain(SDF[domain_kind], dim, prm.ctypes.data, prm.size)
    if on_device:
        xx, zz, yy = x, z, y
        n, p = x.shape[0], z.shape[0]
    else:
        xx, zz, yy = _f64(x), _f64(z), _f64(y)
        n, p = xx.shape[0], zz.shape[0]
    cw = _f64(cell_weights)
    o = BuildOpts(precision, max_steps, stream, _ptr(cw), cell_samples, threads_per_block, ctas_per_sm, hash_in_smem,
                  1 if record_walks else 0, instance, 1 if on_device else 0, float(lookup_grid_scale),
                  _ptr(yy), 0 if yy is None else yy.shape[0], int(walk_kernel))
    h = ctypes.c_void_p()
    st = lib().ewos_toolbox_build(ctypes.byref(dom), _ptr(xx), n, _ptr(zz), p, int(walks), float(eps), int(seed),
                                  ctypes.byref(o), ctypes.byref(h))
    _check(st, "toolbox build", allow=(OK, ESTEPCAP))
    tb = Toolbox(h.value)
    tb.status = st
    return tb


def build_toolbox_noalloc(domain_kind, dim, params, x_dev, z_dev, walks, eps, P, KH, Hc, seed=0, max_steps=0,
                          stream=None):
    """FP32 build into caller-owned device buffers (torch tensors): x_dev [n][d] and z_dev [p][d]
    float64, P [(d+1)][n][n] float32, KH [(d+1)][n][p] float32, Hc [n][p] int32/uint32 storage.
    The library allocates no device memory for it (see ewos_toolbox_build_noalloc)."""
    prm = _f64(params)
    dom = _Domain(SDF[domain_kind], dim, prm.ctypes.data, prm.size)
    rep = BuildReport()
    st = lib().ewos_toolbox_build_noalloc(ctypes.byref(dom), x_dev.data_ptr(), x_dev.shape[0], z_dev.data_ptr(),
                                          z_dev.shape[0], int(walks), float(eps), int(seed), int(max_steps), stream,
                                          P.data_ptr(), KH.data_ptr(), Hc.data_ptr(), ctypes.byref(rep))
    _check(st, "toolbox build (no allocation)", allow=(OK, ESTEPCAP))
    return st, rep.as_dict()


def build_workload(w, **kw):
    """Build the toolbox of a workloads.Workload."""
    kw.setdefault("precision", w.precision)
    if w.lam is not None:
        kw.setdefault("cell_weights", w.lam)
    return build_toolbox(w.domain.kind, w.domain.dim, w.domain.params, w.x, w.z, w.walks, w.eps, seed=w.seed, **kw)


def build_batch(domains, xs, zs, walks, eps, seed=0, precision=32, max_steps=0, instance=0, cell_samples=0,
                threads_per_block=0, ctas_per_sm=0, stream=None):
    """Several toolboxes in one persistent walk launch (ewos_toolbox_build_batch).  domains:
    list of (kind, dim, params); instance k uses Philox instance `instance + k`.  Returns
    (list of Toolbox, batch report dict, status)."""
    count = len(domains)
    prms = [_f64(pr) for _, _, pr in domains]
    doms = (_Domain * count)(*[_Domain(SDF[k], d, pr.ctypes.data, pr.size) for (k, d, _), pr in zip(domains, prms)])
    xa = [_f64(x) for x in xs]
    za = [_f64(z) for z in zs]
    xp = (ctypes.c_void_p * count)(*[a.ctypes.data for a in xa])
    zp = (ctypes.c_void_p * count)(*[a.ctypes.data for a in za])
    ns = (ctypes.c_int64 * count)(*[a.shape[0] for a in xa])
    ps = (ctypes.c_int64 * count)(*[a.shape[0] for a in za])
    o = BuildOpts()
    o.precision = precision
    o.max_steps = max_steps
    o.stream = stream
    o.cell_samples = cell_samples
    o.threads_per_block = threads_per_block
    o.ctas_per_sm = ctas_per_sm
    o.hash_in_smem = -1
    o.instance = instance
    out = (ctypes.c_void_p * count)()
    rep = BuildReport()
    st = lib().ewos_toolbox_build_batch(count, ctypes.cast(doms, ctypes.c_void_p), ctypes.cast(xp, ctypes.c_void_p),
                                        ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(zp, ctypes.c_void_p),
                                        ctypes.cast(ps, ctypes.c_void_p), walks, eps, seed, ctypes.byref(o),
                                        ctypes.cast(out, ctypes.c_void_p), ctypes.byref(rep))
    _check(st, "build_batch", allow=(OK, ESTEPCAP))
    return [Toolbox(out[k]) for k in range(count)], rep.as_dict(), st


def toolbox_from_host(dim, x, z, G, gradG, H, gradH, lam, precision=64, stream=None):
    arrs = [_f64(a) for a in (x, z, G, gradG, H, gradH, lam)]
    h = ctypes.c_void_p()
    n, p = arrs[0].shape[0], arrs[1].shape[0]
    _check(lib().ewos_toolbox_from_host(dim, n, p, *[a.ctypes.data for a in arrs], precision, stream, ctypes.byref(h)),
           "toolbox from host")
    return Toolbox(h.value, keep=arrs)


def save_toolbox(tb, path):
    """Write a toolbox to a file (ewos_toolbox_save): arrays, shape and build parameters."""
    _check(lib().ewos_toolbox_save(tb._h, os.fsencode(path)), "toolbox save")


def load_toolbox(path, stream=None):
    """Read a toolbox written by save_toolbox into device memory (ewos_toolbox_load)."""
    h = ctypes.c_void_p()
    _check(lib().ewos_toolbox_load(os.fsencode(path), stream, ctypes.byref(h)), "toolbox load")
    return Toolbox(h.value)


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().ewos_launch_count())


def debug_philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _check(lib().ewos_debug_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data, c.shape[0]), "philox")
    return out


def debug_tc_gemm(A, B, split=False, sym=False, f16=False):
    """C = A^T B on the tensor cores (TF32 inputs, FP32 accumulation; split: 3xTF32; f16: three
    products of scaled FP16 halves); A [K][M], B [K][N].  sym: a split form with the symmetric
    launch (tiles on and below the diagonal, mirrored)."""
    a = np.ascontiguousarray(A, dtype=np.float32)
    b = np.ascontiguousarray(B, dtype=np.float32)
    K, M = a.shape
    N = b.shape[1]
    c = np.zeros((M, N), dtype=np.float32)
    _check(lib().ewos_debug_tc_gemm(a.ctypes.data, b.ctypes.data, c.ctypes.data, M, N, K,
                                    (4 if sym else 3) if f16 else (2 if sym else (1 if split else 0))), "tc gemm")
    return c


def debug_tc_assemble(P, M, sym=False, f16=True):
    """Lambda = P^T Q, Q_i = M_i P_i, by the tensor-core assembly of the mixed solve: P [D+1][n][m],
    M [n][D+1][D+1]; f16: scaled FP16 halves (else three TF32 products); sym: mirrored lower half."""
    p = np.ascontiguousarray(P, dtype=np.float32)
    mm = np.ascontiguousarray(M, dtype=np.float64)
    E, n, m = p.shape
    assert mm.shape == (n, E, E)
    c = np.zeros((m, m), dtype=np.float32)
    _check(lib().ewos_debug_tc_assemble(p.ctypes.data, mm.ctypes.data, n, m, E - 1, c.ctypes.data,
                                        1 if sym else 0, 1 if f16 else 0), "tc assemble")
    return c


def debug_tc_update(A, B, C, f16=True):
    """C - A B by the tensor-core trailing update of the LU (A [M][K], B [K][N], C [M][N]; FP32):
    f16: rows of A and columns of B scaled by powers of two and split into FP16 halves (the
    rank-512 updates), else three TF32 products."""
    a = np.ascontiguousarray(A, dtype=np.float32)
    b = np.ascontiguousarray(B, dtype=np.float32)
    c = np.array(C, dtype=np.float32, order="C", copy=True)
    M, K = a.shape
    N = b.shape[1]
    assert b.shape[0] == K and c.shape == (M, N)
    _check(lib().ewos_debug_tc_update(a.ctypes.data, b.ctypes.data, c.ctypes.data, M, N, K, 1 if f16 else 0),
           "tc update")
    return c


def debug_set_flow_wait_limit(polls):
    """Test hook: polls before the dataflow solves' flag waits give up (< 0: default)."""
    _check(lib().ewos_debug_set_flow_wait_limit(int(polls)), "flow wait limit")


def debug_fail_allocations(after):
    """Test hook: the device allocation after `after` more successful ones fails (< 0: cancel)."""
    lib().ewos_debug_fail_allocations(int(after))


def debug_green_radius(u, precision=32):
    dt = np.float32 if precision == 32 else np.float64
    uu = np.ascontiguousarray(u, dtype=dt)
    R = np.zeros_like(uu)
    _check(lib().ewos_debug_green_radius(uu.ctypes.data, R.ctypes.data, uu.size, precision), "green radius")
    return R


class Server:
    """Request server of include/ewos.h (ewos_server_*): submit() queues a solve on a resident
    toolbox and returns a ticket; wait() returns (u, s, report, timing)."""

    def __init__(self, max_slots=4, memory_fraction=0.8, reserve_bytes=0, budget_bytes=0):
        o = ServerOpts(int(max_slots), float(memory_fraction), int(reserve_bytes), int(budget_bytes))
        h = ctypes.c_void_p()
        _check(lib().ewos_server_create(ctypes.byref(o), ctypes.byref(h)), "server create")
        self._h = h
        self._pending = {}

    def submit(self, tb, A, f, g, b=None, c=None, kind="linear", coef=None, mode="mixed", rcond=-1.0, tol=0.0,
               max_iter=0, pivoting=0):
        Ad, fd, gd, bd, cd = _f64(A), _f64(f), _f64(g), _f64(b), _f64(c)
        nrhs = fd.shape[0] if fd.ndim == 2 else 1
        cf = _f64(coef) if coef is not None else None
        pb = _Problem(_ptr(Ad), _ptr(bd), _ptr(cd), _ptr(fd), _ptr(gd), nrhs, NL[kind], _ptr(cf),
                      0 if cf is None else cf.size, MODE[mode], float(rcond), float(tol), int(max_iter), 0, None,
                      int(pivoting), 1)
        t = ctypes.c_uint64()
        _check(lib().ewos_server_submit(self._h, tb._h, ctypes.byref(pb), ctypes.byref(t)), "server submit")
        self._pending[t.value] = (tb.n, tb.m, nrhs, fd.ndim == 1)
        return t.value

    def wait(self, ticket, timeout_s=0.0, want_s=False):
        n, m, nrhs, single = self._pending.pop(ticket)
        u = np.zeros((nrhs, n))
        s = np.zeros((nrhs, m)) if want_s else None
        rep = SolveReport()
        tm = RequestTiming()
        st = lib().ewos_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s), u.ctypes.data, _ptr(s),
                                    ctypes.byref(rep), ctypes.byref(tm))
        if st == ETIMEOUT:
            self._pending[ticket] = (n, m, nrhs, single)
        _check(st, "server wait", allow=(OK, ENOCONV))
        r = rep.as_dict()
        r["status"] = st
        if single:
            u = u[0]
            s = None if s is None else s[0]
        return u, s, r, tm.as_dict()

    def stats(self):
        st = ServerStats()
        _check(lib().ewos_server_query(self._h, ctypes.byref(st)), "server query")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().ewos_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
