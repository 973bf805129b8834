"""Thin Python binding of the C-ABI in include/bi.h (argument marshalling only).

Every numerical step runs in libbi_gb300.so; PyTorch provides device memory and the
CUDA stream.  The library is loaded on first use and a missing or unloadable
library raises -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbi_gb300.so")

BI_OK = 0
BI_ERR_ARG = -1
BI_ERR_MESH = -2
BI_ERR_OOM = -3
BI_ERR_CUDA = -4
BI_ERR_NOT_CONVERGED = -5
BI_ERR_TIMEOUT = -6
BI_ERR_BUSY = -7
_NAMES = {0: "BI_OK", -1: "BI_ERR_ARG", -2: "BI_ERR_MESH", -3: "BI_ERR_OOM", -4: "BI_ERR_CUDA",
          -5: "BI_ERR_NOT_CONVERGED", -6: "BI_ERR_TIMEOUT", -7: "BI_ERR_BUSY"}

# entry points declared in include/bi.h
EXPORTS = ["bi_default_params", "bi_setup", "bi_num_unknowns", "bi_rwg_edges", "bi_get_info", "bi_matvec",
           "bi_matvec_host", "bi_rhs_planewave", "bi_solve", "bi_solve_refined", "bi_farfield", "bi_farfield_noalloc", "bi_debug_copy", "bi_debug_set_wait_limit", "bi_tuned_config", "bi_profile_stages", "bi_stage_name", "bi_last_error", "bi_device_status", "bi_set_coupling", "bi_coupling_blocks", "bi_matvec_coupled", "bi_plan_create", "bi_plan_info", "bi_plan_get",
           "bi_plan_last_error", "bi_plan_destroy",
           "bi_destroy", "bi_server_default_params", "bi_server_create", "bi_submit", "bi_poll", "bi_result",
           "bi_release", "bi_server_last_error", "bi_server_stats", "bi_server_destroy"]


# qsolve(user, in, out, nrhs, stream) of bi_set_coupling
QSOLVE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)


class _DeviceView:
    """A raw device buffer seen by torch (argument marshalling for the qsolve callback)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


class BIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, code), msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("digits", ctypes.c_int), ("leaf_box", ctypes.c_double), ("levels", ctypes.c_int),
                ("interp_order", ctypes.c_int), ("precision", ctypes.c_int), ("op_mode", ctypes.c_int),
                ("max_rhs", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("precond", ctypes.c_int), ("k_im", ctypes.c_double),
                ("eps_re", ctypes.c_double), ("eps_im", ctypes.c_double), ("core_tris", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n_rwg", ctypes.c_int64), ("n_unknowns", ctypes.c_int64), ("levels", ctypes.c_int),
                ("leaf_level", ctypes.c_int), ("boxes", ctypes.c_int * 32), ("L", ctypes.c_int * 32),
                ("K", ctypes.c_int * 32), ("near_pairs", ctypes.c_int64), ("interactions", ctypes.c_int64 * 32),
                ("device_bytes", ctypes.c_int64), ("root_size", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("setup_near_regular_ms", ctypes.c_double), ("setup_near_special_ms", ctypes.c_double),
                ("near_special_entries", ctypes.c_int64), ("setup_sai_ms", ctypes.c_double)]


class ServerParams(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int), ("queue_capacity", ctypes.c_int),
                ("share_operators", ctypes.c_int), ("max_batch_rhs", ctypes.c_int), ("setup_threads", ctypes.c_int)]


SERVER_STATS = ("jobs", "operators_built", "cache_hits", "merged_requests", "evictions", "cached_operators",
                "held_bytes")


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libbi_gb300.so not built: run paper_2210_04892_gb300/build.py (or __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.bi_default_params.argtypes = [ctypes.POINTER(Params)]
    L.bi_default_params.restype = None
    L.bi_setup.argtypes = [vp, i, vp, i, d, i, ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.bi_num_unknowns.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.bi_rwg_edges.argtypes = [vp, vp]
    L.bi_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.bi_matvec.argtypes = [vp, vp, vp, i]
    L.bi_matvec_host.argtypes = [vp, vp, vp, i]
    L.bi_rhs_planewave.argtypes = [vp, vp, vp, i, vp]
    L.bi_solve.argtypes = [vp, vp, vp, i, d, vp, vp]
    L.bi_solve_refined.argtypes = [vp, vp, vp, vp, i, d, vp, vp]
    L.bi_farfield.argtypes = [vp, vp, i, vp, i, vp]
    L.bi_farfield_noalloc.argtypes = [vp, vp, i, vp, i, vp]
    L.bi_debug_copy.argtypes = [vp, i, i, vp, i64]
    L.bi_debug_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    L.bi_tuned_config.argtypes = [vp, ctypes.c_char_p, i64]
    L.bi_profile_stages.argtypes = [vp, vp, vp, i, i, vp]
    L.bi_stage_name.argtypes = [i]
    L.bi_stage_name.restype = ctypes.c_char_p
    L.bi_last_error.argtypes = [vp]
    L.bi_last_error.restype = ctypes.c_char_p
    L.bi_device_status.argtypes = [vp]
    L.bi_set_coupling.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, QSOLVE, vp]
    L.bi_coupling_blocks.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp]
    L.bi_matvec_coupled.argtypes = [vp, vp, vp, i]
    L.bi_plan_create.argtypes = [vp, i, vp, i, d, ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.bi_plan_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.bi_plan_get.argtypes = [vp, i, i, vp, i64, ctypes.POINTER(i64)]
    L.bi_plan_last_error.argtypes = []
    L.bi_plan_last_error.restype = ctypes.c_char_p
    L.bi_plan_destroy.argtypes = [vp]
    L.bi_plan_destroy.restype = None
    L.bi_destroy.argtypes = [vp]
    L.bi_destroy.restype = None
    L.bi_server_default_params.argtypes = [ctypes.POINTER(ServerParams)]
    L.bi_server_default_params.restype = None
    L.bi_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(vp)]
    L.bi_submit.argtypes = [vp, vp, i, vp, i, d, ctypes.POINTER(Params), i, vp, vp, d, ctypes.POINTER(i64)]
    L.bi_poll.argtypes = [vp, i64, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.bi_server_stats.argtypes = [vp, vp, i]
    L.bi_result.argtypes = [vp, i64, vp, i64, vp, vp, ctypes.POINTER(d), ctypes.POINTER(d)]
    L.bi_release.argtypes = [vp, i64]
    L.bi_server_last_error.argtypes = [vp]
    L.bi_server_last_error.restype = ctypes.c_char_p
    L.bi_server_destroy.argtypes = [vp]
    L.bi_server_destroy.restype = None
    _lib = L
    return L


def default_params() -> Params:
    p = Params()
    load().bi_default_params(ctypes.byref(p))
    return p


def _check(rc, h=None):
    if rc != BI_OK:
        raise BIError(rc, load().bi_last_error(h).decode())


class Operator:
    """The boundary-integral operator C (Eqs. 43-46) of one closed surface, on the GPU.

    op_mode 0: C block (2N unknowns, J then M); op_mode 1: PEC combined field (N).
    precision "fp32" (complex64 vectors) or "fp64" (complex128).  k0 may be complex
    (k0.real > 0 >= k0.imag: a lossy medium); its imaginary part goes to bi_params.k_im.
    op_mode 2: a homogeneous body of relative permittivity eps_r (two-region equations);
    op_mode 4: a PEC core (the last core_tris triangles) under a coat of permittivity eps_r."""

    def __init__(self, verts, tris, k0, digits=3, precision="fp32", op_mode=0, leaf_box=0.25, levels=0,
                 interp_order=10, max_rhs=1, gmres_restart=100, gmres_maxit=1000, stream=None, precond=0,
                 eps_r=1.0, core_tris=0):
        import torch
        L = load()
        p = default_params()
        p.digits = int(digits)
        p.leaf_box = float(leaf_box)
        p.levels = int(levels)
        p.interp_order = int(interp_order)
        p.precision = 0 if precision == "fp64" else 1
        p.op_mode = int(op_mode)
        p.max_rhs = int(max_rhs)
        p.gmres_restart = int(gmres_restart)
        p.gmres_maxit = int(gmres_maxit)
        p.precond = int(precond)
        k0 = complex(k0)
        p.k_im = k0.imag
        eps_r = complex(eps_r)
        p.eps_re, p.eps_im = eps_r.real, eps_r.imag
        p.core_tris = int(core_tris)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        p.stream = ctypes.c_void_p(stream.cuda_stream)
        v = np.ascontiguousarray(verts, np.float64)
        t = np.ascontiguousarray(tris, np.int32)
        self._v, self._t = v, t
        h = ctypes.c_void_p()
        rc = L.bi_setup(v.ctypes.data, len(v), t.ctypes.data, len(t), k0.real, int(digits), ctypes.byref(p),
                        ctypes.byref(h))
        _check(rc, None)
        self.h = h
        self.params = p
        self.precision = precision
        self.cdtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.np_cdtype = np.complex128 if precision == "fp64" else np.complex64
        n, nu = ctypes.c_int64(), ctypes.c_int64()
        L.bi_num_unknowns(h, ctypes.byref(n), ctypes.byref(nu))
        self.n_rwg, self.n_unknowns = n.value, nu.value
        self.max_rhs = int(max_rhs)
        self.k0 = k0.real if k0.imag == 0 else k0

    # ---------------------------------------------------------------- queries
    def info(self) -> dict:
        I = Info()
        _check(load().bi_get_info(self.h, ctypes.byref(I)), self.h)
        nl = I.levels
        return dict(n_rwg=I.n_rwg, n_unknowns=I.n_unknowns, levels=nl, leaf_level=I.leaf_level,
                    boxes=list(I.boxes[:nl]), L=list(I.L[:nl]), K=list(I.K[:nl]), near_pairs=I.near_pairs,
                    interactions=list(I.interactions[:nl]), device_bytes=I.device_bytes, root_size=I.root_size,
                    setup_ms=I.setup_ms, setup_near_regular_ms=I.setup_near_regular_ms,
                    setup_near_special_ms=I.setup_near_special_ms, near_special_entries=I.near_special_entries,
                    setup_sai_ms=I.setup_sai_ms)

    def edges(self) -> np.ndarray:
        e = np.zeros((self.n_rwg, 2), np.int32)
        _check(load().bi_rwg_edges(self.h, e.ctypes.data), self.h)
        return e

    # ---------------------------------------------------------------- products
    def _vec(self, x, nrhs=None):
        import torch
        if x.dtype != self.cdtype or not x.is_cuda or not x.is_contiguous():
            raise TypeError("expected a contiguous CUDA %s tensor" % self.cdtype)
        if x.dim() == 1:
            x = x.view(1, -1)
        if x.shape[-1] != self.n_unknowns:
            raise ValueError("last dimension must be n_unknowns = %d" % self.n_unknowns)
        return x

    def matvec(self, x, out=None):
        """y = C x for x of shape [nrhs, n_unknowns] (CUDA complex tensor); queued on the stream."""
        import torch
        x = self._vec(x)
        if out is None:
            out = torch.empty_like(x)
        _check(load().bi_matvec(self.h, x.data_ptr(), out.data_ptr(), x.shape[0]), self.h)
        return out

    def matvec_host(self, x, out=None):
        """y = C x with host buffers (numpy arrays, or CPU torch tensors -- pinned for
        asynchronous copies); the call copies in, multiplies, copies out and synchronises."""
        if hasattr(x, "data_ptr"):
            if x.is_cuda or not x.is_contiguous() or x.shape[-1] != self.n_unknowns:
                raise TypeError("expected a contiguous CPU tensor with last dimension n_unknowns")
            y = out if out is not None else x.new_empty(x.shape)
            n = 1 if x.dim() == 1 else x.shape[0]
            _check(load().bi_matvec_host(self.h, x.data_ptr(), y.data_ptr(), n), self.h)
            return y
        x = np.ascontiguousarray(np.atleast_2d(x), self.np_cdtype)
        y = np.empty_like(x) if out is None else out
        _check(load().bi_matvec_host(self.h, x.ctypes.data, y.ctypes.data, x.shape[0]), self.h)
        return y

    def rhs_planewave(self, khat, phat):
        import torch
        kh = np.ascontiguousarray(np.atleast_2d(khat), np.float64)
        ph = np.ascontiguousarray(np.atleast_2d(phat), np.float64)
        b = torch.empty((len(kh), self.n_unknowns), dtype=self.cdtype, device="cuda")
        _check(load().bi_rhs_planewave(self.h, kh.ctypes.data, ph.ctypes.data, len(kh), b.data_ptr()), self.h)
        return b

    def solve(self, b, tol=1e-3):
        """GMRES solve of C x = b; returns (x, iterations, relative residuals)."""
        import torch
        b = self._vec(b)
        x = torch.empty_like(b)
        R = b.shape[0]
        its = np.zeros(R, np.int32)
        rel = np.zeros(R, np.float64)
        rc = load().bi_solve(self.h, b.data_ptr(), x.data_ptr(), R, float(tol), its.ctypes.data, rel.ctypes.data)
        if rc not in (BI_OK, BI_ERR_NOT_CONVERGED):
            _check(rc, self.h)
        return x, its, rel

    def solve_refined(self, ref, b, tol=1e-4):
        """Iterative refinement: inner GMRES on this operator, residuals with the FP64 operator
        `ref` of the same surface; b complex128 on the GPU.  Returns (x complex128, iterations,
        relative FP64 residuals)."""
        import torch
        b = b.to(torch.complex128).contiguous()
        if b.dim() == 1:
            b = b.view(1, -1)
        x = torch.empty_like(b)
        R = b.shape[0]
        its = np.zeros(R, np.int32)
        rel = np.zeros(R, np.float64)
        rc = load().bi_solve_refined(self.h, ref.h, b.data_ptr(), x.data_ptr(), R, float(tol), its.ctypes.data,
                                     rel.ctypes.data)
        if rc not in (BI_OK, BI_ERR_NOT_CONVERGED):
            _check(rc, self.h)
        return x, its, rel

    def profile_stages(self, x, reps=10):
        """Mean device milliseconds of each stage of one product (serialised stages)."""
        x = self._vec(x)
        import torch
        y = torch.empty_like(x)
        ms = np.zeros(8, np.float64)
        _check(load().bi_profile_stages(self.h, x.data_ptr(), y.data_ptr(), x.shape[0], int(reps), ms.ctypes.data),
               self.h)
        return {load().bi_stage_name(i).decode(): float(ms[i]) for i in range(8)}

    def coupling_blocks(self, conforming=False):
        """The coupling blocks of Eqs. 40a/b, 47, 48 on this surface, computed on the GPU:
        returns (n_lambda, dlx, dxl) with dlx = (ptr, col, val) of D^{Lambda X} and dxl of
        D^{X Lambda} as CUDA tensors, ready for set_coupling."""
        import torch
        L = load()
        sizes = np.zeros(3, np.int64)
        _check(L.bi_coupling_blocks(self.h, int(bool(conforming)), sizes.ctypes.data, None, None, None, None, None,
                                    None), self.h)
        nL, nxl, nlx = (int(v) for v in sizes)
        i32 = dict(dtype=torch.int32, device="cuda")
        xl = (torch.empty(self.n_unknowns + 1, **i32), torch.empty(nxl, **i32),
              torch.empty(nxl, dtype=self.cdtype, device="cuda"))
        lx = (torch.empty(nL + 1, **i32), torch.empty(nlx, **i32), torch.empty(nlx, dtype=self.cdtype, device="cuda"))
        _check(L.bi_coupling_blocks(self.h, int(bool(conforming)), sizes.ctypes.data, xl[0].data_ptr(),
                                    xl[1].data_ptr(), xl[2].data_ptr(), lx[0].data_ptr(), lx[1].data_ptr(),
                                    lx[2].data_ptr()), self.h)
        return nL, lx, xl

    def set_coupling(self, n_int, dlx, dxl, qsolve):
        """Couple to an interior discretisation (Eq. 52).  dlx = (ptr, col, val) of
        D^{Lambda X} (n_int rows), dxl = (ptr, col, val) of D^{X Lambda} (n_unknowns rows):
        torch CUDA tensors (int32, int32, complex of the handle precision).  qsolve(inp, out,
        stream) writes Q^{-1} inp into out (torch views [nrhs, n_int] on the device), queueing
        its work on the given torch stream.  qsolve=None clears the coupling."""
        import torch
        L = load()
        if qsolve is None:
            _check(L.bi_set_coupling(self.h, 0, None, None, None, None, None, None, QSOLVE(), None), self.h)
            self._cpl = None
            return
        ts = "<c16" if self.precision == "fp64" else "<c8"
        n_int = int(n_int)
        for name, (ptr, col, val), rows in (("dlx", dlx, n_int), ("dxl", dxl, self.n_unknowns)):
            if not (ptr.is_cuda and col.is_cuda and val.is_cuda):
                raise TypeError("%s: CSR arrays must be CUDA tensors" % name)
            if ptr.dtype != torch.int32 or col.dtype != torch.int32 or val.dtype != self.cdtype:
                raise TypeError("%s: CSR arrays must be (int32, int32, %s)" % (name, self.cdtype))
            if ptr.numel() != rows + 1 or col.numel() != val.numel():
                raise ValueError("%s: ptr must have %d entries and col, val the same length" % (name, rows + 1))

        def _cb(user, pin, pout, nrhs, stream):
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                a = torch.as_tensor(_DeviceView(pin, (nrhs, n_int), ts), device="cuda")
                b = torch.as_tensor(_DeviceView(pout, (nrhs, n_int), ts), device="cuda")
                qsolve(a, b, st)

        cb = QSOLVE(_cb)
        arrs = [t.contiguous() for t in (*dlx, *dxl)]
        _check(L.bi_set_coupling(self.h, n_int, *[t.data_ptr() for t in arrs], cb, None), self.h)
        self._cpl = (cb, arrs)   # keep the callback and the arrays alive while set

    def matvec_coupled(self, x, out=None):
        """y = (C - D^{X Lambda} Q^{-1} D^{Lambda X}) x (Eq. 52's operator); queued on the stream."""
        import torch
        x = self._vec(x)
        if out is None:
            out = torch.empty_like(x)
        _check(load().bi_matvec_coupled(self.h, x.data_ptr(), out.data_ptr(), x.shape[0]), self.h)
        return out

    def status(self):
        """Synchronise and raise BIError if a product kernel gave up a bounded device wait."""
        _check(load().bi_device_status(self.h), self.h)

    def tuned_config(self):
        """Kernel forms chosen by the autotuner (one line per pass, level and E)."""
        buf = ctypes.create_string_buffer(1 << 16)
        _check(load().bi_tuned_config(self.h, buf, len(buf)), self.h)
        return buf.value.decode()

    def set_wait_limit(self, cycles):
        """Diagnostics: limit of the bulk-copy waits in SM cycles (<= 0: the default)."""
        _check(load().bi_debug_set_wait_limit(self.h, int(cycles)), self.h)

    def debug_buffer(self, what, level=0):
        """Copy of an internal device buffer (diagnostics; see bi_debug_copy in bi.h)."""
        inf = self.info()
        E = 2 * self.max_rhs
        if what in (0, 1):
            shape = (self.n_rwg, inf["K"][inf["leaf_level"]] // 2, 2)
        elif what == 2:
            shape = (343, inf["K"][level])
        elif what in (3, 4):
            shape = (inf["boxes"][level], inf["K"][level], E)
        else:
            out = np.zeros(self.n_rwg, np.int32)
            _check(load().bi_debug_copy(self.h, what, level, out.ctypes.data, out.nbytes), self.h)
            return out
        out = np.zeros(shape, self.np_cdtype)
        _check(load().bi_debug_copy(self.h, what, level, out.ctypes.data, out.nbytes), self.h)
        return out

    def farfield(self, x, dirs):
        """Far-field vectors F [nrhs, ndir, 3] (complex128, CUDA) of currents x; sigma = 4 pi |F|^2."""
        import torch
        x = self._vec(x)
        d = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(dirs), np.float64)).cuda()
        F = torch.empty((x.shape[0], d.shape[0], 3), dtype=torch.complex128, device="cuda")
        _check(load().bi_farfield(self.h, x.data_ptr(), x.shape[0], d.data_ptr(), d.shape[0], F.data_ptr()), self.h)
        return F

    def rcs(self, x, dirs):
        """Bistatic RCS sigma [nrhs, ndir] (area units) of currents x."""
        F = self.farfield(x, dirs)
        return (4 * np.pi * (F.abs() ** 2).sum(-1)).cpu().numpy()

    def close(self):
        if getattr(self, "h", None):
            load().bi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (bi_server_* in include/bi.h)."""

    def __init__(self, mem_budget_bytes=0, max_active=8, queue_capacity=4096, share_operators=True, max_batch_rhs=64,
                 setup_threads=2):
        L = load()
        p = ServerParams()
        L.bi_server_default_params(ctypes.byref(p))
        p.mem_budget_bytes = int(mem_budget_bytes)
        p.max_active = int(max_active)
        p.queue_capacity = int(queue_capacity)
        p.share_operators = int(bool(share_operators))
        p.max_batch_rhs = int(max_batch_rhs)
        p.setup_threads = int(setup_threads)
        h = ctypes.c_void_p()
        rc = L.bi_server_create(ctypes.byref(p), ctypes.byref(h))
        if rc != BI_OK:
            raise BIError(rc, "bi_server_create failed")
        self.h = h
        self._meta = {}

    def submit(self, verts, tris, k0, khat, phat, tol=1e-3, digits=3, precision="fp32", op_mode=1, leaf_box=0.25,
               levels=0, interp_order=10, gmres_restart=100, gmres_maxit=1000, precond=0):
        L = load()
        p = default_params()
        p.precond = int(precond)
        p.digits, p.leaf_box, p.levels, p.interp_order = int(digits), float(leaf_box), int(levels), int(interp_order)
        p.precision = 0 if precision == "fp64" else 1
        p.op_mode = int(op_mode)
        p.gmres_restart, p.gmres_maxit = int(gmres_restart), int(gmres_maxit)
        v = np.ascontiguousarray(verts, np.float64)
        t = np.ascontiguousarray(tris, np.int32)
        kh = np.ascontiguousarray(np.atleast_2d(khat), np.float64)
        ph = np.ascontiguousarray(np.atleast_2d(phat), np.float64)
        req = ctypes.c_int64()
        rc = L.bi_submit(self.h, v.ctypes.data, len(v), t.ctypes.data, len(t), float(k0), ctypes.byref(p), len(kh),
                         kh.ctypes.data, ph.ctypes.data, float(tol), ctypes.byref(req))
        if rc != BI_OK:
            raise BIError(rc, L.bi_server_last_error(self.h).decode())
        nt = len(t)
        nrwg = 3 * nt // 2
        self._meta[req.value] = (len(kh), nrwg * (2 if op_mode == 0 else 1), np.complex128 if precision == "fp64"
                                 else np.complex64)
        return req.value

    def poll(self, req):
        done, st = ctypes.c_int(), ctypes.c_int()
        rc = load().bi_poll(self.h, int(req), ctypes.byref(done), ctypes.byref(st))
        if rc != BI_OK:
            raise BIError(rc, "bi_poll")
        return bool(done.value), st.value

    def result(self, req):
        nrhs, nun, dt = self._meta[req]
        x = np.zeros((nrhs, nun), dt)
        its = np.zeros(nrhs, np.int32)
        rel = np.zeros(nrhs, np.float64)
        lat, st = ctypes.c_double(), ctypes.c_double()
        rc = load().bi_result(self.h, int(req), x.ctypes.data, x.nbytes, its.ctypes.data, rel.ctypes.data,
                              ctypes.byref(lat), ctypes.byref(st))
        return dict(status=rc, x=x, iters=its, relres=rel, latency_ms=lat.value, setup_ms=st.value)

    def wait(self, req, timeout=600.0):
        import time
        t0 = time.time()
        while True:
            done, st = self.poll(req)
            if done:
                return self.result(req)
            if time.time() - t0 > timeout:
                raise TimeoutError("request %d not finished" % req)
            time.sleep(0.002)

    def stats(self):
        """Server counters (SERVER_STATS names)."""
        out = np.zeros(len(SERVER_STATS), np.int64)
        _check(load().bi_server_stats(self.h, out.ctypes.data, len(out)), None)
        return dict(zip(SERVER_STATS, (int(v) for v in out)))

    def release(self, req):
        load().bi_release(self.h, int(req))
        self._meta.pop(req, None)

    def close(self):
        if getattr(self, "h", None):
            load().bi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_PLAN_DOUBLE = {20, 21, 24, 26, 30, 33, 41}


class Plan:
    """Host-only plan of the set-up (bi_plan_*): lists and tables as numpy arrays, no GPU."""

    def __init__(self, verts, tris, k0, digits=3, op_mode=0, leaf_box=0.25, levels=0, interp_order=10):
        L = load()
        p = default_params()
        p.digits, p.leaf_box, p.levels, p.interp_order = int(digits), float(leaf_box), int(levels), int(interp_order)
        p.op_mode = int(op_mode)
        k0 = complex(k0)
        p.k_im = k0.imag
        v = np.ascontiguousarray(verts, np.float64)
        t = np.ascontiguousarray(tris, np.int32)
        h = ctypes.c_void_p()
        rc = L.bi_plan_create(v.ctypes.data, len(v), t.ctypes.data, len(t), k0.real, ctypes.byref(p), ctypes.byref(h))
        if rc != BI_OK:
            raise BIError(rc, L.bi_plan_last_error().decode())
        self.h = h

    def info(self) -> dict:
        I = Info()
        _check(load().bi_plan_info(self.h, ctypes.byref(I)), None)
        nl = I.levels
        return dict(n_rwg=I.n_rwg, n_unknowns=I.n_unknowns, levels=nl, leaf_level=I.leaf_level,
                    boxes=list(I.boxes[:nl]), L=list(I.L[:nl]), K=list(I.K[:nl]), near_pairs=I.near_pairs,
                    interactions=list(I.interactions[:nl]), root_size=I.root_size)

    def get(self, what, level=0):
        L = load()
        n = ctypes.c_int64()
        rc = L.bi_plan_get(self.h, int(what), int(level), None, 0, ctypes.byref(n))
        if rc != BI_OK:
            raise BIError(rc, "bi_plan_get(%d, %d)" % (what, level))
        out = np.zeros(n.value, np.float64 if what in _PLAN_DOUBLE else np.int32)
        _check(L.bi_plan_get(self.h, int(what), int(level), out.ctypes.data, out.nbytes, ctypes.byref(n)), None)
        return out

    def close(self):
        if self.h:
            load().bi_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
