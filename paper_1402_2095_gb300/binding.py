"""Thin Python binding of libfth.so (the C ABI declared in include/fth.h).

Argument marshalling only: every step of the f-thermostat path runs in the
library's CUDA kernels.  PyTorch supplies the device workspace (one uint8 tensor)
and the CUDA stream.  There is no CPU fallback: if libfth.so is missing the import
of this module's FTH class fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfth.so")

FTH_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "UNSUPPORTED", 4: "WORKSPACE", 5: "CUDA",
          6: "TIMEOUT", 7: "NONFINITE", 8: "NOT_TRACKED"}
DENSE, CSR = 0, 1
F32, F64 = 0, 1
PRECISION = {"fp32": 0, "tf32": 1, "bf16x3": 2, "fp64": 3}
TRACK = {"list": 0, "diag": 1, "all": 2}
OBSERVABLE = {"p": 0, "q": 1}
PLANE = {"q": 0, "p": 1, "s": 2}

# Every symbol include/fth.h declares.
EXPORTS = ("fth_workspace_size", "fth_create", "fth_run", "fth_elements", "fth_get_state",
           "fth_set_state", "fth_info", "fth_status_poll", "fth_last_error", "fth_destroy",
           "fth_gle_propagator", "fth_version", "fth_profile_enable", "fth_profile_read",
           "fth_dense_step_noalloc", "fth_pool_create", "fth_pool_footprint", "fth_pool_add",
           "fth_pool_remove", "fth_pool_run", "fth_pool_elements", "fth_pool_get_state",
           "fth_pool_problem_info",
           "fth_pool_stats", "fth_pool_profile", "fth_pool_progress", "fth_pool_last_error",
           "fth_pool_destroy", "fth_server_create", "fth_server_submit", "fth_server_step",
           "fth_server_result", "fth_server_clock", "fth_server_pool", "fth_server_last_error",
           "fth_server_destroy", "fth_functional_bytes", "fth_functional_add", "fth_functional",
           "fth_test_stall", "fth_fit_gle", "fth_gle_response", "fth_functional_operator_terms",
           "fth_functional_add_operator", "fth_spectral_map", "fth_gle_scale", "fth_untransform",
           "fth_untransform_trace")
KERNEL_CLASSES = ("force_fp32", "force_tc", "gle_dense", "csr_step", "pair_accum", "syrk_fp32",
                  "syrk_tc", "flush", "fp64_dense", "fp64_noise")


class FthError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fth: {STATUS.get(status, status)}: {msg}")
        self.status = status


class fth_matrix(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("on_device", ctypes.c_int),
                ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("values", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p)]


class fth_gle(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("a_p", ctypes.c_double * 25), ("c_p", ctypes.c_double * 25)]


class fth_options(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int64), ("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("burnin", ctypes.c_int64), ("block", ctypes.c_int64), ("observable", ctypes.c_int),
                ("precision", ctypes.c_int), ("track", ctypes.c_int), ("pairs", ctypes.c_void_p),
                ("npairs", ctypes.c_int64), ("stack", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("replica_offset", ctypes.c_int64)]


class fth_pool_options(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int64), ("precision", ctypes.c_int),
                ("max_problems", ctypes.c_int64), ("graph_steps", ctypes.c_int64),
                ("stream", ctypes.c_void_p)]


class fth_problem_options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dt", ctypes.c_double), ("burnin", ctypes.c_int64),
                ("block", ctypes.c_int64), ("observable", ctypes.c_int), ("pairs", ctypes.c_void_p),
                ("npairs", ctypes.c_int64), ("replica_offset", ctypes.c_int64)]


class fth_pool_stats_t(ctypes.Structure):
    _fields_ = [("live", ctypes.c_int64), ("slab_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t), ("force_items", ctypes.c_int64),
                ("gle_items", ctypes.c_int64), ("csr_items", ctypes.c_int64),
                ("tuned_variant", ctypes.c_int), ("tuned_grid", ctypes.c_int),
                ("tuned_us", ctypes.c_double), ("gle_variant", ctypes.c_int),
                ("gle_us", ctypes.c_double), ("graphs", ctypes.c_int64)]


class fth_server_options(ctypes.Structure):
    _fields_ = [("pool", fth_pool_options), ("chunk_steps", ctypes.c_int64),
                ("min_blocks", ctypes.c_int64), ("max_bypass", ctypes.c_int64)]


class fth_server_counts(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("retired", ctypes.c_int64),
                ("running", ctypes.c_int64), ("queued", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("used_bytes", ctypes.c_size_t), ("slab_bytes", ctypes.c_size_t)]


class fth_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("steps", ctypes.c_int64), ("rel_err", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("npairs", ctypes.c_int64)]


REQUEST_STATE = {0: "queued", 1: "running", 2: "done", 3: "budget", 4: "failed"}


class fth_fit_options(ctypes.Structure):
    _fields_ = [("observable", ctypes.c_int), ("npts", ctypes.c_int), ("starts", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("delta", ctypes.c_double), ("w_tau", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("threads", ctypes.c_int), ("objective", ctypes.c_int)]


class fth_fit_report(ctypes.Structure):
    _fields_ = [("max_rel_err", ctypes.c_double), ("rms_rel_err", ctypes.c_double),
                ("max_abs_err", ctypes.c_double), ("tail_max", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("lambda_tau_max", ctypes.c_double),
                ("cost", ctypes.c_double), ("evaluations", ctypes.c_int64), ("grid", ctypes.c_int),
                ("objective", ctypes.c_int)]


FUNCTION = {"inv_sqrt": 0, "fermi": 1, "log": 2, "exp": 3, "power": 4}
FIT_OBJECTIVE = {"auto": 0, "log": 1, "abs": 2}


class fth_info_t(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("accumulated", ctypes.c_int64), ("blocks", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("primed", ctypes.c_int), ("precision", ctypes.c_int),
                ("n", ctypes.c_int64), ("replicas", ctypes.c_int64), ("tracked", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfth.so and declare its signatures; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FthError(5, f"{path} not found: build it with paper_1402_2095_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    P, I64, INT, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "fth_workspace_size": ([P, P, P, P], INT),
        "fth_create": ([P, P, P, P, ctypes.c_size_t, P], INT),
        "fth_run": ([P, I64], INT),
        "fth_elements": ([P, P, I64, P, P], INT),
        "fth_get_state": ([P, INT, P], INT),
        "fth_set_state": ([P, INT, P], INT),
        "fth_info": ([P, P], INT),
        "fth_status_poll": ([P], INT),
        "fth_last_error": ([P], ctypes.c_char_p),
        "fth_destroy": ([P], None),
        "fth_gle_propagator": ([P, D, P, P], INT),
        "fth_version": ([], ctypes.c_char_p),
        "fth_profile_enable": ([P, INT], INT),
        "fth_profile_read": ([P, P, P], INT),
        "fth_test_stall": ([P, ctypes.c_uint64], INT),
        "fth_fit_gle": ([INT, P, D, D, INT, D, P, P, P], INT),
        "fth_gle_response": ([P, D, INT, P, I64, P, P], INT),
        "fth_functional_operator_terms": ([P, P, P], INT),
        "fth_functional_add_operator": ([P, P, P, ctypes.c_size_t, P], INT),
        "fth_spectral_map": ([D, D, D, D, P, P], INT),
        "fth_gle_scale": ([P, D, D, P], INT),
        "fth_untransform": ([INT, P, P, I64, P, P], INT),
        "fth_untransform_trace": ([INT, P, I64, P, P], INT),
        "fth_dense_step_noalloc": ([P, I64, I64, P, P, P, I64, I64, INT, P, P, D,
                                    ctypes.c_uint64, ctypes.c_uint32, INT, P, P], INT),
        "fth_pool_create": ([P, P, ctypes.c_size_t, P], INT),
        "fth_pool_footprint": ([P, P, P, P, P], INT),
        "fth_pool_add": ([P, P, P, P, P], INT),
        "fth_pool_remove": ([P, I64], INT),
        "fth_pool_run": ([P, I64], INT),
        "fth_pool_elements": ([P, I64, P, I64, P, P], INT),
        "fth_pool_get_state": ([P, I64, INT, P], INT),
        "fth_pool_problem_info": ([P, I64, P], INT),
        "fth_pool_stats": ([P, P], INT),
        "fth_pool_profile": ([P, I64, P, P], INT),
        "fth_pool_progress": ([P, P, P], INT),
        "fth_functional_bytes": ([I64], ctypes.c_size_t),
        "fth_functional_add": ([P, P, P, I64, P, ctypes.c_size_t, P], INT),
        "fth_functional": ([P, I64, P, P], INT),
        "fth_server_create": ([P, P, ctypes.c_size_t, P], INT),
        "fth_server_submit": ([P, P, P, P, D, I64, P], INT),
        "fth_server_step": ([P, P], INT),
        "fth_server_result": ([P, I64, P, P, P], INT),
        "fth_server_clock": ([P], D),
        "fth_server_pool": ([P], P),
        "fth_server_last_error": ([P], ctypes.c_char_p),
        "fth_server_destroy": ([P], None),
        "fth_pool_last_error": ([P], ctypes.c_char_p),
        "fth_pool_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status, ctx=None):
    if status != FTH_OK:
        msg = load().fth_last_error(ctx)
        raise FthError(status, msg.decode() if msg else "")


def make_gle(a_p, c_p) -> fth_gle:
    a_p = np.asarray(a_p, dtype=np.float64)
    c_p = np.asarray(c_p, dtype=np.float64)
    ns = a_p.shape[0]
    g = fth_gle()
    g.s = ns - 1
    for k, x in enumerate(a_p.ravel()):
        g.a_p[k] = x
    for k, x in enumerate(c_p.ravel()):
        g.c_p[k] = x
    return g


def gle_propagator(a_p, c_p, dt):
    """The library's own FP64 (T, S) of the O half-step."""
    g = make_gle(a_p, c_p)
    ns = g.s + 1
    T = np.zeros(ns * ns)
    S = np.zeros(ns * ns)
    _check(load().fth_gle_propagator(ctypes.byref(g), dt, T.ctypes.data, S.ctypes.data))
    return T.reshape(ns, ns), S.reshape(ns, ns)


def fit_gle(kind, params, lam_min, lam_max, dt, s=4, *, observable="p", npts=120, starts=6,
            max_iter=400, delta=1e-3, w_tau=0.2, seed=0, threads=0, objective="auto"):
    """fth_fit_gle: (a_p, c_p, report dict) of the GLE fitted to f over [lam_min, lam_max]."""
    o = fth_fit_options()
    o.observable = OBSERVABLE[observable]
    o.npts, o.starts, o.max_iter = int(npts), int(starts), int(max_iter)
    o.delta, o.w_tau = float(delta), float(w_tau)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.threads = int(threads)
    o.objective = FIT_OBJECTIVE[objective]
    par = np.ascontiguousarray(np.asarray(list(params) + [0.0] * 4, dtype=np.float64))
    out = fth_gle()
    rep = fth_fit_report()
    _check(load().fth_fit_gle(FUNCTION[kind], par.ctypes.data, float(lam_min), float(lam_max),
                              int(s), float(dt), ctypes.byref(o), ctypes.byref(out),
                              ctypes.byref(rep)))
    ns = out.s + 1
    a = np.array(out.a_p[:ns * ns]).reshape(ns, ns)
    c = np.array(out.c_p[:ns * ns]).reshape(ns, ns)
    r = {f: getattr(rep, f) for f, _ in fth_fit_report._fields_}
    r["objective"] = {1: "log", 2: "abs"}.get(r["objective"], r["objective"])
    return a, c, r


def gle_response(a_p, c_p, dt, lams, observable="p", tau=False):
    """fth_gle_response: exact per-mode <x^2> of the integrator (and its correlation time
    of x^2 in samples when tau=True) for each eigenvalue."""
    g = make_gle(a_p, c_p)
    lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lams, dtype=np.float64)))
    out = np.zeros(lam.size)
    t = np.zeros(lam.size) if tau else None
    _check(load().fth_gle_response(ctypes.byref(g), float(dt), OBSERVABLE[observable],
                                   lam.ctypes.data, lam.size, out.ctypes.data,
                                   t.ctypes.data if tau else None))
    return (out, t) if tau else out


class FTH:
    """One f-thermostat problem instance on the current CUDA device.

    M: dense (N x N numpy array or torch tensor, host or device) or csr=(rowptr, col,
    val, n).  a_p, c_p: the fitted GLE.  The workspace is a torch uint8 tensor held by
    this object; work runs on `stream` (default: torch's current stream)."""

    def __init__(self, M=None, csr=None, *, a_p, c_p, dt, replicas, seed=0, burnin=0,
                 block=1000, observable="p", precision="fp32", track="list", pairs=None,
                 stack=0, stream=None, replica_offset=0):
        import torch

        L = load()
        self._keep = []
        mat = fth_matrix()
        if (M is None) == (csr is None):
            raise ValueError("give exactly one of M or csr")
        if M is not None:
            mat.kind = DENSE
            if isinstance(M, torch.Tensor):
                t = M.contiguous()
                mat.dtype = F64 if t.dtype == torch.float64 else F32
                if t.dtype not in (torch.float32, torch.float64):
                    t = t.float()
                mat.on_device = 1 if t.is_cuda else 0
                mat.values = t.data_ptr()
                mat.n = t.shape[0]
                self._keep.append(t)
            else:
                a = np.ascontiguousarray(M)
                if a.dtype not in (np.float32, np.float64):
                    a = a.astype(np.float64)
                mat.dtype = F64 if a.dtype == np.float64 else F32
                mat.on_device = 0
                mat.values = a.ctypes.data
                mat.n = a.shape[0]
                self._keep.append(a)
        else:
            rowptr, col, val, n = csr
            rp = np.ascontiguousarray(rowptr, dtype=np.int32)
            ci = np.ascontiguousarray(col, dtype=np.int32)
            va = np.ascontiguousarray(val)
            if va.dtype not in (np.float32, np.float64):
                va = va.astype(np.float64)
            mat.kind = CSR
            mat.dtype = F64 if va.dtype == np.float64 else F32
            mat.on_device = 0
            mat.n = int(n)
            mat.nnz = int(ci.size)
            mat.values = va.ctypes.data
            mat.rowptr = rp.ctypes.data
            mat.colind = ci.ctypes.data
            self._keep += [rp, ci, va]
        self.n = int(mat.n)
        self.replicas = int(replicas)
        gle = make_gle(a_p, c_p)
        self.s = gle.s
        opt = fth_options()
        opt.replicas = int(replicas)
        opt.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        opt.dt = float(dt)
        opt.burnin = int(burnin)
        opt.block = int(block)
        opt.observable = OBSERVABLE[observable]
        opt.precision = PRECISION[precision]
        opt.track = TRACK[track]
        if pairs is not None:
            pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
            self._keep.append(pr)
            opt.pairs = pr.ctypes.data
            opt.npairs = pr.shape[0]
        opt.stack = int(stack)
        opt.replica_offset = int(replica_offset)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt.stream = self.stream.cuda_stream
        nbytes = ctypes.c_size_t(0)
        _check(L.fth_workspace_size(ctypes.byref(mat), ctypes.byref(gle), ctypes.byref(opt),
                                    ctypes.byref(nbytes)))
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8,
                                         device="cuda")
        ctx = ctypes.c_void_p()
        _check(L.fth_create(ctypes.byref(mat), ctypes.byref(gle), ctypes.byref(opt),
                            self.workspace.data_ptr(), self.workspace.numel(), ctypes.byref(ctx)))
        self.ctx = ctx
        self._func_bufs = []
        self._keep_inputs = self._keep  # host copies are only read during create
        self._keep = []

    # -------------------------------------------------------------- hot path
    def run(self, steps: int):
        _check(load().fth_run(self.ctx, int(steps)), self.ctx)

    def elements(self, pairs):
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        k = pr.shape[0]
        vals = np.zeros(k)
        errs = np.zeros(k)
        _check(load().fth_elements(self.ctx, pr.ctypes.data, k, vals.ctypes.data, errs.ctypes.data),
               self.ctx)
        return vals, errs

    # -------------------------------------------------------------- state
    def get_state(self, plane: str):
        shape = (self.replicas, self.s, self.n) if plane == "s" else (self.replicas, self.n)
        out = np.zeros(shape)
        if out.size:
            _check(load().fth_get_state(self.ctx, PLANE[plane], out.ctypes.data), self.ctx)
        return out

    def set_state(self, plane: str, arr):
        shape = (self.replicas, self.s, self.n) if plane == "s" else (self.replicas, self.n)
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(shape))
        if a.size:
            _check(load().fth_set_state(self.ctx, PLANE[plane], a.ctypes.data), self.ctx)

    def add_functional(self, pairs, weights):
        """Register L = sum_k w_k <x_i x_j> over tracked pairs (before the first sample);
        returns its id.  add_trace() builds the terms of Tr f(M) and Tr O f(M)."""
        import torch
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
        if w.shape[0] != pr.shape[0]:
            raise ValueError("one weight per pair")
        L = load()
        nbytes = int(L.fth_functional_bytes(pr.shape[0]))
        with torch.cuda.stream(self.stream):
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (buf.data_ptr() + 255) // 256 * 256
        fid = ctypes.c_int64(-1)
        _check(L.fth_functional_add(self.ctx, pr.ctypes.data, w.ctypes.data, pr.shape[0], ptr,
                                    nbytes, ctypes.byref(fid)), self.ctx)
        self._func_bufs.append(buf)
        return int(fid.value)

    def add_trace(self, O=None):
        """Register Tr O f(M) = <p^T O p> (O symmetric: dense array, torch tensor, scipy
        sparse matrix or csr=(rowptr, col, val, n) tuple; None: Tr f(M)); the weights are
        built by the library (fth_functional_add_operator).  Returns the functional's id."""
        import torch
        L = load()
        keep = []
        optr = None
        if O is not None:
            try:
                import scipy.sparse as sp
                if sp.issparse(O):
                    C = sp.csr_matrix(O)
                    O = {"csr": (C.indptr, C.indices, C.data, C.shape[0])}
            except ImportError:
                pass
            if isinstance(O, dict):
                mat = _matrix_struct(csr=O["csr"], keep=keep)
            elif isinstance(O, tuple):
                mat = _matrix_struct(csr=O, keep=keep)
            else:
                mat = _matrix_struct(M=O, keep=keep)
            optr = ctypes.byref(mat)
        nt = ctypes.c_int64(0)
        _check(L.fth_functional_operator_terms(self.ctx, optr, ctypes.byref(nt)), self.ctx)
        nbytes = int(L.fth_functional_bytes(nt.value))
        with torch.cuda.stream(self.stream):
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (buf.data_ptr() + 255) // 256 * 256
        fid = ctypes.c_int64(-1)
        _check(L.fth_functional_add_operator(self.ctx, optr, ptr, nbytes, ctypes.byref(fid)),
               self.ctx)
        self._func_bufs.append(buf)
        return int(fid.value)

    def functional(self, fid):
        """(value, block error bar) of a registered functional."""
        v = ctypes.c_double()
        e = ctypes.c_double()
        _check(load().fth_functional(self.ctx, int(fid), ctypes.byref(v), ctypes.byref(e)), self.ctx)
        return v.value, e.value

    def info(self) -> dict:
        i = fth_info_t()
        _check(load().fth_info(self.ctx, ctypes.byref(i)), self.ctx)
        return {f: getattr(i, f) for f, _ in fth_info_t._fields_}

    def profile(self, enable: bool = True):
        """Turn per-launch CUDA-event timing on or off."""
        _check(load().fth_profile_enable(self.ctx, 1 if enable else 0), self.ctx)

    def profile_read(self) -> dict:
        """{kernel class: (total device ms, launches)} since the last read."""
        n = len(KERNEL_CLASSES)
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        _check(load().fth_profile_read(self.ctx, ms.ctypes.data, cnt.ctypes.data), self.ctx)
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES) if cnt[i]}

    def poll(self):
        _check(load().fth_status_poll(self.ctx), self.ctx)

    def test_stall(self, limit_ns: int):
        """Test hook: later force launches end through the device timeout path."""
        _check(load().fth_test_stall(self.ctx, int(limit_ns)), self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            load().fth_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------- problem pools
def _matrix_struct(M=None, csr=None, keep=None):
    import torch
    mat = fth_matrix()
    if M is not None:
        mat.kind = DENSE
        if isinstance(M, torch.Tensor):
            t = M.contiguous()
            if t.dtype not in (torch.float32, torch.float64):
                t = t.float()
            mat.dtype = F64 if t.dtype == torch.float64 else F32
            mat.on_device = 1 if t.is_cuda else 0
            mat.values = t.data_ptr()
            mat.n = t.shape[0]
            keep.append(t)
        else:
            a = np.ascontiguousarray(M)
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
            mat.dtype = F64 if a.dtype == np.float64 else F32
            mat.values = a.ctypes.data
            mat.n = a.shape[0]
            keep.append(a)
    else:
        rowptr, col, val, n = csr
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        va = np.ascontiguousarray(val)
        if va.dtype not in (np.float32, np.float64):
            va = va.astype(np.float64)
        mat.kind = CSR
        mat.dtype = F64 if va.dtype == np.float64 else F32
        mat.n = int(n)
        mat.nnz = int(ci.size)
        mat.values = va.ctypes.data
        mat.rowptr = rp.ctypes.data
        mat.colind = ci.ctypes.data
        keep += [rp, ci, va]
    return mat


def _pool_check(status, pool):
    if status != FTH_OK:
        msg = load().fth_pool_last_error(pool)
        raise FthError(status, msg.decode() if msg else "")


class Pool:
    """Many independent problems resident on the GPU, stepped together (ragged batches,
    continuous batching).  `workspace_bytes` of device memory (a torch tensor) is the
    admission capacity."""

    def __init__(self, workspace_bytes, *, replicas=32, precision="bf16x3", max_problems=1024,
                 graph_steps=0, stream=None):
        import torch
        L = load()
        # a stream of its own by default: graphs cannot be captured on the legacy stream
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._aux = {}
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device="cuda")
        o = fth_pool_options()
        o.replicas = int(replicas)
        o.precision = PRECISION[precision]
        o.max_problems = int(max_problems)
        o.graph_steps = int(graph_steps)
        o.stream = self.stream.cuda_stream
        self.replicas = int(replicas)
        self.max_problems = int(max_problems)
        h = ctypes.c_void_p()
        _check(L.fth_pool_create(ctypes.byref(o), self.workspace.data_ptr(), self.workspace.numel(),
                                 ctypes.byref(h)))
        self.pool = h

    def _problem(self, M, csr, a_p, c_p, dt, seed, burnin, block, observable, pairs,
                 replica_offset):
        keep = []
        mat = _matrix_struct(M, csr, keep)
        gle = make_gle(a_p, c_p)
        po = fth_problem_options()
        po.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        po.dt = float(dt)
        po.burnin = int(burnin)
        po.block = int(block)
        po.observable = OBSERVABLE[observable]
        pr = np.ascontiguousarray(np.asarray(pairs if pairs is not None else np.zeros((0, 2)),
                                             dtype=np.int64).reshape(-1, 2))
        keep.append(pr)
        po.pairs = pr.ctypes.data
        po.npairs = pr.shape[0]
        po.replica_offset = int(replica_offset)
        return mat, gle, po, keep

    def footprint(self, M=None, csr=None, *, a_p, c_p, dt, pairs=None, **kw):
        mat, gle, po, keep = self._problem(M, csr, a_p, c_p, dt, 0, 0, 1, "p", pairs, 0)
        b = ctypes.c_size_t(0)
        _pool_check(load().fth_pool_footprint(self.pool, ctypes.byref(mat), ctypes.byref(gle),
                                              ctypes.byref(po), ctypes.byref(b)), self.pool)
        return int(b.value)

    def add(self, M=None, csr=None, *, a_p, c_p, dt, seed=0, burnin=0, block=1000,
            observable="p", pairs=None, replica_offset=0):
        """Admit a problem; returns its handle.  Raises FthError(WORKSPACE) if it does
        not fit."""
        mat, gle, po, keep = self._problem(M, csr, a_p, c_p, dt, seed, burnin, block, observable,
                                           pairs, replica_offset)
        h = ctypes.c_int64(-1)
        _pool_check(load().fth_pool_add(self.pool, ctypes.byref(mat), ctypes.byref(gle),
                                        ctypes.byref(po), ctypes.byref(h)), self.pool)
        self._aux[int(h.value)] = int(gle.s)
        return int(h.value)

    def remove(self, handle):
        _pool_check(load().fth_pool_remove(self.pool, int(handle)), self.pool)
        self._aux.pop(int(handle), None)

    def run(self, steps):
        _pool_check(load().fth_pool_run(self.pool, int(steps)), self.pool)

    def elements(self, handle, pairs):
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        k = pr.shape[0]
        vals = np.zeros(k)
        errs = np.zeros(k)
        _pool_check(load().fth_pool_elements(self.pool, int(handle), pr.ctypes.data, k,
                                             vals.ctypes.data, errs.ctypes.data), self.pool)
        return vals, errs

    def get_state(self, handle, plane: str):
        """State plane of one problem: q, p as (R, n); s as (R, s, n)."""
        info = self.info(handle)
        n = int(info["n"])
        if plane == "s":
            ns = self._aux[handle]
            out = np.zeros((self.replicas, ns, n))
        else:
            out = np.zeros((self.replicas, n))
        if out.size:
            _pool_check(load().fth_pool_get_state(self.pool, int(handle), PLANE[plane],
                                                  out.ctypes.data), self.pool)
        return out

    def info(self, handle) -> dict:
        i = fth_info_t()
        _pool_check(load().fth_pool_problem_info(self.pool, int(handle), ctypes.byref(i)), self.pool)
        return {f: getattr(i, f) for f, _ in fth_info_t._fields_}

    def stats(self) -> dict:
        s = fth_pool_stats_t()
        _check(load().fth_pool_stats(self.pool, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in fth_pool_stats_t._fields_}

    POOL_KERNELS = ("pool_force", "pool_gle", "pool_csr", "pool_accum")

    def profile(self, steps):
        """Run `steps` real steps with each launch timed: {class: (total ms, launches)}."""
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int64)
        _pool_check(load().fth_pool_profile(self.pool, int(steps), ms.ctypes.data, cnt.ctypes.data),
                    self.pool)
        return {k: (float(ms[c]), int(cnt[c])) for c, k in enumerate(self.POOL_KERNELS) if cnt[c]}

    def progress(self):
        """(rel_err, blocks) per handle slot: normwise relative error bar over each
        problem's tracked elements (NaN before 2 blocks / empty slot), complete blocks."""
        n = self.max_problems
        rel = np.zeros(n)
        blk = np.zeros(n, dtype=np.int64)
        _pool_check(load().fth_pool_progress(self.pool, rel.ctypes.data, blk.ctypes.data), self.pool)
        return rel, blk

    def close(self):
        if getattr(self, "pool", None):
            load().fth_pool_destroy(self.pool)
            self.pool = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------- serving loop
class Server:
    """Continuous-batching serving loop over a pool (C++ in libfth): submit requests at
    any time, call step() repeatedly; each step admits what fits, runs chunk_steps steps
    of everything admitted and retires what met its target."""

    def __init__(self, workspace_bytes, *, replicas=32, precision="bf16x3", max_problems=256,
                 graph_steps=0, chunk_steps=500, min_blocks=4, max_bypass=8, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device="cuda")
        o = fth_server_options()
        o.pool.replicas = int(replicas)
        o.pool.precision = PRECISION[precision]
        o.pool.max_problems = int(max_problems)
        o.pool.graph_steps = int(graph_steps)
        o.pool.stream = self.stream.cuda_stream
        o.chunk_steps = int(chunk_steps)
        o.min_blocks = int(min_blocks)
        o.max_bypass = int(max_bypass)
        h = ctypes.c_void_p()
        _check(load().fth_server_create(ctypes.byref(o), self.workspace.data_ptr(),
                                        self.workspace.numel(), ctypes.byref(h)))
        self.srv = h
        self.replicas = int(replicas)
        self._np = {}

    def _err(self, st):
        if st != FTH_OK:
            msg = load().fth_server_last_error(self.srv)
            raise FthError(st, msg.decode() if msg else "")

    def submit(self, M=None, csr=None, *, a_p, c_p, dt, target, max_steps=0, seed=0, burnin=0,
               block=1000, observable="p", pairs, replica_offset=0):
        keep = []
        mat = _matrix_struct(M, csr, keep)
        gle = make_gle(a_p, c_p)
        po = fth_problem_options()
        po.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        po.dt = float(dt)
        po.burnin = int(burnin)
        po.block = int(block)
        po.observable = OBSERVABLE[observable]
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        po.pairs = pr.ctypes.data
        po.npairs = pr.shape[0]
        po.replica_offset = int(replica_offset)
        rid = ctypes.c_int64(-1)
        self._err(load().fth_server_submit(self.srv, ctypes.byref(mat), ctypes.byref(gle),
                                           ctypes.byref(po), float(target), int(max_steps),
                                           ctypes.byref(rid)))
        self._np[int(rid.value)] = pr.shape[0]
        return int(rid.value)

    def step(self) -> dict:
        c = fth_server_counts()
        self._err(load().fth_server_step(self.srv, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in fth_server_counts._fields_}

    def result(self, rid):
        """(info dict, values, errbars); values/errbars are None until retired."""
        info = fth_request_info()
        k = self._np[int(rid)]
        vals = np.full(k, np.nan)
        errs = np.full(k, np.nan)
        self._err(load().fth_server_result(self.srv, int(rid), ctypes.byref(info),
                                           vals.ctypes.data, errs.ctypes.data))
        d = {f: getattr(info, f) for f, _ in fth_request_info._fields_}
        d["state"] = REQUEST_STATE[d["state"]]
        if d["state"] in ("done", "budget"):
            return d, vals, errs
        return d, None, None

    def clock(self) -> float:
        return load().fth_server_clock(self.srv)

    def close(self):
        if getattr(self, "srv", None):
            load().fth_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------- transforms
UNTRANSFORM = {"log": 0, "exp": 1, "power": 2}


def spectral_map(spec, target):
    """fth_spectral_map: (r, m) with r spec[0] + m = target[0], r spec[1] + m = target[1]."""
    r, m = ctypes.c_double(), ctypes.c_double()
    _check(load().fth_spectral_map(float(spec[0]), float(spec[1]), float(target[0]),
                                   float(target[1]), ctypes.byref(r), ctypes.byref(m)))
    return r.value, m.value


def gle_scale(a_p, c_p, alpha=1.0, gamma=1.0):
    """fth_gle_scale: (alpha A_p, gamma C_p)."""
    g = make_gle(a_p, c_p)
    _check(load().fth_gle_scale(ctypes.byref(g), float(alpha), float(gamma), ctypes.byref(g)))
    ns = g.s + 1
    return (np.array(g.a_p[:ns * ns]).reshape(ns, ns), np.array(g.c_p[:ns * ns]).reshape(ns, ns))


def untransform(kind, params, pairs, values, errbars=None):
    """fth_untransform: wanted elements from sampled ones ("log": params (r,), "exp":
    (a, m), "power": (r, k)); returns (values, errbars) as new arrays."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    v = np.array(values, dtype=np.float64, copy=True).reshape(-1)
    e = None if errbars is None else np.array(errbars, dtype=np.float64, copy=True).reshape(-1)
    par = np.ascontiguousarray(np.asarray(list(params) + [0.0] * 2, dtype=np.float64))
    _check(load().fth_untransform(UNTRANSFORM[kind], par.ctypes.data, pr.ctypes.data, pr.shape[0],
                                  v.ctypes.data, None if e is None else e.ctypes.data))
    return v, e


def untransform_trace(kind, params, n, value, errbar=None):
    """fth_untransform_trace: the wanted trace (and its error bar) from the sampled one."""
    par = np.ascontiguousarray(np.asarray(list(params) + [0.0] * 2, dtype=np.float64))
    v = ctypes.c_double(float(value))
    e = ctypes.c_double(float(errbar) if errbar is not None else 0.0)
    _check(load().fth_untransform_trace(UNTRANSFORM[kind], par.ctypes.data, int(n),
                                        ctypes.byref(v), ctypes.byref(e)))
    return (v.value, e.value) if errbar is not None else v.value
