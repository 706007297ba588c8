"""ctypes binding of libspnet (include/spnet.h): argument marshalling only.

Arrays may be numpy arrays (host memory, SPNET_MEM_HOST) or CUDA torch
tensors (device memory, SPNET_MEM_DEVICE); every computation runs in the
library's CUDA kernels.  If the library is missing or cannot be loaded the
import of the handles raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERRORS = {
    -1: "BAD_INPUT", -2: "NOT_SPD", -3: "NO_MEMORY", -4: "NO_CONVERGENCE", -5: "TIMEOUT",
    -6: "CUDA", -7: "UNSUPPORTED", -8: "BAD_H",
}
ERR_BAD_INPUT, ERR_NOT_SPD, ERR_NO_MEMORY, ERR_NO_CONVERGENCE = -1, -2, -3, -4
ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, ERR_BAD_H = -5, -6, -7, -8
ERR_CANCELLED = -9
MEM_HOST, MEM_DEVICE = 0, 1
MODEL_SCALAR, MODEL_TRUSS3 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
STARS_INTERIOR, STARS_ALL = 0, 1
PATCH_ELEMENT, PATCH_SUPPORT = 0, 1
COARSE_Q1, COARSE_P1 = 0, 1
EXPORT_ELEMENTS, EXPORT_Q1, EXPORT_COARSE_MAP, EXPORT_STAR_SIZES = 0, 1, 2, 3
EXPORT_STAR_MESH, EXPORT_A0, EXPORT_STAR_LEVELS, EXPORT_STAR_CORE = 4, 5, 6, 7

EXPORTED = [
    "spnet_assemble", "build_network_operator", "setup_preconditioner", "pcg_solve",
    "spnet_op_destroy", "spnet_pc_destroy", "spnet_last_error", "spnet_op_get_info",
    "spnet_pc_get_info", "spnet_spmv", "spnet_pc_apply", "spnet_pc_restrict", "spnet_pc_coarse",
    "spnet_pc_prolong", "spnet_pc_stars", "spnet_pc_export", "spnet_launch_count",
    "spnet_profile_enable", "spnet_profile_read", "spnet_profile_reset", "spnet_pc_restrict_static",
    "spnet_pc_record_iterates",
    "spnet_server_create", "spnet_server_submit", "spnet_server_wait", "spnet_server_destroy",
    "spnet_pc_apply_batch", "spnet_server_poll", "spnet_server_cancel", "spnet_server_estimate",
    "spnet_server_budget", "spnet_tune_cache_load", "spnet_tune_cache_save", "spnet_tune_cache_clear",
    "spnet_tune_counts", "spnet_assemble_beam",
]
KERNELS = ["spmv", "update", "restrict", "stars", "coarse", "combine", "direction",
           "star_symbolic", "star_numeric", "sweep", "galerkin"]


class SpnetError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("star_set", C.c_int), ("flexible", C.c_int),
                ("max_restarts", C.c_int), ("batch_rhs", C.c_int), ("star_map", C.c_int),
                ("patch", C.c_int), ("no_panels", C.c_int), ("coarse_space", C.c_int), ("reserved", C.c_int * 7)]


class Request(C.Structure):
    _fields_ = [("model", C.c_int), ("dim", C.c_int), ("n_nodes", C.c_int64), ("n_edges", C.c_int64),
                ("edges", C.c_void_p), ("coef", C.c_void_p), ("dirs", C.c_void_p), ("coords", C.c_void_p),
                ("domain_hi", C.c_double * 3), ("n_dirichlet", C.c_int64), ("dirichlet_dofs", C.c_void_p),
                ("nrhs", C.c_int), ("f", C.c_void_p), ("g", C.c_void_p), ("x", C.c_void_p),
                ("H", C.c_double), ("gamma_faces", C.c_int * 3), ("opts", Options), ("rtol", C.c_double),
                ("maxit", C.c_int), ("reserved", C.c_int * 7)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("relres", C.c_double),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double), ("device_start_ms", C.c_double),
                ("device_end_ms", C.c_double), ("message", C.c_char * 256)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("status", C.c_int), ("relres", C.c_double), ("relres_recursive", C.c_double),
                ("solve_ms", C.c_double), ("reserved", C.c_double * 4)]


class OpInfo(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("n_free", C.c_int64), ("n_dirichlet", C.c_int64),
                ("nnz_ff", C.c_int64), ("nnz_fd", C.c_int64), ("dim", C.c_int), ("ndof", C.c_int),
                ("reserved", C.c_int64 * 6)]


class PcInfo(C.Structure):
    _fields_ = [("nH", C.c_int * 3), ("n_elem", C.c_int), ("n_mesh", C.c_int), ("m0", C.c_int),
                ("n_stars", C.c_int), ("max_star", C.c_int), ("sum_star", C.c_int64),
                ("factor_nnz", C.c_int64), ("total_levels", C.c_int64), ("max_levels", C.c_int),
                ("precision", C.c_int), ("star_set", C.c_int), ("flexible", C.c_int),
                ("setup_ms", C.c_double), ("device_bytes", C.c_int64), ("star_stream_bytes", C.c_int64),
                ("star_warps_per_block", C.c_int64), ("coarse_dropped", C.c_int64),
                ("panel_stars", C.c_int64), ("tuned", C.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libspnet.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libspnet is not built ({path} missing)")
    lib = C.CDLL(path)
    P = C.c_void_p
    i64, i32, dbl = C.c_int64, C.c_int, C.c_double
    lib.spnet_assemble.argtypes = [i32, i64, i64, P, P, P, i32, P, P, P, P, i64, C.POINTER(i64)]
    lib.build_network_operator.argtypes = [i32, i32, i64, P, P, P, P, i64, P, P, i32, P, C.POINTER(P)]
    lib.setup_preconditioner.argtypes = [P, dbl, C.POINTER(C.c_int), C.POINTER(Options), C.POINTER(P)]
    lib.pcg_solve.argtypes = [P, P, i32, P, P, P, i32, dbl, i32, i32, C.POINTER(Stats)]
    lib.spnet_op_destroy.argtypes = [P]
    lib.spnet_pc_destroy.argtypes = [P]
    lib.spnet_last_error.argtypes = [C.c_char_p, C.c_size_t]
    lib.spnet_op_get_info.argtypes = [P, C.POINTER(OpInfo)]
    lib.spnet_pc_get_info.argtypes = [P, C.POINTER(PcInfo)]
    for name in ("spnet_spmv", "spnet_pc_apply", "spnet_pc_restrict", "spnet_pc_coarse",
                 "spnet_pc_prolong", "spnet_pc_stars"):
        getattr(lib, name).argtypes = [P, P, P, i32]
    lib.spnet_pc_export.argtypes = [P, i32, P, C.c_size_t]
    lib.spnet_launch_count.argtypes = [C.POINTER(i64)]
    lib.spnet_pc_restrict_static.argtypes = [P, P, P]
    lib.spnet_pc_record_iterates.argtypes = [P, P, i64]
    lib.spnet_profile_enable.argtypes = [i32]
    lib.spnet_profile_read.argtypes = [i32, C.POINTER(i64), C.POINTER(dbl)]
    lib.spnet_profile_reset.argtypes = []
    lib.spnet_pc_apply_batch.argtypes = [P, i32, P, P, i32, i32]
    lib.spnet_server_create.argtypes = [i32, i64, C.POINTER(P)]
    lib.spnet_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(i64)]
    lib.spnet_server_wait.argtypes = [P, i64, C.POINTER(Result)]
    lib.spnet_server_poll.argtypes = [P, i64, C.POINTER(Result), C.POINTER(C.c_int)]
    lib.spnet_server_cancel.argtypes = [P, i64, C.POINTER(C.c_int)]
    lib.spnet_server_estimate.argtypes = [C.POINTER(Request), C.POINTER(i64)]
    lib.spnet_server_budget.argtypes = [P, C.POINTER(i64)]
    lib.spnet_tune_cache_load.argtypes = [C.c_char_p]
    lib.spnet_tune_cache_save.argtypes = [C.c_char_p]
    lib.spnet_tune_cache_clear.argtypes = []
    lib.spnet_tune_counts.argtypes = [C.POINTER(i64), C.POINTER(i64)]
    lib.spnet_assemble_beam.argtypes = [i64, i64, P, P, P, i64, P, dbl, i32, P, P, P, P, i64, C.POINTER(i64)]
    lib.spnet_server_destroy.argtypes = [P]
    for name in EXPORTED:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def last_error() -> str:
    buf = C.create_string_buffer(4096)
    load().spnet_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def launch_count() -> int:
    n = C.c_int64(0)
    _check(load().spnet_launch_count(C.byref(n)))
    return int(n.value)


def profile_enable(on: bool = True):
    _check(load().spnet_profile_enable(1 if on else 0))


def profile_reset():
    _check(load().spnet_profile_reset())


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last reset."""
    lib = load()
    out = {}
    for k, name in enumerate(KERNELS):
        n, ms = C.c_int64(0), C.c_double(0.0)
        _check(lib.spnet_profile_read(k, C.byref(n), C.byref(ms)))
        out[name] = (int(n.value), float(ms.value))
    return out


def tune_cache_load(path):
    """Add the tuner's choices saved in a file to the process-wide cache."""
    _check(load().spnet_tune_cache_load(os.fsencode(path)))


def tune_cache_save(path):
    """Write the tuner's measured choices to a file."""
    _check(load().spnet_tune_cache_save(os.fsencode(path)))


def tune_cache_clear():
    _check(load().spnet_tune_cache_clear())


def tune_counts():
    """(choices measured, choices taken from the cache) since the last clear."""
    m, r = C.c_int64(0), C.c_int64(0)
    _check(load().spnet_tune_counts(C.byref(m), C.byref(r)))
    return int(m.value), int(r.value)


def _check(rc):
    if rc != OK:
        raise SpnetError(rc, last_error())
    return rc


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, dtype):
    """(pointer, mem, keep-alive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        if not a.is_cuda:
            a = a.numpy()
        else:
            return C.c_void_p(a.data_ptr()), MEM_DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), MEM_HOST, arr


def _same_mem(*mems):
    ms = {m for m in mems if m is not None}
    if len(ms) > 1:
        raise ValueError("all arrays of one call must live in the same memory (host or device)")
    return ms.pop() if ms else MEM_HOST


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def assemble(model, n_nodes, edges, coef, dirs=None, stream=None):
    """K on all dofs as host CSR arrays (row_ptr int64, col int32, val float64)."""
    lib = load()
    ndof = 1 if model == MODEL_SCALAR else 3
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    m = edges.shape[0]
    cap = ndof * ndof * (n_nodes + 2 * m)
    rp = np.zeros(n_nodes * ndof + 1, np.int64)
    col = np.zeros(max(cap, 1), np.int32)
    val = np.zeros(max(cap, 1), np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    d = np.ascontiguousarray(dirs, dtype=np.float64) if dirs is not None else None
    nnz = C.c_int64(0)
    _check(lib.spnet_assemble(model, n_nodes, m, edges.ctypes.data, coef.ctypes.data,
                              d.ctypes.data if d is not None else None, MEM_HOST,
                              _stream_ptr(stream), rp.ctypes.data, col.ctypes.data,
                              val.ctypes.data, cap, C.byref(nnz)))
    n = nnz.value
    return rp, col[:n].copy(), val[:n].copy()


def assemble_beam(n_nodes, edges, coords, coef, triples, EI, stream=None):
    """spnet_assemble_beam: K of the planar beam model (3 dofs per node) as host CSR arrays."""
    lib = load()
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    triples = np.ascontiguousarray(triples, dtype=np.int64).reshape(-1, 4)
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    # a node's rows hold at most itself, its neighbours and the members of its triples
    deg = np.bincount(edges.ravel(), minlength=n_nodes)
    tcnt = np.bincount(triples[:, :3].ravel(), minlength=n_nodes)
    cap = int(9 * (n_nodes + deg.sum() + 2 * tcnt.sum()))
    rp = np.zeros(3 * n_nodes + 1, np.int64)
    col = np.zeros(max(cap, 1), np.int32)
    val = np.zeros(max(cap, 1), np.float64)
    nnz = C.c_int64(0)
    _check(lib.spnet_assemble_beam(int(n_nodes), edges.shape[0], edges.ctypes.data, coords.ctypes.data,
                                   coef.ctypes.data, triples.shape[0], triples.ctypes.data if triples.size else None,
                                   float(EI), MEM_HOST, _stream_ptr(stream), rp.ctypes.data, col.ctypes.data,
                                   val.ctypes.data, cap, C.byref(nnz)))
    n = nnz.value
    return rp, col[:n].copy(), val[:n].copy()


class Operator:
    """build_network_operator: A = K_II and K_ID of a network problem."""

    def __init__(self, dim, ndof, coords, row_ptr, col, val, dirichlet_dofs, domain, stream=None):
        lib = load()
        self._lib = lib
        self.handle = C.c_void_p()
        X, m1, k1 = _arg(coords, np.float64)
        rp, m2, k2 = _arg(row_ptr, np.int64)
        cl, m3, k3 = _arg(col, np.int32)
        vl, m4, k4 = _arg(val, np.float64)
        dd, m5, k5 = _arg(dirichlet_dofs, np.int64)
        mem = _same_mem(m1, m2, m3, m4, m5)
        if mem == MEM_DEVICE:
            import torch
            torch.cuda.current_stream(k1.device).synchronize()
        dom = np.ascontiguousarray(domain, dtype=np.float64)
        n_nodes = int(np.asarray(coords.shape)[0])
        nd = 0 if dirichlet_dofs is None else int(len(dirichlet_dofs))
        self.stream = stream
        _check(lib.build_network_operator(dim, ndof, n_nodes, X, rp, cl, vl, nd, dd,
                                          dom.ctypes.data, mem, _stream_ptr(stream),
                                          C.byref(self.handle)))
        self.dim, self.ndof, self.n_nodes = dim, ndof, n_nodes
        self.info = self.get_info()

    @classmethod
    def from_problem(cls, problem, stream=None, device=False):
        """Assemble K with the library and build the operator of a networks.Problem."""
        net = problem.net
        if problem.model == "scalar":
            rp, col, val = assemble(MODEL_SCALAR, net.n_nodes, net.edges, net.cond, stream=stream)
        elif problem.model == "beam":
            EI = float(net.stiff[0]) * problem.meta["r_w"] ** 2 / 4.0
            rp, col, val = assemble_beam(net.n_nodes, net.edges, net.coords, net.stiff, problem.meta["triples"], EI,
                                         stream=stream)
        else:
            rp, col, val = assemble(MODEL_TRUSS3, net.n_nodes, net.edges, net.stiff, net.dirs,
                                    stream=stream)
        arrs = [net.coords, rp, col, val, problem.dirichlet_dofs]
        if device:
            import torch
            arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
        return cls(net.dim, problem.ndof, *arrs, domain=net.domain, stream=stream)

    def get_info(self):
        info = OpInfo()
        _check(self._lib.spnet_op_get_info(self.handle, C.byref(info)))
        return info

    def spmv(self, x):
        xp, mem, keep = _arg(x, np.float64)
        if mem == MEM_DEVICE:
            import torch
            y = torch.empty_like(keep)
            torch.cuda.current_stream(keep.device).synchronize()
            _check(self._lib.spnet_spmv(self.handle, xp, C.c_void_p(y.data_ptr()), mem))
            return y
        y = np.zeros(self.info.n_free)
        _check(self._lib.spnet_spmv(self.handle, xp, y.ctypes.data, mem))
        return y

    def close(self):
        if self.handle:
            _check(self._lib.spnet_op_destroy(self.handle))
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_static_restrict_args(r, rc, n_free, m0):
    """Arguments of spnet_pc_restrict_static, checked before any launch: both torch
    CUDA tensors on the same device, float64, contiguous; r of n_free entries, rc
    of at least m0 (the kernels read r[0..n_free) and write rc[0..m0))."""
    for name, t in (("r", r), ("rc", rc)):
        if not _is_torch(t) or not t.is_cuda:
            raise ValueError(f"restrict_static: {name} must be a CUDA tensor")
        if str(t.dtype) != "torch.float64":
            raise ValueError(f"restrict_static: {name} must be float64, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"restrict_static: {name} must be contiguous")
    if r.device != rc.device:
        raise ValueError("restrict_static: r and rc must be on the same device")
    if r.numel() != n_free:
        raise ValueError(f"restrict_static: r has {r.numel()} entries, the operator {n_free} free dofs")
    if rc.numel() < m0:
        raise ValueError(f"restrict_static: rc has {rc.numel()} entries, fewer than m0 = {m0}")


def check_record_args(buf, n_free):
    """Argument of spnet_pc_record_iterates, checked before the library is called: a
    contiguous float64 torch CUDA tensor of shape (max_iterates, n_free)."""
    if not _is_torch(buf) or not buf.is_cuda:
        raise ValueError("record_iterates: buf must be a CUDA tensor")
    if str(buf.dtype) != "torch.float64":
        raise ValueError(f"record_iterates: buf must be float64, not {buf.dtype}")
    if not buf.is_contiguous() or buf.dim() != 2:
        raise ValueError("record_iterates: buf must be a contiguous 2-D tensor")
    if buf.shape[1] != n_free or buf.shape[0] < 1:
        raise ValueError(f"record_iterates: buf has shape {tuple(buf.shape)}, wanted (k >= 1, {n_free})")


class Preconditioner:
    """setup_preconditioner: the two-level additive Schwarz preconditioner."""

    def __init__(self, op: Operator, H, gamma_faces, precision=PREC_MIXED, star_set=STARS_INTERIOR,
                 flexible=-1, max_restarts=2, batch_rhs=1, star_map=0, patch=PATCH_ELEMENT, panels=True,
                 coarse=COARSE_Q1):
        self._lib = op._lib
        self.op = op
        self.handle = C.c_void_p()
        o = Options()
        o.precision, o.star_set, o.flexible, o.max_restarts = precision, star_set, flexible, max_restarts
        o.batch_rhs = batch_rhs
        o.star_map = star_map
        o.no_panels = 0 if panels else 1
        o.patch = patch if isinstance(patch, int) else (PATCH_SUPPORT if patch == "support"
                                                         else PATCH_ELEMENT)
        o.coarse_space = coarse if isinstance(coarse, int) else (COARSE_P1 if coarse == "p1" else COARSE_Q1)
        gf = (C.c_int * 3)(*(list(gamma_faces) + [0, 0, 0])[:3])
        _check(self._lib.setup_preconditioner(op.handle, float(H), gf, C.byref(o),
                                              C.byref(self.handle)))
        self.info = self.get_info()

    def get_info(self):
        info = PcInfo()
        _check(self._lib.spnet_pc_get_info(self.handle, C.byref(info)))
        return info

    def _vec_call(self, fn, v, n_out):
        vp, mem, keep = _arg(v, np.float64)
        if mem == MEM_DEVICE:
            import torch
            out = torch.zeros(max(n_out, 1), dtype=torch.float64, device=keep.device)[:n_out]
            torch.cuda.current_stream(keep.device).synchronize()
            _check(fn(self.handle, vp, C.c_void_p(out.data_ptr()), mem))
            return out
        out = np.zeros(n_out)
        _check(fn(self.handle, vp, out.ctypes.data if n_out else C.c_void_p(), mem))
        return out

    def apply(self, r):
        return self._vec_call(self._lib.spnet_pc_apply, r, self.op.info.n_free)

    def stars(self, r):
        return self._vec_call(self._lib.spnet_pc_stars, r, self.op.info.n_free)

    def apply_batch(self, R, which=0):
        """spnet_pc_apply_batch: z_j = B r_j (which 0), the coarse term (1) or the star
        term (2) for the rows r_j of R, shape (k, n_free), 1 <= k <= 32, in one pass."""
        R = np.ascontiguousarray(np.atleast_2d(np.asarray(R, np.float64)))
        k, _ = R.shape
        Z = np.zeros(R.shape)
        _check(self._lib.spnet_pc_apply_batch(self.handle, int(k), C.c_void_p(R.ctypes.data),
                                              C.c_void_p(Z.ctypes.data), int(which), MEM_HOST))
        return Z

    def restrict(self, r):
        return self._vec_call(self._lib.spnet_pc_restrict, r, self.info.m0)

    def restrict_static(self, r, rc):
        """r_c = R_0 r into the caller's device tensor rc, allocating nothing.

        r and rc must be contiguous float64 CUDA tensors on one device, r of length
        n_free and rc of at least m0 entries; anything else raises ValueError before
        the library is called."""
        check_static_restrict_args(r, rc, self.op.info.n_free, self.info.m0)
        import torch
        torch.cuda.current_stream(r.device).synchronize()
        _check(self._lib.spnet_pc_restrict_static(self.handle, C.c_void_p(r.data_ptr()),
                                                  C.c_void_p(rc.data_ptr())))
        return rc

    def record_iterates(self, buf=None):
        """spnet_pc_record_iterates: later one-at-a-time solves write u^(l) (free dofs) to
        row l of buf, a contiguous float64 CUDA tensor (max_iterates, n_free) on the
        preconditioner's device; None stops recording."""
        if buf is None:
            _check(self._lib.spnet_pc_record_iterates(self.handle, None, 0))
            self._rec = None
            return
        check_record_args(buf, self.op.info.n_free)
        import torch
        torch.cuda.current_stream(buf.device).synchronize()
        _check(self._lib.spnet_pc_record_iterates(self.handle, C.c_void_p(buf.data_ptr()), int(buf.shape[0])))
        self._rec = buf  # the library writes into it until recording stops

    def coarse(self, rc):
        return self._vec_call(self._lib.spnet_pc_coarse, rc, self.info.m0)

    def prolong(self, zc):
        return self._vec_call(self._lib.spnet_pc_prolong, zc, self.op.info.n_free)

    def export(self, what):
        i = self.info
        nfree = self.op.info.n_free
        spec = {
            EXPORT_ELEMENTS: (np.int32, (nfree,)),
            EXPORT_Q1: (np.float64, (nfree, 2 ** self.op.dim)),
            EXPORT_COARSE_MAP: (np.int32, (i.n_mesh * self.op.ndof,)),
            EXPORT_STAR_SIZES: (np.int32, (i.n_stars,)),
            EXPORT_STAR_MESH: (np.int32, (i.n_stars,)),
            EXPORT_STAR_LEVELS: (np.int32, (i.n_stars,)),
            EXPORT_STAR_CORE: (np.int32, (i.n_stars,)),
            EXPORT_A0: (np.float64, (i.m0, i.m0)),
        }[what]
        out = np.zeros(spec[1], dtype=spec[0])
        _check(self._lib.spnet_pc_export(self.handle, what, out.ctypes.data, out.nbytes))
        return out

    def close(self):
        if self.handle:
            _check(self._lib.spnet_pc_destroy(self.handle))
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcg_solve(op: Operator, pc: Preconditioner, f, g, x0=None, rtol=1e-8, maxit=1000,
              raise_on_noconv=True):
    """Solve for one or several right-hand sides.

    f: (n_dof,) or (nrhs, n_dof); g: (n_dir,) or (nrhs, n_dir).  Returns
    (u_hat, stats) with u_hat of the same leading shape as f.
    """
    lib = op._lib
    single = len(f.shape) == 1
    nrhs = 1 if single else int(f.shape[0])
    fp, m1, kf = _arg(f, np.float64)
    gp, m2, kg = _arg(g, np.float64)
    mem = _same_mem(m1, m2)
    stats = (Stats * nrhs)()
    if mem == MEM_DEVICE:
        import torch
        if x0 is not None:
            x = x0.to(torch.float64).clone().contiguous()
        else:
            x = torch.zeros(tuple(f.shape), dtype=torch.float64, device=kf.device)
        # torch filled x and may have produced f, g on its current stream; the
        # library works on the operator's stream
        torch.cuda.current_stream(kf.device).synchronize()
        xp = C.c_void_p(x.data_ptr())
    else:
        x = np.zeros(tuple(f.shape)) if x0 is None else np.array(x0, dtype=np.float64)
        xp = C.c_void_p(x.ctypes.data)
    rc = lib.pcg_solve(op.handle, pc.handle, nrhs, fp, gp, xp, 1 if x0 is not None else 0,
                       float(rtol), int(maxit), mem, stats)
    if rc != OK and (rc != -4 or raise_on_noconv):
        _check(rc)
    return x, [stats[k] for k in range(nrhs)]


class Server:
    """spnet_server_*: continuous batching of solve requests (host arrays in, host solutions out).

    submit() copies nothing: the arrays of a request are kept alive here until
    wait() returns its solutions.
    """

    def __init__(self, max_inflight=4, reserve_bytes=2 << 30):
        self._lib = load()
        self.handle = C.c_void_p()
        _check(self._lib.spnet_server_create(int(max_inflight), C.c_int64(int(reserve_bytes)),
                                             C.byref(self.handle)))
        self._live = {}

    def submit(self, problem, f=None, g=None, precision=PREC_MIXED, rtol=1e-8, maxit=2000,
               star_set=None, flexible=-1, max_restarts=2, batch_rhs=1):
        """Queue one request for `problem` (a networks.Problem); f: (n_dof,) or (nrhs, n_dof),
        default problem.f; g likewise over the Dirichlet dofs, default problem.dirichlet_vals."""
        live = make_request(problem, f, g, precision, rtol, maxit, star_set, flexible, max_restarts,
                            batch_rhs)
        ticket = C.c_int64(0)
        _check(self._lib.spnet_server_submit(self.handle, C.byref(live[0]), C.byref(ticket)))
        self._live[ticket.value] = live
        return ticket.value

    def _result(self, ticket, res):
        live = self._live.pop(ticket)
        out = {k: getattr(res, k) for k in ("status", "iterations", "relres", "queue_ms", "latency_ms",
                                              "device_start_ms", "device_end_ms")}
        out["message"] = res.message.decode(errors="replace")
        return live[-1], out

    def wait(self, ticket):
        """Block until the request is done: (x of shape (nrhs, n_dof), result dict)."""
        res = Result()
        _check(self._lib.spnet_server_wait(self.handle, C.c_int64(ticket), C.byref(res)))
        return self._result(ticket, res)

    def poll(self, ticket):
        """(x, result dict) if the request has finished, else None (non-blocking)."""
        res = Result()
        done = C.c_int(0)
        _check(self._lib.spnet_server_poll(self.handle, C.c_int64(ticket), C.byref(res), C.byref(done)))
        return self._result(ticket, res) if done.value else None

    def cancel(self, ticket):
        """Withdraw a queued request; True if it had not been admitted yet."""
        c = C.c_int(0)
        _check(self._lib.spnet_server_cancel(self.handle, C.c_int64(ticket), C.byref(c)))
        return bool(c.value)

    def budget(self):
        b = C.c_int64(0)
        _check(self._lib.spnet_server_budget(self.handle, C.byref(b)))
        return int(b.value)

    def close(self):
        if self.handle:
            self._lib.spnet_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_estimate(problem, f=None, **kw):
    """Device bytes the server's admission charges for a request (spnet_server_estimate)."""
    live = make_request(problem, f, None, **kw)
    b = C.c_int64(0)
    _check(load().spnet_server_estimate(C.byref(live[0]), C.byref(b)))
    return int(b.value)


def make_request(problem, f=None, g=None, precision=PREC_MIXED, rtol=1e-8, maxit=2000, star_set=None,
                 flexible=-1, max_restarts=2, batch_rhs=1):
    """A spnet_request for `problem` and the arrays it points to (keep them alive with it):
    (request, edges, coef, dirs, coords, dirichlet dofs, f, g, x)."""
    net = problem.net
    f = problem.f if f is None else f
    f = np.ascontiguousarray(np.atleast_2d(np.asarray(f, np.float64)))
    nrhs = f.shape[0]
    g = problem.dirichlet_vals if g is None else g
    g = np.ascontiguousarray(np.broadcast_to(np.atleast_2d(np.asarray(g, np.float64)),
                                             (nrhs, len(problem.dirichlet_dofs))))
    x = np.zeros((nrhs, problem.n_dof), np.float64)
    edges = np.ascontiguousarray(net.edges, np.int64)
    scalar = problem.model == "scalar"
    coef = np.ascontiguousarray(net.cond if scalar else net.stiff, np.float64)
    dirs = None if scalar else np.ascontiguousarray(net.dirs, np.float64)
    coords = np.ascontiguousarray(net.coords, np.float64)
    dd = np.ascontiguousarray(problem.dirichlet_dofs, np.int64)
    q = Request()
    q.model = MODEL_SCALAR if scalar else MODEL_TRUSS3
    q.dim = net.dim
    q.n_nodes = net.n_nodes
    q.n_edges = net.n_edges
    q.edges = edges.ctypes.data
    q.coef = coef.ctypes.data
    q.dirs = dirs.ctypes.data if dirs is not None else None
    q.coords = coords.ctypes.data
    for a in range(3):
        q.domain_hi[a] = float(net.domain[a]) if a < net.dim else 1.0
    q.n_dirichlet = len(dd)
    q.dirichlet_dofs = dd.ctypes.data if len(dd) else None
    q.nrhs = nrhs
    q.f = f.ctypes.data
    q.g = g.ctypes.data if g.size else x.ctypes.data
    q.x = x.ctypes.data
    q.H = float(problem.H)
    for a, v in enumerate((list(problem.gamma_faces) + [0, 0, 0])[:3]):
        q.gamma_faces[a] = int(v)
    q.opts.precision = precision
    ss = problem.star_set if star_set is None else star_set
    q.opts.star_set = ss if isinstance(ss, int) else (STARS_ALL if ss == "all" else STARS_INTERIOR)
    q.opts.patch = PATCH_SUPPORT if getattr(problem, "patch", "element") == "support" \
        else PATCH_ELEMENT
    q.opts.flexible = flexible
    q.opts.max_restarts = max_restarts
    q.opts.batch_rhs = batch_rhs
    q.rtol = float(rtol)
    q.maxit = int(maxit)
    return (q, edges, coef, dirs, coords, dd, f, g, x)
