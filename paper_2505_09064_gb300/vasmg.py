"""Thin ctypes binding of libvasmg (include/vasmg.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Vectors may be
numpy arrays (host) or torch tensors (host or CUDA); pointers are passed
through unchanged and all arithmetic runs in the library's CUDA kernels.  If
the library is missing this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvasmg.so")

VASMG_OK, VASMG_NOT_CONVERGED = 0, 1
VASMG_ERR_INVALID_ARG, VASMG_ERR_DEGENERATE_ELEMENT, VASMG_ERR_OOM = -1, -2, -3
VASMG_ERR_CUDA, VASMG_ERR_BREAKDOWN, VASMG_ERR_TIMEOUT, VASMG_ERR_UNSUPPORTED = -4, -5, -6, -7
VASMG_FP64, VASMG_FP32_VCYCLE, VASMG_FP32_VCYCLE_BF16_SMOOTH = 0, 1, 2
PRECISIONS = {"fp64": VASMG_FP64, "fp32": VASMG_FP32_VCYCLE, "bf16": VASMG_FP32_VCYCLE_BF16_SMOOTH}

(EXPORT_MORTON, EXPORT_LEAF, EXPORT_CELLS, EXPORT_LATTICE, EXPORT_P_RP, EXPORT_P_CI, EXPORT_P_W, EXPORT_A_RP,
 EXPORT_A_CI, EXPORT_A_V, EXPORT_DEAD, EXPORT_COLOUR, EXPORT_DINV, EXPORT_BOX, EXPORT_LIFT, EXPORT_VOL,
 EXPORT_DENSE, EXPORT_LANES, EXPORT_STAGED) = (0, 1, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19)
OP_MATVEC, OP_SMOOTH_FWD, OP_SMOOTH_BWD, OP_RESIDUAL, OP_RESTRICT, OP_PROLONG, OP_COARSE, OP_VCYCLE, OP_PRECOND = range(9)
KERNEL_SPMV64, KERNEL_SWEEP, KERNEL_VCYCLE, KERNEL_DOWN, KERNEL_UP = 0, 1, 2, 3, 4
KERNEL_FWD_SWEEP, KERNEL_RESIDUAL, KERNEL_RESTRICT, KERNEL_PROLONG, KERNEL_TAIL = 5, 6, 7, 8, 9

# symbols declared in include/vasmg.h
EXPORTED = ["vasmg_default_options", "vasmg_setup", "vasmg_assemble_load", "vasmg_solve", "vasmg_solve_batch",
            "vasmg_num_levels", "vasmg_level_info", "vasmg_export", "vasmg_apply", "vasmg_time_kernel",
            "vasmg_last_launch_count", "vasmg_destroy", "vasmg_error_string", "vasmg_last_error_detail",
            "vasmg_coarse_solve_noalloc", "vasmg_server_default_opts", "vasmg_server_create",
            "vasmg_server_submit", "vasmg_server_poll", "vasmg_server_destroy", "vasmg_update_data",
            "vasmg_probe_wait_timeout", "vasmg_probe_fp64_rate", "vasmg_solve_multi", "vasmg_time_kernel_multi"]

OK, NOT_CONVERGED, PENDING = 0, 1, 2
NOALLOC_MAX_DOFS = 4096  # VASMG_NOALLOC_MAX_DOFS


class vasmg_problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("coords", C.c_void_p), ("n_elements", C.c_int64),
                ("elements", C.c_void_p), ("lambda_", C.c_void_p), ("mu", C.c_void_p), ("lambda_const", C.c_double),
                ("mu_const", C.c_double), ("n_dirichlet", C.c_int64), ("dirichlet_dofs", C.c_void_p),
                ("dirichlet_values", C.c_void_p)]


class vasmg_options(C.Structure):
    _fields_ = [("leaf_threshold", C.c_int32), ("n_pre", C.c_int32), ("n_post", C.c_int32),
                ("precision", C.c_int32), ("coarse_max_dofs", C.c_int64), ("max_iters", C.c_int32),
                ("use_graph", C.c_int32), ("max_ctas", C.c_int32), ("dense_coarse", C.c_int32),
                ("autotune", C.c_int32), ("stream", C.c_void_p), ("cycle", C.c_int32), ("additive", C.c_int32)]


class vasmg_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("precision", C.c_int32), ("max_iters", C.c_int32), ("tol", C.c_double),
                ("memory_budget", C.c_int64), ("batch", C.c_int32)]


class vasmg_request_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_rhs", C.c_int32), ("iterations", C.c_int32),
                ("max_iterations", C.c_int32), ("max_rel_res", C.c_double), ("queue_ms", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("latency_ms", C.c_double),
                ("footprint_bytes", C.c_int64)]


class vasmg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("rel_res", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("n_levels", C.c_int32), ("op_complexity", C.c_double),
                ("res_history", C.c_void_p), ("res_history_cap", C.c_int32)]


class VasmgError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        lib = load()
        detail = lib.vasmg_last_error_detail().decode()
        super().__init__(f"{where}: {lib.vasmg_error_string(code).decode()} ({code}) {detail}")


_lib = None


def load():
    """Load libvasmg.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libvasmg.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.vasmg_default_options.argtypes = [C.c_int, C.POINTER(vasmg_options)]
    lib.vasmg_setup.argtypes = [C.POINTER(vasmg_problem), C.POINTER(vasmg_options), C.POINTER(P)]
    lib.vasmg_assemble_load.argtypes = [P, P, P]
    lib.vasmg_solve.argtypes = [P, P, P, C.c_double, C.POINTER(vasmg_stats)]
    lib.vasmg_solve_batch.argtypes = [C.c_int32, P, P, P, C.c_double, P]
    lib.vasmg_solve_multi.argtypes = [P, C.c_int32, P, P, C.c_double, P]
    lib.vasmg_time_kernel_multi.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
    lib.vasmg_num_levels.argtypes = [P]
    lib.vasmg_level_info.argtypes = [P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int32)]
    lib.vasmg_export.argtypes = [P, C.c_int32, C.c_int32, P, C.POINTER(C.c_int64)]
    lib.vasmg_apply.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.vasmg_time_kernel.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
    lib.vasmg_coarse_solve_noalloc.argtypes = [P, P, P, P]
    lib.vasmg_update_data.argtypes = [P, P, P, C.c_double, C.c_double, P]
    lib.vasmg_server_default_opts.argtypes = [C.POINTER(vasmg_server_opts)]
    lib.vasmg_server_create.argtypes = [C.POINTER(vasmg_server_opts), C.POINTER(P)]
    lib.vasmg_server_submit.argtypes = [P, C.POINTER(vasmg_problem), C.c_int32, P, P, C.POINTER(C.c_uint64)]
    lib.vasmg_server_poll.argtypes = [P, C.c_uint64, C.c_int32, C.POINTER(vasmg_request_stats)]
    lib.vasmg_server_destroy.argtypes = [P]
    lib.vasmg_last_launch_count.argtypes = [P]
    lib.vasmg_last_launch_count.restype = C.c_int64
    lib.vasmg_destroy.argtypes = [P]
    lib.vasmg_error_string.argtypes = [C.c_int]
    lib.vasmg_error_string.restype = C.c_char_p
    lib.vasmg_last_error_detail.argtypes = []
    lib.vasmg_last_error_detail.restype = C.c_char_p
    lib.vasmg_probe_wait_timeout.argtypes = [C.POINTER(C.c_double)]
    lib.vasmg_probe_wait_timeout.restype = C.c_int
    lib.vasmg_probe_fp64_rate.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.vasmg_probe_fp64_rate.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p)
    raise TypeError(type(a))


def _check_vec(a, n, name):
    """A vector argument must be a contiguous float64 numpy array or torch
    tensor of exactly n entries (the library reads / writes n doubles)."""
    if hasattr(a, "data_ptr"):
        import torch

        if a.dtype != torch.float64:
            raise TypeError(f"{name} must be float64, got {a.dtype}")
        size = a.numel()
    elif isinstance(a, np.ndarray):
        if a.dtype != np.float64:
            raise TypeError(f"{name} must be float64, got {a.dtype}")
        size = a.size
    else:
        raise TypeError(f"{name} must be a numpy array or a torch tensor, got {type(a).__name__}")
    if size != n:
        raise ValueError(f"{name} has {size} entries, expected {n}")


def _check(rc, where, allow_not_converged=False):
    if rc == VASMG_OK or (allow_not_converged and rc == VASMG_NOT_CONVERGED):
        return rc
    raise VasmgError(rc, where)


def vasmg_default_options(dim: int) -> vasmg_options:
    o = vasmg_options()
    _check(load().vasmg_default_options(dim, C.byref(o)), "vasmg_default_options")
    return o


def _problem_struct(prob: dict):
    """vasmg_problem for a problem dict, and the arrays it points into."""
    dim = int(prob["dim"])
    coords = np.ascontiguousarray(prob["coords"], dtype=np.float64)
    elems = np.ascontiguousarray(prob["elems"], dtype=np.int32)
    ne = elems.shape[0]
    lam = np.ascontiguousarray(np.broadcast_to(np.asarray(prob["lam"], dtype=np.float64), (ne,)))
    mu = np.ascontiguousarray(np.broadcast_to(np.asarray(prob["mu"], dtype=np.float64), (ne,)))
    dd = np.ascontiguousarray(prob.get("dirichlet_dofs", np.zeros(0)), dtype=np.int64)
    dv = prob.get("dirichlet_values")
    dv = None if dv is None else np.ascontiguousarray(dv, dtype=np.float64)
    p = vasmg_problem(dim, coords.shape[0], _ptr(coords), ne, _ptr(elems), _ptr(lam), _ptr(mu), 0.0, 0.0, dd.size,
                      _ptr(dd), _ptr(dv))
    return p, (coords, elems, lam, mu, dd, dv)


def vasmg_setup(prob: dict, options: vasmg_options | None = None):
    """prob: dict with dim, coords, elems, lam, mu (per element or scalar),
    dirichlet_dofs, dirichlet_values (optional).  Returns (handle, keepalive)."""
    lib = load()
    dim = int(prob["dim"])
    p, _keep = _problem_struct(prob)
    if options is None:
        options = vasmg_default_options(dim)
    h = C.c_void_p()
    _check(lib.vasmg_setup(C.byref(p), C.byref(options), C.byref(h)), "vasmg_setup")
    return h


def vasmg_assemble_load(h, body_force, F):
    f = np.ascontiguousarray(body_force, dtype=np.float64)
    _check(load().vasmg_assemble_load(h, _ptr(f), _ptr(F)), "vasmg_assemble_load")


def vasmg_solve(h, F, U, tol: float = 1e-6, history_cap: int = 0):
    """Returns (status, vasmg_stats, history ndarray)."""
    st = vasmg_stats()
    hist = np.zeros(max(1, history_cap))
    if history_cap:
        st.res_history = hist.ctypes.data_as(C.c_void_p)
        st.res_history_cap = history_cap
    rc = _check(load().vasmg_solve(h, _ptr(F), _ptr(U), float(tol), C.byref(st)), "vasmg_solve",
                allow_not_converged=True)
    return rc, st, hist[: min(st.iterations, history_cap)]


def vasmg_solve_batch(handles, Fs, Us, tol: float = 1e-6):
    k = len(handles)
    H = (C.c_void_p * k)(*[h.value for h in handles])
    Fp = (C.c_void_p * k)(*[_ptr(F).value for F in Fs])
    Up = (C.c_void_p * k)(*[_ptr(U).value for U in Us])
    st = (vasmg_stats * k)()
    rc = _check(load().vasmg_solve_batch(k, H, Fp, Up, float(tol), st), "vasmg_solve_batch",
                allow_not_converged=True)
    return rc, list(st)


def vasmg_solve_multi(h, Fs, Us, tol: float = 1e-6, history_cap: int = 0):
    """k right-hand sides on one hierarchy.  Returns (status, [vasmg_stats],
    [history ndarray])."""
    k = len(Fs)
    Fp = (C.c_void_p * k)(*[_ptr(F).value for F in Fs])
    Up = (C.c_void_p * k)(*[_ptr(U).value for U in Us])
    st = (vasmg_stats * k)()
    hists = [np.zeros(max(1, history_cap)) for _ in range(k)]
    if history_cap:
        for i in range(k):
            st[i].res_history = hists[i].ctypes.data_as(C.c_void_p)
            st[i].res_history_cap = history_cap
    rc = _check(load().vasmg_solve_multi(h, k, Fp, Up, float(tol), st), "vasmg_solve_multi",
                allow_not_converged=True)
    return rc, list(st), [hists[i][: min(st[i].iterations, history_cap)] for i in range(k)]


def vasmg_time_kernel_multi(h, which: int, level: int, k: int, reps: int = 10):
    ms, nbytes = C.c_double(), C.c_double()
    _check(load().vasmg_time_kernel_multi(h, which, level, k, reps, C.byref(ms), C.byref(nbytes)),
           "vasmg_time_kernel_multi")
    return ms.value, nbytes.value


def vasmg_probe_wait_timeout():
    """Run the sweeps' bounded wait against a word nothing publishes; returns
    (return code, kernel milliseconds).  The code is VASMG_ERR_TIMEOUT."""
    ms = C.c_double()
    rc = load().vasmg_probe_wait_timeout(C.byref(ms))
    return rc, ms.value


def vasmg_probe_fp64_rate():
    """(FP64 TFLOP/s, ms per launch) of an FMA-chain kernel on the current device."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().vasmg_probe_fp64_rate(C.byref(tf), C.byref(ms)), "vasmg_probe_fp64_rate")
    return tf.value, ms.value


def vasmg_num_levels(h) -> int:
    n = load().vasmg_num_levels(h)
    if n < 0:
        raise VasmgError(n, "vasmg_num_levels")
    return n


def vasmg_level_info(h, level: int):
    nv, nnzb, nc = C.c_int64(), C.c_int64(), C.c_int32()
    _check(load().vasmg_level_info(h, level, C.byref(nv), C.byref(nnzb), C.byref(nc)), "vasmg_level_info")
    return nv.value, nnzb.value, nc.value


def vasmg_export(h, what: int, level: int = 0, dtype=np.int64):
    lib = load()
    nbytes = C.c_int64()
    _check(lib.vasmg_export(h, what, level, None, C.byref(nbytes)), "vasmg_export")
    buf = np.empty(nbytes.value // np.dtype(dtype).itemsize, dtype=dtype)
    _check(lib.vasmg_export(h, what, level, _ptr(buf), C.byref(nbytes)), "vasmg_export")
    return buf


def vasmg_apply(h, op: int, level: int, x, y):
    _check(load().vasmg_apply(h, op, level, _ptr(x), _ptr(y)), "vasmg_apply")


def vasmg_time_kernel(h, which: int, level: int = 0, reps: int = 10):
    ms, nbytes = C.c_double(), C.c_double()
    _check(load().vasmg_time_kernel(h, which, level, reps, C.byref(ms), C.byref(nbytes)), "vasmg_time_kernel")
    return ms.value, nbytes.value


def vasmg_update_data(h, lam=None, mu=None, lam_const=0.0, mu_const=0.0, dirichlet_values=None):
    """New Lame parameters (per element, or constants) and / or Dirichlet
    values on the same mesh and constrained dofs, reusing the hierarchy."""
    lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
    mu = None if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
    dv = None if dirichlet_values is None else np.ascontiguousarray(dirichlet_values, dtype=np.float64)
    _check(load().vasmg_update_data(h, _ptr(lam), _ptr(mu), float(lam_const), float(mu_const), _ptr(dv)),
           "vasmg_update_data")


def vasmg_coarse_solve_noalloc(h, b, x, stream=None, n=None):
    """x = A_L^{-1} b on the coarsest level without allocating (b, x: CUDA
    float64 tensors of n = dim * coarsest-vertices entries, canonical order, on
    the current device).  Enqueued on `stream` (an int cudaStream_t or None);
    the caller synchronises.  n, if given, is checked against both vectors."""
    import torch

    for a, name in ((b, "b"), (x, "x")):
        if not (hasattr(a, "data_ptr") and a.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
        if a.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {a.device}, not on the current device")
        if n is not None:
            _check_vec(a, n, name)
        elif a.dtype != torch.float64:
            raise TypeError(f"{name} must be float64, got {a.dtype}")
    if b.numel() != x.numel():
        raise ValueError(f"b has {b.numel()} entries and x {x.numel()}")
    s = C.c_void_p(stream) if isinstance(stream, int) else stream
    _check(load().vasmg_coarse_solve_noalloc(h, _ptr(b), _ptr(x), s), "vasmg_coarse_solve_noalloc")


def vasmg_last_launch_count(h) -> int:
    return int(load().vasmg_last_launch_count(h))


def vasmg_destroy(h):
    if h is not None and h.value:
        _check(load().vasmg_destroy(h), "vasmg_destroy")
        h.value = None


class Solver:
    """Convenience owner of one hierarchy: setup in the constructor, destroy on close."""

    def __init__(self, prob: dict, precision: str = "fp64", stream=None, threshold: int = 0,
                 coarse_max_dofs: int = 0, max_iters: int = 1000, use_graph: bool = True, max_ctas: int = 0,
                 dense_coarse: bool = True, autotune: bool = True, cycle: int = 1, additive: bool = False):
        self.dim = int(prob["dim"])
        self.n = int(np.asarray(prob["coords"]).shape[0]) * self.dim
        o = vasmg_default_options(self.dim)
        o.precision = PRECISIONS[precision]
        if threshold:
            o.leaf_threshold = threshold
        o.coarse_max_dofs = coarse_max_dofs
        o.max_iters = max_iters
        o.use_graph = 1 if use_graph else 0
        o.max_ctas = max_ctas
        o.dense_coarse = 1 if dense_coarse else 0
        o.autotune = 1 if autotune else 0
        o.cycle = int(cycle)
        o.additive = 1 if additive else 0
        o.stream = C.c_void_p(stream) if isinstance(stream, int) else stream
        self.options = o
        self.h = vasmg_setup(prob, o)

    def close(self):
        vasmg_destroy(getattr(self, "h", None))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self):
        return vasmg_num_levels(self.h)

    def level_info(self, l):
        return vasmg_level_info(self.h, l)

    def export(self, what, level=0, dtype=np.int64):
        return vasmg_export(self.h, what, level, dtype)

    def assemble_load(self, f, F):
        if np.asarray(f).size != self.dim:
            raise ValueError(f"body force has {np.asarray(f).size} components, expected {self.dim}")
        _check_vec(F, self.n, "F")
        vasmg_assemble_load(self.h, f, F)

    def solve(self, F, U, tol=1e-6, history_cap=0):
        _check_vec(F, self.n, "F")
        _check_vec(U, self.n, "U")
        return vasmg_solve(self.h, F, U, tol, history_cap)

    def apply(self, op, level, x, y):
        vasmg_apply(self.h, op, level, x, y)

    def solve_multi(self, Fs, Us, tol=1e-6, history_cap=0):
        if len(Fs) != len(Us):
            raise ValueError(f"{len(Fs)} right-hand sides and {len(Us)} solutions")
        for i, (F, U) in enumerate(zip(Fs, Us)):
            _check_vec(F, self.n, f"F[{i}]")
            _check_vec(U, self.n, f"U[{i}]")
        return vasmg_solve_multi(self.h, Fs, Us, tol, history_cap)

    def coarse_solve_noalloc(self, b, x, stream=None):
        """vasmg_coarse_solve_noalloc with both vectors checked against the
        coarsest level's dof count."""
        n = self.level_info(self.num_levels - 1)[0] * self.dim
        vasmg_coarse_solve_noalloc(self.h, b, x, stream, n=n)

    def update(self, prob: dict):
        """Take the material and Dirichlet values of `prob` (same mesh and
        constrained dofs as at construction) without a new setup."""
        ne = np.asarray(prob["elems"]).shape[0]
        lam = np.broadcast_to(np.asarray(prob["lam"], dtype=np.float64), (ne,))
        mu = np.broadcast_to(np.asarray(prob["mu"], dtype=np.float64), (ne,))
        dv = prob.get("dirichlet_values")
        if dv is None:
            dv = np.zeros(np.asarray(prob.get("dirichlet_dofs", np.zeros(0))).size)
        vasmg_update_data(self.h, lam, mu, 0.0, 0.0, dv)


PRECISIONS_SERVER = {"fp64": 0, "fp32": 1, "bf16": 2}


class Server:
    """vasmg_server_*: continuous admission of independent requests.

    submit() copies the problem and the right-hand sides; the U arrays passed
    in (float64 numpy arrays of n entries) are written by the server and kept
    referenced here until poll() reports the request done."""

    def __init__(self, slots: int = 4, precision: str = "fp32", tol: float = 1e-6, max_iters: int = 1000,
                 memory_budget: int = 0, batch: bool = False):
        lib = load()
        o = vasmg_server_opts()
        _check(lib.vasmg_server_default_opts(C.byref(o)), "vasmg_server_default_opts")
        o.slots, o.precision, o.tol, o.max_iters, o.memory_budget = (slots, PRECISIONS_SERVER[precision], tol,
                                                                      max_iters, memory_budget)
        o.batch = 1 if batch else 0
        self.s = C.c_void_p()
        _check(lib.vasmg_server_create(C.byref(o), C.byref(self.s)), "vasmg_server_create")
        self._keep = {}

    def submit(self, prob: dict, Fs, Us) -> int:
        p, keep = _problem_struct(prob)
        Fs = [np.ascontiguousarray(F, dtype=np.float64) for F in Fs]
        k = len(Fs)
        Fp = (C.c_void_p * k)(*[_ptr(F).value for F in Fs])
        Up = (C.c_void_p * k)(*[_ptr(U).value for U in Us])
        t = C.c_uint64()
        _check(load().vasmg_server_submit(self.s, C.byref(p), k, Fp, Up, C.byref(t)), "vasmg_server_submit")
        self._keep[t.value] = (list(Us), keep)
        return t.value

    def poll(self, ticket: int, wait_ms: int = -1):
        """Stats dict once the request is done, None while it is pending."""
        st = vasmg_request_stats()
        rc = load().vasmg_server_poll(self.s, ticket, wait_ms, C.byref(st))
        if rc == PENDING:
            return None
        _check(rc, "vasmg_server_poll")
        self._keep.pop(ticket, None)
        return {f: getattr(st, f) for f, _ in vasmg_request_stats._fields_}

    def close(self):
        if getattr(self, "s", None) is not None and self.s.value:
            _check(load().vasmg_server_destroy(self.s), "vasmg_server_destroy")
            self.s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
