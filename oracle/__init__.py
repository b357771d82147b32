"""CPU FP64 oracle for V-ASMG-PCG -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library in
``paper_2505_09064_gb300`` never does, and this package never imports the
library: the two share no code.  The arithmetic lives in ``vasmg_oracle.cpp``
(plain C++, IEEE FP64, no FMA contraction); this module only compiles it and
marshals arrays through ctypes.  ``Oracle(prob, threads=k)`` with k > 1 loads a
second build of the same file with OpenMP, whose independent row loops run on
k threads and give the same bits as the single-threaded build.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vasmg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

# export selectors (match the enum in vasmg_oracle.cpp)
MORTON, LEAF, LEAF_SORTED, CELLS, LATTICE, P_RP, P_CI, P_W, A_RP, A_CI, A_V, DEAD, COLOUR, DINV, BOX, LIFT, VOL = range(17)


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile liboracle.so (or, parallel=True, liboracle_omp.so: the same
    source with -fopenmp) next to its source (plain g++, IEEE semantics)."""
    out = _LIB_OMP if parallel else _LIB
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
            if parallel:
                cmd.append("-fopenmp")
            subprocess.run(cmd + [_SRC, "-o", tmp], check=True)
            os.replace(tmp, out)
    return out


def _load(parallel: bool = False):
    lib = _libs.get(parallel)
    if lib is None:
        lib = C.CDLL(build(parallel=parallel))
        P = C.c_void_p
        lib.or_setup.argtypes = [C.c_int, C.c_int64, P, C.c_int64, P, P, P, C.c_int64, P, P, C.c_int, C.c_int64,
                                 P, C.POINTER(C.c_void_p)]
        lib.or_setup.restype = C.c_int
        lib.or_set_smoother.argtypes = [P, C.c_int]
        lib.or_set_smoother.restype = C.c_int
        lib.or_setup_fine.argtypes = [C.c_int, C.c_int64, P, C.c_int64, P, P, P, C.c_int64, P, P, C.c_int,
                                      C.POINTER(C.c_void_p)]
        lib.or_setup_fine.restype = C.c_int
        lib.or_destroy.argtypes = [P]
        lib.or_num_levels.argtypes = [P]
        lib.or_level_info.argtypes = [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int32)]
        lib.or_export.argtypes = [P, C.c_int, C.c_int, P]
        lib.or_export.restype = C.c_int64
        lib.or_assemble_load.argtypes = [P, P, P]
        lib.or_apply_A.argtypes = [P, C.c_int, P, P]
        lib.or_gs_sweep.argtypes = [P, C.c_int, P, P, C.c_int]
        lib.or_vcycle.argtypes = [P, C.c_int, P, P]
        lib.or_restrict.argtypes = [P, C.c_int, P, P]
        lib.or_prolong_add.argtypes = [P, C.c_int, P, P]
        lib.or_coarse_solve.argtypes = [P, P, P]
        lib.or_solve.argtypes = [P, P, P, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), P,
                                 C.c_int, C.c_int]
        lib.or_splitmix64.argtypes = [C.c_uint64]
        lib.or_splitmix64.restype = C.c_uint64
        lib.or_set_cycle.argtypes = [P, C.c_int, C.c_int]
        lib.or_set_cycle.restype = C.c_int
        lib.or_precondition.argtypes = [P, P, P]
        lib.or_precondition.restype = C.c_int
        lib.or_set_threads.argtypes = [C.c_int]
        lib.or_set_threads.restype = C.c_int
        _libs[parallel] = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """Setup + solve of V-ASMG-PCG on the CPU in FP64 (one hierarchy)."""

    def __init__(self, prob: dict, threshold: int = 0, coarse_max_dofs: int = 0, insertion_order=None,
                 fine_only: bool = False, threads: int = 1):
        """fine_only: assembly, Dirichlet rows and keys only (apply_A(0), the
        load, keys and sorted-key leaves work; nothing of the hierarchy).
        threads > 1: the OpenMP build, its row loops on that many threads
        (self.threads is the count it reports)."""
        lib = _load(parallel=threads > 1)
        self.threads = int(lib.or_set_threads(int(threads))) if threads > 1 else 1
        self.dim = int(prob["dim"])
        self.coords = np.ascontiguousarray(prob["coords"], dtype=np.float64)
        self.elems = np.ascontiguousarray(prob["elems"], dtype=np.int32)
        self.nv = self.coords.shape[0]
        self.n = self.nv * self.dim
        lam = np.ascontiguousarray(np.broadcast_to(prob["lam"], (self.elems.shape[0],)), dtype=np.float64)
        mu = np.ascontiguousarray(np.broadcast_to(prob["mu"], (self.elems.shape[0],)), dtype=np.float64)
        dd = np.ascontiguousarray(prob.get("dirichlet_dofs", np.zeros(0, np.int64)), dtype=np.int64)
        dv = prob.get("dirichlet_values")
        dv = None if dv is None else np.ascontiguousarray(dv, dtype=np.float64)
        order = None if insertion_order is None else np.ascontiguousarray(insertion_order, dtype=np.int64)
        h = C.c_void_p()
        if fine_only:
            rc = lib.or_setup_fine(self.dim, self.nv, _ptr(self.coords), self.elems.shape[0], _ptr(self.elems),
                                   _ptr(lam), _ptr(mu), dd.size, _ptr(dd), _ptr(dv), int(threshold), C.byref(h))
        else:
            rc = lib.or_setup(self.dim, self.nv, _ptr(self.coords), self.elems.shape[0], _ptr(self.elems), _ptr(lam),
                              _ptr(mu), dd.size, _ptr(dd), _ptr(dv), int(threshold), int(coarse_max_dofs),
                              _ptr(order), C.byref(h))
        if rc != 0:
            raise RuntimeError(f"oracle setup failed ({rc})")
        self._h = h
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_destroy(h)
            self._h = None

    # -- structure -----------------------------------------------------------------
    @property
    def num_levels(self) -> int:
        return self._lib.or_num_levels(self._h)

    def level_info(self, l: int):
        nv, nnzb, nc = C.c_int64(), C.c_int64(), C.c_int32()
        if self._lib.or_level_info(self._h, l, C.byref(nv), C.byref(nnzb), C.byref(nc)) != 0:
            raise IndexError(l)
        return nv.value, nnzb.value, nc.value

    def export(self, what: int, level: int = 0, dtype=np.int64):
        nbytes = self._lib.or_export(self._h, what, level, None)
        if nbytes < 0:
            raise ValueError("bad export")
        buf = np.empty(nbytes // np.dtype(dtype).itemsize, dtype=dtype)
        self._lib.or_export(self._h, what, level, _ptr(buf))
        return buf

    def operator(self, l: int):
        """(rowptr int64, cols int32, blocks f64[nnzb, d, d]) of level l."""
        rp = self.export(A_RP, l, np.int64)
        ci = self.export(A_CI, l, np.int32)
        v = self.export(A_V, l, np.float64).reshape(-1, self.dim, self.dim)
        return rp, ci, v

    def prolongation(self, l: int):
        return (self.export(P_RP, l, np.int64), self.export(P_CI, l, np.int32), self.export(P_W, l, np.float64))

    def colours(self, l: int):
        return self.export(COLOUR, l, np.int32)

    def dead(self, l: int):
        return self.export(DEAD, l, np.uint8)

    def lattice(self, l: int):
        return self.export(LATTICE, l, np.uint64)

    def cells(self, l: int):
        return self.export(CELLS, l, np.int64).reshape(-1, 2)

    def leaves(self, sorted_method: bool = False):
        return self.export(LEAF_SORTED if sorted_method else LEAF, 0, np.int64).reshape(-1, 2)

    def morton(self):
        return self.export(MORTON, 0, np.uint64)

    def box(self):
        return self.export(BOX, 0, np.float64)

    def volumes(self):
        return self.export(VOL, 0, np.float64)

    def nv_level(self, l: int) -> int:
        return self.level_info(l)[0]

    # -- arithmetic ------------------------------------------------------------------
    def assemble_load(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        F = np.empty(self.n)
        self._lib.or_assemble_load(self._h, _ptr(f), _ptr(F))
        return F

    def apply_A(self, l: int, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        self._lib.or_apply_A(self._h, l, _ptr(x), _ptr(y))
        return y

    def set_smoother(self, smoother: str):
        """'multicolour' (point-block GS by colours, the GPU path's smoother) or
        'lexicographic' (the paper's scalar GS in component-major order)."""
        rc = self._lib.or_set_smoother(self._h, {"multicolour": 0, "lexicographic": 1}[smoother])
        if rc != 0:
            raise RuntimeError("or_set_smoother failed")

    def set_cycle(self, gamma: int = 1, additive: bool = False):
        """gamma coarse corrections per level (1: V-cycle, 2: W-cycle);
        additive: the preconditioner B_h = S_h + Pi B_0 Pi^T (Sec. 4), with
        S_h symmetric GS and B_0 the cycle on level 1."""
        if self._lib.or_set_cycle(self._h, int(gamma), 1 if additive else 0) != 0:
            raise RuntimeError("or_set_cycle failed")

    def precondition(self, r):
        """z = B r, the preconditioner PCG applies (current cycle variant)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty_like(r)
        self._lib.or_precondition(self._h, _ptr(r), _ptr(z))
        return z

    def gs_sweep(self, l: int, b, x, forward=True):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.array(x, dtype=np.float64, copy=True)
        self._lib.or_gs_sweep(self._h, l, _ptr(b), _ptr(x), 1 if forward else 0)
        return x

    def vcycle(self, b, level: int = 0):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        self._lib.or_vcycle(self._h, level, _ptr(b), _ptr(x))
        return x

    def restrict(self, l: int, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        bc = np.empty(self.nv_level(l + 1) * self.dim)
        self._lib.or_restrict(self._h, l, _ptr(r), _ptr(bc))
        return bc

    def prolong_add(self, l: int, ec, x):
        ec = np.ascontiguousarray(ec, dtype=np.float64)
        x = np.array(x, dtype=np.float64, copy=True)
        self._lib.or_prolong_add(self._h, l, _ptr(ec), _ptr(x))
        return x

    def coarse_solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        self._lib.or_coarse_solve(self._h, _ptr(b), _ptr(x))
        return x

    def solve(self, F, tol=1e-6, max_iters=1000, precondition=True, hist_cap=0):
        """PCG (Alg. 2).  Returns (U, iterations, rel_res, status, history)."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        U = np.empty(self.n)
        it, rr = C.c_int(), C.c_double()
        hist = np.zeros(max(hist_cap, 1))
        st = self._lib.or_solve(self._h, _ptr(F), _ptr(U), float(tol), int(max_iters), C.byref(it), C.byref(rr),
                                _ptr(hist), int(hist_cap), 1 if precondition else 0)
        return U, it.value, rr.value, st, hist[: min(it.value, hist_cap)]


def splitmix64(x: int) -> int:
    return int(_load().or_splitmix64(C.c_uint64(x)))
