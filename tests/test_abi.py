"""The C-ABI library builds, loads without a GPU, and exports every symbol that
include/vasmg.h declares.  No compute call is made here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09064_gb300 import _build, vasmg

    _build.build()
    return vasmg.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "vasmg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vasmg_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2505_09064_gb300", "libvasmg.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for n in names:
        assert n in exported, n
        assert getattr(lib, n) is not None


def test_binding_lists_the_same_symbols():
    from paper_2505_09064_gb300 import vasmg

    assert sorted(vasmg.EXPORTED) == _declared()


def test_host_only_calls(lib):
    from paper_2505_09064_gb300 import vasmg

    o = vasmg.vasmg_default_options(2)
    assert o.leaf_threshold == 4 and o.n_pre == 1 and o.max_iters == 1000
    o3 = vasmg.vasmg_default_options(3)
    assert o3.leaf_threshold == 8
    assert lib.vasmg_default_options(4, C.byref(o)) == vasmg.VASMG_ERR_INVALID_ARG
    assert lib.vasmg_error_string(vasmg.VASMG_ERR_BREAKDOWN).decode().startswith("PCG breakdown")
    h = C.c_void_p()
    assert lib.vasmg_setup(None, None, C.byref(h)) == vasmg.VASMG_ERR_INVALID_ARG
    assert lib.vasmg_num_levels(None) == vasmg.VASMG_ERR_INVALID_ARG
    assert lib.vasmg_destroy(None) == vasmg.VASMG_ERR_INVALID_ARG
    so = vasmg.vasmg_server_opts()
    assert lib.vasmg_server_default_opts(C.byref(so)) == 0
    assert so.slots == 4 and so.tol == 1e-6 and so.precision == 1 and so.memory_budget == 0
    assert lib.vasmg_server_poll(None, 1, 0, None) == vasmg.VASMG_ERR_INVALID_ARG
    assert lib.vasmg_server_destroy(None) == vasmg.VASMG_ERR_INVALID_ARG
    assert lib.vasmg_coarse_solve_noalloc(None, None, None, None) == vasmg.VASMG_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    """ctypes mirrors of the structs have the sizes of the C structs."""
    from paper_2505_09064_gb300 import vasmg

    # sizes computed by the C compiler from the header itself
    prog = ('#include <stdio.h>\n#include "vasmg.h"\nint main(){printf("%zu %zu %zu %zu %zu\\n", '
            'sizeof(vasmg_problem), sizeof(vasmg_options), sizeof(vasmg_stats), sizeof(vasmg_server_opts), '
            'sizeof(vasmg_request_stats));return 0;}\n')
    import tempfile

    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "p.c")
        exe = os.path.join(td, "p")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert sizes == [C.sizeof(vasmg.vasmg_problem), C.sizeof(vasmg.vasmg_options), C.sizeof(vasmg.vasmg_stats),
                     C.sizeof(vasmg.vasmg_server_opts), C.sizeof(vasmg.vasmg_request_stats)]


def test_vector_arguments_are_checked_before_the_call():
    """Solver.solve / assemble_load pass raw pointers: a vector of another
    dtype or length is refused in Python, before the library reads it."""
    import torch

    from paper_2505_09064_gb300 import vasmg

    vasmg._check_vec(np.zeros(6), 6, "F")
    vasmg._check_vec(torch.zeros(6, dtype=torch.float64), 6, "F")
    with pytest.raises(TypeError):
        vasmg._check_vec(np.zeros(6, dtype=np.float32), 6, "F")
    with pytest.raises(TypeError):
        vasmg._check_vec(torch.zeros(6, dtype=torch.float32), 6, "F")
    with pytest.raises(ValueError):
        vasmg._check_vec(np.zeros(5), 6, "U")
    with pytest.raises(TypeError):
        vasmg._check_vec([0.0] * 6, 6, "U")


def test_noalloc_binding_refuses_host_vectors_before_the_call():
    """vasmg_coarse_solve_noalloc reads its vectors on the device: the binding
    refuses numpy arrays and CPU tensors before any pointer reaches the
    library (the handle is never touched, so a dummy one suffices)."""
    import ctypes as C

    import torch

    from paper_2505_09064_gb300 import vasmg

    dummy = C.c_void_p(1)
    with pytest.raises(TypeError):
        vasmg.vasmg_coarse_solve_noalloc(dummy, np.zeros(8), np.zeros(8))
    with pytest.raises(TypeError):
        vasmg.vasmg_coarse_solve_noalloc(dummy, torch.zeros(8, dtype=torch.float64),
                                         torch.zeros(8, dtype=torch.float64))
