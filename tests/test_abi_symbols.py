"""The C-ABI library builds, loads and exports every function declared in
include/*.h (no GPU needed: nothing is computed here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double|int64_t)\s*\**\s*(\w+)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ef_plan_create", "ef_assemble", "rt0_assemble", "ned_assemble", "ef_plan_pattern",
                     "ef_plan_topology", "ef_plan_destroy", "ef_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1409_4618_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1409_4618_gb300 import edgefem as ef

    lib = ef.load()
    assert lib.ef_status_string(ef.EF_ERR_DEGENERATE).decode().startswith("degenerate")
    assert lib.ef_status_string(12345).decode() == "unknown status"


def test_argument_errors_need_no_gpu():
    """Argument checks run before any CUDA call."""
    from paper_1409_4618_gb300 import edgefem as ef

    lib = ef.load()
    h = ctypes.c_void_p()
    assert lib.ef_plan_create(3, 3, 10, 1, None, None, ctypes.byref(h)) == ef.EF_ERR_ARG      # bad kind
    assert lib.ef_plan_create(1, 4, 10, 1, None, None, ctypes.byref(h)) == ef.EF_ERR_ARG      # bad dim
    assert lib.ef_plan_create(1, 3, 10, 5, None, None, ctypes.byref(h)) == ef.EF_ERR_ARG      # no elements
    assert lib.ef_plan_create(1, 3, 2642246, 1, ctypes.c_void_p(16), None,
                              ctypes.byref(h)) == ef.EF_ERR_KEY_OVERFLOW
    assert lib.ef_plan_create(2, 3, 1 << 31, 1, ctypes.c_void_p(16), None, ctypes.byref(h)) == ef.EF_ERR_SIZE
    assert lib.ef_plan_create(2, 3, 100, 1 << 28, ctypes.c_void_p(16), None, ctypes.byref(h)) == ef.EF_ERR_SIZE
    assert lib.ef_assemble(None, None, None, None, None, None) == ef.EF_ERR_ARG
    assert lib.ef_assemble_noalloc(None, None, None, None, None, None) == ef.EF_ERR_ARG
    assert lib.ef_plan_set_fused(None, None, 128, None) == ef.EF_ERR_ARG
    assert lib.ef_batch_assemble(None, None, None, None, None, None) == ef.EF_ERR_ARG
    assert lib.ef_batch_plan_create(1, 3, 0, None, None, None, None, ctypes.byref(h)) == ef.EF_ERR_ARG
    assert lib.ef_batch_plan_create(3, 3, 1, None, None, None, None, ctypes.byref(h)) == ef.EF_ERR_ARG
    rate, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.ef_fp64_probe(7, 10, ctypes.c_void_p(16), ctypes.byref(rate), ctypes.byref(ms), None) == ef.EF_ERR_ARG
    assert lib.ef_int_mul_check(ctypes.c_int64(-1), ctypes.c_uint64(0), ctypes.c_void_p(16), None) == ef.EF_ERR_ARG
    assert lib.ef_int_mul_check(ctypes.c_int64(10), ctypes.c_uint64(0), None, None) == ef.EF_ERR_ARG
    assert lib.ef_fp64_probe(0, 0, ctypes.c_void_p(16), ctypes.byref(rate), ctypes.byref(ms), None) == ef.EF_ERR_ARG
    assert lib.ef_fp64_probe(0, 10, None, ctypes.byref(rate), ctypes.byref(ms), None) == ef.EF_ERR_ARG
    assert h.value is None


def test_binding_rejects_wrong_sizes_before_the_library():
    """The C ABI takes plain pointers; the binding checks every tensor against
    the plan's sizes first (no GPU needed: the checks run before any call)."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    plan = ef.Plan.__new__(ef.Plan)
    plan.kind, plan.dim, plan.n_nodes, plan.n_elems = ef.EF_NED1, 3, 27, 48
    plan.n_dofs, plan.nnz, plan.nloc = 98, 1000, 6
    plan._h = None
    ok = torch.zeros(27 * 3, dtype=torch.float64)
    for call in (lambda: plan.assemble(torch.zeros(80, dtype=torch.float64)),
                 lambda: plan.assemble(ok, torch.zeros(47, dtype=torch.float64)),
                 lambda: plan.assemble(ok, None, torch.zeros(999, dtype=torch.float64)),
                 lambda: plan.fe_curl(ok, torch.zeros(97, dtype=torch.float64)),
                 lambda: plan.load_vector(ok, torch.zeros((8, 48, 2), dtype=torch.float64), 2),
                 lambda: plan.load_vector(ok, torch.zeros((27, 48, 3), dtype=torch.float64), 2),
                 lambda: plan.load_derivative(ok, torch.zeros((8, 48, 1), dtype=torch.float64), 2),
                 lambda: plan.norm_l2(ok, torch.zeros((8, 47, 3), dtype=torch.float64), 2),
                 lambda: plan.norm_l2_derivative(ok, torch.zeros((8, 48, 3), dtype=torch.float64), 2,
                                                 torch.zeros(99, dtype=torch.float64)),
                 lambda: plan.adjoint(ok, None, torch.zeros(98, dtype=torch.float64),
                                      torch.zeros(97, dtype=torch.float64)),
                 lambda: plan.assemble_noalloc(ok, None, torch.zeros(999, dtype=torch.float64)),
                 lambda: plan.set_fused(torch.zeros(80, dtype=torch.float64), 128)):
        with pytest.raises(ValueError, match="entries|shape"):   # not the closed-handle error
            call()


def test_batch_binding_rejects_wrong_sizes_before_the_library():
    """The batch calls take host tables of device pointers; the binding checks
    the number of meshes and each buffer's size first (no GPU needed)."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    b = ef.Batch.__new__(ef.Batch)
    b.kind, b.dim, b.n = ef.EF_NED1, 3, 2
    b.n_nodes, b.n_elems, b.nnz, b.n_dofs = [27, 8], [48, 6], [1000, 100], [98, 19]
    b._h = None
    nodes = [torch.zeros(81, dtype=torch.float64), torch.zeros(24, dtype=torch.float64)]
    K = [torch.zeros(1000, dtype=torch.float64), torch.zeros(100, dtype=torch.float64)]
    with pytest.raises(ValueError, match="meshes"):
        b.tables(nodes[:1], None, K, K)
    with pytest.raises(ValueError, match="entries"):
        b.tables(nodes, None, [K[0], torch.zeros(99, dtype=torch.float64)], K)
    with pytest.raises(ValueError, match="entries"):
        b.tables(nodes, [torch.zeros(48, dtype=torch.float64), torch.zeros(5, dtype=torch.float64)], K, K)
