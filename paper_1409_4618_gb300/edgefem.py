"""Python binding of libedgefem.so (include/edgefem.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch only provides device
memory and the current stream. There is no CPU path: if the library is not
built or no CUDA device is present, the calls raise.

Names follow the C ABI: ``ef_plan_create``, ``ef_assemble``, ...; ``Plan``
bundles a plan handle with its sizes, ``rt0_assemble`` / ``ned_assemble``
are the one-shot calls, and ``energy`` wraps ``ef_adjoint`` as a
differentiable function of the node coordinates and coefficients.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

EF_RT0 = 1
EF_NED1 = 2

EF_OK = 0
EF_ERR_ARG = -1
EF_ERR_RANGE = -2
EF_ERR_DEGENERATE = -3
EF_ERR_KEY_OVERFLOW = -4
EF_ERR_OOM = -5
EF_ERR_CUDA = -6
EF_ERR_TIMEOUT = -7
EF_ERR_SIZE = -8

_lock = threading.Lock()
_lib = None


class EdgeFemError(RuntimeError):
    def __init__(self, code: int, text: str, detail: str = ""):
        msg = f"edgefem status {code}: {text}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)
        self.code = code


class PlanInfo(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("nnz", C.c_int64), ("n_upper", C.c_int64), ("n_contrib", C.c_int64),
                ("assemble_launches", C.c_int32), ("fused_block", C.c_int32), ("fused_blocks", C.c_int64),
                ("fused_partial", C.c_int64), ("pipeline_chunks", C.c_int32), ("fused_sfc", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchConfig(C.Structure):
    _fields_ = [("elems_per_tile", C.c_int32), ("sum_tile", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("dynamic", C.c_int32), ("largest_first", C.c_int32), ("elem_ctas", C.c_int32),
                ("two_launch", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _CSR(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("nnz", C.c_int64), ("d_rowptr", C.c_void_p), ("d_colidx", C.c_void_p),
                ("d_K", C.c_void_p), ("d_M", C.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libedgefem.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libedgefem.so not found at {_build.LIB}; run python -m paper_1409_4618_gb300.build")
        lib = C.CDLL(_build.LIB)
        P, I64, I = C.c_void_p, C.c_int64, C.c_int
        sig = {
            "ef_plan_create": ([I, I, I64, I64, P, P, C.POINTER(P)], I),
            "ef_plan_sizes": ([P, C.POINTER(I64), C.POINTER(I64)], I),
            "ef_plan_pattern": ([P, P, P, P], I),
            "ef_plan_info": ([P, C.POINTER(PlanInfo)], I),
            "ef_plan_set_block": ([P, I, P], I),
            "ef_plan_set_fused": ([P, P, I, P], I),
            "ef_plan_set_pipeline": ([P, I, P], I),
            "ef_plan_inject_stall": ([P, I, P], I),
            "ef_plan_tune": ([P, P, P, P, P, I, C.POINTER(C.c_int), P], I),
            "ef_plan_profile": ([P, I], I),
            "ef_plan_profile_read": ([P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)], I),
            "ef_plan_topology": ([P, P, P, P, P], I),
            "ef_assemble": ([P, P, P, P, P, P], I),
            "ef_assemble_two_pass": ([P, P, P, P, P, P], I),
            "ef_assemble2": ([P, P, P, P, P, P, P], I),
            "ef_assemble_host": ([P, P, P, P, P, P], I),
            "ef_assemble_noalloc": ([P, P, P, P, P, P], I),
            "ef_plan_check": ([P, P], I),
            "ef_adjoint": ([P, P, P, P, P, P, P, P, P], I),
            "ef_plan_destroy": ([P], None),
            "rt0_assemble": ([I, P, I64, P, I64, P, C.POINTER(_CSR), P], I),
            "ned_assemble": ([I, P, I64, P, I64, P, C.POINTER(_CSR), P], I),
            "ef_csr_free": ([C.POINTER(_CSR)], None),
            "ef_batch_create": ([I, I, I, P, P, P, P, C.POINTER(P)], I),
            "ef_batch_sizes": ([P, P, P], I),
            "ef_batch_pattern": ([P, I, P, P, P], I),
            "ef_batch_bind": ([P, P, P, P, P, P], I),
            "ef_batch_assemble_bound": ([P, P], I),
            "ef_batch_plan_create": ([I, I, I, P, P, P, P, C.POINTER(P)], I),
            "ef_batch_assemble": ([P, P, P, P, P, P], I),
            "ef_batch_plan_destroy": ([P], None),
            "ef_batch_tune": ([P, I, C.POINTER(BatchConfig), P], I),
            "ef_batch_get_config": ([P, C.POINTER(BatchConfig)], I),
            "ef_batch_set_config": ([P, C.POINTER(BatchConfig), P], I),
            "ef_batch_check": ([P, P], I),
            "ef_batch_destroy": ([P], None),
            "ef_quad_rule": ([I, I, P, P, I, C.POINTER(C.c_int)], I),
            "ef_quad_points": ([P, P, I, P, P], I),
            "ef_fe_values": ([P, P, P, I, P, P], I),
            "ef_norm_l2": ([P, P, I, I, P, P, P, P, P], I),
            "ef_fe_curl": ([P, P, P, P, P], I),
            "ef_norm_l2_derivative": ([P, P, I, P, P, P, P, P], I),
            "ef_load_vector": ([P, P, I, P, P, P], I),
            "ef_load_derivative": ([P, P, I, P, P, P], I),
            "ef_fp64_probe": ([I, I64, P, C.POINTER(C.c_double), C.POINTER(C.c_double), P], I),
            "ef_int_mul_check": ([I64, C.c_uint64, P, P], I),
            "ef_status_string": ([I], C.c_char_p),
            "ef_last_error": ([], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(st: int):
    if st != EF_OK:
        lib = load()
        raise EdgeFemError(st, lib.ef_status_string(st).decode(), lib.ef_last_error().decode())


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")
    return C.c_void_p(t.data_ptr())


def _host(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CPU tensor of dtype {dtype}")
    return C.c_void_p(t.data_ptr())


def ef_plan_create(kind: int, dim: int, n_nodes: int, elems: torch.Tensor, stream=None) -> C.c_void_p:
    lib = load()
    h = C.c_void_p()
    _check(lib.ef_plan_create(kind, dim, int(n_nodes), int(elems.shape[0]), _dev(elems, torch.int32, "elems"),
                              _stream_ptr(stream), C.byref(h)))
    return h


def ef_plan_sizes(plan) -> tuple[int, int]:
    n, z = C.c_int64(), C.c_int64()
    _check(load().ef_plan_sizes(plan, C.byref(n), C.byref(z)))
    return n.value, z.value


def ef_plan_info(plan) -> dict:
    info = PlanInfo()
    _check(load().ef_plan_info(plan, C.byref(info)))
    return info.as_dict()


def ef_plan_profile(plan, max_calls: int):
    _check(load().ef_plan_profile(plan, int(max_calls)))


def ef_plan_profile_read(plan) -> tuple[float, float, int]:
    """(ms of the first kernel, ms of the second, calls) summed over the recorded ef_assemble calls."""
    a, b, n = C.c_double(), C.c_double(), C.c_int()
    _check(load().ef_plan_profile_read(plan, C.byref(a), C.byref(b), C.byref(n)))
    return a.value, b.value, n.value


def ef_plan_set_block(plan, block: int, stream=None):
    _check(load().ef_plan_set_block(plan, int(block), _stream_ptr(stream)))


def ef_plan_pattern(plan, rowptr: torch.Tensor, colidx: torch.Tensor, stream=None):
    _check(load().ef_plan_pattern(plan, _dev(rowptr, torch.int64, "rowptr"), _dev(colidx, torch.int32, "colidx"),
                                  _stream_ptr(stream)))


def ef_plan_topology(plan, elem2dof=None, signbits=None, dof2nodes=None, stream=None):
    _check(load().ef_plan_topology(plan, _dev(elem2dof, torch.int32, "elem2dof"), _dev(signbits, torch.uint8, "signbits"),
                                   _dev(dof2nodes, torch.int32, "dof2nodes"), _stream_ptr(stream)))


def ef_assemble(plan, nodes, coeff, K, M, stream=None):
    _check(load().ef_assemble(plan, _dev(nodes, torch.float64, "nodes"), _dev(coeff, torch.float64, "coeff"),
                              _dev(K, torch.float64, "K"), _dev(M, torch.float64, "M"), _stream_ptr(stream)))


def ef_assemble2(plan, nodes, coeff_K, coeff_M, K, M, stream=None):
    _check(load().ef_assemble2(plan, _dev(nodes, torch.float64, "nodes"), _dev(coeff_K, torch.float64, "coeff_K"),
                               _dev(coeff_M, torch.float64, "coeff_M"), _dev(K, torch.float64, "K"),
                               _dev(M, torch.float64, "M"), _stream_ptr(stream)))


def ef_assemble_two_pass(plan, nodes, coeff, K, M, stream=None):
    _check(load().ef_assemble_two_pass(plan, _dev(nodes, torch.float64, "nodes"), _dev(coeff, torch.float64, "coeff"),
                                       _dev(K, torch.float64, "K"), _dev(M, torch.float64, "M"), _stream_ptr(stream)))


def ef_assemble_noalloc(plan, nodes, coeff, K, M, stream=None):
    _check(load().ef_assemble_noalloc(plan, _dev(nodes, torch.float64, "nodes"), _dev(coeff, torch.float64, "coeff"),
                                      _dev(K, torch.float64, "K"), _dev(M, torch.float64, "M"), _stream_ptr(stream)))


def ef_assemble_host(plan, nodes, coeff, K, M, stream=None):
    _check(load().ef_assemble_host(plan, _host(nodes, torch.float64, "nodes"), _host(coeff, torch.float64, "coeff"),
                                   _host(K, torch.float64, "K"), _host(M, torch.float64, "M"), _stream_ptr(stream)))


def ef_adjoint(plan, nodes, coeff, u, v, J=None, grad_nodes=None, grad_coeff=None, stream=None):
    _check(load().ef_adjoint(plan, _dev(nodes, torch.float64, "nodes"), _dev(coeff, torch.float64, "coeff"),
                             _dev(u, torch.float64, "u"), _dev(v, torch.float64, "v"), _dev(J, torch.float64, "J"),
                             _dev(grad_nodes, torch.float64, "grad_nodes"), _dev(grad_coeff, torch.float64, "grad_coeff"),
                             _stream_ptr(stream)))


def ef_fp64_probe(op: int, iters: int, stream=None) -> tuple[float, float]:
    """(lane operations per second, ms) for op 0 = DFMA, 1 = DADD, 2 = DMUL,
    3 = the integer-pipe multiply, 4 = DFMA and the integer-pipe multiply in
    half of the chains each, 5 = DFMA with literal operands, 6 = an addition as
    a DFMA with a per-thread 1.0."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    rate, ms = C.c_double(), C.c_double()
    _check(load().ef_fp64_probe(int(op), int(iters), C.c_void_p(sink.data_ptr()), C.byref(rate), C.byref(ms),
                                _stream_ptr(stream)))
    return rate.value, ms.value


def ef_int_mul_check(n: int, seed: int, stream=None) -> tuple[int, int]:
    """(pairs handed to the FP64 instruction, mismatching pairs) of the
    integer-pipe multiply against the FP64 multiply on n generated pairs."""
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    _check(load().ef_int_mul_check(int(n), C.c_uint64(int(seed) & (2**64 - 1)), C.c_void_p(counts.data_ptr()),
                                   _stream_ptr(stream)))
    flagged, mismatched = counts.cpu().tolist()
    return flagged, mismatched


def ef_plan_check(plan, stream=None):
    _check(load().ef_plan_check(plan, _stream_ptr(stream)))


def ef_plan_destroy(plan):
    load().ef_plan_destroy(plan)


class _DevArray:
    """Exposes a raw device pointer through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}


def _one_shot(fn, dim, nodes, elems, coeff, stream):
    lib = load()
    csr = _CSR()
    _check(getattr(lib, fn)(dim, _dev(nodes, torch.float64, "nodes"), int(nodes.shape[0]),
                            _dev(elems, torch.int32, "elems"), int(elems.shape[0]),
                            _dev(coeff, torch.float64, "coeff"), C.byref(csr), _stream_ptr(stream)))
    try:
        out = {}
        for key, ptr, n, ts, dt in (("rowptr", csr.d_rowptr, csr.n_dofs + 1, "<i8", torch.int64),
                                    ("colidx", csr.d_colidx, csr.nnz, "<i4", torch.int32),
                                    ("K", csr.d_K, csr.nnz, "<f8", torch.float64),
                                    ("M", csr.d_M, csr.nnz, "<f8", torch.float64)):
            if n > 0:
                out[key] = torch.as_tensor(_DevArray(ptr, n, ts), device=nodes.device).clone()
            else:
                out[key] = torch.zeros(0, dtype=dt, device=nodes.device)
        torch.cuda.current_stream().synchronize()
        return out
    finally:
        lib.ef_csr_free(C.byref(csr))


def rt0_assemble(dim: int, nodes: torch.Tensor, elems: torch.Tensor, coeff=None, stream=None) -> dict:
    """One-shot RT0 assembly -> dict(rowptr, colidx, K, M) of CUDA tensors."""
    return _one_shot("rt0_assemble", dim, nodes, elems, coeff, stream)


def ned_assemble(dim: int, nodes: torch.Tensor, elems: torch.Tensor, coeff=None, stream=None) -> dict:
    """One-shot Nedelec assembly -> dict(rowptr, colidx, K, M) of CUDA tensors."""
    return _one_shot("ned_assemble", dim, nodes, elems, coeff, stream)


class Plan:
    """A per-mesh plan (topology + CSR pattern) and the calls that use it."""

    def __init__(self, kind: int, dim: int, n_nodes: int, elems: torch.Tensor, stream=None):
        self.kind, self.dim, self.n_nodes = kind, dim, int(n_nodes)
        self.n_elems = int(elems.shape[0])
        self.device = elems.device
        self._h = ef_plan_create(kind, dim, n_nodes, elems, stream)
        self.n_dofs, self.nnz = ef_plan_sizes(self._h)
        self.nloc = 3 if dim == 2 else (4 if kind == EF_RT0 else 6)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("plan is closed")
        return self._h

    # The C ABI takes plain pointers and cannot see buffer sizes; the binding
    # knows the plan's and rejects a wrong-sized tensor before the library
    # would read or write past its end.
    def _need(self, t, numel: int, name: str):
        if t is not None and isinstance(t, torch.Tensor) and t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} entries; this plan needs {numel}")

    def _need_mesh(self, nodes, coeff=None, K=None, M=None, coeff_name="coeff"):
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need(coeff, self.n_elems, coeff_name)
        self._need(K, self.nnz, "K")
        self._need(M, self.nnz, "M")

    def _need_points(self, t, n: int, ncomp: int, name: str):
        shape = (int(n) ** self.dim, self.n_elems, ncomp)
        if not isinstance(t, torch.Tensor) or tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape} (points, elements, components)")

    def info(self) -> dict:
        return ef_plan_info(self.handle)

    def profile(self, max_calls: int):
        """Record per-kernel CUDA events for the next max_calls assemble calls (0 stops)."""
        ef_plan_profile(self.handle, max_calls)

    def profile_read(self) -> tuple[float, float, int]:
        return ef_plan_profile_read(self.handle)

    def set_block(self, block: int, stream=None):
        ef_plan_set_block(self.handle, block, stream)

    def set_fused(self, nodes, block: int, stream=None):
        """Element-block path with blocks along the Morton curve of the centroids under `nodes` (0: leave it)."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        _check(load().ef_plan_set_fused(self.handle, _dev(nodes, torch.float64, "nodes"), int(block),
                                        _stream_ptr(stream)))

    def set_pipeline(self, chunks: int, stream=None):
        _check(load().ef_plan_set_pipeline(self.handle, int(chunks), _stream_ptr(stream)))

    def inject_stall(self, on: bool, stream=None):
        """Fault injection for tests: the queue's sums wait for a tile that never completes, give up after about
        a second and the next check() raises EF_ERR_TIMEOUT; inject_stall(False) restores the schedule."""
        _check(load().ef_plan_inject_stall(self.handle, int(bool(on)), _stream_ptr(stream)))

    def tune(self, nodes, coeff=None, K=None, M=None, reps: int = 5, stream=None) -> int:
        """Pick the fastest ef_assemble schedule for this plan: 0 (two-pass), chunks*100 + elem_ctas*10 + (tile
        == 256) (persistent queue), -block (element-block path in mesh order) or -(block + 1) (element-block path
        along the Morton curve of the centroids)."""
        self._need_mesh(nodes, coeff, K, M)
        K, M = self._vals(K, M)
        chosen = C.c_int(0)
        _check(load().ef_plan_tune(self.handle, _dev(nodes, torch.float64, "nodes"), _dev(coeff, torch.float64, "coeff"),
                                   _dev(K, torch.float64, "K"), _dev(M, torch.float64, "M"), int(reps),
                                   C.byref(chosen), _stream_ptr(stream)))
        return chosen.value

    def pattern(self, stream=None):
        rowptr = torch.empty(self.n_dofs + 1, dtype=torch.int64, device=self.device)
        colidx = torch.empty(max(self.nnz, 0), dtype=torch.int32, device=self.device)
        ef_plan_pattern(self.handle, rowptr, colidx, stream)
        return rowptr, colidx

    def topology(self, stream=None):
        e2d = torch.empty((self.n_elems, self.nloc), dtype=torch.int32, device=self.device)
        sb = torch.empty(self.n_elems, dtype=torch.uint8, device=self.device)
        ent = 3 if (self.kind == EF_RT0 and self.dim == 3) else 2
        d2n = torch.empty((self.n_dofs, ent), dtype=torch.int32, device=self.device)
        ef_plan_topology(self.handle, e2d, sb, d2n, stream)
        return e2d, sb, d2n

    def _vals(self, K, M):
        if K is None:
            K = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        if M is None:
            M = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        return K, M

    def assemble(self, nodes, coeff=None, K=None, M=None, stream=None):
        self._need_mesh(nodes, coeff, K, M)
        K, M = self._vals(K, M)
        ef_assemble(self.handle, nodes, coeff, K, M, stream)
        return K, M

    def assemble_two_pass(self, nodes, coeff=None, K=None, M=None, stream=None):
        self._need_mesh(nodes, coeff, K, M)
        K, M = self._vals(K, M)
        ef_assemble_two_pass(self.handle, nodes, coeff, K, M, stream)
        return K, M

    def assemble_noalloc(self, nodes, coeff=None, K=None, M=None, stream=None):
        """ef_assemble_noalloc: the library allocates nothing (pass K and M to allocate nothing here either)."""
        self._need_mesh(nodes, coeff, K, M)
        K, M = self._vals(K, M)
        ef_assemble_noalloc(self.handle, nodes, coeff, K, M, stream)
        return K, M

    def assemble2(self, nodes, coeff_K=None, coeff_M=None, K=None, M=None, stream=None):
        """K weighted by coeff_K, M by coeff_M (e.g. 1/mu and kappa)."""
        self._need_mesh(nodes, coeff_K, K, M, "coeff_K")
        self._need(coeff_M, self.n_elems, "coeff_M")
        K, M = self._vals(K, M)
        ef_assemble2(self.handle, nodes, coeff_K, coeff_M, K, M, stream)
        return K, M

    def assemble_host(self, nodes, coeff=None, K=None, M=None, stream=None):
        self._need_mesh(nodes, coeff, K, M)
        if K is None:
            K = torch.empty(self.nnz, dtype=torch.float64, pin_memory=True)
        if M is None:
            M = torch.empty(self.nnz, dtype=torch.float64, pin_memory=True)
        ef_assemble_host(self.handle, nodes, coeff, K, M, stream)
        return K, M

    def quad_points(self, nodes, n: int, stream=None):
        """Physical quadrature points [nq, n_elems, dim] (point-major)."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        nq = n ** self.dim
        x = torch.empty((nq, self.n_elems, self.dim), dtype=torch.float64, device=self.device)
        _check(load().ef_quad_points(self.handle, _dev(nodes, torch.float64, "nodes"), int(n),
                                     C.c_void_p(x.data_ptr()), _stream_ptr(stream)))
        return x

    def fe_values(self, nodes, v, n: int, stream=None):
        """Values [nq, n_elems, dim] of the FE function with DOF vector v at the quadrature points."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need(v, self.n_dofs, "v")
        nq = n ** self.dim
        out = torch.empty((nq, self.n_elems, self.dim), dtype=torch.float64, device=self.device)
        _check(load().ef_fe_values(self.handle, _dev(nodes, torch.float64, "nodes"), _dev(v, torch.float64, "v"),
                                   int(n), C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def norm_l2_derivative(self, nodes, g, n: int, v=None, per_element: bool = False, stream=None):
        """Squared L2 norm of g - D v_h (D = div for RT0, curl for Nedelec; D v_h omitted without v), g given at
        the quadrature points [nq, n_elems, nc] (nc 3 for 3D Nedelec, else 1): (total [1], per-element or None)."""
        nc = 3 if (self.kind == EF_NED1 and self.dim == 3) else 1
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need_points(g, n, nc, "g")
        self._need(v, self.n_dofs, "v")
        total = torch.empty(1, dtype=torch.float64, device=self.device)
        elem = torch.empty(self.n_elems, dtype=torch.float64, device=self.device) if per_element else None
        _check(load().ef_norm_l2_derivative(self.handle, _dev(nodes, torch.float64, "nodes"), int(n),
                                            _dev(g, torch.float64, "g"), _dev(v, torch.float64, "v"),
                                            None if elem is None else C.c_void_p(elem.data_ptr()),
                                            C.c_void_p(total.data_ptr()), _stream_ptr(stream)))
        return total, elem

    def fe_curl(self, nodes, v, stream=None):
        """Per-element curl (Nedelec: [n_elems] in 2D, [n_elems, 3] in 3D) or divergence (RT0: [n_elems])."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need(v, self.n_dofs, "v")
        shape = (self.n_elems, 3) if (self.kind == EF_NED1 and self.dim == 3) else (self.n_elems,)
        out = torch.empty(shape, dtype=torch.float64, device=self.device)
        _check(load().ef_fe_curl(self.handle, _dev(nodes, torch.float64, "nodes"), _dev(v, torch.float64, "v"),
                                 C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def load_vector(self, nodes, F, n: int, stream=None):
        """b_i = int F . eta_i, F given at the quadrature points [nq, n_elems, dim]."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need_points(F, n, self.dim, "F")
        b = torch.empty(self.n_dofs, dtype=torch.float64, device=self.device)
        _check(load().ef_load_vector(self.handle, _dev(nodes, torch.float64, "nodes"), int(n),
                                     _dev(F, torch.float64, "F"), C.c_void_p(b.data_ptr()), _stream_ptr(stream)))
        return b

    def load_derivative(self, nodes, g, n: int, stream=None):
        """b_i = int g . D eta_i (D = div for RT0, curl for Nedelec), g given at the quadrature points
        [nq, n_elems, nc] (nc 3 for 3D Nedelec, else 1)."""
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need_points(g, n, 3 if (self.kind == EF_NED1 and self.dim == 3) else 1, "g")
        b = torch.empty(self.n_dofs, dtype=torch.float64, device=self.device)
        _check(load().ef_load_derivative(self.handle, _dev(nodes, torch.float64, "nodes"), int(n),
                                         _dev(g, torch.float64, "g"), C.c_void_p(b.data_ptr()), _stream_ptr(stream)))
        return b

    def norm_l2(self, nodes, f, n: int, v=None, per_element: bool = False, stream=None):
        """Squared L2 norm of f (values [nq, n_elems, ncomp] at the quadrature points), minus the FE
        function of v if given: (total [1], per-element [n_elems] or None)."""
        if not isinstance(f, torch.Tensor) or f.dim() != 3:
            raise ValueError("f must be a [nq, n_elems, ncomp] tensor")
        self._need(nodes, self.n_nodes * self.dim, "nodes")
        self._need_points(f, n, int(f.shape[2]), "f")
        self._need(v, self.n_dofs, "v")
        total = torch.empty(1, dtype=torch.float64, device=self.device)
        elem = torch.empty(self.n_elems, dtype=torch.float64, device=self.device) if per_element else None
        _check(load().ef_norm_l2(self.handle, _dev(nodes, torch.float64, "nodes"), int(n), int(f.shape[2]),
                                 _dev(f, torch.float64, "f"), _dev(v, torch.float64, "v"),
                                 _dev(elem, torch.float64, "elem"), C.c_void_p(total.data_ptr()),
                                 _stream_ptr(stream)))
        return total, elem

    def adjoint(self, nodes, coeff, u, v, stream=None):
        """(J, dJ/dnodes, dJ/dcoeff) of J = u^T K u + v^T M v (3D Nedelec)."""
        self._need_mesh(nodes, coeff)
        self._need(u, self.n_dofs, "u")
        self._need(v, self.n_dofs, "v")
        J = torch.empty(1, dtype=torch.float64, device=self.device)
        gx = torch.empty((self.n_nodes, self.dim), dtype=torch.float64, device=self.device)
        gs = torch.empty(self.n_elems, dtype=torch.float64, device=self.device)
        ef_adjoint(self.handle, nodes, coeff, u, v, J, gx, gs, stream)
        return J, gx, gs

    def check(self, stream=None):
        ef_plan_check(self.handle, stream)

    def close(self):
        if self._h is not None:
            ef_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(tensors, dtype, name, allow_none=False):
    out = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        if t is None:
            if not allow_none:
                raise TypeError(f"{name}[{i}] is None")
            out[i] = None
        else:
            out[i] = _dev(t, dtype, f"{name}[{i}]")
    return out


def ef_quad_rule(dim: int, n: int):
    """Reference points [nq, dim] and weights [nq] of the library's rule (host)."""
    import numpy as np

    nq = C.c_int()
    _check(load().ef_quad_rule(dim, n, None, None, 0, C.byref(nq)))
    x = np.zeros((nq.value, dim))
    w = np.zeros(nq.value)
    _check(load().ef_quad_rule(dim, n, C.c_void_p(x.ctypes.data), C.c_void_p(w.ctypes.data), nq.value, C.byref(nq)))
    return x, w


class _Energy(torch.autograd.Function):
    """J = u^T K u + v^T M v as a function of (nodes, coeff); the gradient is
    the one ef_adjoint computes together with J."""

    @staticmethod
    def forward(ctx, nodes, coeff, u, v, plan):
        J, gx, gs = plan.adjoint(nodes, coeff, u, v)
        ctx.save_for_backward(gx, gs)
        ctx.has_coeff = coeff is not None
        return J.reshape(())

    @staticmethod
    def backward(ctx, gJ):
        gx, gs = ctx.saved_tensors
        return gJ * gx, (gJ * gs if ctx.has_coeff else None), None, None, None


def energy(plan: "Plan", nodes: torch.Tensor, coeff, u: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Differentiable J(nodes, coeff) = u^T K u + v^T M v of a 3D Nedelec plan
    (u, v fixed DOF vectors; no gradient flows to them)."""
    if u.requires_grad or v.requires_grad:
        raise ValueError("energy: u and v are constants (the library gives dJ/dnodes and dJ/dcoeff only)")
    return _Energy.apply(nodes, coeff, u, v, plan)


class Batch:
    """Many independent meshes, each to its own CSR (ef_batch_plan_create / ef_batch_assemble and the other
    ef_batch_* calls): buffers either passed per call (tables + assemble_tables) or bound once (bind +
    assemble)."""

    def __init__(self, kind: int, dim: int, n_nodes, elems, stream=None):
        lib = load()
        self.kind, self.dim, self.n = kind, dim, len(elems)
        self.device = elems[0].device
        nn = (C.c_int64 * self.n)(*[int(v) for v in n_nodes])
        ne = (C.c_int64 * self.n)(*[int(e.shape[0]) for e in elems])
        ep = _ptr_array(elems, torch.int32, "elems")
        self._h = C.c_void_p()
        _check(lib.ef_batch_plan_create(kind, dim, self.n, nn, ne, ep, _stream_ptr(stream), C.byref(self._h)))
        nd = (C.c_int64 * self.n)()
        nz = (C.c_int64 * self.n)()
        _check(lib.ef_batch_sizes(self._h, nd, nz))
        self.n_dofs, self.nnz = list(nd), list(nz)
        self.n_elems = [int(e.shape[0]) for e in elems]
        self.n_nodes = [int(v) for v in n_nodes]

    def pattern(self, mesh: int, stream=None):
        rowptr = torch.empty(self.n_dofs[mesh] + 1, dtype=torch.int64, device=self.device)
        colidx = torch.empty(self.nnz[mesh], dtype=torch.int32, device=self.device)
        _check(load().ef_batch_pattern(self._h, mesh, _dev(rowptr, torch.int64, "rowptr"),
                                       _dev(colidx, torch.int32, "colidx"), _stream_ptr(stream)))
        return rowptr, colidx

    def _check_sizes(self, nodes, coeff, K, M):
        # per-mesh sizes checked here: the C ABI takes plain pointer tables
        for name, ts, sizes in (("nodes", nodes, [v * self.dim for v in self.n_nodes]),
                                ("coeff", coeff, self.n_elems), ("K", K, self.nnz), ("M", M, self.nnz)):
            if ts is None:
                continue
            if len(ts) != self.n:
                raise ValueError(f"{name}: {len(ts)} tensors for {self.n} meshes")
            for m, (t, z) in enumerate(zip(ts, sizes)):
                if t is not None and t.numel() != z:
                    raise ValueError(f"{name}[{m}] has {t.numel()} entries; mesh {m} needs {z}")

    def bind(self, nodes, coeff, K, M, stream=None):
        self._check_sizes(nodes, coeff, K, M)
        self._bound = (list(nodes), None if coeff is None else list(coeff), list(K), list(M))  # keep alive
        cp = None if coeff is None else _ptr_array(coeff, torch.float64, "coeff", allow_none=True)
        _check(load().ef_batch_bind(self._h, _ptr_array(nodes, torch.float64, "nodes"), cp,
                                    _ptr_array(K, torch.float64, "K"), _ptr_array(M, torch.float64, "M"),
                                    _stream_ptr(stream)))

    def assemble(self, stream=None):
        """ef_batch_assemble_bound: every mesh into the buffers given to bind()."""
        _check(load().ef_batch_assemble_bound(self._h, _stream_ptr(stream)))

    def tables(self, nodes, coeff, K, M):
        """Per-mesh pointer tables for assemble_tables (sizes checked here); holds the tensors alive."""
        self._check_sizes(nodes, coeff, K, M)
        cp = None if coeff is None else _ptr_array(coeff, torch.float64, "coeff", allow_none=True)
        return (_ptr_array(nodes, torch.float64, "nodes"), cp, _ptr_array(K, torch.float64, "K"),
                _ptr_array(M, torch.float64, "M"), (list(nodes), coeff, list(K), list(M)))

    def assemble_tables(self, tables, stream=None):
        """ef_batch_assemble: every mesh into the buffers of `tables` (from tables()), passed with the call."""
        _check(load().ef_batch_assemble(self._h, tables[0], tables[1], tables[2], tables[3], _stream_ptr(stream)))

    def tune(self, reps: int = 3, stream=None) -> dict:
        cfg = BatchConfig()
        _check(load().ef_batch_tune(self._h, reps, C.byref(cfg), _stream_ptr(stream)))
        return cfg.as_dict()

    def config(self) -> dict:
        cfg = BatchConfig()
        _check(load().ef_batch_get_config(self._h, C.byref(cfg)))
        return cfg.as_dict()

    def set_config(self, stream=None, **kw):
        cfg = BatchConfig(**{**self.config(), **kw})
        _check(load().ef_batch_set_config(self._h, C.byref(cfg), _stream_ptr(stream)))

    def check(self, stream=None):
        _check(load().ef_batch_check(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            load().ef_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
