"""CPU FP64 oracle for edge-element assembly (RT0 / Nedelec), ctypes binding.

TEST INFRASTRUCTURE ONLY. The oracle is the reference the CUDA library is
checked against: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. The product package never
does, and the oracle never imports the product package.

The C source (``edgefem_oracle.c``) states, function by function, which
definition of the paper it follows. Functions:

* ``assemble(kind, dim, nodes, elems, coeff)`` -> dict with topology
  (``elem2dof``, ``sign``, ``dof2nodes``), CSR pattern (``rowptr``,
  ``colidx``) and values (``K``, ``M`` and the sums of absolute local
  contributions ``Kabs``, ``Mabs``).
* ``topology(kind, dim, nodes, elems)``: the first three only.
* ``local(kind, dim, P, sign, coeff)``: one element's K and M.
* ``adjoint(kind, dim, nodes, elems, coeff, u, v)`` -> (J, dJ/dx, dJ/dsigma).
* ``quadrature(dim, rule, n)`` and ``ref_basis(kind, dim, x)``.
* Integration (Sec. 3.1): ``quad_points``, ``norm_l2``, ``fe_values``,
  ``fe_curl`` (per-element curl or divergence), ``load_vector``
  (int F . eta_i) and ``load_derivative`` (int g . D eta_i, D = div or curl).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

RT0 = 1
NED1 = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SOURCES = ("edgefem_oracle.c", "local_body.inc")

_STATUS = {
    0: "ok",
    -1: "invalid argument",
    -2: "node id out of range",
    -3: "degenerate element (det B_K = 0)",
    -5: "out of memory",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}: {_STATUS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, -O2, no target-specific flags)."""
    src = os.path.join(_HERE, "edgefem_oracle.c")
    newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= newest:
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Result(C.Structure):
    _fields_ = [
        ("n_elems", C.c_int64),
        ("n_dofs", C.c_int64),
        ("nnz", C.c_int64),
        ("nloc", C.c_int32),
        ("ent_nodes", C.c_int32),
        ("elem2dof", C.POINTER(C.c_int32)),
        ("sign", C.POINTER(C.c_int8)),
        ("dof2nodes", C.POINTER(C.c_int32)),
        ("rowptr", C.POINTER(C.c_int64)),
        ("colidx", C.POINTER(C.c_int32)),
        ("K", C.POINTER(C.c_double)),
        ("M", C.POINTER(C.c_double)),
        ("Kabs", C.POINTER(C.c_double)),
        ("Mabs", C.POINTER(C.c_double)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.ora_free.argtypes = [C.POINTER(_Result)]
        lib.ora_nloc.argtypes = [C.c_int, C.c_int]
        lib.ora_quadrature.argtypes = [C.c_int, C.c_int, C.c_int, P, P, C.c_int]
        lib.ora_ref_basis.argtypes = [C.c_int, C.c_int, P, P, P]
        lib.ora_local.argtypes = [C.c_int, C.c_int, P, P, C.c_double, C.c_int, C.c_int, P, P]
        lib.ora_topology.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, C.POINTER(_Result)]
        lib.ora_assemble.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, P, C.c_int, C.c_int,
                                     C.POINTER(_Result)]
        lib.ora_assemble2.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, P, P, C.c_int, C.c_int,
                                      C.POINTER(_Result)]
        lib.ora_quad_points.argtypes = [C.c_int, C.c_int64, P, C.c_int64, P, C.c_int, P]
        lib.ora_norm_l2.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, C.c_int, C.c_int, P, P, P, P]
        lib.ora_load_vector.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, C.c_int, P, P]
        lib.ora_load_derivative.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, C.c_int, P, P]
        lib.ora_fe_values.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, C.c_int, P, P]
        lib.ora_fe_curl.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, P, P]
        lib.ora_adjoint.argtypes = [C.c_int, C.c_int, C.c_int64, P, C.c_int64, P, P, P, P, C.c_int, C.c_int,
                                    P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _prep(nodes, elems, coeff=None):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    if coeff is not None:
        coeff = np.ascontiguousarray(coeff, dtype=np.float64)
        if coeff.shape != (elems.shape[0],):
            raise ValueError("coeff must have one value per element")
    return nodes, elems, coeff


def _copy(ptr, n, dtype, shape=None):
    if n == 0:
        out = np.zeros(0, dtype=dtype)
    else:
        out = np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)
    return out if shape is None else out.reshape(shape)


def _unpack(res: _Result, with_values: bool) -> dict:
    T, N, nl, ne = res.n_elems, res.n_dofs, res.nloc, res.ent_nodes
    out = {
        "n_dofs": int(N),
        "elem2dof": _copy(res.elem2dof, T * nl, np.int32, (T, nl)),
        "sign": _copy(res.sign, T * nl, np.int8, (T, nl)),
        "dof2nodes": _copy(res.dof2nodes, N * ne, np.int32, (N, ne)),
    }
    if with_values:
        nnz = res.nnz
        out.update(
            nnz=int(nnz),
            rowptr=_copy(res.rowptr, N + 1, np.int64),
            colidx=_copy(res.colidx, nnz, np.int32),
            K=_copy(res.K, nnz, np.float64),
            M=_copy(res.M, nnz, np.float64),
            Kabs=_copy(res.Kabs, nnz, np.float64),
            Mabs=_copy(res.Mabs, nnz, np.float64),
        )
    return out


def topology(kind: int, dim: int, nodes, elems) -> dict:
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems)
    res = _Result()
    st = lib.ora_topology(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), C.byref(res))
    if st:
        raise OracleError(st)
    try:
        return _unpack(res, False)
    finally:
        lib.ora_free(C.byref(res))


def assemble(kind: int, dim: int, nodes, elems, coeff=None, rule: int = 0, n: int = 0) -> dict:
    lib = _load()
    nodes, elems, coeff = _prep(nodes, elems, coeff)
    res = _Result()
    st = lib.ora_assemble(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), _ptr(coeff),
                          rule, n, C.byref(res))
    if st:
        raise OracleError(st)
    try:
        return _unpack(res, True)
    finally:
        lib.ora_free(C.byref(res))


def assemble2(kind: int, dim: int, nodes, elems, coeff_K=None, coeff_M=None, rule: int = 0, n: int = 0) -> dict:
    """Assembly with K scaled by coeff_K and M by coeff_M (None: unit)."""
    lib = _load()
    nodes, elems, coeff_K = _prep(nodes, elems, coeff_K)
    coeff_M = None if coeff_M is None else np.ascontiguousarray(coeff_M, dtype=np.float64)
    res = _Result()
    st = lib.ora_assemble2(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), _ptr(coeff_K),
                           _ptr(coeff_M), rule, n, C.byref(res))
    if st:
        raise OracleError(st)
    try:
        return _unpack(res, True)
    finally:
        lib.ora_free(C.byref(res))


def quad_points(dim: int, nodes, elems, n: int):
    """Physical points [nq, T, dim] of the collapsed Gauss-Legendre rule (n per direction)."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    T = elems.shape[0]
    nq = n ** dim
    x = np.zeros((nq, T, dim))
    m = lib.ora_quad_points(dim, nodes.shape[0], _ptr(nodes), T, _ptr(elems), n, _ptr(x))
    if m < 0:
        raise OracleError(m)
    return x


def norm_l2(kind: int, dim: int, nodes, elems, n: int, f, v=None):
    """(total, per-element) squared L2 norm of f - v_h, f: [nq, T, ncomp] at quad_points."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    f = np.ascontiguousarray(f, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    elem = np.zeros(elems.shape[0])
    total = np.zeros(1)
    st = lib.ora_norm_l2(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), n, f.shape[2],
                         _ptr(f), _ptr(v), _ptr(elem), _ptr(total))
    if st:
        raise OracleError(st)
    return float(total[0]), elem


def load_vector(kind: int, dim: int, nodes, elems, n: int, F):
    """b_i = int F . eta_i, F: [nq, T, dim] at quad_points (n per direction)."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    F = np.ascontiguousarray(F, dtype=np.float64)
    N = topology(kind, dim, nodes, elems)["n_dofs"]
    b = np.zeros(N)
    st = lib.ora_load_vector(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), n, _ptr(F), _ptr(b))
    if st:
        raise OracleError(st)
    return b


def load_derivative(kind: int, dim: int, nodes, elems, n: int, g):
    """b_i = int g . D eta_i (D = div for RT0, curl for Nedelec), g: [nq, T, ncomp] at quad_points (ncomp 3 for
    3D Nedelec, else 1; a [nq, T] array is taken as ncomp 1)."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    g = np.ascontiguousarray(g, dtype=np.float64)
    N = topology(kind, dim, nodes, elems)["n_dofs"]
    b = np.zeros(N)
    st = lib.ora_load_derivative(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), n, _ptr(g),
                                 _ptr(b))
    if st:
        raise OracleError(st)
    return b


def fe_values(kind: int, dim: int, nodes, elems, n: int, v):
    """Values [nq, T, dim] of v_h at quad_points."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros((n ** dim, elems.shape[0], dim))
    st = lib.ora_fe_values(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), n, _ptr(v), _ptr(out))
    if st:
        raise OracleError(st)
    return out


def fe_curl(kind: int, dim: int, nodes, elems, v):
    """Per-element curl (Nedelec) or divergence (RT0) of v_h: [T] or [T, 3] (3D Nedelec)."""
    lib = _load()
    nodes, elems, _ = _prep(nodes, elems, None)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros((elems.shape[0], 3) if (kind == NED1 and dim == 3) else elems.shape[0])
    st = lib.ora_fe_curl(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), _ptr(v), _ptr(out))
    if st:
        raise OracleError(st)
    return out


def local(kind: int, dim: int, P, sign, coeff: float = 1.0, rule: int = 0, n: int = 0):
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    nl = lib.ora_nloc(kind, dim)
    if nl < 0:
        raise OracleError(nl)
    sign = np.ascontiguousarray(sign, dtype=np.float64)
    K = np.zeros((nl, nl))
    M = np.zeros((nl, nl))
    st = lib.ora_local(kind, dim, _ptr(P), _ptr(sign), float(coeff), rule, n, _ptr(K), _ptr(M))
    if st:
        raise OracleError(st)
    return K, M


def adjoint(kind: int, dim: int, nodes, elems, coeff, u, v, rule: int = 0, n: int = 0):
    lib = _load()
    nodes, elems, coeff = _prep(nodes, elems, coeff)
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    J = np.zeros(1)
    gx = np.zeros_like(nodes)
    gs = np.zeros(elems.shape[0])
    st = lib.ora_adjoint(kind, dim, nodes.shape[0], _ptr(nodes), elems.shape[0], _ptr(elems), _ptr(coeff),
                         _ptr(u), _ptr(v), rule, n, _ptr(J), _ptr(gx), _ptr(gs))
    if st:
        raise OracleError(st)
    return float(J[0]), gx, gs


def quadrature(dim: int, rule: int = 0, n: int = 0):
    lib = _load()
    cap = 4096
    x = np.zeros((cap, 3))
    w = np.zeros(cap)
    m = lib.ora_quadrature(dim, rule, n, _ptr(x), _ptr(w), cap)
    if m < 0:
        raise OracleError(m)
    return x[:m, :dim].copy(), w[:m].copy()


def ref_basis(kind: int, dim: int, xh):
    lib = _load()
    xh = np.ascontiguousarray(np.resize(np.asarray(xh, dtype=np.float64), 3))
    nl = lib.ora_nloc(kind, dim)
    nd = 3 if (kind == NED1 and dim == 3) else 1
    val = np.zeros((nl, dim))
    dval = np.zeros((nl, nd))
    st = lib.ora_ref_basis(kind, dim, _ptr(xh), _ptr(val), _ptr(dval))
    if st < 0:
        raise OracleError(st)
    return val, dval


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
