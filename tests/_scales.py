"""Per-entry error scales for the GPU parity tests, from the oracle.

A global quantity (a load-vector entry, a node gradient, a per-element curl)
is a sum of element contributions, and each contribution is itself a sum
(over quadrature points, local DOFs or terms of a derivative). The rounding
error of either side is bounded by a small multiple of eps times the sum of
the ABSOLUTE values of those terms, not by the entry itself, which may be
small by cancellation. These helpers compute such sums of absolute values
entry by entry, so that a test can assert |gpu - oracle| <= tol * scale_i on
every entry instead of against the largest entry of the vector.

The per-element terms come from the oracle run on the "disjoint" copy of the
mesh: every element gets its own copies of its nodes, numbered so that the
copies keep the relative order of the original global ids. The orientation
signs of Sec. 2.3 and the lexicographic DOF numbering of Sec. 3 depend only
on that order, so in the disjoint mesh element K's DOFs are 6K..6K+5 (3 or 4
in the other kinds) in the order of its global DOF ids, with the same signs
and the same geometry (local node order is unchanged).
"""
from __future__ import annotations

import numpy as np


def disjoint_mesh(nodes: np.ndarray, elems: np.ndarray):
    """(nodes', elems') with element K on nodes' nv*K .. nv*K + nv - 1, the
    copies of its nodes ordered by their original global id."""
    T, nv = elems.shape
    rank = np.argsort(np.argsort(elems, axis=1, kind="stable"), axis=1, kind="stable")
    elems_d = (nv * np.arange(T)[:, None] + rank).astype(np.int32)
    nodes_d = np.empty((T * nv, nodes.shape[1]))
    nodes_d[elems_d.ravel()] = nodes[elems.ravel()]
    return nodes_d, elems_d


def sorted_dofs(elem2dof: np.ndarray) -> np.ndarray:
    """Global DOF of the r-th DOF of element K in the disjoint mesh (its r-th smallest global DOF)."""
    return np.sort(elem2dof, axis=1)


def _abs_scatter(n: int, idx: np.ndarray, vals: np.ndarray) -> np.ndarray:
    out = np.zeros(n)
    np.add.at(out, idx.ravel(), np.abs(vals).ravel())
    return out


def _unit_by_rank(T: int, nl: int, r: int) -> np.ndarray:
    v = np.zeros(T * nl)
    v[r::nl] = 1.0
    return v


def load_vector_scale(ora, kind: int, dim: int, nodes, elems, n: int, F, derivative: bool = False) -> np.ndarray:
    """s_i = sum over elements K containing DOF i of sum_q w_q |det B_K| |F(x_q) . eta_i(x_q)|
    (derivative=True: |g(x_q) . D eta_i| with D = div or curl), F / g given at the
    points of the rule with n points per direction, [nq][T][components]."""
    topo = ora.topology(kind, dim, nodes, elems)
    gdof = sorted_dofs(topo["elem2dof"])
    T, nl = gdof.shape
    nd, ed = disjoint_mesh(nodes, elems)
    _, w = ora.quadrature(dim, 1, n)
    B = np.stack([nodes[elems[:, a]] - nodes[elems[:, 0]] for a in range(1, dim + 1)], axis=2)
    adet = np.abs(np.linalg.det(B))                       # [T]
    F = np.asarray(F).reshape(len(w), T, -1)
    contrib = np.zeros((T, nl))
    for r in range(nl):
        e = _unit_by_rank(T, nl, r)
        if derivative:
            d = ora.fe_curl(kind, dim, nd, ed, e).reshape(1, T, -1)          # constant per element
            term = np.abs((F * d).sum(axis=2))
        else:
            vals = ora.fe_values(kind, dim, nd, ed, n, e).reshape(len(w), T, dim)
            term = np.abs((F * vals).sum(axis=2))
        contrib[:, r] = adet * (w[:, None] * term).sum(axis=0)
    return _abs_scatter(topo["n_dofs"], gdof, contrib)


def fe_curl_scale(ora, kind: int, dim: int, nodes, elems, v) -> np.ndarray:
    """Per element (and component): sum_k |v_k| |D eta_k| over the element's DOFs, D = curl or div."""
    topo = ora.topology(kind, dim, nodes, elems)
    gdof = sorted_dofs(topo["elem2dof"])
    T, nl = gdof.shape
    nd, ed = disjoint_mesh(nodes, elems)
    out = 0.0
    for r in range(nl):
        d = ora.fe_curl(kind, dim, nd, ed, _unit_by_rank(T, nl, r)).reshape(T, -1)
        out = out + np.abs(v[gdof[:, r]])[:, None] * np.abs(d)
    return out.reshape(ora.fe_curl(kind, dim, nodes, elems, v).shape)


def adjoint_node_scale(ora, kind: int, dim: int, nodes, elems, coeff, u, v) -> np.ndarray:
    """Per node and coordinate: sum over elements K of |d J_K / d x_a|, J_K the
    element's share sigma_K (u_K^T K_K u_K + v_K^T M_K v_K)."""
    topo = ora.topology(kind, dim, nodes, elems)
    gdof = sorted_dofs(topo["elem2dof"])
    nd, ed = disjoint_mesh(nodes, elems)
    _, gxd, _ = ora.adjoint(kind, dim, nd, ed, coeff, u[gdof].ravel(), v[gdof].ravel())
    # node copy ed[K, a] is the copy of the original node elems[K, a]
    out = np.zeros_like(nodes)
    np.add.at(out, elems.ravel(), np.abs(gxd[ed.ravel()]))
    return out
