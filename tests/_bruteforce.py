"""Brute-force global assembly in physical coordinates (numpy, tiny meshes).

Independent of the oracle's reference-element / Piola / sign machinery: the
global basis functions are written directly on each physical element from
barycentric coordinates (np.linalg.inv of the vertex matrix), oriented by the
global rule (edge {a < b} directed from b to a; 2D RT edge normal
R_cw(X_a - X_b); face {a < b < c} normal (X_b - X_a) x (X_c - X_a)), and
integrated with a collapsed Gauss-Legendre product rule built from
numpy.polynomial.legendre.leggauss. The local entities of an element are
enumerated with itertools.combinations, not with the paper's local numbering.

Used only by the tests.
"""
from __future__ import annotations

import itertools

import numpy as np

RT0, NED1 = 1, 2


def numbering(kind: int, dim: int, elems: np.ndarray):
    """Global DOFs = sorted node tuples of edges (or faces for 3D RT0), ranked
    lexicographically. Returns (dof2nodes [N, m], dict tuple -> id)."""
    m = 3 if (kind == RT0 and dim == 3) else 2
    tuples = set()
    for el in elems.tolist():
        for c in itertools.combinations(sorted(el), m):
            tuples.add(c)
    d2n = np.array(sorted(tuples), dtype=np.int64).reshape(-1, m)
    return d2n, {tuple(t): i for i, t in enumerate(d2n.tolist())}


def collapsed_rule(dim: int, n: int):
    t, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    if dim == 2:
        for i in range(n):
            for j in range(n):
                u, v = t[i], t[j]
                pts.append((u, v * (1 - u)))
                wts.append(w[i] * w[j] * (1 - u))
    else:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    u, v, s = t[i], t[j], t[k]
                    pts.append((u, v * (1 - u), s * (1 - u) * (1 - v)))
                    wts.append(w[i] * w[j] * w[k] * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def _cross(a, b):
    return np.cross(a, b)


def brute_force(kind: int, dim: int, nodes: np.ndarray, elems: np.ndarray, coeff=None, nq: int = 4):
    """Dense global K and M (N x N) and dof2nodes."""
    d2n, ids = numbering(kind, dim, elems)
    N = d2n.shape[0]
    K = np.zeros((N, N))
    M = np.zeros((N, N))
    xh, wh = collapsed_rule(dim, nq)
    m = d2n.shape[1]
    for e, el in enumerate(elems.tolist()):
        X = nodes[el]                                    # (d+1, d)
        A = np.vstack([np.ones(dim + 1), X.T])           # (d+1, d+1)
        Ainv = np.linalg.inv(A)                          # row i: lambda_i = Ainv[i,0] + Ainv[i,1:] . x
        grad = Ainv[:, 1:]
        B = (X[1:] - X[0]).T
        vol = abs(np.linalg.det(B)) / (2.0 if dim == 2 else 6.0)
        xq = X[0] + xh @ B.T                             # physical points
        wq = wh * abs(np.linalg.det(B))
        lam = Ainv[:, 0][None, :] + xq @ grad.T          # (nq, d+1)
        sig = 1.0 if coeff is None else float(coeff[e])
        funcs = []                                       # (dof, values (nq,d), div/curl (nq,) or (nq,3))
        for loc in itertools.combinations(range(dim + 1), m):
            g = tuple(sorted(el[i] for i in loc))
            dof = ids[g]
            pos = [el.index(gi) for gi in g]             # local vertex of each sorted global node
            if kind == NED1:
                pa, pb = pos                             # global a < b; direction b -> a
                val = lam[:, [pb]] * grad[pa][None, :] - lam[:, [pa]] * grad[pb][None, :]
                if dim == 3:
                    c = 2.0 * _cross(grad[pb], grad[pa])
                    dv = np.tile(c, (len(wq), 1))
                else:
                    c = 2.0 * (grad[pb][0] * grad[pa][1] - grad[pb][1] * grad[pa][0])
                    dv = np.full((len(wq), 1), c)
            else:
                opp = [i for i in range(dim + 1) if i not in loc][0]
                Xa = X[pos[0]]
                if dim == 2:
                    t = X[pos[0]] - X[pos[1]]
                    Nrm = np.array([t[1], -t[0]])
                else:
                    Nrm = _cross(X[pos[1]] - X[pos[0]], X[pos[2]] - X[pos[0]])
                out = 1.0 if Nrm @ (Xa - X[opp]) > 0 else -1.0
                # flux 1 through an edge (2D); flux 1/2 through a face (3D, Sec. 2.1 basis as printed)
                scale = out / (2.0 * vol) if dim == 2 else out / (6.0 * vol)
                val = scale * (xq - X[opp])
                dv = np.full((len(wq), 1), scale * dim)
            funcs.append((dof, val, dv))
        for (i, vi, di) in funcs:
            for (j, vj, dj) in funcs:
                M[i, j] += sig * np.sum(wq * np.sum(vi * vj, axis=1))
                K[i, j] += sig * np.sum(wq * np.sum(di * dj, axis=1))
    return K, M, d2n


def to_dense(res: dict, key: str) -> np.ndarray:
    N = res["n_dofs"]
    A = np.zeros((N, N))
    rp, ci = res["rowptr"], res["colidx"]
    for i in range(N):
        A[i, ci[rp[i]:rp[i + 1]]] = res[key][rp[i]:rp[i + 1]]
    return A
