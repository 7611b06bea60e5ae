"""Majorant minimisation (Sec. 4.1, Algorithm 1) for the Poisson problem with
the bubble solution u = prod_i x_i (x_i - 1) on the unit square: test helper.

The approximation v is the P1 Galerkin solution (test-side numpy and scipy:
nodal elements are not part of the library). Step (a) of the algorithm
solves, for fixed beta, the Raviart-Thomas discretisation of the quadratic
minimisation problem

    (1 + beta) C^2 int div y div phi + (1 + 1/beta) int y . phi
        = -(1 + beta) C^2 int f div phi + (1 + 1/beta) int grad v . phi,

with C = 1 / (pi sqrt(d)) the Friedrichs constant of the unit square / cube;
step (b) sets beta = ||grad v - y|| / (C ||div y + f||), Eq. (betaoptimal).
The majorant of Eq. (majorantestimate) squared by Young's inequality is

    M = (1 + 1/beta) ||grad v - y||^2 + (1 + beta) C^2 ||div y + f||^2,

and I_eff = sqrt(M) / ||grad (u - v)||. The RT0 matrices, the two load
vectors and the three norms (one of them of div y + f) come from a backend:
the oracle or the GPU library. The linear systems are solved by scipy (neither has a solver).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

RT0 = 1


def bubble_gradient(x):
    """grad u at points x [..., dim]."""
    a = x * (x - 1.0)
    g = 2.0 * x - 1.0
    dim = x.shape[-1]
    return np.stack([g[..., i] * np.prod(np.delete(a, i, axis=-1), axis=-1) for i in range(dim)], -1)


def source(x):
    """f = -Laplace u = -2 sum_i prod_{j != i} x_j (x_j - 1)."""
    a = x * (x - 1.0)
    dim = x.shape[-1]
    return -2.0 * sum(np.prod(np.delete(a, i, axis=-1), axis=-1) for i in range(dim))


def p1_solution(nodes, elems, xhat, w):
    """P1 Galerkin solution v of -Laplace u = f, u = 0 on the boundary of the
    unit square / cube, with the load integrated by the reference rule (xhat
    [nq, dim], w [nq]); returns grad v per element [T, dim]."""
    d = nodes.shape[1]
    V = nodes.shape[0]
    P = nodes[elems]
    B = np.transpose(P[:, 1:, :] - P[:, :1, :], (0, 2, 1))          # columns: edge vectors
    det = np.linalg.det(B)
    G = np.linalg.inv(B)                                           # rows: grad lambda_1..d
    G = np.concatenate([-G.sum(1, keepdims=True), G], 1)           # grad lambda_0..d
    vol = np.abs(det) / math.factorial(d)
    Kl = vol[:, None, None] * np.einsum("tid,tjd->tij", G, G)
    rows = np.repeat(elems, d + 1, axis=1).ravel()
    cols = np.tile(elems, (1, d + 1)).ravel()
    A = sps.csr_matrix((Kl.ravel(), (rows, cols)), shape=(V, V))
    lam = np.concatenate([1.0 - xhat.sum(1, keepdims=True), xhat], 1)
    x = P[:, 0, None, :] + np.einsum("tcd,qd->tqc", B, xhat)
    bl = np.abs(det)[:, None] * np.einsum("q,tq,qi->ti", w, source(x), lam)
    b = np.zeros(V)
    np.add.at(b, elems.ravel(), bl.ravel())
    free = ~np.any((nodes < 1e-12) | (nodes > 1.0 - 1e-12), axis=1)
    v = np.zeros(V)
    v[free] = spla.spsolve(A[free][:, free].tocsc(), b[free])
    return np.einsum("ti,tid->td", v[elems], G)


def minimise(backend, nodes, elems, iters, n=4, record=None):
    """Algorithm 1 from beta = 1 for `iters` iterations: [(beta, sqrt(M),
    I_eff)] of each iteration (beta the value used in that iteration). With a
    dict `record`, also keeps the backend's quantities (K, M, the two load
    vectors, the norms and each iteration's y) for comparison."""
    d = nodes.shape[1]
    T = elems.shape[0]
    xhat, w = backend.ref_rule(n)
    gradv = p1_solution(nodes, elems, xhat, w)
    C = 1.0 / (math.pi * math.sqrt(d))
    K, M = backend.rt0_matrices()
    x = backend.quad_points(n)                                     # [nq, T, d]
    nq = x.shape[0]
    gv = np.ascontiguousarray(np.broadcast_to(gradv[None], (nq, T, d)))
    fx = source(x)                                                 # [nq, T]
    b_grad = backend.load_vector(gv, n)                            # int grad v . phi_i
    b_div = backend.load_derivative(np.ascontiguousarray(fx[..., None]), n)   # int f div phi_i
    err_v = backend.norm_l2(np.ascontiguousarray(bubble_gradient(x) - gv), n)  # ||grad (u - v)||^2
    if record is not None:
        record.update(K=K, M=M, x=x, gv=gv, fx=fx, b_grad=b_grad, b_div=b_div, err_v=err_v, ys=[], t1=[], t2=[])
    beta = 1.0
    out = []
    for _ in range(iters):
        A = (1.0 + beta) * C * C * K + (1.0 + 1.0 / beta) * M
        rhs = -(1.0 + beta) * C * C * b_div + (1.0 + 1.0 / beta) * b_grad
        y = spla.spsolve(A.tocsc(), rhs)
        t1 = backend.norm_l2(gv, n, y)                             # ||grad v - y||^2
        t2 = backend.norm_derivative(np.ascontiguousarray(-fx[..., None]), n, y)   # ||div y + f||^2
        if record is not None:
            record["ys"].append(y)
            record["t1"].append(t1)
            record["t2"].append(t2)
        Mv = (1.0 + 1.0 / beta) * t1 + (1.0 + beta) * C * C * t2
        out.append((beta, math.sqrt(Mv), math.sqrt(Mv / err_v)))
        beta = math.sqrt(t1) / (C * math.sqrt(t2))
    return out


class OracleBackend:
    """RT0 matrices, integrals and divergence from the CPU oracle."""

    def __init__(self, ora, nodes, elems):
        self.ora, self.nodes, self.elems = ora, nodes, elems
        self.dim = nodes.shape[1]

    def ref_rule(self, n):
        return self.ora.quadrature(self.dim, 1, n)

    def rt0_matrices(self):
        r = self.ora.assemble(RT0, self.dim, self.nodes, self.elems)
        N = r["n_dofs"]
        K = sps.csr_matrix((r["K"], r["colidx"], r["rowptr"]), shape=(N, N))
        M = sps.csr_matrix((r["M"], r["colidx"], r["rowptr"]), shape=(N, N))
        return K, M

    def quad_points(self, n):
        return self.ora.quad_points(self.dim, self.nodes, self.elems, n)

    def load_vector(self, F, n):
        return self.ora.load_vector(RT0, self.dim, self.nodes, self.elems, n, F)

    def load_derivative(self, g, n):
        return self.ora.load_derivative(RT0, self.dim, self.nodes, self.elems, n, g)

    def norm_l2(self, f, n, v=None):
        return self.ora.norm_l2(RT0, self.dim, self.nodes, self.elems, n, f, v)[0]

    def norm_derivative(self, g, n, v):
        """||g - div v_h||^2: the oracle's per-element divergence and norm."""
        d = self.ora.fe_curl(RT0, self.dim, self.nodes, self.elems, v)
        return self.norm_l2(np.ascontiguousarray(g - d[None, :, None]), n)


class GpuBackend:
    """The same from the CUDA library (C ABI through the binding)."""

    def __init__(self, nodes, elems):
        import torch

        from paper_1409_4618_gb300 import edgefem as ef

        self.torch, self.ef = torch, ef
        self.dev = torch.device("cuda")
        self.dim = nodes.shape[1]
        self.tn = torch.from_numpy(nodes).to(self.dev)
        self.plan = ef.Plan(RT0, self.dim, nodes.shape[0], torch.from_numpy(elems).to(self.dev))

    def _t(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)

    def ref_rule(self, n):
        return self.ef.ef_quad_rule(self.dim, n)

    def rt0_matrices(self):
        K, M = self.plan.assemble(self.tn)
        self.plan.check()
        rowptr, colidx = self.plan.pattern()
        N = self.plan.n_dofs
        rp, ci = rowptr.cpu().numpy(), colidx.cpu().numpy()
        return (sps.csr_matrix((K.cpu().numpy(), ci, rp), shape=(N, N)),
                sps.csr_matrix((M.cpu().numpy(), ci, rp), shape=(N, N)))

    def quad_points(self, n):
        return self.plan.quad_points(self.tn, n).cpu().numpy()

    def load_vector(self, F, n):
        return self.plan.load_vector(self.tn, self._t(F), n).cpu().numpy()

    def load_derivative(self, g, n):
        return self.plan.load_derivative(self.tn, self._t(g), n).cpu().numpy()

    def norm_l2(self, f, n, v=None):
        total, _ = self.plan.norm_l2(self.tn, self._t(f), n, None if v is None else self._t(v))
        return float(total[0])

    def norm_derivative(self, g, n, v):
        total, _ = self.plan.norm_l2_derivative(self.tn, self._t(g), n, self._t(v))
        return float(total[0])

    def close(self):
        self.plan.check()
        self.plan.close()
