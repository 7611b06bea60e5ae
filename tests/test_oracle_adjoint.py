"""Pins of the oracle's adjoint (no GPU).

J(x, sigma) = u^T K(x, sigma) u + v^T M(x, sigma) v, with K, M the global
matrices. The oracle differentiates the local quadrature in forward mode.
Checked against:
* central finite differences of J computed from the oracle's assembled
  matrices (relative 1e-6), on the 4^3-cube sub-mesh with seed 55;
* exact identities: J is linear in sigma (sum sigma dJ/dsigma = J); J is
  invariant under translation (sum of node gradients = 0) and rotation (zero
  net torque); J_K and J_M are homogeneous in the coordinates, so
  sum x . dJ/dx = p_K J_K + p_M J_M with (p_K, p_M) = (-1, 1) for 3D
  Nedelec, (-2, 0) for 2D Nedelec and 2D RT, (-3, -1) for 3D RT.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg

RT0, NED1 = 1, 2
DEGREES = {(NED1, 3): (-1, 1), (NED1, 2): (-2, 0), (RT0, 2): (-2, 0), (RT0, 3): (-3, -1)}


def _energy(ora, kind, dim, nodes, elems, coeff, u, v):
    r = ora.assemble(kind, dim, nodes, elems, coeff)
    rows = np.repeat(np.arange(r["n_dofs"]), np.diff(r["rowptr"]))
    cols = r["colidx"]
    JK = float(np.sum(u[rows] * r["K"] * u[cols]))
    JM = float(np.sum(v[rows] * r["M"] * v[cols]))
    return JK, JM


def _setup(ora, kind, dim, n, seed):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(n, 0.2, seed)
    else:
        nodes, elems = mg.kuhn_square(n, 0.2, seed)
    coeff = mg.log_uniform_coeff(seed, elems.shape[0])
    N = ora.topology(kind, dim, nodes, elems)["n_dofs"]
    u = mg.normal(seed, mg.STREAM_U, N)
    v = mg.normal(seed, mg.STREAM_V, N)
    return nodes, elems, coeff, u, v


@pytest.mark.parametrize("kind,dim,n", [(NED1, 3, 4), (RT0, 3, 3), (NED1, 2, 5), (RT0, 2, 5)])
def test_adjoint_vs_central_differences(ora, kind, dim, n):
    nodes, elems, coeff, u, v = _setup(ora, kind, dim, n, 55)
    J, gx, gs = ora.adjoint(kind, dim, nodes, elems, coeff, u, v)
    JK, JM = _energy(ora, kind, dim, nodes, elems, coeff, u, v)
    assert abs(J - (JK + JM)) < 1e-12 * (abs(JK) + abs(JM))
    rng = np.random.default_rng(0)
    h = 1e-6 / n
    for _ in range(12):
        a, c = rng.integers(nodes.shape[0]), rng.integers(dim)
        xp, xm = nodes.copy(), nodes.copy()
        xp[a, c] += h
        xm[a, c] -= h
        fd = (sum(_energy(ora, kind, dim, xp, elems, coeff, u, v)) -
              sum(_energy(ora, kind, dim, xm, elems, coeff, u, v))) / (2 * h)
        assert abs(fd - gx[a, c]) <= 1e-6 * max(abs(gx[a, c]), 1e-3 * np.abs(gx).max()), (a, c, fd, gx[a, c])
    for _ in range(6):
        e = rng.integers(elems.shape[0])
        cp, cm = coeff.copy(), coeff.copy()
        hs = 1e-6 * coeff[e]
        cp[e] += hs
        cm[e] -= hs
        fd = (sum(_energy(ora, kind, dim, nodes, elems, cp, u, v)) -
              sum(_energy(ora, kind, dim, nodes, elems, cm, u, v))) / (2 * hs)
        assert abs(fd - gs[e]) <= 1e-6 * max(abs(gs[e]), 1e-3 * np.abs(gs).max())


@pytest.mark.parametrize("kind,dim", list(DEGREES))
def test_adjoint_identities(ora, kind, dim):
    nodes, elems, coeff, u, v = _setup(ora, kind, dim, 3, 8)
    J, gx, gs = ora.adjoint(kind, dim, nodes, elems, coeff, u, v)
    JK, JM = _energy(ora, kind, dim, nodes, elems, coeff, u, v)
    scale = np.abs(gx).max() * np.abs(nodes).max()
    assert abs(np.sum(coeff * gs) - J) < 1e-12 * abs(J)
    assert np.abs(gx.sum(axis=0)).max() < 1e-11 * np.abs(gx).max() * nodes.shape[0] ** 0.5
    if dim == 3:
        torque = np.cross(nodes, gx).sum(axis=0)
    else:
        torque = np.array([np.sum(nodes[:, 0] * gx[:, 1] - nodes[:, 1] * gx[:, 0])])
    assert np.abs(torque).max() < 1e-11 * scale * nodes.shape[0] ** 0.5
    pK, pM = DEGREES[(kind, dim)]
    euler = float(np.sum(nodes * gx))
    assert abs(euler - (pK * JK + pM * JM)) < 1e-11 * (abs(JK) + abs(JM))
