"""Pins of the vectorised integration (Sec. 3.1, norm_L2) (no GPU).

* The library's reference rule (ef_quad_rule, host code) integrates every
  monomial x^a y^b (z^c) of total degree <= 2n - dim exactly: the closed form
  over the reference simplex is a! b! c! / (a + b + c + dim)!.
* The oracle's norm: |Omega| for f = 1; closed-form integrals of polynomial
  fields over the unit square / cube; ||v_h||^2 = v^T M v with the oracle's
  pinned mass matrix (unit coefficient); the interpolant of a constant field
  c reproduces c at every quadrature point, so ||c - v_h||^2 vanishes and
  ||v_h||^2 = |Omega| |c|^2. A wrong Piola map, sign, weight or Jacobian
  fails one of these.
"""
import math

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._bruteforce import to_dense

RT0, NED1 = 1, 2
CASES = [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)]


def _mesh(dim, n, seed):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(n, 0.2, seed)
    else:
        nodes, elems = mg.kuhn_square(n, 0.2, seed)
    return nodes, mg.shuffle_local_order(elems, seed + 100)


def _constant_dofs(kind, dim, nodes, d2n, c):
    Xa, Xb = nodes[d2n[:, 0]], nodes[d2n[:, 1]]
    if kind == NED1:
        return (Xa - Xb) @ c
    if dim == 2:
        t = Xa - Xb
        return np.stack([t[:, 1], -t[:, 0]], 1) @ c
    return np.cross(Xb - Xa, nodes[d2n[:, 2]] - Xa) @ c


@pytest.mark.parametrize("dim", [2, 3])
def test_library_rule_exactness(dim):
    from paper_1409_4618_gb300 import edgefem as ef

    for n in range(1 if dim == 2 else 2, 9):
        x, w = ef.ef_quad_rule(dim, n)
        assert x.shape == (n ** dim, dim) and np.all(w > 0)
        deg = 2 * n - dim
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                for c in (range(deg + 1 - a - b) if dim == 3 else [0]):
                    exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + dim)
                    mono = x[:, 0] ** a * x[:, 1] ** b * (x[:, 2] ** c if dim == 3 else 1.0)
                    assert abs(w @ mono - exact) <= 1e-14 * exact, (n, a, b, c)
        # points inside the reference simplex
        assert np.all(x >= 0) and np.all(x.sum(1) <= 1 + 1e-15)


def test_library_rule_rejects_bad_arguments():
    from paper_1409_4618_gb300 import edgefem as ef

    for dim, n in ((3, 0), (2, 9), (4, 2)):
        with pytest.raises(ef.EdgeFemError):
            ef.ef_quad_rule(dim, n)


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_norm_of_polynomials(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 31)
    n = 4
    x = ora.quad_points(dim, nodes, elems, n)
    one = np.ones(x.shape[:2] + (1,))
    assert abs(ora.norm_l2(kind, dim, nodes, elems, n, one)[0] - 1.0) < 1e-14
    if dim == 3:
        f = (x[..., 0] * x[..., 1] + x[..., 2])[..., None]
        exact = 1.0 / 9 + 1.0 / 4 + 1.0 / 3
    else:
        f = (x[..., 0] * x[..., 1] + 1.0)[..., None]
        exact = 1.0 / 9 + 1.0 / 2 + 1.0
    total, elem = ora.norm_l2(kind, dim, nodes, elems, n, f)
    assert abs(total - exact) < 1e-13 * exact
    assert abs(elem.sum() - total) < 1e-14 * total


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_norm_of_fe_function_is_mass_energy(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 33)
    r = ora.assemble(kind, dim, nodes, elems)
    M = to_dense(r, "M")
    v = mg.normal(33, mg.STREAM_V, r["n_dofs"])
    n = 3
    zero = np.zeros((n ** dim, elems.shape[0], dim))
    total, _ = ora.norm_l2(kind, dim, nodes, elems, n, zero, v)
    assert abs(total - v @ M @ v) < 1e-13 * (v @ M @ v)


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_interpolant_of_constant_is_exact(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 35)
    r = ora.topology(kind, dim, nodes, elems)
    c = np.array([0.7, -1.3, 0.4])[:dim]
    u = _constant_dofs(kind, dim, nodes, r["dof2nodes"], c)
    n = 2
    cf = np.broadcast_to(c, (n ** dim, elems.shape[0], dim)).copy()
    err, _ = ora.norm_l2(kind, dim, nodes, elems, n, cf, u)
    assert err < 1e-26
    zero = np.zeros_like(cf)
    energy, _ = ora.norm_l2(kind, dim, nodes, elems, n, zero, u)
    assert abs(energy - c @ c) < 1e-13


def _linear_dofs(kind, dim, nodes, d2n, A, c):
    """DOFs of the affine field E(x) = A x + c: edge line integrals (Nedelec,
    from the larger to the smaller node id), edge fluxes through R_cw(X_a - X_b)
    (2D RT0), and N_f . E(centroid) with N_f = (X_b - X_a) x (X_c - X_a) (3D
    RT0, the printed basis of flux 1/2), all exact for affine E."""
    E = lambda x: x @ A.T + c
    Xa, Xb = nodes[d2n[:, 0]], nodes[d2n[:, 1]]
    if kind == NED1:
        return np.einsum("ij,ij->i", E(0.5 * (Xa + Xb)), Xa - Xb)
    if dim == 2:
        t = Xa - Xb
        return np.einsum("ij,ij->i", E(0.5 * (Xa + Xb)), np.stack([t[:, 1], -t[:, 0]], 1))
    Xc = nodes[d2n[:, 2]]
    return np.einsum("ij,ij->i", E((Xa + Xb + Xc) / 3.0), np.cross(Xb - Xa, Xc - Xa))


def _affine(dim, seed):
    A = mg.normal(seed, 12, dim * dim).reshape(dim, dim)
    return A, mg.normal(seed, 13, dim)


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_load_vector_pins(ora, kind, dim):
    """b . v = int F . v_h: for F = c and v its interpolant, |Omega| |c|^2;
    for F = v_h(u), b = M u (mass matrix, unit coefficient)."""
    nodes, elems = _mesh(dim, 3, 37)
    r = ora.assemble(kind, dim, nodes, elems)
    n = 3
    c = np.array([0.7, -1.3, 0.4])[:dim]
    cf = np.broadcast_to(c, (n ** dim, elems.shape[0], dim)).copy()
    b = ora.load_vector(kind, dim, nodes, elems, n, cf)
    u_c = _constant_dofs(kind, dim, nodes, r["dof2nodes"], c)
    assert abs(b @ u_c - c @ c) < 1e-13
    u = mg.normal(37, mg.STREAM_U, r["n_dofs"])
    vh = ora.fe_values(kind, dim, nodes, elems, n, u)
    b2 = ora.load_vector(kind, dim, nodes, elems, n, vh)
    Mu = to_dense(r, "M") @ u
    assert np.max(np.abs(b2 - Mu)) < 1e-13 * np.max(np.abs(Mu))


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_curl_of_interpolant_is_exact(ora, kind, dim):
    """The interpolant of an affine field has the field's constant curl (or
    divergence) on every element (commuting diagram)."""
    nodes, elems = _mesh(dim, 3, 39)
    topo = ora.topology(kind, dim, nodes, elems)
    A, c = _affine(dim, 39)
    u = _linear_dofs(kind, dim, nodes, topo["dof2nodes"], A, c)
    got = ora.fe_curl(kind, dim, nodes, elems, u)
    if kind == RT0:
        expect = np.trace(A)
    elif dim == 2:
        expect = A[1, 0] - A[0, 1]
    else:
        expect = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    assert np.max(np.abs(got - expect)) < 1e-12 * (1 + np.abs(A).max())
    # lowest-order elements reproduce constants only: the interpolation error
    # of the affine field at the points is first order, bounded by about h |A|
    vals = ora.fe_values(kind, dim, nodes, elems, 2, u)
    x = ora.quad_points(dim, nodes, elems, 2)
    assert np.abs(vals - (x @ A.T + c)).max() < 2.0 * np.abs(A).sum() / 3


def _bubble_and_gradient(x):
    """b(x) = prod_i x_i (x_i - 1), which vanishes on the boundary of the unit
    square / cube, and its gradient, at points x [..., dim]."""
    a = x * (x - 1.0)
    g = 2.0 * x - 1.0
    dim = x.shape[-1]
    b = np.prod(a, axis=-1)
    grad = np.stack([g[..., i] * np.prod(np.delete(a, i, axis=-1), axis=-1) for i in range(dim)], -1)
    return b, grad


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_derivative_load_vector_by_parts(ora, kind, dim):
    """int g D eta_i for a g vanishing on the boundary equals, by integration
    by parts, a plain load vector of derivatives of g: div (RT0):
    int b div eta = -int grad b . eta; 2D curl: int b curl eta = int (d_y b,
    -d_x b) . eta; 3D curl with G = b c: int G . curl eta = int (grad b x c) .
    eta. The rule is exact for both sides (degree 2 dim + 1 <= 2n - dim)."""
    nodes, elems = _mesh(dim, 3, 41)
    n = 4 if dim == 2 else 5
    x = ora.quad_points(dim, nodes, elems, n)
    b, gb = _bubble_and_gradient(x)
    if kind == RT0:
        lhs = ora.load_derivative(kind, dim, nodes, elems, n, b[..., None])
        rhs = -ora.load_vector(kind, dim, nodes, elems, n, gb)
    elif dim == 2:
        lhs = ora.load_derivative(kind, dim, nodes, elems, n, b[..., None])
        rhs = ora.load_vector(kind, dim, nodes, elems, n, np.stack([gb[..., 1], -gb[..., 0]], -1))
    else:
        c = np.array([0.3, -1.1, 0.8])
        lhs = ora.load_derivative(kind, dim, nodes, elems, n, b[..., None] * c)
        rhs = ora.load_vector(kind, dim, nodes, elems, n, np.cross(gb, c))
    assert np.max(np.abs(lhs)) > 1e-4
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(lhs))


@pytest.mark.parametrize("kind,dim", CASES)
def test_oracle_derivative_load_vector_is_stiffness_energy(ora, kind, dim):
    """With g = D u_h (its per-element curl or divergence) the derivative load
    vector is K u: b_i = int D u_h . D eta_i, K the pinned stiffness matrix
    (unit coefficient)."""
    nodes, elems = _mesh(dim, 3, 43)
    r = ora.assemble(kind, dim, nodes, elems)
    u = mg.normal(43, mg.STREAM_U, r["n_dofs"])
    d = ora.fe_curl(kind, dim, nodes, elems, u).reshape(elems.shape[0], -1)
    n = 2
    g = np.broadcast_to(d, (n ** dim,) + d.shape).copy()
    b = ora.load_derivative(kind, dim, nodes, elems, n, g)
    Ku = to_dense(r, "K") @ u
    assert np.max(np.abs(b - Ku)) < 1e-13 * np.max(np.abs(Ku))
