"""Pins of the oracle's reference element, basis and quadrature (no GPU).

* The oracle's reference basis satisfies the defining DOF property of
  Eqs. RTdofs / NEDdofs (Sec. 2.1-2.2): the functional of DOF i applied to
  basis j is delta_ij, with the outer unit normals and the tangent directions
  of Fig. 1. For the 3D RT basis as printed in Sec. 2.1 every face flux is
  1/2 (not 1): that reading is pinned here too.
* Divergence / curl returned by the oracle equal central differences of its
  basis values (the fields are affine, so differences are exact to rounding).
* Quadrature rules integrate monomials exactly up to their degree
  (x^a y^b z^c over the unit simplex = a! b! c! / (a+b+c+d)!).
* Local matrices on the reference element (B = I, all signs +1) equal the
  exact rational integrals of the paper's basis, computed here with
  Fractions by monomial integration (a different method from quadrature).
"""
import itertools
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

RT0, NED1 = 1, 2


def _gl(n):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1), 0.5 * w


# reference edges / faces: (points spanning it, unit normal or tangent, measure), from Fig. 1
S2 = math.sqrt(2.0)
EDGES2 = [  # (start, end) in the tangent direction; outer normal
    ((1, 0), (0, 1), (1 / S2, 1 / S2)),
    ((0, 1), (0, 0), (-1.0, 0.0)),
    ((0, 0), (1, 0), (0.0, -1.0)),
]
EDGES3 = [((0, 0, 0), (1, 0, 0)), ((0, 0, 0), (0, 1, 0)), ((0, 0, 0), (0, 0, 1)),
          ((1, 0, 0), (0, 1, 0)), ((0, 1, 0), (0, 0, 1)), ((0, 0, 1), (1, 0, 0))]
S3 = math.sqrt(3.0)
FACES3 = [  # three vertices, outer unit normal
    ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, -1.0)),
    ((0, 0, 0), (1, 0, 0), (0, 0, 1), (0, -1.0, 0)),
    ((0, 0, 0), (0, 1, 0), (0, 0, 1), (-1.0, 0, 0)),
    ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1 / S3, 1 / S3, 1 / S3)),
]


def _edge_integral(ora, kind, dim, a, b, direction):
    t, w = _gl(4)
    a, b = np.array(a, float), np.array(b, float)
    L = np.linalg.norm(b - a)
    acc = 0.0
    for ti, wi in zip(t, w):
        val, _ = ora.ref_basis(kind, dim, a + ti * (b - a))
        acc = acc + wi * L * (val @ np.array(direction))
    return acc


@pytest.mark.parametrize("kind", [RT0, NED1])
def test_dof_functionals_2d(ora, kind):
    D = np.zeros((3, 3))
    for i, (a, b, nrm) in enumerate(EDGES2):
        tangent = (np.array(b, float) - np.array(a, float))
        tangent /= np.linalg.norm(tangent)
        direction = nrm if kind == RT0 else tangent
        D[i] = _edge_integral(ora, kind, 2, a, b, direction)
    np.testing.assert_allclose(D, np.eye(3), atol=1e-14)


def test_dof_functionals_ned3d(ora):
    D = np.zeros((6, 6))
    for i, (a, b) in enumerate(EDGES3):
        tangent = np.array(b, float) - np.array(a, float)
        D[i] = _edge_integral(ora, NED1, 3, a, b, tangent / np.linalg.norm(tangent))
    np.testing.assert_allclose(D, np.eye(6), atol=1e-14)


def test_dof_functionals_rt3d_printed_basis_has_half_flux(ora):
    """The 3D RT basis printed in Sec. 2.1 has flux 1/2 through its own face
    and 0 through the others (the text claims delta_ij; the printed
    functions, which define the paper's matrices, give delta_ij / 2)."""
    x2, w2 = ora.quadrature(2, 1, 4)        # collapsed rule on the unit triangle
    D = np.zeros((4, 4))
    for i, (p0, p1, p2, nrm) in enumerate(FACES3):
        p0, p1, p2 = (np.array(p, float) for p in (p0, p1, p2))
        area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0))
        for (s, t), w in zip(x2, w2):
            val, _ = ora.ref_basis(RT0, 3, p0 + s * (p1 - p0) + t * (p2 - p0))
            D[i] += 2.0 * area * w * (val @ np.array(nrm))
    np.testing.assert_allclose(D, 0.5 * np.eye(4), atol=1e-14)


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (RT0, 3), (NED1, 2), (NED1, 3)])
def test_div_curl_match_differences(ora, kind, dim):
    rng = np.random.default_rng(1)
    x = rng.random(dim) * 0.3
    h = 1e-3
    _, dval = ora.ref_basis(kind, dim, x)
    J = np.zeros((dval.shape[0], dim, dim))       # J[k, r, c] = d val_r / d x_c
    for c in range(dim):
        e = np.zeros(dim)
        e[c] = h
        vp, _ = ora.ref_basis(kind, dim, x + e)
        vm, _ = ora.ref_basis(kind, dim, x - e)
        J[:, :, c] = (vp - vm) / (2 * h)
    if kind == RT0:
        expect = np.trace(J, axis1=1, axis2=2)[:, None]
    elif dim == 2:
        expect = (J[:, 1, 0] - J[:, 0, 1])[:, None]
    else:
        expect = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=1)
    np.testing.assert_allclose(dval, expect, atol=1e-9)


def _simplex_monomial(exps):
    d = len(exps)
    return math.prod(math.factorial(a) for a in exps) / math.factorial(sum(exps) + d)


@pytest.mark.parametrize("dim", [2, 3])
def test_degree2_rule_exact(ora, dim):
    x, w = ora.quadrature(dim, 0)
    assert abs(w.sum() - (0.5 if dim == 2 else 1 / 6)) < 1e-16
    for exps in itertools.product(range(3), repeat=dim):
        if sum(exps) > 2:
            continue
        got = np.sum(w * np.prod(x ** np.array(exps), axis=1))
        assert abs(got - _simplex_monomial(exps)) < 1e-16, exps
    # and it is not exact for every cubic (guards against a rule that is silently wrong in the other direction)
    errs = [abs(np.sum(w * np.prod(x ** np.array(e), axis=1)) - _simplex_monomial(e))
            for e in itertools.product(range(4), repeat=dim) if sum(e) == 3]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("dim,n", [(2, 3), (2, 6), (3, 3), (3, 5)])
def test_collapsed_rule_exact(ora, dim, n):
    x, w = ora.quadrature(dim, 1, n)
    top = 2 * n - 1 - (dim - 1)
    for exps in itertools.product(range(top + 1), repeat=dim):
        if sum(exps) > top:
            continue
        got = np.sum(w * np.prod(x ** np.array(exps), axis=1))
        assert abs(got - _simplex_monomial(exps)) < 1e-15, exps


# ---- exact rational local matrices on the reference element -------------
# Basis functions of Sec. 2.1-2.2 as polynomials: component -> {exponents: coefficient}
def _p(**terms):
    out = {}
    for k, v in terms.items():
        e = {"c": (0, 0, 0), "x1": (1, 0, 0), "x2": (0, 1, 0), "x3": (0, 0, 1)}[k]
        out[e] = Fr(v)
    return out


PAPER_BASIS = {
    (RT0, 2): [[_p(x1=1), _p(x2=1)], [_p(x1=1, c=-1), _p(x2=1)], [_p(x1=1), _p(x2=1, c=-1)]],
    (RT0, 3): [[_p(x1=1), _p(x2=1), _p(x3=1, c=-1)], [_p(x1=1), _p(x2=1, c=-1), _p(x3=1)],
               [_p(x1=1, c=-1), _p(x2=1), _p(x3=1)], [_p(x1=1), _p(x2=1), _p(x3=1)]],
    (NED1, 2): [[_p(x2=-1), _p(x1=1)], [_p(x2=-1), _p(x1=1, c=-1)], [_p(c=1, x2=-1), _p(x1=1)]],
    (NED1, 3): [[_p(c=1, x3=-1, x2=-1), _p(x1=1), _p(x1=1)],
                [_p(x2=1), _p(c=1, x3=-1, x1=-1), _p(x2=1)],
                [_p(x3=1), _p(x3=1), _p(c=1, x2=-1, x1=-1)],
                [_p(x2=-1), _p(x1=1), {}],
                [{}, _p(x3=-1), _p(x2=1)],
                [_p(x3=1), {}, _p(x1=-1)]],
}


def _mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(a + b for a, b in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return out


def _int(p, dim):
    tot = Fr(0)
    for e, c in p.items():
        if any(e[dim:]):
            raise AssertionError("variable outside the dimension")
        tot += c * Fr(math.prod(math.factorial(a) for a in e[:dim]), math.factorial(sum(e[:dim]) + dim))
    return tot


def _deriv(p, var):
    out = {}
    for e, c in p.items():
        if e[var]:
            ne = list(e)
            ne[var] -= 1
            out[tuple(ne)] = out.get(tuple(ne), 0) + c * e[var]
    return out


def _const(p):
    assert all(sum(e) == 0 for e in p), "expected a constant"
    return sum(p.values(), Fr(0))


def exact_reference_matrices(kind, dim):
    basis = PAPER_BASIS[(kind, dim)]
    n = len(basis)
    M = [[Fr(0)] * n for _ in range(n)]
    K = [[Fr(0)] * n for _ in range(n)]
    meas = Fr(1, 2) if dim == 2 else Fr(1, 6)
    dv = []
    for f in basis:
        if kind == RT0:
            dv.append([sum((_const(_deriv(f[r], r)) for r in range(dim)), Fr(0))])
        elif dim == 2:
            dv.append([_const(_deriv(f[1], 0)) - _const(_deriv(f[0], 1))])
        else:
            dv.append([_const(_deriv(f[2], 1)) - _const(_deriv(f[1], 2)),
                       _const(_deriv(f[0], 2)) - _const(_deriv(f[2], 0)),
                       _const(_deriv(f[1], 0)) - _const(_deriv(f[0], 1))])
    for k in range(n):
        for l in range(n):
            M[k][l] = sum((_int(_mul(basis[k][r], basis[l][r]), dim) for r in range(dim)), Fr(0))
            K[k][l] = meas * sum((a * b for a, b in zip(dv[k], dv[l])), Fr(0))
    return K, M


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (RT0, 3), (NED1, 2), (NED1, 3)])
def test_reference_local_matrices_exact(ora, kind, dim):
    Kx, Mx = exact_reference_matrices(kind, dim)
    P = np.vstack([np.zeros(dim), np.eye(dim)])
    n = len(Kx)
    K, M = ora.local(kind, dim, P, np.ones(n))
    np.testing.assert_allclose(K, np.array(Kx, dtype=float), rtol=0, atol=2e-16)
    np.testing.assert_allclose(M, np.array(Mx, dtype=float), rtol=0, atol=2e-16)
    # spot values of the closed forms: 3D Nedelec mass diagonal 1/12, 3D RT0 div-div 3/2
    if (kind, dim) == (NED1, 3):
        assert Mx[0][0] == Fr(1, 12) and Mx[3][3] == Fr(1, 30) and Kx[0][0] == Fr(4, 3)
    if (kind, dim) == (RT0, 3):
        assert Kx[0][1] == Fr(3, 2) and Mx[3][3] == Fr(1, 20)


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (RT0, 3), (NED1, 2), (NED1, 3)])
def test_local_matrices_rule_independent(ora, kind, dim):
    """A degree-2 rule and a high-order collapsed rule agree on a general element."""
    rng = np.random.default_rng(7)
    P = rng.random((dim + 1, dim))
    n = 3 if dim == 2 else (4 if kind == RT0 else 6)
    s = rng.choice([-1.0, 1.0], size=n)
    K0, M0 = ora.local(kind, dim, P, s, 2.5)
    K1, M1 = ora.local(kind, dim, P, s, 2.5, rule=1, n=6)
    np.testing.assert_allclose(K0, K1, rtol=1e-13, atol=1e-13 * np.abs(K0).max())
    np.testing.assert_allclose(M0, M1, rtol=1e-13, atol=1e-13 * np.abs(M0).max())
