"""Pins of the oracle's global matrices (no GPU).

* Brute force: on tiny jittered meshes with shuffled local node order (so
  det B_K takes both signs), the oracle's CSR equals a dense assembly of
  globally oriented basis functions written directly in physical
  coordinates (tests/_bruteforce.py), to ~1e-13 relative.
* Invariants of the exact matrices (Sec. 2.4 definitions):
  symmetry, positive definite M, curl K . grad = 0 (Nedelec), div K . rot = 0
  (2D RT), div K . curl = 0 (3D RT), curl . grad = 0, the interpolant of a
  constant field c has energy |Omega| |c|^2, kernel dimensions V-1 and E-V+1,
  invariance under local node order and element order, the 2D rotation
  identity M_Ned = M_RT and K_Ned = K_RT, linearity in the coefficient.
* Separate coefficients for K and M (assemble2): K from the brute force with
  the K coefficient, M from the brute force with the M coefficient; equal
  arrays reproduce assemble() bit for bit.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._bruteforce import brute_force, to_dense

RT0, NED1 = 1, 2
CASES = [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)]


def _mesh(dim, n, seed, shuffle=True, jitter=0.2):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(n, jitter, seed)
    else:
        nodes, elems = mg.kuhn_square(n, jitter, seed)
    if shuffle:
        elems = mg.shuffle_local_order(elems, seed + 100)
    return nodes, elems


@pytest.mark.parametrize("kind,dim", CASES)
def test_bruteforce_agreement(ora, kind, dim):
    n = 3 if dim == 3 else 4
    nodes, elems = _mesh(dim, n, 21)
    coeff = mg.log_uniform_coeff(21, elems.shape[0])
    r = ora.assemble(kind, dim, nodes, elems, coeff)
    Kb, Mb, d2n = brute_force(kind, dim, nodes, elems, coeff, nq=5)
    np.testing.assert_array_equal(r["dof2nodes"], d2n)
    K, M = to_dense(r, "K"), to_dense(r, "M")
    # the pattern holds every pair the brute force touches
    touched = (np.abs(Kb) + np.abs(Mb)) > 0
    patt = to_dense({**r, "P": np.ones(r["nnz"])}, "P") > 0
    assert not np.any(touched & ~patt)
    np.testing.assert_allclose(K, Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())
    np.testing.assert_allclose(M, Mb, rtol=0, atol=1e-13 * np.abs(Mb).max())


def _incidence_G(d2n, V):
    """Discrete gradient: edge {a < b} directed from b to a, (G p)_e = p_a - p_b."""
    G = np.zeros((d2n.shape[0], V))
    G[np.arange(d2n.shape[0]), d2n[:, 0]] = 1.0
    G[np.arange(d2n.shape[0]), d2n[:, 1]] = -1.0
    return G


def _curl_C(f2n, e2n):
    """Discrete curl: circulation around face a -> b -> c -> a against edges directed large -> small."""
    eid = {tuple(e): i for i, e in enumerate(e2n.tolist())}
    C = np.zeros((f2n.shape[0], e2n.shape[0]))
    for f, (a, b, c) in enumerate(f2n.tolist()):
        C[f, eid[(a, b)]] = -1.0
        C[f, eid[(b, c)]] = -1.0
        C[f, eid[(a, c)]] = 1.0
    return C


@pytest.mark.parametrize("kind,dim", CASES)
def test_symmetry_and_spd(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 5)
    coeff = mg.log_uniform_coeff(5, elems.shape[0])
    r = ora.assemble(kind, dim, nodes, elems, coeff)
    K, M = to_dense(r, "K"), to_dense(r, "M")
    assert np.array_equal(K, K.T) and np.array_equal(M, M.T)
    w = np.linalg.eigvalsh(M)
    assert w.min() > 1e-8 * w.max()
    wk = np.linalg.eigvalsh(K)
    assert wk.min() > -1e-12 * wk.max()


@pytest.mark.parametrize("kind,dim", CASES)
def test_kernels(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 9)
    V = nodes.shape[0]
    r = ora.assemble(kind, dim, nodes, elems, mg.log_uniform_coeff(9, elems.shape[0]))
    K = to_dense(r, "K")
    scale = np.abs(K).max()
    if kind == NED1 or dim == 2:
        # Nedelec: curl grad = 0; 2D RT: div rot = 0, rot = same incidence as grad
        G = _incidence_G(r["dof2nodes"], V)
        assert np.abs(K @ G).max() < 1e-12 * scale
        null_expect = V - 1
    else:
        e2n = ora.topology(NED1, 3, nodes, elems)["dof2nodes"]
        C = _curl_C(r["dof2nodes"], e2n)
        assert np.abs(K @ C).max() < 1e-12 * scale
        assert np.abs(C @ _incidence_G(e2n, V)).max() == 0.0
        null_expect = e2n.shape[0] - V + 1
    w = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == null_expect


def test_kernel_catches_a_wrong_sign(ora):
    """A planted mistake (one flipped face sign) breaks div K . curl = 0."""
    nodes, elems = _mesh(3, 2, 4)
    r = ora.assemble(RT0, 3, nodes, elems)
    e2n = ora.topology(NED1, 3, nodes, elems)["dof2nodes"]
    C = _curl_C(r["dof2nodes"], e2n)
    K = to_dense(r, "K")
    e0 = r["elem2dof"][0]                  # flip the sign of one face in ONE element only
    Kbad = K.copy()
    Kl, _ = ora.local(RT0, 3, nodes[elems[0]], r["sign"][0].astype(float))
    Kl2, _ = ora.local(RT0, 3, nodes[elems[0]], r["sign"][0].astype(float) * np.array([-1, 1, 1, 1]))
    for a in range(4):
        for b in range(4):
            Kbad[e0[a], e0[b]] += Kl2[a, b] - Kl[a, b]
    assert np.abs(Kbad @ C).max() > 1e-3 * np.abs(K).max()


@pytest.mark.parametrize("kind,dim", CASES)
def test_constant_field_energy(ora, kind, dim):
    nodes, elems = _mesh(dim, 4, 13)
    r = ora.assemble(kind, dim, nodes, elems)
    M = to_dense(r, "M")
    c = np.array([0.7, -1.3, 0.4])[:dim]
    d2n = r["dof2nodes"]
    Xa, Xb = nodes[d2n[:, 0]], nodes[d2n[:, 1]]
    if kind == NED1:
        u = (Xa - Xb) @ c                               # tangential integral along b -> a
    elif dim == 2:
        t = Xa - Xb
        u = np.stack([t[:, 1], -t[:, 0]], 1) @ c         # flux through R_cw(X_a - X_b)
    else:
        Nf = np.cross(Xb - Xa, nodes[d2n[:, 2]] - Xa)
        u = Nf @ c                                       # flux / (1/2) of the printed basis
    assert abs(u @ M @ u - c @ c) < 1e-12 * (c @ c)


@pytest.mark.parametrize("kind,dim", CASES)
def test_order_invariance(ora, kind, dim):
    nodes, elems = _mesh(dim, 3, 17, shuffle=False)
    coeff = mg.log_uniform_coeff(17, elems.shape[0])
    r0 = ora.assemble(kind, dim, nodes, elems, coeff)
    el1 = mg.shuffle_local_order(elems, 77)
    perm = np.argsort(mg.uniform(3, 1, np.arange(elems.shape[0])))
    r1 = ora.assemble(kind, dim, nodes, el1[perm], coeff[perm])
    np.testing.assert_array_equal(r0["rowptr"], r1["rowptr"])
    np.testing.assert_array_equal(r0["colidx"], r1["colidx"])
    for key in ("K", "M"):
        np.testing.assert_allclose(r0[key], r1[key], rtol=0, atol=1e-13 * np.abs(r0[key]).max())


def test_rotation_identity_2d(ora):
    nodes, elems = _mesh(2, 6, 31)
    coeff = mg.log_uniform_coeff(31, elems.shape[0])
    a = ora.assemble(RT0, 2, nodes, elems, coeff)
    b = ora.assemble(NED1, 2, nodes, elems, coeff)
    np.testing.assert_array_equal(a["colidx"], b["colidx"])
    for key in ("K", "M"):
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-14 * np.abs(a[key]).max())


@pytest.mark.parametrize("kind,dim", CASES)
def test_coefficient_linearity(ora, kind, dim):
    nodes, elems = _mesh(dim, 2, 3)
    c = mg.log_uniform_coeff(3, elems.shape[0])
    r1 = ora.assemble(kind, dim, nodes, elems, c)
    r2 = ora.assemble(kind, dim, nodes, elems, 2.0 * c)
    for key in ("K", "M"):
        np.testing.assert_allclose(r2[key], 2.0 * r1[key], rtol=1e-15, atol=1e-300)


@pytest.mark.parametrize("kind,dim", CASES)
def test_separate_coefficients(ora, kind, dim):
    n = 3 if dim == 3 else 4
    nodes, elems = _mesh(dim, n, 23)
    T = elems.shape[0]
    cK = mg.log_uniform_coeff(23, T)
    cM = mg.log_uniform_coeff(24, T)
    r = ora.assemble2(kind, dim, nodes, elems, cK, cM)
    Kb, _, _ = brute_force(kind, dim, nodes, elems, cK, nq=5)
    _, Mb, _ = brute_force(kind, dim, nodes, elems, cM, nq=5)
    np.testing.assert_allclose(to_dense(r, "K"), Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())
    np.testing.assert_allclose(to_dense(r, "M"), Mb, rtol=0, atol=1e-13 * np.abs(Mb).max())
    one = ora.assemble(kind, dim, nodes, elems, cK)
    same = ora.assemble2(kind, dim, nodes, elems, cK, cK.copy())
    for key in ("K", "M"):
        np.testing.assert_array_equal(same[key], one[key])
    unitM = ora.assemble2(kind, dim, nodes, elems, cK, None)
    np.testing.assert_array_equal(unitM["K"], one["K"])
    np.testing.assert_array_equal(unitM["M"], ora.assemble(kind, dim, nodes, elems, None)["M"])


@pytest.mark.parametrize("kind,dim", CASES)
def test_abs_sums_and_element_order_of_accumulation(ora, kind, dim):
    """Kabs / Mabs (the tolerance scale of the parity tests) are the sums of
    |local entries| over the elements; K / M are the plain sums."""
    nodes, elems = _mesh(dim, 2, 6)
    coeff = mg.log_uniform_coeff(6, elems.shape[0])
    r = ora.assemble(kind, dim, nodes, elems, coeff)
    N = r["n_dofs"]
    Ka, Ma, Ks, Ms = (np.zeros((N, N)) for _ in range(4))
    for e in range(elems.shape[0]):
        Kl, Ml = ora.local(kind, dim, nodes[elems[e]], r["sign"][e].astype(float), coeff[e])
        d = r["elem2dof"][e]
        Ka[np.ix_(d, d)] += np.abs(Kl)
        Ma[np.ix_(d, d)] += np.abs(Ml)
        Ks[np.ix_(d, d)] += Kl
        Ms[np.ix_(d, d)] += Ml
    np.testing.assert_array_equal(to_dense(r, "Kabs"), Ka)
    np.testing.assert_array_equal(to_dense(r, "Mabs"), Ma)
    np.testing.assert_array_equal(to_dense(r, "K"), Ks)
    np.testing.assert_array_equal(to_dense(r, "M"), Ms)
