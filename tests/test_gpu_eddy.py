"""The paper's Table 5 through the GPU library (needs a GB300).

K + M, the load vector of F, the error norms and the per-element curls all
come from the C ABI (ef_assemble, ef_quad_points, ef_load_vector,
ef_norm_l2, ef_fe_curl); scipy solves the Galerkin system on the host. The
energy errors must equal the printed ones to their last digit. Also: the load
vector and the per-element curls against the oracle, entry by entry: each
entry within 1e-12 of the sum of the absolute values of the terms that make
it up (tests/_scales.py), the bound on either side's rounding error.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._eddy import exact, rhs
from tests._scales import fe_curl_scale, load_vector_scale
from tests.test_oracle_eddy import _levels
from tests.test_oracle_integration import _affine, _linear_dofs

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2
CASES = [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)]


def eddy_error_gpu(m, n=6):
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_square(m)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(NED1, 2, nodes.shape[0], torch.from_numpy(elems).to(dev))
    K, M = plan.assemble(tn, None)
    rowptr, colidx = plan.pattern()
    x = plan.quad_points(tn, n).cpu().numpy()
    cen = nodes[elems].mean(1)
    inside = np.broadcast_to(cen[:, 0] > cen[:, 1], x.shape[:2])
    F1, F2 = rhs(x[..., 0], x[..., 1], inside)
    b = plan.load_vector(tn, torch.from_numpy(np.ascontiguousarray(np.stack([F1, F2], -1))).to(dev), n)
    N = plan.n_dofs
    A = sps.csr_matrix(((K + M).cpu().numpy(), colidx.cpu().numpy(), rowptr.cpu().numpy()), shape=(N, N))
    v = torch.from_numpy(spla.spsolve(A.tocsc(), b.cpu().numpy())).to(dev)
    E1, E2, curlE = exact(x[..., 0], x[..., 1], inside)
    l2, _ = plan.norm_l2(tn, torch.from_numpy(np.ascontiguousarray(np.stack([E1, E2], -1))).to(dev), n, v=v)
    c2, _ = plan.norm_l2_derivative(tn, torch.from_numpy(np.ascontiguousarray(curlE[..., None])).to(dev), n, v=v)
    plan.check()
    plan.close()
    return N, float(np.sqrt(float(l2) + float(c2)))


@pytest.mark.parametrize("level", [0, 1, 2])
def test_table5_energy_errors_gpu(level):
    lv = _levels()[level]
    N, err = eddy_error_gpu(lv["m"])
    assert N == lv["edges"]
    assert abs(err - lv["error"]) <= 1e-6 * lv["error"]


@pytest.mark.parametrize("kind,dim", CASES)
def test_load_vector_and_curl_parity(ora, kind, dim):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(7, 0.2, 47) if dim == 3 else mg.kuhn_square(19, 0.2, 47)
    elems = mg.shuffle_local_order(elems, 147)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(kind, dim, nodes.shape[0], torch.from_numpy(elems).to(dev))
    A, c = _affine(dim, 47)
    n = 3
    xg = plan.quad_points(tn, n).cpu().numpy()
    bg = plan.load_vector(tn, torch.from_numpy(np.ascontiguousarray(xg @ A.T + c)).to(dev), n).cpu().numpy()
    xo = ora.quad_points(dim, nodes, elems, n)
    bo = ora.load_vector(kind, dim, nodes, elems, n, xo @ A.T + c)
    sb = load_vector_scale(ora, kind, dim, nodes, elems, n, xo @ A.T + c)
    assert np.all(np.abs(bg - bo) <= 1e-12 * sb), float((np.abs(bg - bo) / sb).max())
    v = mg.normal(47, mg.STREAM_V, plan.n_dofs)
    cg = plan.fe_curl(tn, torch.from_numpy(v).to(dev)).cpu().numpy()
    co = ora.fe_curl(kind, dim, nodes, elems, v)
    sc = fe_curl_scale(ora, kind, dim, nodes, elems, v)
    assert np.all(np.abs(cg - co) <= 1e-12 * sc), float((np.abs(cg - co) / sc).max())
    # the interpolant of an affine field: exact curl / divergence on every element
    d2n = plan.topology()[2].cpu().numpy()
    u = torch.from_numpy(_linear_dofs(kind, dim, nodes, d2n, A, c)).to(dev)
    cu = plan.fe_curl(tn, u).cpu().numpy()
    if kind == RT0:
        expect = np.trace(A)
    elif dim == 2:
        expect = A[1, 0] - A[0, 1]
    else:
        expect = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    assert np.max(np.abs(cu - expect)) < 1e-11 * (1 + np.abs(A).max())
    # load vector sums repeat bit for bit
    b2 = plan.load_vector(tn, torch.from_numpy(np.ascontiguousarray(xg @ A.T + c)).to(dev), n).cpu().numpy()
    assert np.array_equal(bg.view(np.uint64), b2.view(np.uint64))
    plan.check()
    plan.close()


@pytest.mark.parametrize("kind,dim", CASES)
def test_load_derivative_parity(ora, kind, dim):
    """ef_load_derivative (int g . D eta_i, D = div or curl) against the
    oracle for a smooth g on a jittered mesh with shuffled local order; the
    sums repeat bit for bit."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(7, 0.2, 53) if dim == 3 else mg.kuhn_square(19, 0.2, 53)
    elems = mg.shuffle_local_order(elems, 153)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(kind, dim, nodes.shape[0], torch.from_numpy(elems).to(dev))
    nc = 3 if (kind == NED1 and dim == 3) else 1
    w = np.array([1.3, -0.7, 0.4])[:dim]
    amp = np.array([0.9, -1.6, 0.5])[:nc]

    def g(x):
        return np.ascontiguousarray(np.sin(x @ w + 0.3)[..., None] * amp)

    n = 3
    xg = plan.quad_points(tn, n).cpu().numpy()
    bg = plan.load_derivative(tn, torch.from_numpy(g(xg)).to(dev), n).cpu().numpy()
    go = g(ora.quad_points(dim, nodes, elems, n))
    bo = ora.load_derivative(kind, dim, nodes, elems, n, go)
    assert np.max(np.abs(bo)) > 1e-3
    sb = load_vector_scale(ora, kind, dim, nodes, elems, n, go, derivative=True)
    assert np.all(np.abs(bg - bo) <= 1e-12 * sb), float((np.abs(bg - bo) / sb).max())
    b2 = plan.load_derivative(tn, torch.from_numpy(g(xg)).to(dev), n).cpu().numpy()
    assert np.array_equal(bg.view(np.uint64), b2.view(np.uint64))
    plan.check()
    plan.close()


@pytest.mark.parametrize("kind,dim", CASES)
def test_norm_of_derivative_parity(ora, kind, dim):
    """ef_norm_l2_derivative (||g - D v_h||^2, D = div or curl) against the
    oracle's per-element derivative and norm, per element and in total; with
    g = D v_h it vanishes."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(6, 0.2, 59) if dim == 3 else mg.kuhn_square(17, 0.2, 59)
    elems = mg.shuffle_local_order(elems, 159)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(kind, dim, nodes.shape[0], torch.from_numpy(elems).to(dev))
    nc = 3 if (kind == NED1 and dim == 3) else 1
    n = 3
    w = np.array([0.8, 1.7, -0.6])[:dim]
    amp = np.array([1.2, 0.3, -0.9])[:nc]
    xg = plan.quad_points(tn, n).cpu().numpy()
    g = np.ascontiguousarray(np.cos(xg @ w)[..., None] * amp)
    v = mg.normal(59, mg.STREAM_V, plan.n_dofs)
    tot, per = plan.norm_l2_derivative(tn, torch.from_numpy(g).to(dev), n, v=torch.from_numpy(v).to(dev),
                                       per_element=True)
    d = ora.fe_curl(kind, dim, nodes, elems, v).reshape(elems.shape[0], nc)
    xo = ora.quad_points(dim, nodes, elems, n)
    go = np.cos(xo @ w)[..., None] * amp
    to, po = ora.norm_l2(kind, dim, nodes, elems, n, go - d[None])
    assert abs(float(tot[0]) - to) <= 1e-12 * to
    assert np.max(np.abs(per.cpu().numpy() - po)) <= 1e-12 * np.max(po)
    dg = plan.fe_curl(tn, torch.from_numpy(v).to(dev)).reshape(1, -1, nc).expand(n ** dim, -1, -1).contiguous()
    zero, _ = plan.norm_l2_derivative(tn, dg, n, v=torch.from_numpy(v).to(dev))
    assert float(zero[0]) <= 1e-24 * to
    plan.check()
    plan.close()
