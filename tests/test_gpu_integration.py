"""GPU vectorised integration (Sec. 3.1, norm_L2) through the C ABI.

Against the oracle: per-element squared L2 norms of E - v_h for an affine
field E and a random DOF vector v, on every element kind with shuffled local
node order (det B_K of both signs); both sides use exact rules for these
quadratic integrands (their own points), so they agree to rounding. Also:
|Omega| and int x_c^2 = 1/3 from the physical points, the interpolant of a
constant field reproduced at every point, fixed-order totals that repeat bit
for bit, argument errors.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests.test_oracle_integration import _constant_dofs

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2
CASES = [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)]


def _mesh(dim, n, seed):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(n, 0.2, seed)
    else:
        nodes, elems = mg.kuhn_square(n, 0.2, seed)
    elems = mg.shuffle_local_order(elems, seed + 100)
    perm = np.argsort(mg.uniform(seed, 11, np.arange(elems.shape[0])))
    return nodes, np.ascontiguousarray(elems[perm])


def _plan(kind, dim, nodes, elems):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    return ef.Plan(kind, dim, nodes.shape[0], torch.from_numpy(elems).cuda()), torch.from_numpy(nodes).cuda()


def _affine_field(dim, seed):
    A = mg.normal(seed, 12, dim * dim).reshape(dim, dim)
    b = mg.normal(seed, 13, dim)
    return A, b


@pytest.mark.parametrize("kind,dim", CASES)
def test_l2_error_parity(ora, kind, dim):
    import torch

    nodes, elems = _mesh(dim, 9 if dim == 3 else 23, 41)
    plan, tn = _plan(kind, dim, nodes, elems)
    A, b = _affine_field(dim, 41)
    v = mg.normal(41, mg.STREAM_V, plan.n_dofs)
    n = 3
    xg = plan.quad_points(tn, n)
    fg = torch.einsum("qec,rc->qer", xg, torch.from_numpy(A).cuda()) + torch.from_numpy(b).cuda()
    tv = torch.from_numpy(v).cuda()
    total_g, elem_g = plan.norm_l2(tn, fg.contiguous(), n, v=tv, per_element=True)
    xo = ora.quad_points(dim, nodes, elems, n)
    fo = xo @ A.T + b
    total_o, elem_o = ora.norm_l2(kind, dim, nodes, elems, n, fo, v)
    # scale: (||E||_K + ||v_h||_K)^2 per element, from the oracle
    e_only = ora.norm_l2(kind, dim, nodes, elems, n, fo)[1]
    vh_only = ora.norm_l2(kind, dim, nodes, elems, n, np.zeros_like(fo), v)[1]
    scale = (np.sqrt(e_only) + np.sqrt(vh_only)) ** 2
    eg = elem_g.cpu().numpy()
    assert np.all(np.abs(eg - elem_o) <= 1e-12 * scale)
    assert abs(float(total_g) - total_o) <= 1e-12 * scale.sum()
    plan.close()


@pytest.mark.parametrize("kind,dim", CASES)
def test_points_measure_and_constants(kind, dim):
    import torch

    nodes, elems = _mesh(dim, 5 if dim == 3 else 11, 43)
    plan, tn = _plan(kind, dim, nodes, elems)
    n = 3
    x = plan.quad_points(tn, n)
    T = elems.shape[0]
    one, _ = plan.norm_l2(tn, torch.ones((n ** dim, T, 1), dtype=torch.float64, device="cuda"), n)
    assert abs(float(one) - 1.0) < 1e-13
    for c in range(dim):
        sq, _ = plan.norm_l2(tn, x[..., c:c + 1].contiguous(), n)
        assert abs(float(sq) - 1.0 / 3.0) < 1e-13
    # interpolant of a constant field: v_h = c at every point
    topo = plan.topology()
    d2n = topo[2].cpu().numpy()
    cvec = np.array([0.7, -1.3, 0.4])[:dim]
    u = torch.from_numpy(_constant_dofs(kind, dim, nodes, d2n, cvec)).cuda()
    vals = plan.fe_values(tn, u, n)
    assert torch.max(torch.abs(vals - torch.from_numpy(cvec).cuda())).item() < 1e-12
    cf = torch.from_numpy(np.broadcast_to(cvec, (n ** dim, T, dim)).copy()).cuda()
    err, _ = plan.norm_l2(tn, cf, n, v=u)
    assert float(err) < 1e-24
    plan.check()
    plan.close()


def test_totals_repeat_and_errors():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = _mesh(3, 7, 45)
    plan, tn = _plan(NED1, 3, nodes, elems)
    v = torch.from_numpy(mg.normal(45, mg.STREAM_V, plan.n_dofs)).cuda()
    f = plan.quad_points(tn, 4)
    a, ea = plan.norm_l2(tn, f, 4, v=v, per_element=True)
    b, eb = plan.norm_l2(tn, f, 4, v=v, per_element=True)
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    assert torch.equal(ea.view(torch.int64), eb.view(torch.int64))
    with pytest.raises(ef.EdgeFemError):
        plan.quad_points(tn, 9)
    with pytest.raises(ef.EdgeFemError):
        plan.norm_l2(tn, f[..., :2].contiguous(), 4, v=v)     # ncomp must equal dim with v
    plan.close()
