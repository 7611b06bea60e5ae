"""GPU adjoint of J = u^T K u + v^T M v (3D Nedelec), through the C ABI.

Checked against the oracle's forward-mode (dual number) adjoint (every node
gradient within 1e-11 of the sum of its elements' absolute gradients), against
central finite differences of J computed from the GPU's own assembled
matrices on the 4^3 sub-mesh (seed 55), and for bitwise run-to-run
reproducibility.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._scales import adjoint_node_scale

pytestmark = pytest.mark.gpu

NED1 = 2


def _setup(n, seed, shuffle=False):
    nodes, elems = mg.kuhn_cube(n, 0.2, seed)
    if shuffle:
        elems = mg.shuffle_local_order(elems, seed)
    coeff = mg.log_uniform_coeff(seed, elems.shape[0])
    return nodes, elems, coeff


def _gpu_adjoint(nodes, elems, coeff, u, v):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    plan = ef.Plan(NED1, 3, nodes.shape[0], t(elems.astype(np.int32)))
    J, gx, gs = plan.adjoint(t(nodes), t(coeff), t(u), t(v))
    plan.check()
    out = float(J.cpu()[0]), gx.cpu().numpy(), gs.cpu().numpy()
    plan.close()
    return out


def _gpu_energy(plan, nodes, coeff, u, v):
    import torch

    K, M = plan.assemble(torch.from_numpy(nodes).cuda(), torch.from_numpy(coeff).cuda())
    rowptr, colidx = plan.pattern()
    rows = torch.repeat_interleave(torch.arange(plan.n_dofs, device="cuda"), torch.diff(rowptr))
    cols = colidx.long()
    tu, tv = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    return float((tu[rows] * K * tu[cols]).sum() + (tv[rows] * M * tv[cols]).sum())


@pytest.mark.parametrize("n,seed,shuffle", [(4, 55, False), (7, 3, True), (12, 4, False)])
def test_adjoint_vs_oracle(ora, n, seed, shuffle):
    nodes, elems, coeff = _setup(n, seed, shuffle)
    N = ora.topology(NED1, 3, nodes, elems)["n_dofs"]
    u = mg.normal(seed, mg.STREAM_U, N)
    v = mg.normal(seed, mg.STREAM_V, N)
    Jo, gxo, gso = ora.adjoint(NED1, 3, nodes, elems, coeff, u, v)
    Jg, gxg, gsg = _gpu_adjoint(nodes, elems, coeff, u, v)
    assert abs(Jg - Jo) <= 1e-12 * abs(Jo) * 10
    # per node and coordinate: within 1e-11 of sum_K |dJ_K/dx| (the element
    # gradients summed into it; their cancellation is what makes an entry small)
    scale_x = adjoint_node_scale(ora, NED1, 3, nodes, elems, coeff, u, v)
    assert np.all(np.abs(gxg - gxo) <= 1e-11 * scale_x), float((np.abs(gxg - gxo) / scale_x).max())
    np.testing.assert_allclose(gsg, gso, rtol=1e-11, atol=1e-13 * np.abs(gso).max())


def test_adjoint_vs_central_differences_4cube():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems, coeff = _setup(4, 55)
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    u = mg.normal(55, mg.STREAM_U, plan.n_dofs)
    v = mg.normal(55, mg.STREAM_V, plan.n_dofs)
    J, gx, gs = _gpu_adjoint(nodes, elems, coeff, u, v)
    assert abs(_gpu_energy(plan, nodes, coeff, u, v) - J) <= 1e-12 * abs(J) * 10
    rng = np.random.default_rng(1)
    # fourth-order central differences: truncation O(h^4), rounding eps |J| / h
    h = 1e-4

    def shifted(a, c, d):
        x = nodes.copy()
        x[a, c] += d
        return _gpu_energy(plan, x, coeff, u, v)

    for _ in range(16):
        a, c = rng.integers(nodes.shape[0]), rng.integers(3)
        fd = (8 * (shifted(a, c, h) - shifted(a, c, -h)) - (shifted(a, c, 2 * h) - shifted(a, c, -2 * h))) / (12 * h)
        assert abs(fd - gx[a, c]) <= 1e-6 * max(abs(gx[a, c]), 1e-3 * np.abs(gx).max())
    for _ in range(8):
        e = rng.integers(elems.shape[0])
        cp, cm = coeff.copy(), coeff.copy()
        hs = 0.5 * coeff[e]            # J is linear in sigma: the difference quotient is exact up to rounding
        cp[e] += hs
        cm[e] -= hs
        fd = (_gpu_energy(plan, nodes, cp, u, v) - _gpu_energy(plan, nodes, cm, u, v)) / (2 * hs)
        assert abs(fd - gs[e]) <= 1e-6 * max(abs(gs[e]), 1e-3 * np.abs(gs).max())
    plan.close()


def test_adjoint_bitwise_repeatable():
    nodes, elems, coeff = _setup(9, 6)
    N = 6 * 9 ** 3 + 1000
    from paper_1409_4618_gb300 import edgefem as ef  # noqa: F401

    import oracle

    N = oracle.topology(NED1, 3, nodes, elems)["n_dofs"]
    u = mg.normal(6, mg.STREAM_U, N)
    v = mg.normal(6, mg.STREAM_V, N)
    a = _gpu_adjoint(nodes, elems, coeff, u, v)
    b = _gpu_adjoint(nodes, elems, coeff, u, v)
    assert a[0] == b[0]
    assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64))
    assert np.array_equal(a[2].view(np.uint64), b[2].view(np.uint64))


def test_energy_autograd_wrapper():
    """edgefem.energy is J(nodes, coeff) with the library's gradient: the value
    and (scaled) gradients through torch.autograd equal ef_adjoint's."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems, coeff = _setup(5, 21)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    plan = ef.Plan(NED1, 3, nodes.shape[0], t(elems.astype(np.int32)))
    u = t(mg.normal(21, mg.STREAM_U, plan.n_dofs))
    v = t(mg.normal(21, mg.STREAM_V, plan.n_dofs))
    J0, gx0, gs0 = plan.adjoint(t(nodes), t(coeff), u, v)
    x = t(nodes).requires_grad_(True)
    s = t(coeff).requires_grad_(True)
    J = ef.energy(plan, x, s, u, v)
    assert J.shape == () and float(J.detach()) == float(J0[0])
    (3.0 * J).backward()
    assert torch.equal(x.grad, 3.0 * gx0)
    assert torch.equal(s.grad, 3.0 * gs0)
    with pytest.raises(ValueError):
        ef.energy(plan, x, s, u.clone().requires_grad_(True), v)
    plan.close()
