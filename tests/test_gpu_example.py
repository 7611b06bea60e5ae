"""The documented usage example, run as written: plan, assembly, pattern,
check, differentiable energy with its adjoint gradient, quadrature points and
an L2 norm (needs a GB300). The energy and its gradient are checked against
an assembly of the same plan, and against the Euler identity
sum_i x_i . dJ/dx_i = u^T M u - u^T K u (K scales like 1/length, M like
length)."""
import pytest

pytestmark = pytest.mark.gpu


def test_documented_example():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef, meshgen as mg

    nodes, elems = mg.kuhn_cube(64, 0.2, 2)
    coeff = mg.log_uniform_coeff(2, elems.shape[0])
    dev = torch.device("cuda")
    tn, tc = torch.from_numpy(nodes).to(dev), torch.from_numpy(coeff).to(dev)

    plan = ef.Plan(ef.EF_NED1, 3, nodes.shape[0], torch.from_numpy(elems).to(dev))
    K, M = plan.assemble(tn, tc)
    rowptr, colidx = plan.pattern()
    plan.check()

    u = torch.randn(plan.n_dofs, dtype=torch.float64, device=dev)
    tn.requires_grad_(True)
    J = ef.energy(plan, tn, tc, u, u)
    J.backward()

    x = plan.quad_points(tn, 3)
    err2, _ = plan.norm_l2(tn, torch.ones_like(x), 3, v=u)

    rows = torch.repeat_interleave(torch.arange(plan.n_dofs, device=dev), torch.diff(rowptr))
    uKu = float((u[rows] * K * u[colidx.long()]).sum())
    uMu = float((u[rows] * M * u[colidx.long()]).sum())
    assert abs(float(J.detach()) - (uKu + uMu)) <= 1e-10 * (abs(uKu) + abs(uMu))
    euler = float((tn.detach() * tn.grad).sum())
    assert abs(euler - (uMu - uKu)) <= 1e-9 * (abs(uKu) + abs(uMu))
    assert x.shape == (27, elems.shape[0], 3) and float(err2[0]) > 0.0
    plan.check()
    plan.close()
