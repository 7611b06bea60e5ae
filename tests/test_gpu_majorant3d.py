"""Algorithm 1 (Sec. 4.1) on tetrahedra through the GPU library, against the
same chain run on the oracle: the unit cube as 12^3 Kuhn cubes (10,368
tetrahedra, the size of Table 4's first mesh). Every library quantity of the
chain is compared entry by entry: the 3D RT0 K and M (ef_assemble; pattern
bit for bit, values as in the other parity tests), the load vectors
int grad v . phi_i (ef_load_vector) and int f div phi_i (ef_load_derivative),
each within 1e-12 of the sum of the absolute values of its terms, the norms
||grad(u - v)||^2, ||grad v - y||^2 (ef_norm_l2) and ||div y + f||^2
(ef_norm_l2_derivative) of every iteration within a relative 1e-12 (each
side's norm taken of the same flux y), and the iterates (beta, sqrt(M),
I_eff), which also pass through scipy's solves, within a relative 1e-9.
The P1 approximation and the linear solves are host numpy / scipy. Table 4's
own meshes are not stated: its printed values are not a pin."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sps

from paper_1409_4618_gb300 import meshgen as mg
from tests._majorant import GpuBackend, OracleBackend, minimise
from tests._parity import compare
from tests._scales import load_vector_scale

pytestmark = pytest.mark.gpu

RT0 = 1


def test_majorant_3d_chain_gpu_vs_oracle(ora):
    nodes, elems = mg.kuhn_cube(12)
    ro, rg = {}, {}
    got_o = minimise(OracleBackend(ora, nodes, elems), nodes, elems, 4, record=ro)
    gpu = GpuBackend(nodes, elems)
    got_g = minimise(gpu, nodes, elems, 4, record=rg)
    # RT0 3D matrices: the parity of the other tests
    o = ora.assemble(RT0, 3, nodes, elems)
    e2d, sb, d2n = gpu.plan.topology()
    rowptr, colidx = gpu.plan.pattern()
    g = {"n_dofs": gpu.plan.n_dofs, "nnz": gpu.plan.nnz, "elem2dof": e2d.cpu().numpy(), "signbits": sb.cpu().numpy(),
         "dof2nodes": d2n.cpu().numpy(), "rowptr": rowptr.cpu().numpy(), "colidx": colidx.cpu().numpy(),
         "K": sps.csr_matrix(rg["K"]).data, "M": sps.csr_matrix(rg["M"]).data}
    compare(g, o)
    # load vectors, entry by entry (each side's own quadrature points, the same rule)
    n = 4
    s_grad = load_vector_scale(ora, RT0, 3, nodes, elems, n, ro["gv"])
    assert np.all(np.abs(rg["b_grad"] - ro["b_grad"]) <= 1e-12 * s_grad)
    s_div = load_vector_scale(ora, RT0, 3, nodes, elems, n, np.ascontiguousarray(ro["fx"][..., None]),
                              derivative=True)
    assert np.all(np.abs(rg["b_div"] - ro["b_div"]) <= 1e-12 * s_div)
    # norms: ||grad(u - v)||^2, then each iteration's two norms of the oracle's own flux y
    assert abs(rg["err_v"] - ro["err_v"]) <= 1e-12 * ro["err_v"]
    for y, t1, t2 in zip(ro["ys"], ro["t1"], ro["t2"]):
        g1 = gpu.norm_l2(rg["gv"], n, y)
        g2 = gpu.norm_derivative(np.ascontiguousarray(-rg["fx"][..., None]), n, y)
        assert abs(g1 - t1) <= 1e-12 * t1 and abs(g2 - t2) <= 1e-12 * t2
    for a, b in zip(got_g, got_o):
        for x, z in zip(a, b):
            assert abs(x - z) <= 1e-9 * abs(z), (got_g, got_o)
    gpu.close()
    path = os.environ.get("EF_PARITY_STATS")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": "majorant_3d_kuhn12", "iterates_gpu": got_g, "iterates_oracle": got_o}) + "\n")
