"""Elements that the integer-pipe multiply hands back to the FP64 multiply.

The element kernels form their products on the integer pipes (csrc/ef_intmul.cuh)
for operands and products in the normal range and zero; an element with a
subnormal operand is recomputed with the FP64 multiply. Here the nodes on the
x = 0 face of a jittered Kuhn cube are moved to distinct subnormal x values, so
that the edge vectors between them have subnormal components and every element
touching the face takes the FP64 repeat. Checked: parity with the oracle on all
four element kinds, and for 3D RT0 the same bits as the element-block kernel,
which forms every product with the FP64 multiply (and so never repeats).
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._parity import compare, run_gpu

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2


def _mesh(dim, seed):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(6, 0.2, seed)
    else:
        nodes, elems = mg.kuhn_square(12, 0.2, seed)
    nodes = nodes.copy()
    face = np.flatnonzero(nodes[:, 0] == 0.0)
    assert face.size > 2
    # 3, 6, 9, ... times the smallest subnormal: distinct, their differences subnormal too
    nodes[face, 0] = 3 * np.arange(1, face.size + 1) * 5e-324
    assert np.all(nodes[face, 0] > 0) and np.all(nodes[face, 0] < 2.2250738585072014e-308)
    return nodes, elems, mg.log_uniform_coeff(seed, elems.shape[0])


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)])
def test_subnormal_operands_parity(ora, kind, dim):
    nodes, elems, coeff = _mesh(dim, 31)
    o = ora.assemble(kind, dim, nodes, elems, coeff)
    g = run_gpu(kind, dim, nodes, elems, coeff, path="two_pass")
    compare(g, o)


def test_subnormal_operands_same_bits_as_fp64_products():
    nodes, elems, coeff = _mesh(3, 32)
    a = run_gpu(RT0, 3, nodes, elems, coeff, path="two_pass")   # integer products, FP64 repeat on the face
    b = run_gpu(RT0, 3, nodes, elems, coeff, path="fused256")   # FP64 products throughout
    np.testing.assert_array_equal(a["K"].view(np.int64), b["K"].view(np.int64))
    np.testing.assert_array_equal(a["M"].view(np.int64), b["M"].view(np.int64))
