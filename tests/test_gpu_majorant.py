"""Table 3 (Sec. 4.1, majorant minimisation by Algorithm 1) through the
library: RT0 2D matrices (ef_assemble), quadrature points, the load vectors
int grad v . phi (ef_load_vector) and int f div phi (ef_load_derivative),
and the three norms (ef_norm_l2; ef_norm_l2_derivative for div y + f) on
the GPU; the P1
approximation and the linear solves by scipy in the test. Every printed
iterate of the 512- and 131,072-triangle meshes to the printed digits."""
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._majorant import GpuBackend, minimise
from tests.test_oracle_majorant import _table, check_iterates

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh", [0, 1])
def test_table3_majorant_iterates_gpu(mesh):
    t = _table()
    case = t["meshes"][mesh]
    nodes, elems = mg.kuhn_square(case["m"])
    backend = GpuBackend(nodes, elems)
    got = minimise(backend, nodes, elems, len(case["iterations"]))
    backend.close()
    check_iterates(got, case["iterations"], t["decimals"])
