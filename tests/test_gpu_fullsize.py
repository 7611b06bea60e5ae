"""GPU parity on the full-size workloads, against the full oracle (needs a GB300).

3D Nedelec 64^3 (1,572,864 tets), 3D RT0 128^3 (12,582,912 tets) and 3D
Nedelec 96^3 (5,308,416 tets), jittered +-0.2h, coefficient log-uniform in
[0.1, 10]: topology and CSR pattern bit for bit, K and M within 1e-12 of
max(|oracle|, sum |contributions|), through the same ef_assemble launch the
benchmark times. Oracle time on one core is about 12 s, 80 s and 50 s.
"""
import gc

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._parity import compare, run_gpu

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2


@pytest.mark.parametrize("name,kind,n,seed", [("ned3d_64", NED1, 64, 2), ("rt3d_128", RT0, 128, 3),
                                              ("ned3d_96", NED1, 96, 5)])
def test_fullsize_parity(ora, name, kind, n, seed):
    nodes, elems = mg.kuhn_cube(n, 0.2, seed)
    coeff = mg.log_uniform_coeff(seed, elems.shape[0])
    g = run_gpu(kind, 3, nodes, elems, coeff)
    o = ora.assemble(kind, 3, nodes, elems, coeff)
    stats = compare(g, o)
    print(name, stats)
    del g, o
    gc.collect()
