"""End-to-end pin against numbers the paper prints: the 2D eddy-current
example of Sec. 4.2, Table 5 (no GPU).

The oracle assembles K + M (Nedelec, unit coefficients), the load vector of
F = curlv curl E + E by quadrature (36 points per triangle), scipy solves the
Galerkin system, and the oracle integrates the error against the exact E and
curl E. The energy errors must equal the printed ones to their last digit.
"""
import json
import os

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._eddy import exact, rhs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table5_eddy_errors.json")
NED1 = 2


def _levels():
    with open(GOLD) as f:
        return json.load(f)["levels"]


def eddy_error_oracle(ora, m, n=6):
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla

    nodes, elems = mg.kuhn_square(m)
    r = ora.assemble(NED1, 2, nodes, elems)
    N = r["n_dofs"]
    A = sps.csr_matrix((r["K"] + r["M"], r["colidx"], r["rowptr"]), shape=(N, N))
    x = ora.quad_points(2, nodes, elems, n)
    cen = nodes[elems].mean(1)
    inside = np.broadcast_to(cen[:, 0] > cen[:, 1], x.shape[:2])
    F1, F2 = rhs(x[..., 0], x[..., 1], inside)
    b = ora.load_vector(NED1, 2, nodes, elems, n, np.stack([F1, F2], -1))
    v = spla.spsolve(A.tocsc(), b)
    E1, E2, curlE = exact(x[..., 0], x[..., 1], inside)
    l2, _ = ora.norm_l2(NED1, 2, nodes, elems, n, np.stack([E1, E2], -1), v)
    cv = ora.fe_curl(NED1, 2, nodes, elems, v)
    c2, _ = ora.norm_l2(NED1, 2, nodes, elems, n, (curlE - cv[None, :])[..., None])
    return N, float(np.sqrt(l2 + c2))


@pytest.mark.parametrize("level", [0, 1])
def test_table5_energy_errors(ora, level):
    lv = _levels()[level]
    N, err = eddy_error_oracle(ora, lv["m"])
    assert N == lv["edges"]
    assert abs(err - lv["error"]) <= 1e-6 * lv["error"]
