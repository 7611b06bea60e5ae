"""Pins of the oracle's mesh topology, DOF numbering and signs (no GPU).

* Edge / face counts equal the matrix sizes printed in Tables 1, 2 and 5.
* elem2dof / dof2nodes equal an independent numpy ranking of sorted node
  tuples (global numbering = rows of edges2nodes / faces2nodes, Sec. 3).
* The oracle decides signs geometrically; they must equal the combinatorial
  rules: the paper's 2D rule (Sec. 3, edge from node 2 to node 3 gets +1 iff
  its global node ids satisfy node2 > node3), applied to every directed local
  edge, and for faces s = -parity of (sorted face nodes, opposite node).
* nnz of the CSR pattern equals the closed-form count for the Kuhn meshes.
"""
import json
import os

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg

RT0, NED1 = 1, 2
GOLD = os.path.join(os.path.dirname(__file__), "golden")

EDGE2 = [(1, 2), (2, 0), (0, 1)]
EDGE3 = [(0, 1), (0, 2), (0, 3), (1, 2), (2, 3), (3, 1)]
FACE3 = [(0, 1, 2, 3), (0, 1, 3, 2), (0, 2, 3, 1), (1, 2, 3, 0)]


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_table2_cube_sizes(ora, level):
    g = _load("table2_cube_sizes.json")["levels"][str(level)]
    nodes, elems = mg.kuhn_cube(6 * 2 ** (level - 1))
    assert ora.topology(NED1, 3, nodes, elems)["n_dofs"] == g["ned_edges"]
    assert ora.topology(RT0, 3, nodes, elems)["n_dofs"] == g["rt_faces"]


@pytest.mark.parametrize("level", [5, 6, 7])
def test_table1_lshape_sizes(ora, level):
    g = _load("table1_lshape_sizes.json")["levels"][str(level)]
    nodes, elems = mg.lshape(level)
    assert elems.shape[0] == 6 * 4 ** level
    assert ora.topology(RT0, 2, nodes, elems)["n_dofs"] == g
    assert ora.topology(NED1, 2, nodes, elems)["n_dofs"] == g


def test_table5_square_sizes(ora):
    rows = _load("table5_square_sizes.json")["rows"]
    for T, E in rows[:2]:
        m = int(round((T // 2) ** 0.5))
        nodes, elems = mg.kuhn_square(m)
        assert elems.shape[0] == T
        assert ora.topology(NED1, 2, nodes, elems)["n_dofs"] == E


def test_printed_sizes_follow_the_mesh_family():
    """Every printed size (also the levels too large to mesh here) follows the
    Kuhn-family counting formulas, so the synthetic family is the paper's."""
    for lvl, g in _load("table2_cube_sizes.json")["levels"].items():
        n = 6 * 2 ** (int(lvl) - 1)
        V, T = (n + 1) ** 3, 6 * n ** 3
        E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
        F = 1 - V + E + T                       # Euler: V - E + F - T = 1
        assert (E, F) == (g["ned_edges"], g["rt_faces"])
    for lvl, g in _load("table1_lshape_sizes.json")["levels"].items():
        m = 2 ** int(lvl)
        V = (2 * m + 1) ** 2 - m * m
        assert V + 6 * m * m - 1 == g          # Euler: V - E + T = 1
    for T, E in _load("table5_square_sizes.json")["rows"]:
        m = int(round((T // 2) ** 0.5))
        assert 3 * m * m + 2 * m == E


def _independent_numbering(kind, dim, elems):
    nl = {(RT0, 2): 3, (NED1, 2): 3, (RT0, 3): 4, (NED1, 3): 6}[(kind, dim)]
    if kind == RT0 and dim == 3:
        ent = np.stack([np.sort(elems[:, list(f[:3])], axis=1) for f in FACE3], axis=1)
    else:
        loc = EDGE2 if dim == 2 else EDGE3
        ent = np.stack([np.sort(elems[:, list(e)], axis=1) for e in loc], axis=1)
    flat = ent.reshape(-1, ent.shape[-1])
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    return uniq, inv.reshape(-1, nl)


def _combinatorial_signs(kind, dim, elems):
    if kind == RT0 and dim == 3:
        s = np.empty((elems.shape[0], 4), dtype=np.int8)
        for k, f in enumerate(FACE3):
            sub = elems[:, list(f[:3])]
            order = np.argsort(sub, axis=1, kind="stable")
            perm = np.concatenate([np.array(f[:3])[order], np.full((elems.shape[0], 1), f[3])], axis=1)
            inv = np.zeros(elems.shape[0], dtype=np.int64)
            for a in range(4):
                for b in range(a + 1, 4):
                    inv += perm[:, a] > perm[:, b]
            parity = np.where(inv % 2 == 0, 1, -1)
            s[:, k] = -parity
        return s
    loc = EDGE2 if dim == 2 else EDGE3
    return np.stack([np.where(elems[:, t] > elems[:, h], 1, -1) for (t, h) in loc], axis=1).astype(np.int8)


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)])
@pytest.mark.parametrize("shuffle", [False, True])
def test_numbering_and_signs(ora, kind, dim, shuffle):
    if dim == 3:
        nodes, elems = mg.kuhn_cube(5, 0.2, 11)
    else:
        nodes, elems = mg.kuhn_square(9, 0.2, 11)
    if shuffle:
        elems = mg.shuffle_local_order(elems, 3)
    t = ora.topology(kind, dim, nodes, elems)
    uniq, e2d = _independent_numbering(kind, dim, elems)
    np.testing.assert_array_equal(t["dof2nodes"], uniq)
    np.testing.assert_array_equal(t["elem2dof"], e2d)
    np.testing.assert_array_equal(t["sign"], _combinatorial_signs(kind, dim, elems))


def test_paper_2d_rule_edge1(ora):
    """Sec. 3: the first edge of K_i runs from node 2 to node 3 and gets +1 iff
    elems2nodes(i,2) > elems2nodes(i,3)."""
    nodes, elems = mg.kuhn_square(6, 0.1, 2)
    elems = mg.shuffle_local_order(elems, 8)
    for kind in (RT0, NED1):
        s = ora.topology(kind, 2, nodes, elems)["sign"]
        np.testing.assert_array_equal(s[:, 0], np.where(elems[:, 1] > elems[:, 2], 1, -1))


def _nnz_formula(kind, dim, n):
    if dim == 3 and kind == NED1:
        return 115 * n ** 3 + 45 * n ** 2 + 3 * n
    if dim == 3:
        V, E, T = (n + 1) ** 3, 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3, 6 * n ** 3
        F = 1 - V + E + T
        return 7 * F - 36 * n * n
    E = 3 * n * n + 2 * n
    return 5 * E - 8 * n


@pytest.mark.parametrize("kind,dim,n", [(NED1, 3, 3), (NED1, 3, 6), (RT0, 3, 4), (RT0, 3, 7),
                                        (RT0, 2, 8), (NED1, 2, 13)])
def test_nnz_formula(ora, kind, dim, n):
    nodes, elems = mg.kuhn_cube(n) if dim == 3 else mg.kuhn_square(n)
    r = ora.assemble(kind, dim, nodes, elems)
    assert r["nnz"] == _nnz_formula(kind, dim, n)
    # every row is sorted, unique, and holds its diagonal
    rp, ci = r["rowptr"], r["colidx"]
    for i in range(r["n_dofs"]):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row


def test_error_codes(ora):
    nodes, elems = mg.kuhn_cube(2)
    bad = elems.copy()
    bad[3, 2] = nodes.shape[0]
    with pytest.raises(ora.OracleError) as e:
        ora.topology(NED1, 3, nodes, bad)
    assert e.value.code == -2
    bad = elems.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(ora.OracleError) as e:
        ora.topology(NED1, 3, nodes, bad)
    assert e.value.code == -1
    flat = nodes.copy()
    flat[:, 2] = 0.0
    with pytest.raises(ora.OracleError) as e:
        ora.assemble(RT0, 3, flat, elems)
    assert e.value.code == -3


@pytest.mark.parametrize("kind", [1, 2])
def test_fig3_shared_edge_signs(ora, kind):
    """The paper's worked orientation example (Fig. 3): with node c > node a the
    shared edge gets +1 in K_n and the opposite sign in K_m, for RT0 (normal)
    and Nedelec (tangential) alike, and both elements point to the same
    global edge."""
    with open(os.path.join(GOLD, "fig3_shared_edge_signs.json")) as f:
        g = json.load(f)
    nodes = np.array(g["nodes"])
    elems = np.array([g["elems"]["K_n"], g["elems"]["K_m"]], dtype=np.int32)
    r = ora.topology(kind, 2, nodes, elems)
    ex = g["expected"]
    kn, km = ex["K_n_shared_local_edge"], ex["K_m_shared_local_edge"]
    assert r["sign"][0][kn] == ex["K_n_sign"]
    assert r["sign"][1][km] == ex["K_m_sign"]
    assert r["elem2dof"][0][kn] == r["elem2dof"][1][km]
    a, c = g["node_names"]["a"], g["node_names"]["c"]
    assert sorted(r["dof2nodes"][r["elem2dof"][0][kn]].tolist()) == sorted([a, c])
