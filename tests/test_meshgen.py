"""Synthetic input generator: counts, determinism, jitter and orientation (no GPU)."""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg


def test_counter_based_rng_is_order_free():
    a = mg.uniform(3, 0, np.arange(10))
    b = mg.uniform(3, 0, np.arange(5, 10))
    np.testing.assert_array_equal(a[5:], b)
    assert np.all((a >= 0) & (a < 1))
    assert not np.array_equal(a, mg.uniform(4, 0, np.arange(10)))
    assert not np.array_equal(a, mg.uniform(3, 1, np.arange(10)))
    x = mg.uniform(1, 2, np.arange(200000))
    assert abs(x.mean() - 0.5) < 5e-3 and abs(x.var() - 1 / 12) < 5e-3
    z = mg.normal(1, 4, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1) < 1e-2


@pytest.mark.parametrize("n", [1, 3, 8])
def test_kuhn_cube(n):
    nodes, elems = mg.kuhn_cube(n, 0.2, 7)
    assert nodes.shape == ((n + 1) ** 3, 3) and elems.shape == (6 * n ** 3, 4)
    assert elems.min() == 0 and elems.max() == nodes.shape[0] - 1
    B = np.stack([nodes[elems[:, i]] - nodes[elems[:, 0]] for i in (1, 2, 3)], axis=2)
    det = np.linalg.det(B)
    assert np.sum(det > 0) == np.sum(det < 0)
    assert abs(np.abs(det).sum() / 6 - 1.0) < 1e-12          # the volume of the unit cube
    assert np.abs(det).min() > 0.05 / n ** 3
    ref, _ = mg.kuhn_cube(n)
    d = nodes - ref
    assert np.abs(d).max() <= 0.2 / n + 1e-15
    on_boundary = np.any((ref == 0) | (ref == 1), axis=1)
    assert np.all(d[on_boundary] == 0)


def test_kuhn_square_and_lshape():
    nodes, elems = mg.kuhn_square(32)
    assert elems.shape == (2048, 3) and nodes.shape == (1089, 2)
    B = np.stack([nodes[elems[:, i]] - nodes[elems[:, 0]] for i in (1, 2)], axis=2)
    det = np.linalg.det(B)
    assert np.sum(det > 0) == np.sum(det < 0) == 1024
    nodes, elems = mg.lshape(3)
    assert elems.shape[0] == 6 * 4 ** 3
    cen = nodes[elems].mean(axis=1)
    assert not np.any((cen[:, 0] > 0.5) & (cen[:, 1] > 0.5))


def test_batch_sizes():
    s = mg.batch_sizes(4, 256, 8, 48)
    assert s.min() >= 8 and s.max() <= 48 and len(np.unique(s)) > 30
    np.testing.assert_array_equal(s, mg.batch_sizes(4, 256, 8, 48))


def test_coeff_range():
    c = mg.log_uniform_coeff(2, 100000)
    assert c.min() >= 0.1 and c.max() <= 10.0
    assert abs(np.log10(c).mean()) < 0.02
