"""Batched assembly (ef_batch_*) on the GPU: one persistent launch (or the
two-launch form) over many uneven meshes gives, mesh by mesh, exactly the bits
of ef_assemble on that mesh (and so the oracle's values), under every schedule
the autotuner can pick, and when replayed from a CUDA graph."""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._parity import compare

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2


def _meshes(kind, count, lo, hi, seed):
    sizes = mg.batch_sizes(seed, count, lo, hi)
    out = []
    for b, n in enumerate(sizes):
        nodes, elems = mg.kuhn_cube(int(n), 0.2, 1000 * seed + b)
        coeff = mg.log_uniform_coeff(1000 * seed + b, elems.shape[0])
        out.append((nodes, elems, coeff))
    return out


def _setup(kind, meshes):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    nodes = [t(m[0]) for m in meshes]
    elems = [t(m[1]) for m in meshes]
    coeff = [t(m[2]) for m in meshes]
    batch = ef.Batch(kind, 3, [m[0].shape[0] for m in meshes], elems)
    K = [torch.full((z,), float("nan"), dtype=torch.float64, device="cuda") for z in batch.nnz]
    M = [torch.full((z,), float("nan"), dtype=torch.float64, device="cuda") for z in batch.nnz]
    batch.bind(nodes, coeff, K, M)
    ref = []
    for i in range(len(meshes)):
        plan = ef.Plan(kind, 3, meshes[i][0].shape[0], elems[i])
        k, m = plan.assemble(nodes[i], coeff[i])
        ref.append((k.clone(), m.clone()))
        plan.close()
    return batch, nodes, elems, coeff, K, M, ref


def _same_bits(K, M, ref):
    import torch

    torch.cuda.synchronize()
    for (k, m), (rk, rm) in zip(zip(K, M), ref):
        assert torch.equal(k.view(torch.int64), rk.view(torch.int64))
        assert torch.equal(m.view(torch.int64), rm.view(torch.int64))


@pytest.mark.parametrize("kind", [NED1, RT0])
def test_batch_equals_per_mesh_assembly(ora, kind):
    meshes = _meshes(kind, 12, 1, 9, 7)
    batch, nodes, elems, coeff, K, M, ref = _setup(kind, meshes)
    batch.assemble()
    batch.check()
    _same_bits(K, M, ref)
    # and parity with the oracle on two of the meshes
    for i in (0, 5):
        rowptr, colidx = batch.pattern(i)
        g = {"n_dofs": batch.n_dofs[i], "rowptr": rowptr.cpu().numpy(), "colidx": colidx.cpu().numpy(),
             "K": K[i].cpu().numpy(), "M": M[i].cpu().numpy()}
        o = ora.assemble(kind, 3, *meshes[i])
        np.testing.assert_array_equal(g["rowptr"], o["rowptr"])
        np.testing.assert_array_equal(g["colidx"], o["colidx"])
        for key in ("K", "M"):
            from tests._parity import entry_scale
            assert np.all(np.abs(g[key] - o[key]) <= 1e-12 * entry_scale(o, key))
    batch.close()


def test_batch_every_schedule_and_the_tuner():
    meshes = _meshes(NED1, 9, 1, 12, 8)
    batch, nodes, elems, coeff, K, M, ref = _setup(NED1, meshes)
    for tile in (128, 256):
        for dyn, ec in ((0, 0), (1, 0), (1, 1), (1, 3)):
            for lf in (0, 1):
                for st in (256, 4096):
                    batch.set_config(elems_per_tile=tile, dynamic=dyn, largest_first=lf, sum_tile=max(st, tile),
                                     ctas_per_sm=2 if ec else 1, elem_ctas=ec, two_launch=0)
                    for k in K + M:
                        k.fill_(float("nan"))
                    batch.assemble()
                    batch.assemble()          # queue counters reset themselves between launches
                    batch.check()
                    _same_bits(K, M, ref)
    batch.set_config(two_launch=1)
    for k in K + M:
        k.fill_(float("nan"))
    batch.assemble()
    batch.check()
    _same_bits(K, M, ref)
    cfg = batch.tune(reps=2)
    assert cfg["two_launch"] in (0, 1)
    assert cfg["elems_per_tile"] in (128, 256) and cfg["ctas_per_sm"] >= 1
    for k in K + M:
        k.fill_(float("nan"))
    batch.assemble()
    batch.check()
    _same_bits(K, M, ref)
    batch.close()


def test_batch_in_cuda_graph():
    import torch

    meshes = _meshes(NED1, 6, 2, 10, 9)
    batch, nodes, elems, coeff, K, M, ref = _setup(NED1, meshes)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.assemble(stream=s)
        s.synchronize()
        for k in K + M:
            k.fill_(float("nan"))
        with torch.cuda.graph(g, stream=s):
            batch.assemble(stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    batch.check()
    _same_bits(K, M, ref)
    batch.close()


@pytest.mark.parametrize("two_launch", [1, 0])
def test_batch_plan_per_call_buffers_and_graph(two_launch):
    """ef_batch_plan_create / ef_batch_assemble with the per-mesh buffers passed
    as pointer tables on each call: two calls into two different sets of
    buffers, then a CUDA graph of the call replayed twice with new
    coefficients written into the captured buffers, each equal bit for bit to
    per-mesh ef_assemble; under the two-launch and the persistent schedule."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    meshes = _meshes(NED1, 70, 1, 7, 11)           # more than the 64 meshes of one descriptor kernel
    batch, nodes, elems, coeff, K, M, ref = _setup(NED1, meshes)
    batch.set_config(two_launch=two_launch)
    K2 = [torch.full_like(k, float("nan")) for k in K]
    M2 = [torch.full_like(m, float("nan")) for m in M]
    for k in K + M:
        k.fill_(float("nan"))
    batch.assemble_tables(batch.tables(nodes, coeff, K2, M2))
    batch.assemble_tables(batch.tables(nodes, coeff, K, M))
    batch.check()
    _same_bits(K, M, ref)
    _same_bits(K2, M2, ref)
    # graph: captured once, replayed with other coefficients in the same buffers
    tabs = batch.tables(nodes, coeff, K, M)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.assemble_tables(tabs, stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            batch.assemble_tables(tabs, stream=s)
    torch.cuda.synchronize()
    for seed in (3, 4):
        for i, (nd, el, _) in enumerate(meshes):
            coeff[i].copy_(torch.from_numpy(mg.log_uniform_coeff(100 * seed + i, el.shape[0])))
        for k in K + M:
            k.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        want = []
        for i, (nd, el, _) in enumerate(meshes):
            plan = ef.Plan(NED1, 3, nd.shape[0], elems[i])
            k, m = plan.assemble(nodes[i], coeff[i])
            want.append((k.clone(), m.clone()))
            plan.close()
        batch.check()
        _same_bits(K, M, want)
    with pytest.raises(ef.EdgeFemError):
        bad = batch.tables(nodes, coeff, K, M)
        bad[2][0] = None                            # a NULL K for a non-empty mesh
        batch.assemble_tables(bad)
    batch.close()
