"""GPU parity against the oracle, through the C ABI (needs a GB300).

Topology (elem2dof, sign bits, dof2nodes) and the CSR pattern must be bit for
bit the oracle's; K and M values within 1e-12 of the entry scale defined in
tests/_parity.py. Sizes span many 256-element tiles with ragged tails; local
node order and element order are shuffled so that det B_K takes both signs;
edge cases: one element, no element, unused nodes, the L-shaped domain. Every
assembly schedule (the default two-pass kernels, the one-launch persistent
queue, element-block with 128 or 256 elements per CTA in mesh order or along
the Morton curve of the centroids) is checked, and the default path also
inside a CUDA graph.
"""
import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg
from tests._parity import compare, run_gpu

pytestmark = pytest.mark.gpu

RT0, NED1 = 1, 2


def _case(name):
    if name == "c1_rt2d_32":               # the 2D RT0 workload: 32x32 squares, unit coefficient, no jitter
        nodes, elems = mg.kuhn_square(32)
        return RT0, 2, nodes, elems, None
    if name == "ned2d_33_shuffled":
        nodes, elems = mg.kuhn_square(33, 0.2, 7)
        elems = mg.shuffle_local_order(elems, 7)
        return NED1, 2, nodes, elems, mg.log_uniform_coeff(7, elems.shape[0])
    if name == "rt2d_37_shuffled":
        nodes, elems = mg.kuhn_square(37, 0.2, 8)
        elems = mg.shuffle_local_order(elems, 8)
        return RT0, 2, nodes, elems, mg.log_uniform_coeff(8, elems.shape[0])
    if name == "ned3d_8":
        nodes, elems = mg.kuhn_cube(8, 0.2, 2)
        return NED1, 3, nodes, elems, mg.log_uniform_coeff(2, elems.shape[0])
    if name == "ned3d_13_shuffled":
        nodes, elems = mg.kuhn_cube(13, 0.2, 9)
        elems = mg.shuffle_local_order(elems, 9)
        perm = np.argsort(mg.uniform(9, 11, np.arange(elems.shape[0])))
        return NED1, 3, nodes, elems[perm], mg.log_uniform_coeff(9, elems.shape[0])
    if name == "rt3d_8":
        nodes, elems = mg.kuhn_cube(8, 0.2, 3)
        return RT0, 3, nodes, elems, mg.log_uniform_coeff(3, elems.shape[0])
    if name == "rt3d_13_shuffled":
        nodes, elems = mg.kuhn_cube(13, 0.2, 10)
        elems = mg.shuffle_local_order(elems, 10)
        perm = np.argsort(mg.uniform(10, 11, np.arange(elems.shape[0])))
        return RT0, 3, nodes, elems[perm], mg.log_uniform_coeff(10, elems.shape[0])
    if name == "lshape_4_ned2d":
        nodes, elems = mg.lshape(4)
        return NED1, 2, nodes, elems, None
    raise KeyError(name)


CASES = ["c1_rt2d_32", "ned2d_33_shuffled", "rt2d_37_shuffled", "ned3d_8", "ned3d_13_shuffled", "rt3d_8",
         "rt3d_13_shuffled", "lshape_4_ned2d"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("path", ["default", "chunks4", "blocked128", "blocked256", "fused128", "fused256"])
def test_parity(ora, name, path):
    kind, dim, nodes, elems, coeff = _case(name)
    o = ora.assemble(kind, dim, nodes, elems, coeff)
    g = run_gpu(kind, dim, nodes, elems, coeff, path=path)
    compare(g, o)


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (NED1, 2), (RT0, 3), (NED1, 3)])
@pytest.mark.parametrize("path", ["default", "blocked128", "fused256"])
def test_single_element_and_unused_nodes(ora, kind, dim, path):
    rng = np.random.default_rng(5)
    nodes = rng.random((9, dim))
    elems = np.array([[7, 2, 5] + ([1] if dim == 3 else [])], dtype=np.int32)
    o = ora.assemble(kind, dim, nodes, elems, np.array([2.5]))
    g = run_gpu(kind, dim, nodes, elems, np.array([2.5]), path=path)
    compare(g, o)


@pytest.mark.parametrize("kind,dim", [(RT0, 2), (NED1, 3)])
@pytest.mark.parametrize("path", ["default", "fused128"])
def test_empty_mesh(kind, dim, path):
    nodes = np.zeros((4, dim))
    elems = np.zeros((0, dim + 1), dtype=np.int32)
    g = run_gpu(kind, dim, nodes, elems, path=path)
    assert g["n_dofs"] == 0 and g["nnz"] == 0
    np.testing.assert_array_equal(g["rowptr"], [0])


@pytest.mark.parametrize("kind", [NED1, RT0])
def test_paths_agree_bitwise_and_runs_repeat(ora, kind):
    """The persistent queue (several element chunks at 131,712 tets), the plain
    two-pass and the element-block paths (mesh order and Morton order) form the
    same sums in the same order:
    identical bits, run after run; and the queue's result passes parity."""
    nodes, elems = mg.kuhn_cube(28, 0.2, 12)
    coeff = mg.log_uniform_coeff(12, elems.shape[0])
    a = run_gpu(kind, 3, nodes, elems, coeff, path="chunks3")
    others = [run_gpu(kind, 3, nodes, elems, coeff, path=p)
              for p in ("default", "two_pass", "chunks3", "chunks16", "blocked128", "blocked256", "fused128",
                        "fused256")]
    for key in ("K", "M"):
        for other in others:
            assert np.array_equal(a[key].view(np.uint64), other[key].view(np.uint64))
    compare(a, ora.assemble(kind, 3, nodes, elems, coeff))


def test_csr_is_symmetric_bitwise():
    kind, dim, nodes, elems, coeff = _case("rt3d_13_shuffled")
    g = run_gpu(kind, dim, nodes, elems, coeff)
    rows = np.repeat(np.arange(g["n_dofs"]), np.diff(g["rowptr"]))
    cols = g["colidx"]
    order = np.lexsort((rows, cols))          # transposed order
    for key in ("K", "M"):
        v = g[key]
        # entry (i,j) equals entry (j,i) bit for bit
        idx = np.lexsort((cols, rows))
        assert np.array_equal(idx, np.arange(len(v)))
        t = v[order]
        assert np.array_equal(v.view(np.uint64), t.view(np.uint64))


def test_one_shot_and_host_path_match_plan(ora):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    kind, dim, nodes, elems, coeff = _case("ned3d_8")
    g = run_gpu(kind, dim, nodes, elems, coeff)
    tn, te, tc = (torch.from_numpy(x).cuda() for x in (nodes, elems, coeff))
    one = ef.ned_assemble(3, tn, te, tc)
    np.testing.assert_array_equal(one["rowptr"].cpu().numpy(), g["rowptr"])
    np.testing.assert_array_equal(one["colidx"].cpu().numpy(), g["colidx"])
    np.testing.assert_array_equal(one["K"].cpu().numpy(), g["K"])
    np.testing.assert_array_equal(one["M"].cpu().numpy(), g["M"])
    plan = ef.Plan(kind, dim, nodes.shape[0], te)
    hn = torch.from_numpy(nodes).pin_memory()
    hc = torch.from_numpy(coeff).pin_memory()
    K, M = plan.assemble_host(hn, hc)
    np.testing.assert_array_equal(K.numpy(), g["K"])
    np.testing.assert_array_equal(M.numpy(), g["M"])
    plan.close()
    rt = ef.rt0_assemble(2, *(torch.from_numpy(x).cuda() for x in mg.kuhn_square(5)))
    o = ora.assemble(RT0, 2, *mg.kuhn_square(5))
    np.testing.assert_array_equal(rt["colidx"].cpu().numpy(), o["colidx"])
    assert np.abs(rt["K"].cpu().numpy() - o["K"]).max() <= 1e-12 * np.abs(o["K"]).max()


@pytest.mark.parametrize("shuffle", [False, True])
def test_host_path_chunked_copies_only_final_rows(shuffle):
    """ef_assemble_host on a plan with several element chunks copies each CSR
    range back only once every sum in it is done: a first call with other
    coefficients leaves different values in the staging buffers, so a range
    copied too early would differ from the device result. With the elements
    shuffled, rows become final only near the end; the result is the same."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(28, 0.2, 16)                 # 131,712 tets: 4 element chunks
    if shuffle:
        elems = elems[np.argsort(mg.uniform(16, 11, np.arange(elems.shape[0])))]
    coeff = mg.log_uniform_coeff(16, elems.shape[0])
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(np.ascontiguousarray(elems)).cuda())
    assert plan.info()["pipeline_chunks"] == 4
    K0, M0 = plan.assemble(torch.from_numpy(nodes).cuda(), torch.from_numpy(coeff).cuda())
    hn = torch.from_numpy(nodes).pin_memory()
    plan.assemble_host(hn, torch.from_numpy(3.0 * coeff).pin_memory())
    K, M = plan.assemble_host(hn, torch.from_numpy(coeff).pin_memory())
    assert torch.equal(K.view(torch.int64), K0.cpu().view(torch.int64))
    assert torch.equal(M.view(torch.int64), M0.cpu().view(torch.int64))
    plan.close()


def test_tuner_keeps_results_and_picks_a_schedule():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(36, 0.2, 14)           # 279,936 tets: 4, 8 and 16 chunks are tried
    coeff = mg.log_uniform_coeff(14, elems.shape[0])
    tn, tc = torch.from_numpy(nodes).cuda(), torch.from_numpy(coeff).cuda()
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    K0, M0 = plan.assemble_two_pass(tn, tc)
    chosen = plan.tune(tn, tc, reps=2)
    assert chosen in (0, -128, -256) or (chosen // 100 in (4, 8, 16) and (chosen // 10) % 10 in (0, 1, 2))
    K, M = plan.assemble(tn, tc)
    torch.cuda.synchronize()
    assert torch.equal(K.view(torch.int64), K0.view(torch.int64))
    assert torch.equal(M.view(torch.int64), M0.view(torch.int64))
    plan.close()


@pytest.mark.parametrize("name", ["ned2d_33_shuffled", "rt2d_37_shuffled", "ned3d_13_shuffled", "rt3d_13_shuffled"])
def test_separate_coefficients(ora, name):
    """ef_assemble2: K weighted by one coefficient array, M by another, against
    the oracle's assemble2; with equal arrays, ef_assemble's bits."""
    kind, dim, nodes, elems, coeff = _case(name)
    cM = mg.log_uniform_coeff(77, elems.shape[0])
    g = run_gpu(kind, dim, nodes, elems, coeff, coeff_M=cM)
    compare(g, ora.assemble2(kind, dim, nodes, elems, coeff, cM))
    same = run_gpu(kind, dim, nodes, elems, coeff, coeff_M=coeff.copy())
    one = run_gpu(kind, dim, nodes, elems, coeff)
    for key in ("K", "M"):
        assert np.array_equal(same[key].view(np.uint64), one[key].view(np.uint64))


def test_kernel_profile_events():
    """ef_plan_profile records the kernels of exactly the requested number of
    calls; the two-pass schedule reports both kernels, the one-launch queue
    all its time as the first kernel."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(20, 0.2, 15)
    tn = torch.from_numpy(nodes).cuda()
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    K = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    M = torch.empty_like(K)
    assert plan.info()["assemble_launches"] == 2
    plan.profile(3)
    for _ in range(5):
        plan.assemble(tn, None, K, M)
    first, second, calls = plan.profile_read()
    assert calls == 3 and first > 0 and second > 0
    plan.set_pipeline(4)
    plan.profile(2)
    for _ in range(2):
        plan.assemble(tn, None, K, M)
    first, second, calls = plan.profile_read()
    assert calls == 2 and first > 0 and second == 0
    plan.profile(0)
    assert plan.profile_read() == (0.0, 0.0, 0)
    plan.close()


def test_errors_are_reported():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(2)
    te = torch.from_numpy(elems).cuda()
    bad = elems.copy()
    bad[5, 1] = nodes.shape[0]                       # node id out of range
    with pytest.raises(ef.EdgeFemError) as e:
        ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(bad).cuda())
    assert e.value.code == ef.EF_ERR_RANGE
    bad = elems.copy()
    bad[3, 2] = bad[3, 0]                            # repeated node
    with pytest.raises(ef.EdgeFemError) as e:
        ef.Plan(RT0, 3, nodes.shape[0], torch.from_numpy(bad).cuda())
    assert e.value.code == ef.EF_ERR_ARG
    flat = nodes.copy()
    flat[:, 2] = 0.5                                 # every element degenerate
    plan = ef.Plan(NED1, 3, nodes.shape[0], te)
    plan.assemble(torch.from_numpy(flat).cuda())
    with pytest.raises(ef.EdgeFemError) as e:
        plan.check()
    assert e.value.code == ef.EF_ERR_DEGENERATE
    plan.check()                                     # the status word was cleared
    plan.assemble(torch.from_numpy(nodes).cuda())
    plan.check()
    plan.close()
    with pytest.raises(ef.EdgeFemError) as e:
        ef.rt0_assemble(3, torch.from_numpy(flat).cuda(), te)
    assert e.value.code == ef.EF_ERR_DEGENERATE


def test_poisoned_queue_times_out_and_recovers():
    """The one-launch queue's waits are bounded: with the first element
    chunk's completion count raised from the host (a tile that never comes),
    the sums give up after about a second, the call reports EF_ERR_TIMEOUT
    and the GPU stays usable; with the count restored the queue gives the
    two-pass bits again."""
    import time

    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(12, 0.2, 21)
    coeff = mg.log_uniform_coeff(21, elems.shape[0])
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    tn, tc = torch.from_numpy(nodes).cuda(), torch.from_numpy(coeff).cuda()
    K0, M0 = plan.assemble(tn, tc)
    plan.check()
    with pytest.raises(ef.EdgeFemError) as e:        # the two-pass schedule has no waits to poison
        plan.inject_stall(True)
    assert e.value.code == ef.EF_ERR_ARG
    plan.set_pipeline(4)
    plan.inject_stall(True)
    t0 = time.perf_counter()
    plan.assemble(tn, tc)
    with pytest.raises(ef.EdgeFemError) as e:
        plan.check()
    elapsed = time.perf_counter() - t0
    assert e.value.code == ef.EF_ERR_TIMEOUT
    assert 0.5 < elapsed < 20.0, elapsed
    plan.check()                                     # the status word was cleared
    plan.inject_stall(False)
    K1, M1 = plan.assemble(tn, tc)
    plan.check()
    assert torch.equal(K0, K1) and torch.equal(M0, M1)
    plan.close()


def test_cuda_graph_capture_replays_bitwise():
    """ef_assemble (one persistent launch with self-resetting queue counters)
    captured in a CUDA graph and replayed gives the same bits as a direct
    call, also after the coordinates change in place."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(28, 0.2, 13)
    coeff = mg.log_uniform_coeff(13, elems.shape[0])
    tn, tc = torch.from_numpy(nodes).cuda(), torch.from_numpy(coeff).cuda()
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    plan.set_pipeline(3)
    assert plan.info()["pipeline_chunks"] == 3
    K0, M0 = plan.assemble(tn, tc)
    K = torch.zeros_like(K0)
    M = torch.zeros_like(M0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.assemble(tn, tc, K, M, stream=s)            # warm-up outside the capture
        s.synchronize()
        K.zero_()
        M.zero_()
        with torch.cuda.graph(g, stream=s):
            plan.assemble(tn, tc, K, M, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(K.view(torch.int64), K0.view(torch.int64))
    assert torch.equal(M.view(torch.int64), M0.view(torch.int64))
    tn.mul_(1.5)                                          # new coordinates in place, replay again
    g.replay()
    K1, M1 = plan.assemble(tn, tc)
    torch.cuda.synchronize()
    assert torch.equal(K.view(torch.int64), K1.view(torch.int64))
    plan.check()
    plan.close()


@pytest.mark.parametrize("kind", [RT0, NED1])
def test_fig3_shared_edge_signs_gpu(kind):
    """The paper's Fig. 3 orientation example through the C ABI: sign bit of
    K_n's shared edge clear (+1), of K_m's set (-1), same global edge."""
    import json
    import os

    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    with open(os.path.join(os.path.dirname(__file__), "golden", "fig3_shared_edge_signs.json")) as f:
        g = json.load(f)
    elems = np.array([g["elems"]["K_n"], g["elems"]["K_m"]], dtype=np.int32)
    plan = ef.Plan(kind, 2, len(g["nodes"]), torch.from_numpy(elems).cuda())
    e2d, sb, _ = plan.topology()
    e2d, sb = e2d.cpu().numpy(), sb.cpu().numpy()
    ex = g["expected"]
    kn, km = ex["K_n_shared_local_edge"], ex["K_m_shared_local_edge"]
    assert ((sb[0] >> kn) & 1) == (0 if ex["K_n_sign"] > 0 else 1)
    assert ((sb[1] >> km) & 1) == (0 if ex["K_m_sign"] > 0 else 1)
    assert e2d[0][kn] == e2d[1][km]
    plan.close()


def test_fused_order_from_other_coordinates_and_graph():
    """The Morton grouping of ef_plan_set_fused comes from one set of
    coordinates; assembling with other coordinates and coefficients still
    gives the two-pass bits, call after call and from a CUDA graph (the split
    nonzeros' tickets reset themselves)."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(17, 0.2, 31)
    elems = mg.shuffle_local_order(elems, 31)
    perm = np.argsort(mg.uniform(31, 11, np.arange(elems.shape[0])))
    elems = elems[perm]
    dev = torch.device("cuda")
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).to(dev))
    other, _ = mg.kuhn_cube(17, 0.2, 32)
    plan.set_fused(torch.from_numpy(other * 3.0 + 1.0).to(dev), 128)
    info = plan.info()
    assert info["fused_sfc"] == 1 and info["assemble_launches"] == 1 and info["fused_block"] == 128
    tn = torch.from_numpy(nodes).to(dev)
    for seed in (1, 2):
        tc = torch.from_numpy(mg.log_uniform_coeff(seed, elems.shape[0])).to(dev)
        K0, M0 = plan.assemble_two_pass(tn, tc)
        for _ in range(2):
            K, M = plan.assemble(tn, tc)
            assert torch.equal(K.view(torch.int64), K0.view(torch.int64))
            assert torch.equal(M.view(torch.int64), M0.view(torch.int64))
    K = torch.full_like(K0, float("nan"))
    M = torch.full_like(M0, float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.assemble(tn, tc, K, M, stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.assemble(tn, tc, K, M, stream=s)
    for _ in range(3):
        K.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(K.view(torch.int64), K0.view(torch.int64))
        assert torch.equal(M.view(torch.int64), M0.view(torch.int64))
    plan.check()
    plan.close()
