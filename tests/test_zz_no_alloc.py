"""ef_assemble_noalloc: the assembly entry point that allocates nothing.

Callers that must not allocate device memory while they assemble (inside an
open global-mode stream capture, in latency-bound loops, under a foreign
allocator's fixed budget) use ef_assemble_noalloc, whose scratch is a static
device array of the library. This test calls it through the C ABI twice in a
row, with different coefficients the second time (the array keeps the first
call's contents), and compares each result with ef_assemble's within the
parity tolerance of the other tests; it also checks that a plan too large for
the array is refused. It sits in its own file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

NED1, RT0 = 2, 1
TOL = 1e-12


@pytest.mark.parametrize("kind,n", [(NED1, 12), (RT0, 10)])
def test_noalloc_matches_ef_assemble_twice(kind, n):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    lib = ef.load()
    nodes, elems = mg.kuhn_cube(n, 0.2, 21)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(kind, 3, nodes.shape[0], torch.from_numpy(elems).to(dev))
    stream = torch.cuda.current_stream()
    for seed in (21, 22):                     # two calls in a row on the shared static scratch
        tc = torch.from_numpy(mg.log_uniform_coeff(seed, elems.shape[0])).to(dev)
        K0, M0 = plan.assemble(tn, tc)
        K = torch.full_like(K0, float("nan"))
        M = torch.full_like(M0, float("nan"))
        st = lib.ef_assemble_noalloc(plan.handle, ctypes.c_void_p(tn.data_ptr()), ctypes.c_void_p(tc.data_ptr()),
                                     ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(M.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == ef.EF_OK, lib.ef_last_error()
        plan.check()
        torch.cuda.synchronize()
        for got, ref in ((K, K0), (M, M0)):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.isfinite(g).all()
            # same sums in the same order: agreement far inside the tolerance of the parity tests
            assert np.abs(g - r).max() <= TOL * np.abs(r).max()
    plan.close()


def test_noalloc_rejects_plans_larger_than_its_array():
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    lib = ef.load()
    nodes, elems = mg.kuhn_cube(33)            # 215,622 tets > 199,728 for 3D Nedelec
    plan = ef.Plan(NED1, 3, nodes.shape[0], torch.from_numpy(elems).cuda())
    K = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    tn = torch.from_numpy(nodes).cuda()
    st = lib.ef_assemble_noalloc(plan.handle, ctypes.c_void_p(tn.data_ptr()), None, ctypes.c_void_p(K.data_ptr()),
                                 ctypes.c_void_p(K.data_ptr()), None)
    assert st == ef.EF_ERR_SIZE
    plan.close()
