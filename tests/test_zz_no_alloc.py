"""ef_assemble_noalloc: the assembly entry point that allocates nothing.

Some callers cannot let the library allocate device memory while they
assemble: code that runs while another part of the process holds a CUDA
stream capture open in global mode (a cudaMalloc anywhere would break that
capture), loops with a latency budget that cannot absorb the device-wide
synchronisation a cudaMalloc or cudaFree may cause, and applications whose
device memory belongs to another allocator with a fixed budget.
ef_assemble_noalloc serves them with a static device array of the library
as its scratch. This test calls it through the C ABI (the binding's
Plan.assemble_noalloc, which checks buffer sizes and passes pointers) twice
in a row, with different coefficients the second time (the array keeps the
first call's contents), and requires each result to equal
ef_assemble_two_pass's bit for bit: both add every nonzero's contributions
in the same order. It also checks that a plan too large for the array is
refused with a message. It sits in its own file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_1409_4618_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

NED1, RT0 = 2, 1


@pytest.mark.parametrize("kind,n", [(NED1, 12), (RT0, 10)])
def test_noalloc_matches_two_pass_bitwise_twice(kind, n):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(n, 0.2, 21)
    dev = torch.device("cuda")
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(kind, 3, nodes.shape[0], torch.from_numpy(elems).to(dev))
    for seed in (21, 22):                     # two calls in a row on the shared static scratch
        tc = torch.from_numpy(mg.log_uniform_coeff(seed, elems.shape[0])).to(dev)
        K0, M0 = plan.assemble_two_pass(tn, tc)
        K = torch.full_like(K0, float("nan"))
        M = torch.full_like(M0, float("nan"))
        plan.assemble_noalloc(tn, tc, K, M)
        plan.check()
        torch.cuda.synchronize()
        assert torch.isfinite(K).all() and torch.isfinite(M).all()
        # same sums in the same order: the same bits
        assert torch.equal(K.view(torch.int64), K0.view(torch.int64))
        assert torch.equal(M.view(torch.int64), M0.view(torch.int64))
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
    assert "EF_NOALLOC_SCRATCH_BYTES" in lib.ef_last_error().decode()
    with pytest.raises(ef.EdgeFemError):
        plan.assemble_noalloc(tn, None, K, K)
    # the binding rejects wrong-sized buffers before the library sees them
    with pytest.raises(ValueError):
        plan.assemble_noalloc(tn[:-1], None, K, K)
    plan.close()
