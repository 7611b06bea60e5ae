"""Helpers of the GPU parity tests: run the CUDA library through its C ABI and
compare with the oracle (topology and pattern bit for bit, values within the
stated tolerance)."""
from __future__ import annotations

import numpy as np

# Per nonzero (i, j): |gpu - oracle| <= TOL * s_ij with
#   s_ij = max(|oracle_ij|, A_ij, sqrt(A_ii A_jj)),
# A_ij = sum over elements of |local contribution| to (i, j). The local K and
# M of every element are symmetric positive semi-definite, so each local entry
# is bounded by sqrt(L_kk L_ll), and the rounding error of an entry computed
# from the element's geometry scales with that bound, not with the entry
# itself (entries that vanish exactly, e.g. on right-angled elements, carry
# only rounding noise on both sides). Summing over elements, by Cauchy-Schwarz
# the error of a global entry is bounded by a multiple of sqrt(A_ii A_jj).
TOL = 1e-12


def entry_scale(ora: dict, key: str) -> np.ndarray:
    rowptr, colidx = ora["rowptr"], ora["colidx"]
    N = ora["n_dofs"]
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    a = ora[key + "abs"]
    diag = np.zeros(N)
    on = rows == colidx
    diag[rows[on]] = a[on]
    return np.maximum(np.maximum(np.abs(ora[key]), a), np.sqrt(diag[rows] * diag[colidx]))


def signbits_from_signs(sign: np.ndarray) -> np.ndarray:
    bits = np.zeros(sign.shape[0], dtype=np.uint8)
    for k in range(sign.shape[1]):
        bits |= ((sign[:, k] < 0).astype(np.uint8) << k)
    return bits


def run_gpu(kind, dim, nodes, elems, coeff=None, path="default", check=True, coeff_M=None):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    dev = torch.device("cuda")
    tn = torch.from_numpy(np.ascontiguousarray(nodes)).to(dev)
    te = torch.from_numpy(np.ascontiguousarray(elems, dtype=np.int32)).to(dev)
    tc = None if coeff is None else torch.from_numpy(np.ascontiguousarray(coeff)).to(dev)
    plan = ef.Plan(kind, dim, nodes.shape[0], te)
    try:
        if coeff_M is not None:
            K, M = plan.assemble2(tn, tc, torch.from_numpy(np.ascontiguousarray(coeff_M)).to(dev))
        elif path == "two_pass":
            K, M = plan.assemble_two_pass(tn, tc)
        elif path.startswith("blocked"):
            plan.set_block(int(path[len("blocked"):]))
            K, M = plan.assemble(tn, tc)
        elif path.startswith("chunks"):
            plan.set_pipeline(int(path[len("chunks"):]))
            K, M = plan.assemble(tn, tc)
        else:
            K, M = plan.assemble(tn, tc)
        if check:
            plan.check()
        rowptr, colidx = plan.pattern()
        e2d, sb, d2n = plan.topology()
        torch.cuda.synchronize()
        return {
            "n_dofs": plan.n_dofs, "nnz": plan.nnz,
            "elem2dof": e2d.cpu().numpy(), "signbits": sb.cpu().numpy(), "dof2nodes": d2n.cpu().numpy(),
            "rowptr": rowptr.cpu().numpy(), "colidx": colidx.cpu().numpy(),
            "K": K.cpu().numpy(), "M": M.cpu().numpy(),
        }
    finally:
        plan.close()


def compare(gpu: dict, ora: dict, tol: float = TOL) -> dict:
    """Assert parity; returns error statistics."""
    assert gpu["n_dofs"] == ora["n_dofs"]
    np.testing.assert_array_equal(gpu["elem2dof"], ora["elem2dof"])
    np.testing.assert_array_equal(gpu["signbits"], signbits_from_signs(ora["sign"]))
    np.testing.assert_array_equal(gpu["dof2nodes"], ora["dof2nodes"])
    np.testing.assert_array_equal(gpu["rowptr"], ora["rowptr"])
    np.testing.assert_array_equal(gpu["colidx"], ora["colidx"])
    stats = {}
    for key in ("K", "M"):
        g, o, a = gpu[key], ora[key], ora[key + "abs"]
        scale = entry_scale(ora, key)
        err = np.abs(g - o)
        bad = err > tol * scale
        assert not bad.any(), (key, int(bad.sum()), float((err / np.where(scale > 0, scale, 1)).max()))
        big = np.abs(o) > 1e-6 * scale          # entries that are not zero up to rounding
        stats[key] = {
            "max_scaled_err": float((err / np.where(scale > 0, scale, 1)).max()) if err.size else 0.0,
            "max_rel_err_large": float((err[big] / np.abs(o[big])).max()) if big.any() else 0.0,
        }
    return stats
