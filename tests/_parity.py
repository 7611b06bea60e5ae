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

# Plain relative error |gpu - oracle| / |oracle| is asserted <= TOL on every
# entry with |oracle_ij| >= REL_FLOOR * sqrt(A_ii A_jj). The scaled error
# above stays below 4e-15 on every workload, so there the plain relative
# error is at most 4e-15 / REL_FLOOR = 4e-13. Below the floor the entry is
# small by cancellation between (or inside) element contributions, and both
# sides' rounding errors, a few eps * sqrt(A_ii A_jj), are no longer small
# against it (measured: up to 1.1e-12 between 1e-3 and 1e-2, up to 3e-9 at
# 1e-6); there the scaled bound is the one that holds.
REL_FLOOR = 1e-2

# bands of |oracle_ij| / sqrt(A_ii A_jj) for the recorded error distribution
BANDS = (1e-2, 1e-3, 1e-6, 1e-9, 1e-12)


def diag_scale(ora: dict, key: str) -> np.ndarray:
    """sqrt(A_ii A_jj) per nonzero, A = sum of |local contributions|."""
    rowptr, colidx = ora["rowptr"], ora["colidx"]
    N = ora["n_dofs"]
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    a = ora[key + "abs"]
    diag = np.zeros(N)
    on = rows == colidx
    diag[rows[on]] = a[on]
    return np.sqrt(diag[rows] * diag[colidx])


def entry_scale(ora: dict, key: str) -> np.ndarray:
    """s_ij = max(|oracle_ij|, A_ij, sqrt(A_ii A_jj)) per nonzero."""
    return np.maximum(np.maximum(np.abs(ora[key]), ora[key + "abs"]), diag_scale(ora, key))


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
        elif path.startswith("fused"):
            plan.set_fused(tn, int(path[len("fused"):]))
            K, M = plan.assemble(tn, tc)
            K, M = plan.assemble(tn, tc, K, M)        # a second call: the tickets were reset by the first
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
    """Assert parity; returns error statistics.

    Topology and pattern bit for bit; every value within tol of its scale
    s_ij (above); and every value at least REL_FLOOR sqrt(A_ii A_jj) in
    magnitude within tol of itself (plain relative error). The statistics
    give, per band of |oracle_ij| / sqrt(A_ii A_jj), the share of entries and
    their largest plain relative error."""
    assert gpu["n_dofs"] == ora["n_dofs"]
    np.testing.assert_array_equal(gpu["elem2dof"], ora["elem2dof"])
    np.testing.assert_array_equal(gpu["signbits"], signbits_from_signs(ora["sign"]))
    np.testing.assert_array_equal(gpu["dof2nodes"], ora["dof2nodes"])
    np.testing.assert_array_equal(gpu["rowptr"], ora["rowptr"])
    np.testing.assert_array_equal(gpu["colidx"], ora["colidx"])
    stats = {}
    for key in ("K", "M"):
        g, o = gpu[key], ora[key]
        scale = entry_scale(ora, key)
        d = diag_scale(ora, key)
        err = np.abs(g - o)
        bad = err > tol * scale
        assert not bad.any(), (key, int(bad.sum()), float((err / np.where(scale > 0, scale, 1)).max()))
        ratio = np.abs(o) / np.where(d > 0, d, 1)
        rel = err / np.where(o != 0, np.abs(o), 1)
        sel = ratio >= REL_FLOOR
        worst = float(rel[sel].max()) if sel.any() else 0.0
        assert worst <= tol, (key, "plain relative error", worst, int((rel[sel] > tol).sum()))
        bands, hi = [], np.inf
        for lo in BANDS + (0.0,):
            m = (ratio >= lo) & (ratio < hi) if lo > 0 else (ratio < hi)
            bands.append({"ratio_ge": lo, "share": float(m.mean()) if m.size else 0.0, "count": int(m.sum()),
                          "max_rel_err": float(rel[m & (o != 0)].max()) if (m & (o != 0)).any() else 0.0,
                          "max_scaled_err": float((err[m] / np.where(scale[m] > 0, scale[m], 1)).max())
                          if m.any() else 0.0})
            hi = lo
        stats[key] = {
            "max_scaled_err": float((err / np.where(scale > 0, scale, 1)).max()) if err.size else 0.0,
            "max_rel_err": worst, "rel_floor": REL_FLOOR, "share_rel_checked": float(sel.mean()) if sel.size else 0.0,
            "bands": bands,
            "exact_zero_gpu_nonzero_oracle": int(((g == 0) & (o != 0)).sum()),
        }
    return stats


def worst_entries(gpu: dict, ora: dict, nodes: np.ndarray, elems: np.ndarray, key: str, k: int = 5) -> list:
    """The k entries of largest plain relative error, each with the elements
    that contribute to it (elements holding both DOFs) and whether every node
    of those elements lies on the boundary of the unit cube / square (where
    the workloads apply no jitter)."""
    g, o = gpu[key], ora[key]
    rows = np.repeat(np.arange(ora["n_dofs"]), np.diff(ora["rowptr"]))
    cols = ora["colidx"]
    rel = np.abs(g - o) / np.where(o != 0, np.abs(o), 1)
    d = diag_scale(ora, key)
    e2d = ora["elem2dof"]
    on_bnd = np.any((nodes <= 0.0) | (nodes >= 1.0), axis=1)
    out = []
    for i in np.argsort(-rel)[:k]:
        r, c = int(rows[i]), int(cols[i])
        els = np.nonzero((e2d == r).any(axis=1) & (e2d == c).any(axis=1))[0]
        out.append({"row": r, "col": c, "oracle": float(o[i]), "gpu": float(g[i]), "rel_err": float(rel[i]),
                    "A_ij": float(ora[key + "abs"][i]), "sqrt_AiiAjj": float(d[i]),
                    "elements": [int(e) for e in els],
                    "all_nodes_on_boundary": bool(on_bnd[elems[els]].all()) if els.size else None})
    return out
