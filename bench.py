#!/usr/bin/env python3
"""Benchmark: assembly of 3D Nedelec K and M into CSR on GB300.

One step = one ef_assemble call (element matrices in closed form + the
fixed-order sum into CSR) on the 3D Nedelec workload: the unit cube as a
64^3 grid of cubes split into 6 tetrahedra (1,572,864 tets), interior nodes
jittered by +-0.2h (seed 2), per-element coefficient log-uniform in
[0.1, 10]. The plan (topology + pattern) is built before timing, as in a
shape-optimisation loop where only coordinates and coefficients change.

Prints one JSON line: throughput (M elements / s), e2e through the host-buffer
C-ABI call, the roofline of the step's dominant kernel (timed per launch by
CUDA events the library records on the launching stream inside the timed
region) against this GPU's FP64 pipe rate measured first by the library's
probe (ef_fp64_probe), the HBM fraction of the whole step, the clocks seen
while timing, the CPU oracle timed on this host, and the other workloads:
batched (256 meshes, one ef_batch_assemble call per step replayed from a
CUDA graph), adjoint (96^3), RT0 (3D 128^3, 2D 32^2) and the vectorised
integration (L2 error at 27 points per element), the library share of the
majorant minimisation (Sec. 4.1) on the 33.5 M-triangle square and on the
5.3 M-tetrahedron cube, and the 2D RT0 and Nedelec assembly on Table 1's
L-shaped domain (level 11).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain FP64 quadrature assembler
that the tests compare against) on a bounded sample of the same workload.
Under torchrun (N > 1) every rank assembles its own replica (the single-mesh
path is not sharded: replicas only) and rank 0 reports the job total.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1409_4618_gb300 import meshgen as mg  # noqa: E402

WORKLOAD = {"name": "ned3d_kuhn64_jitter0.2", "kind": 2, "dim": 3, "n": 64, "jitter": 0.2, "seed": 2}
METRIC = "M elements/s assembled to CSR (K+M), % HBM roofline; batched & adjoint vs plain"
UNIT = "Melem/s"
# FP64 pipe peak: 152 SMs x 2 FP64 results per clock per SM x 2070 MHz (the
# GB300's 1.25 TFLOP/s FP64 with FMA = 2 flops); DADD, DMUL, DFMA count 1 op.
SMS, FP64_PER_CLK_PER_SM, SM_MAX_MHZ = 152, 2, 2070
FP64_PEAK_TOPS = SMS * FP64_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
L2_BYTES = 129 * 1024 * 1024
# FP64 peak the legs divide by: the probe's measured DFMA rate once the fp64
# leg has run (run_gpu runs it first), else the nominal figure above
FP64_PEAK = {"T_ops_per_s": FP64_PEAK_TOPS, "source": "nominal"}
# FP64 arithmetic operations per tetrahedron of the adjoint kernel, counted
# from the source (csrc/ef_adjoint.cu): B 9, H 18, adj(H) 12, det 9, 1/|det|
# 4 (two Newton steps), r^3 2, a 6, a^T H a 9, Whitney coefficients 17, P 30,
# <P, A> 6, J 4, A P 27, scale factors 12, Gamma 36, B Gamma 27, node 0 6,
# sigma J 1. Its products but the last run on the integer pipes: H 6, adj(H)
# 6, det 4, r^3 2, a^T H a 4, P 6, <P, A> 1, J 3, A P 9, scale factors 11,
# Gamma 12, B Gamma 9.
ADJOINT_FP64_OPS_PER_TET = 9 + 18 + 12 + 9 + 4 + 2 + 6 + 9 + 17 + 30 + 6 + 4 + 27 + 12 + 36 + 27 + 6 + 1
ADJOINT_INT_PIPE_OPS_PER_TET = 6 + 6 + 4 + 2 + 4 + 6 + 1 + 3 + 9 + 11 + 12 + 9
ADJOINT_FP64_PIPE_OPS_PER_TET = ADJOINT_FP64_OPS_PER_TET - ADJOINT_INT_PIPE_OPS_PER_TET
# executed FP64 instructions per tetrahedron of the adjoint kernel (ncu sass
# counters on the 24^3 cube: 1 DADD, 161 DFMA, 1 DMUL)
ADJOINT_FP64_EXECUTED_PER_TET = 163
# DRAM bytes (read + write) per element of the Nedelec-3D element kernel of
# the two-pass schedule, from ncu dram__bytes_{read,write}.sum of one launch
# on the 48^3 cube (663,552 tets); the launch's traffic grows in proportion
# to the elements.
ELEMENT_KERNEL_DRAM_BYTES_PER_TET = (75.176192e6 + 177.140224e6) / 663552


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _nvtx(torch, name):
    """Mark the timed region as an NVTX range (a profiler can filter on it)."""
    try:
        if name:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _workload():
    w = WORKLOAD
    nodes, elems = mg.kuhn_cube(w["n"], w["jitter"], w["seed"])
    coeff = mg.log_uniform_coeff(w["seed"], elems.shape[0])
    return nodes, elems, coeff


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def job_timing(ms_local: float, units_local: float, dist=None, device="cpu"):
    """Whole-job timing over the ranks: (max of the ranks' milliseconds, sum of
    the units they processed). Without a process group, the local values."""
    import torch

    t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=device)
    if dist is None:
        return float(t[0]), float(t[1])
    ms = t[:1].clone()
    units = t[1:].clone()
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return float(ms.item()), float(units.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, val in zip(names, r[5:9]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# FP64 instructions per element of each element kernel as executed (ncu
# sm__sass_thread_inst_executed_op_{dadd,dfma,dmul}_pred_on.sum of one launch
# divided by its elements; every FP64 warp instruction had all 32 lanes on):
# (kind, dim) -> DADD, DFMA, DMUL. Measured on the 24^3 cube (3D) and the
# level-5 L-shape (2D); the counts do not depend on the mesh. No DMUL: the
# products run on the integer pipes; the additions are DFMAs with a
# per-thread 1.0 (csrc/ef_fp64.cuh), which run at the FP64 pipe's full rate
# where DADD runs at 84 % of it.
ELEMENT_KERNEL_FP64_EXECUTED = {
    (2, 3): {"dadd": 0, "dfma": 92, "dmul": 0},
    (1, 3): {"dadd": 0, "dfma": 56, "dmul": 0},
    (1, 2): {"dadd": 0, "dfma": 25, "dmul": 0},
    (2, 2): {"dadd": 1, "dfma": 30, "dmul": 0},
}
ELEMENT_KERNEL_FP64_MIX = ELEMENT_KERNEL_FP64_EXECUTED[(2, 3)]


def fp64_executed_per_element(kind: int, dim: int) -> int:
    return sum(ELEMENT_KERNEL_FP64_EXECUTED[(kind, dim)].values())
FP64_PROBE_ITERS = 100_000


def run_fp64_probe(gpu_index: int) -> dict:
    """This GPU's FP64 pipe throughput, measured by the library's probe kernel
    (ef_fp64_probe: independent chains of one operation on every SM) for DFMA,
    DADD and DMUL, three launches each, with the SM clock sampled meanwhile.
    The DFMA rate is the peak of the element kernels' roofline; the rate for
    the element kernel's own instruction mix is reported beside it. Also the
    integer-pipe multiply alone and in half of the chains beside DFMA in the
    other half (the two pipes at once)."""
    from paper_1409_4618_gb300 import edgefem as ef

    rates = {}
    with ClockSampler(gpu_index) as clk:
        for name, op in (("dfma", 0), ("dadd", 1), ("dmul", 2), ("int_mul", 3), ("dfma_and_int_mul", 4),
                         ("dfma_literal_operands", 5), ("add_as_dfma", 6)):
            best = None
            for _ in range(3):
                r, ms = ef.ef_fp64_probe(op, FP64_PROBE_ITERS)
                if best is None or r > best[0]:
                    best = (r, ms)
            rates[name] = {"ops_per_s": best[0], "T_ops_per_s": best[0] / 1e12, "ms_per_launch": best[1]}
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz")
    for v in rates.values():
        v["ops_per_clk_per_sm"] = v["ops_per_s"] / (SMS * mhz * 1e6) if mhz else None
    mix = {k: v for k, v in ELEMENT_KERNEL_FP64_MIX.items() if v}
    t_mix = sum(mix[k] / rates[k]["ops_per_s"] for k in mix)
    return {"rates": rates, "clocks": clocks, "peak_T_ops_per_s": rates["dfma"]["T_ops_per_s"],
            "element_mix_T_ops_per_s": sum(mix.values()) / t_mix / 1e12, "element_mix": mix,
            "how": f"ef_fp64_probe: {SMS} SMs x 4 CTAs x 256 threads x 8 independent chains x "
                   f"{FP64_PROBE_ITERS} rounds per launch, best of 3, CUDA events on the launching stream"}


def fp64_ops_per_element(kind: int, dim: int) -> int:
    """FP64 arithmetic operations (add, multiply, FMA each 1) of one element's
    local matrices in the closed forms of csrc/ef_element.cuh, counted from the
    source; the reciprocal 1/|det| is two Newton steps, 4 FMA. In the element
    kernels the products (and the exact doublings) run on the integer pipes
    (INT_PIPE_OPS_PER_ELEMENT), the rest on the FP64 pipe."""
    if (kind, dim) == (2, 3):
        # B 9, H 18, adj(H) 12, det 9, 1/|det| 4, sigma*r 2, K: 1 + 6 + 15, M: 1 + 6 + 41
        return 9 + 18 + 12 + 9 + 4 + 2 + 22 + 48
    if (kind, dim) == (1, 3):
        # B 9, H 18, det 9, 1/|det| 4, sigma*r 2, row sums 6, c0 5, scales 4, q 3, t 3, entries 12, K 1
        return 9 + 18 + 9 + 4 + 2 + 6 + 5 + 4 + 3 + 3 + 12 + 1
    if (kind, dim) == (1, 2):
        # B 4, H 6, det 2, 1/|det| 4, sigma*r 2, cM 1, row sums 2, c0 3, scales 2, c0s q 3, t 2, entries 6, K 1
        return 4 + 6 + 2 + 4 + 2 + 1 + 2 + 3 + 2 + 3 + 2 + 6 + 1
    # 2D Nedelec: B 4, H 6, det 2, 1/|det| 4, sigma*r 2, cM 1, g 3, g01 g02 2, g00 1, entries 18, K 1
    return 4 + 6 + 2 + 4 + 2 + 1 + 3 + 2 + 1 + 18 + 1


# Of those, the operations that the two-pass element kernel runs on the
# integer pipes (csrc/ef_intmul.cuh, bit for bit the FP64 results): every
# product, and in 2D the exact doublings 2 sigma/|det| (and in 2D Nedelec the
# three doubled diagonal sums), which had been FP64 instructions.
INT_PIPE_OPS_PER_ELEMENT = {
    (2, 3): 6 + 6 + 3 + 1 + 2 + 1 + 6 + 1 + 6,   # H, adj(H), cross, det, sigma*r, cK, h, cM, g: 32
    (1, 3): 6 + 3 + 1 + 2 + 1 + 2 + 1 + 3 + 1,   # H, cross, det, sigma*r, cM, m5 m20, c0s, q, kv: 20
    (1, 2): 3 + 1 + 2 + 1 + 2 + 1 + 2 + 1,       # H, det, sigma*r, cM, m4 m12, c0s, q, kv: 13
    (2, 2): 3 + 1 + 2 + 1 + 3 + 1 + 3,           # H, det, sigma*r, cM, g, kv, diagonals: 14
}


def fp64_pipe_ops_per_element(kind: int, dim: int) -> int:
    """Operations of fp64_ops_per_element that stay on the FP64 pipe."""
    return fp64_ops_per_element(kind, dim) - INT_PIPE_OPS_PER_ELEMENT[(kind, dim)]


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    w = WORKLOAD
    # bounded sample of the same recipe per step, sized so that the whole run
    # stays near one minute of CPU time whatever K and W are (~8e6 tets in total)
    ns = int(max(4, min(64, (8e6 / (6 * (args.steps + args.warmup))) ** (1 / 3))))
    nodes, elems = mg.kuhn_cube(ns, w["jitter"], w["seed"])
    coeff = mg.log_uniform_coeff(w["seed"], elems.shape[0])
    for _ in range(args.warmup):
        oracle.assemble(w["kind"], w["dim"], nodes, elems, coeff)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.assemble(w["kind"], w["dim"], nodes, elems, coeff)
    dt = time.perf_counter() - t0
    value = args.steps * elems.shape[0] / dt / 1e6
    sample = f"{ns}^3 cubes x 6 tets ({elems.shape[0]} tets) of the same jitter/coefficient recipe per step, end to end"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "sample_tets": int(elems.shape[0])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, dev, plain_rate):
    """256 independent cubes, n ~ U{8..48} (seed 4, mesh b jittered with seed
    4000 + b), all assembled per step by one ef_batch_assemble call with the
    per-mesh buffers passed as pointer tables, captured once in a CUDA graph
    and timed as graph replays: under the two-launch schedule (element kernel
    and sum kernel over all meshes) and under the one-launch persistent
    queue (its best configuration over a small sweep). Rate = all elements of
    the batch per second, of the faster schedule. Compared with the same
    meshes as 256 separate ef_assemble calls and with one Kuhn cube of about
    the batch's element count."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    sizes = mg.batch_sizes(4, args.batch_meshes, 8, 48)
    nodes, elems, coeff = [], [], []
    for b, n in enumerate(sizes):
        nd, el = mg.kuhn_cube(int(n), 0.2, 4000 + b)
        nodes.append(torch.from_numpy(nd).to(dev))
        elems.append(torch.from_numpy(el).to(dev))
        coeff.append(torch.from_numpy(mg.log_uniform_coeff(4000 + b, el.shape[0])).to(dev))
    t0 = time.perf_counter()
    batch = ef.Batch(2, 3, [x.shape[0] for x in nodes], elems)
    plan_s = time.perf_counter() - t0
    K = [torch.empty(z, dtype=torch.float64, device=dev) for z in batch.nnz]
    M = [torch.empty(z, dtype=torch.float64, device=dev) for z in batch.nnz]
    batch.bind(nodes, coeff, K, M)
    t0 = time.perf_counter()
    tuned = batch.tune(reps=2)
    tune_s = time.perf_counter() - t0
    tabs = batch.tables(nodes, coeff, K, M)
    stream = torch.cuda.current_stream()
    T = int(sum(batch.n_elems))

    def graph_ms(steps):
        """ms per replay of a CUDA graph holding one ef_batch_assemble call."""
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            batch.assemble_tables(tabs, stream=side)
            side.synchronize()
            with torch.cuda.graph(g, stream=side):
                batch.assemble_tables(tabs, stream=side)
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        batch.check()
        del g
        return a.elapsed_time(b) / steps

    schedules = {}
    batch.set_config(two_launch=1)
    schedules["two_launch"] = {"ms_per_step": graph_ms(max(args.batch_steps // 2, 3)), "launches_per_step": 2 + (
        len(sizes) + 63) // 64, "config": batch.config()}
    best = None
    for tile in (128, 256):
        for su in (512, 2048):
            for ec in (0, 1):
                for lf in (0, 1):
                    batch.set_config(elems_per_tile=tile, sum_tile=max(su, tile), elem_ctas=ec, dynamic=1,
                                     largest_first=lf, two_launch=0, ctas_per_sm=0)
                    ms = graph_ms(3)
                    if best is None or ms < best[0]:
                        best = (ms, batch.config())
    batch.set_config(**best[1])
    schedules["persistent"] = {"ms_per_step": graph_ms(max(args.batch_steps // 2, 3)),
                               "launches_per_step": 1 + (len(sizes) + 63) // 64, "config": best[1]}
    for v in schedules.values():
        v["value"] = T / (v["ms_per_step"] / 1e3) / 1e6
        v["unit"] = UNIT
    fast = min(schedules, key=lambda k: schedules[k]["ms_per_step"])
    # the timed steps: the faster schedule, graph replays inside the NVTX range
    batch.set_config(**schedules[fast]["config"])
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        batch.assemble_tables(tabs, stream=side)
        side.synchronize()
        with torch.cuda.graph(g, stream=side):
            batch.assemble_tables(tabs, stream=side)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    _nvtx(torch, "timed")
    e0.record(stream)
    for _ in range(args.batch_steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    _nvtx(torch, None)
    batch.check()
    del g
    ms = e0.elapsed_time(e1) / args.batch_steps
    rate = T / (ms / 1e3) / 1e6
    out = {"value": rate, "unit": UNIT, "meshes": len(sizes), "elements": T, "nnz": int(sum(batch.nnz)),
           "ms_per_step": ms, "graph": True, "call": "ef_batch_assemble (per-call pointer tables)",
           "schedule": fast, "launches_per_step": schedules[fast]["launches_per_step"],
           "schedules": schedules, "persistent_vs_two_launch":
               schedules["two_launch"]["ms_per_step"] / schedules["persistent"]["ms_per_step"],
           "vs_plain": rate / plain_rate, "plain": "the single-mesh ef_assemble rate of this run",
           "tuned_config": tuned, "plan_s": plan_s, "tune_s": tune_s}
    batch.close()
    del batch
    torch.cuda.empty_cache()
    if args.no_batch_baselines:
        return out

    def timed(fn, steps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    # the same meshes as separate ef_assemble calls, one plan each, into the
    # same buffers (the default two-pass schedule: 2 launches per mesh)
    plans = [ef.Plan(2, 3, nd.shape[0], el) for nd, el in zip(nodes, elems)]

    def plain_calls():
        for pl, nd, c, k, m in zip(plans, nodes, coeff, K, M):
            ef.ef_assemble(pl.handle, nd, c, k, m, stream)

    ms_p = timed(plain_calls, max(args.batch_steps // 2, 3))
    for pl in plans:
        pl.check()
        pl.close()
    del plans
    out["separate_calls"] = {"value": T / (ms_p / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms_p,
                             "launches_per_step": 2 * len(sizes), "batched_vs": rate / (T / (ms_p / 1e3) / 1e6)}
    del K, M, nodes, elems, coeff
    torch.cuda.empty_cache()
    # one mesh of about the batch's element count (Kuhn cube, 6 n^3 tets)
    n1 = int(round((T / 6) ** (1.0 / 3.0)))
    nd1, el1 = mg.kuhn_cube(n1, 0.2, 4)
    c1 = torch.from_numpy(mg.log_uniform_coeff(4, el1.shape[0])).to(dev)
    nd1 = torch.from_numpy(nd1).to(dev)
    pl1 = ef.Plan(2, 3, nd1.shape[0], torch.from_numpy(el1).to(dev))
    K1 = torch.empty(pl1.nnz, dtype=torch.float64, device=dev)
    M1 = torch.empty_like(K1)
    ms_1 = timed(lambda: ef.ef_assemble(pl1.handle, nd1, c1, K1, M1, stream), max(args.batch_steps // 2, 3))
    pl1.check()
    T1 = el1.shape[0]
    out["one_mesh_equal_T"] = {"workload": f"ned3d_kuhn{n1}_jitter0.2", "elements": int(T1),
                               "value": T1 / (ms_1 / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms_1,
                               "batched_vs": rate / (T1 / (ms_1 / 1e3) / 1e6)}
    pl1.close()
    del K1, M1, pl1, nd1, c1
    torch.cuda.empty_cache()
    return out


def _fp64_leg(kind: int, dim: int, T: int, ms: float) -> dict:
    """An element kernel's launch against the FP64 pipe peak: by the source
    count of the operations on that pipe and by the executed FP64
    instructions; beside them all FP64 operations of the routine (products
    included, which run on the integer pipes) per second."""
    src, exe = fp64_pipe_ops_per_element(kind, dim), fp64_executed_per_element(kind, dim)
    tot = fp64_ops_per_element(kind, dim)
    peak = FP64_PEAK["T_ops_per_s"]
    a_src, a_exe = src * T / (ms / 1e3) / 1e12, exe * T / (ms / 1e3) / 1e12
    return {"ops_per_elem": src, "achieved": a_src, "peak": peak, "unit": "T fp64-pipe-ops/s", "frac": a_src / peak,
            "executed_per_elem": exe, "achieved_executed": a_exe, "frac_executed": a_exe / peak,
            "all_fp64_ops_per_elem": tot, "int_pipe_ops_per_elem": INT_PIPE_OPS_PER_ELEMENT[(kind, dim)],
            "all_fp64_ops_T_per_s": tot * T / (ms / 1e3) / 1e12,
            "ms_per_launch": ms, "peak_source": FP64_PEAK["source"]}


def _timed_calls(torch, fn, steps, stream) -> float:
    """ms per call of fn, CUDA events on the launching stream around `steps`
    calls (no per-call events inside the timed region)."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _kernel_split(ef, plan, fn, steps):
    """Per-kernel ms of ef_assemble from the library's own events
    (ef_plan_profile), recorded over `steps` further calls outside the timed
    region: their three event records per call would add host time to
    launch-bound calls."""
    plan.profile(steps)
    for _ in range(steps):
        fn()
    k1, k2, calls = plan.profile_read()
    plan.profile(0)
    return k1, k2, calls


def _two_pass_ms(ef, torch, plan, tn, tc, K, M, steps, stream) -> float:
    """ms per call of the two-pass schedule (ef_assemble_two_pass) on the same
    buffers, CUDA events on the launching stream: the tuned schedule's
    comparison."""
    for _ in range(3):
        ef.ef_assemble_two_pass(plan.handle, tn, tc, K, M, stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ef.ef_assemble_two_pass(plan.handle, tn, tc, K, M, stream)
    b.record(stream)
    torch.cuda.synchronize()
    plan.check()
    return a.elapsed_time(b) / steps


def run_rt0(args, dev, peaks):
    """The two RT0 workloads: 3D RT0 on the 128^3 cube (12,582,912 tets,
    jitter 0.2h seed 3, log-uniform coefficient; the large, memory-heavy case)
    and 2D RT0 on the 32^2 square (2,048 triangles, unit coefficient, no
    jitter; launch-latency-bound). Same ef_assemble call, tuned, per-kernel
    CUDA events, HBM fraction on the algorithmic bytes per call."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    out = {}
    for name, dim, n, jitter, seed, unit in ((f"rt0_3d_kuhn{args.rt0_cube}_jitter0.2", 3, args.rt0_cube, 0.2, 3,
                                              False),
                                             ("rt0_2d_square32", 2, 32, 0.0, 0, True)):
        if dim == 3:
            nodes, elems = mg.kuhn_cube(n, jitter, seed)
        else:
            nodes, elems = mg.kuhn_square(n)
        coeff = None if unit else mg.log_uniform_coeff(seed, elems.shape[0])
        tn = torch.from_numpy(nodes).to(dev)
        tc = None if coeff is None else torch.from_numpy(coeff).to(dev)
        plan = ef.Plan(1, dim, nodes.shape[0], torch.from_numpy(elems).to(dev))
        K = torch.empty(plan.nnz, dtype=torch.float64, device=dev)
        M = torch.empty_like(K)
        tuned = plan.tune(tn, tc, K, M, reps=3)
        steps = args.rt0_steps if dim == 3 else 10 * args.rt0_steps
        stream = torch.cuda.current_stream()
        for _ in range(3):
            ef.ef_assemble(plan.handle, tn, tc, K, M, stream)
        torch.cuda.synchronize()
        call = lambda: ef.ef_assemble(plan.handle, tn, tc, K, M, stream)
        ms = _timed_calls(torch, call, steps, stream)
        k1, k2, calls = _kernel_split(ef, plan, call, steps)
        plan.check()
        T, V, nnz = elems.shape[0], nodes.shape[0], plan.nnz
        alg = (4 * (dim + 1) + (0 if coeff is None else 8)) * T + 8 * dim * V + 16 * nnz
        gbs = alg / (ms / 1e3) / 1e9
        out[name] = {"value": T / (ms / 1e3) / 1e6, "unit": UNIT, "elements": int(T), "nnz": int(nnz),
                     "ms_per_step": ms, "tuned_choice": tuned,
                     "kernels_ms": {"first": k1 / max(calls, 1), "second": k2 / max(calls, 1)},
                     "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                             "algorithmic_bytes_per_step": int(alg), "bytes_per_elem": alg / T}}
        if tuned == 0 and calls:
            # the element kernel of the two-pass schedule against the FP64 pipe
            out[name]["fp64_element_kernel"] = _fp64_leg(1, dim, T, k1 / calls)
        else:
            tp = _two_pass_ms(ef, torch, plan, tn, tc, K, M, steps, stream)
            out[name]["two_pass"] = {"ms_per_step": tp, "tuned_speedup": tp / ms}
        plan.close()
        del K, M
        torch.cuda.empty_cache()
    return out


def run_lshape(args, dev, peaks):
    """The 2D assembly of Table 1: RT0 and Nedelec K and M on the L-shaped
    domain (0,1)^2 minus (1/2,1)^2 at level L (6 4^L triangles; L = 11:
    25,165,824 triangles, 37,756,928 edges, the matrix size Table 1 prints),
    unit coefficient as in the paper, no jitter. Same tuned ef_assemble call
    and per-kernel CUDA events as the other legs."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.lshape(args.lshape_level)
    tn = torch.from_numpy(nodes).to(dev)
    te = torch.from_numpy(elems).to(dev)
    T, V = elems.shape[0], nodes.shape[0]
    del elems
    out = {"workload": f"lshape2d_L{args.lshape_level}", "elements": int(T)}
    stream = torch.cuda.current_stream()
    for kind, name in ((1, "rt0"), (2, "nedelec")):
        plan = ef.Plan(kind, 2, V, te)
        K = torch.empty(plan.nnz, dtype=torch.float64, device=dev)
        M = torch.empty_like(K)
        tuned = plan.tune(tn, None, K, M, reps=3)
        steps = args.rt0_steps
        for _ in range(3):
            ef.ef_assemble(plan.handle, tn, None, K, M, stream)
        torch.cuda.synchronize()
        call = lambda: ef.ef_assemble(plan.handle, tn, None, K, M, stream)
        _nvtx(torch, "timed")
        ms = _timed_calls(torch, call, steps, stream)
        _nvtx(torch, None)
        k1, k2, calls = _kernel_split(ef, plan, call, steps)
        plan.check()
        alg = 12 * T + 16 * V + 16 * plan.nnz
        gbs = alg / (ms / 1e3) / 1e9
        leg = {"value": T / (ms / 1e3) / 1e6, "unit": UNIT, "dofs": int(plan.n_dofs), "nnz": int(plan.nnz),
               "ms_per_step": ms, "tuned_choice": tuned,
               "kernels_ms": {"first": k1 / max(calls, 1), "second": k2 / max(calls, 1)},
               "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                       "algorithmic_bytes_per_step": int(alg), "bytes_per_elem": alg / T}}
        if tuned == 0 and calls:
            leg["fp64_element_kernel"] = _fp64_leg(kind, 2, T, k1 / calls)
        else:
            tp = _two_pass_ms(ef, torch, plan, tn, None, K, M, steps, stream)
            leg["two_pass"] = {"ms_per_step": tp, "tuned_speedup": tp / ms}
        out[name] = leg
        plan.close()
        del K, M
        torch.cuda.empty_cache()
    return out


def run_integration(args, dev, peaks):
    """Vectorised integration (Sec. 3.1): squared L2 error ||E - v_h||^2 of an
    affine field E against the Nedelec function of a random DOF vector on the
    64^3 workload, 27-point rule (n = 3), E given at the points (point-major,
    resident in HBM). Timed: ef_norm_l2 (per-element norms + fixed-order total)."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    w = WORKLOAD
    nodes, elems, _ = _workload()
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(w["kind"], w["dim"], nodes.shape[0], torch.from_numpy(elems).to(dev))
    n = 3
    x = plan.quad_points(tn, n)
    A = torch.from_numpy(mg.normal(7, 12, 9).reshape(3, 3)).to(dev)
    f = (torch.einsum("qec,rc->qer", x, A) + 1.0).contiguous()
    del x
    v = torch.from_numpy(mg.normal(7, mg.STREAM_V, plan.n_dofs)).to(dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        plan.norm_l2(tn, f, n, v=v, per_element=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = args.integration_steps
    _nvtx(torch, "timed")
    a.record(stream)
    for _ in range(steps):
        plan.norm_l2(tn, f, n, v=v, per_element=True)
    b.record(stream)
    torch.cuda.synchronize()
    _nvtx(torch, None)
    plan.check()
    ms = a.elapsed_time(b) / steps
    T, V = elems.shape[0], nodes.shape[0]
    nq = n ** 3
    alg = (nq * 3 * 8 + 16 + 24 + 1 + 8) * T + 24 * V + 8 * plan.n_dofs
    gbs = alg / (ms / 1e3) / 1e9
    out = {"value": T / (ms / 1e3) / 1e6, "unit": UNIT, "workload": w["name"] + "_l2error_q27",
           "elements": int(T), "points_per_element": nq, "ms_per_step": ms,
           "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                   "algorithmic_bytes_per_step": int(alg), "bytes_per_elem": alg / T}}
    plan.close()
    del f
    torch.cuda.empty_cache()
    return out


def run_majorant(args, dev, peaks, dim=2):
    """The library's share of the majorant minimisation (Sec. 4.1, Algorithm 1)
    with the 16-point (2D) or 64-point (3D) rule (n = 4), on the unit square
    with 2 m^2 triangles (m = 4096: Table 3's largest mesh, 33,554,432
    triangles) or the unit cube with 6 c^3 Kuhn tetrahedra (c = 96: the size
    of Table 4's largest mesh, 5,308,416 tetrahedra): RT0 K and M, the load
    vectors int grad v . phi (ef_load_vector) and int f div phi
    (ef_load_derivative), the error ||grad(u - v)||^2, and for each of the 3
    iterations the tables print ||grad v - y||^2 (ef_norm_l2) and
    ||div y + f||^2 (ef_norm_l2_derivative). The host solves are not part of
    it; grad v (per element) and y are seeded normal values drawn on the
    device (they do not change the work), f and grad u are the bubble
    problem's. Rate = elements / time of all these calls (one step)."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    if dim == 2:
        m = args.majorant_m
        nodes, elems = mg.kuhn_square(m)
        name = f"rt2d_square{m}_majorant_q16"
    else:
        m = args.majorant_cube
        nodes, elems = mg.kuhn_cube(m)
        name = f"rt3d_kuhn{m}_majorant_q64"
    T, V = elems.shape[0], nodes.shape[0]
    tn = torch.from_numpy(nodes).to(dev)
    plan = ef.Plan(1, dim, V, torch.from_numpy(elems).to(dev))
    del elems
    n = 4
    nq = n ** dim
    x = plan.quad_points(tn, n)                                       # [nq, T, dim]
    a = x * (x - 1.0)
    # -f = 2 sum_i prod_{j != i} a_j;  (grad u)_i = (2 x_i - 1) prod_{j != i} a_j
    others = [torch.prod(torch.cat([a[..., :c], a[..., c + 1:]], -1), -1) for c in range(dim)]
    mf = (2.0 * sum(others)).unsqueeze(-1).contiguous()
    gu = torch.stack([(2.0 * x[..., c] - 1.0) * others[c] for c in range(dim)], -1)
    del x, a, others
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    gvt = torch.randn((T, dim), generator=gen, dtype=torch.float64, device=dev)
    gv = gvt.unsqueeze(0).expand(nq, T, dim).contiguous()
    gerr = (gu - gv).contiguous()
    del gu, gvt
    f = (-mf).contiguous()
    y = torch.randn(plan.n_dofs, generator=gen, dtype=torch.float64, device=dev)
    K = torch.empty(plan.nnz, dtype=torch.float64, device=dev)
    M = torch.empty_like(K)
    iters = 3

    def step():
        plan.assemble(tn, None, K, M)
        plan.load_vector(tn, gv, n)
        plan.load_derivative(tn, f, n)
        plan.norm_l2(tn, gerr, n)
        for _ in range(iters):
            plan.norm_l2(tn, gv, n, v=y)
            plan.norm_l2_derivative(tn, mf, n, v=y)

    stream = torch.cuda.current_stream()
    for _ in range(3):
        step()
    plan.check()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = args.majorant_steps
    _nvtx(torch, "timed")
    a0.record(stream)
    for _ in range(steps):
        step()
    a1.record(stream)
    torch.cuda.synchronize()
    _nvtx(torch, None)
    plan.check()
    ms = a0.elapsed_time(a1) / steps
    # algorithmic bytes of one step: per element the values at the points each
    # call reads (8 B per component and point), connectivity (4 (dim + 1) B)
    # and the gathered coordinates (8 dim V / T) per call; the CSR values K, M
    # (16 nnz); the local load entries written and re-read and the load vectors
    # written; DOF ids, signs and the gathered y of the norms with y
    nloc = dim + 1 if dim == 3 else 3
    calls = 4 + 2 * iters
    per_pts = nq * 8 * (dim + 1 + dim + iters * (dim + 1))
    alg = (per_pts + calls * 4 * (dim + 1)) * T + calls * 8 * dim * V + 16 * plan.nnz \
        + 2 * (2 * nloc * 8 * T + 8 * plan.n_dofs) + 2 * iters * (4 * nloc + 1 + nloc * 8) * T
    gbs = alg / (ms / 1e3) / 1e9
    out = {"value": T / (ms / 1e3) / 1e6, "unit": UNIT, "workload": name,
           "elements": int(T), "dofs": int(plan.n_dofs), "iterations": iters, "points_per_element": nq,
           "ms_per_step": ms,
           "calls_per_step": {"ef_assemble": 1, "ef_load_vector": 1, "ef_load_derivative": 1,
                              "ef_norm_l2": 1 + iters, "ef_norm_l2_derivative": iters},
           "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                   "algorithmic_bytes_per_step": int(alg), "bytes_per_elem": alg / T}}
    plan.close()
    del gv, gerr, mf, f, K, M
    torch.cuda.empty_cache()
    return out


def run_adjoint(args, dev):
    """Adjoint of u^T K u + v^T M v on the 96^3 Nedelec workload (5,308,416
    tets, seed 5), against plain ef_assemble on the same mesh."""
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    nodes, elems = mg.kuhn_cube(args.adjoint_cube, 0.2, 5)
    coeff = mg.log_uniform_coeff(5, elems.shape[0])
    tn, tc = torch.from_numpy(nodes).to(dev), torch.from_numpy(coeff).to(dev)
    plan = ef.Plan(2, 3, nodes.shape[0], torch.from_numpy(elems).to(dev))
    u = torch.from_numpy(mg.normal(5, mg.STREAM_U, plan.n_dofs)).to(dev)
    v = torch.from_numpy(mg.normal(5, mg.STREAM_V, plan.n_dofs)).to(dev)
    J = torch.empty(1, dtype=torch.float64, device=dev)
    gx = torch.empty_like(tn)
    gs = torch.empty_like(tc)
    K = torch.empty(plan.nnz, dtype=torch.float64, device=dev)
    M = torch.empty_like(K)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _nvtx(torch, "timed")
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        _nvtx(torch, None)
        return a.elapsed_time(b) / steps

    ms_adj = timed(lambda: ef.ef_adjoint(plan.handle, tn, tc, u, v, J, gx, gs, stream), args.adjoint_steps)
    ms_asm = timed(lambda: ef.ef_assemble(plan.handle, tn, tc, K, M, stream), args.adjoint_steps)
    plan.check()
    T = elems.shape[0]
    ops = ADJOINT_FP64_PIPE_OPS_PER_TET * T
    out = {"value": T / (ms_adj / 1e3) / 1e6, "unit": UNIT, "workload": f"ned3d_kuhn{args.adjoint_cube}_jitter0.2",
           "elements": int(T), "ms_per_step": ms_adj,
           "plain_same_mesh": {"value": T / (ms_asm / 1e3) / 1e6, "ms_per_step": ms_asm},
           "vs_plain": ms_asm / ms_adj,
           "fp64": {"ops_per_elem": ADJOINT_FP64_PIPE_OPS_PER_TET, "achieved": ops / (ms_adj / 1e3) / 1e12,
                    "peak": FP64_PEAK["T_ops_per_s"], "unit": "T fp64-pipe-ops/s",
                    "all_fp64_ops_per_elem": ADJOINT_FP64_OPS_PER_TET,
                    "int_pipe_ops_per_elem": ADJOINT_INT_PIPE_OPS_PER_TET,
                    "all_fp64_ops_T_per_s": ADJOINT_FP64_OPS_PER_TET * T / (ms_adj / 1e3) / 1e12,
                    "frac": ops / (ms_adj / 1e3) / 1e12 / FP64_PEAK["T_ops_per_s"],
                    "peak_source": FP64_PEAK["source"],
                    "executed_per_elem": ADJOINT_FP64_EXECUTED_PER_TET,
                    "frac_executed": ADJOINT_FP64_EXECUTED_PER_TET * T / (ms_adj / 1e3) / 1e12
                    / FP64_PEAK["T_ops_per_s"],
                    "note": "whole ef_adjoint call (element kernel ~92 % of it)"}}
    plan.close()
    return out


ALL_CORES_CUBE = 48   # cubes per axis of each process's sample in the all-cores oracle run


def _oracle_process(barrier, n):
    """One process of the all-cores oracle run: its own n^3 sample of the
    workload recipe, timed between a start aligned with the other processes
    and its end (wall clock)."""
    import oracle

    nodes, elems = mg.kuhn_cube(n, WORKLOAD["jitter"], WORKLOAD["seed"])
    coeff = mg.log_uniform_coeff(WORKLOAD["seed"], elems.shape[0])
    oracle.assemble(WORKLOAD["kind"], WORKLOAD["dim"], *mg.kuhn_cube(2, 0.0, 0))   # load the library
    barrier.wait()
    t0 = time.time()
    oracle.assemble(WORKLOAD["kind"], WORKLOAD["dim"], nodes, elems, coeff)
    return elems.shape[0], t0, time.time()


def _oracle_all_cores(cores):
    """The oracle as it stands on every host core: `cores` independent
    processes (spawned, so none inherits the parent's CUDA context), each
    assembling its own sample; rate = all their elements / the time from the
    common start to the last end."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        barrier = manager.Barrier(cores)
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_process, [(barrier, ALL_CORES_CUBE)] * cores)
    T = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": T / wall / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each its own {ALL_CORES_CUBE}^3 x 6 tets ({res[0][0]} tets) of the "
                      f"workload recipe, topology + pattern + quadrature assembly, {wall:.1f} s"}


def cpu_baseline():
    """The oracle as it stands, timed on this host: the full workload, one
    thread; and on every host core (independent processes, one sample each)."""
    import oracle

    oracle.build()
    nodes, elems, coeff = _workload()
    t0 = time.perf_counter()
    oracle.assemble(WORKLOAD["kind"], WORKLOAD["dim"], nodes, elems, coeff)
    dt = time.perf_counter() - t0
    out = {"value": elems.shape[0] / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the full workload ({elems.shape[0]} tets), topology + pattern + quadrature assembly, "
                     f"single thread, {dt:.1f} s"}
    cores = os.cpu_count() or 1
    if cores > 1:
        try:
            out["all_cores"] = _oracle_all_cores(cores)
        except Exception as exc:   # a host that cannot start the processes: report why
            out["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"}
    return out


def run_gpu(args):
    import torch

    from paper_1409_4618_gb300 import edgefem as ef

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.only:
        # one workload by itself (for profiling): its JSON object on one line
        dev = torch.device("cuda", local)
        peaks, _ = _peaks()
        legs = {"batched": lambda: run_batched(args, dev, float("nan")), "adjoint": lambda: run_adjoint(args, dev),
                "rt0": lambda: run_rt0(args, dev, peaks), "integration": lambda: run_integration(args, dev, peaks),
                "majorant": lambda: run_majorant(args, dev, peaks), "lshape": lambda: run_lshape(args, dev, peaks),
                "majorant3d": lambda: run_majorant(args, dev, peaks, dim=3)}
        print(json.dumps({"leg": args.only, **legs[args.only]()}), flush=True)
        return 0
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if args.no_fp64_probe:
        probe = {"peak_T_ops_per_s": FP64_PEAK_TOPS, "element_mix_T_ops_per_s": FP64_PEAK_TOPS,
                 "clocks": {"sm_mhz": None}, "skipped": "--no-fp64-probe (nominal peak)"}
    else:
        probe = run_fp64_probe(local)
        FP64_PEAK.update(T_ops_per_s=probe["peak_T_ops_per_s"], source="measured (bench fp64 leg: ef_fp64_probe DFMA)")
    nodes, elems, coeff = _workload()
    w = WORKLOAD
    tn = torch.from_numpy(nodes).to(dev)
    tc = torch.from_numpy(coeff).to(dev)
    te = torch.from_numpy(elems).to(dev)
    # a small plan first, so that module loading is not in the plan-build time
    _, small = mg.kuhn_cube(2, 0.0, 0)
    ef.Plan(w["kind"], w["dim"], 27, torch.from_numpy(small).to(dev)).close()
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    plan = ef.Plan(w["kind"], w["dim"], nodes.shape[0], te)    # topology, pattern, work order (synchronises)
    plan_ms = (time.perf_counter() - t_plan) * 1e3
    T, V, nnz = elems.shape[0], nodes.shape[0], plan.nnz
    K = torch.empty(nnz, dtype=torch.float64, device=dev)
    M = torch.empty(nnz, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    path = args.path
    tuned = None
    if path.startswith("blocked"):
        plan.set_block(int(path[len("blocked"):]))
    elif path.startswith("fused"):
        plan.set_fused(tn, int(path[len("fused"):]))
    elif path == "default":
        tuned = plan.tune(tn, tc, K, M, reps=5)      # library autotuner: pipeline chunks / element-block

    def step():
        if path == "two_pass":
            ef.ef_assemble_two_pass(plan.handle, tn, tc, K, M, stream)
        else:
            ef.ef_assemble(plan.handle, tn, tc, K, M, stream)

    for _ in range(args.warmup):
        step()
    plan.check()
    torch.cuda.synchronize()

    # ---- timed region: K steps, device time by CUDA events on the launching stream;
    # the library records its own per-kernel events on that stream for the same K calls
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if path != "two_pass":
        plan.profile(args.steps)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        _nvtx(torch, "timed")
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        _nvtx(torch, None)
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    plan.check()
    k_first, k_second, k_calls = plan.profile_read() if path != "two_pass" else (0.0, 0.0, 0)
    plan.profile(0)
    ms, units = job_timing(ms, T * args.steps, dist, dev)
    ms_step = ms / args.steps
    value = units / (ms / 1e3) / 1e6

    # ---- end to end through the host-buffer C-ABI call
    hn = torch.from_numpy(nodes).pin_memory()
    hc = torch.from_numpy(coeff).pin_memory()
    hK = torch.empty(nnz, dtype=torch.float64, pin_memory=True)
    hM = torch.empty(nnz, dtype=torch.float64, pin_memory=True)
    # (each call synchronises; per-step CUDA events, median over the steps,
    # max over ranks)
    e2e_steps = max(3, min(args.steps, 20))
    plan.assemble_host(hn, hc, hK, hM)
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(e2e_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.assemble_host(hn, hc, hK, hM)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms, e2e_units = job_timing(statistics.median(e2e_times), T, dist, dev)
    e2e = {"value": e2e_units / (e2e_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": e2e_ms,
           "steps": e2e_steps, "timing": "median of per-step CUDA events around ef_assemble_host",
           "h2d_bytes_per_step": int(hn.numel() * 8 + hc.numel() * 8),
           "d2h_bytes_per_step": int(2 * nnz * 8)}

    # ---- rooflines: the dominant kernel (per-launch CUDA events), and HBM for the whole step
    peaks, src = _peaks()
    alg_bytes = 16 * T + 8 * T + 8 * w["dim"] * V + 16 * nnz
    achieved_gbs = alg_bytes / (ms_step / 1e3) / 1e9
    info = plan.info()
    U = info["n_upper"]
    n_pairs = info["n_contrib"] // T
    elem_ops = T * fp64_pipe_ops_per_element(w["kind"], w["dim"])
    elem_ops_all = T * fp64_ops_per_element(w["kind"], w["dim"])
    sum_ops = 2 * (T * n_pairs - U)
    sum_bytes = 2 * n_pairs * 8 * T + 14 * U + 16 * nnz   # list, indices + store orders, CSR values
    if k_calls > 0 and info["fused_block"] == 0 and info["assemble_launches"] == 2:
        ms_e, ms_s = k_first / k_calls, k_second / k_calls
        kernels = {"element": {"ms_per_launch": ms_e, "share": ms_e / (ms_e + ms_s)},
                   "sum": {"ms_per_launch": ms_s, "share": ms_s / (ms_e + ms_s),
                           "achieved_gbs": sum_bytes / (ms_s / 1e3) / 1e9,
                           "frac_hbm": sum_bytes / (ms_s / 1e3) / 1e9 / peaks["hbm_gbs"],
                           "algorithmic_bytes": int(sum_bytes)}}
        dom_name, dom_ms, dom_ops = "k_element_local (two-pass element kernel)", ms_e, elem_ops
        traffic = (None if ELEMENT_KERNEL_DRAM_BYTES_PER_TET is None
                   else ELEMENT_KERNEL_DRAM_BYTES_PER_TET * T)
    else:
        one = k_first / k_calls if k_calls else ms_step
        kernels = {"step": {"ms_per_launch": one}}
        dom_name, dom_ms, dom_ops, traffic = "ef_assemble (" + path + ")", one if k_calls else ms_step, \
            elem_ops + sum_ops, None
    achieved_ops = dom_ops / (dom_ms / 1e3) / 1e12
    peak = probe["peak_T_ops_per_s"]
    exec_ops = sum(ELEMENT_KERNEL_FP64_MIX.values()) * T if dom_ops == elem_ops else None
    roofline = {
        "bound": "alu", "unit": "T fp64-pipe-ops/s", "achieved": achieved_ops, "peak": peak,
        "frac": achieved_ops / peak, "traffic": traffic,
        "peak_source": ("measured (bench fp64 leg: ef_fp64_probe DFMA lane-ops/s on this GPU, "
                        f"median SM clock {probe['clocks'].get('sm_mhz')} MHz during the probe)"
                        if "skipped" not in probe else "nominal (" + probe["skipped"] + ")"),
        "peak_nominal": FP64_PEAK_TOPS,
        "peak_nominal_source": f"{SMS} SMs x {FP64_PER_CLK_PER_SM} FP64 ops/clk/SM x {SM_MAX_MHZ} MHz",
        "kernel": dom_name, "ms_per_launch": dom_ms,
        "fp64_ops_per_launch": int(dom_ops), "fp64_ops_per_elem": dom_ops / T,
        "fp64_ops_source": ("counted from the source (csrc/ef_element.cuh): the operations on the FP64 pipe; "
                            "the products run on the integer pipes (csrc/ef_intmul.cuh)"),
        "all_fp64_ops": (None if dom_ops != elem_ops else
                         {"per_elem": elem_ops_all / T,
                          "int_pipe_per_elem": INT_PIPE_OPS_PER_ELEMENT[(w["kind"], w["dim"])],
                          "T_per_s": elem_ops_all / (dom_ms / 1e3) / 1e12,
                          "of_fp64_pipe_peak": elem_ops_all / (dom_ms / 1e3) / 1e12 / peak}),
        "executed": (None if exec_ops is None else
                     {"fp64_ops_per_elem": exec_ops / T, "source": "ncu sass FP64 instruction counters",
                      "achieved": exec_ops / (dom_ms / 1e3) / 1e12,
                      "frac": exec_ops / (dom_ms / 1e3) / 1e12 / peak,
                      "frac_of_mix_peak": exec_ops / (dom_ms / 1e3) / 1e12 / probe["element_mix_T_ops_per_s"]}),
        "fp64_probe": probe,
        "kernels": kernels,
        "hbm_step": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved_gbs / peaks["hbm_gbs"],
                     "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_step": int(alg_bytes), "bytes_per_elem": alg_bytes / T},
    }
    info = plan.info()
    launches = (2 if path == "two_pass" else info["assemble_launches"]) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "elements": T, "nodes": V, "dofs": plan.n_dofs, "nnz": nnz,
                   "plan_build_ms": plan_ms,
                   "path": path, "tuned_choice": tuned, "plan": info, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": f"no flush: each step moves {alg_bytes / 1e6:.0f} MB (algorithmic) > 129 MB L2"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }
    plan.close()
    if not args.no_batched:
        line["batched"] = run_batched(args, dev, value / ws)
    if not args.no_adjoint:
        line["adjoint"] = run_adjoint(args, dev)
    if not args.no_rt0:
        line["rt0"] = run_rt0(args, dev, peaks)
    if not args.no_integration:
        line["integration"] = run_integration(args, dev, peaks)
    if not args.no_majorant:
        line["majorant"] = run_majorant(args, dev, peaks)
        line["majorant3d"] = run_majorant(args, dev, peaks, dim=3)
    if not args.no_lshape:
        line["lshape"] = run_lshape(args, dev, peaks)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--path", default="default",
                    choices=["default", "two_pass", "blocked128", "blocked256", "fused128", "fused256"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-rt0", action="store_true")
    ap.add_argument("--only", choices=["batched", "adjoint", "rt0", "integration", "majorant", "majorant3d",
                                       "lshape"],
                    help="run one of the other workloads by itself (profiling)")
    ap.add_argument("--adjoint-cube", type=int, default=96)
    ap.add_argument("--no-integration", action="store_true")
    ap.add_argument("--integration-steps", type=int, default=50)
    ap.add_argument("--no-majorant", action="store_true")
    ap.add_argument("--majorant-m", type=int, default=4096,
                    help="squares per axis of the majorant workload (2 m^2 triangles)")
    ap.add_argument("--majorant-steps", type=int, default=5)
    ap.add_argument("--majorant-cube", type=int, default=96,
                    help="cubes per axis of the 3D majorant workload (6 c^3 tetrahedra)")
    ap.add_argument("--no-lshape", action="store_true")
    ap.add_argument("--lshape-level", type=int, default=11,
                    help="level of the 2D L-shaped workload (6 4^L triangles)")
    ap.add_argument("--rt0-steps", type=int, default=20)
    ap.add_argument("--rt0-cube", type=int, default=128, help="cubes per axis of the 3D RT0 workload")
    ap.add_argument("--no-fp64-probe", action="store_true",
                    help="skip the FP64 throughput probe (profiling runs); rooflines then use the nominal peak")
    ap.add_argument("--batch-meshes", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-batch-baselines", action="store_true",
                    help="skip the batch's comparisons (separate calls, one mesh of equal size)")
    ap.add_argument("--adjoint-steps", type=int, default=50)
    ap.add_argument("--cube", type=int, default=64,
                    help="cubes per axis of the single-mesh workload (smaller values: profiling cases)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.cube != WORKLOAD["n"]:
        if args.cube < 4:
            ap.error("--cube must be >= 4")
        WORKLOAD.update(n=args.cube, name=f"ned3d_kuhn{args.cube}_jitter0.2")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
