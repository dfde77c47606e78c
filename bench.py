#!/usr/bin/env python3
"""Benchmark: SP2 spectral projection driven by SpAMM on one GB300.

Workload (the large single SP2): the N = 65536 tight-binding Hamiltonian on
Morton-ordered 3-D three-site clusters, h_ij = -exp(-r_ij / 1.0 A) cut at
1e-12, on-site -/+2 by site parity, Ne = N/2, Gershgorin start, tau = 1e-8,
leaf 32.  F is stored sparsely (leaves with ||leaf||_F <= 1e-12 are not
stored); the iterates use the dense leaf grid.  One step is one complete
SP2 solve: norm quadtree, culling, leaf products and the fused SP2 update
for every iteration until the stopping rule fires.

Printed metric: SP2 solve time and SpAMM leaf throughput, mixed precision vs
plain FP64.  `value` is the useful SpAMM leaf throughput of the mixed solve,
2 b^3 x (surviving leaf triples summed over iterations) / solve time, in
TFLOP/s; `ms_per_step` is the mixed SP2 solve time.  The timed steps use the
mixed-precision leaf products (exact BF16 slices on the tensor cores, FP64
norms, traces and updates); the same workload is then solved with FP64 leaf
products, and the line reports that solve time, the speedup and
||P_mixed - P_FP64||_F.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec ozaki|fp64] [--slices S] [--bench-n N]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)
  python bench.py --study precision [--n 16384] [--taus ...]   (modes vs FP64 SP2)
  python bench.py --study batch [--batch 64] [--batch-prec tf32] (many SpAMMs, one launch)
  python bench.py --study large [--n-large 65536]   (one large SP2, mixed vs FP64)
  python bench.py --study spamm [--spamm-n 1024]     (single products, time per product)

N > 1 runs independent replicas (one solve per GPU); without torchrun in
the environment, `--gpus N` starts the N ranks itself through
torch.distributed.run.  value = all ranks' useful FLOPs / the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "sp2_tb_hamiltonian_large", "n": 65536, "leaf": 32, "tau": 1e-8,
            "ne": 32768, "decay_A": 1.0, "onsite": 2.0, "cut": 1e-12, "drop": 1e-12,
            "storage": "F: sparse leaves (||leaf||_F > 1e-12 stored); X, X^2: dense leaf grid",
            "start": "gershgorin", "stop": "trace+idempotency or stagnation"}
METRIC = "SP2 solve time & SpAMM leaf TFLOP/s, mixed vs FP64 plain, at ||ΔP||_F≤1e-6"
UNIT = "TFLOP/s"
L2_BYTES = 129 * 1024 * 1024
# Principal block of the Hamiltonian that the CPU oracle solves as its
# bounded sample (one SP2 iteration): all cores / one core / reference arm.
CPU_SAMPLE_N = 16384
CPU_SAMPLE_N_ONE_CORE = 4096
REF_SAMPLE_N = 8192
# DRAM bytes (read + write) per launch of the tensor-core leaf-product kernel
# on this workload (mean over the launches of one solve) from an ncu capture,
# with the SHA-256 prefix of the kernel source it was taken on: the figure is
# reported only while tc_kernel.cuh is unchanged.
TC_TRAFFIC = {"source_sha256_16": "6ca06abd3c613e01", "bytes_per_launch": 17.86e9}


def _tc_traffic():
    src = os.path.join(ROOT, "paper_1403_7458_gb300", "csrc", "tc_kernel.cuh")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if TC_TRAFFIC["source_sha256_16"] == sha:
        return TC_TRAFFIC["bytes_per_launch"]
    return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_peak_tflops():
    """FP64 FMA peak: 152 SMs x 2 DFMA/clk/SM x 2 FLOP x 2.07 GHz = 1.26
    TFLOP/s (the nominal 1.25 TFLOP/s FP64 rate at the maximum SM clock)."""
    return 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi's start-up (NVML initialisation) must not overlap the
            # timed region: wait for its first sample, count only later ones
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 10:
                time.sleep(0.01)
            self.start = len(self.lines)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken inside the region (the last one before it if none)
        for ln in (self.lines[self.start:] or self.lines[-1:]):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_ours(args):
    import torch
    from paper_1403_7458_gb300 import spamm, synth

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    spamm.load()
    prec = spamm.OZAKI_BF16 if args.prec == "ozaki" else spamm.FP64
    slices = args.slices if prec == spamm.OZAKI_BF16 else 0
    n, b, tau = args.bench_n, WORKLOAD["leaf"], WORKLOAD["tau"]
    ne = n // 2
    decay, drop = WORKLOAD["decay_A"], WORKLOAD["drop"]
    gib = lambda x: x / 2.0 ** 30
    t_gen = time.perf_counter()
    h = synth.tb_hamiltonian_torch(n, seed=rank, decay=decay)   # built on the device
    F = spamm.tree_build(h, leaf=b, drop=drop)                  # sparse leaf storage
    torch.cuda.synchronize()
    # host copy of F for the end-to-end leg (pinned: its H2D is timed there)
    # and the CPU baseline's sample
    e2e_steps = min(args.steps, args.e2e_steps)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    h_pin = None
    if e2e_steps > 0 or want_cpu:
        h_pin = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        h_pin.copy_(h)
    del h
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t_gen
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    P = None

    def solve(timing=False, p=prec, sl=slices, out=None):
        return spamm.sp2_solve(F, ne, tau, P=out, prec=p, slices=sl, timing=timing)

    for _ in range(args.warmup):  # same settings as the timed steps
        P, _ = solve(timing=True, out=P)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM ----
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flops = tflops = gemm_ms = cull_ms = upd_ms = 0.0
    iters = launches = 0
    step_ms = []
    with ClockSampler(local) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        total_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()                       # evict L2 between steps
            ev0.record(stream)
            P, rep = solve(timing=True, out=P)
            ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1)
            step_ms.append(ms)
            total_ms += ms
            flops += rep["flops_useful"]
            tflops += rep["flops_tensor"]
            gemm_ms += rep["ms_gemm"]
            cull_ms += rep["ms_cull"]
            upd_ms += rep["ms_update"]
            iters += rep["iters"]
            launches += rep["launches"]
        torch.cuda.synchronize()
        _barrier(world)
    clocks = clk.summary()
    t_max = reduce_max_over_ranks(total_ms, world, dev)
    flops_all = reduce_sum_over_ranks(flops, world, dev)
    value = flops_all / (t_max * 1e-3) / 1e12
    mem_free_mixed = gib(torch.cuda.mem_get_info()[0])
    main_rep = rep
    spamm.release_scratch(P)

    # ---- the same workload with FP64 leaf products (one solve) ----
    fp64 = None
    if prec != spamm.FP64 and not args.no_fp64_leg:
        flush.zero_()
        ev0.record(stream)
        P64, r64 = solve(p=spamm.FP64, sl=0, timing=True)
        ev1.record(stream)
        ev1.synchronize()
        f_ms = ev0.elapsed_time(ev1)
        spamm.release_scratch(P64)
        spamm.trim()
        d = spamm.to_dense(P)
        trace_err = abs(torch.trace(d).item() - ne)
        p64 = spamm.to_dense(P64)
        P64.free()
        d.sub_(p64)                             # P_mixed - P_FP64, in place
        del p64
        dP = torch.linalg.norm(d).item()
        del d
        torch.cuda.empty_cache()
        fp64 = {"solve_ms": f_ms, "iters": r64["iters"], "stop_reason": r64["stop_reason"],
                "symmetric": r64["symmetric"], "speedup_mixed_vs_fp64": f_ms / (t_max / args.steps),
                "dP_fro_mixed_vs_fp64": dP, "value_fp64": r64["flops_useful"] / (f_ms * 1e-3) / 1e12,
                "ms_cull": r64["ms_cull"], "ms_gemm": r64["ms_gemm"], "ms_update": r64["ms_update"],
                "gemm_useful_tflops": r64["flops_useful"] / (r64["ms_gemm"] * 1e-3) / 1e12,
                "gemm_executed_tflops": r64["flops_tensor"] / (r64["ms_gemm"] * 1e-3) / 1e12,
                "gemm_frac_of_fp64_peak": r64["flops_tensor"] / (r64["ms_gemm"] * 1e-3) / 1e12 / fp64_peak_tflops()}
    else:
        spamm.trim()
        d = spamm.to_dense(P)
        trace_err = abs(torch.trace(d).item() - ne)
        del d
        torch.cuda.empty_cache()
    P.free()
    spamm.trim()

    # ---- end to end through the C ABI with host buffers ----
    p_pin = torch.empty((n, n), dtype=torch.float64, pin_memory=True) if e2e_steps > 0 else None
    e2e_flops = 0.0
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        F2 = spamm.tree_build(h_pin.numpy(), leaf=b, drop=drop)   # host pointer: H2D inside
        P2, rep2 = spamm.sp2_solve(F2, ne, tau, prec=prec, slices=slices)
        spamm.to_dense(P2, out=p_pin.numpy())                     # host pointer: D2H inside
        e2e_flops += rep2["flops_useful"]
        F2.free()
        P2.free()
    torch.cuda.synchronize()
    e2e_s = reduce_max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = reduce_sum_over_ranks(e2e_flops, world, dev) / e2e_s / 1e12 if e2e_steps > 0 else None

    # ---- roofline of the dominant kernel (grouped leaf products) ----
    peaks, peak_src = _peaks()
    if prec == spamm.FP64:
        peak = fp64_peak_tflops()
        bound = "alu"
        kern = "k_gemm_fp64<32>"
        peak_note = "FP64 FMA: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s)"
        alg_flops = flops
        traffic = None
        burst = None
    else:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        burst = peaks.get("bf16_tflops", 1900.0)
        bound = "tensor"
        kern = "k_gemm_tc (%d exact BF16 slices, leaf 32)" % slices
        peak_note = ("bf16 tensor, sustained (the kernel runs inside a ~1 s solve), %s (MEASURED_PEAKS.json)"
                     % peak_src)
        # tensor work of the surviving products: each slice pair that is not
        # identically zero, on the tiles actually formed (symmetric half)
        alg_flops = tflops
        traffic = _tc_traffic() if slices == 7 and n == WORKLOAD["n"] else None
    achieved = alg_flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": kern, "peak_source": peak_note,
                "frac_of_burst_peak": (achieved / burst) if (achieved and burst) else None,
                "launches_per_solve": main_rep["iters"],
                "useful_leaf_tflops_in_kernel": flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms else None,
                "kernel_share_of_step": gemm_ms / total_ms if total_ms else None}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == spamm.FP64 else "bf16-slices/f32-acc/f64",
        "data": "synthetic (seeded tight-binding Hamiltonian, Morton-ordered 3-D clusters, built on the device)",
        "config": dict(WORKLOAD, n=n, ne=ne, prec=args.prec, slices=slices,
                       parallelism="replicas" if world > 1 else "1gpu",
                       l2="flushed between steps; working set > L2"),
        "sp2": {"iters_per_solve": iters / args.steps, "solve_ms": t_max / args.steps,
                "step_ms": step_ms, "idempotency": main_rep["idem_err"], "trace_err": trace_err,
                "stop_reason": main_rep["stop_reason"], "symmetric": main_rep["symmetric"],
                "sums_rounded": main_rep["sums_rounded"],
                "ms_cull_per_solve": cull_ms / args.steps, "ms_gemm_per_solve": gemm_ms / args.steps,
                "ms_update_per_solve": upd_ms / args.steps,
                "tensor_over_useful_flops": tflops / flops if flops else None,
                "stored_leaves_F": F.stored, "hbm_free_gib_during_mixed": mem_free_mixed,
                "setup_s": gen_s},
        "fp64_plain": fp64,
        "roofline": roofline,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n * n,
                "d2h_bytes_per_step": 8 * n * n, "seconds": e2e_s, "steps": e2e_steps,
                "path": "spamm_tree_build(host F, sparse) + sp2_solve + spamm_to_dense(host P), pinned buffers"},
        "gpu_launches": launches,
    }
    del p_pin
    if want_cpu:
        line["cpu_baseline"] = cpu_baseline(h_pin.numpy(), n)
    F.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _oracle_sp2_sample(f, tau, leaf, nthreads=0):
    """One SP2 iteration by the CPU oracle (Gershgorin bounds, X0, X0^2 by
    the recursive SpAMM of Algorithm 1) on the matrix f; (useful FLOPs,
    seconds)."""
    import oracle
    m = f.shape[0]
    t0 = time.perf_counter()
    _, hist, _ = oracle.sp2(f, leaf, m // 2, tau, fixed_iters=1, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return 2.0 * leaf ** 3 * hist[:, oracle.H_TASKS].sum(), dt


def cpu_baseline(h=None, n=None):
    """The FP64 CPU oracle on the host cores, on a bounded sample of the same
    workload: one SP2 iteration of the leading principal block (the first
    sites along the Morton curve) of the Hamiltonian; useful leaf FLOPs /
    wall time.  Also on one core, on a smaller block."""
    import numpy as np
    import oracle
    from paper_1403_7458_gb300 import synth
    n = n or WORKLOAD["n"]
    b, tau, decay = WORKLOAD["leaf"], WORKLOAD["tau"], WORKLOAD["decay_A"]
    m = min(CPU_SAMPLE_N, n)
    m1 = min(CPU_SAMPLE_N_ONE_CORE, n)
    blk = (np.ascontiguousarray(h[:m, :m]) if h is not None
           else synth.tb_hamiltonian_block(n, m, seed=0, decay=decay))
    flops, dt = _oracle_sp2_sample(blk, tau, b)
    flops1, dt1 = _oracle_sp2_sample(np.ascontiguousarray(blk[:m1, :m1]), tau, b, nthreads=1)
    return {"value": flops / dt / 1e12, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": ("one SP2 iteration (Gershgorin bounds, X0, X0^2 by the recursive SpAMM) of the "
                       "leading %d x %d principal block of the N=%d Hamiltonian (first %d sites along "
                       "the Morton curve), leaf %d, tau %g" % (m, m, n, m, b, tau)),
            "one_core": {"value": flops1 / dt1 / 1e12, "unit": UNIT, "cores": 1, "seconds": dt1,
                         "sample": "the same on the leading %d x %d block" % (m1, m1)}}


def run_precision_study(args):
    """SP2 on the tight-binding Hamiltonian (N = args.n, default 16384) for
    each tau, with FP64 leaf products as the reference and each mixed mode at
    the reference's iteration count: ||P - P_FP64||_F, idempotency, trace,
    Tr[F (P - P_FP64)] and solve time.  One JSON line per (tau, mode)."""
    import torch
    from paper_1403_7458_gb300 import spamm, synth
    spamm.load()
    torch.cuda.set_device(0)
    n = args.n
    h = synth.tb_hamiltonian(n, seed=0)
    hd = torch.from_numpy(h).cuda()
    F = spamm.tree_build(hd, leaf=32)
    ne = n // 2
    modes = [("bf16", spamm.BF16, 0), ("bf16x3", spamm.BF16X3, 0), ("tf32", spamm.TF32, 0),
             ("tf32x3", spamm.TF32X3, 0), ("ozaki5", spamm.OZAKI_BF16, 5),
             ("ozaki6", spamm.OZAKI_BF16, 6), ("ozaki7", spamm.OZAKI_BF16, 7)]
    for tau in args.taus:
        spamm.sp2_solve(F, ne, tau)                       # warm-up
        P64, r64 = spamm.sp2_solve(F, ne, tau)
        p64 = spamm.to_dense(P64)
        base = {"study": "precision", "n": n, "tau": tau, "ne": ne}
        print(json.dumps(dict(base, mode="fp64", solve_ms=r64["ms_total"], iters=r64["iters"],
                              stop=r64["stop_reason"], idem=r64["idem_err"], trace_err=r64["trace_err"],
                              dP=0.0, dE=0.0, tasks=r64["tasks_total"])), flush=True)
        for name, prec, sl in modes:
            spamm.sp2_solve(F, ne, tau, prec=prec, slices=sl, fixed_iters=r64["iters"])
            P, r = spamm.sp2_solve(F, ne, tau, prec=prec, slices=sl, fixed_iters=r64["iters"])
            p = spamm.to_dense(P)
            d = p - p64
            line = dict(base, mode=name, solve_ms=r["ms_total"], iters=r["iters"], stop=r["stop_reason"],
                        idem=r["idem_err"], trace_err=r["trace_err"], dP=torch.linalg.norm(d).item(),
                        dE=float((hd * d.T).sum().item()), tasks=r["tasks_total"],
                        speedup_vs_fp64=r64["ms_total"] / r["ms_total"])
            # the same mode with its own stopping rule (time to solution)
            P2, r2 = spamm.sp2_solve(F, ne, tau, prec=prec, slices=sl)
            line.update(own_stop_ms=r2["ms_total"], own_stop_iters=r2["iters"],
                        own_stop_reason=r2["stop_reason"])
            print(json.dumps(line), flush=True)
            del P, P2, p, d
        del P64, p64
        torch.cuda.empty_cache()


def run_batch_study(args):
    """Many independent SpAMMs in one persistent launch: `args.batch` products
    C_m = A_m A_m of sizes log-uniform in [512, 8192] (multiples of 32, seeds
    0..count-1, decay length uniform in [1, 2] A, the decaying-matrix
    generator), tau = 1e-6, TF32 leaves with FP32 accumulation.  The leaf size
    and tile schedule come from the library's autotuner; the batched call is
    captured into a CUDA graph and replayed.  Compared with the same products
    as sequential spamm_multiply calls (plain and graph-captured) and with the
    FP64 batched form.  One JSON line."""
    import torch
    from paper_1403_7458_gb300 import spamm, synth
    spamm.load()
    torch.cuda.set_device(0)
    prec = {"tf32": spamm.TF32, "tf32x3": spamm.TF32X3, "bf16x3": spamm.BF16X3,
            "ozaki": spamm.OZAKI_BF16}[args.batch_prec]
    slices = 7 if prec == spamm.OZAKI_BF16 else 0
    tau = args.batch_tau
    sizes, decays = synth.batch_sizes(args.batch, seed=0)
    t0 = time.perf_counter()
    mats = [torch.from_numpy(synth.decaying_matrix(n, seed=q, decay=d)).cuda()
            for q, (n, d) in enumerate(zip(sizes, decays))]
    gen_s = time.perf_counter() - t0
    tune = spamm.autotune_batched(mats, mats, tau, prec=prec, slices=slices, reps=3)
    leaf, flags = tune["leaf"], tune["flags"]
    A = [spamm.tree_build(m, leaf=leaf) for m in mats]
    C, st = spamm.multiply_batched(A, A, tau, prec=prec, slices=slices, flags=flags, stats=True)
    _, stt = spamm.multiply_batched(A, A, tau, C=C, prec=prec, slices=slices, flags=flags, timing=True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = []
        for _ in range(steps):
            flush.zero_()
            ev0.record()
            fn()
            ev1.record()
            ev1.synchronize()
            out.append(ev0.elapsed_time(ev1))
        out.sort()
        return out[len(out) // 2]

    def capture(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn(side.cuda_stream)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return g

    def batched(stream=None):
        spamm.multiply_batched(A, A, tau, C=C, prec=prec, slices=slices, flags=flags, stream=stream)

    Cs = [None] * len(A)

    def sequential(stream=None):
        for q in range(len(A)):
            Cs[q], _ = spamm.multiply(A[q], A[q], tau, C=Cs[q], prec=prec, slices=slices, flags=flags,
                                      stream=stream)

    steps = max(args.steps, 3)
    for _ in range(args.warmup):
        batched()
        sequential()
    torch.cuda.synchronize()
    ms_batched = timed(batched, steps)
    ms_seq = timed(sequential, steps)
    gb = capture(batched)
    ms_batched_graph = timed(gb.replay, steps)
    gs = capture(sequential)
    ms_seq_graph = timed(gs.replay, steps)
    # FP64 batched at the same leaf size: reference values (same task set)
    C64, st64 = spamm.multiply_batched(A, A, tau, stats=True)
    rel = 0.0
    for q in range(len(A)):
        x = spamm.to_dense(C[q])
        y = spamm.to_dense(C64[q])
        rel = max(rel, (torch.linalg.norm(x - y) / torch.linalg.norm(y)).item())
        del x, y
    del C64
    # FP64 batched at its own tuned leaf size: the plain form's best time
    tune64 = spamm.autotune_batched(mats, mats, tau, reps=1)
    A64 = [spamm.tree_build(m, leaf=tune64["leaf"]) for m in mats]
    D64, sd64 = spamm.multiply_batched(A64, A64, tau, stats=True)
    ms_fp64 = timed(lambda: spamm.multiply_batched(A64, A64, tau, C=D64), max(2, steps // 2))
    peaks, peak_src = _peaks()
    # nominal dense TF32 : BF16 = 1.1 : 2.25 PFLOP/s applied to the measured BF16 peak
    tf32_peak = peaks.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
    line = {
        "study": "batch", "products": len(A), "prec": args.batch_prec, "tau": tau,
        "sizes": {"min": min(sizes), "max": max(sizes), "median": sorted(sizes)[len(sizes) // 2],
                  "sum_n2": int(sum(n * n for n in sizes))},
        "autotune": tune, "autotune_fp64": tune64, "tasks": st["tasks"], "candidates": st["candidates"],
        "useful_tflop_per_batch": st["flops_useful"] / 1e12,
        "ms": {"batched_graph": ms_batched_graph, "batched": ms_batched,
               "sequential": ms_seq, "sequential_graph": ms_seq_graph, "fp64_batched": ms_fp64,
               "split_cull_gemm_norm": [stt["ms_cull"], stt["ms_gemm"], stt["ms_norm"]]},
        "value_tflops": st["flops_useful"] / (ms_batched_graph * 1e-3) / 1e12,
        "speedup_vs_sequential": ms_seq / ms_batched_graph,
        "speedup_vs_sequential_graph": ms_seq_graph / ms_batched_graph,
        "speedup_vs_fp64_batched": ms_fp64 / ms_batched_graph,
        "fp64_batched_tflops": sd64["flops_useful"] / (ms_fp64 * 1e-3) / 1e12,
        "roofline": {"bound": "tensor", "kernel": "k_gemm_tc (one batched launch)",
                     "achieved": st["flops_issued"] / (stt["ms_gemm"] * 1e-3) / 1e12,
                     "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": st["flops_issued"] / (stt["ms_gemm"] * 1e-3) / 1e12 / tf32_peak,
                     "peak_source": "TF32 = 1.1/2.25 x the %s sustained BF16 peak (nominal ratio)" % peak_src,
                     "note": "issued tensor work (tiles of 128 rows; culled leaf rows masked out of the MMA)"},
        "max_rel_err_vs_fp64": rel,
        "generation_s": gen_s,
        "l2": "flushed between steps",
    }
    print(json.dumps(line), flush=True)


def run_large_study(args):
    """SP2 at N = args.n_large (default 65536) on the tight-binding
    Hamiltonian with decay length 1.0 A, tau = 1e-8, leaf 32, Ne = N/2: FP64
    leaf products with their own stopping rule, then exact BF16 slices (7)
    at the same iteration count (||P - P_FP64||_F, Tr[F (P - P_FP64)]) and
    with their own stopping rule (time to solution).  The Hamiltonian is
    generated on the device.  One JSON line."""
    import torch
    from paper_1403_7458_gb300 import spamm, synth
    spamm.load()
    torch.cuda.set_device(0)
    n, leaf, tau = args.n_large, 32, 1e-8
    ne = n // 2
    gib = lambda b: b / 2.0 ** 30
    mem = {"total_gib": gib(torch.cuda.mem_get_info()[1])}
    t0 = time.perf_counter()
    h = synth.tb_hamiltonian_torch(n, seed=0, decay=1.0)
    # sparse leaf storage: leaves with ||leaf||_F <= 1e-12 are not stored
    F = spamm.tree_build(h, leaf=leaf, drop=1e-12)
    torch.cuda.synchronize()
    del h
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    nb = F.nb
    fill = lambda M: float((spamm.norms(M, M.depth)[:nb, :nb] > 1e-24).mean())
    fill_h = fill(F)

    P64, r64 = spamm.sp2_solve(F, ne, tau, timing=True)
    fill_p = fill(P64)
    mem["free_after_fp64_gib"] = gib(torch.cuda.mem_get_info()[0])
    p64 = spamm.to_dense(P64)
    P64.free()
    torch.cuda.synchronize()

    P, r = spamm.sp2_solve(F, ne, tau, prec=spamm.OZAKI_BF16, slices=7, fixed_iters=r64["iters"], timing=True)
    mem["free_with_mixed_scratch_gib"] = gib(torch.cuda.mem_get_info()[0])
    spamm.release_scratch(P)
    torch.cuda.synchronize()
    d = spamm.to_dense(P)
    d.sub_(p64)                                  # P_mixed - P_FP64, in place
    dP = torch.linalg.norm(d).item()
    del p64
    torch.cuda.empty_cache()
    hh = synth.tb_hamiltonian_torch(n, seed=0, decay=1.0)
    dE = 0.0
    for r0 in range(0, n, 4096):                 # Tr[F dP] = sum_ij F_ij dP_ji
        dE += float((hh[r0:r0 + 4096] * d[:, r0:r0 + 4096].T).sum().item())
    del hh, d
    torch.cuda.empty_cache()

    P2, r2 = spamm.sp2_solve(F, ne, tau, P=P, prec=spamm.OZAKI_BF16, slices=7, timing=True)
    peaks, peak_src = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    keys = ("iters", "stop_reason", "ms_total", "ms_cull", "ms_gemm", "ms_update", "tasks_total",
            "flops_useful", "flops_tensor", "idem_err", "trace_err", "launches", "symmetric")
    line = {
        "study": "large", "n": n, "leaf": leaf, "tau": tau, "ne": ne, "decay_A": 1.0,
        "storage": "F: sparse leaves (norm > 1e-12 stored, %d of %d); X, X^2: dense leaf grid" % (F.stored, nb * nb),
        "leaf_fill": {"H_n2_gt_1e-24": fill_h, "P_n2_gt_1e-24": fill_p},
        "fp64": {k: r64[k] for k in keys},
        "mixed_same_iters": {k: r[k] for k in keys},
        "mixed_own_stop": {k: r2[k] for k in keys},
        "dP_fro": dP, "dE_trF": dE,
        "speedup_same_iters": r64["ms_total"] / r["ms_total"],
        "speedup_time_to_solution": r64["ms_total"] / r2["ms_total"],
        "useful_tflops": {"fp64": r64["flops_useful"] / (r64["ms_total"] * 1e-3) / 1e12,
                          "mixed": r["flops_useful"] / (r["ms_total"] * 1e-3) / 1e12},
        "roofline": {"fp64": {"bound": "alu", "kernel": "k_gemm_fp64<32>", "unit": "TFLOP/s",
                              # the leaf products the kernel formed (the mirrored
                              # half of a symmetric X^2 is stored, not formed)
                              "achieved": r64["flops_tensor"] / (r64["ms_gemm"] * 1e-3) / 1e12,
                              "peak": fp64_peak_tflops()},
                     "mixed": {"bound": "tensor", "kernel": "k_gemm_tc<7,2,32,1>", "unit": "TFLOP/s",
                               "achieved": r["flops_tensor"] / (r["ms_gemm"] * 1e-3) / 1e12,
                               "peak": bf16, "peak_source": "bf16 sustained, %s" % peak_src}},
        "memory": mem, "generation_s": gen_s,
    }
    for k in ("fp64", "mixed"):
        rf = line["roofline"][k]
        rf["frac"] = rf["achieved"] / rf["peak"]
    print(json.dumps(line), flush=True)


def run_spamm_study(args):
    """Single SpAMM products of the decaying matrix (N = 1024, leaf 32, tau =
    1e-6; a_ij = u_ij exp(-r_ij / 1.5 A), seed 0): device time per product
    (plain launches and graph-captured), FP64 and mixed precision, with the
    task count.  One JSON line."""
    import torch
    from paper_1403_7458_gb300 import spamm, synth
    spamm.load()
    torch.cuda.set_device(0)
    n, tau = args.spamm_n, 1e-6
    a = torch.from_numpy(synth.decaying_matrix(n, 0)).cuda()
    A = spamm.tree_build(a, leaf=32)
    out = {"study": "spamm", "n": n, "leaf": 32, "tau": tau}
    for name, prec, sl in (("fp64", spamm.FP64, 0), ("ozaki7", spamm.OZAKI_BF16, 7), ("tf32", spamm.TF32, 0)):
        C, st = spamm.multiply(A, A, tau, prec=prec, slices=sl, stats=True, timing=True)

        def one(stream=None):
            spamm.multiply(A, A, tau, C=C, prec=prec, slices=sl, stream=stream)

        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        for _ in range(5):
            one()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            one()
        ev1.record()
        ev1.synchronize()
        plain_us = ev0.elapsed_time(ev1) / reps * 1e3
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            one(side.cuda_stream)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            one(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            g.replay()
        ev1.record()
        ev1.synchronize()
        graph_us = ev0.elapsed_time(ev1) / reps * 1e3
        out[name] = {"tasks": st["tasks"], "candidates": st["candidates"], "us_per_product": plain_us,
                     "us_per_product_graph": graph_us, "ms_cull": st["ms_cull"], "ms_gemm": st["ms_gemm"],
                     "ms_norm": st["ms_norm"], "useful_tflops_graph": st["flops_useful"] / (graph_us * 1e-6) / 1e12}
    print(json.dumps(out), flush=True)


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1403_7458_gb300 import synth
    n, b, tau, decay = args.bench_n, WORKLOAD["leaf"], WORKLOAD["tau"], WORKLOAD["decay_A"]
    m = min(REF_SAMPLE_N, n)
    blk = synth.tb_hamiltonian_block(n, m, seed=0, decay=decay)
    for _ in range(args.warmup):
        _oracle_sp2_sample(blk, tau, b)
    flops = secs = 0.0
    for _ in range(args.steps):
        f, dt = _oracle_sp2_sample(blk, tau, b)
        flops += f
        secs += dt
    value = flops / secs / 1e12
    sample = ("one SP2 iteration (Gershgorin bounds, X0, X0^2 by the recursive SpAMM) of the leading "
              "%d x %d principal block of the N=%d Hamiltonian per step" % (m, m, n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, n=n, ne=n // 2, prec="fp64", parallelism="cpu", sample_n=m),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _spawn_ranks(args, argv):
    """Start args.gpus ranks of this script through torch.distributed.run (one
    process per GPU) when it was not launched that way."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(args.gpus), "--master-addr", "127.0.0.1",
           "--master-port", str(port), os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp64", "ozaki"], default="ozaki")
    ap.add_argument("--slices", type=int, default=7)
    ap.add_argument("--bench-n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--study", choices=["none", "precision", "batch", "large", "spamm"], default="none")
    ap.add_argument("--spamm-n", type=int, default=1024)
    ap.add_argument("--n-large", type=int, default=65536)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--batch-prec", choices=["tf32", "tf32x3", "bf16x3", "ozaki"], default="tf32")
    ap.add_argument("--batch-tau", type=float, default=1e-6)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--taus", type=float, nargs="+", default=[1e-4, 1e-6, 1e-8, 1e-10])
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and args.study == "none":
        sys.exit(_spawn_ranks(args, sys.argv[1:] if argv is None else argv))
    if args.study == "none" and args.gpus != world:
        sys.exit("bench.py: --gpus %d but WORLD_SIZE=%d" % (args.gpus, world))
    if args.study == "precision":
        run_precision_study(args)
    elif args.study == "batch":
        run_batch_study(args)
    elif args.study == "large":
        run_large_study(args)
    elif args.study == "spamm":
        run_spamm_study(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
