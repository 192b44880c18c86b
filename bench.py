"""Benchmark: block-sparse contraction TFLOP/s, split precision vs FP64, on one GB300.

One step = one pass of the whole hot path on the 40/240 spin-orbital
coupled-cluster-doubles workload (tiles 20/40, spin block sparsity): vvvv
ladder, W = W0 copy, intermediate W += V_oovv T, oooo ladder, ring term with
the P(ab)P(ij) antisymmetriser, T1 term, and the energy.  The headline runs
every contraction in split precision (six BF16 slices per FP64 operand on the
tcgen05 tensor cores); an FP64 pass of the same step gives the FP64 rate and
the split-precision error.  Throughput counts nonzero-block flops (2*M*N*K
over every stored block pair), the same count for every precision.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): independent replicas of the step, one
per GPU, no collective on the data path (weak scaling).  ``--impl reference``
times the FP64 CPU oracle on bounded samples of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "block-sparse contraction TFLOP/s: split-precision vs FP64, rel err ≤1e-10"
UNIT = "TFLOP/s"
WORKLOAD = ("ccsd_doubles_O40_V240: vvvv ladder + W copy + intermediate + oooo ladder + ring with P(ab)P(ij) + "
            "T1 term + energy")
SLICES = 6
# DRAM bytes (read + write) per launch of the split-precision GEMM kernel, averaged over the five GEMM
# launches of an O=40 V=240 doubles step, from an ncu capture of this bench command's GEMM launches,
# keyed by the hash of the kernel sources it was taken on; a changed kernel reports null until it is
# captured again.
MEASURED_TRAFFIC = {"2c7bdc1ea544cab5": 8.035e9}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("ozaki.cu", "ozaki.h", "ozaki_device.cuh", "ozaki_fused.cu", "sm100.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2201_01257_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ multi-rank

def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's); identity without dist."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, flops_per_rank_step: float, ms_per_step: float) -> float:
    """Whole-job TFLOP/s: every rank runs its own full step (weak scaling), timed by the slowest rank."""
    return world * flops_per_rank_step / (ms_per_step * 1e-3) / 1e12


# ------------------------------------------------------------------ ours

def run_ours(args, rank: int, world: int) -> dict | None:
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl
    import tamm_synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{dev}"))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = wl.ccsd_doubles_o40_v240()
    ctx = tg.Context(dev)
    spaces, T = gw.build(ctx, w, fill=False)
    host = {}
    for name, spec in w.tensors.items():
        if spec.sigma == 0.0:
            continue
        t = T[name]
        h = torch.empty(t.n_elems, dtype=torch.float64, pin_memory=True)
        lo, ext = t.block_lo_ext()
        tamm_synth.fill_boxes(w.seed, spec.stream, spec.sigma, [m.n for m in t.modes], spec.anti01, spec.anti23,
                              lo, ext, t.block_offsets, h.numpy(), sym01=spec.sym01)
        host[name] = h
        ctx.copy_from_host(t, h.numpy())
    ctx.sync()
    run = gw.Runner(ctx, w, spaces, T)
    flops = sum(run.flops(s) for s in w.steps)

    energy_dev = torch.zeros(1, dtype=torch.float64, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()

    # split-precision configuration per contraction: autotuned (slices, chunk, tile policy) for
    # rel err <= 1e-10 with a factor-2 margin, or a fixed slice count
    tuned = None
    if args.slices == 0:
        # one FP64 step first, so that intermediates (W) hold the values the step's contractions see
        run.run("f64", 0, energy_out=energy_dev.data_ptr())
        t0 = time.time()
        tuned = run.autotune(1e-10)
        tune_s = time.time() - t0
    oz_slices = args.slices

    def step(prec):
        run.run("ozaki_bf16" if prec == "oz" else "f64", oz_slices if prec == "oz" else 0,
                energy_out=energy_dev.data_ptr())

    # --- device-resident timed region (split precision) ---
    for _ in range(args.warmup):
        step("oz")
    barrier()
    ctx.profile_read()
    ctx.profile(True)
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clocks:
        barrier()
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed steps' launches
        ev0.record(stream)
        for _ in range(args.steps):
            step("oz")
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.launch_count() - l0
    ctx.profile(False)
    prof = ctx.profile_read()
    r_oz = T["R"].download()
    w_oz = T["W"].download()
    e_oz = float(energy_dev.item())

    # --- FP64 pass of the same step: its rate and the split-precision error ---
    step("f64")
    ctx.sync()
    f64_steps = max(1, min(2, args.steps))
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(f64_steps):
        step("f64")
    ev3.record(stream)
    torch.cuda.synchronize()
    ms_f64 = ev2.elapsed_time(ev3) / f64_steps
    r_64, w_64, e_64 = T["R"].download(), T["W"].download(), float(energy_dev.item())
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    # measured FP64 throughput of this GPU: the FP64 path's roofline denominator
    fp64_peak = {"dfma": round(ctx.fp64_peak("dfma"), 4), "dmma": round(ctx.fp64_peak("dmma"), 4)}

    # --- each contraction alone (not the headline): split precision and FP64 ---
    per_contraction = {}
    for st in w.steps:
        if not isinstance(st, wl.ContractSpec):
            continue
        res = {"nonzero_block_flops": run.flops(st)}
        for prec, reps in (("oz", 3), ("f64", 1)):
            go = lambda: run.run("ozaki_bf16" if prec == "oz" else "f64", oz_slices if prec == "oz" else 0,
                                 steps=[st])
            go()
            ctx.profile_read()
            ctx.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                go()
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.profile(False)
            kp = ctx.profile_read()
            t = e0.elapsed_time(e1) / reps
            res["split_ms" if prec == "oz" else "f64_ms"] = round(t, 3)
            res["split_TFLOP/s" if prec == "oz" else "f64_TFLOP/s"] = round(res["nonzero_block_flops"] / t / 1e9, 3)
            if prec == "oz" and kp["gemm_ozaki"][0] > 0:
                # this contraction's own GEMM launches against the sustained BF16 peak, in slice products
                s_used = tuned[st.name]["slices"] if tuned else oz_slices
                g_ms = kp["gemm_ozaki"][0] / reps
                res["split_gemm_ms"] = round(g_ms, 3)
                res["split_gemm_frac_of_sustained_bf16"] = round(
                    res["nonzero_block_flops"] * (s_used * (s_used + 1) // 2) / (g_ms * 1e-3) / 1e12
                    / measured_peaks().get("bf16_tflops_sustained", 1700.0), 4)
        per_contraction[st.name] = res

    # --- the two transposed permuted adds of the step alone (tiled through shared memory): GB/s ---
    add_bw = {}
    ring = next(st for st in w.steps if st.name == "ring")
    X, lx = run.scratch_for(ring)
    from paper_2201_01257_gb300 import workload as gw_

    for name, fn, nbytes in (
            ("ring_antisymmetriser", lambda: ctx.add(T["R"], "abij", 1.0, X, gw_.antisym_terms("abij", lx)),
             T["R"].n_elems * 8 * (4 + 2)),  # four source terms read, R read and written
            ("transposition_ij", lambda: ctx.add(T["R"], "abij", 1.0, X, [(1.0, gw_.antisym_terms("abij", lx)[2][1])]),
             T["R"].n_elems * 8 * (1 + 2))):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        t_ms = a.elapsed_time(b) / 5
        add_bw[name] = {"ms": round(t_ms, 4), "GB/s": round(nbytes / (t_ms * 1e-3) / 1e9, 1),
                        "frac_of_hbm": round(nbytes / (t_ms * 1e-3) / 1e9 / measured_peaks()["hbm_gbs"], 3)}

    # --- end to end through the C ABI: pinned host inputs in, result out, every step ---
    # Every step copies all of its inputs from pinned host memory and reads R and the energy back.
    # Pipelined (the reported figure): the inputs of step k+1 are copied, on a second stream through
    # a second context, into the other of two device buffer sets while step k computes; each step
    # binds its set.  Serial: the copies, the step and the read-back one after another on one stream.
    out_host = torch.empty(T["R"].n_elems, dtype=torch.float64, pin_memory=True)
    e_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
    h2d = sum(T[k].n_elems * 8 for k in host)
    d2h = T["R"].n_elems * 8 + 8
    e2e_k = max(1, args.steps)

    def e2e_serial_step():
        for k, h in host.items():
            ctx.copy_from_host(T[k], h.numpy())
        step("oz")
        ctx.copy_to_host(T["R"], out_host.numpy())
        e_host.copy_(energy_dev, non_blocking=True)

    e2e_serial_step()
    barrier()
    ev4, ev5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev4.record(stream)
    for _ in range(e2e_k):
        e2e_serial_step()
    ev5.record(stream)
    barrier()
    ms_e2e_serial = ev4.elapsed_time(ev5) / e2e_k

    copy_stream = torch.cuda.Stream(dev)
    cctx = tg.Context(dev, stream=copy_stream)
    sets = [{k: T[k].data for k in host}, {k: torch.empty_like(T[k].data) for k in host}]
    r_sets = [T["R"].data, torch.empty_like(T["R"].data)]
    e_sets = [energy_dev, torch.zeros_like(energy_dev)]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    computed = [torch.cuda.Event(), torch.cuda.Event()]
    read_back = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_pipelined(n_steps):
        # Every transfer runs on one copy stream, one at a time (concurrent host-to-device and
        # device-to-host copies slow each other down on this link): the inputs of step k+1, then the
        # result of step k, while step k+1 computes.  Inputs, R and the energy alternate between two
        # device sets, so a set is rewritten only after the step that read it (inputs) or its read-back
        # (R, energy) is done.
        for k, h in host.items():
            T[k].bind(sets[0][k])
            cctx.copy_from_host(T[k], h.numpy())
        copied[0].record(copy_stream)
        for i in range(n_steps):
            cur, nxt = i % 2, (i + 1) % 2
            stream.wait_event(copied[cur])
            if i >= 2:
                stream.wait_event(read_back[cur])
            for k in host:
                T[k].bind(sets[cur][k])
            T["R"].bind(r_sets[cur])
            run.run("ozaki_bf16", oz_slices, energy_out=e_sets[cur].data_ptr())
            computed[cur].record(stream)
            if i + 1 < n_steps:
                if i >= 1:
                    copy_stream.wait_event(computed[nxt])
                for k, h in host.items():
                    T[k].bind(sets[nxt][k])
                    cctx.copy_from_host(T[k], h.numpy())
                copied[nxt].record(copy_stream)
            copy_stream.wait_event(computed[cur])
            T["R"].bind(r_sets[cur])
            cctx.copy_to_host(T["R"], out_host.numpy())
            with torch.cuda.stream(copy_stream):
                e_host.copy_(e_sets[cur], non_blocking=True)
            read_back[cur].record(copy_stream)
        for k in host:
            T[k].bind(sets[0][k])
        T["R"].bind(r_sets[0])

    e2e_pipelined(2)
    torch.cuda.synchronize()
    barrier()
    ev6, ev7 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev6.record(copy_stream)
    e2e_pipelined(e2e_k)
    ev7.record(copy_stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = ev6.elapsed_time(ev7) / e2e_k
    r_e2e = out_host.numpy().copy()

    # the copy bound of e2e: the same pinned host inputs copied alone (cudaMemcpyAsync, one per tensor)
    plain = {k: torch.empty_like(T[k].data) for k in host}
    for k, h in host.items():
        plain[k][: h.numel()].copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    ev8, ev9 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev8.record(stream)
    for _ in range(2):
        for k, h in host.items():
            plain[k][: h.numel()].copy_(h, non_blocking=True)
    ev9.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 2 * h2d / (ev8.elapsed_time(ev9) * 1e-3) / 1e9
    del plain

    ms, ms_e2e, ms_f64 = (max_over_ranks(x, dist, f"cuda:{dev}") for x in (ms, ms_e2e, ms_f64))
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return None

    peaks = measured_peaks()
    gemm_ms, gemm_n = prof["gemm_ozaki"]
    dominant = max(prof, key=lambda k: prof[k][0])
    # BF16 slice products per step (algorithmic): S(S+1)/2 products of every nonzero block pair
    def n_products(s):
        return s * (s + 1) // 2

    tensor_flops_per_step = sum(run.flops(st) * n_products(tuned[st.name]["slices"] if tuned else oz_slices)
                                for st in w.steps if isinstance(st, wl.ContractSpec))
    achieved = tensor_flops_per_step * args.steps / (gemm_ms * 1e-3) / 1e12 if gemm_ms else None
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    traffic = MEASURED_TRAFFIC.get(kernel_source_hash())
    value = job_throughput(world, flops, ms)
    return {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16 slices (f32 accumulate, f64 reconstruct)",
        "data": "synthetic (seeded Philox normals, antisymmetrised; V~N(0,0.1), T~N(0,0.01))",
        "config": {
            "workload": WORKLOAD,
            "O": 40, "V": 240, "tiles": [20, 40], "symmetry": "spin",
            "precision": "ozaki_bf16",
            "slices": ({k: v["slices"] for k, v in tuned.items()} if tuned else oz_slices),
            "autotuned": ({k: {"slices": v["slices"], "chunk_k": v["chunk_k"], "tile_policy": v["tile_policy"],
                               "persistent": v["persistent"], "shared_scale": v["shared_scale"],
                               "fused_a": v["fused_a"],
                               "rel_err_vs_f64_gpu": v["rel_err"],
                               "ms": round(v["ms"], 3)}
                           for k, v in tuned.items()} if tuned else None),
            "autotune_seconds": round(tune_s, 2) if tuned else None,
            "nonzero_block_flops_per_step": flops,
            "l2": "inputs larger than L2 (V_vvvv 9.95 GB per step)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        },
        "f64": {"value": round(job_throughput(world, flops, ms_f64), 4), "unit": UNIT,
                "ms_per_step": round(ms_f64, 2), "steps": f64_steps,
                "peak_measured_tflops": fp64_peak,
                "frac_of_measured_peak": round(job_throughput(world, flops, ms_f64) / max(fp64_peak.values()), 4)},
        "speedup_vs_f64": round(ms_f64 / ms, 2),
        "per_contraction": per_contraction,
        "permuted_adds": add_bw,
        "rel_err_vs_f64": {"R": rel(r_oz, r_64), "W": rel(w_oz, w_64), "energy": abs(e_oz - e_64) / abs(e_64)},
        "e2e": {"value": round(job_throughput(world, flops, ms_e2e), 3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e, 3),
                "steps": e2e_k, "pipelined": "inputs of step k+1, then the result of step k, copied on one copy stream during step k+1 "
                             "(two device sets of inputs, R and energy)",
                "serial": {"value": round(job_throughput(world, flops, ms_e2e_serial), 3),
                           "ms_per_step": round(ms_e2e_serial, 3)},
                "rel_err_R_vs_device_step": rel(r_e2e, r_oz),
                "plain_pinned_h2d_GBps": round(h2d_gbs, 1),
                "copy_bound_ms": round(h2d / (h2d_gbs * 1e9) * 1e3, 3)},
        "gpu_launches": launches,
        "kernel_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in prof.items()},
        "roofline": {
            "kernel": "ozaki_gemm_kernel (tcgen05 BF16 slice products)",
            "dominant_by_time": dominant,
            "bound": "tensor",
            "achieved": round(achieved, 2) if achieved else None,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4) if achieved else None,
            "peak_source": f"{peaks['_source']} bf16_tflops_sustained",
            "algorithmic_flops_per_launch": tensor_flops_per_step / max(1, gemm_n // max(1, args.steps)),
            "avg_launch_ms": round(gemm_ms / gemm_n, 4) if gemm_n else None,
            "traffic": traffic,
        },
        "clocks": clocks.summary(),
        "cpu_baseline": cpu_baseline(seconds=args.cpu_seconds) if world == 1 or rank == 0 else None,
    }


# ---------------------------------------------------------- CPU (oracle)

def oracle_sample(w, target_flops: float, seed: int = 0, box: int = 4):
    """Oracle tensors with only the blocks a seeded sample needs filled, and the sample:
    for every contraction, box^4 sub-boxes of randomly chosen output blocks.

    Returns (tensors, [(step, cblocks, lo, ext)], total nonzero-block flops of the sample)."""
    import itertools

    import oracle as O
    import tamm_synth
    from tamm_synth import workloads as wl

    spaces = {k: O.Space.from_spec(s) for k, s in w.spaces.items()}
    T = {n: O.Tensor([spaces[m] for m in t.modes], t.n_upper, t.sym) for n, t in w.tensors.items()}
    rng = np.random.default_rng(seed)
    steps = [s for s in w.steps if isinstance(s, wl.ContractSpec)]
    plan, need, total = [], {n: set() for n in T}, 0.0
    per_step = target_flops / len(steps)
    for s in steps:
        C, A, B = T[s.c], T[s.a], T[s.b]
        lab = {}
        for X, l in ((C, s.lc), (A, s.la), (B, s.lb)):
            for m, ch in enumerate(l):
                lab[ch] = X.modes[m]
        summed = [ch for ch in s.la if ch not in s.lc]
        _, ext_all = C.block_lo_ext()
        kcache = {}

        def k_eff(cb):
            if cb not in kcache:
                tile = {ch: int(C.block_tiles[cb, m]) for m, ch in enumerate(s.lc)}
                k, blocks = 0, []
                for kt in itertools.product(*[range(lab[ch].n_tiles) for ch in summed]):
                    tile.update(dict(zip(summed, kt)))
                    ab = A.find_block([tile[ch] for ch in s.la])
                    bb = B.find_block([tile[ch] for ch in s.lb])
                    if ab < 0 or bb < 0:
                        continue
                    blocks.append((ab, bb))
                    kk = 1
                    for ch in summed:
                        kk *= lab[ch].tiles[tile[ch]][1]
                    k += kk
                kcache[cb] = (k, blocks)
            return kcache[cb]

        cbs, los, exts, fl = [], [], [], 0.0
        guard = 0
        # boxes come from two output blocks per contraction, so few input blocks need filling
        pool = [int(x) for x in rng.permutation(C.n_blocks)[:2]]
        while fl < per_step and guard < 100000:
            guard += 1
            cb = pool[guard % len(pool)]
            k, blocks = k_eff(cb)
            if k == 0:
                continue
            ext = [min(box, int(e)) for e in ext_all[cb]]
            lo = [int(rng.integers(0, int(e) - x + 1)) for e, x in zip(ext_all[cb], ext)]
            cbs.append(cb)
            los.append(lo)
            exts.append(ext)
            fl += 2.0 * float(np.prod(ext)) * k
            for ab, bb in blocks:
                need[s.a].add(ab)
                need[s.b].add(bb)
        plan.append((s, cbs, los, exts))
        total += fl
    for n, blocks in need.items():
        if not blocks:
            continue
        spec = w.tensors[n]
        if spec.sigma == 0.0:
            continue
        X = T[n]
        lo, ext = X.block_lo_ext()
        idx = np.array(sorted(blocks))
        tamm_synth.fill_boxes(w.seed, spec.stream, spec.sigma, X.dense_shape(), spec.anti01, spec.anti23,
                              lo[idx], ext[idx], X.block_off[idx], X.data, sym01=spec.sym01)
    return T, plan, total


def time_oracle_sample(T, plan) -> float:
    import oracle as O

    t0 = time.perf_counter()
    for s, cbs, los, exts in plan:
        O.contract_boxes(s.alpha, T[s.c], s.lc, T[s.a], s.la, T[s.b], s.lb, cbs, los, exts)
    return time.perf_counter() - t0


def cpu_baseline(seconds: float = 15.0) -> dict:
    """The FP64 oracle (as it stands) on a bounded sample of the same workload."""
    from tamm_synth import workloads as wl

    w = wl.ccsd_doubles_o40_v240()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # calibrate on a small sample, then size the timed sample to about `seconds`
    T, plan, fl = oracle_sample(w, 1e9, seed=1)
    dt = time_oracle_sample(T, plan)
    T, plan, fl = oracle_sample(w, fl / max(dt, 1e-6) * seconds, seed=2)
    dt = time_oracle_sample(T, plan)
    return {"value": round(fl / dt / 1e12, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle on seeded 4x4x4x4 sub-boxes of output blocks of each of the five "
                      f"contractions of ccsd_doubles_O40_V240 ({fl:.3e} nonzero-block flops, {dt:.1f} s)",
            "seconds": round(dt, 2)}


def run_reference(args, rank: int) -> dict | None:
    if rank != 0:
        return None
    from tamm_synth import workloads as wl

    w = wl.ccsd_doubles_o40_v240()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    T, plan, fl = oracle_sample(w, 1e9, seed=1)
    dt = time_oracle_sample(T, plan)
    per_step_flops = fl / dt * args.ref_seconds
    T, plan, fl = oracle_sample(w, per_step_flops, seed=3)
    for _ in range(args.warmup):
        time_oracle_sample(T, plan)
    times = [time_oracle_sample(T, plan) for _ in range(args.steps)]
    ms = 1e3 * float(np.sum(times)) / args.steps
    value = fl / (ms * 1e-3) / 1e12
    sample = (f"FP64 oracle on seeded 4x4x4x4 sub-boxes of output blocks of the five contractions of "
              f"ccsd_doubles_O40_V240 ({fl:.3e} nonzero-block flops per step)")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "O": 40, "V": 240, "tiles": [20, 40], "symmetry": "spin",
                       "precision": "f64 (CPU oracle; each step a bounded sample of the workload, see cpu_baseline)"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ladder_case(args) -> dict:
    """A single split-precision vvvv ladder at a chosen size (small cases for profiling)."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    O_, V_ = (int(x) for x in args.ladder.split(","))
    w = wl._doubles(wl._vt(2, O_, V_, 20, 40, f"ladder_O{O_}_V{V_}"))
    ctx = tg.Context(0)
    _, T = gw.build(ctx, w, only={"V_vvvv", "T", "R"})
    fl = ctx.flops(T["R"], "abij", T["V_vvvv"], "abef", T["T"], "efij")
    go = lambda: ctx.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", "ozaki_bf16", SLICES)
    for _ in range(args.warmup):
        go()
    ctx.sync()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        go()
    e.record()
    ctx.sync()
    ms = s.elapsed_time(e) / args.steps
    return {"case": f"vvvv ladder O={O_} V={V_} tiles 20/40, split precision", "ms": round(ms, 3),
            "TFLOP/s": round(fl / ms / 1e9, 3), "nonzero_block_flops": fl}


def run_irrep_case(args) -> dict:
    """Uneven D2h blocks (O=64, V=384): the ladder and the ring as one contraction group, eager and as a
    CUDA graph, against the same contractions launched one by one and the FP64 path."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    O_, V_ = (int(x) for x in args.irrep.split(",")) if args.irrep else (64, 384)
    w = wl.irrep_doubles(O=O_, V=V_)
    stream = torch.cuda.Stream(0)
    ctx = tg.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        sp, T = gw.build(ctx, w)
    run = gw.Runner(ctx, w, sp, T)
    flops = sum(run.flops(s) for s in w.steps)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        ctx.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        ctx.sync()
        return a.elapsed_time(b) / k

    out = {"case": f"{w.name}: vvvv ladder + ring with P(ab)P(ij), D2h irreps, tiles U{{8..96}}",
           "nonzero_block_flops": flops, "blocks": {k: T[k].n_blocks for k in ("V_vvvv", "T", "R")}}
    with torch.cuda.stream(stream):
        # the one-time cost of a plan (block-pair enumeration, slicing and work-item records, their upload):
        # the first grouped call on a fresh context against the next one, host wall clock, synchronised
        ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, 1)
        walls = []
        for _ in range(2):
            ctx.sync()
            t0 = time.perf_counter()
            run.run_grouped(w.steps, "ozaki_bf16", SLICES)
            ctx.sync()
            walls.append((time.perf_counter() - t0) * 1e3)
        out["plan_once"] = {"first_call_ms": round(walls[0], 2), "next_call_ms": round(walls[1], 2),
                            "plan_ms": round(walls[0] - walls[1], 2)}
        for policy in (0, 1, 2):
            ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, policy)
            ms_g = timed(lambda: run.run_grouped(w.steps, "ozaki_bf16", SLICES), args.steps)
            ms_s = timed(lambda: run.run("ozaki_bf16", SLICES), args.steps)
            run.run_grouped(w.steps, "ozaki_bf16", SLICES)
            ctx.sync()
            ctx.graph_begin()
            try:
                run.run_grouped(w.steps, "ozaki_bf16", SLICES)
            finally:
                g = ctx.graph_end()
            ms_graph = timed(g.launch, args.steps)
            out[f"tile_policy_{policy}"] = {
                "grouped_ms": round(ms_g, 3), "separate_ms": round(ms_s, 3), "graph_ms": round(ms_graph, 3),
                "graph_kernels": g.kernel_launches, "TFLOP/s_graph": round(flops / ms_graph / 1e9, 3)}
            g.destroy()
        ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, 1)
        ms64 = timed(lambda: run.run("f64", 0), max(1, min(args.steps, 2)))
    out["f64_ms"] = round(ms64, 3)
    out["f64_TFLOP/s"] = round(flops / ms64 / 1e9, 4)
    return out


def run_batch_case(args) -> dict:
    """The 32 independent ladders R = 1/2 V_vvvv T of sizes O in [16, 64], V in [64, 320] (tiles 20/40),
    in sub-batches that fit the free HBM; each sub-batch runs as one contraction group captured in a CUDA
    graph.  The stored V_vvvv of all 32 (162 GB in FP64 for these sizes) plus their slice images exceed
    one GPU, so sub-batches run one after another; inputs are seeded normals drawn on the device
    (torch generator, sigma 0.1 / 0.01): a throughput measurement (parity of the same path is tested on
    the scaled batch and on the O=64 V=384 irrep problem)."""
    import gc

    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    sizes = wl.ladder_batch_sizes()
    stream = torch.cuda.Stream(0)
    ctx = tg.Context(0, stream=stream)
    free, _ = torch.cuda.mem_get_info(0)
    budget = 0.8 * free
    per = [wl.batch_memory_bytes(o, v, SLICES) * 1.08 for o, v in sizes]  # + tile padding
    subs, cur, acc = [], [], 0.0
    for k, b in enumerate(per):
        if cur and acc + b > budget:
            subs.append(cur)
            cur, acc = [], 0.0
        cur.append(k)
        acc += b
    subs.append(cur)
    gen = torch.Generator(device="cuda:0")
    total_flops, total_ms, report = 0.0, 0.0, []
    for sub in subs:
        with torch.cuda.stream(stream):
            probs = []
            for k in sub:
                o, v = sizes[k]
                w = wl.ladder_problem(o, v, wl.SEED_BASE + 300 + k)
                sp, T = gw.build(ctx, w, fill=False)
                for name, sigma in (("V_vvvv", 0.1), ("T", 0.01)):
                    gen.manual_seed(wl.SEED_BASE + 1000 * k + (1 if name == "V_vvvv" else 2))
                    T[name].data.normal_(0.0, sigma, generator=gen)
                probs.append((w, T))
            flops = sum(ctx.flops(T["R"], "abij", T["V_vvvv"], "abef", T["T"], "efij") for _, T in probs)

            def step():
                with ctx.group():
                    for _, T in probs:
                        ctx.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij", "ozaki_bf16",
                                     SLICES)

            step()  # plans and the group's scratch
            ctx.sync()
            ctx.graph_begin()
            try:
                step()
            finally:
                g = ctx.graph_end()
            for _ in range(max(1, args.warmup)):
                g.launch()
            ctx.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                g.launch()
            b.record(stream)
            ctx.sync()
            ms = a.elapsed_time(b) / args.steps
        report.append({"problems": len(sub), "nonzero_block_flops": flops, "graph_ms": round(ms, 3),
                       "graph_kernels": g.kernel_launches, "TFLOP/s": round(flops / ms / 1e9, 3)})
        total_flops += flops
        total_ms += ms
        g.destroy()
        del probs, T, sp
        gc.collect()
        torch.cuda.empty_cache()
    return {"case": "32 independent vvvv ladders, O in [16,64], V in [64,320], tiles 20/40, split precision "
                    f"({SLICES} slices), sub-batches of one grouped launch in one CUDA graph each",
            "sizes": sizes, "sub_batches": report, "nonzero_block_flops": total_flops,
            "ms": round(total_ms, 3), "TFLOP/s": round(total_flops / total_ms / 1e9, 3)}


def _device_fill(T, spec, seed):
    import torch

    gen = torch.Generator(device=T.data.device)
    gen.manual_seed(seed)
    T.data.normal_(0.0, spec.sigma, generator=gen)


def run_doubles_o80_case(args) -> dict:
    """The O=80 V=320 doubles contractions at full size (tiles 40/64; V_vvvv 31.5 GB): ladder, oooo and ring each
    autotuned for 1e-10, timed alone in split precision and in FP64.  Inputs are seeded normals drawn on
    the device (the host generator would take minutes for 4e9 elements); parity of this size is tested
    on sampled sub-blocks with the host-generated inputs."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    w = wl.ccsd_doubles_o80_v320()
    ctx = tg.Context(0)
    sp, T = gw.build(ctx, w, fill=False)
    for k, (name, spec) in enumerate(w.tensors.items()):
        if spec.sigma:
            _device_fill(T[name], spec, w.seed * 16 + k)
    run = gw.Runner(ctx, w, sp, T)
    run.run("f64")  # intermediates (W) hold the values the contractions see
    ctx.sync()
    out = {"case": f"{w.name}: vvvv ladder, oooo ladder, ring with P(ab)P(ij); split precision autotuned "
                   "for rel err 1e-10, and FP64", "contractions": {}}
    stream = torch.cuda.current_stream()
    for st in w.steps:
        if not isinstance(st, wl.ContractSpec):
            continue
        tuned = run.autotune(1e-10, steps=[st])[st.name]
        res = {"nonzero_block_flops": run.flops(st), "autotuned": tuned}
        for prec, reps in (("ozaki_bf16", max(1, args.steps)), ("f64", 1)):
            run.run(prec, 0, steps=[st])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run.run(prec, 0, steps=[st])
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps
            key = "split" if prec == "ozaki_bf16" else "f64"
            res[f"{key}_ms"] = round(t, 3)
            res[f"{key}_TFLOP/s"] = round(res["nonzero_block_flops"] / t / 1e9, 3)
        out["contractions"][st.name] = res
    return out


def run_dense4d_case(args) -> dict:
    """The paper's dense 4-D benchmark C(a,b,c,d) = A(a,b,m,n) B(m,n,c,d) (Sec. V), every extent N, on
    one GPU in split precision (6 slices); FP64 as well when N <= 128.  Inputs are device-seeded normals."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    N, tile = (int(x) for x in args.dense4d.split(","))
    w = wl.dense4d(N, tile)
    ctx = tg.Context(0)
    sp, T = gw.build(ctx, w, fill=False)
    for k, name in enumerate(("A", "B")):
        _device_fill(T[name], w.tensors[name], w.seed * 16 + k)
    run = gw.Runner(ctx, w, sp, T)
    st = w.steps[0]
    flops = run.flops(st)
    stream = torch.cuda.current_stream()
    out = {"case": f"{w.name}: C(abcd) = A(abmn) B(mncd), all blocks stored", "nonzero_block_flops": flops}
    precs = [("ozaki_bf16", max(1, args.steps))] + ([("f64", 1)] if N <= 128 else [])
    results = {}
    for prec, reps in precs:
        run.run(prec, SLICES if prec == "ozaki_bf16" else 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run.run(prec, SLICES if prec == "ozaki_bf16" else 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        results[prec] = T["C"].download() if N <= 128 else None
        key = "split" if prec == "ozaki_bf16" else "f64"
        out[f"{key}_ms"] = round(t, 3)
        out[f"{key}_TFLOP/s"] = round(flops / t / 1e9, 3)
    if results.get("f64") is not None:
        a, b = results["ozaki_bf16"], results["f64"]
        out["split_rel_err_vs_f64"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return out


def run_cholesky_case(args) -> dict:
    """The ladder R = 1/2 V T with V_vvvv never stored: a lambda tensor formed slab by slab from 560
    Cholesky vectors (Eq. cc12) inside the contraction, O=40 V=240 (tiles 20/40).  Split precision
    (6 slices, formation included) and FP64; flops count forming V once plus the ladder."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    w = wl.cholesky_ladder_o40_v240()
    ctx = tg.Context(0)
    sp, T = gw.build(ctx, w, slab_bytes=int(args.slab_gb * (1 << 30)))
    run = gw.Runner(ctx, w, sp, T)
    st = w.steps[0]
    V = T["V_chol"]
    flops = run.flops(st)
    out = {"case": f"{w.name}: R = 1/2 V_vvvv T, V_vvvv formed on the fly from Cholesky vectors",
           "V_vvvv_bytes_not_stored": V.n_elems * 8, "slab_buffer_bytes": V.buffer_bytes, "slabs": V.n_slabs,
           "form_flops": V.form_flops, "ladder_flops": flops - V.form_flops, "nonzero_block_flops": flops}
    stream = torch.cuda.current_stream()
    results = {}
    for prec, reps in (("ozaki_bf16", max(1, args.steps)), ("f64", 1)):
        run.run(prec, SLICES if prec == "ozaki_bf16" else 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run.run(prec, SLICES if prec == "ozaki_bf16" else 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        results[prec] = T["R"].download()
        key = "split" if prec == "ozaki_bf16" else "f64"
        out[f"{key}_ms"] = round(t, 3)
        out[f"{key}_TFLOP/s"] = round(flops / t / 1e9, 3)
    a, b = results["ozaki_bf16"], results["f64"]
    out["split_rel_err_vs_f64"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    ctx.profile(True)
    run.run("ozaki_bf16", SLICES)
    prof = ctx.profile_read()
    ctx.profile(False)
    out["split_kernel_ms"] = {k: round(v[0], 3) for k, v in prof.items() if v[1]}
    out["split_kernel_launches"] = {k: v[1] for k, v in prof.items() if v[1]}
    return out


def run_doubles_term_case(args) -> dict:
    """One contraction of the doubles recipe at a chosen size (tiles 20/40), split precision (6 slices):
    small cases for profiling a single term."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    O_, V_, name = args.term.split(",")
    w = wl._doubles(wl._vt(2, int(O_), int(V_), 20, 40, f"ccsd_doubles_O{O_}_V{V_}"))
    w.steps = wl.doubles_steps()
    ctx = tg.Context(0)
    sp, T = gw.build(ctx, w)
    run = gw.Runner(ctx, w, sp, T)
    run.run("f64")
    st = next(x for x in w.steps if x.name == name)
    if args.term_config:
        chunk, policy, persistent, mode = (int(x) for x in args.term_config.split(","))
        for opt, val in ((tg.TAMM_OPT_OZAKI_CHUNK_K, chunk), (tg.TAMM_OPT_OZAKI_TILE_POLICY, policy),
                         (tg.TAMM_OPT_OZAKI_PERSISTENT, persistent), (tg.TAMM_OPT_OZAKI_SHARED_SCALE, int(mode == 1)),
                         (tg.TAMM_OPT_OZAKI_FUSED_A, int(mode == 2))):
            ctx.set_option(opt, val)
        slices = 6
        tuned = {"slices": 6, "chunk_k": chunk, "tile_policy": policy, "persistent": persistent, "mode": mode}
    else:
        tuned = run.autotune(1e-10, steps=[st])[st.name]  # slices, chunk, tile policy, grid and scaling
        slices = 0
    for _ in range(max(1, args.warmup)):
        run.run("ozaki_bf16", slices, steps=[st])
    ctx.sync()
    ctx.profile_read()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for _ in range(args.steps):
        run.run("ozaki_bf16", slices, steps=[st])
    e1.record()
    torch.cuda.nvtx.range_pop()
    ctx.sync()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    return {"case": f"{w.name} {name}, split precision, " + ("fixed configuration" if args.term_config else "autotuned"),
            "ms": round(ms, 3),
            "TFLOP/s": round(run.flops(st) / ms / 1e9, 3), "nonzero_block_flops": run.flops(st), "tuned": tuned,
            "kernel_ms": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]}}


def run_triples_case(args) -> dict:
    """The perturbative triples correction E(T) (Sec. IV.B, Eqs. cc14, tensort, tensort2) of the ``triples``
    recipe (default O=32 V=160, tiles 16/80): split precision (4..6 slices, the fastest configuration whose
    E(T) is within 5e-11 of the FP64 value) and FP64, CUDA events per
    evaluation, kernel classes timed by the library.  Throughput counts the block-GEMM flops of the U
    accumulations (2 M N K over stored block pairs); the fused energy kernel's time is included."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    O_, V_, to, tv = (int(x) for x in (args.triples or "32,160,16,80").split(","))
    w = wl.triples(O_, V_, to, tv)
    ctx = tg.Context(0)
    _, T = gw.build(ctx, w)
    eo, ev = wl.orbital_energies(w)
    deo = torch.tensor(eo, dtype=torch.float64, device="cuda:0")
    dev = torch.tensor(ev, dtype=torch.float64, device="cuda:0")
    out_e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    ins = (T["T"], T["t1"], T["V_ooov"], T["V_vovv"], T["V_oovv"])
    info = ctx.triples_info(*ins)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    out = {"case": f"{w.name}: E(T) fused to a scalar, tiles {to}/{tv}", "n_triples": info["n_triples"],
           "gemm_flops": info["gemm_flops"], "n_batches": info["n_batches"]}
    energies = {}

    def timed_run(prec, slices, reps, warm):
        run = lambda: ctx.triples_energy(*ins, deo.data_ptr(), dev.data_ptr(), out_e.data_ptr(), prec, slices)
        for _ in range(warm):
            run()
        ctx.sync()
        ctx.profile_read()
        ctx.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.profile(False)
        return e0.elapsed_time(e1) / reps, ctx.profile_read(), float(out_e.item())

    # FP64 first: its E(T) is the reference the split configurations are held to
    ms64, prof64, energies["f64"] = timed_run("f64", 0, 1, 1)
    out["f64_ms"] = round(ms64, 3)
    out["f64_TFLOP/s"] = round(info["gemm_flops"] / ms64 / 1e9, 3)
    out["f64_kernel_ms"] = {k: round(v[0], 3) for k, v in prof64.items() if v[1]}
    # split precision: slice count, tile policy (output columns per work item), grid kind and scaling picked
    # by timing like the autotuner, among the configurations whose E(T) is within half the 1e-10 target of
    # the FP64 value (the slice count and the scaling change the arithmetic; the rest only the work split)
    cfg_ms, cfg_err = {}, {}
    fixed = tuple(int(x) for x in args.triples_config.split(",")) if getattr(args, "triples_config", "") else None
    for slices in ((fixed[0],) if fixed else (6, 5, 4)):
        for policy in ((fixed[1],) if fixed else (1, 3)):
            for persistent in ((fixed[2],) if fixed else (0, 1)):
                for shared in ((fixed[3],) if fixed else (0, 1)):
                    ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, policy)
                    ctx.set_option(tg.TAMM_OPT_OZAKI_PERSISTENT, persistent)
                    ctx.set_option(tg.TAMM_OPT_OZAKI_SHARED_SCALE, shared)
                    t, _, e = timed_run("ozaki_bf16", slices, 1, 1)
                    cfg_ms[(slices, policy, persistent, shared)] = t
                    cfg_err[(slices, policy, persistent, shared)] = abs(e - energies["f64"]) / abs(energies["f64"])
    ok = [k for k in cfg_ms if cfg_err[k] <= 0.5e-10]
    best = min(ok or list(cfg_ms), key=cfg_ms.get)
    for opt, val in zip((tg.TAMM_OPT_OZAKI_TILE_POLICY, tg.TAMM_OPT_OZAKI_PERSISTENT, tg.TAMM_OPT_OZAKI_SHARED_SCALE),
                        best[1:]):
        ctx.set_option(opt, val)
    out["split_config_ms"] = {f"slices{k[0]}_policy{k[1]}_persistent{k[2]}_shared{k[3]}": round(v, 3)
                              for k, v in cfg_ms.items()}
    out["split_config_rel_err"] = {f"slices{k[0]}_policy{k[1]}_persistent{k[2]}_shared{k[3]}": float(f"{v:.3g}")
                                   for k, v in cfg_err.items()}
    out["split_config"] = {"slices": best[0], "tile_policy": best[1], "persistent": best[2], "shared_scale": best[3]}
    s_best = best[0]
    ms, prof, energies["split"] = timed_run("ozaki_bf16", s_best, max(1, args.steps), max(1, args.warmup))
    out["split_ms"] = round(ms, 3)
    out["split_TFLOP/s"] = round(info["gemm_flops"] / ms / 1e9, 3)
    out["split_kernel_ms"] = {k: round(v[0] / max(1, args.steps), 3) for k, v in prof.items() if v[1]}
    g_ms = prof["gemm_ozaki"][0] / max(1, args.steps)
    tf = info["gemm_flops"] * s_best * (s_best + 1) // 2 / (g_ms * 1e-3) / 1e12 if g_ms else None
    out["split_gemm_roofline"] = {"achieved": round(tf, 1) if tf else None, "unit": "TFLOP/s",
                                  "peak": peaks["bf16_tflops_sustained"],
                                  "frac": round(tf / peaks["bf16_tflops_sustained"], 4) if tf else None,
                                  "peak_source": f"{peaks['_source']} bf16_tflops_sustained"}
    out["energy"] = energies
    out["split_rel_err_vs_f64"] = abs(energies["split"] - energies["f64"]) / abs(energies["f64"])
    return out


def run_residual_case(args) -> dict:
    """One full CCSD residual (T1 and T2 equations, Stanton-Gauss intermediates, the energy and the
    residual norms: 55 library operations in 11 dependency levels) at O=40 V=240, tiles 20/40 by default:
    operation by operation, through the scheduler (each level's split-precision contractions as one
    grouped launch), and that scheduled run captured in one CUDA graph; split precision (every contraction
    autotuned for 1e-10; also six slices with the default options, operation by operation) and FP64.  Inputs are seeded normals drawn on the device.  Throughput counts the nonzero-block flops of
    the 36 contractions."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    O_, V_, to, tv = (int(x) for x in (args.residual or "40,240,20,40").split(","))
    w = wl.ccsd_residual(O_, V_, to, tv)
    stream = torch.cuda.Stream(0)
    ctx = tg.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        sp, T = gw.build(ctx, w, fill=False)
        for k, (name, spec) in enumerate(w.tensors.items()):
            if spec.sigma:
                _device_fill(T[name], spec, w.seed * 64 + k)
        run = gw.Runner(ctx, w, sp, T)
        flops = sum(run.flops(st) for st in w.steps if isinstance(st, wl.ContractSpec))
        e = torch.zeros(8, dtype=torch.float64, device="cuda:0")

        def timed(fn, k, warm):
            for _ in range(warm):
                fn()
            ctx.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                fn()
            b.record(stream)
            ctx.sync()
            return a.elapsed_time(b) / k

        out = {"case": f"{w.name}: CCSD T1 + T2 residual, energy and norms, tiles {to}/{tv}", "operations": len(w.steps),
               "contractions": sum(isinstance(st, wl.ContractSpec) for st in w.steps), "nonzero_block_flops": flops}
        k = max(1, args.steps)
        # FP64 first: the reference, and the values every intermediate holds when the autotuner looks at it
        ms64 = timed(lambda: run.run("f64", 0, energy_out=e.data_ptr()), 1, 1)
        r2_64 = T["R2"].download()
        e_64 = e.cpu().numpy()[:4].copy()
        # six slices with the context's default options, operation by operation
        ms_fixed = timed(lambda: run.run("ozaki_bf16", SLICES, energy_out=e.data_ptr()), k, max(1, args.warmup))
        # every contraction autotuned (slices, chunk, tile policy, grid, scaling) for 1e-10, then slices = 0
        run.run("f64", 0, energy_out=e.data_ptr())
        t0 = time.time()
        tuned = run.autotune(1e-10)
        out["autotune_seconds"] = round(time.time() - t0, 2)
        out["autotuned_slices"] = sorted({v["slices"] for v in tuned.values()})
        ms_seq = timed(lambda: run.run("ozaki_bf16", 0, energy_out=e.data_ptr()), k, max(1, args.warmup))
        sch = run.scheduled("ozaki_bf16", 0, energy_out=e.data_ptr())
        out["levels"] = max(sch.levels()) + 1
        ms_sch = timed(sch.execute, k, 1)
        ctx.profile_read()
        ctx.profile(True)
        sch.execute()
        ctx.sync()
        ctx.profile(False)
        prof = ctx.profile_read()
        with ctx.capture() as cap:
            sch.execute()
        g = cap.graph
        ms_graph = timed(g.launch, k, 1)
        r2_split = T["R2"].download()
        e_split = e.cpu().numpy()[:4].copy()
    out.update({
        "split_fixed6_sequential_ms": round(ms_fixed, 3),
        "split_fixed6_sequential_TFLOP/s": round(flops / ms_fixed / 1e9, 3),
        "split_sequential_ms": round(ms_seq, 3), "split_scheduled_ms": round(ms_sch, 3),
        "split_graph_ms": round(ms_graph, 3), "graph_kernels": g.kernel_launches,
        "split_sequential_TFLOP/s": round(flops / ms_seq / 1e9, 3),
        "split_scheduled_TFLOP/s": round(flops / ms_sch / 1e9, 3),
        "split_graph_TFLOP/s": round(flops / ms_graph / 1e9, 3),
        "f64_ms": round(ms64, 3), "f64_TFLOP/s": round(flops / ms64 / 1e9, 4),
        "scheduled_kernel_ms": {kk: round(v[0], 3) for kk, v in prof.items() if v[1]},
        "split_rel_err_vs_f64": {"R2": float(np.linalg.norm(r2_split - r2_64) / np.linalg.norm(r2_64)),
                                 "energy_t2": float(abs(e_split[0] - e_64[0]) / abs(e_64[0]))},
    })
    g.destroy()
    return out


def run_gradients_case(args) -> dict:
    """Differentiation (O=32 V=192, tiles 16/32): E = 1/4 V_oovv(ijab) T'(abij), T' = T + 1/2 V_vvvv(abef) T(efij),
    forward and backward through torch.autograd (the hand-written adjoint: two adjoint contractions and two
    scaled permuted adds), split precision (6 slices), BF16x3 and FP64, storing T' or recomputing it.  Each
    pass ends with the library's status check.  Throughput counts the three contractions (forward ladder and
    the two adjoint GEMMs, 2 M N K over stored block pairs)."""
    import torch

    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import autograd as ga
    from paper_2201_01257_gb300 import workload as gw
    from tamm_synth import workloads as wl

    w = wl.ladder_energy_o32_v192()
    ctx = tg.Context(0)
    _, T = gw.build(ctx, w)
    run = gw.Runner(ctx, w, _, T)
    ladder = next(st for st in w.steps if st.name == "ladder")
    flops = 3 * run.flops(ladder)  # forward ladder + dT and dV_vvvv adjoints (same block pairs)
    stream = torch.cuda.current_stream()
    out = {"case": f"{w.name}: E and dE/dT, dE/dV_vvvv, dE/dV_oovv through torch.autograd",
           "contraction_flops_per_pass": flops}
    grads = {}
    for prec, slices, recompute, reps in (("ozaki_bf16", SLICES, False, max(1, args.steps)),
                                         ("ozaki_bf16", SLICES, True, max(1, args.steps)),
                                         ("bf16x3", 0, False, max(1, args.steps)), ("f64", 0, False, 1)):
        def step():
            v = T["V_vvvv"].data.detach().requires_grad_(True)
            t = T["T"].data.detach().requires_grad_(True)
            voo = T["V_oovv"].data.detach().requires_grad_(True)
            E = ga.ladder_energy(ctx, T["V_vvvv"], v, T["T"], t, T["V_oovv"], voo, prec, slices, recompute)
            E.backward()
            return E, v, t, voo
        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            E, v, t, voo = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        key = f"{prec}{'_recompute' if recompute else ''}"
        out[f"{key}_ms"] = round(ms, 3)
        out[f"{key}_TFLOP/s"] = round(flops / ms / 1e9, 3)
        grads[key] = {"E": float(E.item()), "T": t.grad.detach().cpu().numpy(), "V": v.grad.detach().cpu().numpy()}
    ref = grads["f64"]
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out["rel_err_vs_f64"] = {k: {"E": abs(g["E"] - ref["E"]) / abs(ref["E"]), "dT": rel(g["T"], ref["T"]),
                                 "dV_vvvv": rel(g["V"], ref["V"])} for k, g in grads.items() if k != "f64"}
    return out


def _oracle_row(name: str) -> dict:
    """One CPU-baseline row: the FP64 oracle, as it stands, on one workload (OMP_NUM_THREADS sets its cores)."""
    import oracle as O
    import tamm_synth
    from tamm_synth import workloads as wl

    def fill(w, T, names, blocks=None):
        for n in names:
            spec, X = w.tensors[n], T[n]
            lo, ext = X.block_lo_ext()
            idx = np.arange(X.n_blocks) if blocks is None or n not in blocks else np.array(sorted(blocks[n]))
            if len(idx):
                tamm_synth.fill_boxes(w.seed, spec.stream, spec.sigma, X.dense_shape(), spec.anti01, spec.anti23,
                                      lo[idx], ext[idx], X.block_off[idx], X.data)

    def tensors(w, names):
        sp = {k: O.Space.from_spec(v) for k, v in w.spaces.items()}
        return {n: O.Tensor([sp[m] for m in w.tensors[n].modes], w.tensors[n].n_upper, w.tensors[n].sym)
                for n in names}

    if name == "ladder_O8_V32":  # configuration 1, in full
        w = wl.ladder_o8_v32()
        T = tensors(w, ("V_vvvv", "T", "R"))
        fill(w, T, ("V_vvvv", "T"))
        t0 = time.perf_counter()
        O.contract(0.5, T["R"], "abij", 0.0, T["V_vvvv"], "abef", T["T"], "efij")
        return {"seconds": time.perf_counter() - t0, "flops": 2.097152e7}
    if name == "oooo_O40_V240":  # the configuration-2 oooo ladder, in full
        w = wl.ccsd_doubles_o40_v240()
        T = tensors(w, ("T", "W0", "R"))
        fill(w, T, ("T", "W0"))
        t0 = time.perf_counter()
        O.contract(0.25, T["R"], "abij", 0.0, T["T"], "abmn", T["W0"], "mnij")
        return {"seconds": time.perf_counter() - t0, "flops": 4.608e10}
    if name == "gradients_O32_V192":  # configuration 4: forward and the closed-form reference gradient
        w = wl.ladder_energy_o32_v192()
        T = tensors(w, ("V_vvvv", "T", "V_oovv"))
        fill(w, T, ("V_vvvv", "T", "V_oovv"))
        t0 = time.perf_counter()
        Tp = O.Tensor(T["T"].modes, 2)
        Tp.data[:] = T["T"].data
        O.contract(0.5, Tp, "abij", 1.0, T["V_vvvv"], "abef", T["T"], "efij")
        O.energy(0.25, T["V_oovv"], "ijab", Tp, "abij")
        G = O.Tensor(T["T"].modes, 2)
        O.add(0.25, G, "abij", 0.0, T["V_oovv"], "ijab")
        dT = O.Tensor(T["T"].modes, 2)
        dT.data[:] = G.data
        O.contract(0.5, dT, "efij", 1.0, T["V_vvvv"], "abef", G, "abij")
        dV = O.Tensor(T["V_vvvv"].modes, 2)
        O.contract(0.5, dV, "abef", 0.0, G, "abij", T["T"], "efij")
        return {"seconds": time.perf_counter() - t0, "flops": 3 * 4.349e11}
    if name == "doubles_O80_V320_sample":  # configuration 5: 256 seeded 8^4 sub-blocks (ladder, ring, oooo)
        w = wl.ccsd_doubles_o80_v320()
        T = tensors(w, ("V_vvvv", "T", "W0", "V_ovvo", "R"))
        rng = np.random.default_rng(5)
        R = T["R"]
        _, ext = R.block_lo_ext()
        pool = [int(x) for x in rng.permutation(R.n_blocks)[:2]]  # boxes from two output blocks: few V blocks
        terms = {"ladder": (0.5, "V_vvvv", "abef", "T", "efij"), "oooo": (0.25, "T", "abmn", "W0", "mnij"),
                 "ring": (1.0, "T", "aeim", "V_ovvo", "mbej")}
        boxes = {k: [] for k in terms}
        for _ in range(256):
            k = ["ladder", "ring", "oooo"][int(rng.integers(3))]
            b = pool[int(rng.integers(len(pool)))]
            boxes[k].append((b, [int(rng.integers(0, e - 8 + 1)) for e in ext[b]]))
        need = {"V_vvvv": set()}
        tv = [T["V_vvvv"].modes[0].tiles[t] for t in range(T["V_vvvv"].modes[0].n_tiles)]
        for b, _ in boxes["ladder"]:
            ta, tb = R.block_tiles[b][0], R.block_tiles[b][1]
            for te in range(len(tv)):
                for tf in range(len(tv)):
                    vb = T["V_vvvv"].find_block([ta, tb, te, tf])
                    if vb >= 0:
                        need["V_vvvv"].add(vb)
        fill(w, T, ("V_vvvv", "T", "W0", "V_ovvo"), need)
        t0 = time.perf_counter()
        fl = 0.0
        for k, (al, a, la, bb, lb) in terms.items():
            if boxes[k]:
                O.contract_boxes(al, R, "abij", T[a], la, T[bb], lb, [x[0] for x in boxes[k]], [x[1] for x in boxes[k]],
                                 [[8] * 4] * len(boxes[k]))
        dt = time.perf_counter() - t0
        # flops of the sample: 2 x 8^4 x (stored summed extent of the box's output block) per box
        import itertools

        for k, (al, a, la, bb, lb) in terms.items():
            lab = {}
            for X, l in ((R, "abij"), (T[a], la), (T[bb], lb)):
                for m, ch in enumerate(l):
                    lab[ch] = X.modes[m]
            summed = [ch for ch in la if ch not in "abij"]
            for b, _ in boxes[k]:
                tile = {ch: int(R.block_tiles[b, m]) for m, ch in enumerate("abij")}
                keff = 0
                for kt in itertools.product(*[range(lab[ch].n_tiles) for ch in summed]):
                    tile.update(dict(zip(summed, kt)))
                    if T[a].find_block([tile[ch] for ch in la]) < 0 or T[bb].find_block([tile[ch] for ch in lb]) < 0:
                        continue
                    keff += int(np.prod([lab[ch].tiles[tile[ch]][1] for ch in summed]))
                fl += 2.0 * 8 ** 4 * keff
        full = 2.097e13 + 5.243e12 + 1.311e12  # ladder, ring, oooo over all stored blocks
        return {"seconds": dt, "flops": fl, "full_flops": full, "extrapolated_full_seconds": dt * full / fl}
    raise ValueError(name)


def run_cpu_rows(args) -> dict:
    """The CPU-baseline rows: the FP64 oracle, as it stands, on the machine's host cores (all of them, and one
    core where asked): configuration 1 in full, the configuration-2 oooo ladder in full, configuration 4
    forward and reference gradient, and configuration 5's 256 seeded 8^4 sub-blocks with the full time
    extrapolated.  Each row runs in a child process so that OMP_NUM_THREADS takes effect."""
    cores = os.cpu_count() or 1
    rows = {}
    plan = [("ladder_O8_V32", cores), ("ladder_O8_V32", 1), ("oooo_O40_V240", cores), ("oooo_O40_V240", 1),
            ("gradients_O32_V192", cores), ("doubles_O80_V320_sample", cores)]
    for name, n in plan:
        env = dict(os.environ, OMP_NUM_THREADS=str(n))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-row", name], env=env,
                           capture_output=True, text=True, check=True)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        d["cores"] = n
        d["TFLOP/s"] = d["flops"] / d["seconds"] / 1e12
        rows[f"{name}_{n}core" + ("s" if n > 1 else "")] = d
    cpu = ""
    try:
        cpu = next(l.split(":", 1)[1].strip() for l in open("/proc/cpuinfo") if "model name" in l or "CPU part" in l)
    except (OSError, StopIteration):
        pass
    return {"case": "FP64 oracle (C, OpenMP over output blocks) on the host", "nproc": cores, "cpu": cpu,
            "rows": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="size of the CPU-baseline sample")
    ap.add_argument("--ref-seconds", type=float, default=6.0, help="CPU work per reference-arm step")
    ap.add_argument("--ladder", default="", help="O,V: time one split-precision ladder of that size instead")
    ap.add_argument("--slices", type=int, default=0,
                    help="split-precision slices per operand; 0 = autotune every contraction for 1e-10")
    ap.add_argument("--irrep-doubles", action="store_true", help="time the uneven-irrep grouped ladder + ring instead")
    ap.add_argument("--irrep", default="", help="O,V: with --irrep-doubles, spin-orbital counts (default 64,384)")
    ap.add_argument("--batch", action="store_true", help="time the 32 independent ladders in sub-batches instead")
    ap.add_argument("--doubles-o80", action="store_true", help="time the O=80 V=320 contractions alone instead")
    ap.add_argument("--dense4d", default="", help="N,tile: time the dense 4-D contraction instead")
    ap.add_argument("--term", default="", help="O,V,name: time one doubles contraction of that size instead")
    ap.add_argument("--term-config", default="", help="chunk,policy,persistent,mode: with --term, this split "
                    "configuration (6 slices; mode 0 per-block scaling, 1 shared, 2 A sliced in the GEMM) "
                    "instead of the autotuner's")
    ap.add_argument("--cholesky", action="store_true",
                    help="time the ladder with V_vvvv formed on the fly from Cholesky vectors instead")
    ap.add_argument("--slab-gb", type=float, default=0.0, help="with --cholesky: slab buffer bound (0 = default)")
    ap.add_argument("--cpu-rows", action="store_true", help="time the oracle's CPU-baseline rows instead")
    ap.add_argument("--cpu-row", default="", help=argparse.SUPPRESS)
    ap.add_argument("--gradients", action="store_true",
                    help="time the O=32 V=192 ladder-energy forward + backward through autograd instead")
    ap.add_argument("--residual", nargs="?", const="40,240,20,40", default="",
                    help="O,V,to,tv: time one full CCSD residual, sequential vs scheduled vs graph, instead")
    ap.add_argument("--triples-config", default="", help="slices,policy,persistent,shared: with --triples, this "
                    "split configuration instead of the sweep")
    ap.add_argument("--triples", nargs="?", const="32,160,16,80", default="",
                    help="O,V,to,tv: time the (T) correction instead (default 32,160,16,80)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.ladder:
        out = run_ladder_case(args)
    elif args.irrep_doubles:
        out = run_irrep_case(args)
    elif args.batch:
        out = run_batch_case(args)
    elif args.doubles_o80:
        out = run_doubles_o80_case(args)
    elif args.dense4d:
        out = run_dense4d_case(args)
    elif args.term:
        out = run_doubles_term_case(args)
    elif args.cholesky:
        out = run_cholesky_case(args)
    elif args.triples:
        out = run_triples_case(args)
    elif args.residual:
        out = run_residual_case(args)
    elif args.gradients:
        out = run_gradients_case(args)
    elif args.cpu_rows:
        out = run_cpu_rows(args)
    elif args.cpu_row:
        out = _oracle_row(args.cpu_row)
    elif args.impl == "reference":
        out = run_reference(args, rank)
    else:
        out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
