#!/usr/bin/env python3
"""Throughput of k-input RNS-CKKS ciphertext multiplication on GB300.

Workload (one "step"): for every k in 4..12, one batched k-input multiply of
16 independent products with Table II's partition, N = 2^16, 24 x 50-bit Q
primes, 8 x 60-bit P primes, dnum = 3, input level 24, evaluation keys
ek_2..ek_12 resident in HBM. 144 products per step. Inputs are uniform
residues (the distribution of RLWE ciphertexts) drawn on the device with a
seeded generator; they total ~27 GB, far above the 129 MB L2, so no L2 flush
is needed between steps.

Printed JSON line: value = products per second over the whole step (all N
ranks), e2e = the same with host buffers (pinned host -> device copies of the
step's inputs and device -> host copies of its outputs inside the timed
region), roofline of the dominant kernel class (CUDA-event timed inside the
timed region), per-k comparisons against chained standard 2-input
multiplies (Table VII's binary tree) and one product per launch, and the CPU
oracle timed on a bounded sample.

--impl reference times the CPU oracle (the only reference: the paper has no
code) on the same workload, one full-size k = 4 product per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "k-input ct-mults/s at N=2^16 (k=4..12, batch 16 per k)"
UNIT = "ct-mults/s"
KS = list(range(4, 13))
BATCH = 16
CONFIG = {
    "workload": "k-input CKKS multiply, N=2^16, L=24x50-bit q + K=8x60-bit p, dnum=3, level 24, "
                "k=4..12 (Table II partitions), batch 16 per k",
    "N": 65536, "L": 24, "K": 8, "dnum": 3, "level": 24, "ks": KS, "batch_per_k": BATCH,
    "products_per_step": BATCH * len(KS),
    "l2": "inputs (~27 GB) larger than L2; no flush",
}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "traffic.json")


PRIMES = {"chain": "the largest primes below 2^50 / 2^60 that are 1 mod 2^17 (the default reading)",
          "q1": "the largest primes below 2^50 / 2^60 that are 1 mod 2^32 (cheaper modular-product forms)"}


def congruence(args) -> int:
    import synth
    return synth.Q1_CONGRUENCE if args.primes == "q1" else synth.NTT_CONGRUENCE


def reduce_max(value: float, world: int, device=None) -> float:
    """Largest value over the ranks (the slowest rank's time); identity for
    one rank. Works with any initialised process group (nccl or gloo)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def binary_tree(k):
    if k == 1:
        return None
    a = 1 << (k - 1).bit_length() - 1
    if k == 2:
        return (1, 1)
    return (a, k - a)


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2601_15401_gb300 as G
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    params = synth.params_large(congruence=congruence(args))
    N, L, K = params.N, params.L, params.K
    ks = [int(x) for x in args.ks.split(",")] if args.ks else KS
    B = args.batch
    t_max = max(ks)
    ctx = G.Context.from_params(params, device=local_rank)

    # evaluation keys ek_2..ek_tmax, generated on the device from seeded draws
    g = synth.rng(3, 0, stream=1)
    s = torch.from_numpy(synth.ternary_secret(g, N)).to(dev)
    e = torch.from_numpy(__import__("numpy").stack(
        [[synth.gaussian(g, N) for _ in range(params.dnum)] for _ in range(t_max - 1)])).to(dev)
    a = synth.uniform_residues_torch(list(params.q) + list(params.p), (t_max - 1, params.dnum), N, 0x51, dev)
    keys = torch.empty((t_max - 1, params.dnum, 2, L + K, N), dtype=torch.uint64, device=dev)
    kws = torch.empty(ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device=dev)
    ctx.keygen_evk(t_max, s, a, e, keys, kws)
    del a, kws
    evk = ctx.evk_set(t_max, keys)

    # inputs / outputs per k (batched tensors [B][k][2][L][N])
    inp, outs, tup, otup, depth = {}, {}, {}, {}, {}
    ws_bytes = 0
    for k in ks:
        d = ctx.plan_describe(k)["depth"]
        depth[k] = d
        inp[k] = synth.uniform_residues_torch(params.q, (B, k, 2), N, 1000 + k + 97 * rank, dev)
        outs[k] = torch.empty((B, 2, L - d, N), dtype=torch.uint64, device=dev)
        tup[k] = [[G.Tuple(inp[k][b, u], 2, L, L, 1, 2.0 ** 50) for u in range(k)] for b in range(B)]
        otup[k] = [G.Tuple(outs[k][b], 2, L - d, L - d) for b in range(B)]
        ws_bytes = max(ws_bytes, ctx.workspace_size(k, L, B))
    ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.uint64, device=dev)
    torch.cuda.synchronize()
    tuned = None
    if args.tune:
        # fixed tunables (e.g. to profile the autotuner's choice without
        # running the autotuner)
        tuned = {}
        for kv in args.tune:
            key, val = kv.split("=")
            ctx.tune_set(key, int(val))
            tuned[key] = int(val)
    elif not args.no_tune:
        from paper_2601_15401_gb300.executor import autotune
        tuned = autotune(ctx, evk, k=8, batch=4)["choice"]

    stream = torch.cuda.current_stream()
    lat = {k: [] for k in ks}
    ex = None
    wave = None
    if args.engine == "waves":
        # the whole step (every k, every batch element) as one cross-shape
        # wave: each stage of all 144 products is one launch
        wave = G.Wave(ctx, [(tup[k][b], otup[k][b], None) for k in ks for b in range(B)], evk)
        wave_bufs = wave.buffers(dev)
        ws = None
        torch.cuda.empty_cache()
        wave.run(*wave_bufs, stream=stream)  # writes the job tables
        torch.cuda.synchronize()
    elif args.streams > 1:
        # the step through the batched executor: one group per k, groups
        # spread over streams, the whole step captured in one CUDA graph
        from paper_2601_15401_gb300.executor import BatchExecutor, MulRequest
        ex = BatchExecutor({16: (ctx, evk)}, n_streams=args.streams, device=dev)
        reqs = [MulRequest(16, k, L, None, 1000 * k + b) for k in ks for b in range(B)]
        ex.plan(reqs)
        for k in ks:
            gi = ex.slot_of[1000 * k][0]
            ex.groups[gi].inp.copy_(inp[k])
        ws = None
        torch.cuda.empty_cache()
        ex.capture()

    def step(record=False):
        if ex is not None:
            ex.replay()
            return []
        if wave is not None:
            wave.run(*wave_bufs, stream=stream)
            return []
        evs = []
        for k in ks:
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            ctx.mul_k_batch(tup[k], evk, otup[k], ws, stream=stream)
            if record:
                e1.record(stream)
                evs.append((k, e0, e1))
        return evs

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.check()
    q1_forms = all(int(x) % (1 << 32) == 1 for x in list(params.q) + list(params.p)) and \
        ctx.tune_get("q1_forms") == 1
    int_peaks = measure_int_peaks(G, params, q1_forms)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ctx.counters(reset=True)
    ctx.profile(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    all_evs = []
    t0.record(stream)
    for _ in range(args.steps):
        all_evs += step(record=True)
    t1.record(stream)
    t1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.profile(False)
    ms_total = t0.elapsed_time(t1)
    prof = ctx.profile_read()
    launches = ctx.counters()["kernels"]
    ctx.check()
    for k, e0, e1 in all_evs:
        lat[k].append(e0.elapsed_time(e1))
    ms_step = reduce_max(ms_total / args.steps, world, dev)
    products = B * len(ks) * world
    value = products / (ms_step / 1e3)

    # dominant kernel class and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"]) if prof else (None, None)
    roofline = None
    if dom[0]:
        st = dom[1]
        achieved_gbs = st["alg_bytes"] / (st["total_ms"] / 1e3) / 1e9
        traffic = None
        busy = None
        try:
            ts = json.load(open(PROFILE_SUMMARY))
            ent = ts.get("kernels", {}).get(dom[0])
            if ent and ent.get("source_hash") == source_hash(dom[0]):
                # DRAM bytes per algorithmic byte from an ncu capture of this
                # kernel class, scaled to this run's launches
                traffic = round(ent["dram_bytes_per_alg_byte"] * st["alg_bytes"] / st["launches"])
                busy = ent.get("fmaheavy_busy")
        except Exception:
            pass
        unit_peak = int_peaks.get(op_unit(dom[0]))
        achieved_ops = st["int_ops"] / (st["total_ms"] / 1e3) / 1e9
        roofline = {"bound": "alu", "kernel": dom[0],
                    "achieved": round(achieved_ops, 2), "peak": round(unit_peak / 1e9, 2) if unit_peak else None,
                    "unit": "G Shoup products/s" if dom[0].startswith("ntt") else "G 128-bit MACs/s",
                    "frac": round(achieved_ops * 1e9 / unit_peak, 4) if unit_peak else None,
                    "traffic": traffic,
                    "peak_source": "measured in this run (ckks_peak_int: register-only stream of lazy NTT butterflies "
                                   "/ 128-bit MACs over every SM, CUDA events, best of 5), the integer-multiply "
                                   "roofline of this GPU for the operation the kernel is built from"
                                   + (", the butterfly in the Shoup form for primes = 1 mod 2^32 that the kernels run"
                                      if q1_forms else ""),
                    "alg_ops_per_launch": st["int_ops"] / st["launches"],
                    "alg_bytes_per_launch": st["alg_bytes"] / st["launches"],
                    "avg_launch_us": st["total_ms"] * 1e3 / st["launches"],
                    "hbm": {"achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                            "frac": round(achieved_gbs / hbm_peak, 4),
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"},
                    "fmaheavy_busy": busy,
                    "limiter": "integer multiply (fmaheavy) pipe and the latency around it, not HBM: ncu shows the "
                               "pipe 63-72 % busy in the NTT phases (95 % in the register-only butterfly stream the "
                               "peak comes from), 59-61 of its instructions per element for 4 butterflies, the rest "
                               "of the issue slots lost to long-scoreboard and dependent-multiply stalls, DRAM at a "
                               "quarter of peak and traffic at most the algorithmic bytes "
                               "(profiles/ntt_phase_N65536_batch8.md, int_peaks_gb300.md)"}
    def int_frac(n, v):
        pk = int_peaks.get(op_unit(n))
        return round(v["int_ops"] / (v["total_ms"] / 1e3) / pk, 4) if pk and v["int_ops"] else None

    kernel_table = {n: {"launches": v["launches"] // args.steps, "ms_per_step": round(v["total_ms"] / args.steps, 3),
                        "share": round(v["total_ms"] / sum(x["total_ms"] for x in prof.values()), 4),
                        "GBps": round(v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9, 1),
                        "hbm_frac": round(v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9 / hbm_peak, 4),
                        "int_frac": int_frac(n, v)}
                    for n, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"])}
    # whole-step algorithmic bytes: inputs + outputs + keys once per step
    in_bytes = sum(B * k * 2 * L * N * 8 for k in ks)
    out_bytes = sum(B * 2 * (L - depth[k]) * N * 8 for k in ks)
    lat_all = [x for k in ks for x in lat[k]] or [ms_step]
    per_k = {}
    for k in ks:
        if not lat[k]:
            # the step ran as one wave: time each k's batched call alone
            # (outside the timed region) for the per-k comparisons
            wsk = torch.empty(ctx.workspace_size(k, L, B) // 8 + 1, dtype=torch.uint64, device=dev)
            for r in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.mul_k_batch(tup[k], evk, otup[k], wsk, stream=stream)
                e1.record(stream)
                e1.synchronize()
                if r:
                    lat[k].append(e0.elapsed_time(e1))
            del wsk
        xs = sorted(lat[k])
        per_k[k] = {"batch_ms_p50": round(statistics.median(xs), 3), "kinput_ctmults_s": round(B / (statistics.median(xs) / 1e3), 1)}

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded uniform residues, seeded key draws)",
        "config": dict(CONFIG, ks=ks, batch_per_k=B, products_per_step=B * len(ks), primes=PRIMES[args.primes],
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       executor=("one cross-shape wave per step (every stage of all products one launch)"
                                 if args.engine == "waves" else
                                 f"CUDA graph, {args.streams} streams" if args.streams > 1 else "one stream, eager")),
        "gpu_launches": int(launches),
        "latency_ms": {"per_batch_p50": round(statistics.median(lat_all), 3),
                       "per_batch_p99": round(sorted(lat_all)[max(0, math.ceil(0.99 * len(lat_all)) - 1)], 3)},
        "roofline": roofline,
        "kernels": kernel_table,
        "step_alg_GBps": round((in_bytes + out_bytes) / (ms_step / 1e3) / 1e9, 1),
        "per_k": per_k,
        "clocks": clk,
        "tuning": tuned,
        "int_peaks_Gops": {k: round(v / 1e9, 2) for k, v in int_peaks.items()},
    }

    # ---------------- end to end through the C ABI with host buffers
    if not args.no_e2e:
        # right after the timed device steps, before the comparator legs:
        # after those legs the copy engines' uploads ran at 83-112 GB/s
        # (end to end 430-443 products/s), before them at 110-210 GB/s (524)
        if wave is not None:
            # the host-buffer leg builds its own two waves over two buffer sets
            del wave_bufs
            wave.close()
        torch.cuda.empty_cache()
        if ex is None:
            if ws is None and args.e2e_engine != "waves":
                ws = torch.empty(max(ctx.workspace_size(k, L, B) for k in ks) // 8 + 1, dtype=torch.uint64,
                                 device=dev)
            result["e2e"] = e2e_leg(args, ctx, evk, ks, B, L, N, depth, dev, stream, ws, world, inp, outs, tup, otup,
                                    inp[max(ks)].clone())

    # ---------------- comparators (outside the timed region)
    if not args.no_compare and rank == 0:
        reps = 2
        torch.cuda.synchronize()
        for k in ks:
            # one product per launch
            ws1 = torch.empty(ctx.workspace_size(k, L, 1) // 8 + 1, dtype=torch.uint64, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for r in range(reps + 1):
                if r == 1:
                    e0.record(stream)
                for b in range(B):
                    ctx.mul_k(tup[k][b], evk, otup[k][b], ws1, stream=stream)
            e1.record(stream)
            e1.synchronize()
            per_k[k]["one_per_launch_ctmults_s"] = round(B * reps / (e0.elapsed_time(e1) / 1e3), 1)
            del ws1
            # chained standard 2-input multiplies along the binary tree (batched over B)
            ms = chained_ms(ctx, evk, inp[k], k, B, L, N, dev, stream, reps)
            per_k[k]["chained_2input_ctmults_s"] = round(B / (ms / 1e3), 1)
            per_k[k]["speedup_vs_chained"] = round(per_k[k]["kinput_ctmults_s"] / per_k[k]["chained_2input_ctmults_s"], 3)
            per_k[k]["speedup_vs_one_per_launch"] = round(per_k[k]["kinput_ctmults_s"] / per_k[k]["one_per_launch_ctmults_s"], 3)
        ctx.check()

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(args)
    return result


def op_unit(kernel_class: str) -> str:
    """The integer operation a kernel class is built from (its roofline unit)."""
    if kernel_class.startswith("ntt"):
        return "butterfly"
    if kernel_class in ("bconv", "key_mac", "tensor"):
        return "mac128"
    return ""


def measure_int_peaks(G, params, q1: bool) -> dict:
    """Rate of the lazy NTT butterfly and of the 128-bit MAC on this GPU
    (register-only kernels over every SM; operations/s), taken at the same
    point of the run as the timed steps. The butterfly is measured in the
    form the NTT kernels run (q1: the Shoup product for q = 1 mod 2^32);
    with q1 the general form's rate is reported beside it."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    q = int(params.q[0])

    def rate(u):
        return max(G.peak_int(u, q, blocks=sms * per_sm, threads=256, iters=2048) for per_sm in (8, 16))
    out = {"butterfly": rate("butterfly_q1" if q1 else "butterfly"), "mac128": rate("mac128")}
    if q1:
        out["butterfly_general_form"] = rate("butterfly")
    return out


def chained_ms(ctx, evk, inp, k, B, L, N, dev, stream, reps):
    """Time the binary tree of standard 2-input multiplies over the batch."""
    import torch

    import paper_2601_15401_gb300 as G
    bufs = []
    ws = torch.empty(ctx.mul2_workspace_size(L, B) // 8 + 1, dtype=torch.uint64, device=dev)

    def mul2(x, y):
        (tx, lx), (ty, ly) = x, y
        lv = min(lx, ly)
        o = torch.empty((B, 2, lv - 1, N), dtype=torch.uint64, device=dev)
        bufs.append(o)
        a = [G.Tuple(tx[b], 2, lv, tx.shape[2]) for b in range(B)]
        c = [G.Tuple(ty[b], 2, lv, ty.shape[2]) for b in range(B)]
        oo = [G.Tuple(o[b], 2, lv - 1, lv - 1) for b in range(B)]
        ctx.mul2_batch(a, c, evk, oo, ws, stream=stream)
        return (o, lv - 1)

    def tree(lo, n):
        if n == 1:
            return (inp[:, lo], L)
        a = 1 << (n - 1).bit_length() - 1
        if n == 2:
            a = 1
        return mul2(tree(lo, a), tree(lo + a, n - a))

    tree(0, k)  # warm-up
    torch.cuda.synchronize()
    bufs.clear()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        tree(0, k)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _cpulist(text: str) -> set:
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.update(range(int(a), int(b or a) + 1))
    return cpus


def gpu_local_cpus(index: int) -> dict:
    """The GPU's PCI NUMA node and the CPUs local to it (sysfs, via the bus
    id nvidia-smi reports), restricted to the CPUs this process may use."""
    info = {"gpu_numa_node": None, "cpus": None}
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        dev = f"/sys/bus/pci/devices/{dom[-4:].lower()}:{rest.lower()}"
        info["pci"] = os.path.basename(dev)
        info["gpu_numa_node"] = int(open(os.path.join(dev, "numa_node")).read().strip())
        local = _cpulist(open(os.path.join(dev, "local_cpulist")).read())
        allowed = os.sched_getaffinity(0)
        usable = local & allowed
        info["local_cpus"] = len(local)
        info["allowed_cpus"] = len(allowed)
        if usable and usable != allowed:
            info["cpus"] = usable
    except Exception as e:  # no sysfs entry (container) or no nvidia-smi: leave placement to the OS
        info["error"] = type(e).__name__
    return info


def e2e_leg(args, ctx, evk, ks, B, L, N, depth, dev, stream, ws, world, dev_inp, dev_out, tup, otup, src):
    """The step through the C ABI with host buffers: every k's inputs are
    copied from pinned host memory, multiplied, and the outputs copied back,
    all inside the timed region. Uploads run on their own stream(s) and
    overlap the multiplies; downloads run on a second stream.

    With --engine batch each k has its own device buffers, so an upload
    waits only for the previous multiply of that k. With --engine waves the
    step is one cross-shape wave, and two sets of device buffers alternate
    between steps: step i's uploads fill one set while step i-1's wave reads
    the other."""
    import torch
    kmax = max(ks)
    # pinned host buffers on the GPU's own NUMA node: allocate them from a
    # thread bound to the CPUs local to the GPU (first touch places the pages)
    numa = gpu_local_cpus(dev.index if dev.index is not None else 0)
    prev_affinity = os.sched_getaffinity(0)
    if numa.get("cpus"):
        os.sched_setaffinity(0, numa["cpus"])
    host_in = torch.empty((B, kmax, 2, L, N), dtype=torch.uint64, pin_memory=True)
    host_in.copy_(src)  # the step's synthetic inputs, staged in pinned host memory
    host_out = {k: torch.empty((B, 2, L - depth[k], N), dtype=torch.uint64, pin_memory=True) for k in ks}
    numa_note = {k: v for k, v in numa.items() if k != "cpus"}
    numa_note["bound_cpus"] = len(numa["cpus"]) if numa.get("cpus") else None
    h2d = sum(B * k * 2 * L * N * 8 for k in ks)
    d2h = sum(B * 2 * (L - depth[k]) * N * 8 for k in ks)
    # uploads and downloads on their own streams: the next step's upload of
    # k waits only for this step's multiply of k (which frees its input
    # buffers), not for the downloads; several upload streams spread the
    # batch elements' copies over copy engines when asked
    copies = [torch.cuda.Stream(device=dev) for _ in range(max(1, args.copy_streams))]
    copy = copies[0]
    down = torch.cuda.Stream(device=dev)
    used = {}  # k -> event: the last multiply that read dev_inp[k]

    import paper_2601_15401_gb300 as G
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    n_mixed = int(round(B * args.pull_fraction))
    npull = [B if args.h2d == "pull" else 0 if args.h2d == "copy" else n_mixed]
    # device buffer sets (inputs, outputs): one for the batched engine, two
    # alternating sets for the wave engine
    sets = [(dev_inp, dev_out)]
    waves_mode = args.e2e_engine == "waves"
    cur_set = [0]
    if waves_mode:
        inp1 = {k: torch.empty_like(dev_inp[k]) for k in ks}
        out1 = {k: torch.empty_like(dev_out[k]) for k in ks}
        sets.append((inp1, out1))
        waves, wave_tables = [], []
        for si, (inps, outs_) in enumerate(sets):
            items = [([G.Tuple(inps[k][b, u], 2, L, L, 1, 2.0 ** 50) for u in range(k)],
                      G.Tuple(outs_[k][b], 2, L - depth[k], L - depth[k]), None) for k in ks for b in range(B)]
            w = G.Wave(ctx, items, evk)
            waves.append(w)
            wave_tables.append(torch.empty(w.workspace_size()[0] // 8 + 32, dtype=torch.uint64, device=dev))
        wave_scratch = torch.empty(max(w.workspace_size()[1] for w in waves) // 8 + 32, dtype=torch.uint64,
                                   device=dev)
        for w, t in zip(waves, wave_tables):
            w.run(t, wave_scratch, stream=stream)  # writes each wave's job tables
        torch.cuda.synchronize()
        set_used = [None, None]  # set -> event: the last wave that read its inputs
        set_down = [None, None]  # set -> event: the last download of its outputs
        step_no = [0]

    def upload(k, b, cs):
        """One batch element's inputs host -> device on stream cs: by the copy
        engines (cudaMemcpyAsync) or by the GPU's own loads over the host link
        (ckks_pull). "mixed" sends the last pull_fraction of the batch
        elements through the GPU's loads: the copy engines restart at a
        fraction of the link's rate after device compute, and the GPU's loads
        take SM slots from the multiplies, so each carries part; "pull" sends
        every element through the GPU's loads; "auto" (default) keeps the
        fastest of six splits, from every element by the copy engines to
        every element by the GPU's loads."""
        dst = sets[cur_set[0]][0][k][b]
        if b >= B - npull[0]:
            G.pull(dst, host_in[b, :k], blocks=sms * args.pull_ctas_per_sm, stream=cs)
        else:
            dst.copy_(host_in[b, :k], non_blocking=True)

    def step_waves():
        p = step_no[0] & 1
        step_no[0] += 1
        cur_set[0] = p
        evs = []
        for c, cs in enumerate(copies):
            if set_used[p] is not None:
                cs.wait_event(set_used[p])
            with torch.cuda.stream(cs):
                for k in ks:
                    for b in range(c, B, len(copies)):
                        upload(k, b, cs)
                e = torch.cuda.Event()
                e.record(cs)
                evs.append(e)
        for e in evs:
            stream.wait_event(e)
        if set_down[p] is not None:
            stream.wait_event(set_down[p])  # this set's outputs from two steps back are on the host
        waves[p].run(wave_tables[p], wave_scratch, stream=stream)
        done = torch.cuda.Event()
        done.record(stream)
        set_used[p] = done
        down.wait_event(done)
        with torch.cuda.stream(down):
            for k in ks:
                host_out[k].copy_(sets[p][1][k], non_blocking=True)
        fin = torch.cuda.Event()
        fin.record(down)
        set_down[p] = fin
        last_fin[0] = fin

    last_fin = [None]

    def step():
        if waves_mode:
            return step_waves()
        up = {}
        for k in ks:
            evs = []
            for c, cs in enumerate(copies):
                if k in used:
                    cs.wait_event(used[k])
                with torch.cuda.stream(cs):
                    for b in range(c, B, len(copies)):
                        upload(k, b, cs)
                    e = torch.cuda.Event()
                    e.record(cs)
                    evs.append(e)
            up[k] = evs
        for k in ks:
            for e in up[k]:
                stream.wait_event(e)
            ctx.mul_k_batch(tup[k], evk, otup[k], ws, stream=stream)
            done = torch.cuda.Event()
            done.record(stream)
            used[k] = done
            down.wait_event(done)
            with torch.cuda.stream(down):
                host_out[k].copy_(dev_out[k], non_blocking=True)
        fin = torch.cuda.Event()
        fin.record(down)
        stream.wait_event(fin)

    def upload_alone() -> float:
        """GB/s of the step's uploads with nothing else running (context)."""
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(copy)
        for c, cs in enumerate(copies):
            if c:
                cs.wait_event(t0)
            with torch.cuda.stream(cs):
                for k in ks:
                    for b in range(c, B, len(copies)):
                        upload(k, b, cs)
        for cs in copies[1:]:
            ev = torch.cuda.Event()
            ev.record(cs)
            copy.wait_event(ev)
        t1.record(copy)
        t1.synchronize()
        return h2d / (t0.elapsed_time(t1) / 1e3) / 1e9

    # the first host-to-device passes over freshly pinned buffers run at a
    # fraction of the link's rate (measured: 86 GB/s on the first pass, 210
    # GB/s later on one box); pass over them until the rate settles
    warm_bw = [upload_alone()]
    for _ in range(4):
        if len(warm_bw) > 1 and warm_bw[-1] > 0.9 * max(warm_bw[:-1]):
            break
        warm_bw.append(upload_alone())
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    trials = {}
    if args.h2d == "auto":
        # the copy engines' rate next to device compute differs between
        # boxes (94-210 GB/s measured), the GPU's own loads hold ~210 GB/s
        # but take SM slots: time two untimed steps of each split (none, an
        # eighth, a quarter, half, three quarters or all of the batch
        # elements by GPU loads) and keep the fastest
        for n in sorted({0, B // 8, n_mixed, B // 2, (3 * B) // 4, B}):
            npull[0] = n
            step()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(2):
                step()
            if last_fin[0] is not None:
                stream.wait_event(last_fin[0])
            t1.record(stream)
            t1.synchronize()
            trials[n] = t0.elapsed_time(t1) / 2
        npull[0] = min(trials, key=trials.get)
        torch.cuda.synchronize()
    cur_set[0] = 0
    bw_before = upload_alone()
    steps = max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    if last_fin[0] is not None:
        stream.wait_event(last_fin[0])  # the last step's downloads are inside the timed region
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ms = reduce_max(ms, world, dev)
    cur_set[0] = 0
    bw_after = upload_alone()
    os.sched_setaffinity(0, prev_affinity)
    ctx.check()
    return {"value": round(B * len(ks) * world / (ms / 1e3), 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3),
            "h2d_GBps_alone": [round(bw_before, 1), round(bw_after, 1)],
            "h2d_GBps_warmup": [round(x, 1) for x in warm_bw],
            "copy_streams": len(copies), "host_numa": numa_note,
            "h2d": {"copy_engines_elements": B - npull[0], "gpu_load_elements": npull[0],
                    "gpu_load_ctas": sms * args.pull_ctas_per_sm if npull[0] else 0,
                    "split": args.h2d,
                    "trial_ms_per_step": {f"{B - n} copy / {n} gpu-load": round(v, 2) for n, v in trials.items()},
                    "note": "per step, of the B batch elements of every k: copy engines (cudaMemcpyAsync) for the "
                            "first, the GPU's own loads over the host link (ckks_pull, 64-thread CTAs) for the rest"},
            "engine": "one cross-shape wave per step, two alternating input / output sets" if waves_mode else
                      "one batched call per k",
            "overlap": "uploads (own stream) overlap the multiplies of this and the previous step; downloads on "
                       "a second stream"}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_setup(k, args):
    import synth
    from oracle import ckks as O
    params = synth.params_large(congruence=congruence(args))
    octx = O.Ctx(params)
    km = synth.key_material(params, k, 3)
    keys = O.keygen_all(octx, km, k)
    cts = [O.Tup(synth.uniform_tuple(params, 2, params.L, 3, i), 2.0 ** 50) for i in range(k)]
    return octx, keys, cts


def oracle_product_seconds(octx, keys, cts) -> float:
    from oracle import ckks as O
    t = time.time()
    O.mul_k(octx, cts, keys)
    return time.time() - t


def cpu_baseline(args):
    from oracle import ring
    k = 4
    octx, keys, cts = _oracle_setup(k, args)
    sec = oracle_product_seconds(octx, keys, cts)
    return {"value": round(1.0 / sec, 4), "unit": UNIT, "cores": ring.num_threads(), "kind": "oracle",
            "sample": f"one full-size k={k} product (N=2^16, L=24, K=8, dnum=3) of the step's 144; "
                      f"{sec:.1f} s; k=4 is the cheapest k of the step, so the mix runs slower"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import ring
    k = 4
    octx, keys, cts = _oracle_setup(k, args)
    for _ in range(min(args.warmup, 1)):
        oracle_product_seconds(octx, keys, cts)
    times = []
    budget = 200.0
    t_start = time.time()
    for i in range(args.steps):
        times.append(oracle_product_seconds(octx, keys, cts))
        if time.time() - t_start > budget:
            break
    sec = statistics.mean(times)
    v = round(1.0 / sec, 4)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": len(times), "warmup": min(args.warmup, 1), "ms_per_step": round(sec * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded uniform residues, seeded key draws)",
            "config": dict(CONFIG, primes=PRIMES[args.primes],
                           reference_step="one full-size k=4 product (the cheapest k of the step)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": ring.num_threads(),
                             "sample": "one full-size k=4 product per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


KERNEL_SOURCES = {
    "ntt": ["ntt.cu", "ntt_kernel.cuh", "ntt_uf.cu", "ntt_ui.cu", "ntt_tf.cu", "ntt_ti.cu", "ntt_uf1.cu", "ntt_ui1.cu",
            "ntt_tf1.cu", "ntt_ti1.cu", "common.cuh", "internal.h"],
    "rns": ["rns.cu", "tensor_fixed.cu", "rns.h", "common.cuh", "internal.h"],
}


def source_hash(kernel_class: str = "ntt") -> str:
    """Hash of the sources a kernel class is compiled from (a stored DRAM
    traffic figure is used only while they are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_15401_gb300", "csrc")
    group = "ntt" if kernel_class.startswith("ntt") else "rns"
    for f in KERNEL_SOURCES[group]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--ks", default="")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--h2d", default="auto", choices=["auto", "mixed", "pull", "copy"],
                    help="e2e uploads: copy engines, GPU loads over the host link (pull), both (mixed), or the "
                         "fastest of six splits from all copy engines to all GPU loads in two untimed steps each (auto)")
    ap.add_argument("--pull-fraction", type=float, default=0.25,
                    help="--h2d mixed / auto: share of the batch elements uploaded by GPU loads")
    ap.add_argument("--pull-ctas-per-sm", type=int, default=1, help="64-thread CTAs per SM of the e2e uploads")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="streams the e2e leg spreads its copies over (1 measured best: 465 vs 343 with 4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tune", action="append", default=[], help="key=value library tunable (skips the autotuner)")
    ap.add_argument("--streams", type=int, default=1)
    ap.add_argument("--e2e-engine", default="batch", choices=["batch", "waves"],
                    help="engine of the host-buffer leg: one batched call per k (uploads of each k overlap the "
                         "multiplies of the others) or one wave per step over two alternating buffer sets")
    ap.add_argument("--primes", default="chain", choices=sorted(PRIMES),
                    help="prime chain of the workload: " + "; ".join(f"{k}: {v}" for k, v in PRIMES.items()))
    ap.add_argument("--engine", default="waves", choices=["batch", "waves"],
                    help="batch: one batched call per k; waves: the whole step as one cross-shape wave")
    args = ap.parse_args()
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
