"""Batched execution of uneven k-input multiplications in one CUDA graph.

A workload is a list of requests, each a k-input product at its own ring
degree N, input level and k. Two executors:

* WaveExecutor (cross-shape): the requests of one ring degree form waves of
  any mix of k, level and partition; every stage of all products of a wave
  is one launch (ckks_wave_*, device job tables), so a wave of 128 products
  takes a few dozen launches whatever its mix.
* BatchExecutor (per shape): requests with the same (N, k, level,
  partition) form a group that runs as one batched library call
  (ckks_mul_k_batch); groups are spread over several streams.

Either schedule is captured once into a CUDA graph; replaying it launches
the entire workload with one cudaGraphLaunch. Workspaces are allocated up
front, so nothing is allocated while the graph runs.

The library calls are the only device work; this module only arranges
buffers, streams and the graph.
"""
from __future__ import annotations

import json
import os
from collections import defaultdict
from dataclasses import dataclass, field

import torch

from . import Context, Tuple


@dataclass
class MulRequest:
    """One product: k ciphertexts at `level` in the context for `log_n`."""
    log_n: int
    k: int
    level: int
    partition: str | None = None
    rid: int = 0


@dataclass
class _Group:
    log_n: int
    k: int
    level: int
    partition: str | None
    rids: list = field(default_factory=list)
    inp: object = None      # [B][k][2][level][N]
    out: object = None      # [B][2][level - depth][N]
    tuples: list = None
    outs: list = None
    depth: int = 0
    ws_bytes: int = 0
    stream: int = 0


class BatchExecutor:
    """contexts: {log_n: (Context, EvkSet)} with keys up to the largest k."""

    def __init__(self, contexts: dict, n_streams: int = 8, device=None):
        self.contexts = contexts
        self.n_streams = n_streams
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.groups: list[_Group] = []
        self.slot_of: dict[int, tuple] = {}
        self.graph = None
        self.streams = []
        self.ws = []

    # -------------------------------------------------------------- planning
    def plan(self, requests: list[MulRequest]):
        by_shape = defaultdict(list)
        for r in requests:
            by_shape[(r.log_n, r.k, r.level, r.partition)].append(r.rid)
        self.groups = []
        for (log_n, k, level, part), rids in sorted(by_shape.items(), key=lambda kv: -len(kv[1]) * kv[0][1]):
            ctx, _ = self.contexts[log_n]
            g = _Group(log_n, k, level, part, rids)
            g.depth = ctx.plan_describe(k, part)["depth"]
            B, N = len(rids), ctx.N
            g.inp = torch.empty((B, k, 2, level, N), dtype=torch.uint64, device=self.device)
            g.out = torch.empty((B, 2, level - g.depth, N), dtype=torch.uint64, device=self.device)
            g.tuples = [[Tuple(g.inp[b, u], 2, level, level) for u in range(k)] for b in range(B)]
            g.outs = [Tuple(g.out[b], 2, level - g.depth, level - g.depth) for b in range(B)]
            g.ws_bytes = ctx.workspace_size(k, level, B, part)
            for b, rid in enumerate(rids):
                self.slot_of[rid] = (len(self.groups), b)
            self.groups.append(g)
        # balance the groups over the streams by workspace size (a proxy for work)
        load = [0] * self.n_streams
        need = [0] * self.n_streams
        for g in sorted(self.groups, key=lambda g: -g.ws_bytes):
            s = min(range(self.n_streams), key=lambda i: load[i])
            g.stream = s
            load[s] += g.ws_bytes
            need[s] = max(need[s], g.ws_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.n_streams)]
        self.ws = [torch.empty(max(1, n // 8 + 1), dtype=torch.uint64, device=self.device) for n in need]
        self.graph = None

    def input_view(self, rid: int):
        """[k][2][level][N] device slot of a request (write its ciphertexts here)."""
        gi, b = self.slot_of[rid]
        return self.groups[gi].inp[b]

    def output_view(self, rid: int):
        gi, b = self.slot_of[rid]
        return self.groups[gi].out[b]

    def output_tuple(self, rid: int) -> Tuple:
        gi, b = self.slot_of[rid]
        return self.groups[gi].outs[b]

    # -------------------------------------------------------------- running
    def _enqueue(self, main: torch.cuda.Stream):
        start = torch.cuda.Event()
        start.record(main)
        done = []
        for s in self.streams:
            s.wait_event(start)
        for g in self.groups:
            ctx, evk = self.contexts[g.log_n]
            st = self.streams[g.stream]
            ctx.mul_k_batch(g.tuples, evk, g.outs, self.ws[g.stream], partition=g.partition, stream=st)
        for s in self.streams:
            e = torch.cuda.Event()
            e.record(s)
            done.append(e)
        for e in done:
            main.wait_event(e)

    def run_eager(self):
        """Every group's batched call, stream-ordered, without a graph."""
        self._enqueue(torch.cuda.current_stream(self.device))

    def capture(self):
        """Capture the whole schedule into one CUDA graph."""
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=self.device)
        with torch.cuda.graph(g, stream=cap):
            self._enqueue(cap)
        self.graph = g
        torch.cuda.synchronize(self.device)
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()


class WaveExecutor:
    """Uneven requests as cross-shape waves (ckks_wave_*): the requests of
    one ring degree are split, in order, into waves of at most `max_wave`
    products of any k, level and partition; each wave runs every stage of
    all its products as one launch per stage. The waves of one ring degree
    run one after another on that degree's stream and share one scratch
    buffer (each keeps its own job-table buffer); ring degrees run side by
    side. capture() records the whole schedule in one CUDA graph.
    contexts: {log_n: (Context, EvkSet)} with keys up to the largest k."""

    def __init__(self, contexts: dict, max_wave: int = 128, device=None):
        self.contexts = contexts
        self.max_wave = max_wave
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.waves = []          # (log_n, Wave, tables)
        self.scratch = {}        # log_n -> buffer
        self.streams = {}
        self.slot_of = {}        # rid -> (inp tensor [k][2][level][N], out Tuple)
        self.graph = None
        self._first_run = True

    def plan(self, requests: list[MulRequest]):
        from . import Wave
        by_n = defaultdict(list)
        for r in requests:
            by_n[r.log_n].append(r)
        self.waves, self.scratch, self.slot_of = [], {}, {}
        need = defaultdict(int)
        for log_n, reqs in sorted(by_n.items()):
            ctx, evk = self.contexts[log_n]
            for i in range(0, len(reqs), self.max_wave):
                items = []
                for r in reqs[i:i + self.max_wave]:
                    depth = ctx.plan_describe(r.k, r.partition)["depth"]
                    inp = torch.empty((r.k, 2, r.level, ctx.N), dtype=torch.uint64, device=self.device)
                    out = Tuple(torch.empty((2, r.level - depth, ctx.N), dtype=torch.uint64, device=self.device),
                                2, r.level - depth, r.level - depth)
                    self.slot_of[r.rid] = (inp, out)
                    items.append(([Tuple(inp[u], 2, r.level, r.level) for u in range(r.k)], out, r.partition))
                w = Wave(ctx, items, evk)
                t, n = w.workspace_size()
                tables = torch.empty(t // 8 + 32, dtype=torch.uint64, device=self.device)
                self.waves.append((log_n, w, tables))
                need[log_n] = max(need[log_n], n)
        for log_n, n in need.items():
            self.scratch[log_n] = torch.empty(n // 8 + 32, dtype=torch.uint64, device=self.device)
            self.streams[log_n] = torch.cuda.Stream(device=self.device)
        self.graph = None
        self._first_run = True

    def input_view(self, rid: int):
        return self.slot_of[rid][0]

    def output_view(self, rid: int):
        return self.slot_of[rid][1].data

    def launches(self) -> int:
        return sum(w.describe()["launches"] for _, w, _ in self.waves)

    def _enqueue(self, main: torch.cuda.Stream):
        start = torch.cuda.Event()
        start.record(main)
        for s in self.streams.values():
            s.wait_event(start)
        for log_n, w, tables in self.waves:
            w.run(tables, self.scratch[log_n], stream=self.streams[log_n])
        for s in self.streams.values():
            e = torch.cuda.Event()
            e.record(s)
            main.wait_event(e)

    def run_eager(self):
        self._enqueue(torch.cuda.current_stream(self.device))
        self._first_run = False

    def capture(self):
        """Capture the schedule in one CUDA graph (after one eager run, which
        writes every wave's job tables)."""
        if self._first_run:
            self.run_eager()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=self.device)
        with torch.cuda.graph(g, stream=cap):
            self._enqueue(cap)
        self.graph = g
        torch.cuda.synchronize(self.device)
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()


def one_per_launch(contexts, requests, executor: BatchExecutor):
    """Reference schedule: every product as its own ckks_mul_k call on one
    stream (reads the executor's input slots, writes its output slots)."""
    ws_need = 0
    for r in requests:
        ctx, _ = contexts[r.log_n]
        ws_need = max(ws_need, ctx.workspace_size(r.k, r.level, 1, r.partition))
    ws = torch.empty(ws_need // 8 + 1, dtype=torch.uint64, device=executor.device)
    for r in requests:
        ctx, evk = contexts[r.log_n]
        gi, b = executor.slot_of[r.rid]
        g = executor.groups[gi]
        ctx.mul_k(g.tuples[b], evk, g.outs[b], ws, partition=r.partition)
    return ws


# ---------------------------------------------------------------------------
# autotuner
# ---------------------------------------------------------------------------
TUNE_SPACE = {
    "ntt_tile_cols": [2048, 4096, 8192],
    "ntt_tile_blocks": [1024, 2048, 4096],
    "bconv_threads": [128, 256, 512],
    "mac_threads": [128, 256, 512],
}
# the library's defaults (Context in csrc/internal.h): the reference every
# candidate's output is compared with
TUNE_DEFAULTS = {"ntt_tile_cols": 4096, "ntt_tile_blocks": 4096, "bconv_threads": 256, "mac_threads": 256}


def _cache_path() -> str:
    return os.environ.get("CKKS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ckks_mulk",
                                                          "autotune.json"))


def tune_key(ctx: Context) -> str:
    """Cache key: GPU, parameter shape and the hash of the library sources, so
    that a choice made for other kernels is never applied to these."""
    from .build import source_hash
    name = torch.cuda.get_device_name(ctx.device).replace(" ", "_")
    return f"{name}/logN{ctx.log_n}/L{ctx.L}/K{ctx.K}/dnum{ctx.dnum}/src{source_hash()}"


def autotune(ctx: Context, evk, k: int = 8, batch: int = 4, reps: int = 3, cache: str | None = None,
             force: bool = False) -> dict:
    """Pick each tunable by timing a batched k-input product (coordinate
    descent over TUNE_SPACE, CUDA events), store the choice in a JSON cache
    keyed by GPU, N, the prime-chain shape and the library's source hash, and
    apply it to `ctx`.

    Every candidate's output is compared, residue for residue, with the
    output of the library defaults on the same inputs; a candidate that
    differs is rejected (never chosen), and a cached choice is re-checked the
    same way before it is applied."""
    import synth
    path = cache or _cache_path()
    key = tune_key(ctx)
    db = {}
    if os.path.exists(path):
        try:
            db = json.load(open(path))
        except Exception:
            db = {}
    level = ctx.L
    depth = ctx.plan_describe(k)["depth"]
    dev = torch.device("cuda", ctx.device)
    inp = synth.uniform_residues_torch(ctx.q[:level], (batch, k, 2), ctx.N, 0x7E57, dev)
    out = torch.empty((batch, 2, level - depth, ctx.N), dtype=torch.uint64, device=dev)
    tup = [[Tuple(inp[b, u], 2, level, level) for u in range(k)] for b in range(batch)]
    outs = [Tuple(out[b], 2, level - depth, level - depth) for b in range(batch)]
    ws = torch.empty(ctx.workspace_size(k, level, batch) // 8 + 1, dtype=torch.uint64, device=dev)

    def apply(choice: dict):
        for n, v in choice.items():
            ctx.tune_set(n, v)

    def run_once():
        out.zero_()
        ctx.mul_k_batch(tup, evk, outs, ws)
        torch.cuda.synchronize(dev)
        ctx.check()

    apply(TUNE_DEFAULTS)
    run_once()
    reference = out.clone()

    def same() -> bool:
        return torch.equal(out.view(torch.int64), reference.view(torch.int64))

    if key in db and not force:
        apply(db[key]["choice"])
        run_once()
        if same():
            return db[key]
        apply(TUNE_DEFAULTS)  # a cached choice that no longer matches: search again

    def timed() -> float:
        run_once()
        if not same():
            return None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.mul_k_batch(tup, evk, outs, ws)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    choice = dict(TUNE_DEFAULTS)
    trials, rejected = {}, []
    for name, values in TUNE_SPACE.items():
        best = None
        for v in values:
            ctx.tune_set(name, v)
            ms = timed()
            if ms is None:
                rejected.append(f"{name}={v}")
                continue
            trials[f"{name}={v}"] = round(ms, 4)
            if best is None or ms < best[0]:
                best = (ms, v)
        choice[name] = best[1] if best else TUNE_DEFAULTS[name]
        ctx.tune_set(name, choice[name])
    # the combination, checked once more as a whole
    run_once()
    if not same():
        rejected.append("combined choice " + json.dumps(choice))
        choice = dict(TUNE_DEFAULTS)
        apply(choice)
    entry = {"choice": choice, "ms": min(trials.values()), "trials": trials, "rejected": rejected,
             "verified": "every candidate's output equal to the library defaults' output",
             "workload": f"k={k} batch={batch}"}
    db[key] = entry
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        json.dump(db, open(path, "w"), indent=1)
    except OSError:
        pass
    return entry


# ---------------------------------------------------------------------------
# the uneven-batch measurement: 1024 products with k uniform in 2..12, N in
# {2^14, 2^15, 2^16}, input level uniform in [k, 24], in one graph launch
# ---------------------------------------------------------------------------
def _time_replays(fn, reps: int) -> float:
    fn()  # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    import argparse
    import numpy as np

    from .serve import build_gpu_state

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=1024)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--max-wave", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--log-ns", default="14,15,16")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--skip-groups", action="store_true", help="time only the wave executor and one per launch")
    args = ap.parse_args()
    log_ns = [int(x) for x in args.log_ns.split(",")]
    contexts, pools = build_gpu_state(tuple(log_ns))
    tuned = {}
    if not args.no_tune:
        for ln, (ctx, evk) in contexts.items():
            tuned[ln] = autotune(ctx, evk, k=8, batch=4)["choice"]
    g = np.random.default_rng(args.seed)
    reqs, srcs = [], {}
    for i in range(args.requests):
        k = int(g.integers(2, 13))
        log_n = int(g.choice(log_ns))
        level = int(g.integers(k, 25))
        reqs.append(MulRequest(log_n, k, level, None, i))
        srcs[i] = [int(x) for x in g.integers(0, pools[log_n].shape[0], size=k)]

    def fill(ex):
        for r in reqs:
            src = pools[r.log_n].view(torch.int64)[srcs[r.rid]][:, :, :r.level]
            ex.input_view(r.rid).view(torch.int64).copy_(src)
        torch.cuda.synchronize()

    res = {"workload": f"{args.requests} k-input products, k in 2..12, N in {[1 << x for x in log_ns]}, "
                       "level in [k, 24], L=24x50-bit q, K=8x60-bit p, dnum=3", "tuning": tuned}
    # cross-shape waves, one CUDA graph
    wx = WaveExecutor(contexts, max_wave=args.max_wave)
    wx.plan(reqs)
    fill(wx)
    wx.capture()
    wave_ms = _time_replays(wx.replay, args.reps)
    wave_out = {r.rid: wx.output_view(r.rid).clone() for r in reqs}
    res.update({"waves": len(wx.waves), "wave_launches": wx.launches(), "wave_graph_ms": round(wave_ms, 3),
                "wave_ctmults_s": round(args.requests / (wave_ms / 1e3), 1)})
    del wx
    torch.cuda.empty_cache()
    # per-shape groups on several streams, one CUDA graph
    ex = BatchExecutor(contexts, n_streams=args.streams)
    ex.plan(reqs)
    fill(ex)
    if not args.skip_groups:
        ex.capture()
        graph_ms = _time_replays(ex.replay, args.reps)
        same_groups = all(torch.equal(wave_out[r.rid].view(torch.int64), ex.output_view(r.rid).view(torch.int64))
                          for r in reqs)
        res.update({"groups": len(ex.groups), "streams": args.streams, "group_graph_ms": round(graph_ms, 3),
                    "group_ctmults_s": round(args.requests / (graph_ms / 1e3), 1),
                    "waves_equal_groups": bool(same_groups)})
    # reference schedule: one product per library call, one stream, eager
    single_ms = _time_replays(lambda: one_per_launch(contexts, reqs, ex), args.reps)
    same = all(torch.equal(wave_out[r.rid].view(torch.int64), ex.output_view(r.rid).view(torch.int64)) for r in reqs)
    res.update({"one_per_launch_ms": round(single_ms, 3),
                "one_per_launch_ctmults_s": round(args.requests / (single_ms / 1e3), 1),
                "waves_equal_one_per_launch": bool(same),
                "speedup_waves_vs_one_per_launch": round(single_ms / wave_ms, 3)})
    if "group_graph_ms" in res:
        res["speedup_waves_vs_groups"] = round(res["group_graph_ms"] / wave_ms, 3)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
