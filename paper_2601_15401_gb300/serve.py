"""Continuous-batching server for k-input multiplications.

Evaluation keys and a pool of ciphertexts stay resident on the device, one
set per ring degree. A request names k pool ciphertexts, a level and
(optionally) a partition. The scheduler keeps a queue of arrived requests
and, whenever a stream is free and the device-memory budget allows, launches
a batch: the pending requests of one shape (N, k, level, partition), oldest
first, up to `max_batch`. Requests that arrive while other batches run join
the next batches (continuous batching); batches on different streams run
side by side on the device. A request's footprint (its input slot, output
and its share of the batch workspace) is admitted only under the memory cap;
otherwise it waits. Latency = completion (CUDA event observed) - arrival.

The scheduling logic is independent of the device: `Scheduler` drives any
backend with launch / poll; `GpuBackend` runs batches through the library
(ckks_mul_k_batch), `tests` drive the scheduler with a host-only fake.

Run `python -m paper_2601_15401_gb300.serve --rate 2000 --seconds 30` for the
Poisson-arrival measurement (p50 / p99 latency, sustained products/s).
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    log_n: int
    k: int
    level: int
    cts: tuple           # pool indices of the k input ciphertexts
    arrival: float = 0.0
    partition: str | None = None
    admitted: float = -1.0
    done: float = -1.0
    error: str | None = None
    batch: int = -1          # id of the batch that ran it
    slots: object = None     # plaintext requests: [k][N/2] complex slot vectors (cts unused)
    seed: int = 0            # plaintext requests: seed of the encryption noise

    @property
    def shape(self):
        return (self.log_n, self.k, self.level, self.partition)


@dataclass
class Batch:
    bid: int
    shape: tuple
    reqs: list
    stream: int
    footprint: int
    handle: object = None
    launched: float = 0.0


class Scheduler:
    """Continuous batching with admission by memory footprint.

    backend must provide: n_streams, footprint(shape, batch) -> bytes,
    launch(batch) -> handle, poll(handle) -> bool, and optional finish(batch)."""

    def __init__(self, backend, cap_bytes: int, max_batch: int = 8, max_queue: int = 100000,
                 timeout_s: float | None = None):
        self.be = backend
        # requests that may share a batch: the backend's grouping key if it
        # has one (cross-shape batches group by ring degree only), else the
        # full shape (N, k, level, partition)
        self.key = getattr(backend, "group_key", None) or (lambda r: r.shape)
        self.timeout_s = timeout_s      # watchdog: a batch running longer is failed
        self.failed: list[Request] = []
        self.cap = cap_bytes
        self.max_batch = max_batch
        self.max_queue = max_queue
        self.queues: "OrderedDict[tuple, deque]" = OrderedDict()
        self.free_streams = deque(range(backend.n_streams))
        self.running: list[Batch] = []
        self.in_use = 0
        self.next_bid = 0
        self.completed: list[Request] = []
        self.rejected = 0
        self.admitted_batches = 0

    def submit(self, r: Request) -> bool:
        if sum(len(q) for q in self.queues.values()) >= self.max_queue:
            self.rejected += 1
            return False
        self.queues.setdefault(self.key(r), deque()).append(r)
        return True

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def _pick(self):
        """Shape whose oldest request arrived first."""
        best = None
        for shape, q in self.queues.items():
            if q and (best is None or q[0].arrival < self.queues[best][0].arrival):
                best = shape
        return best

    def step(self, now: float) -> int:
        """Retire finished batches, then launch as many batches as streams and
        memory allow. Returns the number of batches launched."""
        still = []
        for b in self.running:
            if self.timeout_s is not None and now is not None and now - b.launched > self.timeout_s \
                    and not self.be.poll(b.handle):
                # the batch missed its deadline: fail its requests and keep its
                # stream and memory out of use (the work may still be running)
                for r in b.reqs:
                    r.done = now
                    r.error = "timeout"
                self.failed.extend(b.reqs)
                abandon = getattr(self.be, "abandon", None)
                if abandon:
                    abandon(b)
                continue
            if self.be.poll(b.handle):
                t = time.perf_counter() if now is None else now
                for r in b.reqs:
                    r.done = t
                self.completed.extend(b.reqs)
                self.in_use -= b.footprint
                self.free_streams.append(b.stream)
                fin = getattr(self.be, "finish", None)
                if fin:
                    fin(b)
            else:
                still.append(b)
        self.running = still
        launched = 0
        while self.free_streams:
            shape = self._pick()
            if shape is None:
                break
            q = self.queues[shape]
            n = min(len(q), self.max_batch)
            fits = getattr(self.be, "fits", None)
            by_reqs = getattr(self.be, "footprint_reqs", None)

            def fp_of(n):
                return by_reqs([q[i] for i in range(n)]) if by_reqs else self.be.footprint(shape, n)

            def fits_n(n):
                if not fits:
                    return True
                return fits([q[i] for i in range(n)]) if by_reqs else fits(shape, n)
            while n > 0 and (self.in_use + fp_of(n) > self.cap or not fits_n(n)):
                n -= 1
            if n == 0:
                break  # wait for memory to free up
            fp = fp_of(n)
            reqs = [q.popleft() for _ in range(n)]
            if not q:
                del self.queues[shape]
            b = Batch(self.next_bid, shape, reqs, self.free_streams.popleft(), fp)
            self.next_bid += 1
            for r in reqs:
                r.admitted = now
                r.batch = b.bid
            b.launched = now
            b.handle = self.be.launch(b)
            self.in_use += fp
            self.running.append(b)
            self.admitted_batches += 1
            launched += 1
        return launched

    def idle(self) -> bool:
        return not self.running and self.pending() == 0

    def healthy_streams(self) -> int:
        """Streams not lost to timed-out batches."""
        return len(self.free_streams) + len(self.running)


# ---------------------------------------------------------------------------
# device backend
# ---------------------------------------------------------------------------
class GpuBackend:
    """Runs batches through the library; contexts: {log_n: (Context, EvkSet)},
    pools: {log_n: tensor [P][2][L][N]} of resident ciphertexts (NTT domain).

    Every stream owns one workspace of `ws_bytes` allocated up front, so a
    batch allocates only its gathered inputs and its outputs; a shape whose
    workspace for n requests exceeds `ws_bytes` runs with fewer requests."""

    def __init__(self, contexts, pools, n_streams: int = 8, ws_bytes: int = 4 << 30, keep_results: bool = False):
        import torch
        self.torch = torch
        self.keep_results = keep_results
        self.contexts = contexts
        self.pools = pools
        self.n_streams = n_streams
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.ws_bytes = ws_bytes
        self.ws = [torch.empty(ws_bytes // 8, dtype=torch.uint64, device="cuda") for _ in range(n_streams)]
        self.results = {}
        self._fp_cache = {}
        self._ws_cache = {}

    def resident_bytes(self) -> int:
        """Keys, pools, contexts' tables and the stream workspaces."""
        return self.torch.cuda.memory_allocated()

    def fits(self, shape, n: int) -> bool:
        key = (shape, n)
        if key not in self._ws_cache:
            log_n, k, level, part = shape
            ctx, _ = self.contexts[log_n]
            self._ws_cache[key] = ctx.workspace_size(k, level, n, part)
        return self._ws_cache[key] <= self.ws_bytes

    def footprint(self, shape, n: int) -> int:
        """Device bytes a batch allocates: gathered inputs and outputs."""
        key = (shape, n)
        if key not in self._fp_cache:
            log_n, k, level, part = shape
            ctx, _ = self.contexts[log_n]
            depth = ctx.plan_describe(k, part)["depth"]
            self._fp_cache[key] = n * (k * 2 * level + 2 * (level - depth)) * ctx.N * 8
        return self._fp_cache[key]

    def launch(self, b: Batch):
        torch = self.torch
        from . import Tuple
        log_n, k, level, part = b.shape
        ctx, evk = self.contexts[log_n]
        depth = ctx.plan_describe(k, part)["depth"]
        st = self.streams[b.stream]
        n = len(b.reqs)
        pool = self.pools[log_n]
        with torch.cuda.stream(st):
            idx = torch.tensor([c for r in b.reqs for c in r.cts], device=pool.device)
            # gather only the active limbs, on an int64 view (same bits; uint64
            # has no CUDA gather)
            inp = pool.view(torch.int64)[:, :, :level].index_select(0, idx).view(torch.uint64)
            inp = inp.view(n, k, 2, level, ctx.N)
            out = torch.empty((n, 2, level - depth, ctx.N), dtype=torch.uint64, device=pool.device)
            tup = [[Tuple(inp[i, u], 2, level, level) for u in range(k)] for i in range(n)]
            outs = [Tuple(out[i], 2, level - depth, level - depth) for i in range(n)]
            ctx.mul_k_batch(tup, evk, outs, self.ws[b.stream], partition=part, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        # keep the buffers alive until the event completes
        return (ev, inp, out)

    def poll(self, handle) -> bool:
        return handle[0].query()

    def abandon(self, b: Batch):
        """A timed-out batch: keep its buffers alive (the device may still be
        using them) and never reuse its stream."""
        self._abandoned = getattr(self, "_abandoned", [])
        self._abandoned.append(b.handle)

    def finish(self, b: Batch):
        """Completed batch: hand results over (kept only when asked; a
        served result otherwise goes back to the allocator)."""
        if self.keep_results:
            out = b.handle[2]
            for i, r in enumerate(b.reqs):
                self.results[r.rid] = out[i]
        b.handle = None


class WaveBackend:
    """Cross-shape batches: the pending requests of one ring degree, any mix
    of k, level and partition, run as one wave (ckks_wave_*: every stage of
    every product in one launch). Inputs are read in place from the resident
    pool (a wave item points at its pool ciphertexts, no gather); each batch
    allocates only its outputs and its job tables; every stream owns a
    scratch buffer of `ws_bytes` allocated up front, and a batch whose
    scratch would not fit it runs with fewer requests.

    contexts: {log_n: (Context, EvkSet)}, pools: {log_n: tensor [P][2][L][N]}."""

    def __init__(self, contexts, pools, n_streams: int = 4, ws_bytes: int = 16 << 30, keep_results: bool = False):
        import torch
        self.torch = torch
        self.contexts = contexts
        self.pools = pools
        self.n_streams = n_streams
        self.keep_results = keep_results
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.ws_bytes = ws_bytes
        self.scratch = [torch.empty(ws_bytes // 8, dtype=torch.uint64, device="cuda") for _ in range(n_streams)]
        self.results = {}
        self._need = {}

    @staticmethod
    def group_key(r: Request):
        return (r.log_n,)

    def resident_bytes(self) -> int:
        return self.torch.cuda.memory_allocated()

    def _req_bytes(self, r: Request) -> tuple:
        """(scratch, output) bytes of one product (scratch as ckks_mul_k's
        workspace for it alone, which is the wave's per-product layout)."""
        key = (r.log_n, r.k, r.level, r.partition)
        if key not in self._need:
            ctx, _ = self.contexts[r.log_n]
            depth = ctx.plan_describe(r.k, r.partition)["depth"]
            self._need[key] = (ctx.workspace_size(r.k, r.level, 1, r.partition),
                               2 * (r.level - depth) * ctx.N * 8)
        return self._need[key]

    def fits(self, reqs) -> bool:
        return sum(self._req_bytes(r)[0] for r in reqs) <= self.ws_bytes

    def footprint_reqs(self, reqs) -> int:
        """Device bytes a batch allocates: its outputs (the job tables are
        small; inputs stay in the pool)."""
        return sum(self._req_bytes(r)[1] for r in reqs)

    def footprint(self, shape, n: int) -> int:  # for the scheduler's fallback path
        return 0

    def launch(self, b: Batch):
        torch = self.torch
        from . import Tuple, Wave
        (log_n,) = b.shape
        ctx, evk = self.contexts[log_n]
        pool = self.pools[log_n]
        L = pool.shape[2]
        st = self.streams[b.stream]
        items, outs = [], []
        with torch.cuda.stream(st):
            for r in b.reqs:
                depth = ctx.plan_describe(r.k, r.partition)["depth"]
                ol = r.level - depth
                out = Tuple(torch.empty((2, ol, ctx.N), dtype=torch.uint64, device=pool.device), 2, ol, ol)
                outs.append(out)
                items.append(([Tuple(pool[c], 2, r.level, L) for c in r.cts], out, r.partition))
            w = Wave(ctx, items, evk)
            t, _ = w.workspace_size()
            tables = torch.empty(t // 8 + 32, dtype=torch.uint64, device=pool.device)
            w.run(tables, self.scratch[b.stream], stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        # the wave (host staging), tables and outputs live until the event completes
        return (ev, w, tables, outs)

    def poll(self, handle) -> bool:
        return handle[0].query()

    def abandon(self, b: Batch):
        self._abandoned = getattr(self, "_abandoned", [])
        self._abandoned.append(b.handle)

    def finish(self, b: Batch):
        if self.keep_results:
            for r, o in zip(b.reqs, b.handle[3]):
                self.results[r.rid] = o.data
        b.handle[1].close()
        b.handle = None


class PlaintextBackend(GpuBackend):
    """Plaintext in, plaintext out: a batch of requests carrying slot vectors
    runs encode -> encrypt (batched) -> k-input product -> decrypt (batched)
    -> decode on its stream, every step in the library. This is the pipeline
    of the party that holds the secret (e.g. a client batching its own
    products); the encryption noise of a request is drawn from its own seed,
    so its result does not depend on the batch it lands in.

    keys: {log_n: (s, pk)} device secret (int64 [N]) and public key [2][L][N]."""

    def __init__(self, contexts, keys, scale: float = 2.0 ** 50, **kw):
        super().__init__(contexts, pools={}, **kw)
        self.keys = keys
        self.scale = scale

    def footprint(self, shape, n: int) -> int:
        key = ("pt", shape, n)
        if key not in self._fp_cache:
            log_n, k, level, part = shape
            ctx, _ = self.contexts[log_n]
            N = ctx.N
            depth = ctx.plan_describe(k, part)["depth"]
            cts = n * k * 2 * level * N * 8 + n * 2 * (level - depth) * N * 8
            plain = n * k * N * (16 + 8 + 3 * 8) + n * N * (8 + 16)
            enc_ws = ctx.encrypt_batch_workspace_size(level, n * k) + ctx.decrypt_batch_workspace_size(n)
            emb_ws = ctx.embed_workspace_size(n * k)
            self._fp_cache[key] = cts + plain + enc_ws + emb_ws
        return self._fp_cache[key]

    def _noise(self, r: Request, N: int, k: int):
        import synth
        torch = self.torch
        g = torch.Generator(device="cuda")
        g.manual_seed(int(r.seed))
        v = torch.randint(-1, 2, (k, N), generator=g, device="cuda", dtype=torch.int64)
        e = torch.randn((2, k, N), generator=g, device="cuda", dtype=torch.float64) * synth.SIGMA
        e = e.round().clamp_(-synth.ERR_CLIP, synth.ERR_CLIP).to(torch.int64)
        return v, e[0], e[1]

    def launch(self, b: Batch):
        torch = self.torch
        import numpy as np
        from . import Tuple
        log_n, k, level, part = b.shape
        ctx, evk = self.contexts[log_n]
        s, pk = self.keys[log_n]
        N = ctx.N
        depth = ctx.plan_describe(k, part)["depth"]
        st = self.streams[b.stream]
        n = len(b.reqs)
        with torch.cuda.stream(st):
            z = torch.from_numpy(np.ascontiguousarray(np.concatenate([r.slots for r in b.reqs]), dtype=np.complex128))
            z = z.pin_memory().to("cuda", non_blocking=True)                      # [n k][N/2]
            emb_ws = torch.empty(ctx.embed_workspace_size(n * k) // 8 + 1, dtype=torch.uint64, device="cuda")
            m = torch.empty((n * k, N), dtype=torch.int64, device="cuda")
            ctx.encode(z, self.scale, m, emb_ws, stream=st)
            noise = [self._noise(r, N, k) for r in b.reqs]
            v = torch.cat([x[0] for x in noise])
            e0 = torch.cat([x[1] for x in noise])
            e1 = torch.cat([x[2] for x in noise])
            ct = torch.empty((n * k, 2, level, N), dtype=torch.uint64, device="cuda")
            cts = [Tuple(ct[i], 2, level, level, scale=self.scale) for i in range(n * k)]
            enc_ws = torch.empty(ctx.encrypt_batch_workspace_size(level, n * k) // 8 + 1, dtype=torch.uint64,
                                 device="cuda")
            ctx.encrypt_batch(m, v, e0, e1, pk, level, cts, enc_ws, stream=st)
            for t in cts:
                t.scale = self.scale
            out = torch.empty((n, 2, level - depth, N), dtype=torch.uint64, device="cuda")
            outs = [Tuple(out[i], 2, level - depth, level - depth) for i in range(n)]
            tup = [cts[i * k:(i + 1) * k] for i in range(n)]
            ctx.mul_k_batch(tup, evk, outs, self.ws[b.stream], partition=part, stream=st)
            dec = torch.empty((n, N), dtype=torch.float64, device="cuda")
            dec_ws = torch.empty(ctx.decrypt_batch_workspace_size(n) // 8 + 1, dtype=torch.uint64, device="cuda")
            ctx.decrypt_batch(outs, s, dec, dec_ws, stream=st)
            zo = torch.empty((n, N // 2), dtype=torch.complex128, device="cuda")
            ctx.decode(dec, outs[0].scale, zo, emb_ws, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, zo, (z, m, v, e0, e1, ct, out, dec, emb_ws, enc_ws, dec_ws))

    def finish(self, b: Batch):
        if self.keep_results:
            zo = b.handle[1].cpu().numpy()
            for i, r in enumerate(b.reqs):
                self.results[r.rid] = zo[i]
        b.handle = None


def build_plaintext_keys(contexts, device=0, secret_h=None):
    """Public key of each context's secret (the secret of build_gpu_state,
    with the same secret_h)."""
    import torch

    import synth
    keys = {}
    for log_n, (ctx, _) in contexts.items():
        N = ctx.N
        g = synth.rng(5, log_n, stream=1)
        s = torch.from_numpy(synth.secret(g, N, secret_h)).cuda()
        pa = synth.uniform_residues_torch(list(ctx.q), (), N, 0x7A + log_n, "cuda")
        pe = torch.from_numpy(synth.gaussian(synth.rng(6, log_n, stream=4), N)).cuda()
        pk = torch.empty((2, ctx.L, N), dtype=torch.uint64, device="cuda")
        ws = torch.empty(ctx.encrypt_workspace_size() // 8, dtype=torch.uint64, device="cuda")
        ctx.public_key(s, pa, pe, pk, ws)
        keys[log_n] = (s, pk)
    torch.cuda.synchronize()
    return keys


def poisson_arrivals(rate: float, seconds: float, rng) -> list[float]:
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        out.append(t)


def run_open_loop(sched: Scheduler, requests: list[Request], timeout: float = 600.0) -> float:
    """Feed requests at their arrival times (seconds from start) and run the
    scheduler until all complete. Returns the wall time."""
    t0 = time.perf_counter()
    i = 0
    n = len(requests)
    while True:
        now = time.perf_counter() - t0
        while i < n and requests[i].arrival <= now:
            requests[i].arrival = t0 + requests[i].arrival
            sched.submit(requests[i])
            i += 1
        sched.step(time.perf_counter())
        if i >= n and sched.idle():
            break
        if now > timeout:
            raise TimeoutError("serving run did not drain")
        if i < n and not sched.running and sched.pending() == 0:
            time.sleep(max(0.0, min(0.0005, requests[i].arrival - now)))
    return time.perf_counter() - t0


def latency_stats(reqs: list[Request]) -> dict:
    lat = sorted((r.done - r.arrival) * 1e3 for r in reqs)
    if not lat:
        return {}
    p = lambda f: lat[min(len(lat) - 1, max(0, math.ceil(f * len(lat)) - 1))]
    return {"p50_ms": round(p(0.50), 3), "p99_ms": round(p(0.99), 3), "mean_ms": round(statistics.mean(lat), 3),
            "max_ms": round(lat[-1], 3), "n": len(lat)}


# ---------------------------------------------------------------------------
# the mixed workload (k uniform in 2..12, N in {2^14, 2^15, 2^16},
# level uniform in [k, 24]) served at a Poisson rate
# ---------------------------------------------------------------------------
def mixed_requests(rate, seconds, seed, log_ns=(14, 15, 16), L=24, pool_size=64, k_range=(2, 12), partitions=None):
    import numpy as np
    g = np.random.default_rng(seed)
    arr = poisson_arrivals(rate, seconds, g)
    reqs = []
    for i, t in enumerate(arr):
        k = int(g.integers(k_range[0], k_range[1] + 1))
        log_n = int(g.choice(log_ns))
        level = int(g.integers(k, L + 1))
        cts = tuple(int(x) for x in g.integers(0, pool_size, size=k))
        reqs.append(Request(i, log_n, k, level, cts, arrival=t, partition=(partitions or {}).get(k)))
    return reqs


def plaintext_requests(rate, seconds, seed, log_ns=(14, 15, 16), L=24, pool_size=16, k_range=(2, 12),
                       partitions=None):
    """The mixed workload with slot vectors instead of pool ciphertexts: each
    request multiplies k slot vectors taken from a per-N pool of unit-disk
    vectors; its encryption noise is seeded by the request."""
    import numpy as np

    import synth
    g = np.random.default_rng(seed)
    pools = {log_n: [synth.unit_disk_slots(synth.rng(7, log_n * 100 + i, stream=6), 1 << (log_n - 1))
                     for i in range(pool_size)] for log_n in log_ns}
    reqs = []
    for i, t in enumerate(poisson_arrivals(rate, seconds, g)):
        k = int(g.integers(k_range[0], k_range[1] + 1))
        log_n = int(g.choice(log_ns))
        level = int(g.integers(k, L + 1))
        idx = [int(x) for x in g.integers(0, pool_size, size=k)]
        reqs.append(Request(i, log_n, k, level, tuple(idx), arrival=t, partition=(partitions or {}).get(k),
                            slots=np.stack([pools[log_n][j] for j in idx]), seed=seed * 1000003 + i))
    return reqs


def build_gpu_state(log_ns, L=24, K=8, dnum=3, t_max=12, pool_size=64, device=0, secret_h=None):
    """Contexts, resident keys (generated on the device) and ciphertext pools.
    secret_h: Hamming weight of the secret (None: uniform ternary)."""
    import numpy as np
    import torch

    import synth

    from . import Context
    contexts, pools = {}, {}
    for log_n in log_ns:
        params = synth.params_large(log_n=log_n, L=L, K=K, dnum=dnum)
        ctx = Context.from_params(params, device=device)
        g = synth.rng(5, log_n, stream=1)
        N = params.N
        s = torch.from_numpy(synth.secret(g, N, secret_h)).cuda()
        e = torch.from_numpy(np.stack([[synth.gaussian(g, N) for _ in range(dnum)] for _ in range(t_max - 1)])).cuda()
        a = synth.uniform_residues_torch(list(params.q) + list(params.p), (t_max - 1, dnum), N, 0x5E + log_n, "cuda")
        keys = torch.empty((t_max - 1, dnum, 2, L + K, N), dtype=torch.uint64, device="cuda")
        ws = torch.empty(ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device="cuda")
        ctx.keygen_evk(t_max, s, a, e, keys, ws)
        del a, ws
        evk = ctx.evk_set(t_max, keys)
        contexts[log_n] = (ctx, evk)
        pools[log_n] = synth.uniform_residues_torch(params.q, (pool_size, 2), N, 0x9000 + log_n, "cuda")
    torch.cuda.synchronize()
    return contexts, pools


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seconds", type=float, default=30.0)
    ap.add_argument("--streams", type=int, default=None, help="default: 4 for waves, 8 for groups")
    ap.add_argument("--max-batch", type=int, default=None, help="default: 64 for waves, 8 for groups")
    ap.add_argument("--cap-gb", type=float, default=150.0)
    ap.add_argument("--ws-gb", type=float, default=None,
                    help="workspace (scratch) per stream; default: 16 for waves, 6 for groups")
    ap.add_argument("--log-ns", default="14,15,16")
    ap.add_argument("--seed", type=int, default=2026)
    ap.add_argument("--secret-h", type=int, default=0,
                    help="Hamming weight of the secret (0: uniform ternary)")
    ap.add_argument("--plaintext", action="store_true",
                    help="requests carry slot vectors: encode, encrypt, multiply, decrypt, decode on the device")
    ap.add_argument("--k-max", type=int, default=12)
    ap.add_argument("--jsonl", default=None, help="write one JSON line per completed request to this file")
    ap.add_argument("--warmup-seconds", type=float, default=3.0,
                    help="untimed serving at the same rate first: the first launch of each (N, k, level, batch) "
                         "shape pays one-time costs (kernel loading, new allocator blocks) that otherwise "
                         "queue up the opening seconds")
    ap.add_argument("--criterion", default="table2", choices=["table2", "precision"],
                    help="partitions: Table II, or the precision search's (smallest inner tuple degree)")
    ap.add_argument("--engine", default="waves", choices=["waves", "groups"],
                    help="waves: cross-shape batches of one ring degree (any k, level, partition); "
                         "groups: batches of one (N, k, level, partition) shape")
    args = ap.parse_args()
    waves = args.engine == "waves" and not args.plaintext
    args.streams = args.streams or (4 if waves else 8)
    args.max_batch = args.max_batch or (64 if waves else 8)
    args.ws_gb = args.ws_gb or (16.0 if waves else 6.0)
    parts = None
    if args.criterion == "precision":
        from . import plan_optimize
        parts = {k: plan_optimize(k, "precision", 24, 8, 8)[0] for k in range(2, args.k_max + 1)}
    log_ns = tuple(int(x) for x in args.log_ns.split(","))
    h = args.secret_h or None
    contexts, pools = build_gpu_state(log_ns, pool_size=1 if args.plaintext else 64, secret_h=h)
    if args.plaintext:
        be = PlaintextBackend(contexts, build_plaintext_keys(contexts, secret_h=h), n_streams=args.streams,
                              ws_bytes=int(args.ws_gb * (1 << 30)), keep_results=True)

        def make(rate, seconds, seed, lns):
            return plaintext_requests(rate, seconds, seed, lns, k_range=(2, args.k_max), partitions=parts)
    else:
        if args.engine == "waves":
            be = WaveBackend(contexts, pools, n_streams=args.streams, ws_bytes=int(args.ws_gb * (1 << 30)))
        else:
            be = GpuBackend(contexts, pools, n_streams=args.streams, ws_bytes=int(args.ws_gb * (1 << 30)))

        def make(rate, seconds, seed, lns):
            return mixed_requests(rate, seconds, seed, lns, k_range=(2, args.k_max), partitions=parts)
    # the cap covers everything on the device: keys, pools, tables and stream
    # workspaces are resident; batches are admitted within what is left
    resident = be.resident_bytes()
    budget = int(args.cap_gb * 1e9) - resident
    if budget <= 0:
        raise SystemExit(f"resident state ({resident / 1e9:.1f} GB) exceeds the cap")
    warm = make(args.rate, args.warmup_seconds, args.seed + 1, log_ns)
    run_open_loop(Scheduler(be, budget, args.max_batch), warm)
    reqs = make(args.rate, args.seconds, args.seed, log_ns)
    sched = Scheduler(be, budget, args.max_batch)
    wall = run_open_loop(sched, reqs, timeout=args.seconds * 20 + 120)
    stats = latency_stats(sched.completed)
    if args.jsonl:
        t0 = min(r.arrival for r in reqs)
        with open(args.jsonl, "w") as f:
            for r in sorted(sched.completed, key=lambda r: r.arrival):
                f.write(json.dumps({"rid": r.rid, "log_n": r.log_n, "k": r.k, "level": r.level, "batch": r.batch,
                                    "arrival_s": round(r.arrival - t0, 6), "admitted_s": round(r.admitted - t0, 6),
                                    "done_s": round(r.done - t0, 6),
                                    "latency_ms": round((r.done - r.arrival) * 1e3, 3)}) + "\n")
    extra = {}
    if args.plaintext:
        import numpy as np
        err = {}
        for r in sched.completed:
            e = float(np.abs(be.results[r.rid] - np.prod(r.slots, axis=0)).max())
            err[r.k] = max(err.get(r.k, 0.0), e)
        extra = {"mode": "plaintext in / plaintext out", "max_abs_slot_error_per_k": dict(sorted(err.items())),
                 "secret": f"Hamming weight {h}" if h else "uniform ternary", "partitions": args.criterion}
    print(json.dumps({"metric": "served k-input ct-mults/s (Poisson arrivals, mixed k, N, level)",
                      "offered_rate": args.rate, "seconds": args.seconds, "warmup_seconds": args.warmup_seconds,
                      "requests": len(reqs),
                      "completed": len(sched.completed), "wall_s": round(wall, 3),
                      "sustained_ctmults_s": round(len(sched.completed) / wall, 1), "latency": stats,
                      "batches": sched.admitted_batches, "mean_batch": round(len(reqs) / max(1, sched.admitted_batches), 2),
                      "engine": "plaintext" if args.plaintext else args.engine,
                      "streams": args.streams, "max_batch": args.max_batch, "cap_gb": args.cap_gb,
                      "resident_gb": round(resident / 1e9, 2), "peak_allocated_gb": round(
                          __import__("torch").cuda.max_memory_allocated() / 1e9, 2), **extra}))


if __name__ == "__main__":
    main()
