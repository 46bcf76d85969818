"""Small, self-contained launches of single library steps for timing and for
profiler captures (one kernel class at a time, a few GB on the device).

  python -m paper_2601_15401_gb300.microbench --op ntt --batch 16
  python -m paper_2601_15401_gb300.microbench --op mul_k --k 8 --batch 4
  python -m paper_2601_15401_gb300.microbench --op rotate --batch 16
  python -m paper_2601_15401_gb300.microbench --op precision --batch 4 --secret-h 64
  python -m paper_2601_15401_gb300.microbench --op peak

--op peak measures the GPU's rate of each integer operation of the hot path
(lazy Shoup product, lazy NTT butterfly, 64 x 64 -> 128-bit MAC, Montgomery
product) with register-only kernels over a sweep of grid sizes, for a 50-bit
and a 60-bit prime: the integer roofline the NTT / BConv / MAC fractions are
taken against.

--op precision prints, per k = 2..12, the largest slot error of the device
round trip encode -> encrypt -> k-input product -> decrypt -> decode
against the FP64 product of the slot vectors (no timing).

Prints one JSON line: per kernel class, launches, average event time and
achieved algorithmic GB/s (the library's timing hook).
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    import paper_2601_15401_gb300 as G
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["ntt", "mul_k", "mul2", "chain3", "rotate", "encode", "decode", "precision",
                                         "peak", "tensor_rates", "h2d"], default="ntt")
    ap.add_argument("--log-n", type=int, default=16)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--tune", action="append", default=[], help="key=value library tunable")
    ap.add_argument("--partition", default=None, help="partition text for --op mul_k (default Table II)")
    ap.add_argument("--primes", default="chain", choices=["chain", "q1"],
                    help="chain: the largest primes of each size that are 1 mod 2^17 (default); q1: primes = 1 "
                         "mod 2^32, for which the kernels take cheaper modular-product forms")
    ap.add_argument("--params", default="large", choices=["large", "mid", "small"],
                    help="large: 24 x 50-bit q, 8 x 60-bit p, dnum 3; mid: q_0 60-bit + 11 x 45-bit, 4 x 60-bit p, "
                         "dnum 3; small: 4 x 50-bit q, one 60-bit p, dnum 1")
    ap.add_argument("--graph", action="store_true", help="capture one rep in a CUDA graph and time its replays")
    ap.add_argument("--latency", action="store_true",
                    help="also time each rep alone on the host (launch to completion, synchronised)")
    ap.add_argument("--secret-h", type=int, default=0, help="--op precision: Hamming weight of s (0: uniform)")
    ap.add_argument("--scale-bits", type=int, default=50, help="--op precision: log2 of the encoding scale")
    ap.add_argument("--criterion", default="table2", choices=["table2", "precision"],
                    help="--op precision: Table II partitions or the precision search's")
    ap.add_argument("--seconds-compute", type=float, default=3.0, help="--op h2d: device work between probes")
    args = ap.parse_args()
    if args.op == "precision":
        return precision(args)
    if args.op == "peak":
        return peak(args)
    if args.op == "tensor_rates":
        return tensor_rates(args)
    if args.op == "h2d":
        return h2d(args)
    cong = synth.Q1_CONGRUENCE if args.primes == "q1" else synth.NTT_CONGRUENCE
    if args.params == "small":
        p = synth.params_small(log_n=args.log_n, congruence=cong)
    elif args.params == "mid":
        p = synth.params_mid(log_n=args.log_n, congruence=cong)
    else:
        p = synth.params_large(log_n=args.log_n, congruence=cong)
    ctx = G.Context.from_params(p)
    L, N, B = p.L, p.N, args.batch
    for kv in args.tune:
        key, val = kv.split("=")
        ctx.tune_set(key, int(val))
    if args.op == "ntt":
        x = synth.uniform_residues_torch(p.q, (B * 2,), N, 7, "cuda")  # [2B][L][N]
        T = G.Tuple(x, 2 * B, L, L, 0)

        def run():
            ctx.ntt(T)
            ctx.intt(T)
    elif args.op in ("encode", "decode"):
        z = torch.randn((B, N // 2), dtype=torch.complex128, device="cuda") * 0.5
        m = torch.empty((B, N), dtype=torch.int64, device="cuda")
        mf = torch.empty((B, N), dtype=torch.float64, device="cuda")
        ews = torch.empty(ctx.embed_workspace_size(B) // 8, dtype=torch.uint64, device="cuda")
        ctx.encode(z, 2.0 ** 40, m, ews)
        mf.copy_(m)

        def run():
            if args.op == "encode":
                ctx.encode(z, 2.0 ** 40, m, ews)
            else:
                ctx.decode(mf, 2.0 ** 40, z, ews)
    elif args.op == "rotate":
        import numpy as np
        g_el = ctx.galois_element(1)
        gen = synth.rng(9, 0, stream=1)
        s = torch.from_numpy(synth.ternary_secret(gen, N)).cuda()
        e = torch.from_numpy(np.stack([synth.gaussian(gen, N) for _ in range(p.dnum)])).cuda()
        a = synth.uniform_residues_torch(list(p.q) + list(p.p), (p.dnum,), N, 0x32, "cuda")
        keys = torch.empty((p.dnum, 2, L + p.K, N), dtype=torch.uint64, device="cuda")
        kws = torch.empty(ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device="cuda")
        ctx.keygen_galois(g_el, s, a, e, keys, kws)
        del a, kws
        gk = ctx.evk_set(2, keys)
        inp = synth.uniform_residues_torch(p.q, (B, 2), N, 13, "cuda")
        out = torch.empty((B, 2, L, N), dtype=torch.uint64, device="cuda")
        cts = [G.Tuple(inp[b], 2, L, L) for b in range(B)]
        outs = [G.Tuple(out[b], 2, L, L) for b in range(B)]
        ws = torch.empty(ctx.rotate_workspace_size(L, B) // 8 + 1, dtype=torch.uint64, device="cuda")

        def run():
            ctx.rotate_batch(cts, g_el, gk, outs, ws)
    else:
        t_max = max(args.k, 2)
        g = synth.rng(9, 0, stream=1)
        s = torch.from_numpy(synth.ternary_secret(g, N)).cuda()
        import numpy as np
        e = torch.from_numpy(np.stack([[synth.gaussian(g, N) for _ in range(p.dnum)] for _ in range(t_max - 1)])).cuda()
        a = synth.uniform_residues_torch(list(p.q) + list(p.p), (t_max - 1, p.dnum), N, 0x31, "cuda")
        keys = torch.empty((t_max - 1, p.dnum, 2, L + p.K, N), dtype=torch.uint64, device="cuda")
        kws = torch.empty(ctx.keygen_workspace_size() // 8, dtype=torch.uint64, device="cuda")
        ctx.keygen_evk(t_max, s, a, e, keys, kws)
        del a, kws
        evk = ctx.evk_set(t_max, keys)
        if args.op == "mul_k":
            k = args.k
            depth = ctx.plan_describe(k, args.partition)["depth"]
            inp = synth.uniform_residues_torch(p.q, (B, k, 2), N, 11, "cuda")
            out = torch.empty((B, 2, L - depth, N), dtype=torch.uint64, device="cuda")
            tup = [[G.Tuple(inp[b, u], 2, L, L) for u in range(k)] for b in range(B)]
            outs = [G.Tuple(out[b], 2, L - depth, L - depth) for b in range(B)]
            ws = torch.empty(ctx.workspace_size(k, L, B, args.partition) // 8 + 1, dtype=torch.uint64, device="cuda")

            def run():
                ctx.mul_k_batch(tup, evk, outs, ws, partition=args.partition)
        elif args.op == "chain3":
            # three inputs through two standard 2-input multiplies: (a b) c
            inp = synth.uniform_residues_torch(p.q, (B, 3, 2), N, 14, "cuda")
            ab = torch.empty((B, 2, L - 1, N), dtype=torch.uint64, device="cuda")
            out = torch.empty((B, 2, L - 2, N), dtype=torch.uint64, device="cuda")
            a_ = [G.Tuple(inp[b, 0], 2, L, L) for b in range(B)]
            b_ = [G.Tuple(inp[b, 1], 2, L, L) for b in range(B)]
            c_ = [G.Tuple(inp[b, 2], 2, L, L) for b in range(B)]
            abt = [G.Tuple(ab[b], 2, L - 1, L - 1) for b in range(B)]
            outs = [G.Tuple(out[b], 2, L - 2, L - 2) for b in range(B)]
            ws = torch.empty(ctx.mul2_workspace_size(L, B) // 8 + 1, dtype=torch.uint64, device="cuda")

            def run():
                ctx.mul2_batch(a_, b_, evk, abt, ws)
                ctx.mul2_batch(abt, c_, evk, outs, ws)
        else:
            inp = synth.uniform_residues_torch(p.q, (B, 2, 2), N, 12, "cuda")
            out = torch.empty((B, 2, L - 1, N), dtype=torch.uint64, device="cuda")
            a_ = [G.Tuple(inp[b, 0], 2, L, L) for b in range(B)]
            b_ = [G.Tuple(inp[b, 1], 2, L, L) for b in range(B)]
            outs = [G.Tuple(out[b], 2, L - 1, L - 1) for b in range(B)]
            ws = torch.empty(ctx.mul2_workspace_size(L, B) // 8 + 1, dtype=torch.uint64, device="cuda")

            def run():
                ctx.mul2_batch(a_, b_, evk, outs, ws)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    step = run
    if args.graph:
        import time as _t
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            run()  # one eager pass on the capture stream first
            side.synchronize()
            with torch.cuda.graph(graph, stream=side):
                run()
        torch.cuda.synchronize()

        def step():
            graph.replay()
    ctx.counters(reset=True)
    ctx.profile(not args.graph)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        step()
    e1.record()
    e1.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read() if not args.graph else {}
    latency = None
    if args.latency:
        import time as _t
        lat = []
        for _ in range(max(20, args.reps)):
            t = _t.perf_counter()
            step()
            torch.cuda.synchronize()
            lat.append((_t.perf_counter() - t) * 1e3)
        lat.sort()
        latency = {"p50_ms": round(lat[len(lat) // 2], 4), "min_ms": round(lat[0], 4), "n": len(lat)}
    ctx.check()
    print(json.dumps({
        "op": args.op, "params": args.params, "log_n": args.log_n, "batch": B, "k": args.k, "tune": args.tune,
        "partition": args.partition, "graph": args.graph, "latency": latency,
        "ms_per_rep": round(e0.elapsed_time(e1) / args.reps, 4), "counters_per_rep": {n: v // args.reps for n, v in ctx.counters().items()},
        "kernels": {n: {"launches": v["launches"], "avg_us": round(v["total_ms"] * 1e3 / v["launches"], 2),
                        "GBps": round(v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9, 1),
                        "Gops": round(v["int_ops"] / (v["total_ms"] / 1e3) / 1e9, 2)} for n, v in prof.items()}}))


def h2d(args):
    """Host-to-device bandwidth from pinned memory, 4 GiB: the copy engines
    (cudaMemcpyAsync through torch) against the GPU's own loads (ckks_pull
    over the mapped host memory); then the same after device-to-host traffic
    into a second pinned buffer and after seconds of device compute (the
    state a benchmark step leaves behind), and for host memory backed by
    transparent huge pages and registered with the driver."""
    import mmap

    import torch

    import paper_2601_15401_gb300 as G
    nbytes = 4 << 30
    words = nbytes // 8
    host = torch.empty(words, dtype=torch.int64, pin_memory=True)
    host.copy_(torch.arange(words, dtype=torch.int64))
    dev = torch.empty(words, dtype=torch.int64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {"op": "h2d", "bytes": nbytes}

    def rate(fn, n=nbytes, reps=3):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            out.append(round(n / (e0.elapsed_time(e1) / 1e3) / 1e9, 1))
        return out

    def probe(tag, src):
        res[f"{tag}/copy_engine_GBps"] = rate(lambda: dev.copy_(src, non_blocking=True))
        try:
            G.host_device_pointer(src)
        except G.CkksError:
            res[f"{tag}/pull_GBps"] = "host memory not mapped"
            return
        res[f"{tag}/pull_GBps"] = rate(lambda: G.pull(dev, src, blocks=sms * 8))

    probe("fresh", host)
    # device-to-host traffic into another pinned buffer
    back = torch.empty(words // 2, dtype=torch.int64, pin_memory=True)
    res["d2h_GBps"] = rate(lambda: back.copy_(dev[:words // 2], non_blocking=True), n=nbytes // 2)
    probe("after_d2h", host)
    # seconds of device work over 24 GiB of HBM
    big = torch.empty(3 * words, dtype=torch.int64, device="cuda")
    t_end = __import__("time").time() + args.seconds_compute
    while __import__("time").time() < t_end:
        big.add_(1)
        torch.cuda.synchronize()
    del big
    probe("after_compute", host)
    # transparent-huge-page host memory registered with the driver
    mm = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    try:
        mm.madvise(mmap.MADV_HUGEPAGE)
        res["thp"] = True
    except (AttributeError, OSError):
        res["thp"] = False
    thp = torch.frombuffer(mm, dtype=torch.int64)
    thp.copy_(host)
    rc = torch.cuda.cudart().cudaHostRegister(thp.data_ptr(), nbytes, 0)
    res["register_rc"] = int(rc.value if hasattr(rc, "value") else rc)
    if res["register_rc"] == 0:
        probe("thp_registered", thp)
        torch.cuda.cudart().cudaHostUnregister(thp.data_ptr())
    print(json.dumps(res))


def tensor_rates(args):
    """Dense tensor-core rates of this GPU through the vendor GEMMs (context
    for the BConv-as-GEMM question: an exact byte-split BConv would run as
    an INT8 GEMM with int32 accumulation): int8 x int8 -> int32
    (torch._int_mm) and bf16 (torch.matmul), 8192^3, best of 10 after
    warm-up, CUDA events."""
    import torch
    n = 8192
    res = {"op": "tensor_rates", "gpu": torch.cuda.get_device_name(0), "shape": [n, n, n]}

    def best(fn, flops):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return round(flops / (min(ms) / 1e3) / 1e12, 1)
    a8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device="cuda")
    b8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device="cuda")
    try:
        res["int8_tops"] = best(lambda: torch._int_mm(a8, b8), 2.0 * n ** 3)
    except Exception as e:  # no int8 GEMM in this torch build
        res["int8_error"] = str(e)[:200]
    ab = torch.randn((n, n), dtype=torch.bfloat16, device="cuda")
    bb = torch.randn((n, n), dtype=torch.bfloat16, device="cuda")
    res["bf16_tflops"] = best(lambda: ab @ bb, 2.0 * n ** 3)
    print(json.dumps(res))


def peak(args):
    import torch

    import paper_2601_15401_gb300 as G
    import synth
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {"op": "peak", "sms": sms, "gpu": torch.cuda.get_device_name(0), "unit": "G operations/s", "rates": {}}
    for bits in (50, 60):
        q = synth.prime_chain(bits, 1)[0]
        q1 = synth.prime_chain(bits, 1, congruence=1 << 32)[0]
        for kind in G.PEAK_KINDS:
            if kind.startswith("transpose") and bits == 60:
                continue
            best = 0.0
            for per_sm in (1, 2, 4, 8, 16):
                r = G.peak_int(kind, q1 if kind.endswith("_q1") else q, blocks=sms * per_sm, threads=256,
                               iters=2048)
                best = max(best, r)
                res["rates"][f"{kind}/{bits}bit/{per_sm}x256 per SM"] = round(r / 1e9, 2)
            res["rates"][f"{kind}/{bits}bit/best"] = round(best / 1e9, 2)
    print(json.dumps(res))


def precision(args):
    import numpy as np
    import torch

    import paper_2601_15401_gb300 as G
    import synth
    from .serve import build_gpu_state, build_plaintext_keys
    h = args.secret_h or None
    contexts, _ = build_gpu_state((args.log_n,), pool_size=1, secret_h=h)
    keys = build_plaintext_keys(contexts, secret_h=h)
    ctx, evk = contexts[args.log_n]
    s, pk = keys[args.log_n]
    N, L, B, scale = ctx.N, ctx.L, args.batch, 2.0 ** args.scale_bits
    rows = {}
    parts = {}
    for k in range(2, 13):
        part = None if args.criterion == "table2" else G.plan_optimize(k, "precision", L, ctx.K, ctx.alpha)[0]
        parts[k] = part or G.TABLE_II[k]
        zs = np.stack([synth.unit_disk_slots(synth.rng(11, k * 100 + i, stream=6), N // 2) for i in range(B * k)])
        ews = torch.empty(ctx.embed_workspace_size(B * k) // 8 + 1, dtype=torch.uint64, device="cuda")
        m = torch.empty((B * k, N), dtype=torch.int64, device="cuda")
        ctx.encode(torch.from_numpy(zs).cuda(), scale, m, ews)
        g = torch.Generator(device="cuda")
        g.manual_seed(1000 + k)
        v = torch.randint(-1, 2, (B * k, N), generator=g, device="cuda", dtype=torch.int64)
        e = (torch.randn((2, B * k, N), generator=g, device="cuda", dtype=torch.float64) * synth.SIGMA).round()
        e = e.clamp_(-synth.ERR_CLIP, synth.ERR_CLIP).to(torch.int64)
        ct = torch.empty((B * k, 2, L, N), dtype=torch.uint64, device="cuda")
        cts = [G.Tuple(ct[i], 2, L, L, scale=scale) for i in range(B * k)]
        ws = torch.empty(ctx.encrypt_batch_workspace_size(L, B * k) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.encrypt_batch(m, v, e[0].contiguous(), e[1].contiguous(), pk, L, cts, ws)
        for t in cts:
            t.scale = scale
        depth = ctx.plan_describe(k, part)["depth"]
        out = torch.empty((B, 2, L - depth, N), dtype=torch.uint64, device="cuda")
        outs = [G.Tuple(out[b], 2, L - depth, L - depth) for b in range(B)]
        mws = torch.empty(ctx.workspace_size(k, L, B, part) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.mul_k_batch([cts[b * k:(b + 1) * k] for b in range(B)], evk, outs, mws, partition=part)
        dec = torch.empty((B, N), dtype=torch.float64, device="cuda")
        dws = torch.empty(ctx.decrypt_batch_workspace_size(B) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.decrypt_batch(outs, s, dec, dws)
        zo = torch.empty((B, N // 2), dtype=torch.complex128, device="cuda")
        ctx.decode(dec, outs[0].scale, zo, ews)
        want = np.prod(zs.reshape(B, k, N // 2), axis=1)
        err = float(np.abs(zo.cpu().numpy() - want).max())
        rows[k] = {"max_abs_err": err, "log2": round(float(np.log2(err)), 1) if err > 0 else None,
                   "partition": parts[k]}
        del ct, ws, mws, out, dec, ews, m
        torch.cuda.empty_cache()
    print(json.dumps({"op": "precision", "log_n": args.log_n, "L": L, "K": ctx.K, "dnum": ctx.dnum,
                      "scale_bits": args.scale_bits, "batch": B, "criterion": args.criterion,
                      "secret": f"Hamming weight {h}" if h else "uniform ternary", "per_k": rows}))


if __name__ == "__main__":
    main()
