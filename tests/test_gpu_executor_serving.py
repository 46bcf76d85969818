"""Batched uneven workloads in one CUDA graph, and the continuous-batching
server: every result equals the same product computed alone (bit-exact)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def state():
    from paper_2601_15401_gb300.serve import build_gpu_state
    return build_gpu_state((10, 11), L=8, K=2, dnum=2, t_max=6, pool_size=24)


def _alone(contexts, pools, log_n, k, level, cts, partition=None):
    import torch

    import paper_2601_15401_gb300 as G
    ctx, evk = contexts[log_n]
    pool = pools[log_n]
    depth = ctx.plan_describe(k, partition)["depth"]
    ins = [G.Tuple(pool[c].contiguous(), 2, level, pool.shape[2]) for c in cts]
    out = G.Tuple.wrap(torch.zeros((2, level - depth, ctx.N), dtype=torch.uint64, device="cuda"))
    ws = torch.empty(ctx.workspace_size(k, level, 1, partition) // 8 + 1, dtype=torch.uint64, device="cuda")
    ctx.mul_k(ins, evk, out, ws, partition=partition)
    return out.data.cpu().numpy()


def test_graph_executor_uneven_batch_equals_alone(state):
    import torch

    from paper_2601_15401_gb300.executor import BatchExecutor, MulRequest
    contexts, pools = state
    g = np.random.default_rng(7)
    reqs, srcs = [], {}
    for i in range(40):
        k = int(g.integers(2, 7))
        log_n = int(g.choice([10, 11]))
        level = int(g.integers(k, 9)) if k > 2 else int(g.integers(2, 9))
        cts = tuple(int(x) for x in g.integers(0, 24, size=k))
        reqs.append(MulRequest(log_n, k, level, None, i))
        srcs[i] = cts
    ex = BatchExecutor(contexts, n_streams=4)
    ex.plan(reqs)
    for r in reqs:
        pool = pools[r.log_n]
        src = pool.view(torch.int64)[list(srcs[r.rid])][:, :, :r.level]
        ex.input_view(r.rid).view(torch.int64).copy_(src)
    ex.capture()
    ex.replay()
    torch.cuda.synchronize()
    for r in reqs[::3]:
        want = _alone(contexts, pools, r.log_n, r.k, r.level, srcs[r.rid])
        assert np.array_equal(ex.output_view(r.rid).cpu().numpy(), want)
    # a second replay gives the same results
    first = {r.rid: ex.output_view(r.rid).cpu().numpy() for r in reqs}
    ex.replay()
    torch.cuda.synchronize()
    for r in reqs:
        assert np.array_equal(ex.output_view(r.rid).cpu().numpy(), first[r.rid])


def test_serving_mix_equals_alone(state):
    from paper_2601_15401_gb300.serve import GpuBackend, Scheduler, mixed_requests, run_open_loop
    contexts, pools = state
    reqs = mixed_requests(400.0, 0.15, 11, log_ns=(10, 11), L=8, pool_size=24, k_range=(2, 6))
    assert len(reqs) > 20
    be = GpuBackend(contexts, pools, n_streams=4, ws_bytes=256 << 20, keep_results=True)
    sched = Scheduler(be, cap_bytes=int(8e9), max_batch=4)
    run_open_loop(sched, reqs, timeout=120)
    assert len(sched.completed) == len(reqs)
    assert any(len(b) > 0 for b in [sched.completed])
    for r in reqs:
        want = _alone(contexts, pools, r.log_n, r.k, r.level, r.cts)
        got = be.results[r.rid].cpu().numpy()
        assert np.array_equal(got, want), r


def test_wave_executor_uneven_batch_equals_alone(state):
    """The cross-shape executor (waves of any k and level, one CUDA graph):
    every product equals ckks_mul_k alone, also on a second replay."""
    import torch

    from paper_2601_15401_gb300.executor import MulRequest, WaveExecutor
    contexts, pools = state
    g = np.random.default_rng(8)
    reqs, srcs = [], {}
    for i in range(40):
        k = int(g.integers(2, 7))
        log_n = int(g.choice([10, 11]))
        level = int(g.integers(k, 9)) if k > 2 else int(g.integers(2, 9))
        reqs.append(MulRequest(log_n, k, level, None, i))
        srcs[i] = tuple(int(x) for x in g.integers(0, 24, size=k))
    ex = WaveExecutor(contexts, max_wave=16)
    ex.plan(reqs)
    for r in reqs:
        src = pools[r.log_n].view(torch.int64)[list(srcs[r.rid])][:, :, :r.level]
        ex.input_view(r.rid).view(torch.int64).copy_(src)
    ex.capture()
    ex.replay()
    torch.cuda.synchronize()
    first = {}
    for r in reqs:
        got = ex.output_view(r.rid).cpu().numpy()
        assert np.array_equal(got, _alone(contexts, pools, r.log_n, r.k, r.level, srcs[r.rid])), r
        first[r.rid] = got
    ex.replay()
    torch.cuda.synchronize()
    for r in reqs:
        assert np.array_equal(ex.output_view(r.rid).cpu().numpy(), first[r.rid])
    assert len(ex.waves) == sum(-(-sum(1 for r in reqs if r.log_n == n) // 16) for n in (10, 11))


def test_wave_serving_mix_equals_alone(state):
    """Continuous batching with cross-shape batches: requests of one ring
    degree share a batch whatever their k and level; every result equals the
    product computed alone."""
    from paper_2601_15401_gb300.serve import Scheduler, WaveBackend, mixed_requests, run_open_loop
    contexts, pools = state
    reqs = mixed_requests(400.0, 0.15, 12, log_ns=(10, 11), L=8, pool_size=24, k_range=(2, 6))
    assert len(reqs) > 20
    be = WaveBackend(contexts, pools, n_streams=2, ws_bytes=512 << 20, keep_results=True)
    sched = Scheduler(be, cap_bytes=int(8e9), max_batch=16)
    run_open_loop(sched, reqs, timeout=120)
    assert len(sched.completed) == len(reqs)
    for r in reqs:
        want = _alone(contexts, pools, r.log_n, r.k, r.level, r.cts)
        assert np.array_equal(be.results[r.rid].cpu().numpy(), want), r
