"""The allocation-free rescale entry point (ckks_rescale_multi_noalloc).

It exists for callers that cannot allocate device memory where they rescale
(a component holding only device pointers handed to it, or a loop that must
not call cudaMalloc). Through the C ABI it must give the same residues as
ckks_rescale_multi with a caller workspace, on two calls in a row (the first
call also resolves the library's scratch array on this device), leave the
device's free memory unchanged, work in place, fill its fixed scratch
exactly at N = 2^16 with a 2-polynomial tuple at level 32 (checked against
the oracle's sequential rescales), and reject sizes beyond that scratch with
CKKS_ENOMEM. This file is collected last on purpose."""
import numpy as np
import pytest

import synth
from oracle import ckks as O

pytestmark = pytest.mark.gpu


def test_noalloc_rescale_matches_workspace_rescale():
    import torch

    import paper_2601_15401_gb300 as G
    params = synth.make_params(12, [50] * 8, 2, 2)
    ctx = G.Context.from_params(params)
    g = synth.rng(404)
    N, L = params.N, params.L
    for call, (polys, mu) in enumerate([(3, 2), (2, 5)]):
        A = np.stack([synth.uniform_residues(g, params.q, N) for _ in range(polys)])
        src = torch.from_numpy(A).cuda()
        ref = G.Tuple.wrap(torch.zeros((polys, L - mu, N), dtype=torch.uint64, device="cuda"))
        ws = torch.empty(ctx.rescale_workspace_size(polys, L, mu) // 8 + 1, dtype=torch.uint64, device="cuda")
        ctx.rescale_multi(G.Tuple.wrap(src.clone()), mu, ref, ws)
        got = G.Tuple.wrap(torch.zeros((polys, L - mu, N), dtype=torch.uint64, device="cuda"))
        inp = G.Tuple.wrap(src.clone())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        ctx.rescale_multi_noalloc(inp, mu, got)
        torch.cuda.synchronize()
        if call:  # after the first call has loaded the kernels and resolved the scratch
            assert torch.cuda.mem_get_info()[0] == free_before
        assert got.level == ref.level == L - mu
        assert np.array_equal(got.data.cpu().numpy(), ref.data.cpu().numpy()), f"call {call}"
    ctx.check()


def test_noalloc_follows_algorithm1_under_other_rescale_forms():
    """The entry point always runs Algorithm 1; the context's other rescale
    forms give the same residues through the workspace path."""
    import torch

    import paper_2601_15401_gb300 as G
    params = synth.make_params(11, [50] * 6, 2, 2)
    ctx = G.Context.from_params(params)
    g = synth.rng(405)
    N, L, polys, mu = params.N, params.L, 2, 3
    A = np.stack([synth.uniform_residues(g, params.q, N) for _ in range(polys)])
    want = np.stack([O.multi_rs_sequential(O.Ctx(params), A[p], mu) for p in range(polys)])
    for form in (1, 2):
        ctx.tune_set("inner_rescale", form)
        got = G.Tuple.wrap(torch.zeros((polys, L - mu, N), dtype=torch.uint64, device="cuda"))
        ctx.rescale_multi_noalloc(G.Tuple.wrap(torch.from_numpy(A).cuda()), mu, got)
        torch.cuda.synchronize()
        assert np.array_equal(got.data.cpu().numpy(), want), f"inner_rescale={form}"
    ctx.tune_set("inner_rescale", 0)
    ctx.check()


def test_noalloc_fills_capacity_at_full_size_and_in_place():
    """N = 2^16, a 2-polynomial tuple at level 32: the scratch is exactly the
    32 MiB capacity. Out of place and in place, equal to the oracle's mu
    sequential rescales (Eq. 6)."""
    import torch

    import paper_2601_15401_gb300 as G
    params = synth.make_params(16, [50] * 32, 2, 4)
    ctx = G.Context.from_params(params)
    octx = O.Ctx(params)
    N, L, polys = params.N, params.L, 2
    assert polys * L * N * 8 == G.Context.rescale_noalloc_capacity()
    g = synth.rng(406)
    A = np.stack([synth.uniform_residues(g, params.q, N) for _ in range(polys)])
    for mu, in_place in ((3, False), (5, True)):
        want = np.stack([O.multi_rs_sequential(octx, A[p], mu) for p in range(polys)])
        src = torch.from_numpy(A).cuda()
        inp = G.Tuple.wrap(src)
        if in_place:
            out = G.Tuple(src, polys, L - mu, L)
        else:
            out = G.Tuple.wrap(torch.zeros((polys, L - mu, N), dtype=torch.uint64, device="cuda"))
        ctx.rescale_multi_noalloc(inp, mu, out)
        torch.cuda.synchronize()
        got = out.data.cpu().numpy()[:, :L - mu]
        assert out.level == L - mu
        assert np.array_equal(got, want), f"mu={mu} in_place={in_place}"
    ctx.check()


def test_noalloc_rejects_sizes_beyond_capacity():
    import torch

    import paper_2601_15401_gb300 as G
    params = synth.make_params(16, [50] * 24, 2, 3)
    ctx = G.Context.from_params(params)
    assert G.Context.rescale_noalloc_capacity() == 32 << 20
    # 3 polynomials x 24 limbs x 512 KiB of scratch = 36 MiB > 32 MiB
    t = G.Tuple(torch.zeros((3, 24, params.N), dtype=torch.uint64, device="cuda"), 3, 24, 24)
    out = G.Tuple(torch.zeros((3, 23, params.N), dtype=torch.uint64, device="cuda"), 3, 23, 23)
    with pytest.raises(G.CkksError) as e:
        ctx.rescale_multi_noalloc(t, 1, out)
    assert e.value.code == -4
    # the timing hook on: refused rather than switched off
    ctx.profile(True)
    small = G.Tuple(torch.zeros((2, 24, params.N), dtype=torch.uint64, device="cuda"), 2, 24, 24)
    sout = G.Tuple(torch.zeros((2, 23, params.N), dtype=torch.uint64, device="cuda"), 2, 23, 23)
    with pytest.raises(G.CkksError) as e:
        ctx.rescale_multi_noalloc(small, 1, sout)
    assert e.value.code == -1
    ctx.profile(False)
    ctx.rescale_multi_noalloc(small, 1, sout)
    torch.cuda.synchronize()
    ctx.check()
