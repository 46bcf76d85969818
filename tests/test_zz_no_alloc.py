"""The allocation-free rescale entry point (ckks_rescale_multi_noalloc),
for callers that cannot allocate device memory where they rescale: through
the C ABI it must give the same residues as ckks_rescale_multi with a
caller workspace, on two calls in a row (the first call also resolves the
library's scratch array on this device), and reject sizes beyond its fixed
scratch with CKKS_ENOMEM. This file is collected last on purpose."""
import numpy as np
import pytest

import synth

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
        ctx.rescale_multi_noalloc(G.Tuple.wrap(src.clone()), mu, got)
        torch.cuda.synchronize()
        assert got.level == ref.level == L - mu
        assert np.array_equal(got.data.cpu().numpy(), ref.data.cpu().numpy()), f"call {call}"
    ctx.check()


def test_noalloc_rejects_sizes_beyond_capacity():
    import torch

    import paper_2601_15401_gb300 as G
    params = synth.make_params(16, [50] * 24, 2, 3)
    ctx = G.Context.from_params(params)
    assert G.Context.rescale_noalloc_capacity() == 32 << 20
    # 13 polynomials x 24 limbs x 512 KiB of scratch > 32 MiB
    t = G.Tuple(torch.zeros((13, 24, params.N), dtype=torch.uint64, device="cuda"), 13, 24, 24)
    out = G.Tuple(torch.zeros((13, 23, params.N), dtype=torch.uint64, device="cuda"), 13, 23, 23)
    with pytest.raises(G.CkksError) as e:
        ctx.rescale_multi_noalloc(t, 1, out)
    assert e.value.code == -4
