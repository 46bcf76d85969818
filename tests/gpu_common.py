"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
CUDA library (through the C ABI) and to the CPU oracle."""
from __future__ import annotations

import numpy as np

import synth
from oracle import ckks as O


def torch():
    import torch as T
    return T


def dev(a: np.ndarray):
    T = torch()
    return T.from_numpy(np.ascontiguousarray(a, dtype=np.uint64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy()


class Setup:
    """GPU context + oracle context + keys for one parameter set."""

    def __init__(self, params, t_max: int, config: int, gpu_keygen: bool = False):
        import paper_2601_15401_gb300 as G
        T = torch()
        self.params = params
        self.t_max = t_max
        self.octx = O.Ctx(params)
        self.ctx = G.Context.from_params(params)
        self.km = synth.key_material(params, t_max, config)
        self.okeys = O.keygen_all(self.octx, self.km, t_max)
        plain = np.stack([np.stack([np.stack([k[0], k[1]]) for k in row]) for row in self.okeys])
        if gpu_keygen:
            a = np.stack([np.stack(row) for row in self.km.a])
            e = np.stack([np.stack(row) for row in self.km.e])
            keys = T.empty(plain.shape, dtype=T.uint64, device="cuda")
            ws = T.empty(self.ctx.keygen_workspace_size() // 8, dtype=T.uint64, device="cuda")
            self.ctx.keygen_evk(t_max, T.from_numpy(self.km.s).cuda(), dev(a), T.from_numpy(e).cuda(), keys, ws)
            self.gpu_plain_keys = keys.clone()
        else:
            keys = dev(plain)
        self.plain_keys = plain
        self.evk = self.ctx.evk_set(t_max, keys)
        T.cuda.synchronize()

    def ws(self, nbytes: int):
        T = torch()
        return T.empty(max(1, (nbytes + 7) // 8), dtype=T.uint64, device="cuda")

    def tuple(self, arr: np.ndarray, level=None, scale=1.0):
        import paper_2601_15401_gb300 as G
        return G.Tuple.wrap(dev(arr), level=level, scale=scale)


def oracle_tuple(arr, scale=1.0):
    return O.Tup(np.ascontiguousarray(arr, dtype=np.uint64), scale)
