"""Python binding of libckks_mulk.so (include/ckks_mulk.h): argument
marshalling only. Every step of the multiplication runs in the library's CUDA
kernels; there is no CPU or PyTorch fallback: the first call into the library
(e.g. creating a Context) raises ImportError when libckks_mulk.so is missing.

Device memory and streams come from PyTorch: tuples are torch.uint64 CUDA
tensors shaped [n_polys][poly_stride][N] (or [batch][n_polys][stride][N]).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from ._lib import ERRORS, CkksError, lib, library_path

__all__ = ["Context", "Tuple", "Wave", "CkksError", "library_path", "lib", "TABLE_II", "plan_optimize"]

TABLE_II = {
    2: "(1,1)", 3: "(1,1,1)", 4: "(2,2)", 5: "(2,2,1)", 6: "(3,3)", 7: "(4,3)|(2,2)",
    8: "(4,4)|(2,2),(2,2)", 9: "(3,3,3)", 10: "(3,3,4)|(2,2)", 11: "(4,4,3)|(2,2),(2,2)",
    12: "(6,6)|(3,3),(3,3)",
}


def _as_real_pairs(z):
    """A contiguous complex128 or float64 [..., 2] tensor as float64 pairs."""
    import torch
    if z.dtype == torch.complex128:
        z = torch.view_as_real(z)
    if z.dtype != torch.float64 or not z.is_contiguous():
        raise ValueError("slots must be a contiguous complex128 (or float64 [..., 2]) tensor")
    return z


class _Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("L", ctypes.c_uint32), ("K", ctypes.c_uint32),
                ("dnum", ctypes.c_uint32), ("q", ctypes.POINTER(ctypes.c_uint64)),
                ("p", ctypes.POINTER(ctypes.c_uint64))]


class _Tuple(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n_polys", ctypes.c_uint32), ("level", ctypes.c_uint32),
                ("poly_stride", ctypes.c_uint32), ("ntt_form", ctypes.c_uint32), ("scale", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("ct", ctypes.c_void_p), ("k", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("evk", ctypes.c_void_p), ("plan", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class _WaveItem(ctypes.Structure):
    _fields_ = [("ct", ctypes.c_void_p), ("k", ctypes.c_uint32), ("plan", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class _KStats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("int_ops", ctypes.c_double)]


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("limb_ntt", "limb_intt", "ntt_phase", "intt_phase", "bconv", "kernels")]


def _check(rc: int, what: str):
    if rc != 0:
        raise CkksError(rc, f"{what}: {ERRORS.get(rc, rc)} ({lib().ckks_strerror(rc).decode()})")


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


@dataclass
class Tuple:
    """A tuple of polynomials in device memory.

    data: torch.uint64 CUDA tensor; polynomial a, limb j lives at
    data.view(-1)[(a * poly_stride + j) * N : ...]."""
    data: object
    n_polys: int
    level: int
    poly_stride: int
    ntt_form: int = 1
    scale: float = 1.0

    def c(self) -> _Tuple:
        return _Tuple(self.data.data_ptr(), self.n_polys, self.level, self.poly_stride, self.ntt_form, self.scale)

    @staticmethod
    def wrap(t, level=None, ntt_form=1, scale=1.0) -> "Tuple":
        """t: [n_polys][stride][N] tensor."""
        n_polys, stride = int(t.shape[0]), int(t.shape[1])
        return Tuple(t, n_polys, level if level is not None else stride, stride, ntt_form, scale)

    def limbs(self):
        """View [n_polys][level][N] of the active limbs."""
        return self.data[:, :self.level]


class Context:
    """One parameter set (N, Q, P, dnum) on one device."""

    def __init__(self, log_n: int, q, p, dnum: int, device: int = 0):
        self.log_n, self.N = log_n, 1 << log_n
        self.q, self.p = [int(x) for x in q], [int(x) for x in p]
        self.L, self.K, self.dnum = len(self.q), len(self.p), dnum
        self.alpha = -(-self.L // dnum)
        self.device = device
        qa = (ctypes.c_uint64 * self.L)(*self.q)
        pa = (ctypes.c_uint64 * self.K)(*self.p)
        prm = _Params(log_n, self.L, self.K, dnum, qa, pa)
        h = ctypes.c_void_p()
        _check(lib().ckks_context_create(ctypes.byref(prm), device, ctypes.byref(h)), "ckks_context_create")
        self._h = h
        self._plans = {}

    @classmethod
    def from_params(cls, params, device: int = 0) -> "Context":
        return cls(params.log_n, params.q, params.p, params.dnum, device)

    def close(self):
        if getattr(self, "_h", None):
            for pl in self._plans.values():
                lib().ckks_plan_destroy(pl)
            self._plans = {}
            lib().ckks_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ keys
    def keygen_workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_keygen_workspace_size(self._h, ctypes.byref(n)), "ckks_keygen_workspace_size")
        return n.value

    def keygen_evk(self, t_max, s, a, e, keys, workspace, stream=None):
        _check(lib().ckks_keygen_evk(self._h, t_max, s.data_ptr(), a.data_ptr(), e.data_ptr(), keys.data_ptr(),
                                     workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                     _stream(stream)), "ckks_keygen_evk")

    # ------------------------------------------------------- around the product
    def encrypt_workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_encrypt_workspace_size(self._h, ctypes.byref(n)), "ckks_encrypt_workspace_size")
        return n.value

    def check_residues(self, t: "Tuple", stream=None) -> int:
        """Number of residues outside [0, q) in the tuple's active limbs."""
        c = t.c()
        n = ctypes.c_uint64()
        _check(lib().ckks_check_residues(self._h, ctypes.byref(c), ctypes.byref(n), _stream(stream)),
               "ckks_check_residues")
        return n.value

    def embed_workspace_size(self, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_embed_workspace_size(self._h, batch, ctypes.byref(n)), "ckks_embed_workspace_size")
        return n.value

    def encode(self, z, scale: float, m, workspace, stream=None):
        """z: complex128 (or float64 [..., 2]) CUDA tensor [batch][N/2];
        m: int64 CUDA tensor [batch][N] <- rounded canonical-embedding coefficients."""
        zr = _as_real_pairs(z)
        batch = zr.numel() // self.N
        _check(lib().ckks_encode(self._h, zr.data_ptr(), batch, float(scale), m.data_ptr(), workspace.data_ptr(),
                                 workspace.numel() * workspace.element_size(), _stream(stream)), "ckks_encode")
        return m

    def decode(self, m, scale: float, z, workspace, stream=None):
        """m: float64 CUDA tensor [batch][N]; z: complex128 CUDA tensor [batch][N/2]."""
        zr = _as_real_pairs(z)
        batch = m.numel() // self.N
        _check(lib().ckks_decode(self._h, m.data_ptr(), batch, float(scale), zr.data_ptr(), workspace.data_ptr(),
                                 workspace.numel() * workspace.element_size(), _stream(stream)), "ckks_decode")
        return z

    def public_key(self, s, a, e, pk, workspace, stream=None):
        _check(lib().ckks_public_key(self._h, s.data_ptr(), a.data_ptr(), e.data_ptr(), pk.data_ptr(),
                                     workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                     _stream(stream)), "ckks_public_key")

    def encrypt(self, m, v, e0, e1, pk, level: int, out: Tuple, workspace, stream=None) -> Tuple:
        o = out.c()
        _check(lib().ckks_encrypt(self._h, m.data_ptr(), v.data_ptr(), e0.data_ptr(), e1.data_ptr(), pk.data_ptr(),
                                  level, ctypes.byref(o), workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(), _stream(stream)), "ckks_encrypt")
        out.level, out.n_polys, out.ntt_form, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.poly_stride
        return out

    def encrypt_batch_workspace_size(self, level: int, batch: int) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_encrypt_batch_workspace_size(self._h, level, batch, ctypes.byref(n)),
               "ckks_encrypt_batch_workspace_size")
        return n.value

    def encrypt_batch(self, m, v, e0, e1, pk, level: int, outs, workspace, stream=None):
        """m, v, e0, e1: int64 CUDA tensors [batch][N]; outs: evenly strided Tuples."""
        B = len(outs)
        oo = (_Tuple * B)(*[t.c() for t in outs])
        _check(lib().ckks_encrypt_batch(self._h, m.data_ptr(), v.data_ptr(), e0.data_ptr(), e1.data_ptr(), B,
                                        pk.data_ptr(), level, oo, workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_encrypt_batch")
        for o, r in zip(outs, oo):
            o.level, o.n_polys, o.ntt_form, o.poly_stride = r.level, r.n_polys, r.ntt_form, r.poly_stride
        return outs

    def decrypt_batch_workspace_size(self, batch: int) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_decrypt_batch_workspace_size(self._h, batch, ctypes.byref(n)),
               "ckks_decrypt_batch_workspace_size")
        return n.value

    def decrypt_batch(self, cts, s, out, workspace, stream=None):
        """cts: evenly strided Tuples; out: float64 CUDA tensor [batch][N]."""
        B = len(cts)
        cc = (_Tuple * B)(*[t.c() for t in cts])
        _check(lib().ckks_decrypt_batch(self._h, cc, B, s.data_ptr(), out.data_ptr(), workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_decrypt_batch")
        return out

    def decrypt(self, ct: Tuple, s, out, workspace, stream=None):
        """out: float64 CUDA tensor [N] <- centred c_0 + c_1 s (two lowest limbs)."""
        c = ct.c()
        _check(lib().ckks_decrypt(self._h, ctypes.byref(c), s.data_ptr(), out.data_ptr(), workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(), _stream(stream)), "ckks_decrypt")
        return out

    # -------------------------------------------------------------- rotation
    def galois_element(self, r: int) -> int:
        """g = 5^r mod 2N (the automorphism that rotates the slots by r)."""
        g = ctypes.c_uint32()
        _check(lib().ckks_galois_element(self._h, int(r), ctypes.byref(g)), "ckks_galois_element")
        return g.value

    def automorphism(self, t: Tuple, g: int, out: Tuple, stream=None) -> Tuple:
        c, o = t.c(), out.c()
        _check(lib().ckks_automorphism(self._h, ctypes.byref(c), g, ctypes.byref(o), _stream(stream)),
               "ckks_automorphism")
        out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride
        return out

    def keygen_galois(self, g: int, s, a, e, keys, workspace, stream=None):
        """keys [dnum][2][L+K][N] <- the Galois key of g; adopt with evk_set(2, keys)."""
        _check(lib().ckks_keygen_galois(self._h, g, s.data_ptr(), a.data_ptr(), e.data_ptr(), keys.data_ptr(),
                                        workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "ckks_keygen_galois")

    def rotate_workspace_size(self, level: int, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_rotate_workspace_size(self._h, level, batch, ctypes.byref(n)), "ckks_rotate_workspace_size")
        return n.value

    def rotate_batch(self, cts, g: int, gk, outs, workspace, stream=None):
        """cts, outs: lists over the batch of Tuples (evenly strided)."""
        B = len(cts)
        ii = (_Tuple * B)(*[t.c() for t in cts])
        oo = (_Tuple * B)(*[t.c() for t in outs])
        _check(lib().ckks_rotate_batch(self._h, ii, B, g, gk._h, oo, workspace.data_ptr(),
                                       workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_rotate_batch")
        for o, r in zip(outs, oo):
            o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride = r.level, r.n_polys, r.ntt_form, r.scale, r.poly_stride
        return outs

    def rotate(self, ct: Tuple, g: int, gk, out: Tuple, workspace, stream=None) -> Tuple:
        return self.rotate_batch([ct], g, gk, [out], workspace, stream)[0]

    def evk_set(self, t_max: int, keys, stream=None) -> "EvkSet":
        h = ctypes.c_void_p()
        _check(lib().ckks_evk_set_create(self._h, t_max, keys.data_ptr(), _stream(stream), ctypes.byref(h)),
               "ckks_evk_set_create")
        return EvkSet(self, h, keys, t_max)

    # ----------------------------------------------------------------- plans
    def plan(self, k: int, partition: str | None = None):
        key = (k, partition)
        if key not in self._plans:
            h = ctypes.c_void_p()
            part = partition.encode() if partition else None
            _check(lib().ckks_plan_create(self._h, k, part, ctypes.byref(h)), f"ckks_plan_create({k}, {partition})")
            self._plans[key] = h
        return self._plans[key]

    def plan_describe(self, k: int, partition: str | None = None):
        d, r, n = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().ckks_plan_describe(self.plan(k, partition), ctypes.byref(d), ctypes.byref(r), ctypes.byref(n)),
               "ckks_plan_describe")
        return {"depth": d.value, "rs_units": r.value, "nodes": n.value}

    def plan_optimize(self, k: int, criterion: str = "transforms", level: int | None = None):
        """Cheapest valid partition of k inputs: criterion "rs_units" (Table
        II's count) or "transforms" (limb (I)NTTs at `level`, default L)."""
        return plan_optimize(k, criterion, level if level is not None else self.L, self.K, self.alpha)

    def plan_cost(self, k: int, partition: str | None = None, criterion: str = "transforms",
                  level: int | None = None) -> float:
        v = ctypes.c_double()
        crit = {"rs_units": 0, "transforms": 1, "precision": 2}[criterion]
        _check(lib().ckks_plan_cost(self.plan(k, partition), crit, level if level is not None else self.L, self.K,
                                    self.alpha, ctypes.byref(v)), "ckks_plan_cost")
        return v.value

    def workspace_size(self, k: int, level: int, batch: int = 1, partition: str | None = None) -> int:
        n = ctypes.c_size_t()
        _check(lib().ckks_workspace_size(self._h, self.plan(k, partition), level, batch, ctypes.byref(n)),
               "ckks_workspace_size")
        return n.value

    # -------------------------------------------------------------- multiply
    def mul_k(self, cts, evk, out: Tuple, workspace, partition=None, stream=None) -> Tuple:
        k = len(cts)
        arr = (_Tuple * k)(*[c.c() for c in cts])
        o = out.c()
        _check(lib().ckks_mul_k(self._h, arr, k, evk._h, self.plan(k, partition), ctypes.byref(o),
                                workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                _stream(stream)), "ckks_mul_k")
        out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride
        return out

    def mul_k_batch(self, cts, evk, outs, workspace, partition=None, stream=None):
        """cts: list over batch of lists of k Tuples (strided views of batched
        tensors); outs: list over batch of Tuples."""
        B, k = len(cts), len(cts[0])
        arr = (_Tuple * (B * k))(*[c.c() for row in cts for c in row])
        oarr = (_Tuple * B)(*[o.c() for o in outs])
        _check(lib().ckks_mul_k_batch(self._h, arr, k, B, evk._h, self.plan(k, partition), oarr,
                                      workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                      _stream(stream)), "ckks_mul_k_batch")
        for o, r in zip(outs, oarr):
            o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride = r.level, r.n_polys, r.ntt_form, r.scale, r.poly_stride
        return outs

    def _requests(self, groups, evk):
        """groups: list of (cts [batch][k] Tuples, outs [batch] Tuples, partition or None)."""
        keep, reqs = [], []
        for cts, outs, part in groups:
            k = len(cts[0])
            arr = (_Tuple * (len(cts) * k))(*[c.c() for row in cts for c in row])
            oarr = (_Tuple * len(outs))(*[o.c() for o in outs])
            keep.append((arr, oarr, outs))
            reqs.append(_Request(ctypes.cast(arr, ctypes.c_void_p), k, len(cts), evk._h, self.plan(k, part),
                                 ctypes.cast(oarr, ctypes.c_void_p)))
        return (_Request * len(reqs))(*reqs), keep

    def requests_workspace_size(self, groups, evk) -> int:
        rr, _ = self._requests(groups, evk)
        n = ctypes.c_size_t()
        _check(lib().ckks_requests_workspace_size(self._h, rr, len(groups), ctypes.byref(n)),
               "ckks_requests_workspace_size")
        return n.value

    def mul_k_requests(self, groups, evk, workspace, stream=None) -> int:
        """Uneven groups of k-input products in one call (see the header);
        returns the number of groups enqueued."""
        rr, keep = self._requests(groups, evk)
        done = ctypes.c_uint32()
        _check(lib().ckks_mul_k_requests(self._h, rr, len(groups), ctypes.byref(done), workspace.data_ptr(),
                                         workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_mul_k_requests")
        for arr, oarr, outs in keep:
            for o, r in zip(outs, oarr):
                o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride = r.level, r.n_polys, r.ntt_form, r.scale, r.poly_stride
        return done.value

    def rescale(self, t: Tuple, out: Tuple, workspace, stream=None) -> Tuple:
        c, o = t.c(), out.c()
        _check(lib().ckks_rescale(self._h, ctypes.byref(c), ctypes.byref(o), workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(), _stream(stream)), "ckks_rescale")
        out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride
        return out

    def mul2_workspace_size(self, level: int, batch: int = 1) -> int:
        v = ctypes.c_size_t()
        _check(lib().ckks_mul2_workspace_size(self._h, level, batch, ctypes.byref(v)), "ckks_mul2_workspace_size")
        return v.value

    def mul2_batch(self, a, b, evk, outs, workspace, stream=None):
        """a, b, outs: lists over the batch of Tuples (evenly strided)."""
        B = len(a)
        aa = (_Tuple * B)(*[t.c() for t in a])
        bb = (_Tuple * B)(*[t.c() for t in b])
        oo = (_Tuple * B)(*[t.c() for t in outs])
        _check(lib().ckks_mul2_batch(self._h, aa, bb, B, evk._h, oo, workspace.data_ptr(),
                                     workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_mul2_batch")
        for o, r in zip(outs, oo):
            o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride = r.level, r.n_polys, r.ntt_form, r.scale, r.poly_stride
        return outs

    def mul2(self, a: Tuple, b: Tuple, evk, out: Tuple, workspace, stream=None) -> Tuple:
        o = out.c()
        ca, cb = a.c(), b.c()
        _check(lib().ckks_mul2(self._h, ctypes.byref(ca), ctypes.byref(cb), evk._h, ctypes.byref(o),
                               workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_mul2")
        out.level, out.n_polys, out.ntt_form, out.scale = o.level, o.n_polys, o.ntt_form, o.scale
        return out

    # ----------------------------------------------------------------- steps
    def tensor(self, ins, out: Tuple, stream=None) -> Tuple:
        arr = (_Tuple * len(ins))(*[t.c() for t in ins])
        o = out.c()
        _check(lib().ckks_tensor(self._h, arr, len(ins), ctypes.byref(o), _stream(stream)), "ckks_tensor")
        out.level, out.n_polys, out.ntt_form, out.scale = o.level, o.n_polys, o.ntt_form, o.scale
        return out

    def relin_workspace_size(self, n: int, level: int) -> int:
        v = ctypes.c_size_t()
        _check(lib().ckks_relin_workspace_size(self._h, n, level, ctypes.byref(v)), "ckks_relin_workspace_size")
        return v.value

    def relin(self, d: Tuple, evk, out: Tuple, workspace, out_ntt: bool = False, stream=None) -> Tuple:
        cd, o = d.c(), out.c()
        _check(lib().ckks_relin(self._h, ctypes.byref(cd), evk._h, int(out_ntt), ctypes.byref(o),
                                workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                _stream(stream)), "ckks_relin")
        out.level, out.n_polys, out.ntt_form, out.scale = o.level, o.n_polys, o.ntt_form, o.scale
        return out

    def rescale_workspace_size(self, n_polys: int, level: int, mu: int) -> int:
        v = ctypes.c_size_t()
        _check(lib().ckks_rescale_workspace_size(self._h, n_polys, level, mu, ctypes.byref(v)),
               "ckks_rescale_workspace_size")
        return v.value

    def rescale_multi(self, t: Tuple, mu: int, out: Tuple, workspace, stream=None) -> Tuple:
        ci, o = t.c(), out.c()
        _check(lib().ckks_rescale_multi(self._h, ctypes.byref(ci), mu, ctypes.byref(o), workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(), _stream(stream)),
               "ckks_rescale_multi")
        out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride
        return out

    def rescale_multi_noalloc(self, t: Tuple, mu: int, out: Tuple, stream=None) -> Tuple:
        """Algorithm 1 with the library's fixed scratch array (no workspace,
        no allocation); see ckks_rescale_multi_noalloc in the header."""
        ci, o = t.c(), out.c()
        _check(lib().ckks_rescale_multi_noalloc(self._h, ctypes.byref(ci), mu, ctypes.byref(o), _stream(stream)),
               "ckks_rescale_multi_noalloc")
        out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = o.level, o.n_polys, o.ntt_form, o.scale, o.poly_stride
        return out

    @staticmethod
    def rescale_noalloc_capacity() -> int:
        return lib().ckks_rescale_noalloc_capacity()

    def ntt(self, t: Tuple, out: Tuple | None = None, stream=None) -> Tuple:
        out = out or t
        ci, o = t.c(), out.c()
        _check(lib().ckks_ntt(self._h, ctypes.byref(ci), ctypes.byref(o), _stream(stream)), "ckks_ntt")
        out.level, out.n_polys, out.ntt_form = o.level, o.n_polys, o.ntt_form
        return out

    def intt(self, t: Tuple, out: Tuple | None = None, stream=None) -> Tuple:
        out = out or t
        ci, o = t.c(), out.c()
        _check(lib().ckks_intt(self._h, ctypes.byref(ci), ctypes.byref(o), _stream(stream)), "ckks_intt")
        out.level, out.n_polys, out.ntt_form = o.level, o.n_polys, o.ntt_form
        return out

    # ---------------------------------------------------------------- status
    def counters(self, reset: bool = False) -> dict:
        c = _Counters()
        _check(lib().ckks_counters(self._h, ctypes.byref(c), int(reset)), "ckks_counters")
        return {n: getattr(c, n) for n, _ in _Counters._fields_}

    def check(self):
        _check(lib().ckks_check(self._h), "ckks_check")

    def tune_set(self, key: str, value: int):
        _check(lib().ckks_tune_set(self._h, key.encode(), int(value)), f"ckks_tune_set({key})")

    def tune_get(self, key: str) -> int:
        v = ctypes.c_int()
        _check(lib().ckks_tune_get(self._h, key.encode(), ctypes.byref(v)), f"ckks_tune_get({key})")
        return v.value

    def profile(self, enable: bool):
        _check(lib().ckks_profile_enable(self._h, int(enable)), "ckks_profile_enable")

    def profile_read(self) -> dict:
        arr = (_KStats * 16)()
        n = ctypes.c_uint32()
        _check(lib().ckks_profile_read(self._h, arr, 16, ctypes.byref(n)), "ckks_profile_read")
        return {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms,
                                       "alg_bytes": arr[i].alg_bytes, "int_ops": arr[i].int_ops}
                for i in range(n.value)}


class Wave:
    """A cross-shape batch of k-input products of one context (ckks_wave_*):
    items = [(inputs: list of k Tuples, out: Tuple, partition or None)], any
    mix of k, partitions and levels. Every stage of every product runs in one
    launch per stage (job tables on the device); results equal ckks_mul_k on
    each item alone. The wave borrows the tuples' device memory."""

    def __init__(self, ctx: "Context", items, evk):
        self.ctx = ctx
        self._keep = []
        arr = (_WaveItem * len(items))()
        self.outs = []
        for i, (cts, out, part) in enumerate(items):
            k = len(cts)
            ct = (_Tuple * k)(*[c.c() for c in cts])
            o = out.c()
            self._keep += [ct, o]
            arr[i] = _WaveItem(ctypes.cast(ct, ctypes.c_void_p), k, ctx.plan(k, part), ctypes.addressof(o))
            self.outs.append((out, o))
        self._keep.append(arr)
        h = ctypes.c_void_p()
        _check(lib().ckks_wave_create(ctx._h, arr, len(items), evk._h, ctypes.byref(h)), "ckks_wave_create")
        self._h = h

    def workspace_size(self) -> tuple:
        """(table bytes, scratch bytes) of the two device buffers a run needs."""
        t, n = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().ckks_wave_workspace_size(self._h, ctypes.byref(t), ctypes.byref(n)), "ckks_wave_workspace_size")
        return t.value, n.value

    def buffers(self, device="cuda"):
        """Freshly allocated (tables, scratch) uint64 device buffers of the needed sizes."""
        import torch
        t, n = self.workspace_size()
        return (torch.empty(max(1, t // 8 + 32), dtype=torch.uint64, device=device),
                torch.empty(max(1, n // 8 + 32), dtype=torch.uint64, device=device))

    def run(self, tables, scratch, stream=None):
        _check(lib().ckks_wave_run(self._h, tables.data_ptr(), tables.numel() * tables.element_size(),
                                   scratch.data_ptr(), scratch.numel() * scratch.element_size(), _stream(stream)),
               "ckks_wave_run")
        for out, o in self.outs:
            out.level, out.n_polys, out.ntt_form, out.scale, out.poly_stride = (o.level, o.n_polys, o.ntt_form,
                                                                                o.scale, o.poly_stride)

    def describe(self) -> dict:
        n, h = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().ckks_wave_describe(self._h, ctypes.byref(n), ctypes.byref(h)), "ckks_wave_describe")
        return {"launches": n.value, "heights": h.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ckks_wave_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_device_pointer(host_tensor) -> int:
    """Device address of a pinned host tensor's memory."""
    d = ctypes.c_void_p()
    _check(lib().ckks_host_device_pointer(ctypes.c_void_p(host_tensor.data_ptr()), ctypes.byref(d)),
           "ckks_host_device_pointer")
    return d.value


def pull(dst, src, nbytes: int | None = None, blocks: int = 0, stream=None):
    """Copy src -> dst (device tensors, or a pinned host tensor on either side)
    with the GPU's own loads and stores (ckks_pull)."""
    import torch
    nbytes = nbytes if nbytes is not None else dst.numel() * dst.element_size()

    def addr(t):
        return host_device_pointer(t) if not t.is_cuda else t.data_ptr()
    if not blocks:
        blocks = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8
    _check(lib().ckks_pull(ctypes.c_void_p(addr(dst)), ctypes.c_void_p(addr(src)), nbytes, blocks,
                           _stream(stream)), "ckks_pull")


PEAK_KINDS = {"shoup": 0, "butterfly": 1, "mac128": 2, "montgomery": 3, "transpose_shfl": 4, "transpose_smem": 5,
              "butterfly_q1": 6, "shoup_q1": 7}


def peak_int(kind: str, q: int, blocks: int, threads: int = 256, iters: int = 4096, reps: int = 5,
             stream=None) -> float:
    """Measured rate (operations per second, best of `reps` CUDA-event timed
    launches after one warm-up) of one integer operation of the hot path on
    this GPU: "shoup", "butterfly", "mac128" or "montgomery" (ckks_peak_int);
    "shoup_q1" / "butterfly_q1" for a modulus q = 1 (mod 2^32)."""
    import torch
    chains = lib().ckks_peak_chains()
    w = [(q - 1 - 977 * i) % q for i in range(chains)]
    wp = [(x << 64) // q for x in w]
    W = (ctypes.c_uint64 * chains)(*w)
    WP = (ctypes.c_uint64 * chains)(*wp)
    out = torch.empty(blocks * threads, dtype=torch.uint64, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib().ckks_peak_int(PEAK_KINDS[kind], q, W, WP, blocks, threads, iters, out.data_ptr(),
                                   _stream(st)), "ckks_peak_int")
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if r and (best is None or ms < best):
            best = ms
    per_thread = 16 if PEAK_KINDS[kind] in (4, 5) else chains
    return blocks * threads * per_thread * iters / (best / 1e3)


def plan_optimize(k: int, criterion: str = "rs_units", level: int = 0, K: int = 0, alpha: int = 0):
    """(partition text, cost) of the cheapest valid tree; host only."""
    buf = ctypes.create_string_buffer(256)
    v = ctypes.c_double()
    crit = {"rs_units": 0, "transforms": 1, "precision": 2}[criterion]
    _check(lib().ckks_plan_optimize(k, crit, level, K, alpha, buf, 256, ctypes.byref(v)), "ckks_plan_optimize")
    return buf.value.decode(), v.value


class EvkSet:
    def __init__(self, ctx: Context, h, keys, t_max: int):
        self.ctx, self._h, self.keys, self.t_max = ctx, h, keys, t_max

    def verify(self, stream=None) -> bool:
        """True if the resident keys still match the checksum taken at creation."""
        rc = lib().ckks_evk_verify(self._h, _stream(stream))
        if rc == -8:
            return False
        _check(rc, "ckks_evk_verify")
        return True

    def close(self):
        if self._h:
            lib().ckks_evk_set_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
