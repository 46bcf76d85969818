"""Loading libckks_mulk.so and declaring the C ABI of include/ckks_mulk.h."""
from __future__ import annotations

import ctypes
import os
from functools import lru_cache

_HERE = os.path.dirname(os.path.abspath(__file__))

ERRORS = {0: "CKKS_OK", -1: "CKKS_EINVAL", -2: "CKKS_ELEVEL", -3: "CKKS_EKEY", -4: "CKKS_ENOMEM",
          -5: "CKKS_ECUDA", -6: "CKKS_ETIMEOUT", -7: "CKKS_EBUSY", -8: "CKKS_ECHECK"}


class CkksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


def library_path() -> str:
    return os.environ.get("CKKS_MULK_LIB", os.path.join(_HERE, "libckks_mulk.so"))


V, P, I, U32, SZ, D = (ctypes.c_void_p, ctypes.POINTER, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t,
                       ctypes.c_double)

# name -> argument types (return type int unless listed in _VOID / _STR)
SIGNATURES = {
    "ckks_context_create": [V, I, V],
    "ckks_context_destroy": [V],
    "ckks_keygen_workspace_size": [V, V],
    "ckks_keygen_evk": [V, U32, V, V, V, V, V, SZ, V],
    "ckks_evk_set_create": [V, U32, V, V, V],
    "ckks_galois_element": [V, I, V],
    "ckks_automorphism": [V, V, U32, V, V],
    "ckks_keygen_galois": [V, U32, V, V, V, V, V, SZ, V],
    "ckks_rotate_workspace_size": [V, U32, U32, V],
    "ckks_rotate": [V, V, U32, V, V, V, SZ, V],
    "ckks_rotate_batch": [V, V, U32, U32, V, V, V, SZ, V],
    "ckks_evk_verify": [V, V],
    "ckks_rescale": [V, V, V, V, SZ, V],
    "ckks_requests_workspace_size": [V, V, U32, V],
    "ckks_mul_k_requests": [V, V, U32, V, V, SZ, V],
    "ckks_check_residues": [V, V, V, V],
    "ckks_encrypt_workspace_size": [V, V],
    "ckks_encrypt_batch_workspace_size": [V, U32, U32, V],
    "ckks_encrypt_batch": [V, V, V, V, V, U32, V, U32, V, V, SZ, V],
    "ckks_decrypt_batch_workspace_size": [V, U32, V],
    "ckks_decrypt_batch": [V, V, U32, V, V, V, SZ, V],
    "ckks_embed_workspace_size": [V, U32, V],
    "ckks_encode": [V, V, U32, D, V, V, SZ, V],
    "ckks_decode": [V, V, U32, D, V, V, SZ, V],
    "ckks_public_key": [V, V, V, V, V, V, SZ, V],
    "ckks_encrypt": [V, V, V, V, V, V, U32, V, V, SZ, V],
    "ckks_decrypt": [V, V, V, V, V, SZ, V],
    "ckks_evk_set_destroy": [V],
    "ckks_plan_create": [V, U32, ctypes.c_char_p, V],
    "ckks_plan_destroy": [V],
    "ckks_plan_describe": [V, V, V, V],
    "ckks_plan_optimize": [U32, I, U32, U32, U32, ctypes.c_char_p, SZ, V],
    "ckks_plan_cost": [V, I, U32, U32, U32, V],
    "ckks_workspace_size": [V, V, U32, U32, V],
    "ckks_mul_k": [V, V, U32, V, V, V, V, SZ, V],
    "ckks_mul_k_batch": [V, V, U32, U32, V, V, V, V, SZ, V],
    "ckks_mul2_workspace_size": [V, U32, U32, V],
    "ckks_mul2": [V, V, V, V, V, V, SZ, V],
    "ckks_mul2_batch": [V, V, V, U32, V, V, V, SZ, V],
    "ckks_tensor": [V, V, U32, V, V],
    "ckks_relin_workspace_size": [V, U32, U32, V],
    "ckks_relin": [V, V, V, U32, V, V, SZ, V],
    "ckks_rescale_workspace_size": [V, U32, U32, U32, V],
    "ckks_rescale_multi": [V, V, U32, V, V, SZ, V],
    "ckks_rescale_noalloc_capacity": [],
    "ckks_rescale_multi_noalloc": [V, V, U32, V, V],
    "ckks_ntt": [V, V, V, V],
    "ckks_intt": [V, V, V, V],
    "ckks_counters": [V, V, I],
    "ckks_check": [V],
    "ckks_profile_enable": [V, I],
    "ckks_profile_read": [V, V, U32, V],
    "ckks_tune_set": [V, ctypes.c_char_p, I],
    "ckks_tune_get": [V, ctypes.c_char_p, V],
    "ckks_strerror": [I],
    "ckks_peak_chains": [],
    "ckks_host_device_pointer": [V, V],
    "ckks_pull": [V, V, SZ, I, V],
    "ckks_wave_create": [V, V, U32, V, V],
    "ckks_wave_workspace_size": [V, V, V],
    "ckks_wave_run": [V, V, SZ, V, SZ, V],
    "ckks_wave_describe": [V, V, V],
    "ckks_wave_destroy": [V],
    "ckks_peak_int": [I, ctypes.c_uint64, V, V, I, I, I, V, V],
}
_VOID = {"ckks_context_destroy", "ckks_evk_set_destroy", "ckks_plan_destroy", "ckks_wave_destroy"}
_STR = {"ckks_strerror"}
_SIZE = {"ckks_rescale_noalloc_capacity"}


@lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libckks_mulk.so not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2601_15401_gb300.build")
    L = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = None if name in _VOID else (ctypes.c_char_p if name in _STR else
                                                (ctypes.c_size_t if name in _SIZE else ctypes.c_int))
    return L
