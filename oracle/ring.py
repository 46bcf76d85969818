"""Ring Z_q[x]/(x^N + 1) primitives for the oracle (test infrastructure only).

Residue vectors are numpy uint64 arrays with values in [0, q). Products go
through `prims.c` (exact 128-bit products reduced with `%`); sums and
differences use numpy uint64, exact because every q < 2^62.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_prims.so")


def build_prims(force: bool = False) -> str:
    """Compile prims.c with gcc (OpenMP over rows)."""
    src = os.path.join(_HERE, "prims.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


@lru_cache(maxsize=1)
def _lib():
    lib = ctypes.CDLL(build_prims())
    P = ctypes.POINTER(ctypes.c_uint64)
    S = ctypes.c_size_t
    U = ctypes.c_uint64
    sigs = {
        "or_mulmod": [P, P, P, S, U],
        "or_scalar_mulmod": [P, U, P, S, U],
        "or_dot_const": [P, P, S, P, S, U],
        "or_ntt_definition": [P, P, S, U, U],
        "or_intt_definition": [P, P, S, U, U],
        "or_negacyclic_mul": [P, P, P, S, U],
        "or_ntt": [P, S, U, U],
        "or_intt": [P, S, U, U],
        "or_ntt_rows": [P, S, S, P, P],
        "or_intt_rows": [P, S, S, P, P],
        "or_mulmod_rows": [P, P, P, S, S, P],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None
    lib.or_num_threads.restype = ctypes.c_int
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint64)


def num_threads() -> int:
    return _lib().or_num_threads()


# ---------------------------------------------------------------------------
# scalar number theory
# ---------------------------------------------------------------------------
def inv(a: int, q: int) -> int:
    return pow(a % q, -1, q)


def brv(x: int, bits: int) -> int:
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@lru_cache(maxsize=None)
def psi_of(q: int, N: int) -> int:
    """The NTT root for modulus q and degree N: the smallest primitive 2N-th
    root of unity mod q (requires q = 1 mod 2N)."""
    assert (q - 1) % (2 * N) == 0
    g = 2
    while True:
        r = pow(g, (q - 1) // (2 * N), q)
        if pow(r, N, q) == q - 1:
            break
        g += 1
    r2 = r * r % q
    best, cur = r, r
    for _ in range(N - 1):
        cur = cur * r2 % q
        if cur < best:
            best = cur
    return best


# ---------------------------------------------------------------------------
# vector primitives
# ---------------------------------------------------------------------------
def mulmod(a, b, q: int) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    _lib().or_mulmod(_p(a), _p(b), _p(out), a.size, q)
    return out


def smul(a, c: int, q: int) -> np.ndarray:
    """a * c mod q for a scalar c (any a in uint64)."""
    a = _u64(a)
    out = np.empty_like(a)
    _lib().or_scalar_mulmod(_p(a), c % q, _p(out), a.size, q)
    return out


def dot_const(rows: np.ndarray, consts, q: int) -> np.ndarray:
    """sum_j rows[j] * consts[j] mod q (rows [m][n], any uint64 entries)."""
    rows = _u64(rows)
    c = _u64([int(x) % q for x in consts])
    m, n = rows.shape
    out = np.empty(n, dtype=np.uint64)
    _lib().or_dot_const(_p(rows), _p(c), m, _p(out), n, q)
    return out


def addmod(a, b, q: int) -> np.ndarray:
    return (_u64(a) % np.uint64(q) + _u64(b) % np.uint64(q)) % np.uint64(q)


def submod(a, b, q: int) -> np.ndarray:
    qq = np.uint64(q)
    return (_u64(a) % qq + qq - _u64(b) % qq) % qq


def from_signed(x: np.ndarray, q: int) -> np.ndarray:
    """Residues of small signed integers."""
    return np.mod(np.asarray(x, dtype=np.int64), q).astype(np.uint64) if q < (1 << 63) else None


def ntt_definition(a, q: int) -> np.ndarray:
    a = _u64(a)
    out = np.empty_like(a)
    _lib().or_ntt_definition(_p(a), _p(out), a.size, q, psi_of(q, a.size))
    return out


def intt_definition(A, q: int) -> np.ndarray:
    A = _u64(A)
    out = np.empty_like(A)
    _lib().or_intt_definition(_p(A), _p(out), A.size, q, psi_of(q, A.size))
    return out


def negacyclic_mul(a, b, q: int) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    _lib().or_negacyclic_mul(_p(a), _p(b), _p(out), a.size, q)
    return out


def ntt(a, q: int) -> np.ndarray:
    out = _u64(a).copy()
    _lib().or_ntt(_p(out), out.size, q, psi_of(q, out.size))
    return out


def intt(A, q: int) -> np.ndarray:
    out = _u64(A).copy()
    _lib().or_intt(_p(out), out.size, q, psi_of(q, out.size))
    return out


def ntt_rows(a: np.ndarray, primes) -> np.ndarray:
    """Forward transform of each row a[r] modulo primes[r]."""
    out = _u64(a).copy()
    rows, N = out.shape
    qs = _u64(list(primes))
    psis = _u64([psi_of(int(q), N) for q in primes])
    _lib().or_ntt_rows(_p(out), rows, N, _p(qs), _p(psis))
    return out


def intt_rows(A: np.ndarray, primes) -> np.ndarray:
    out = _u64(A).copy()
    rows, N = out.shape
    qs = _u64(list(primes))
    psis = _u64([psi_of(int(q), N) for q in primes])
    _lib().or_intt_rows(_p(out), rows, N, _p(qs), _p(psis))
    return out


def mulmod_rows(a: np.ndarray, b: np.ndarray, primes) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    rows, N = a.shape
    _lib().or_mulmod_rows(_p(a), _p(b), _p(out), rows, N, _p(_u64(list(primes))))
    return out


def addmod_rows(a, b, primes) -> np.ndarray:
    qs = _u64(list(primes))[:, None]
    return (_u64(a) % qs + _u64(b) % qs) % qs


def submod_rows(a, b, primes) -> np.ndarray:
    qs = _u64(list(primes))[:, None]
    return (_u64(a) % qs + qs - _u64(b) % qs) % qs
