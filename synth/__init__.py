"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by
the CPU oracle.

This module draws random numbers and picks parameters. It holds none of the
multiplication method's arithmetic: no NTT, no basis conversion, no key or
ciphertext formula. Every random value the method consumes (secret, key masks,
errors, messages) is drawn here and passed to both sides as an input.

Workload recipe (RNS-CKKS, Section II of the paper):
  * secret s: i.i.d. uniform ternary coefficients in {-1, 0, 1};
  * key masks a: uniform residues in [0, q) per limb, NTT domain;
  * errors e: rounded normal, sigma = 3.2, clipped to +-19 (6 sigma);
  * encryption v: ternary with exactly N/2 non-zero coefficients;
  * messages: N/2 complex slots uniform in the unit disk,
    z = sqrt(U1) * exp(2 pi i U2);
  * ciphertexts for throughput runs: uniform residues in [0, q), which is the
    distribution of RLWE ciphertext components.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x260115401
SIGMA = 3.2
ERR_CLIP = 19  # ceil(6 * sigma)


def rng(config: int, index: int = 0, stream: int = 0) -> np.random.Generator:
    """PCG64 generator seeded from (workload id, request index, stream)."""
    seed = SEED_BASE ^ (config << 32) ^ index ^ (stream << 48)
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# prime chain (parameter choice, not part of the method)
# ----------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


NTT_CONGRUENCE = 1 << 17  # q = 1 mod 2^17 serves every N <= 2^16
# q = 1 mod 2^32 (q = h 2^32 + 1): still NTT-friendly for every N <= 2^31, and
# the modular products of the GPU kernels take a cheaper form for it. Every
# parameter set below takes congruence=Q1_CONGRUENCE to use such primes; the
# default is the 2^17 chain.
Q1_CONGRUENCE = 1 << 32


def prime_chain(bits: int, count: int, exclude=(), congruence: int = NTT_CONGRUENCE) -> list[int]:
    """The `count` largest primes below 2^bits with q = 1 (mod congruence),
    descending (congruence a power of two >= 2N)."""
    out = []
    excl = set(exclude)
    c = ((1 << bits) - 1) // congruence * congruence + 1
    if c >= (1 << bits):
        c -= congruence
    while len(out) < count:
        if c < (1 << (bits - 1)):
            raise ValueError("ran out of primes")
        if c not in excl and is_prime(c):
            out.append(c)
        c -= congruence
    return out


@dataclass(frozen=True)
class Params:
    """RNS-CKKS parameters: ring degree N = 2^log_n, Q = prod q, P = prod p."""
    log_n: int
    q: tuple
    p: tuple
    dnum: int

    @property
    def N(self) -> int:
        return 1 << self.log_n

    @property
    def L(self) -> int:
        return len(self.q)

    @property
    def K(self) -> int:
        return len(self.p)

    @property
    def alpha(self) -> int:
        return -(-self.L // self.dnum)


def make_params(log_n: int, q_bits, k_special: int, dnum: int, p_bits: int = 60,
                congruence: int = NTT_CONGRUENCE) -> Params:
    """q_bits: list of bit sizes, one per Q prime (q_0 first). Primes of the same
    size are taken in descending order; special primes are the next primes of
    p_bits bits not already used; every prime is 1 (mod congruence)."""
    used: list[int] = []
    q = []
    for b in q_bits:
        nxt = prime_chain(b, 1, exclude=used, congruence=congruence)[0]
        q.append(nxt)
        used.append(nxt)
    p = prime_chain(p_bits, k_special, exclude=used, congruence=congruence)
    return Params(log_n, tuple(q), tuple(p), dnum)


# The five workloads (sizes from the paper's 3-input and k-input settings).
def params_small(log_n=10, dnum=1, congruence=NTT_CONGRUENCE):
    """4 x 50-bit Q primes, one 60-bit special prime."""
    return make_params(log_n, [50] * 4, 1, dnum, congruence=congruence)


def params_mid(log_n=14, congruence=NTT_CONGRUENCE):
    """12 Q primes (q_0 60-bit, q_1..q_11 45-bit), 4 x 60-bit special, dnum 3."""
    return make_params(log_n, [60] + [45] * 11, 4, 3, congruence=congruence)


def params_large(log_n=16, L=24, K=8, dnum=3, congruence=NTT_CONGRUENCE):
    """24 x 50-bit Q primes, 8 x 60-bit special primes, dnum 3."""
    return make_params(log_n, [50] * L, K, dnum, congruence=congruence)


# ----------------------------------------------------------------------------
# random draws
# ----------------------------------------------------------------------------
def ternary_secret(g: np.random.Generator, N: int) -> np.ndarray:
    return g.integers(-1, 2, size=N, dtype=np.int64)


def secret(g: np.random.Generator, N: int, h: int | None = None) -> np.ndarray:
    """The secret: uniform ternary (h None), or ternary of Hamming weight h."""
    return ternary_secret(g, N) if not h else ternary_weight(g, N, h)


def ternary_weight(g: np.random.Generator, N: int, h: int) -> np.ndarray:
    v = np.zeros(N, dtype=np.int64)
    idx = g.choice(N, size=h, replace=False)
    v[idx] = g.choice(np.array([-1, 1], dtype=np.int64), size=h)
    return v


def gaussian(g: np.random.Generator, N: int, sigma: float = SIGMA) -> np.ndarray:
    e = np.rint(g.normal(0.0, sigma, size=N)).astype(np.int64)
    return np.clip(e, -ERR_CLIP, ERR_CLIP)


def uniform_residues(g: np.random.Generator, primes, N: int) -> np.ndarray:
    """[len(primes)][N] uint64 residues, uniform in [0, q_j) per row."""
    out = np.empty((len(primes), N), dtype=np.uint64)
    for j, q in enumerate(primes):
        out[j] = g.integers(0, q, size=N, dtype=np.uint64)
    return out


def unit_disk_slots(g: np.random.Generator, n_slots: int) -> np.ndarray:
    r = np.sqrt(g.random(n_slots))
    th = 2.0 * math.pi * g.random(n_slots)
    return r * np.exp(1j * th)


@dataclass
class KeyMaterial:
    """Random inputs of evaluation-key generation for t = 2..t_max.

    a[t-2][beta]: [L+K][N] uniform residues (Q limbs first, then P limbs), NTT domain.
    e[t-2][beta]: [N] small error coefficients (coefficient domain, int64)."""
    s: np.ndarray
    a: list = field(default_factory=list)
    e: list = field(default_factory=list)


def key_material(params: Params, t_max: int, config: int, seed_index: int = 0) -> KeyMaterial:
    g = rng(config, seed_index, stream=1)
    s = ternary_secret(g, params.N)
    km = KeyMaterial(s=s)
    primes = list(params.q) + list(params.p)
    for t in range(2, t_max + 1):
        km.a.append([uniform_residues(g, primes, params.N) for _ in range(params.dnum)])
        km.e.append([gaussian(g, params.N) for _ in range(params.dnum)])
    return km


def uniform_tuple(params: Params, n_polys: int, level: int, config: int, index: int) -> np.ndarray:
    """[n_polys][level][N] uniform residues (NTT domain) for throughput runs."""
    g = rng(config, index, stream=2)
    return np.stack([uniform_residues(g, params.q[:level], params.N) for _ in range(n_polys)])


@dataclass
class EncryptionDraw:
    z: np.ndarray      # N/2 complex message slots
    v: np.ndarray      # ternary, weight N/2
    e0: np.ndarray
    e1: np.ndarray


def encryption_draw(params: Params, config: int, index: int) -> EncryptionDraw:
    g = rng(config, index, stream=3)
    N = params.N
    return EncryptionDraw(z=unit_disk_slots(g, N // 2), v=ternary_weight(g, N, N // 2),
                          e0=gaussian(g, N), e1=gaussian(g, N))


def public_key_draw(params: Params, config: int):
    """(a, e) for the public key: a uniform on every Q limb (NTT domain)."""
    g = rng(config, 0, stream=4)
    return uniform_residues(g, params.q, params.N), gaussian(g, params.N)


# ----------------------------------------------------------------------------
# device-side draws for large throughput runs (same distributions)
# ----------------------------------------------------------------------------
def galois_key_draw(params: Params, config: int, g: int):
    """Random inputs of the Galois key of g: a [dnum] x [L+K][N] uniform
    residues (NTT domain), e [dnum] x [N] small errors."""
    gen = rng(config, g, stream=5)
    primes = list(params.q) + list(params.p)
    a = [uniform_residues(gen, primes, params.N) for _ in range(params.dnum)]
    e = [gaussian(gen, params.N) for _ in range(params.dnum)]
    return a, e


def uniform_residues_torch(primes, shape_prefix, N: int, seed: int, device):
    """Tensor [*shape_prefix][len(primes)][N] of uniform residues, limb j in
    [0, primes[j]), drawn on `device` with a seeded torch generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed & 0x7FFFFFFFFFFFFFFF)
    out = torch.empty((*shape_prefix, len(primes), N), dtype=torch.int64, device=device)
    for j, q in enumerate(primes):
        out[..., j, :] = torch.randint(0, int(q), (*shape_prefix, N), generator=g, dtype=torch.int64, device=device)
    return out.view(torch.uint64)
