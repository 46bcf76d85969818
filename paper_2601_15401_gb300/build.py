"""Build libckks_mulk.so (sm_103a) in-tree with nvcc; no torch extension
machinery and no cmake. Translation units compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.environ.get("CKKS_MULK_LIB", os.path.join(HERE, "libckks_mulk.so"))
SOURCES = ["ntt.cu", "ntt_uf.cu", "ntt_ui.cu", "ntt_tf.cu", "ntt_ti.cu", "ntt_uf1.cu", "ntt_ui1.cu", "ntt_tf1.cu",
           "ntt_ti1.cu", "rns.cu", "tensor_fixed.cu", "context.cu", "engine.cu", "capi.cu", "plan.cpp", "noalloc.cu", "encrypt.cu", "galois.cu", "embed.cu", "check.cu", "peak.cu", "wave.cu", "xfer.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _compile(src: str, extra: list[str]) -> str:
    tag = os.path.basename(LIB).replace(".so", "")
    obj = os.path.join(BUILD, f"{tag}_{os.path.basename(src)}.o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-I", os.path.join(HERE, "..", "include"), "-c",
           os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "ckks_mulk.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def source_hash() -> str:
    """Hash of the library's sources (every file under csrc/ and the public
    header): a tuning choice cached for one build is reused only while the
    kernels it was measured and verified on are unchanged."""
    import hashlib
    h = hashlib.sha256()
    files = sorted(os.listdir(CSRC))
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(HERE, "..", "include", "ckks_mulk.h"), "rb").read())
    return h.hexdigest()[:16]


def build(force: bool = False, extra: list[str] | None = None, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or []) + os.environ.get("CKKS_NVCC_FLAGS", "").split()
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
