"""ctypes binding and build step of the C++ oracle (test infrastructure only).

Parity unpinned: none -- every oracle function is pinned by the tests in
tests/test_oracle_pins.py (worked example, closed forms, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wg_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libwg_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host g++ (seconds)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64pp = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))
        szp = ctypes.POINTER(ctypes.c_size_t)
        for name in ("oracle_tc", "oracle_sg"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [u32p, u32p, ctypes.c_size_t, ctypes.c_uint32, u64pp, szp, u64pp, szp,
                          u32p]
        lib.oracle_tc_rows.restype = ctypes.c_int
        lib.oracle_tc_rows.argtypes = [u32p, u32p, ctypes.c_size_t, u32p, ctypes.c_size_t,
                                       ctypes.c_int, u64pp, szp,
                                       ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, u32p]
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_tc_reach.restype = ctypes.c_int
        lib.oracle_tc_reach.argtypes = [u32p, u32p, ctypes.c_size_t, ctypes.c_int, u64p, u32p,
                                        u64p, ctypes.c_size_t, szp, u64p]
        lib.oracle_triangles.restype = ctypes.c_uint64
        lib.oracle_triangles.argtypes = [u32p, u32p, ctypes.c_size_t, ctypes.c_int]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class OracleResult:
    keys: np.ndarray        # uint64, sorted, (src << 32) | dst
    log: np.ndarray         # uint64: |Delta^0| .. |Delta^iters|
    iters: int
    status: int             # 0 fixpoint reached, 1 iteration cap

    def pairs(self):
        return (self.keys >> np.uint64(32)).astype(np.uint32), \
               (self.keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _run(fn, src, dst, max_iters):
    lib = _load()
    src, dst = _u32(src), _u32(dst)
    assert src.shape == dst.shape
    kp = ctypes.POINTER(ctypes.c_uint64)()
    lp = ctypes.POINTER(ctypes.c_uint64)()
    nk, nl = ctypes.c_size_t(), ctypes.c_size_t()
    it = ctypes.c_uint32()
    st = getattr(lib, fn)(_ptr32(src), _ptr32(dst), src.shape[0], max_iters,
                          ctypes.byref(kp), ctypes.byref(nk), ctypes.byref(lp),
                          ctypes.byref(nl), ctypes.byref(it))
    if st < 0:
        raise MemoryError(fn)
    keys = np.ctypeslib.as_array(kp, shape=(nk.value + 1,))[: nk.value].copy()
    log = np.ctypeslib.as_array(lp, shape=(nl.value + 1,))[: nl.value].copy()
    lib.oracle_free(kp)
    lib.oracle_free(lp)
    return OracleResult(keys, log, int(it.value), int(st))


def oracle_tc(src, dst, max_iters: int = 0xFFFFFFFF) -> OracleResult:
    """Transitive closure, semi-naive (Sec. Background, steps 1-5)."""
    return _run("oracle_tc", src, dst, max_iters)


def oracle_sg(src, dst, max_iters: int = 0xFFFFFFFF) -> OracleResult:
    """Same-generation, semi-naive (Sec. Generalization; base rule x != y)."""
    return _run("oracle_sg", src, dst, max_iters)


def oracle_tc_rows(src, dst, sources, n_threads: int = 1, log_cap: int = 4096):
    """Rows T(x, .) for each x in ``sources`` (row-by-row semi-naive loop).

    Returns (keys, row_len, log_sum, max_row_iters)."""
    lib = _load()
    src, dst, sources = _u32(src), _u32(dst), _u32(sources)
    kp = ctypes.POINTER(ctypes.c_uint64)()
    nk = ctypes.c_size_t()
    row_len = np.zeros(sources.shape[0] + 1, dtype=np.uint64)
    log_sum = np.zeros(log_cap, dtype=np.uint64)
    mx = ctypes.c_uint32()
    st = lib.oracle_tc_rows(_ptr32(src), _ptr32(dst), src.shape[0], _ptr32(sources),
                            sources.shape[0], int(n_threads), ctypes.byref(kp),
                            ctypes.byref(nk),
                            row_len.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            log_sum.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), log_cap,
                            ctypes.byref(mx))
    if st < 0:
        raise MemoryError("oracle_tc_rows")
    keys = np.ctypeslib.as_array(kp, shape=(nk.value + 1,))[: nk.value].copy()
    lib.oracle_free(kp)
    return keys, row_len[: sources.shape[0]], log_sum, int(mx.value)


def oracle_triangles(src, dst, n_threads: int = 1) -> int:
    """Number of tuples of triangle(a,b,c) <- edge(a,b), edge(b,c), edge(c,a)
    (Sec. Generalization, "Triangle Counting"); edges are a set."""
    lib = _load()
    src, dst = _u32(src), _u32(dst)
    assert src.shape == dst.shape
    return int(lib.oracle_triangles(_ptr32(src), _ptr32(dst), src.shape[0], int(n_threads)))


def oracle_tc_reach(src, dst, n_threads: int = 1, log_cap: int = 4096):
    """TC by reachability (breadth-first search from every source): closure
    size, iterations, the Delta-size log and the digest of the sorted closure
    (see digest_keys), without materialising the closure."""
    lib = _load()
    s, d = _u32(src), _u32(dst)
    n = ctypes.c_uint64(0)
    it = ctypes.c_uint32(0)
    log = np.zeros(log_cap, dtype=np.uint64)
    nl = ctypes.c_size_t(0)
    dg = ctypes.c_uint64(0)
    rc = lib.oracle_tc_reach(_ptr32(s), _ptr32(d), s.shape[0], n_threads, ctypes.byref(n),
                             ctypes.byref(it), log.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                             log_cap, ctypes.byref(nl), ctypes.byref(dg))
    if rc != 0:
        raise RuntimeError(f"oracle_tc_reach failed: {rc}")
    return int(n.value), int(it.value), log[: min(nl.value, log_cap)].copy(), int(dg.value)


_PHI = np.uint64(0x9E3779B97F4A7C15)


def digest_keys(keys) -> int:
    """Digest of a sorted packed-key array: sum over i of mix64(key_i + i * phi)
    mod 2^64, mix64 = the SplitMix64 output function (Steele, Lea, Flood 2014)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    tot = 0
    with np.errstate(over="ignore"):
        for a in range(0, k.shape[0], 1 << 24):
            z = k[a:a + (1 << 24)] + np.arange(a, a + min(1 << 24, k.shape[0] - a), dtype=np.uint64) * _PHI
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
            tot = (tot + int(z.sum(dtype=np.uint64))) & 0xFFFFFFFFFFFFFFFF
    return tot
