"""Python binding of libwg (include/wg.h): ctypes argument marshalling only.

Every step of the fixpoint runs in the CUDA library; this module converts
arguments, raises on error codes, and (optionally) hands PyTorch's caching
allocator and a PyTorch stream to the library.  There is no fallback: if
libwg.so is missing the import of the library fails with instructions.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, byref, c_char, c_double, c_int, c_int32,
                    c_size_t, c_uint32, c_uint64, c_void_p)

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwg.so")

WG_OK = 0
WG_E_INVAL, WG_E_NOMEM, WG_E_BUDGET, WG_E_CAPACITY = -1, -2, -3, -4
WG_E_NOT_READY, WG_E_ITER_CAP, WG_E_DEVICE_TIMEOUT, WG_E_CUDA = -5, -6, -7, -8
WG_TC, WG_SG = 0, 1
WG_LOOP_DEVICE, WG_LOOP_HOST, WG_LOOP_HOST_STAGED = 0, 1, 2
WG_FLAG_SEPARATE_STAGES = 1
WG_FLAG_FULL_WIDTH = 2
WG_FLAG_COPY_BACK = 4
WG_FLAG_HASH_JOIN = 8
WG_FLAG_MERGE_EVERY_ITER = 16
WG_FLAG_SIDE_RUN_ALWAYS = 32
WG_PENDING, WG_RUNNING, WG_DONE, WG_FAILED = 0, 1, 2, 3
WG_SORT_SEGMENT16, WG_SORT_SEGMENT8, WG_SORT_PASSES, WG_SORT_SEGMENT_WIDE = 0, 1, 2, 3
ERRORS = {-1: "WG_E_INVAL", -2: "WG_E_NOMEM", -3: "WG_E_BUDGET", -4: "WG_E_CAPACITY",
          -5: "WG_E_NOT_READY", -6: "WG_E_ITER_CAP", -7: "WG_E_DEVICE_TIMEOUT", -8: "WG_E_CUDA"}


class wg_opts(Structure):
    _fields_ = [("max_iters", c_uint32), ("loop", c_uint32), ("profile", c_uint32),
                ("flags", c_uint32), ("reserve_full", c_uint64), ("reserve_cand", c_uint64)]


class wg_status(Structure):
    _fields_ = [("state", c_int32), ("error", c_int32), ("n_tuples", c_uint64),
                ("iterations", c_uint32), ("regrows", c_uint32), ("candidates", c_uint64),
                ("gpu_launches", c_uint64), ("device_ms", c_double)]


class wg_request(Structure):
    _fields_ = [("kind", c_int32), ("reserved0", c_uint32), ("edges", c_uint64), ("opts", wg_opts)]


class wg_tune(Structure):
    _fields_ = [("key_bytes", c_uint32), ("count_tile", c_uint32), ("fuse_tile", c_uint32),
                ("count_cand", c_uint32 * 2), ("fuse_cand", c_uint32 * 2), ("sort_mode", c_uint32),
                ("emit_tile", c_uint32), ("emit_cand", c_uint32 * 2), ("reserved0", c_uint32),
                ("count_ms", c_double * 2), ("fuse_ms", c_double * 2), ("sort_ms", c_double * 4),
                ("emit_ms", c_double * 2)]


class wg_kernel_stat(Structure):
    _fields_ = [("name", c_char * 32), ("launches", c_uint64), ("total_ms", c_double),
                ("bytes", c_double)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)

# name -> (restype, argtypes), exactly the declarations of include/wg.h
SIGNATURES = {
    "wg_init": (c_int, [c_int, c_size_t, ALLOC_FN, FREE_FN, c_void_p, c_void_p, POINTER(c_void_p)]),
    "wg_destroy": (None, [c_void_p]),
    "wg_last_error": (ctypes.c_char_p, []),
    "wg_mem_used": (c_size_t, [c_void_p]),
    "wg_relation_load": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, POINTER(c_uint64)]),
    "wg_relation_load_device": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, POINTER(c_uint64)]),
    "wg_relation_info": (c_int, [c_void_p, c_uint64, POINTER(c_uint64), POINTER(c_uint32),
                                 POINTER(c_uint32)]),
    "wg_relation_free": (None, [c_void_p, c_uint64]),
    "wg_tc": (c_int, [c_void_p, c_uint64, POINTER(wg_opts), POINTER(c_uint64)]),
    "wg_sg": (c_int, [c_void_p, c_uint64, POINTER(wg_opts), POINTER(c_uint64)]),
    "wg_submit": (c_int, [c_void_p, POINTER(wg_request), c_size_t, POINTER(c_uint64)]),
    "wg_serve_step": (c_int, [c_void_p, c_uint32, POINTER(c_size_t)]),
    "wg_poll": (c_int, [c_void_p, c_uint64, POINTER(wg_status)]),
    "wg_take_completed": (c_int, [c_void_p, POINTER(c_uint64), c_size_t, POINTER(c_size_t)]),
    "wg_wait": (c_int, [c_void_p, c_uint64, c_uint64]),
    "wg_result_copy": (c_int, [c_void_p, c_uint64, c_void_p, c_size_t, POINTER(c_size_t)]),
    "wg_result_copy_device": (c_int, [c_void_p, c_uint64, c_void_p, c_size_t, POINTER(c_size_t)]),
    "wg_result_iters": (c_int, [c_void_p, c_uint64, c_void_p, c_size_t, POINTER(c_size_t)]),
    "wg_result_digest": (c_int, [c_void_p, c_uint64, POINTER(c_uint64)]),
    "wg_autotune": (c_int, [c_void_p, c_uint64, c_int, POINTER(wg_tune)]),
    "wg_selftest_wait_timeout": (c_int, [c_void_p]),
    "wg_set_tiles": (c_int, [c_void_p, c_int, c_uint32, c_uint32, c_uint32]),
    "wg_set_sort": (c_int, [c_void_p, c_int, c_uint32]),
    "wg_result_profile": (c_int, [c_void_p, c_uint64, POINTER(wg_kernel_stat), c_size_t,
                                  POINTER(c_size_t)]),
    "wg_query_free": (None, [c_void_p, c_uint64]),
    "wg_sort_keys": (c_int, [c_void_p, c_void_p, c_size_t, c_int, c_uint32]),
    "wg_unique_diff": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_size_t, c_void_p,
                               POINTER(c_size_t), c_int]),
    "wg_merge_disjoint": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_size_t, c_void_p,
                                  c_int]),
    "wg_sort_keys_noalloc": (c_int, [c_void_p, c_size_t, c_int, c_uint32, c_void_p]),
    "wg_triangles": (c_int, [c_void_p, c_uint64, POINTER(c_uint64)]),
}
WG_NOALLOC_MAX_KEYS = 1 << 20

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libwg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_2607_17571_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class WgError(RuntimeError):
    def __init__(self, code, where):
        msg = load_library().wg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, where):
    if rc != WG_OK:
        raise WgError(rc, where)


def _opts(max_iters=0, loop=WG_LOOP_DEVICE, profile=False, reserve_full=0, reserve_cand=0,
          separate_stages=False, full_width=False, copy_back=False, hash_join=False,
          side_run="auto"):
    if side_run not in ("auto", "never", "always"):
        raise ValueError(f"side_run must be 'auto', 'never' or 'always', got {side_run!r}")
    flags = ((WG_FLAG_SEPARATE_STAGES if separate_stages else 0) |
             (WG_FLAG_FULL_WIDTH if full_width else 0) | (WG_FLAG_COPY_BACK if copy_back else 0) |
             (WG_FLAG_HASH_JOIN if hash_join else 0) |
             (WG_FLAG_MERGE_EVERY_ITER if side_run == "never" else 0) |
             (WG_FLAG_SIDE_RUN_ALWAYS if side_run == "always" else 0))
    return wg_opts(max_iters, loop, 1 if profile else 0, flags, reserve_full, reserve_cand)


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def pinned(n: int, dtype=np.uint64) -> np.ndarray:
    """A page-locked host array of n elements (torch's pinned allocator): the
    reusable host side of result copies and of edge uploads."""
    import torch
    t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8, pin_memory=True)
    return t.numpy().view(dtype)  # the array keeps the pinned storage alive


def sort_keys_noalloc(ptr: int, n: int, key_bytes: int, bits: int, stream_ptr=None):
    """wg_sort_keys_noalloc: in-place sort with the library's static scratch
    (no context, no allocation); asynchronous on the given stream."""
    _check(load_library().wg_sort_keys_noalloc(c_void_p(ptr), n, key_bytes, bits,
                                               c_void_p(stream_ptr) if stream_ptr else None),
           "wg_sort_keys_noalloc")


def noalloc_check(stream_ptr=None) -> int:
    """wg_sort_keys_noalloc with n = 0: synchronises the stream and returns
    WG_E_DEVICE_TIMEOUT if an allocation-free sort on this device gave up a
    device wait since the last check (else WG_OK); clears the record."""
    return load_library().wg_sort_keys_noalloc(None, 0, 4, 32,
                                               c_void_p(stream_ptr) if stream_ptr else None)


class Query:
    def __init__(self, ctx, qid):
        self.ctx, self.id = ctx, qid

    def poll(self) -> wg_status:
        st = wg_status()
        _check(self.ctx.lib.wg_poll(self.ctx.h, self.id, byref(st)), "wg_poll")
        return st

    def wait(self, timeout_us: int = 0):
        rc = self.ctx.lib.wg_wait(self.ctx.h, self.id, timeout_us)
        _check(rc, "wg_wait")
        return self.poll()

    def result(self, out: np.ndarray = None) -> np.ndarray:
        """Sorted packed keys (src << 32) | dst, uint64, on the host.

        `out` (optional): a host uint64 array of at least the result size to
        copy into -- e.g. a reusable buffer from `pinned()`, which the copy
        reaches at DMA speed.  Returns the filled prefix."""
        n = c_size_t()
        rc = self.ctx.lib.wg_result_copy(self.ctx.h, self.id, None, 0, byref(n))
        if rc not in (WG_OK, WG_E_CAPACITY):
            _check(rc, "wg_result_copy")
        if out is None:
            out = np.empty(n.value, dtype=np.uint64)
        elif out.dtype != np.uint64 or not out.flags.c_contiguous or out.shape[0] < n.value:
            raise ValueError("out must be a contiguous uint64 array of at least the result size")
        _check(self.ctx.lib.wg_result_copy(self.ctx.h, self.id, out.ctypes.data_as(c_void_p),
                                           out.shape[0], byref(n)), "wg_result_copy")
        return out[: n.value]

    def result_device(self, out_ptr: int, cap: int) -> int:
        n = c_size_t()
        _check(self.ctx.lib.wg_result_copy_device(self.ctx.h, self.id, c_void_p(out_ptr), cap,
                                                  byref(n)), "wg_result_copy_device")
        return n.value

    def digest(self) -> int:
        """wg_result_digest: the device-side digest of the sorted result."""
        d = c_uint64()
        _check(self.ctx.lib.wg_result_digest(self.ctx.h, self.id, byref(d)), "wg_result_digest")
        return int(d.value)

    def delta_sizes(self) -> list:
        n = c_size_t()
        buf = np.zeros(1 << 16, dtype=np.uint64)
        _check(self.ctx.lib.wg_result_iters(self.ctx.h, self.id, buf.ctypes.data_as(c_void_p),
                                            buf.shape[0], byref(n)), "wg_result_iters")
        return buf[: n.value].tolist()

    def profile(self) -> list:
        n = c_size_t()
        arr = (wg_kernel_stat * 64)()
        _check(self.ctx.lib.wg_result_profile(self.ctx.h, self.id, arr, 64, byref(n)),
               "wg_result_profile")
        return [dict(name=arr[i].name.decode(), launches=arr[i].launches,
                     total_ms=arr[i].total_ms, bytes=arr[i].bytes) for i in range(n.value)]

    def free(self):
        if self.id:
            self.ctx.lib.wg_query_free(self.ctx.h, self.id)
            self.id = 0


class Relation:
    def __init__(self, ctx, rid):
        self.ctx, self.id = ctx, rid

    def info(self):
        ne, nv, w = c_uint64(), c_uint32(), c_uint32()
        _check(self.ctx.lib.wg_relation_info(self.ctx.h, self.id, byref(ne), byref(nv), byref(w)),
               "wg_relation_info")
        return dict(n_edges=ne.value, n_vertices=nv.value, field_bits=w.value)

    def free(self):
        if self.id:
            self.ctx.lib.wg_relation_free(self.ctx.h, self.id)
            self.id = 0


class Context:
    """wg_init / wg_destroy.  With torch_memory=True the library allocates
    through PyTorch's caching allocator on a PyTorch stream."""

    def __init__(self, device: int = 0, mem_budget: int = 0, torch_memory: bool = True,
                 stream=None):
        self.lib = load_library()
        self.device = device
        self._keep = []
        alloc, free, sptr = ALLOC_FN(), FREE_FN(), None
        if torch_memory:
            import torch
            self.torch_stream = stream or torch.cuda.Stream(device=device)
            sptr = self.torch_stream.cuda_stream
            if not mem_budget:
                # the library's default is 90% of the free device memory; blocks
                # PyTorch's cache holds unused will serve this context too
                free, _ = torch.cuda.mem_get_info(device)
                cached = torch.cuda.memory_reserved(device) - torch.cuda.memory_allocated(device)
                mem_budget = int(0.9 * (free + max(0, cached)))

            def _alloc(nbytes, stream_, user):
                try:
                    return torch.cuda.caching_allocator_alloc(nbytes, device, stream_ or sptr)
                except RuntimeError:
                    return None

            def _free(ptr, nbytes, stream_, user):
                torch.cuda.caching_allocator_delete(ptr)

            alloc, free = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [alloc, free, _alloc, _free]
        else:
            self.torch_stream = None
            if stream is not None:
                sptr = int(stream)
        h = c_void_p()
        _check(self.lib.wg_init(device, mem_budget, alloc, free, None,
                                c_void_p(sptr) if sptr else None, byref(h)), "wg_init")
        self.h = h

    @property
    def stream_ptr(self):
        return self.torch_stream.cuda_stream if self.torch_stream is not None else None

    def close(self):
        if getattr(self, "h", None):
            self.lib.wg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mem_used(self) -> int:
        return self.lib.wg_mem_used(self.h)

    def load(self, src, dst) -> Relation:
        """wg_relation_load from host arrays."""
        s, d = _u32(src), _u32(dst)
        r = c_uint64()
        _check(self.lib.wg_relation_load(self.h, s.ctypes.data_as(c_void_p),
                                         d.ctypes.data_as(c_void_p), s.shape[0], byref(r)),
               "wg_relation_load")
        return Relation(self, r.value)

    def load_device(self, src_ptr: int, dst_ptr: int, n: int) -> Relation:
        """wg_relation_load_device from device pointers (e.g. tensor.data_ptr())."""
        r = c_uint64()
        _check(self.lib.wg_relation_load_device(self.h, c_void_p(src_ptr), c_void_p(dst_ptr), n,
                                                byref(r)), "wg_relation_load_device")
        return Relation(self, r.value)

    def tc(self, rel: Relation, **opts) -> Query:
        q = c_uint64()
        o = _opts(**opts)
        _check(self.lib.wg_tc(self.h, rel.id, byref(o), byref(q)), "wg_tc")
        return Query(self, q.value)

    def autotune(self, rel: Relation, kind: int = WG_TC) -> dict:
        """wg_autotune: time the compiled tile shapes of the join count, the
        join emit and the fused pass (and the radix-sort modes) on profiled
        fixpoints of `rel` and keep the fastest for engines of its key width."""
        t = wg_tune()
        _check(self.lib.wg_autotune(self.h, rel.id, kind, byref(t)), "wg_autotune")
        return dict(key_bytes=t.key_bytes, count_tile=t.count_tile, fuse_tile=t.fuse_tile,
                    emit_tile=t.emit_tile, sort_mode=t.sort_mode, count_cand=list(t.count_cand),
                    fuse_cand=list(t.fuse_cand), emit_cand=list(t.emit_cand),
                    count_ms=[round(x, 3) for x in t.count_ms],
                    fuse_ms=[round(x, 3) for x in t.fuse_ms],
                    emit_ms=[round(x, 3) for x in t.emit_ms],
                    sort_ms=[round(x, 3) for x in t.sort_ms])

    def selftest_wait_timeout(self) -> int:
        """wg_selftest_wait_timeout: the return code (WG_E_DEVICE_TIMEOUT is
        the expected outcome: the bounded device wait gave up)."""
        return int(self.lib.wg_selftest_wait_timeout(self.h))

    def set_tiles(self, key_bytes: int, count_tile: int = 0, fuse_tile: int = 0,
                  emit_tile: int = 0):
        """wg_set_tiles: tile shapes for engines of this key width (0 = default)."""
        _check(self.lib.wg_set_tiles(self.h, key_bytes, count_tile, fuse_tile, emit_tile),
               "wg_set_tiles")

    def set_sort(self, key_bytes: int, mode: int = WG_SORT_SEGMENT16):
        """wg_set_sort: radix-sort mode of single TC engines of this key width."""
        _check(self.lib.wg_set_sort(self.h, key_bytes, mode), "wg_set_sort")

    def triangles(self, rel: Relation) -> int:
        """wg_triangles: number of tuples of triangle(a,b,c) <- edge(a,b),
        edge(b,c), edge(c,a) over the relation (synchronous)."""
        n = c_uint64()
        _check(self.lib.wg_triangles(self.h, rel.id, byref(n)), "wg_triangles")
        return int(n.value)

    def sg(self, rel: Relation, **opts) -> Query:
        q = c_uint64()
        o = _opts(**opts)
        _check(self.lib.wg_sg(self.h, rel.id, byref(o), byref(q)), "wg_sg")
        return Query(self, q.value)

    def submit(self, reqs) -> list:
        """reqs: iterable of (kind, Relation[, opts dict])."""
        reqs = list(reqs)
        arr = (wg_request * max(1, len(reqs)))()
        for i, r in enumerate(reqs):
            kind, rel = r[0], r[1]
            arr[i].kind = kind
            arr[i].edges = rel.id
            arr[i].opts = _opts(**(r[2] if len(r) > 2 else {}))
        ids = (c_uint64 * max(1, len(reqs)))()
        _check(self.lib.wg_submit(self.h, arr, len(reqs), ids), "wg_submit")
        return [Query(self, ids[i]) for i in range(len(reqs))]

    def take_completed(self, cap: int = 65536) -> list:
        """Ids of batch queries finished since the previous call."""
        ids = (c_uint64 * cap)()
        n = c_size_t()
        _check(self.lib.wg_take_completed(self.h, ids, cap, byref(n)), "wg_take_completed")
        return [ids[i] for i in range(n.value)]

    def serve_step(self, iters: int = 0) -> int:
        n = c_size_t()
        _check(self.lib.wg_serve_step(self.h, iters, byref(n)), "wg_serve_step")
        return n.value

    # sorted-array primitives on device buffers
    def sort_keys(self, ptr: int, n: int, key_bytes: int, bits: int):
        _check(self.lib.wg_sort_keys(self.h, c_void_p(ptr), n, key_bytes, bits), "wg_sort_keys")

    def unique_diff(self, cand: int, n: int, full: int, nf: int, out: int, key_bytes: int) -> int:
        m = c_size_t()
        _check(self.lib.wg_unique_diff(self.h, c_void_p(cand), n, c_void_p(full) if nf else None,
                                       nf, c_void_p(out), byref(m), key_bytes), "wg_unique_diff")
        return m.value

    def merge_disjoint(self, a: int, na: int, b: int, nb: int, out: int, key_bytes: int):
        _check(self.lib.wg_merge_disjoint(self.h, c_void_p(a), na, c_void_p(b), nb, c_void_p(out),
                                          key_bytes), "wg_merge_disjoint")
