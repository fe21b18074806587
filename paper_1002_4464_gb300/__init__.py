"""Python binding of the GB300 GPU Bucket Sort library (``include/bsort.h``).

Argument marshalling only: every step of the sort runs in the CUDA kernels
of ``libbsort.so``; there is no Python or CPU fallback.  The functions below
carry the C names and signatures; ``BucketSorter`` is a convenience wrapper
that takes torch tensors and lets PyTorch own the device workspace.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "BSORT_OK", "BSORT_EINVAL", "BSORT_ENOMEM", "BSORT_ECUDA", "BSORT_ETIMEOUT",
    "BSORT_EBUSY", "BSORT_ENOTREADY", "BSORT_EUNSUPPORTED", "BSORT_EINTERNAL",
    "BSORT_U32", "BSORT_F32", "BSORT_U64", "BSORT_FLAG_TIMING", "BSORT_FLAG_LOW_MEMORY",
    "BSORT_FLAG_GRAPHS", "BSORT_FLAG_MERGE_SORT", "BSORT_FLAG_TEST_STALL_SCAN",
    "BSORT_FLAG_PLAN_MODEL", "BSORT_BUCKETS_AUTO", "BSORT_FLAG_TEST_TWO_LEVEL",
    "bsort_config", "bsort_plan_info", "BsortError", "load_library",
    "bsort_create", "bsort_destroy", "bsort_plan", "bsort_sort_keys",
    "bsort_sort_pairs", "bsort_sort_keys_host", "bsort_sync",
    "bsort_get_intermediate", "bsort_kernel_times", "bsort_kernel_name",
    "bsort_last_error", "bsort_status_string", "bsort_sort_keys_noalloc", "BucketSorter",
    "bsort_batch_info", "bsort_sort_batch", "bsort_plan_batch", "EXPORTED_SYMBOLS",
    "bsort_request", "bsort_result", "bsort_serve_info", "bsort_submit", "bsort_poll",
    "bsort_serve_stats", "bsort_clock_ns", "bsort_poll_any", "SortServer",
]

BSORT_OK, BSORT_EINVAL, BSORT_ENOMEM, BSORT_ECUDA, BSORT_ETIMEOUT = 0, 1, 2, 3, 4
BSORT_EBUSY, BSORT_ENOTREADY, BSORT_EUNSUPPORTED, BSORT_EINTERNAL = 5, 6, 7, 8
BSORT_U32, BSORT_F32, BSORT_U64 = 0, 1, 2
BSORT_FLAG_TIMING = 0x1
BSORT_FLAG_LOW_MEMORY = 0x2
BSORT_FLAG_GRAPHS = 0x4
BSORT_FLAG_MERGE_SORT = 0x8
BSORT_FLAG_TEST_STALL_SCAN = 0x10
BSORT_FLAG_PLAN_MODEL = 0x20
BSORT_FLAG_TEST_TWO_LEVEL = 0x40
BSORT_BUCKETS_AUTO = 0xFFFFFFFF
(BSORT_IM_TILES, BSORT_IM_SAMPLES, BSORT_IM_SPLITTERS, BSORT_IM_COUNTS,
 BSORT_IM_OFFSETS, BSORT_IM_RELOCATED) = range(6)

# every function include/bsort.h declares
EXPORTED_SYMBOLS = (
    "bsort_create", "bsort_destroy", "bsort_plan", "bsort_sort_keys",
    "bsort_sort_pairs", "bsort_sort_keys_host", "bsort_sync",
    "bsort_get_intermediate", "bsort_kernel_times", "bsort_kernel_name",
    "bsort_last_error", "bsort_status_string", "bsort_sort_keys_noalloc",
    "bsort_sort_batch", "bsort_plan_batch", "bsort_submit", "bsort_poll", "bsort_serve_stats",
    "bsort_clock_ns", "bsort_poll_any",
)


class bsort_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("tile", ctypes.c_uint32), ("samples", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("buckets", ctypes.c_uint32),
                ("batch_direct_max", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
                ("serve_budget_bytes", ctypes.c_uint64)]


class bsort_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("n_padded", ctypes.c_uint64),
                ("t", ctypes.c_uint32), ("s", ctypes.c_uint32), ("m", ctypes.c_uint32),
                ("w", ctypes.c_uint32), ("bucket_bound", ctypes.c_uint64),
                ("tile_ctas", ctypes.c_uint32), ("unit_ctas", ctypes.c_uint32),
                ("unit_capacity", ctypes.c_uint64), ("single_tile", ctypes.c_uint32),
                ("num_kernels", ctypes.c_uint32), ("workspace_bytes", ctypes.c_uint64),
                ("b", ctypes.c_uint32), ("unit_small", ctypes.c_uint32),
                ("levels", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class bsort_batch_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("num_segs", ctypes.c_uint32),
                ("direct_segs", ctypes.c_uint32), ("sampled_segs", ctypes.c_uint32),
                ("large_segs", ctypes.c_uint32), ("sublists", ctypes.c_uint32),
                ("buckets", ctypes.c_uint32), ("num_kernels", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32), ("workspace_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad_"}


class bsort_request(ctypes.Structure):
    _fields_ = [("key_type", ctypes.c_int), ("pad_", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("h_keys_in", ctypes.c_void_p), ("h_keys_out", ctypes.c_void_p)]


class bsort_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_uint32),
                ("submit_ns", ctypes.c_uint64), ("start_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64)]


class bsort_serve_info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "arena_bytes", "workspace_bytes", "arena_used_bytes", "arena_peak_bytes", "queued",
        "completed", "batches", "max_batch", "large_jobs", "worker_busy_ns")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class BsortError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (bsort_status_string(status), msg))
        self.status = status


_lib = None


def load_library(rebuild: bool = False):
    """Load ``libbsort.so`` (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None and not rebuild:
        return _lib
    path = _build.build(force=rebuild) if (rebuild or not os.path.exists(_build.LIB)) else _build.LIB
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    vp = ctypes.c_void_p
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "bsort_create": (i32, [ctypes.POINTER(bsort_config), ctypes.POINTER(H)]),
        "bsort_destroy": (i32, [H]),
        "bsort_plan": (i32, [H, i32, u32, u64, ctypes.POINTER(bsort_plan_info)]),
        "bsort_sort_keys": (i32, [H, i32, vp, vp, u64, vp]),
        "bsort_sort_pairs": (i32, [H, i32, vp, vp, vp, vp, u32, u64, vp]),
        "bsort_sort_keys_host": (i32, [H, i32, vp, vp, u64, vp]),
        "bsort_sync": (i32, [H, vp]),
        "bsort_get_intermediate": (i32, [H, i32, vp, u64]),
        "bsort_kernel_times": (i32, [H, ctypes.POINTER(ctypes.c_float), u32,
                                     ctypes.POINTER(u32), ctypes.POINTER(u32)]),
        "bsort_kernel_name": (ctypes.c_char_p, [H, u32]),
        "bsort_last_error": (ctypes.c_char_p, [H]),
        "bsort_status_string": (ctypes.c_char_p, [i32]),
        "bsort_sort_keys_noalloc": (i32, [i32, vp, vp, u64, vp, i32]),
        "bsort_sort_batch": (i32, [H, i32, vp, vp, ctypes.POINTER(u64), u32, vp]),
        "bsort_plan_batch": (i32, [H, i32, ctypes.POINTER(u64), u32,
                                   ctypes.POINTER(bsort_batch_info)]),
        "bsort_submit": (i32, [H, ctypes.POINTER(bsort_request), ctypes.POINTER(u64)]),
        "bsort_poll": (i32, [H, u64, ctypes.POINTER(bsort_result)]),
        "bsort_serve_stats": (i32, [H, ctypes.POINTER(bsort_serve_info)]),
        "bsort_poll_any": (i32, [H, ctypes.POINTER(u64), ctypes.POINTER(bsort_result), u32,
                                 ctypes.POINTER(u32)]),
        "bsort_clock_ns": (u64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------ C-named calls

def bsort_status_string(st):
    return load_library().bsort_status_string(int(st)).decode()


def bsort_last_error(h):
    return load_library().bsort_last_error(h).decode()


def _check(h, st):
    if st != BSORT_OK:
        raise BsortError(st, bsort_last_error(h) if h else "")
    return st


def bsort_create(cfg: bsort_config = None):
    h = ctypes.c_void_p()
    st = load_library().bsort_create(ctypes.byref(cfg) if cfg is not None else None,
                                     ctypes.byref(h))
    if st != BSORT_OK:
        raise BsortError(st, "bsort_create failed")
    return h


def bsort_destroy(h):
    return _check(None, load_library().bsort_destroy(h))


def bsort_plan(h, key_type, val_bytes, n):
    info = bsort_plan_info()
    _check(h, load_library().bsort_plan(h, key_type, val_bytes, n, ctypes.byref(info)))
    return info


def bsort_sort_keys(h, key_type, d_keys_in, d_keys_out, n, stream):
    return _check(h, load_library().bsort_sort_keys(h, key_type, d_keys_in, d_keys_out, n,
                                                    stream))


def bsort_sort_pairs(h, key_type, d_keys_in, d_vals_in, d_keys_out, d_vals_out, val_bytes,
                     n, stream):
    return _check(h, load_library().bsort_sort_pairs(h, key_type, d_keys_in, d_vals_in,
                                                     d_keys_out, d_vals_out, val_bytes, n,
                                                     stream))


def bsort_sort_keys_host(h, key_type, h_keys_in, h_keys_out, n, stream):
    return _check(h, load_library().bsort_sort_keys_host(h, key_type, h_keys_in, h_keys_out,
                                                         n, stream))


def bsort_sync(h, stream):
    return _check(h, load_library().bsort_sync(h, stream))


def bsort_get_intermediate(h, which, h_dst, nbytes):
    return _check(h, load_library().bsort_get_intermediate(h, which, h_dst, nbytes))


def bsort_kernel_times(h, count=64):
    """[(kernel name, summed ms)], number of calls summed."""
    arr = (ctypes.c_float * count)()
    written = ctypes.c_uint32()
    calls = ctypes.c_uint32()
    _check(h, load_library().bsort_kernel_times(h, arr, count, ctypes.byref(written),
                                                ctypes.byref(calls)))
    return [(bsort_kernel_name(h, i), arr[i]) for i in range(written.value)], calls.value


def bsort_sort_keys_noalloc(key_type, d_keys_in, d_keys_out, n, stream, wait=0):
    """Keys-only sort of n <= 2^20 keys that allocates nothing (fixed scratch
    inside the library; see include/bsort.h)."""
    return _check(None, load_library().bsort_sort_keys_noalloc(key_type, d_keys_in, d_keys_out,
                                                               n, stream, wait))


def _offsets_arg(seg_offsets):
    """Host uint64 array of num_segs + 1 offsets, kept alive by the caller."""
    import numpy as np
    arr = np.ascontiguousarray(seg_offsets, dtype=np.uint64)
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), max(arr.size - 1, 0)


def bsort_sort_batch(h, key_type, d_keys_in, d_keys_out, seg_offsets, stream):
    arr, ptr, nseg = _offsets_arg(seg_offsets)
    return _check(h, load_library().bsort_sort_batch(h, key_type, d_keys_in, d_keys_out, ptr,
                                                     nseg, stream))


def bsort_plan_batch(h, key_type, seg_offsets):
    arr, ptr, nseg = _offsets_arg(seg_offsets)
    info = bsort_batch_info()
    _check(h, load_library().bsort_plan_batch(h, key_type, ptr, nseg, ctypes.byref(info)))
    return info


def bsort_submit(h, key_type, h_keys_in, h_keys_out, n):
    req = bsort_request(key_type=key_type, n=n, h_keys_in=h_keys_in, h_keys_out=h_keys_out)
    ticket = ctypes.c_uint64()
    _check(h, load_library().bsort_submit(h, ctypes.byref(req), ctypes.byref(ticket)))
    return ticket.value


def bsort_poll(h, ticket):
    """bsort_result once the job is done, else None."""
    res = bsort_result()
    st = load_library().bsort_poll(h, ticket, ctypes.byref(res))
    if st == BSORT_ENOTREADY:
        return None
    _check(h, st)
    return res


def bsort_poll_any(h, cap=256):
    """[(ticket, bsort_result)] of up to cap finished jobs (released)."""
    tk = (ctypes.c_uint64 * cap)()
    rs = (bsort_result * cap)()
    cnt = ctypes.c_uint32()
    _check(h, load_library().bsort_poll_any(h, tk, rs, cap, ctypes.byref(cnt)))
    return [(tk[i], rs[i]) for i in range(cnt.value)]


def bsort_serve_stats(h):
    info = bsort_serve_info()
    _check(h, load_library().bsort_serve_stats(h, ctypes.byref(info)))
    return info


def bsort_clock_ns():
    return load_library().bsort_clock_ns()


def bsort_kernel_name(h, index):
    return load_library().bsort_kernel_name(h, index).decode()


# ------------------------------------------------------------ torch wrapper

_KEY_TYPES = {"u32": BSORT_U32, "f32": BSORT_F32, "u64": BSORT_U64}


class BucketSorter:
    """One library handle on one CUDA device, its workspace owned by a torch
    tensor.  ``sort_keys``/``sort_pairs`` take CUDA tensors (uint32 keys may be
    given as torch.int32 bit patterns) and run on the current torch stream."""

    def __init__(self, device: int = 0, tile: int = 0, samples: int = 0,
                 timing: bool = False, workspace_bytes: int = 0, low_memory: bool = False,
                 buckets: int = 0, batch_direct_max: int = 0, graphs: bool = False,
                 merge_sort: bool = False, flags: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.flags = ((BSORT_FLAG_TIMING if timing else 0) | (BSORT_FLAG_LOW_MEMORY if low_memory else 0)
                      | (BSORT_FLAG_GRAPHS if graphs else 0)
                      | (BSORT_FLAG_MERGE_SORT if merge_sort else 0) | int(flags))
        self.tile, self.samples, self.buckets = tile, samples, buckets
        self.batch_direct_max = batch_direct_max
        self.ws = None
        self.h = None
        self._make(workspace_bytes)

    def _make(self, nbytes):
        torch = self.torch
        if self.h is not None:
            bsort_destroy(self.h)
            self.h = None
        cfg = bsort_config(device=self.device, tile=self.tile, samples=self.samples,
                           flags=self.flags, buckets=self.buckets,
                           batch_direct_max=self.batch_direct_max)
        if nbytes:
            self.ws = torch.empty(int(nbytes), dtype=torch.uint8,
                                  device="cuda:%d" % self.device)
            cfg.workspace = self.ws.data_ptr()
            cfg.workspace_bytes = int(nbytes)
        self.h = bsort_create(cfg)

    def plan(self, n, key_type="u32", val_bytes=0):
        return bsort_plan(self.h, _KEY_TYPES[key_type], val_bytes, n)

    def _ensure(self, n, key_type, val_bytes, extra=0):
        need = self.plan(n, key_type, val_bytes).workspace_bytes + extra
        if self.ws is None or self.ws.numel() < need:
            self._make(max(need, 256))

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def sort_keys(self, keys, out=None, key_type="u32"):
        n = keys.numel()
        if out is None:
            out = self.torch.empty_like(keys)
        self._ensure(n, key_type, 0)
        bsort_sort_keys(self.h, _KEY_TYPES[key_type], keys.data_ptr(), out.data_ptr(), n,
                        self._stream())
        return out

    def sort_pairs(self, keys, vals, out_keys=None, out_vals=None, key_type="u32"):
        n = keys.numel()
        vb = vals.element_size()
        if out_keys is None:
            out_keys = self.torch.empty_like(keys)
        if out_vals is None:
            out_vals = self.torch.empty_like(vals)
        self._ensure(n, key_type, vb)
        bsort_sort_pairs(self.h, _KEY_TYPES[key_type], keys.data_ptr(), vals.data_ptr(),
                         out_keys.data_ptr(), out_vals.data_ptr(), vb, n, self._stream())
        return out_keys, out_vals

    def plan_batch(self, seg_offsets, key_type="u32"):
        return bsort_plan_batch(self.h, _KEY_TYPES[key_type], seg_offsets)

    def sort_batch(self, keys, seg_offsets, out=None, key_type="u32"):
        """Sort every segment [seg_offsets[q], seg_offsets[q+1]) of keys on
        its own (seg_offsets: host sequence of num_segs + 1 offsets)."""
        if out is None:
            out = self.torch.empty_like(keys)
        need = self.plan_batch(seg_offsets, key_type).workspace_bytes
        if self.ws is None or self.ws.numel() < need:
            self._make(max(need, 256))
        bsort_sort_batch(self.h, _KEY_TYPES[key_type], keys.data_ptr(), out.data_ptr(),
                         seg_offsets, self._stream())
        return out

    def sort_keys_host(self, h_keys, h_out, key_type="u32"):
        """Host tensors (pinned for asynchronous copies) in and out."""
        n = h_keys.numel()
        self._ensure(n, key_type, 0,
                     extra=((n * h_keys.element_size() + 255) // 256) * 256 + 256)
        bsort_sort_keys_host(self.h, _KEY_TYPES[key_type], h_keys.data_ptr(),
                             h_out.data_ptr(), n, self._stream())
        return h_out

    def sync(self):
        return bsort_sync(self.h, self._stream())

    def intermediate(self, which, nbytes, dtype):
        import numpy as np
        buf = np.empty(nbytes // np.dtype(dtype).itemsize, dtype=dtype)
        bsort_get_intermediate(self.h, which, buf.ctypes.data, nbytes)
        return buf

    def kernel_times(self):
        return bsort_kernel_times(self.h)

    def close(self):
        if self.h is not None:
            bsort_destroy(self.h)
            self.h = None
        self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SortServer:
    """A handle that serves sort jobs (bsort_submit / bsort_poll): host
    tensors in and out (pinned for asynchronous copies), results polled by
    ticket.  The handle's device memory is the serving budget."""

    def __init__(self, device: int = 0, budget_bytes: int = 4 << 30, batch_direct_max: int = 0):
        self.h = bsort_create(bsort_config(device=device, serve_budget_bytes=int(budget_bytes),
                                           batch_direct_max=batch_direct_max))
        self._alive = {}

    def submit(self, h_keys, h_out, key_type="u32"):
        t = bsort_submit(self.h, _KEY_TYPES[key_type], h_keys.data_ptr(), h_out.data_ptr(),
                         h_keys.numel())
        self._alive[t] = (h_keys, h_out)  # keep the buffers alive until polled
        return t

    def poll(self, ticket):
        res = bsort_poll(self.h, ticket)
        if res is not None:
            self._alive.pop(ticket, None)
        return res

    def wait(self, ticket, sleep_s=20e-6):
        import time
        while True:
            res = self.poll(ticket)
            if res is not None:
                return res
            time.sleep(sleep_s)

    def poll_any(self, cap=256):
        """[(ticket, bsort_result)] of finished jobs, in completion order."""
        done = bsort_poll_any(self.h, cap)
        for t, _ in done:
            self._alive.pop(t, None)
        return done

    def stats(self):
        return bsort_serve_stats(self.h).as_dict()

    def close(self):
        if self.h is not None:
            bsort_destroy(self.h)
            self.h = None
        self._alive.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
