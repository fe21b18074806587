"""CPU oracle for GPU Bucket Sort -- TEST INFRASTRUCTURE ONLY.

A plain C statement of Algorithm 1 (Dehne & Zaboli, Section 4, Steps 1-9)
plus an independent bottom-up merge sort, compiled with gcc and called via
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package; the CUDA library and
its Python binding never do.

Parity pins (brute force on tiny inputs, the textbook sort, closed-form
bucket sizes, the bucket-size bound) live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsort_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lib = None


def compile_to(src: str, out: str) -> str:
    """Compile a C source of the oracle into the shared library ``out``."""
    tmp = out + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp,
                           src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_to(_SRC, _LIB_PATH)


@contextlib.contextmanager
def use_library(path: str):
    """Run the oracle functions on another build of the oracle source while
    the context is open (the planted-mistake tests compile mutated copies of
    ``bsort_oracle.c`` and check that the pins reject them)."""
    global _lib
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    """Declare the argument and result types of the oracle's C functions."""
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.oracle_paper_sort.restype = ctypes.c_int
    lib.oracle_paper_sort.argtypes = [u64p, u64p, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64] + [u64p] * 13
    lib.oracle_paper_sort_mt.restype = ctypes.c_int
    lib.oracle_paper_sort_mt.argtypes = lib.oracle_paper_sort.argtypes + [ctypes.c_int]
    lib.oracle_textbook_sort.restype = ctypes.c_int
    lib.oracle_textbook_sort.argtypes = [u64p, u64p, ctypes.c_uint64,
                                         u64p, u64p]
    lib.oracle_f32_to_key.restype = ctypes.c_uint32
    lib.oracle_f32_to_key.argtypes = [ctypes.c_uint32]
    lib.oracle_key_to_f32.restype = ctypes.c_uint32
    lib.oracle_key_to_f32.argtypes = [ctypes.c_uint32]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_f32_to_key_array.restype = None
    lib.oracle_f32_to_key_array.argtypes = [u32p, u32p, ctypes.c_uint64]
    lib.oracle_key_to_f32_array.restype = None
    lib.oracle_key_to_f32_array.argtypes = [u32p, u32p, ctypes.c_uint64]
    lib.oracle_num_sublists.restype = ctypes.c_uint64
    lib.oracle_num_sublists.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    return lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


KEY_MAX = {"u32": 0xFFFFFFFF, "f32": 0xFFFFFFFF, "u64": 0xFFFFFFFFFFFFFFFF}


def f32_to_key(bits: np.ndarray) -> np.ndarray:
    """Order-preserving float32-bits -> uint32 map (oracle's own statement)."""
    lib = _load()
    b = np.ascontiguousarray(bits, dtype=np.uint32).ravel()
    out = np.empty_like(b)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_f32_to_key_array(b.ctypes.data_as(u32p), out.ctypes.data_as(u32p), b.size)
    return out


def key_to_f32(keys: np.ndarray) -> np.ndarray:
    lib = _load()
    k = np.ascontiguousarray(keys, dtype=np.uint32).ravel()
    out = np.empty_like(k)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_key_to_f32_array(k.ctypes.data_as(u32p), out.ctypes.data_as(u32p), k.size)
    return out


def _to_u64_keys(keys: np.ndarray, key_type: str) -> np.ndarray:
    if key_type == "f32":
        bits = np.ascontiguousarray(keys).view(np.uint32)
        return f32_to_key(bits).astype(np.uint64)
    if key_type == "u32":
        return np.ascontiguousarray(keys, dtype=np.uint32).astype(np.uint64)
    if key_type == "u64":
        return np.ascontiguousarray(keys, dtype=np.uint64).copy()
    raise ValueError(key_type)


def _from_u64_keys(k: np.ndarray, key_type: str) -> np.ndarray:
    if key_type == "f32":
        return key_to_f32(k.astype(np.uint32)).view(np.float32)
    if key_type == "u32":
        return k.astype(np.uint32)
    return k


def paper_sort(keys: np.ndarray, t: int, s: int, key_type: str = "u32",
               vals: Optional[np.ndarray] = None,
               intermediates: bool = True, b: int = 0, threads: int = 1) -> Dict[str, np.ndarray]:
    """Run Algorithm 1 on the CPU.  Returns the sorted keys (and values) and,
    if ``intermediates``, every intermediate of Steps 2-8 (in the transformed
    key domain for float32).  ``b`` is the number of buckets (0: b = s, the
    paper's choice).  ``threads`` > 1 spreads the per-sublist and per-bucket
    iterations of Steps 2, 6, 8 and 9 over that many threads (same code,
    same result)."""
    lib = _load()
    n = int(np.asarray(keys).size)
    k64 = _to_u64_keys(np.asarray(keys).ravel(), key_type)
    v64 = None if vals is None else np.ascontiguousarray(vals).astype(np.uint64)
    m = int(lib.oracle_num_sublists(n, t)) if n else 0
    npad = m * t
    nb = b if b else s
    out_k = np.zeros(n, np.uint64)
    out_v = np.zeros(n, np.uint64) if vals is not None else None
    res: Dict[str, np.ndarray] = {}
    names = [("tile_keys", npad), ("tile_pos", npad), ("samp_keys", m * s),
             ("samp_p", m * s), ("spl_keys", nb), ("spl_p", nb),
             ("counts", m * nb), ("offsets", m * nb), ("reloc_keys", npad),
             ("reloc_pos", npad), ("bucket_start", nb + 1)]
    bufs = []
    for name, size in names:
        if intermediates and n:
            arr = np.zeros(size, np.uint64)
            res[name] = arr
            bufs.append(arr)
        else:
            bufs.append(None)
    if threads > 1:
        rc = lib.oracle_paper_sort_mt(_ptr(k64), _ptr(v64), n, t, s, b,
                                      KEY_MAX[key_type], _ptr(out_k), _ptr(out_v),
                                      *[_ptr(x) for x in bufs], int(threads))
    else:
        rc = lib.oracle_paper_sort(_ptr(k64), _ptr(v64), n, t, s, b,
                                   KEY_MAX[key_type], _ptr(out_k), _ptr(out_v),
                                   *[_ptr(x) for x in bufs])
    if rc != 0:
        raise ValueError("oracle_paper_sort failed (n=%d t=%d s=%d b=%d)" % (n, t, s, b))
    res["keys"] = _from_u64_keys(out_k, key_type)
    if out_v is not None:
        res["vals"] = out_v.astype(np.asarray(vals).dtype)
    res["m"] = m
    res["n_padded"] = npad
    return res


def textbook_sort(keys: np.ndarray, key_type: str = "u32",
                  vals: Optional[np.ndarray] = None):
    """Independent stable bottom-up merge sort (O2)."""
    lib = _load()
    n = int(np.asarray(keys).size)
    k64 = _to_u64_keys(np.asarray(keys).ravel(), key_type)
    v64 = None if vals is None else np.ascontiguousarray(vals).astype(np.uint64)
    out_k = np.zeros(n, np.uint64)
    out_v = np.zeros(n, np.uint64) if vals is not None else None
    rc = lib.oracle_textbook_sort(_ptr(k64), _ptr(v64), n, _ptr(out_k), _ptr(out_v))
    if rc != 0:
        raise MemoryError("oracle_textbook_sort failed")
    keys_out = _from_u64_keys(out_k, key_type)
    if vals is None:
        return keys_out
    return keys_out, out_v.astype(np.asarray(vals).dtype)


def bucket_bound(n_padded: int, m: int, s: int, b: int = 0) -> int:
    """Upper bound on |B_j| for the sampling rule above: n'/s + (m-1)(w-1)
    for b = s, derived from the positions of the regular samples (tighter
    than the paper's 2n/s, Section 4, Step 8 discussion); with b buckets,
    ceil(m*s/b)*w + (m-1)(w-1)."""
    t = n_padded // m
    w = t // s
    b = b or s
    return -(-(m * s) // b) * w + (m - 1) * (w - 1)
