"""The allocation-free entry point bsort_sort_keys_noalloc, called through
the C ABI: its output equals the oracle's textbook sort and the library's
bsort_sort_keys, on two calls in a row.

Some callers cannot allocate device memory (their allocator or memory budget
is fixed, or cudaMalloc is not allowed where they run); this entry point
serves them from a fixed scratch array inside the library.  The file is
named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1002_4464_gb300 as pkg  # noqa: E402


def _sort_keys(keys_dev, key_type):
    sorter = pkg.BucketSorter()
    out = sorter.sort_keys(keys_dev, key_type=key_type)
    sorter.sync()
    sorter.close()
    return out.cpu().numpy().view(np.uint32)


def _want(keys, key_type):
    if key_type == "f32":
        return oracle.textbook_sort(keys, "f32").view(np.uint32)
    return oracle.textbook_sort(keys, "u32")


def _call(lib, kt, d_in, d_out, n, wait=1):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bsort_sort_keys_noalloc(kt, d_in.data_ptr() if d_in is not None else None,
                                       d_out.data_ptr() if d_out is not None else None,
                                       n, stream, wait)


CASES = [
    ("u32", "uniform", 1 << 20),    # the maximum n
    ("f32", "gaussian", 300001),    # ragged, floats
    ("u32", "staggered", 262144),   # one cluster unit, no sampling
    ("u32", "zero", 1000),          # one CTA, all keys equal
    ("u32", "uniform", 1),
]


@pytest.mark.parametrize("key_type,dist,n", CASES)
def test_noalloc_matches_oracle_and_sort_keys_twice(key_type, dist, n):
    """Two calls in a row (the second reuses the scratch the first left),
    each checked against the oracle's textbook sort and bsort_sort_keys."""
    lib = pkg.load_library()
    kt = pkg.BSORT_U32 if key_type == "u32" else pkg.BSORT_F32
    for rep in range(2):
        seed = synth.seed_for(7, rep, n % 1000)
        keys = synth.keys_u32(dist, n, seed) if key_type == "u32" else \
            synth.keys_f32(dist, n, seed)
        d_in = torch.from_numpy(np.ascontiguousarray(keys).view(np.int32)).cuda()
        d_out = torch.empty_like(d_in)
        st = _call(lib, kt, d_in, d_out, n)
        assert st == pkg.BSORT_OK, pkg.bsort_status_string(st)
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, _want(keys, key_type))  # bit-exact
        assert np.array_equal(got, _sort_keys(d_in, key_type))
        assert np.array_equal(d_in.cpu().numpy().view(np.uint32), keys.view(np.uint32))


def test_noalloc_in_place_and_empty():
    lib = pkg.load_library()
    keys = synth.keys_u32("reverse", 100003, synth.seed_for(7, 2))
    d = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    assert _call(lib, pkg.BSORT_U32, d, d, keys.size) == pkg.BSORT_OK
    assert np.array_equal(d.cpu().numpy().view(np.uint32), _want(keys, "u32"))
    assert _call(lib, pkg.BSORT_U32, None, None, 0) == pkg.BSORT_OK


def test_noalloc_wait0_then_wait1():
    """A call that does not wait, then one that does, on the same stream:
    both outputs are right (the second call reports the status of both)."""
    lib = pkg.load_library()
    a = synth.keys_u32("uniform", 500000, synth.seed_for(7, 3))
    b = synth.keys_u32("bucket", 700001, synth.seed_for(7, 4))
    da, oa = torch.from_numpy(a.view(np.int32)).cuda(), None
    db = torch.from_numpy(b.view(np.int32)).cuda()
    oa, ob = torch.empty_like(da), torch.empty_like(db)
    assert _call(lib, pkg.BSORT_U32, da, oa, a.size, wait=0) == pkg.BSORT_OK
    assert _call(lib, pkg.BSORT_U32, db, ob, b.size, wait=1) == pkg.BSORT_OK
    assert np.array_equal(oa.cpu().numpy().view(np.uint32), _want(a, "u32"))
    assert np.array_equal(ob.cpu().numpy().view(np.uint32), _want(b, "u32"))


def test_noalloc_rejects_too_many_keys():
    lib = pkg.load_library()
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.bsort_sort_keys_noalloc(pkg.BSORT_U32, d.data_ptr(), d.data_ptr(),
                                     (1 << 20) + 1, None, 1)
    assert st == pkg.BSORT_EINVAL
    st = lib.bsort_sort_keys_noalloc(pkg.BSORT_U64, d.data_ptr(), d.data_ptr(), 2, None, 1)
    assert st == pkg.BSORT_EUNSUPPORTED
