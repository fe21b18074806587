"""The allocation-free entry point bsort_sort_keys_noalloc, called through
the C ABI, gives the same keys as bsort_sort_keys on two calls in a row.

Some callers cannot allocate device memory (their allocator or memory budget
is fixed, or cudaMalloc is not allowed where they run); this entry point
serves them from a fixed scratch array inside the library.  The file is
named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1002_4464_gb300 as pkg  # noqa: E402


def _reference(keys_dev, key_type):
    sorter = pkg.BucketSorter()
    out = sorter.sort_keys(keys_dev, key_type=key_type)
    sorter.sync()
    sorter.close()
    return out.cpu().numpy().view(np.uint32)


def test_noalloc_matches_sort_keys_twice():
    lib = pkg.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [
        ("u32", synth.keys_u32("uniform", 1 << 20, synth.seed_for(6, 0))),      # the maximum n
        ("f32", synth.keys_f32("gaussian", 300001, synth.seed_for(6, 1))),      # ragged, floats
    ]
    for key_type, keys in cases:
        d_in = torch.from_numpy(keys.view(np.int32)).cuda()
        want = _reference(d_in, key_type)
        d_out = torch.empty_like(d_in)
        kt = pkg.BSORT_U32 if key_type == "u32" else pkg.BSORT_F32
        st = lib.bsort_sort_keys_noalloc(kt, d_in.data_ptr(), d_out.data_ptr(), keys.size,
                                         stream, 1)
        assert st == pkg.BSORT_OK, pkg.bsort_status_string(st)
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)  # bit-exact, as every sort parity test
        assert np.array_equal(d_in.cpu().numpy().view(np.uint32), keys.view(np.uint32))


def test_noalloc_rejects_too_many_keys():
    lib = pkg.load_library()
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.bsort_sort_keys_noalloc(pkg.BSORT_U32, d.data_ptr(), d.data_ptr(),
                                     (1 << 20) + 1, None, 1)
    assert st == pkg.BSORT_EINVAL
