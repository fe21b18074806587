"""GPU parity of the batched sort (bsort_sort_batch): every segment of the
output equals the textbook sort of that segment of the input, bit for bit,
and keys outside every segment are left untouched."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1002_4464_gb300 as pkg  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _expect(keys, off, key_type="u32"):
    """Per-segment textbook sort (oracle); keys outside segments unchanged."""
    want = keys.copy()
    for q in range(len(off) - 1):
        a, b = int(off[q]), int(off[q + 1])
        if b > a:
            want[a:b] = oracle.textbook_sort(keys[a:b], key_type)
    return want


def _run(sorter, keys, off, key_type="u32", out=None):
    d_in = _dev(keys)
    if out is None:
        d_out = sorter.sort_batch(d_in, off, key_type=key_type)
    else:
        d_out = _dev(out)
        sorter.sort_batch(d_in, off, out=d_out, key_type=key_type)
    sorter.sync()
    return d_out.cpu().numpy().view(np.uint32)


# one segment of every class: empty, one key, direct shapes 2048 .. 8 x 32768,
# sampled segments (ragged last sublist, exact multiples), a plain-sorted one
EDGE_SIZES = [0, 1, 2, 3, 127, 2047, 2048, 2049, 4096, 8191, 16384, 16385, 32768, 32769,
              65536, 65537, 131072, 131073, 163840, 200001, 262144, 300000, 524288, 524289,
              1, 0, 5]


@pytest.mark.parametrize("dist", ["uniform", "zero", "sorted", "reverse", "staggered"])
def test_batch_every_class(dist):
    sizes = np.array(EDGE_SIZES, np.int64)
    off = np.concatenate([[7], 7 + np.cumsum(sizes)]).astype(np.uint64)  # keys 0..6 outside
    n = int(off[-1]) + 11                                                # and 11 after
    keys = synth.keys_u32(dist, n, synth.seed_for(4, synth.DISTRIBUTIONS.index(dist)))
    sorter = pkg.BucketSorter()
    p = sorter.plan_batch(off)
    assert p.direct_segs > 0 and p.sampled_segs > 0 and p.large_segs == 1
    sentinel = np.full(n, 0xA5A5A5A5, np.uint32)
    got = _run(sorter, keys, off, out=sentinel)
    want = _expect(keys, off)
    want[:7] = 0xA5A5A5A5
    want[int(off[-1]):] = 0xA5A5A5A5
    assert np.array_equal(got, want)
    sorter.close()


@pytest.mark.parametrize("direct_max", [2048, 32768, 131072, 262144])
def test_batch_log_uniform(direct_max):
    """A scaled-down batched workload: 400 arrays, log-uniform sizes in
    [2^7, 2^20] (about 2^25 keys in all), uniform keys."""
    sizes = synth.batch_sizes(400, synth.seed_for(4, 0, 1), cap=1 << 27)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    keys = synth.keys_u32("uniform", n, synth.seed_for(4, 0, 2))
    sorter = pkg.BucketSorter(batch_direct_max=direct_max)
    got = _run(sorter, keys, off)
    seg = np.repeat(np.arange(len(sizes)), sizes)
    want = keys[np.lexsort((keys, seg))]  # library sort, segment-major
    assert np.array_equal(got, want)
    sorter.close()


def test_batch_f32_and_in_place():
    sizes = np.array([3000, 140000, 40000, 260000, 9], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    f = synth.keys_f32("gaussian", n, synth.seed_for(4, 3))
    f[:8] = np.array([np.inf, -np.inf, np.nan, -0.0, 0.0, 1e-45, -1e-45, -np.nan], np.float32)
    f[140000:140008] = f[:8]
    sorter = pkg.BucketSorter()
    d = torch.from_numpy(f.copy()).cuda()
    sorter.sort_batch(d, off, out=d, key_type="f32")
    sorter.sync()
    got = d.cpu().numpy().view(np.uint32)
    want = _expect(f, off, "f32").view(np.uint32)
    assert np.array_equal(got, want)
    sorter.close()


def test_batch_equals_one_at_a_time():
    """Each segment's result is the same sorted alone and in the batch."""
    sizes = synth.batch_sizes(200, synth.seed_for(4, 4), cap=1 << 24)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = synth.keys_zipf(int(off[-1]), synth.seed_for(4, 5))
    sorter = pkg.BucketSorter()
    got = _run(sorter, keys, off)
    d_in = _dev(keys)
    alone = np.empty_like(keys)
    for q in range(len(sizes)):
        a, b = int(off[q]), int(off[q + 1])
        o = sorter.sort_keys(d_in[a:b])
        sorter.sync()
        alone[a:b] = o.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, alone)
    # and again: the batch is deterministic
    assert np.array_equal(_run(sorter, keys, off), got)
    sorter.close()


def test_batch_u64():
    """64-bit keys: segments up to 262144 keys sorted whole (CTAs of 16384
    keys, clusters up to 16 where the device schedules a 16-CTA cluster,
    else up to 8 and 131072 keys), larger ones up to 2^20 by the
    segment-aware sample sort (sublists of 16384 keys, s = 256 up to 32
    sublists and 128 above), larger ones by a plain sort each."""
    sizes = np.array([0, 1, 2, 1000, 2048, 2049, 16384, 16385, 65536, 131072, 131073, 200001,
                      262144, 262145, 400000, 524288, 524289, 1 << 20, (1 << 20) + 1, 7],
                     np.int64)
    off = np.concatenate([[3], 3 + np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1]) + 5
    keys = synth.keys_u64(n, synth.seed_for(5, 4))
    keys[::7] &= np.uint64(0xFF)  # duplicates
    sorter = pkg.BucketSorter()
    wide16 = sorter.plan_batch(np.array([0, 262144], np.uint64), "u64").direct_segs == 1
    p = sorter.plan_batch(off, "u64")
    if wide16:
        assert (p.direct_segs, p.sampled_segs, p.large_segs) == (12, 5, 1)
    else:
        assert (p.direct_segs, p.sampled_segs, p.large_segs) == (9, 8, 1)
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.full_like(d_in, 0x5A5A)
    sorter.sort_batch(d_in, off, out=d_out, key_type="u64")
    sorter.sync()
    got = d_out.cpu().numpy().view(np.uint64)
    want = np.full(n, 0x5A5A, np.uint64)
    for q in range(len(sizes)):
        a, b = int(off[q]), int(off[q + 1])
        want[a:b] = oracle.textbook_sort(keys[a:b], "u64")
    assert np.array_equal(got, want)
    sorter.close()


@pytest.mark.parametrize("direct_max", [2048, 16384])
def test_batch_u64_log_uniform(direct_max):
    """64-bit keys with a low direct limit, so that sampled segments of 1 to
    64 sublists occur: 200 arrays, log-uniform sizes in [2^7, 2^20] (at most
    2^25 keys in all), uniform keys with every seventh key cut to 8 bits."""
    sizes = synth.batch_sizes(200, synth.seed_for(4, 7, direct_max), cap=1 << 25)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    keys = synth.keys_u64(n, synth.seed_for(4, 7, 1))
    keys[::7] &= np.uint64(0xFF)
    sorter = pkg.BucketSorter(batch_direct_max=direct_max)
    p = sorter.plan_batch(off, "u64")
    sampled = [x for x in sizes if direct_max < x <= 1 << 20]
    assert p.sampled_segs == len(sampled) and p.large_segs == 0
    assert p.sublists == sum(-(-int(x) // 16384) for x in sampled)
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty_like(d_in)
    sorter.sort_batch(d_in, off, out=d_out, key_type="u64")
    sorter.sync()
    got = d_out.cpu().numpy().view(np.uint64)
    seg = np.repeat(np.arange(len(sizes)), sizes)
    want = keys[np.lexsort((keys, seg))]  # library sort, segment-major
    assert np.array_equal(got, want)
    sorter.close()


def test_batch_u64_sampled_ties():
    """Sampled 64-bit segments whose keys tie: all equal to the largest key
    (the value that pads the last sublist of a segment), 16 distinct values,
    and all zero, beside uniform keys; the ties are ordered by position in
    the samples and splitters, so every bucket stays within its unit."""
    sizes = [300000, 524289, 1 << 20, 700001, 262145]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    keys = synth.keys_u64(n, synth.seed_for(5, 6))
    a = [int(x) for x in off]
    keys[a[0]:a[1]] = np.uint64(0xFFFFFFFFFFFFFFFF)
    keys[a[1]:a[2]] &= np.uint64(0xF000000000000000)
    keys[a[2]:a[3]] = 0
    keys[a[4]:a[5]] |= np.uint64(0xFFFFFFFFFFFFFF00)  # near the largest key
    sorter = pkg.BucketSorter()
    p = sorter.plan_batch(off, "u64")
    assert p.sampled_segs == 5 and p.large_segs == 0
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty_like(d_in)
    sorter.sort_batch(d_in, off, out=d_out, key_type="u64")
    sorter.sync()
    got = d_out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, _expect(keys, off, "u64"))
    # in place
    sorter.sort_batch(d_in, off, out=d_in, key_type="u64")
    sorter.sync()
    assert np.array_equal(d_in.cpu().numpy().view(np.uint64), got)
    sorter.close()


def test_batch_graph_replay():
    """BSORT_FLAG_GRAPHS on bsort_sort_batch: the first call with a segment
    table is captured, later calls with the same table, buffers and stream
    replay the graph, with new key contents each time; a different table is
    captured anew; every result equals the per-segment textbook sort."""
    sizes = [0, 1, 5, 2049, 40000, 131073, 300000, 700001, 17]  # direct, sampled, large
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    side = torch.cuda.Stream()
    sorter = pkg.BucketSorter(graphs=True)
    with torch.cuda.stream(side):
        d_in = torch.empty(n, dtype=torch.int32, device="cuda")
        d_out = torch.empty_like(d_in)
        for rep in range(3):
            keys = synth.keys_u32("uniform" if rep != 1 else "staggered", n,
                                  synth.seed_for(4, 9, rep))
            d_in.copy_(torch.from_numpy(keys.view(np.int32)))
            sorter.sort_batch(d_in, off, out=d_out)
            sorter.sync()
            side.synchronize()
            assert np.array_equal(d_out.cpu().numpy().view(np.uint32), _expect(keys, off))
        off2 = np.concatenate([[0], np.cumsum(sizes[::-1])]).astype(np.uint64)
        keys = synth.keys_u32("gaussian", n, synth.seed_for(4, 9, 7))
        d_in.copy_(torch.from_numpy(keys.view(np.int32)))
        sorter.sort_batch(d_in, off2, out=d_out)
        sorter.sync()
        side.synchronize()
        assert np.array_equal(d_out.cpu().numpy().view(np.uint32), _expect(keys, off2))
    sorter.close()
