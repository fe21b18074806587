"""GPU parity of the radix-sorting CTAs (a unit of 32768 32-bit keys sorted
by one CTA in Step 2 or Step 9 of Algorithm 1 is sorted by 7-bit digits over
the bits that vary in the unit): key ranges at every pass-width boundary,
ragged fills, float keys, single-unit sorts and clusters, and every
intermediate of forced and planner-shaped plans against the CPU oracle, bit
for bit.  The comparison sort (BSORT_FLAG_MERGE_SORT) must give the same
results."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, run on the GPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1002_4464_gb300 as pkg  # noqa: E402


def _rec(k, p):
    return (np.asarray(k).astype(np.uint64) << np.uint64(32)) | np.asarray(p).astype(np.uint64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _sort(sorter, keys, key_type="u32"):
    out = sorter.sort_keys(_dev(keys), key_type=key_type)
    sorter.sync()
    return out.cpu().numpy().view(np.uint32)


def _ranged(n, lo, span, seed):
    """n uint32 keys in [lo, lo + span], both ends present."""
    u = synth.keys_u32("uniform", n, seed).astype(np.uint64)
    k = (np.uint64(lo) + u % np.uint64(span + 1)).astype(np.uint32)
    if n >= 2:
        k[n // 3] = np.uint32(lo)
        k[(2 * n) // 3] = np.uint32(lo + span)
    return k


# spans whose bit counts sit on both sides of the 7-bit digit boundaries
SPANS = [0, 1, 126, 127, 128, (1 << 14) - 1, 1 << 14, (1 << 21) + 5, (1 << 28) + 3,
         0xFFFFFFFF]


@pytest.mark.parametrize("n", [16385, 20000, 32767, 32768])
@pytest.mark.parametrize("span", SPANS)
def test_one_chunk_ranges(n, span):
    """n in (16384, 32768]: one 32768-key radix CTA sorts the whole input."""
    los = [0, 0xFFFFFFFF - span, 0x12345678 % (0xFFFFFFFF - span + 1)]
    sorter = pkg.BucketSorter()
    assert sorter.plan(n).single_tile == 1
    for i, lo in enumerate(los):
        keys = _ranged(n, lo, span, synth.seed_for(6, 1, span % 251 + 7 * i))
        got = _sort(sorter, keys)
        assert np.array_equal(got, oracle.textbook_sort(keys, "u32"))
    sorter.close()


@pytest.mark.parametrize("n", [32769, 40000, 65536, 100001, 262144])
@pytest.mark.parametrize("span", [0, 300, (1 << 21) + 5, 0xFFFFFFFF])
def test_cluster_unit_ranges(n, span):
    """One unit above 32768 keys: a cluster of 2-8 CTAs merged through
    distributed shared memory (each CTA's padding must sort after every real
    key of the cluster); radix and comparison sorts agree."""
    keys = _ranged(n, 0x40000000 if span < 0x40000000 else 0, span,
                   synth.seed_for(6, 2, n % 1000))
    sorter = pkg.BucketSorter()
    got = _sort(sorter, keys)
    assert np.array_equal(got, oracle.textbook_sort(keys, "u32"))
    ref = pkg.BucketSorter(merge_sort=True)
    assert np.array_equal(_sort(ref, keys), got)
    sorter.close()
    ref.close()


@pytest.mark.parametrize("dist", ["uniform", "zero", "sorted", "staggered"])
def test_float_keys_one_chunk(dist):
    n = 30001
    f = synth.keys_f32(dist, n, synth.seed_for(6, 3))
    f[:12] = np.array([np.inf, -np.inf, np.nan, -0.0, 0.0, 1e-45, -1e-45, 3.4e38, -3.4e38,
                       np.float32(-np.nan), 1.0, -1.0], np.float32)
    sorter = pkg.BucketSorter()
    d = torch.from_numpy(f.copy()).cuda()
    out = sorter.sort_keys(d, key_type="f32")
    sorter.sync()
    want = oracle.textbook_sort(f, "f32").view(np.uint32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
    sorter.close()


def _check_intermediates(sorter, want, s, b):
    n_pad, m = want["n_padded"], want["m"]
    got_t = sorter.intermediate(pkg.BSORT_IM_TILES, n_pad * 4, np.uint32)
    assert np.array_equal(got_t, want["tile_keys"].astype(np.uint32)), "Step 2 sublists"
    got_s = sorter.intermediate(pkg.BSORT_IM_SAMPLES, m * s * 8, np.uint64)
    assert np.array_equal(got_s, _rec(want["samp_keys"], want["samp_p"])), "Step 3 samples"
    got_g = sorter.intermediate(pkg.BSORT_IM_SPLITTERS, b * 8, np.uint64)
    assert np.array_equal(got_g, _rec(want["spl_keys"], want["spl_p"])), "Step 5 splitters"
    got_a = sorter.intermediate(pkg.BSORT_IM_COUNTS, m * b * 4, np.uint32)
    assert np.array_equal(got_a, want["counts"].astype(np.uint32)), "Step 6 counts"
    got_l = sorter.intermediate(pkg.BSORT_IM_OFFSETS, m * b * 4, np.uint32)
    assert np.array_equal(got_l, want["offsets"].astype(np.uint32)), "Step 7 offsets"
    got_r = sorter.intermediate(pkg.BSORT_IM_RELOCATED, n_pad * 4, np.uint32)
    assert np.array_equal(got_r, want["reloc_keys"].astype(np.uint32)), "Step 8 relocation"


@pytest.mark.parametrize("n,t,s,b", [
    ((1 << 21) + 777, 32768, 256, 0),   # one radix CTA per sublist, ragged tail
    ((1 << 22) + 5, 65536, 1024, 300),  # 2-CTA sublists, b != s, radix buckets
    (1 << 22, 131072, 2048, 0),         # 4-CTA sublists
])
@pytest.mark.parametrize("dist", ["uniform", "zero", "sorted", "staggered", "narrow"])
@pytest.mark.parametrize("merge", [False, True])
def test_forced_plans_intermediates(n, t, s, b, dist, merge):
    if dist == "narrow":  # few bits vary: most sublists and buckets need one pass
        keys = _ranged(n, 0x9000_0000, 200, synth.seed_for(6, 4, t % 997))
    else:
        keys = synth.keys_u32(dist, n, synth.seed_for(6, 5, synth.DISTRIBUTIONS.index(dist)))
        keys[::11] = keys[::11] & np.uint32(0xFFF)  # duplicates across sublists
    bb = b or s
    want = oracle.paper_sort(keys, t, s, "u32", b=bb)
    sorter = pkg.BucketSorter(tile=t, samples=s, buckets=b, merge_sort=merge)
    got = _sort(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, s, bb)
    sorter.close()


def test_planner_shape_two_tier_keys_intermediates():
    """The shape the planner picks for 2^28 uint32 keys (sublists of 65536
    sorted by 2-CTA clusters, s = 4096, Step 9 in two tiers: a one-CTA radix
    unit per bucket listed by k_units_each, the rare larger buckets sorted by
    looping cluster units) at 2^26 keys, b chosen so that the average bucket
    fills one CTA as at 2^28: every intermediate and the result against the
    oracle."""
    n, t, s = 1 << 26, 65536, 4096
    b = -(-n * 105 // (100 * 32768)) + 1  # average bucket just under 32768 / 1.05
    keys = synth.keys_u32("uniform", n, synth.seed_for(6, 6))
    sorter = pkg.BucketSorter(tile=t, samples=s, buckets=b)
    p = sorter.plan(n)
    assert (p.t, p.s, p.b, p.tile_ctas) == (t, s, b, 2)
    assert p.unit_small == 32768 and p.unit_ctas > 1  # two tiers
    want = oracle.paper_sort(keys, t, s, "u32", b=b)
    got = _sort(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, s, b)
    sorter.close()


def test_radix_equals_merge_sort_planner_plan():
    """2^24 + 3 Gaussian keys on the planner's plan: the radix and the
    comparison sorts agree with each other and with the textbook sort."""
    n = (1 << 24) + 3
    keys = synth.keys_u32("gaussian", n, synth.seed_for(6, 7))
    a = pkg.BucketSorter()
    b = pkg.BucketSorter(merge_sort=True)
    ga, gb = _sort(a, keys), _sort(b, keys)
    assert np.array_equal(ga, oracle.textbook_sort(keys, "u32"))
    assert np.array_equal(ga, gb)
    a.close()
    b.close()


def test_bench_workload_2e28_intermediates():
    """The benchmark workload itself: 2^28 uniform uint32 keys on the
    planner's own plan (two-tier Step 9 with one-CTA radix units): the
    sorted sublists, samples, splitters, counts, offsets, relocated array and
    the result against the oracle run with the same t, s and b."""
    n = 1 << 28
    keys = synth.keys_u32("uniform", n, synth.seed_for(2, 0))
    sorter = pkg.BucketSorter()
    p = sorter.plan(n)
    assert not p.single_tile and p.unit_small == 32768
    got = _sort(sorter, keys)
    want = oracle.paper_sort(keys, p.t, p.s, "u32", b=p.b)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, p.s, p.b)
    sorter.close()
