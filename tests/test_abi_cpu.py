"""The C-ABI library builds, loads and exports every function that
include/bsort.h declares; the host-side planner (Step 1 parameters, the
Step-9 unit, the bucket bound) behaves as documented.  No GPU needed: these
calls touch no device."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1002_4464_gb300 as pkg
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsort.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(bsort_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = pkg.load_library()
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert set(declared) == set(pkg.EXPORTED_SYMBOLS)
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bsort_[a-z_0-9]+)\b", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(lib, f)


def test_status_strings():
    assert pkg.bsort_status_string(pkg.BSORT_OK) == "BSORT_OK"
    assert pkg.bsort_status_string(pkg.BSORT_ETIMEOUT) == "BSORT_ETIMEOUT"


def _handle(tile=0, samples=0, buckets=0):
    return pkg.bsort_create(pkg.bsort_config(device=0, tile=tile, samples=samples,
                                             buckets=buckets))


def test_plan_config1():
    """n = 2^20, m = 256 sublists, s = 64: t = 4096, w = 64,
    bound n/s + (m-1)(w-1) = 16384 + 255*63 = 32449 <= 2n/s = 32768."""
    h = _handle(4096, 64)
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert (p.t, p.s, p.m, p.w) == (4096, 64, 256, 64)
    assert p.n_padded == 1 << 20
    assert p.bucket_bound == 32449 <= 2 * (1 << 20) // 64
    assert p.unit_capacity >= p.bucket_bound
    assert p.single_tile == 0
    pkg.bsort_destroy(h)


@pytest.mark.parametrize("n", [2, 1000, 32768, 32769, 100000, 1 << 20, (1 << 20) + 17, 1 << 24])
def test_plan_auto_bound_fits_unit(n):
    h = _handle()
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, n)
    if p.single_tile:
        assert n <= 8 * 32768 and p.unit_capacity >= n
    else:
        assert p.t % p.s == 0 and p.m * p.t == p.n_padded >= n > p.n_padded - p.t
        w = p.t // p.s
        # b buckets from the m*s samples: ceil(ms/b) sample ranks of w items
        # plus w-1 items of every other sublist
        assert 1 <= p.b <= p.m * p.s
        assert p.bucket_bound == -(-p.m * p.s // p.b) * w + (p.m - 1) * (w - 1)
        assert p.bucket_bound == oracle.bucket_bound(p.n_padded, p.m, p.s, p.b)
        assert p.unit_capacity >= p.bucket_bound
        # about (k + 0.1) average buckets per unit for a whole k
        per_unit = p.unit_capacity * p.b / p.n_padded
        assert per_unit >= 1.0
    pkg.bsort_destroy(h)


def test_plan_bucket_count():
    """b = s when s is given (Section 4, Step 5); a forced b is kept and its
    bound is ceil(ms/b) w + (m-1)(w-1); b beyond m*s or 12288 is refused."""
    h = _handle(4096, 64)
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert p.b == p.s == 64 and p.bucket_bound == 32449
    pkg.bsort_destroy(h)
    h = _handle(4096, 64, 100)
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert p.b == 100
    assert p.bucket_bound == -(-256 * 64 // 100) * 64 + 255 * 63 == 26561
    pkg.bsort_destroy(h)
    h = _handle(4096, 64, 40)  # fewer buckets than samples: bound 41*64 + 16065
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert p.b == 40 and p.bucket_bound == 410 * 64 + 255 * 63
    pkg.bsort_destroy(h)
    h = _handle(4096, 64, 256 * 64 + 1)
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert e.value.status in (pkg.BSORT_EINVAL, pkg.BSORT_EUNSUPPORTED)
    pkg.bsort_destroy(h)
    h = _handle(0, 0, 12289)
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 24)
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    pkg.bsort_destroy(h)
    h = _handle(0, 0, 3000)  # forced b, planner's t and s
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 24)
    assert p.b == 3000 and p.unit_capacity >= p.bucket_bound
    pkg.bsort_destroy(h)


def test_plan_pairs_and_errors():
    h = _handle()
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 4, 1 << 20)
    assert p.unit_capacity >= p.bucket_bound and p.t <= 16384
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 3, 100)
    assert e.value.status == pkg.BSORT_EINVAL
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 35)
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    pkg.bsort_destroy(h)
    h = _handle(4096, 48)  # s must divide t
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 20)
    assert e.value.status == pkg.BSORT_EINVAL
    pkg.bsort_destroy(h)


def test_plan_paper_worked_parameters():
    """Section 4's example: n = 32M, n/m = 2K -> m = 16K sublists; with s = 64
    every bucket holds at most 2n/s = 1M items, more than one Step-9 unit
    holds: the planner refuses it rather than overflow a unit."""
    h = _handle(2048, 64)
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 32 << 20)
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    assert "1032161" in pkg.bsort_last_error(h)  # 2^25/64 + (2^14-1)(32-1)
    pkg.bsort_destroy(h)


def test_plan_batch_classes():
    """Segments up to batch_direct_max keys are sorted whole, larger ones up to
    524288 by the segment-aware sample sort (sublists of 32768, s = 1024, b
    buckets whose bound fits a 32768-key unit), larger ones by a plain sort."""
    sizes = [0, 1, 2, 100, 2048, 2049, 32768, 131072, 131073, 200000, 524288, 524289, 3]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    h = _handle()
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U32, off)
    assert p.num_segs == len(sizes) and p.n == sum(sizes)
    assert p.direct_segs == 7  # 2 .. 131072 (0 and 1 need no sort)
    assert p.sampled_segs == 3 and p.large_segs == 1
    assert p.sublists == 5 + 7 + 16
    b_expect = 0
    for n in (131073, 200000, 524288):
        m = -(-n // 32768)
        b = next(b for b in range(1, m * 1024 + 1)
                 if oracle.bucket_bound(m * 32768, m, 1024, b) <= 32768)
        b_expect += b
    assert p.buckets == b_expect
    pkg.bsort_destroy(h)
    h = pkg.bsort_create(pkg.bsort_config(device=0, batch_direct_max=32768))
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U32, off)
    assert p.direct_segs == 6 and p.sampled_segs == 4
    pkg.bsort_destroy(h)
    with pytest.raises(pkg.BsortError):
        pkg.bsort_create(pkg.bsort_config(device=0, batch_direct_max=262145))


def test_plan_batch_classes_u64():
    """64-bit keys: segments above the direct limit (131072 keys without a
    device, where the 16-CTA cluster is not known to run) up to 2^20 keys
    go through the segment-aware sample sort with sublists of 16384 keys,
    s = 256 samples per sublist up to 32 sublists and 128 above, and b
    buckets whose bound fits a 16384-key unit; larger ones a plain sort."""
    sizes = [5, 131072, 131073, 262145, 524288, 524289, 1 << 20, (1 << 20) + 1, 2]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    h = _handle()
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U64, off)
    assert p.num_segs == len(sizes) and p.n == sum(sizes)
    assert (p.direct_segs, p.sampled_segs, p.large_segs) == (3, 5, 1)
    sampled = (131073, 262145, 524288, 524289, 1 << 20)
    ms = [-(-n // 16384) for n in sampled]
    assert ms == [9, 17, 32, 33, 64]
    assert p.sublists == sum(ms)
    b_expect = 0
    for m in ms:
        s = 256 if m <= 32 else 128
        assert m * s <= 8192  # the records of Steps 4-5 fit one CTA
        b = next(b for b in range(1, m * s + 1)
                 if oracle.bucket_bound(m * 16384, m, s, b) <= 16384)
        b_expect += b
    assert p.buckets == b_expect
    # the plain sort of the 2^20 + 1 keys is counted with the batch's kernels
    assert p.num_kernels > 7
    pkg.bsort_destroy(h)
    # a low direct limit: one-sublist sampled segments, one bucket each
    h = pkg.bsort_create(pkg.bsort_config(device=0, batch_direct_max=2048))
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U64, np.array([0, 2049, 2049 + 16384], np.uint64))
    assert (p.direct_segs, p.sampled_segs, p.sublists, p.buckets) == (0, 2, 2, 2)
    pkg.bsort_destroy(h)


@pytest.mark.parametrize("n,kind", [(300000, "max"), (300000, "16"), (1 << 20, "zero"),
                                    (1 << 20, "uniform")])
def test_u64_sampled_plan_on_the_oracle(n, kind):
    """The plan the batch makes for one sampled 64-bit segment (t = 16384,
    its s and b), run through the oracle's Algorithm 1 on keys that tie:
    every bucket fits the 16384-key Step-9 unit and the result is the
    textbook sort."""
    h = pkg.bsort_create(pkg.bsort_config(device=0, batch_direct_max=2048))
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U64, np.array([0, n], np.uint64))
    pkg.bsort_destroy(h)
    m = -(-n // 16384)
    s = 256 if m <= 32 else 128
    assert p.sampled_segs == 1 and p.sublists == m
    keys = synth.keys_u64(n, synth.seed_for(5, 8, n))
    if kind == "max":
        keys[:] = np.uint64(0xFFFFFFFFFFFFFFFF)
    elif kind == "16":
        keys &= np.uint64(0xF000000000000000)
    elif kind == "zero":
        keys[:] = 0
    r = oracle.paper_sort(keys, 16384, s, "u64", b=p.buckets, threads=4)
    sizes = np.diff(r["bucket_start"].astype(np.int64))
    assert sizes.max() <= 16384
    assert sizes.max() <= oracle.bucket_bound(m * 16384, m, s, p.buckets)
    assert np.array_equal(r["keys"], oracle.textbook_sort(keys, "u64"))


def test_plan_batch_errors():
    h = _handle()
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan_batch(h, pkg.BSORT_U32, np.array([0, 10, 5], np.uint64))
    assert e.value.status == pkg.BSORT_EINVAL
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U64,
                             np.cumsum([0, 10, 131072, 131073, 600000, 1 << 21]).astype(np.uint64))
    assert (p.direct_segs, p.sampled_segs, p.large_segs) == (2, 2, 1)
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan_batch(h, pkg.BSORT_U32, np.array([0, 1 << 32], np.uint64))
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    p = pkg.bsort_plan_batch(h, pkg.BSORT_U32, np.array([0], np.uint64))
    assert p.num_segs == 0 and p.n == 0 and p.num_kernels == 0
    pkg.bsort_destroy(h)


def test_batch_sizes_generator():
    """Log-uniform sizes in [2^7, 2^20], scaled to at most 2^30 keys in all."""
    s = synth.batch_sizes(20000, synth.seed_for(4, 0))
    assert s.size == 20000 and s.min() >= 128 and s.max() <= 1 << 20
    assert s.sum() <= 1 << 30 and s.sum() > 0.99 * (1 << 30)
    small = synth.batch_sizes(100, synth.seed_for(4, 1), cap=1 << 40)
    assert small.min() >= 128 and small.max() < 1 << 20
    # the scaling keeps the order of the sizes
    raw = synth.batch_sizes(20000, synth.seed_for(4, 0), cap=1 << 40)
    assert np.all(np.diff(s[np.argsort(raw, kind="stable")]) >= 0)


def test_plan_u64_keys():
    """64-bit keys sort 64-bit words: CTAs of at most 16384 keys, units of at
    most 8 x 16384; pairs with 64-bit keys plan two passes of the 32-bit pair
    sort (that plan, with the scratch of both passes in its workspace)."""
    h = _handle()
    for n in (100, 131072, 131073, 1 << 20, (1 << 24) + 5, 1 << 28):
        p = pkg.bsort_plan(h, pkg.BSORT_U64, 0, n)
        assert p.unit_capacity <= 8 * 16384
        if p.single_tile:
            assert n <= p.unit_capacity
        else:
            assert p.t <= 8 * 16384 and p.m * p.t == p.n_padded >= n
            assert p.bucket_bound == oracle.bucket_bound(p.n_padded, p.m, p.s, p.b)
            assert p.bucket_bound <= p.unit_capacity
    q = pkg.bsort_plan(h, pkg.BSORT_U32, 4, 1 << 20)
    p = pkg.bsort_plan(h, pkg.BSORT_U64, 8, 1 << 20)
    assert (p.t, p.s, p.b) == (q.t, q.s, q.b)
    assert p.workspace_bytes >= q.workspace_bytes + (1 << 20) * (5 * 4 + 8 + 8)
    assert p.num_kernels == 2 * q.num_kernels + 3
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U64, 8, 1 << 32)
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    pkg.bsort_destroy(h)
    h = _handle(4096, 64)
    p = pkg.bsort_plan(h, pkg.BSORT_U64, 0, 1 << 20)
    assert (p.t, p.s, p.b, p.m) == (4096, 64, 64, 256)
    pkg.bsort_destroy(h)


def test_plan_two_tier_step9():
    """When the bound needs a cluster unit and bucket sizes are regular
    enough, b puts the average bucket four sigmas below a one-CTA unit and
    Step 9 runs in two tiers (unit_small; a unit per bucket, so b may reach
    32768); with s given (b = s), or when b would exceed that limit, in one
    (greedy packing: b at most 12288)."""
    h = _handle()
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 28)
    assert p.unit_ctas > 1 and p.unit_small == 32768
    # average bucket four sigmas (sigma = w sqrt(m/6)) below the one-CTA unit,
    # and those four sigmas within 10% of it
    sigma = p.w * (p.m / 6) ** 0.5
    assert 4 * sigma <= 0.10 * 32768
    assert p.b == -(-p.n_padded // int(32768 - 4 * sigma))
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 4, 1 << 25)
    assert p.unit_ctas > 1 and p.unit_small == 16384
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 22)
    assert p.unit_ctas == 1 and p.unit_small == 0
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 3 << 28)  # two tiers: up to 32768 buckets
    assert p.unit_small == 32768 and 12288 < p.b <= 32768
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 30)  # b capped: one tier
    assert p.unit_small == 0 and p.b <= 12288
    pkg.bsort_destroy(h)
    h = _handle(131072, 8192)
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 28)
    assert p.unit_small == 0 and p.b == 8192
    pkg.bsort_destroy(h)
    h = _handle(131072, 8192, 8602)  # a given b that fits: two tiers
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 28)
    assert p.unit_small == 32768 and p.b == 8602
    pkg.bsort_destroy(h)


def test_plan_invariants_sweep():
    """Over sizes from 2^17 to 3 * 2^28 and every key type: the bucket bound
    of the plan (the oracle's formula) fits the Step-9 unit, one-tier plans
    keep b within the greedy packing's 12288 buckets, two-tier plans within
    32768 with a one-CTA small unit, and b never exceeds the m*s samples."""
    h = _handle()
    sizes = [(1 << k) + d for k in range(17, 29) for d in (0, 12345)] + [3 << 28]
    for kt, vb in ((pkg.BSORT_U32, 0), (pkg.BSORT_F32, 0), (pkg.BSORT_U32, 4),
                   (pkg.BSORT_U32, 8), (pkg.BSORT_U64, 0)):
        for n in sizes:
            try:
                p = pkg.bsort_plan(h, kt, vb, n)
            except pkg.BsortError as e:  # sizes beyond what a plan can hold
                assert e.status == pkg.BSORT_EUNSUPPORTED
                continue
            if p.single_tile:
                assert n <= p.unit_capacity
                continue
            assert p.m * p.t == p.n_padded >= n > (p.m - 1) * p.t
            assert p.t % p.s == 0 and p.w == p.t // p.s
            assert 1 <= p.b <= p.m * p.s
            assert p.bucket_bound == oracle.bucket_bound(p.n_padded, p.m, p.s, p.b)
            assert p.bucket_bound <= p.unit_capacity
            if p.unit_small:
                assert p.b <= 32768 and p.unit_small < p.unit_capacity
                assert p.unit_small == (16384 if (vb or kt == pkg.BSORT_U64) else 32768)
            else:
                assert p.b <= 12288
    pkg.bsort_destroy(h)


def test_create_flags():
    """bsort_create takes the documented flags (timing, low memory, CUDA-graph
    replay, comparison sort, the stalled-scan test, the cost-model planner)
    and refuses unknown bits."""
    ok = (pkg.BSORT_FLAG_TIMING | pkg.BSORT_FLAG_LOW_MEMORY | pkg.BSORT_FLAG_GRAPHS
          | pkg.BSORT_FLAG_MERGE_SORT | pkg.BSORT_FLAG_TEST_STALL_SCAN
          | pkg.BSORT_FLAG_PLAN_MODEL | pkg.BSORT_FLAG_TEST_TWO_LEVEL)
    h = pkg.bsort_create(pkg.bsort_config(device=0, flags=ok))
    pkg.bsort_destroy(h)
    for bad in (0x80, 0x100, 0x80000000):
        with pytest.raises(pkg.BsortError) as e:
            pkg.bsort_create(pkg.bsort_config(device=0, flags=bad))
        assert e.value.status == pkg.BSORT_EINVAL


def test_tuned_plan_table_lookup():
    """Keys-only 32-bit sorts above one unit take (t, s) from the measured
    table for n's size class (b is then the planner's); BSORT_FLAG_PLAN_MODEL,
    pairs, 64-bit keys and the comparison sort use the cost model; a forced
    t/s with BSORT_BUCKETS_AUTO keeps them and lets the planner choose b."""
    import re as _re
    src = open(os.path.join(ROOT, "paper_1002_4464_gb300", "csrc", "bsort_tuned.inc")).read()
    table = [tuple(map(int, m))
             for m in _re.findall(r"^\{(\d+),\s*(\d+),\s*(\d+)\},", src, flags=_re.M)]
    assert table and all(a[0] < b[0] for a, b in zip(table, table[1:]))
    h = _handle()
    model = pkg.bsort_create(pkg.bsort_config(device=0, flags=pkg.BSORT_FLAG_PLAN_MODEL))
    for lg in (19, 20, 21, 24, 26, 28, 30):
        n = (1 << lg) + 3
        want = next(((t, s) for top, t, s in table if n <= (1 << top)), None)
        for kt in (pkg.BSORT_U32, pkg.BSORT_F32):
            p = pkg.bsort_plan(h, kt, 0, n)
            if p.single_tile:
                continue
            if want is not None:
                assert (p.t, p.s) == want, (lg, p.t, p.s)
            assert p.unit_capacity >= p.bucket_bound
            assert p.bucket_bound == oracle.bucket_bound(p.n_padded, p.m, p.s, p.b)
        q = pkg.bsort_plan(model, pkg.BSORT_U32, 0, n)
        assert q.unit_capacity >= q.bucket_bound
    pkg.bsort_destroy(model)
    pkg.bsort_destroy(h)
    h = pkg.bsort_create(pkg.bsort_config(device=0, tile=65536, samples=4096,
                                          buckets=pkg.BSORT_BUCKETS_AUTO))
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 26)
    assert (p.t, p.s) == (65536, 4096) and p.b != p.s
    pkg.bsort_destroy(h)


def test_plan_two_level():
    """Above 2^30 keys (keys-only 32-bit keys, up to 2^34) the plan has two
    levels: sublists of 32768, b buckets of about 2^28 keys whose bound (the
    oracle's formula) stays below 2^32 - 2^16, m*s samples and m*b runs
    within 32 bits; pairs and 64-bit keys stop below 2^32 - 2^16."""
    h = _handle()
    assert pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 30).levels == 1
    for n in ((1 << 30) + 1, (1 << 32) - (1 << 16), (1 << 32) + 12345, 1 << 33, 1 << 34):
        for kt in (pkg.BSORT_U32, pkg.BSORT_F32):
            p = pkg.bsort_plan(h, kt, 0, n)
            assert p.levels == 2 and p.t == 32768 and p.m * p.t == p.n_padded >= n
            assert p.bucket_bound == oracle.bucket_bound(p.n_padded, p.m, p.s, p.b)
            assert p.n_padded // p.b <= p.bucket_bound < (1 << 32) - (1 << 16)
            assert p.bucket_bound <= 1.3 * p.n_padded / p.b  # slack within a quarter
            assert p.m * p.s < 1 << 32 and p.m * p.b < 1 << 32
    for kt, vb in ((pkg.BSORT_U32, 4), (pkg.BSORT_U64, 0)):
        with pytest.raises(pkg.BsortError) as e:
            pkg.bsort_plan(h, kt, vb, 1 << 32)
        assert e.value.status == pkg.BSORT_EUNSUPPORTED
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, (1 << 34) + 1)
    assert e.value.status == pkg.BSORT_EUNSUPPORTED
    pkg.bsort_destroy(h)
    t = pkg.bsort_create(pkg.bsort_config(device=0, flags=pkg.BSORT_FLAG_TEST_TWO_LEVEL))
    p = pkg.bsort_plan(t, pkg.BSORT_U32, 0, (1 << 22) + 777)
    assert p.levels == 2 and p.b == -(-p.n_padded // (1 << 16))
    assert pkg.bsort_plan(t, pkg.BSORT_U32, 4, 1 << 22).levels == 1
    pkg.bsort_destroy(t)


def test_plan_kernel_counts():
    """Launches per sort as the plan reports them: Steps 1-3 (1), Steps 4-5
    by the record radix sort (histogram + 4 digit passes) once the sample
    set spans several chunks, else one chunk sort, Step 6 (2), Steps 7-8
    fused when m is a multiple of 4 (1; else row scan, run index and
    relocation, 3), the unit lists (1) and Step 9 (1, or 2 with two tiers)."""
    h = _handle()
    cases = [(1 << 28, 1 + 5 + 2 + 1 + 1 + 2),       # m = 8192, two tiers
             ((1 << 24) + 77, 1 + 5 + 2 + 3 + 1 + 1),  # m = 513: separate Steps 7 and 8
             (1 << 20, 1 + 1 + 2 + 1 + 1 + 1)]       # one chunk of sample records
    for n, want in cases:
        p = pkg.bsort_plan(h, pkg.BSORT_U32, 0, n)
        assert p.num_kernels == want, (n, p.num_kernels, want)
    pkg.bsort_destroy(h)
