"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element and bit-exactly (sorting is integer work: the bar is
bit-exact for keys, values, intermediates and indices)."""
import os

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


def _to_dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _gpu_sort_keys(sorter, keys, key_type="u32"):
    d_in = _to_dev_u32(keys)
    d_out = sorter.sort_keys(d_in, key_type=key_type)
    sorter.sync()
    return d_out.cpu().numpy().view(np.uint32)


def _check_intermediates(sorter, want, n_pad, m, s, b=0):
    b = b or s
    im = pkg
    got_t = sorter.intermediate(im.BSORT_IM_TILES, n_pad * 4, np.uint32)
    assert np.array_equal(got_t, want["tile_keys"].astype(np.uint32)), "Step 2 sublists"
    got_s = sorter.intermediate(im.BSORT_IM_SAMPLES, m * s * 8, np.uint64)
    assert np.array_equal(got_s, _rec(want["samp_keys"], want["samp_p"])), "Step 3 samples"
    got_g = sorter.intermediate(im.BSORT_IM_SPLITTERS, b * 8, np.uint64)
    assert np.array_equal(got_g, _rec(want["spl_keys"], want["spl_p"])), "Step 5 splitters"
    got_a = sorter.intermediate(im.BSORT_IM_COUNTS, m * b * 4, np.uint32)
    assert np.array_equal(got_a, want["counts"].astype(np.uint32)), "Step 6 counts"
    got_l = sorter.intermediate(im.BSORT_IM_OFFSETS, m * b * 4, np.uint32)
    assert np.array_equal(got_l, want["offsets"].astype(np.uint32)), "Step 7 offsets"
    got_r = sorter.intermediate(im.BSORT_IM_RELOCATED, n_pad * 4, np.uint32)
    assert np.array_equal(got_r, want["reloc_keys"].astype(np.uint32)), "Step 8 relocation"


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_config1_all_intermediates(dist):
    """n = 2^20 uint32 keys, m = 256 sublists, s = 64 samples each."""
    n, t, s = 1 << 20, 4096, 64
    keys = synth.keys_u32(dist, n, synth.seed_for(1, synth.DISTRIBUTIONS.index(dist)))
    want = oracle.paper_sort(keys, t, s, "u32")
    sorter = pkg.BucketSorter(tile=t, samples=s)
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s)
    sorter.close()


@pytest.mark.parametrize("n,t,s,b", [
    (1 << 20, 4096, 64, 67),        # b > s, not a divisor of m*s
    (1 << 20, 4096, 64, 40),        # b < s
    (1 << 18, 4096, 64, 64 * 64),   # every sample a splitter (b = m*s)
    (50000, 4096, 64, 1),           # one bucket: Step 9 sorts everything
    (3 * 4096 + 1000, 4096, 16, 23),
    (200003, 16384, 256, 3001),
])
@pytest.mark.parametrize("dist", ["uniform", "zero", "staggered"])
def test_decoupled_buckets_intermediates(n, t, s, b, dist):
    """b splitters taken from the m*s sorted samples at ranks
    floor((j+1)ms/b) - 1 (b = s is the paper's Step 5), Steps 6-9 over b
    buckets: every intermediate equals the oracle's."""
    m = -(-n // t)
    if oracle.bucket_bound(m * t, m, s, b) > 8 * 32768:
        pytest.skip("bound beyond the largest Step-9 unit")
    keys = synth.keys_u32(dist, n, synth.seed_for(2, 11, b))
    want = oracle.paper_sort(keys, t, s, "u32", b=b)
    sorter = pkg.BucketSorter(tile=t, samples=s, buckets=b)
    p = sorter.plan(n)
    assert (p.t, p.s, p.b) == (t, s, b)
    assert p.bucket_bound == oracle.bucket_bound(m * t, m, s, b)
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s, b)
    sorter.close()
    low = pkg.BucketSorter(tile=t, samples=s, buckets=b, low_memory=True)
    assert np.array_equal(_gpu_sort_keys(low, keys), want["keys"])
    low.close()


def test_auto_buckets_intermediates():
    """The planner's own b (not s) at n = 2^22: intermediates against the
    oracle run with the same t, s and b."""
    n = 1 << 22
    keys = synth.keys_u32("gaussian", n, synth.seed_for(2, 12))
    sorter = pkg.BucketSorter()
    p = sorter.plan(n)
    assert p.b != p.s and not p.single_tile
    want = oracle.paper_sort(keys, p.t, p.s, "u32", b=p.b)
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], p.s, p.b)
    sorter.close()


@pytest.mark.parametrize("n,t,s", [
    (4097, 4096, 64),             # two sublists, the second almost all padding
    (3 * 4096 + 1000, 4096, 16),  # ragged tail
    (123457, 8192, 128),
    (200003, 16384, 256),
    (70001, 2048, 32),
])
def test_ragged_intermediates(n, t, s):
    keys = synth.keys_u32("uniform", n, synth.seed_for(2, 7, n % 97))
    keys[::3] = keys[::3] & np.uint32(0xFF)  # duplicates across sublists
    keys[-5:] = np.uint32(0xFFFFFFFF)        # real maximal keys next to the pads
    want = oracle.paper_sort(keys, t, s, "u32")
    sorter = pkg.BucketSorter(tile=t, samples=s)
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s)
    sorter.close()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 2047, 2048, 4095, 4096, 4097, 32767, 32768,
                               32769, 65536 + 5, 1 << 20, (1 << 20) + 12345, 1 << 22])
def test_auto_plan_sizes(n):
    keys = synth.keys_u32("gaussian", n, synth.seed_for(2, 1, n % 1000)) if n else \
        np.zeros(0, np.uint32)
    sorter = pkg.BucketSorter()
    got = _gpu_sort_keys(sorter, keys) if n else np.zeros(0, np.uint32)
    assert np.array_equal(got, oracle.textbook_sort(keys, "u32"))
    sorter.close()


@pytest.mark.parametrize("dist", ["uniform", "zero", "sorted", "reverse", "staggered"])
def test_f32_keys(dist):
    n = 300001
    f = synth.keys_f32(dist, n, synth.seed_for(2, 3))
    f[:16] = np.array([np.inf, -np.inf, np.nan, -0.0, 0.0, 1e-45, -1e-45, 3.4e38, -3.4e38,
                       np.float32(-np.nan), 1.0, -1.0, 0.5, -0.5, 2.0, -2.0], np.float32)
    sorter = pkg.BucketSorter()
    d_in = torch.from_numpy(f.copy()).cuda()
    d_out = sorter.sort_keys(d_in, key_type="f32")
    sorter.sync()
    got = d_out.cpu().numpy().view(np.uint32)
    want = oracle.textbook_sort(f, "f32").view(np.uint32)
    assert np.array_equal(got, want)
    sorter.close()


@pytest.mark.parametrize("kind", ["zipf", "distinct16", "uniform"])
@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
def test_pairs_stable(kind, vdtype):
    n = 400009
    seed = synth.seed_for(3, 1)
    if kind == "zipf":
        keys = synth.keys_zipf(n, seed)
    elif kind == "distinct16":
        keys = synth.keys_16distinct(n, seed)
    else:
        keys = synth.keys_u32("uniform", n, seed)
    vals = np.arange(n, dtype=vdtype)
    if vdtype == np.uint64:
        vals = vals | (np.uint64(0xABCD) << np.uint64(40))
    sorter = pkg.BucketSorter()
    tdt = torch.int32 if vdtype == np.uint32 else torch.int64
    d_k = _to_dev_u32(keys)
    d_v = torch.from_numpy(vals.view(np.int32 if vdtype == np.uint32 else np.int64)).cuda()
    ok, ov = sorter.sort_pairs(d_k, d_v)
    sorter.sync()
    wk, wv = oracle.textbook_sort(keys, "u32", vals=vals)
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), wk)
    assert np.array_equal(ov.cpu().numpy().view(vdtype), wv)
    assert tdt is not None
    sorter.close()


@pytest.mark.parametrize("b", [0, 97])
def test_pairs_intermediates_forced_plan(b):
    n, t, s = 100000, 4096, 64
    keys = synth.keys_zipf(n, synth.seed_for(3, 2))
    vals = np.arange(n, dtype=np.uint32)
    want = oracle.paper_sort(keys, t, s, "u32", vals=vals, b=b)
    sorter = pkg.BucketSorter(tile=t, samples=s, buckets=b)
    ok, ov = sorter.sort_pairs(_to_dev_u32(keys), _to_dev_u32(vals))
    sorter.sync()
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), want["keys"])
    assert np.array_equal(ov.cpu().numpy().view(np.uint32), want["vals"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s, b)
    sorter.close()


def test_in_place_and_repeat_determinism():
    n = (1 << 21) + 3
    keys = synth.keys_u32("bucket", n, synth.seed_for(2, 5))
    sorter = pkg.BucketSorter()
    d = _to_dev_u32(keys)
    sorter.sort_keys(d, out=d)
    sorter.sync()
    first = d.cpu().numpy().view(np.uint32).copy()
    assert np.array_equal(first, np.sort(keys))
    d2 = _to_dev_u32(keys)
    out = sorter.sort_keys(d2)
    sorter.sync()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), first)
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), keys)  # input untouched
    sorter.close()


def test_host_entry_point():
    n = 1 << 20
    keys = synth.keys_u32("uniform", n, synth.seed_for(2, 6))
    sorter = pkg.BucketSorter()
    h_in = torch.from_numpy(keys.view(np.int32)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    sorter.sort_keys_host(h_in, h_out)
    sorter.sync()
    assert np.array_equal(h_out.numpy().view(np.uint32), np.sort(keys))
    sorter.close()


def _host_pair(a):
    h_in = torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    return h_in, torch.empty_like(h_in).pin_memory()


def test_host_entry_overlapped_intermediates():
    """The host entry's copies overlap Steps 1-3 (chunks of sublists) and
    Step 9 (groups of units by position): the sublists, samples, splitters,
    counts, offsets and relocated array are still the paper's (n = 2^23,
    t = 4096, s = 64: m = 2048 sublists in 4 chunks)."""
    n, t, s = 1 << 23, 4096, 64
    keys = synth.keys_u32("bucket", n, synth.seed_for(1, 7, 3))
    want = oracle.paper_sort(keys, t, s, "u32")
    sorter = pkg.BucketSorter(tile=t, samples=s)
    h_in, h_out = _host_pair(keys)
    sorter.sort_keys_host(h_in, h_out)
    sorter.sync()
    assert np.array_equal(h_out.numpy().view(np.uint32), want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s)
    sorter.close()


@pytest.mark.parametrize("n,dist,kt", [
    ((1 << 24) + 77, "uniform", "u32"),
    ((1 << 25) + 3, "zipf", "u32"),
    ((1 << 26) - 5, "zero", "u32"),
    ((1 << 23) + 5, "gaussian", "f32"),
    (300_001, "sorted", "u32"),
    ((1 << 22) + 5, "gaussian", "f32"),
])
def test_host_entry_overlapped(n, dist, kt):
    """Host entry with copies overlapped (from 2^23 keys: 4, 8 and 16 chunks;
    ragged sizes; one and two Step-9 tiers; float keys) and not (smaller n):
    the output equals the textbook sort bit for bit."""
    seed = synth.seed_for(2, 7, n & 0xFF)
    if kt == "f32":
        keys = synth.keys_f32(dist, n, seed)
        want = oracle.textbook_sort(keys, "f32").view(np.uint32)
    elif dist == "zipf":
        keys = synth.keys_zipf(n, seed)
        want = np.sort(keys)
    else:
        keys = synth.keys_u32(dist, n, seed)
        want = np.sort(keys)
    sorter = pkg.BucketSorter()
    h_in, h_out = _host_pair(keys)
    sorter.sort_keys_host(h_in, h_out, key_type=kt)
    sorter.sync()
    assert np.array_equal(h_out.numpy().view(np.uint32), want)
    assert np.array_equal(h_in.numpy().view(np.uint32), np.asarray(keys).view(np.uint32))
    sorter.close()


def test_host_entry_back_to_back_and_pageable():
    """Two overlapped host sorts issued without a wait between them (the
    second reuses the staging buffer and the copy events), then one from
    pageable host memory, and one with BSORT_FLAG_LOW_MEMORY (no overlap)."""
    n = (1 << 23) + 9
    a = synth.keys_u32("uniform", n, synth.seed_for(2, 8))
    b = synth.keys_u32("reverse", n, synth.seed_for(2, 9))
    sorter = pkg.BucketSorter()
    ha, oa = _host_pair(a)
    hb, ob = _host_pair(b)
    sorter.sort_keys_host(ha, oa)
    sorter.sort_keys_host(hb, ob)
    sorter.sync()
    assert np.array_equal(oa.numpy().view(np.uint32), np.sort(a))
    assert np.array_equal(ob.numpy().view(np.uint32), np.sort(b))
    pa = torch.from_numpy(a.view(np.int32).copy())
    po = torch.empty_like(pa)
    sorter.sort_keys_host(pa, po)
    sorter.sync()
    assert np.array_equal(po.numpy().view(np.uint32), np.sort(a))
    sorter.close()
    low = pkg.BucketSorter(low_memory=True)
    lo = torch.empty_like(pa)
    low.sort_keys_host(pa, lo)
    low.sync()
    assert np.array_equal(lo.numpy().view(np.uint32), np.sort(a))
    low.close()


def test_graph_replay():
    """BSORT_FLAG_GRAPHS: the first call with given buffers is captured as a
    CUDA graph and later calls replay it.  New contents in the same buffers
    sort correctly on every replay, a new size captures again, and key-value
    pairs stay stable."""
    side = torch.cuda.Stream()  # the legacy default stream cannot be captured
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _graph_replay_cases()
    torch.cuda.synchronize()


def _graph_replay_cases():
    sorter = pkg.BucketSorter(graphs=True)
    for n in ((1 << 20) + 3, 1 << 22):
        d_in = torch.empty(n, dtype=torch.int32, device="cuda")
        d_out = torch.empty_like(d_in)
        for rep in range(3):
            keys = synth.keys_u32("uniform", n, synth.seed_for(2, 10, rep))
            d_in.copy_(torch.from_numpy(keys.view(np.int32)))
            sorter.sort_keys(d_in, out=d_out)
            sorter.sync()
            assert np.array_equal(d_out.cpu().numpy().view(np.uint32), np.sort(keys))
    n = (1 << 21) + 5
    kk = torch.empty(n, dtype=torch.int32, device="cuda")
    vv = torch.arange(n, dtype=torch.int32, device="cuda")
    ok = torch.empty_like(kk)
    ov = torch.empty_like(vv)
    for rep in range(2):
        keys = synth.keys_zipf(n, synth.seed_for(2, 11, rep))
        kk.copy_(torch.from_numpy(keys.view(np.int32)))
        sorter.sort_pairs(kk, vv, out_keys=ok, out_vals=ov)
        sorter.sync()
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(ok.cpu().numpy().view(np.uint32), keys[order])
        assert np.array_equal(ov.cpu().numpy(), order.astype(np.int32))
    sorter.close()


def test_workspace_too_small_is_enomem():
    cfg = pkg.bsort_config(device=0)
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    cfg.workspace = ws.data_ptr()
    cfg.workspace_bytes = 4096
    h = pkg.bsort_create(cfg)
    d = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_sort_keys(h, pkg.BSORT_U32, d.data_ptr(), d.data_ptr(), 1 << 20, None)
    assert e.value.status == pkg.BSORT_ENOMEM
    pkg.bsort_destroy(h)


def test_bucket_bound_holds_on_device():
    """Every bucket B_j built on the GPU obeys |B_j| <= n'/s + (m-1)(w-1)."""
    for dist in synth.DISTRIBUTIONS:
        n = 1 << 20
        keys = synth.keys_u32(dist, n, synth.seed_for(2, 9))
        sorter = pkg.BucketSorter(tile=4096, samples=64)
        _gpu_sort_keys(sorter, keys)
        p = sorter.plan(n)
        l = sorter.intermediate(pkg.BSORT_IM_OFFSETS, p.m * p.s * 4, np.uint32).astype(np.int64)
        starts = np.append(l.reshape(p.s, p.m)[:, 0], p.n_padded)
        assert np.diff(starts).max() <= p.bucket_bound <= 2 * p.n_padded // p.s
        sorter.close()


@pytest.mark.parametrize("n,t,s", [
    (1 << 22, 65536, 2048),         # sublists sorted by 2-CTA clusters
    ((1 << 22) + 999, 131072, 1024),  # 4-CTA clusters, ragged tail, 2-CTA units
    (1 << 23, 262144, 1024),        # 8-CTA clusters, 4-CTA units
    (3 << 20, 32768, 256),          # single-CTA sublists, 8-CTA units
])
def test_cluster_plans_intermediates(n, t, s):
    keys = synth.keys_u32("staggered", n, synth.seed_for(2, 6, t))
    keys[::7] = keys[::7] & np.uint32(0xFFF)
    want = oracle.paper_sort(keys, t, s, "u32")
    sorter = pkg.BucketSorter(tile=t, samples=s)
    p = sorter.plan(n)
    assert p.tile_ctas * (32768 if p.tile_ctas > 1 else p.t) == p.t
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s)
    sorter.close()


@pytest.mark.parametrize("n,t,s", [(1 << 21, 65536, 1024), ((1 << 21) + 77, 131072, 2048)])
def test_cluster_plans_pairs(n, t, s):
    keys = synth.keys_zipf(n, synth.seed_for(3, 4))
    vals = np.arange(n, dtype=np.uint32)
    want = oracle.paper_sort(keys, t, s, "u32", vals=vals)
    sorter = pkg.BucketSorter(tile=t, samples=s)
    ok, ov = sorter.sort_pairs(_to_dev_u32(keys), _to_dev_u32(vals))
    sorter.sync()
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), want["keys"])
    assert np.array_equal(ov.cpu().numpy().view(np.uint32), want["vals"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], s)
    sorter.close()


@pytest.mark.parametrize("n", [40000, 100000, 262144])
def test_single_cluster_unit(n):
    """n above one CTA's chunk but within one cluster: one unit, no sampling."""
    keys = synth.keys_u32("reverse", n, synth.seed_for(2, 8))
    sorter = pkg.BucketSorter()
    assert sorter.plan(n).single_tile == 1
    got = _gpu_sort_keys(sorter, keys)
    assert np.array_equal(got, np.sort(keys))
    vals = np.arange(n, dtype=np.uint64)
    ok, ov = sorter.sort_pairs(_to_dev_u32(keys & np.uint32(0xFF)),
                               torch.from_numpy(vals.view(np.int64)).cuda())
    sorter.sync()
    wk, wv = oracle.textbook_sort(keys & np.uint32(0xFF), "u32", vals=vals)
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), wk)
    assert np.array_equal(ov.cpu().numpy().view(np.uint64), wv)
    sorter.close()


@pytest.mark.parametrize("n,kt", [(1 << 26, "u32"), ((1 << 25) + 3, "f32")])
def test_large_auto_plans(n, kt):
    """Large planner-chosen plans (clusters in Steps 2 and 9); the result is
    compared with an independent library sort (numpy) of the same keys."""
    if kt == "u32":
        keys = synth.keys_u32("uniform", n, synth.seed_for(2, 0, 1))
        got = _gpu_sort_keys(pkg.BucketSorter(), keys)
        assert np.array_equal(got, np.sort(keys))
    else:
        f = synth.keys_f32("gaussian", n, synth.seed_for(2, 1, 1))
        sorter = pkg.BucketSorter()
        d = torch.from_numpy(f).cuda()
        out = sorter.sort_keys(d, key_type="f32")
        sorter.sync()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), np.sort(f).view(np.uint32))


def _u32_as_i64(t):
    return t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF


@pytest.mark.parametrize("dist", ["uniform", "staggered"])
def test_full_size_2e28_u32(dist):
    """The benchmark workload itself (2^28 uint32 keys, planner's plan): the
    output equals an independent library sort (torch.sort) of the same keys,
    element by element."""
    n = 1 << 28
    keys = synth.keys_u32_torch(dist, n, synth.seed_for(2, synth.DISTRIBUTIONS.index(dist)),
                                device="cuda")
    sorter = pkg.BucketSorter()
    out = sorter.sort_keys(keys)
    sorter.sync()
    want = torch.sort(_u32_as_i64(keys)).values
    assert torch.equal(_u32_as_i64(out), want)
    sorter.close()


@pytest.mark.parametrize("kind", ["zipf", "distinct16"])
def test_full_size_2e27_pairs(kind):
    """Key-value pairs at 2^27 (value = original index): keys equal an
    independent sort, values are a permutation, and equal keys keep their
    input order (stability), checked on every element."""
    n = 1 << 27
    seed = synth.seed_for(3, 0 if kind == "zipf" else 1)
    k_np = synth.keys_zipf(n, seed) if kind == "zipf" else synth.keys_16distinct(n, seed)
    keys = torch.from_numpy(k_np.view(np.int32)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    sorter = pkg.BucketSorter()
    ok, ov = sorter.sort_pairs(keys, vals)
    sorter.sync()
    ok64, ov64 = _u32_as_i64(ok), ov.to(torch.int64)
    assert torch.equal(ok64, torch.sort(_u32_as_i64(keys)).values)
    # stable: (key, value) strictly increasing lexicographically
    same = ok64[1:] == ok64[:-1]
    assert bool((ov64[1:][same] > ov64[:-1][same]).all())
    assert torch.equal(torch.sort(ov64).values, torch.arange(n, device="cuda"))
    # every value points at an input item with the sorted key
    assert torch.equal(_u32_as_i64(keys)[ov64], ok64)
    sorter.close()


@pytest.mark.parametrize("n,t,s,kind", [
    ((1 << 22) + 5, 65536, 2048, "keys"),
    (1 << 21, 131072, 1024, "pairs"),
    ((1 << 20) + 333, 4096, 64, "pairs"),
])
def test_low_memory_equals_materialised(n, t, s, kind):
    """Step 9 gathering its units straight from the runs A_ij (low-memory
    mode) gives the same result as reading the materialised relocated array."""
    keys = synth.keys_zipf(n, synth.seed_for(3, 7, t))
    outs = []
    for low in (True, False):
        sorter = pkg.BucketSorter(tile=t, samples=s, low_memory=low)
        if kind == "keys":
            outs.append(_gpu_sort_keys(sorter, keys))
        else:
            vals = np.arange(n, dtype=np.uint32)
            ok, ov = sorter.sort_pairs(_to_dev_u32(keys), _to_dev_u32(vals))
            sorter.sync()
            outs.append((ok.cpu().numpy().view(np.uint32), ov.cpu().numpy().view(np.uint32)))
        sorter.close()
    if kind == "keys":
        assert np.array_equal(outs[0], outs[1])
        assert np.array_equal(outs[0], np.sort(keys))
    else:
        wk, wv = oracle.textbook_sort(keys, "u32", vals=np.arange(n, dtype=np.uint32))
        for ok, ov in outs:
            assert np.array_equal(ok, wk) and np.array_equal(ov, wv)


def _check_intermediates_u64(sorter, want, n_pad, m, s, b):
    """Intermediates of a 64-bit-key sort: 8-byte sublist items, 16-byte
    (key, p) sample and splitter records."""
    im = pkg
    got_t = sorter.intermediate(im.BSORT_IM_TILES, n_pad * 8, np.uint64)
    assert np.array_equal(got_t, want["tile_keys"].astype(np.uint64)), "Step 2 sublists"
    got_s = sorter.intermediate(im.BSORT_IM_SAMPLES, m * s * 16, np.uint64).reshape(-1, 2)
    assert np.array_equal(got_s[:, 0], want["samp_keys"].astype(np.uint64)), "Step 3 keys"
    assert np.array_equal(got_s[:, 1], want["samp_p"].astype(np.uint64)), "Step 3 positions"
    got_g = sorter.intermediate(im.BSORT_IM_SPLITTERS, b * 16, np.uint64).reshape(-1, 2)
    assert np.array_equal(got_g[:, 0], want["spl_keys"].astype(np.uint64)), "Step 5 keys"
    assert np.array_equal(got_g[:, 1], want["spl_p"].astype(np.uint64)), "Step 5 positions"
    got_a = sorter.intermediate(im.BSORT_IM_COUNTS, m * b * 4, np.uint32)
    assert np.array_equal(got_a, want["counts"].astype(np.uint32)), "Step 6 counts"
    got_l = sorter.intermediate(im.BSORT_IM_OFFSETS, m * b * 4, np.uint32)
    assert np.array_equal(got_l, want["offsets"].astype(np.uint32)), "Step 7 offsets"
    got_r = sorter.intermediate(im.BSORT_IM_RELOCATED, n_pad * 8, np.uint64)
    assert np.array_equal(got_r, want["reloc_keys"].astype(np.uint64)), "Step 8 relocation"


def _keys_u64(kind, n, seed):
    k = synth.keys_u64(n, seed)
    if kind == "dup":     # few distinct values, equal high words
        k = (k & np.uint64(0xF)) | (np.uint64(0xDEADBEEF) << np.uint64(32))
    elif kind == "zero":
        k = np.zeros(n, np.uint64)
    elif kind == "low":   # differ only in the low 32 bits
        k = k & np.uint64(0xFFFFFFFF)
    return k


def _gpu_sort_u64(sorter, keys):
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = sorter.sort_keys(d_in, key_type="u64")
    sorter.sync()
    return d_out.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("n,t,s,b", [
    (1 << 20, 4096, 64, 0),          # config 1's shape with 64-bit keys
    (123457, 8192, 128, 0),          # ragged tail
    (300001, 32768, 512, 700),       # 2-CTA cluster sublists, b > s
    (500000, 131072, 2048, 1500),    # 8-CTA cluster sublists, b < s
    ((1 << 24) + 3, 65536, 4096, 1160),  # 4-CTA sublists, two-tier Step 9 (the 2^28 plan's shape)
])
@pytest.mark.parametrize("kind", ["uniform", "dup", "zero", "low"])
def test_u64_intermediates(n, t, s, b, kind):
    keys = _keys_u64(kind, n, synth.seed_for(5, 1, n % 1000))
    want = oracle.paper_sort(keys, t, s, "u64", b=b,
                             threads=min(8, os.cpu_count() or 1) if n > (1 << 22) else 1)
    sorter = pkg.BucketSorter(tile=t, samples=s, buckets=b)
    p = sorter.plan(n, "u64")
    assert (p.t, p.s, p.b) == (t, s, b or s)
    got = _gpu_sort_u64(sorter, keys)
    assert np.array_equal(got, want["keys"])
    _check_intermediates_u64(sorter, want, want["n_padded"], want["m"], s, b or s)
    sorter.close()


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2049, 16385, 131072, 131073, 1 << 22,
                               (1 << 24) + 3])
def test_u64_auto_sizes(n):
    keys = _keys_u64("uniform", n, synth.seed_for(5, 2, n % 1000))
    sorter = pkg.BucketSorter()
    got = _gpu_sort_u64(sorter, keys) if n else np.zeros(0, np.uint64)
    assert np.array_equal(got, np.sort(keys))
    sorter.close()


def test_u64_full_size_2e27():
    """2^27 64-bit keys (1 GiB) against the library sort."""
    n = 1 << 27
    keys = synth.keys_u64(n, synth.seed_for(5, 3))
    sorter = pkg.BucketSorter()
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = sorter.sort_keys(d_in, key_type="u64")
    sorter.sync()
    # signed view: flip the top bit so that torch's int64 order is uint64 order
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    want = torch.sort(d_in ^ flip).values ^ flip
    assert torch.equal(d_out, want)
    sorter.close()


def test_u64_full_size_2e28():
    """2^28 64-bit keys (2 GiB) with the planner's plan (t = 65536, two-tier
    Step 9) against the library sort."""
    n = 1 << 28
    keys = synth.keys_u64(n, synth.seed_for(5, 4))
    sorter = pkg.BucketSorter()
    p = sorter.plan(n, "u64")
    assert p.unit_small == 16384
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = sorter.sort_keys(d_in, key_type="u64")
    sorter.sync()
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    want = torch.sort(d_in ^ flip).values ^ flip
    assert torch.equal(d_out, want)
    sorter.close()


def test_u64_host_entry():
    n = (1 << 21) + 9
    keys = synth.keys_u64(n, synth.seed_for(5, 5))
    sorter = pkg.BucketSorter()
    h_in = torch.from_numpy(keys.view(np.int64)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    sorter.sort_keys_host(h_in, h_out, key_type="u64")
    sorter.sync()
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy().view(np.uint64), np.sort(keys))
    sorter.close()


def test_two_tier_step9_pairs_intermediates():
    """The planner's own two-tier plan (buckets up to one CTA's 16384 words
    sorted by one CTA, larger ones by a cluster unit): 2^25 + 3 Zipf pairs,
    every intermediate and the stable result against the oracle."""
    n = (1 << 25) + 3
    keys = synth.keys_zipf(n, synth.seed_for(3, 9))
    vals = np.arange(n, dtype=np.uint32)
    sorter = pkg.BucketSorter()
    p = sorter.plan(n, "u32", 4)
    assert p.unit_small == 16384 and p.unit_ctas > 1
    want = oracle.paper_sort(keys, p.t, p.s, "u32", vals=vals, b=p.b)
    ok, ov = sorter.sort_pairs(_to_dev_u32(keys), _to_dev_u32(vals))
    sorter.sync()
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), want["keys"])
    assert np.array_equal(ov.cpu().numpy().view(np.uint32), want["vals"])
    _check_intermediates(sorter, want, want["n_padded"], want["m"], p.s, p.b)
    sorter.close()


def test_scan_lookback_timeout_is_reported():
    """Step 7's look-back waits are bounded: with its first chunk made never
    to publish a prefix (BSORT_FLAG_TEST_STALL_SCAN: a flag that nothing
    sets), the later chunks give up after a few thousand polls, the kernel
    returns, and bsort_sync reports BSORT_ETIMEOUT; nothing hangs, and the
    device then sorts correctly again."""
    import time
    n, t, s = 1 << 20, 4096, 64  # m*s = 16384 runs: four scan chunks
    keys = synth.keys_u32("uniform", n, synth.seed_for(2, 13))
    stalled = pkg.BucketSorter(tile=t, samples=s, flags=pkg.BSORT_FLAG_TEST_STALL_SCAN)
    d_in = _to_dev_u32(keys)
    t0 = time.perf_counter()
    stalled.sort_keys(d_in)
    with pytest.raises(pkg.BsortError) as e:
        stalled.sync()
    assert e.value.status == pkg.BSORT_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    stalled.sync()  # the error word was read and cleared
    stalled.close()
    sorter = pkg.BucketSorter(tile=t, samples=s)
    assert np.array_equal(_gpu_sort_keys(sorter, keys), oracle.textbook_sort(keys, "u32"))
    sorter.close()


@pytest.mark.parametrize("n,dist,kt", [
    ((1 << 22) + 777, "uniform", "u32"),
    ((1 << 21) + 5, "zero", "u32"),
    ((1 << 21) + 3, "staggered", "u32"),
    ((1 << 21) + 99, "gaussian", "f32"),
])
def test_two_level_forced_intermediates(n, dist, kt):
    """The two-level plan of n >= 2^32 keys, forced at small n with
    top-level buckets of about 2^16 keys (BSORT_FLAG_TEST_TWO_LEVEL): the
    top level's sorted sublists, samples, splitters, counts, 64-bit offsets
    and relocated array equal the oracle's Algorithm 1 with the same t, s, b,
    and the result (every bucket sorted by a plan of its own) equals it."""
    seed = synth.seed_for(8, synth.DISTRIBUTIONS.index(dist), n & 0xFF)
    keys = synth.keys_f32(dist, n, seed) if kt == "f32" else synth.keys_u32(dist, n, seed)
    sorter = pkg.BucketSorter(flags=pkg.BSORT_FLAG_TEST_TWO_LEVEL)
    p = sorter.plan(n, kt)
    assert p.levels == 2 and p.b > 8
    want = oracle.paper_sort(keys, p.t, p.s, kt, b=p.b)
    d_in = torch.from_numpy(np.ascontiguousarray(keys).view(np.int32)).cuda()
    out = sorter.sort_keys(d_in, key_type=kt)
    sorter.sync()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, np.asarray(want["keys"]).view(np.uint32))
    _check_intermediates(sorter, want, want["n_padded"], want["m"], p.s, p.b)
    sorter.close()


def test_two_level_above_2e32():
    """n = 2^32 + 12345 uint32 keys (a two-level plan: 64-bit offsets, 17
    buckets of about 2^28 keys): the output is nondecreasing, has the input's
    multiset (histograms of the high and low 16 bits, wrapping sums of the
    keys and of their squares), and its key at sampled ranks r is the r-th
    smallest input key (fewer than r+1 input keys below it, more than r at
    or below it), all counted on the device in chunks."""
    n = (1 << 32) + 12345
    free, total = torch.cuda.mem_get_info()
    if free < 80 * 2 ** 30:
        pytest.skip("needs about 80 GB of device memory")
    sorter = pkg.BucketSorter()
    p = sorter.plan(n)
    assert p.levels == 2
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    chunk = 1 << 28
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        keys[c0:c1] = synth.keys_u32_torch("uniform", c1 - c0, synth.seed_for(8, 0, c0 // chunk),
                                           device="cuda")
    out = sorter.sort_keys(keys)
    sorter.sync()

    def u64(t):
        return t.to(torch.int64) & 0xFFFFFFFF

    hist_in = torch.zeros(2, 65536, dtype=torch.int64, device="cuda")
    hist_out = torch.zeros_like(hist_in)
    sums_in = torch.zeros(2, dtype=torch.int64, device="cuda")
    sums_out = torch.zeros_like(sums_in)
    prev = None
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        a, o = u64(keys[c0:c1]), u64(out[c0:c1])
        assert bool((o[1:] >= o[:-1]).all()), "not sorted in chunk %d" % (c0 // chunk)
        if prev is not None:
            assert int(o[0]) >= prev
        prev = int(o[-1])
        for src, hist, sums in ((a, hist_in, sums_in), (o, hist_out, sums_out)):
            hist[0] += torch.bincount(src >> 16, minlength=65536)
            hist[1] += torch.bincount(src & 0xFFFF, minlength=65536)
            sums[0] += src.sum()
            sums[1] += (src * src).sum()
        del a, o
    assert torch.equal(hist_in, hist_out) and torch.equal(sums_in, sums_out)
    gen = np.random.default_rng(12345)
    for r in [0, n - 1] + gen.integers(0, n, 6).tolist():
        v = int(u64(out[r:r + 1]))
        less = le = 0
        for c0 in range(0, n, chunk):
            a = u64(keys[c0:min(n, c0 + chunk)])
            less += int((a < v).sum())
            le += int((a <= v).sum())
        assert less <= r < le, (r, v, less, le)
    sorter.close()


@pytest.mark.parametrize("kind", ["uniform", "few", "low_only", "high_only"])
@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
def test_u64_pairs_stable(kind, vdtype):
    """Key-value pairs with 64-bit keys (two stable passes of the 32-bit pair
    sort, low key half first): keys and values equal the oracle's stable
    textbook sort, on keys with many duplicates and on keys that differ only
    in one half."""
    n = 300007
    u = synth.keys_u64(n, synth.seed_for(3, 7, ["uniform", "few", "low_only", "high_only"].index(kind)))
    if kind == "few":
        u = u & np.uint64(0xF00000000000000F)
    elif kind == "low_only":
        u = (u & np.uint64(0xFFFF)) | np.uint64(0xABCD000000000000)
    elif kind == "high_only":
        u = u & np.uint64(0xFFFF000000000000)
    vals = np.arange(n, dtype=vdtype) * vdtype(3)
    sorter = pkg.BucketSorter()
    d_k = torch.from_numpy(u.view(np.int64)).cuda()
    d_v = torch.from_numpy(vals.view(np.int32 if vdtype == np.uint32 else np.int64)).cuda()
    ok, ov = sorter.sort_pairs(d_k, d_v, key_type="u64")
    sorter.sync()
    wk, wv = oracle.textbook_sort(u, "u64", vals=vals)
    assert np.array_equal(ok.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(ov.cpu().numpy().view(vdtype), wv)
    # in place, and the keys and values untouched when not in place
    assert np.array_equal(d_k.cpu().numpy().view(np.uint64), u)
    sorter.sort_pairs(d_k, d_v, out_keys=d_k, out_vals=d_v, key_type="u64")
    sorter.sync()
    assert np.array_equal(d_k.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(d_v.cpu().numpy().view(vdtype), wv)
    sorter.close()


def test_u64_pairs_large():
    n = (1 << 24) + 3
    u = synth.keys_u64(n, synth.seed_for(3, 8))
    u[::5] = u[::5] & np.uint64(0xFFFFFFFF00000000)
    vals = np.arange(n, dtype=np.uint32)
    sorter = pkg.BucketSorter()
    ok, ov = sorter.sort_pairs(torch.from_numpy(u.view(np.int64)).cuda(),
                               torch.from_numpy(vals.view(np.int32)).cuda(), key_type="u64")
    sorter.sync()
    wk, wv = oracle.textbook_sort(u, "u64", vals=vals)
    assert np.array_equal(ok.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(ov.cpu().numpy().view(np.uint32), wv)
    sorter.close()
