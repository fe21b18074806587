"""Pins of the CPU oracle against facts that do not come from the oracle.

- brute force: on inputs of <= 6 keys, the unique stable sorted permutation
  found by enumerating every order of the indices;
- an independent textbook merge sort and Python's own stable sort;
- a hand-worked example of Algorithm 1 (tests/golden/worked_example_n12.txt);
- closed forms: all-equal and strictly monotone inputs give buckets of
  exactly n/s items (regular sampling of Steps 3-5);
- the bucket-size bound of Step 8/9 (the paper's 2n/s, and the tighter
  n'/s + (m-1)(w-1) derived from the sample positions);
- properties of the splitters (Step 5) and of the partition (Step 6) stated
  in the original-index order, which the oracle never uses directly;
- the float32 key transform against IEEE-754 ordering.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _stable_perm_bruteforce(keys):
    """Enumerate all orders of the indices; return the one that is sorted by
    key with ties in index order (it is unique)."""
    n = len(keys)
    found = None
    for perm in itertools.permutations(range(n)):
        ok = True
        for a, b in zip(perm, perm[1:]):
            if keys[a] > keys[b] or (keys[a] == keys[b] and a > b):
                ok = False
                break
        if ok:
            assert found is None, "stable sorted order must be unique"
            found = perm
    return list(found) if found is not None else []


def _plans(n):
    out = []
    for t in (1, 2, 4, 8):
        for s in (1, 2, 4):
            if s <= t and t % s == 0:
                out.append((t, s))
    return out


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6])
def test_bruteforce_tiny(n):
    inputs = [list(p) for p in itertools.permutations(range(n))]
    inputs += [list(x) for x in itertools.product(range(3), repeat=n)]
    if n == 6:
        inputs = inputs[::7]  # keep the run short; still hundreds of inputs
    for keys in inputs:
        perm = _stable_perm_bruteforce(keys)
        want_k = np.array([keys[x] for x in perm], np.uint32)
        for t, s in _plans(n):
            k = np.array(keys, np.uint32)
            v = np.arange(n, dtype=np.uint32)
            r = oracle.paper_sort(k, t, s, "u32", vals=v)
            assert (r["keys"] == want_k).all(), (keys, t, s)
            assert list(r["vals"]) == perm, (keys, t, s)


def _load_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            d[parts[0]] = [int(x) for x in parts[1:]]
    return d


def test_hand_worked_example():
    g = _load_golden("worked_example_n12.txt")
    keys = np.array(g["keys"], np.uint32)
    r = oracle.paper_sort(keys, g["t"][0], g["s"][0], "u32",
                          vals=np.arange(g["n"][0], dtype=np.uint32))
    for name in ("tile_keys", "tile_pos", "samp_keys", "samp_p", "spl_keys",
                 "spl_p", "counts", "offsets", "reloc_keys", "bucket_start"):
        assert list(r[name]) == g[name], name
    assert list(r["keys"]) == g["sorted_keys"]
    assert list(r["vals"]) == g["sorted_vals"]


DISTS_SMALL = synth.DISTRIBUTIONS


@pytest.mark.parametrize("seed", range(6))
def test_against_textbook_and_library(seed):
    rng = np.random.default_rng(seed)
    for trial in range(8):
        n = int(rng.integers(1, 3000))
        t = int(rng.choice([4, 8, 16, 64, 256]))
        s = int(rng.choice([x for x in (1, 2, 4, 8, 16, 32, 64) if x <= t]))
        dist = DISTS_SMALL[(seed + trial) % len(DISTS_SMALL)]
        keys = synth.keys_u32(dist, n, synth.seed_for(9, seed, trial))
        if trial % 3 == 0:
            keys = keys & np.uint32(0x7)  # heavy duplicates
        vals = np.arange(n, dtype=np.uint32)
        r = oracle.paper_sort(keys, t, s, "u32", vals=vals)
        tk, tv = oracle.textbook_sort(keys, "u32", vals=vals)
        order = sorted(range(n), key=lambda x: int(keys[x]))  # Timsort: stable
        assert (r["keys"] == tk).all() and (r["vals"] == tv).all()
        assert (r["keys"] == keys[order]).all()
        assert list(r["vals"]) == order


def test_u64_and_f32_keys():
    n = 2000
    k64 = synth.keys_u64(n, 77)
    k64[::5] = np.uint64(0xFFFFFFFFFFFFFFFF)
    r = oracle.paper_sort(k64, 64, 8, "u64")
    assert (r["keys"] == np.sort(k64)).all()
    f = synth.keys_f32("gaussian", n, 78)
    r = oracle.paper_sort(f, 64, 8, "f32")
    assert (r["keys"].view(np.uint32) == np.sort(f).view(np.uint32)).all()


def _bucket_sizes(r):
    return np.diff(r["bucket_start"].astype(np.int64))


@pytest.mark.parametrize("kind", ["zero", "increasing", "decreasing"])
@pytest.mark.parametrize("t,s,m", [(64, 8, 16), (256, 16, 8), (4096, 64, 4)])
def test_closed_form_equal_buckets(kind, t, s, m):
    n = t * m
    if kind == "zero":
        keys = np.zeros(n, np.uint32)
    else:
        step = (1 << 32) // n
        keys = (np.arange(n, dtype=np.uint64) * step).astype(np.uint32)
        if kind == "decreasing":
            keys = keys[::-1].copy()
    r = oracle.paper_sort(keys, t, s, "u32")
    sizes = _bucket_sizes(r)
    assert (sizes == n // s).all(), sizes


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_bucket_bound_and_partition(dist):
    t, s = 256, 16
    n = 256 * 40 + 77  # ragged: 41 sublists, last one padded
    keys = synth.keys_u32(dist, n, synth.seed_for(1, 5))
    r = oracle.paper_sort(keys, t, s, "u32")
    m, npad = r["m"], r["n_padded"]
    w = t // s
    sizes = _bucket_sizes(r)
    assert sizes.sum() == npad
    # the paper's bound (Section 4, Step 8: at most 2n/s items per B_j)
    assert sizes.max() <= 2 * npad // s
    # the tighter bound from the sample positions
    assert sizes.max() <= oracle.bucket_bound(npad, m, s)
    assert sizes[0] >= npad // s and sizes[-1] <= npad // s
    if s > 2:
        assert sizes[1:-1].min() >= m + w - 1
    # counts and offsets (Steps 6-7) agree with the bucket boundaries
    a = r["counts"].astype(np.int64).reshape(s, m)
    assert (a.sum(axis=1) == sizes).all()
    l = r["offsets"].astype(np.int64)
    assert l[0] == 0 and (l[1:] == (l + a.ravel())[:-1]).all()
    # splitters are samples, strictly increasing, and exactly (j+1)m samples
    # are <= g_j; the last one is the global maximum item
    samples = list(zip(r["samp_keys"].tolist(), r["samp_p"].tolist()))
    spl = list(zip(r["spl_keys"].tolist(), r["spl_p"].tolist()))
    sset = set(samples)
    for j, g in enumerate(spl):
        assert g in sset
        assert sum(1 for x in samples if x <= g) == (j + 1) * m
    assert all(spl[j] < spl[j + 1] for j in range(s - 1))
    assert spl[-1][1] == npad - 1 or spl[-1][0] == oracle.KEY_MAX["u32"]
    # partition: every item of B_j lies in (g_{j-1}, g_j] in (key, original
    # index) order, the splitter's original index read from the tiles
    tile_pos = r["tile_pos"]
    spl_orig = [(int(k), int(tile_pos[p])) for k, p in spl]
    rk, rp = r["reloc_keys"], r["reloc_pos"]
    bs = r["bucket_start"]
    for j in range(s):
        lo = spl_orig[j - 1] if j else None
        hi = spl_orig[j]
        for x in range(int(bs[j]), int(bs[j + 1])):
            item = (int(rk[x]), int(rp[x]))
            assert item <= hi and (lo is None or item > lo)
    # each A_ij is a contiguous run of sorted sublist i, and B_j lists them
    # in sublist order
    for j in range(s):
        pos_seq = [int(p) for p in rp[int(bs[j]):int(bs[j + 1])]]
        tiles_of = [min(p, n) // t if p < n else m - 1 for p in pos_seq]
        assert tiles_of == sorted(tiles_of)


def test_paper_worked_parameters():
    """Section 4: n = 32M items, n/m = 2K -> m = 16K sublists, s = 64,
    s*m = 1M samples, and every B_j has at most 2n/s = 1M items."""
    n, t, s = 32 * 2 ** 20, 2 * 2 ** 10, 64
    m = n // t
    assert m == 16 * 2 ** 10 and s * m == 2 ** 20
    assert 2 * n // s == 2 ** 20
    assert oracle.bucket_bound(n, m, s) <= 2 * n // s


def test_f32_transform_order():
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2 ** 32, size=200000, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000,
                         0x7FC00000, 0xFFC00000, 0x00000001, 0x80000001,
                         0x7F7FFFFF, 0xFF7FFFFF, 0x7F800001, 0xFF800001],
                        np.uint32)
    bits = np.concatenate([bits, specials])
    keys = oracle.f32_to_key(bits)
    # round trip is the identity on every bit pattern
    assert (oracle.key_to_f32(keys) == bits).all()
    f = bits.view(np.float32)
    fin = ~np.isnan(f)
    # for non-NaN values the key order is IEEE order, with -0 below +0
    order = np.argsort(keys[fin], kind="stable")
    fs = f[fin][order]
    assert (np.diff(fs.astype(np.float64)) >= 0).all()
    assert oracle.f32_to_key(np.array([0x80000000], np.uint32))[0] < \
        oracle.f32_to_key(np.array([0x00000000], np.uint32))[0]
    # NaNs with the sign bit sit below -inf, the others above +inf
    k_ninf = oracle.f32_to_key(np.array([0xFF800000], np.uint32))[0]
    k_pinf = oracle.f32_to_key(np.array([0x7F800000], np.uint32))[0]
    nb = bits[~fin]
    nk = keys[~fin]
    assert (nk[(nb >> 31) == 1] < k_ninf).all()
    assert (nk[(nb >> 31) == 0] > k_pinf).all()


def test_generator_reference_value():
    """SplitMix64 with seed 0: first output 0xE220A8397B1DCDAF (published
    test vector of the Steele-Lea-Flood generator)."""
    assert int(synth.draws64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_generators_numpy_torch_agree():
    torch = pytest.importorskip("torch")
    for d in synth.DISTRIBUTIONS:
        a = synth.keys_u32(d, 4096, synth.seed_for(2, 1))
        b = synth.keys_u32_torch(d, 4096, synth.seed_for(2, 1)).numpy().view(np.uint32)
        assert (a == b).all(), d
        fa = synth.keys_f32(d, 1024, 11)
        fb = synth.keys_f32_torch(d, 1024, 11).numpy()
        assert (fa.view(np.uint32) == fb.view(np.uint32)).all(), d


# ---- decoupled bucket count b (extension: b global samples from the m*s samples)

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_bruteforce_tiny_decoupled_buckets(n):
    inputs = [list(x) for x in itertools.product(range(3), repeat=n)]
    inputs += [list(p) for p in itertools.permutations(range(n))][:60]
    for keys in inputs:
        perm = _stable_perm_bruteforce(keys)
        for t, s in ((2, 1), (2, 2), (4, 2), (4, 4)):
            m = -(-n // t)
            for b in range(1, m * s + 1):
                r = oracle.paper_sort(np.array(keys, np.uint32), t, s, "u32",
                                      vals=np.arange(n, dtype=np.uint32), b=b)
                assert list(r["vals"]) == perm, (keys, t, s, b)


@pytest.mark.parametrize("kind", ["zero", "increasing", "decreasing"])
@pytest.mark.parametrize("t,s,m,b", [(64, 8, 16, 5), (256, 16, 8, 37), (4096, 64, 4, 100),
                                     (256, 16, 8, 128)])
def test_closed_form_decoupled_buckets(kind, t, s, m, b):
    """All-equal and strictly monotone keys: samples are every w-th item of
    the global order, so bucket j holds exactly (r_j - r_{j-1}) * w items with
    r_j = floor((j+1) m s / b) - 1."""
    n = t * m
    if kind == "zero":
        keys = np.zeros(n, np.uint32)
    else:
        keys = (np.arange(n, dtype=np.uint64) * ((1 << 32) // n)).astype(np.uint32)
        if kind == "decreasing":
            keys = keys[::-1].copy()
    r = oracle.paper_sort(keys, t, s, "u32", b=b)
    w = t // s
    ranks = [(j + 1) * m * s // b - 1 for j in range(b)]
    want = [(ranks[j] - (ranks[j - 1] if j else -1)) * w for j in range(b)]
    assert list(_bucket_sizes(r)) == want


@pytest.mark.parametrize("dist", ["uniform", "staggered", "zero", "bucket"])
@pytest.mark.parametrize("b", [3, 40, 250])
def test_bound_and_partition_decoupled_buckets(dist, b):
    t, s = 256, 16
    n = 256 * 30 + 11
    keys = synth.keys_u32(dist, n, synth.seed_for(1, 6))
    r = oracle.paper_sort(keys, t, s, "u32", b=b)
    m, npad = r["m"], r["n_padded"]
    sizes = _bucket_sizes(r)
    assert sizes.sum() == npad and len(sizes) == b
    assert sizes.max() <= oracle.bucket_bound(npad, m, s, b)
    samples = list(zip(r["samp_keys"].tolist(), r["samp_p"].tolist()))
    spl = list(zip(r["spl_keys"].tolist(), r["spl_p"].tolist()))
    for j, g in enumerate(spl):
        assert sum(1 for x in samples if x <= g) == (j + 1) * m * s // b
    tile_pos = r["tile_pos"]
    spl_orig = [(int(k), int(tile_pos[p])) for k, p in spl]
    rk, rp, bs = r["reloc_keys"], r["reloc_pos"], r["bucket_start"]
    for j in range(b):
        for x in range(int(bs[j]), int(bs[j + 1])):
            item = (int(rk[x]), int(rp[x]))
            assert item <= spl_orig[j] and (j == 0 or item > spl_orig[j - 1])
    assert (r["keys"] == np.sort(keys)).all()


@pytest.mark.parametrize("dist", ["uniform", "zero", "staggered"])
@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_oracle_is_identical(dist, threads):
    """The threaded form (Steps 2, 6, 8, 9 split into per-sublist and
    per-bucket ranges over threads, used only to time the oracle on all host
    cores) returns exactly the single-threaded result and intermediates."""
    n = 100003
    keys = synth.keys_u32(dist, n, synth.seed_for(9, 1, threads))
    vals = np.arange(n, dtype=np.uint32)
    one = oracle.paper_sort(keys, 2048, 64, "u32", vals=vals, b=97)
    many = oracle.paper_sort(keys, 2048, 64, "u32", vals=vals, b=97, threads=threads)
    assert one.keys() == many.keys()
    for name, a in one.items():
        assert np.array_equal(np.asarray(a), np.asarray(many[name])), name
