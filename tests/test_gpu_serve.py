"""GPU tests of the served stream (bsort_submit / bsort_poll): every job's
result is the sort of its keys, the same alone and in the mix; admission
respects the device budget; a serving handle refuses plain calls."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1002_4464_gb300 as pkg  # noqa: E402

NP = {"u32": np.uint32, "f32": np.float32, "u64": np.uint64}
TORCH = {"u32": torch.int32, "f32": torch.float32, "u64": torch.int64}


def _job_keys(kind, key_type, n, seed):
    if key_type == "u64":
        k = synth.keys_u64(n, seed)
        if kind == "zipf":
            k = synth.keys_zipf_u64(n, seed)
        return k
    if key_type == "f32":
        return synth.keys_f32("gaussian", n, seed)
    return synth.keys_zipf(n, seed) if kind == "zipf" else synth.keys_u32("uniform", n, seed)


def _pinned(a):
    return torch.from_numpy(a.view({4: np.int32, 8: np.int64}[a.itemsize])).pin_memory()


def _mix(count, seed, lo=10, hi=20):
    sizes = synth.batch_sizes(count, seed, lo_log2=lo, hi_log2=hi, cap=1 << 40)
    jobs = []
    for q, n in enumerate(sizes):
        kt = ("u32", "u64", "f32")[q % 3]
        kind = ("uniform", "zipf")[(q // 3) % 2]
        jobs.append((kt, _job_keys(kind, kt, int(n), synth.seed_for(5, q % 7, q))))
    return jobs


def test_served_mix_equals_alone():
    jobs = _mix(48, synth.seed_for(5, 9))
    srv = pkg.SortServer(budget_bytes=1 << 30)
    bufs, tickets = [], []
    for kt, keys in jobs:  # all submitted at once: they batch together
        h_in, h_out = _pinned(keys), _pinned(np.zeros_like(keys))
        bufs.append((h_in, h_out))
        tickets.append(srv.submit(h_in, h_out, kt))
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r.status == pkg.BSORT_OK for r in results)
    assert st["completed"] == len(jobs) and st["max_batch"] >= 2
    assert st["arena_peak_bytes"] <= st["arena_bytes"]
    alone = pkg.BucketSorter()
    for (kt, keys), (h_in, h_out), r in zip(jobs, bufs, results):
        got = h_out.numpy().view(NP[kt])
        want = oracle.textbook_sort(keys, kt)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (kt, keys.size)
        d = torch.from_numpy(keys.view({4: np.int32, 8: np.int64}[keys.itemsize])).cuda()
        o = alone.sort_keys(d, key_type=kt)
        alone.sync()
        assert np.array_equal(o.cpu().numpy().view(np.uint8), got.view(np.uint8))
        assert r.done_ns >= r.start_ns >= r.submit_ns and 1 <= r.batch_size <= len(jobs)
    alone.close()


def test_admission_by_budget():
    """512 MiB budget: a 256 MiB arena holds eight 8M-key jobs at a time;
    twenty jobs (640 MiB of keys) all finish; a job larger than the arena is
    refused."""
    srv = pkg.SortServer(budget_bytes=512 << 20)
    n = 8 << 20
    keys = [synth.keys_u32("uniform", n, synth.seed_for(5, 10, q)) for q in range(20)]
    bufs = [(_pinned(k), _pinned(np.zeros_like(k))) for k in keys]
    tickets = [srv.submit(a, b, "u32") for a, b in bufs]
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    assert all(r.status == pkg.BSORT_OK for r in results)
    assert st["arena_bytes"] == 256 << 20 and st["arena_peak_bytes"] <= st["arena_bytes"]
    assert st["completed"] == 20
    for k, (a, b) in zip(keys, bufs):
        assert np.array_equal(b.numpy().view(np.uint32), np.sort(k))
    big = _pinned(np.zeros(72 << 20, np.uint32))
    with pytest.raises(pkg.BsortError) as e:
        srv.submit(big, big, "u32")
    assert e.value.status == pkg.BSORT_ENOMEM
    srv.close()


def test_serving_handle_refuses_plain_calls_and_empty_jobs_finish():
    srv = pkg.SortServer(budget_bytes=64 << 20)
    e0 = _pinned(np.zeros(0, np.uint32))
    t = srv.submit(e0, e0, "u32")
    assert srv.wait(t).status == pkg.BSORT_OK
    d = torch.zeros(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_sort_keys(srv.h, pkg.BSORT_U32, d.data_ptr(), d.data_ptr(), 1000,
                            torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pkg.BSORT_EBUSY
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_poll(srv.h, 10 ** 9)
    assert e.value.status == pkg.BSORT_EINVAL
    srv.close()


def test_arrivals_while_sorting_form_later_batches():
    """Jobs submitted over time: each is sorted correctly, and jobs that
    arrive while a batch sorts are batched together later."""
    srv = pkg.SortServer(budget_bytes=1 << 30)
    jobs = _mix(60, synth.seed_for(5, 11), lo=14, hi=22)
    tickets, bufs = [], []
    for q, (kt, keys) in enumerate(jobs):
        a, b = _pinned(keys), _pinned(np.zeros_like(keys))
        bufs.append((a, b))
        tickets.append(srv.submit(a, b, kt))
        time.sleep(0.0005)
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["batches"] >= 2
    for (kt, keys), (a, b), r in zip(jobs, bufs, results):
        assert r.status == pkg.BSORT_OK
        want = oracle.textbook_sort(keys, kt)
        assert np.array_equal(b.numpy().view(np.uint8), want.view(np.uint8))


def test_poll_any_returns_every_job_once():
    jobs = _mix(30, synth.seed_for(5, 12))
    srv = pkg.SortServer(budget_bytes=1 << 30)
    bufs, want = {}, {}
    for kt, keys in jobs:
        a, b = _pinned(keys), _pinned(np.zeros_like(keys))
        t = srv.submit(a, b, kt)
        bufs[t] = (kt, keys, b)
    seen = {}
    deadline = time.time() + 60
    while len(seen) < len(jobs) and time.time() < deadline:
        for t, r in srv.poll_any(8):
            assert t not in seen and r.status == pkg.BSORT_OK
            seen[t] = r
        time.sleep(1e-4)
    assert set(seen) == set(bufs)
    for t, (kt, keys, b) in bufs.items():
        assert np.array_equal(b.numpy().view(np.uint8),
                              oracle.textbook_sort(keys, kt).view(np.uint8))
    assert srv.poll_any(8) == []
    srv.close()
