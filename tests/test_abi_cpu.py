"""The C-ABI library builds, loads and exports every function that
include/bsort.h declares; the host-side planner (Step 1 parameters, the
Step-9 unit, the bucket bound) behaves as documented.  No GPU needed: these
calls touch no device."""
import os
import re
import subprocess

import pytest

import paper_1002_4464_gb300 as pkg

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


def _handle(tile=0, samples=0):
    return pkg.bsort_create(pkg.bsort_config(device=0, tile=tile, samples=samples))


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
        assert p.bucket_bound == p.n_padded // p.s + (p.m - 1) * (w - 1)
        assert p.bucket_bound <= 2 * p.n_padded // p.s
        assert p.unit_capacity >= p.bucket_bound
    pkg.bsort_destroy(h)


def test_plan_pairs_and_errors():
    h = _handle()
    p = pkg.bsort_plan(h, pkg.BSORT_U32, 4, 1 << 20)
    assert p.unit_capacity >= p.bucket_bound and p.t <= 16384
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 3, 100)
    assert e.value.status == pkg.BSORT_EINVAL
    with pytest.raises(pkg.BsortError) as e:
        pkg.bsort_plan(h, pkg.BSORT_U32, 0, 1 << 33)
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
