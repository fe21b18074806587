"""Planted mistakes: every plausible slip in the oracle (a wrong index, a
dropped term, a wrong sign or tie rule, a transposed operand) must fail at
least one of the pins in test_oracle_pins.py.  Each case edits one line of a
copy of oracle/bsort_oracle.c, compiles it with gcc into a temporary
directory, runs the pins against it on the CPU, and expects a failure.  The
edits keep every memory access in bounds, so a mutant can only give wrong
answers, never crash the test process.  (A merge that lets the right run win
ties is not among them: items are compared in composite order (key,
position), where no two are equal, so that edit changes nothing.)"""
import os

import pytest

import oracle

import test_oracle_pins as pins

MUTANTS = [
    # Step 3: sample ranks (k+1)w - 1 -> kw (first item of each chunk)
    ("sample rank", "uint64_t r = (k + 1) * w - 1;", "uint64_t r = k * w;"),
    # Step 5: splitter ranks floor((j+1)ms/b) - 1 -> floor(jms/b)
    ("splitter rank", "G[j] = S[(j + 1) * m * s / b - 1];", "G[j] = S[j * m * s / b];"),
    # Step 6: buckets (g_{j-1}, g_j] -> [g_{j-1}, g_j) (the splitter leaves its bucket)
    ("bucket boundary tie rule", "if (rec_less(&G[j], &item)) hi = mid;",
     "if (!rec_less(&item, &G[j])) hi = mid;"),
    # Step 6: composite position i*t + r -> r (dropped term)
    ("composite position", "item.p = i * t + mid;", "item.p = mid;"),
    # Step 1: pads get the smallest key instead of the largest
    ("pad sentinel", "A[x].key = key_max;", "A[x].key = 0;"),
    # Step 8: run copied in reverse order (wrong index)
    ("relocation order", "B[l[j * m + i] + q] = A[src + q];",
     "B[l[j * m + i] + len - 1 - q] = A[src + q];"),
    # Steps 2/9: merge comparison with its operands transposed
    ("local sort comparison", "if (elem_less(&a[y], &a[x])) tmp[o++] = a[y++];",
     "if (elem_less(&a[x], &a[y])) tmp[o++] = a[y++];"),
    # Steps 2/9: equal keys ordered by descending position (unstable)
    ("item tie-break", "    return a->pos < b->pos;", "    return a->pos > b->pos;"),
    # Step 4: sample records compared by key only (transposed tie-break)
    ("sample order tie-break", "    return a->p < b->p;\n}\n\n/* ---- top-down",
     "    return a->p > b->p;\n}\n\n/* ---- top-down"),
    # float transform: negative values not inverted (wrong sign handling)
    ("float transform", "if (bits & 0x80000000u) return ~bits;",
     "if (bits & 0x80000000u) return bits;"),
    # textbook sort: right run wins ties (unstable)
    ("textbook stability", "(y < hi && k0[y] < k0[x])", "(y < hi && k0[y] <= k0[x])"),
]

# the pins, with small parameter sets
PINS = [
    (pins.test_bruteforce_tiny, {"n": 4}),
    (pins.test_bruteforce_tiny, {"n": 5}),
    (pins.test_hand_worked_example, {}),
    (pins.test_against_textbook_and_library, {"seed": 0}),
    (pins.test_u64_and_f32_keys, {}),
    (pins.test_closed_form_equal_buckets, {"kind": "zero", "t": 64, "s": 8, "m": 16}),
    (pins.test_closed_form_equal_buckets, {"kind": "increasing", "t": 64, "s": 8, "m": 16}),
    (pins.test_bucket_bound_and_partition, {"dist": "uniform"}),
    (pins.test_bucket_bound_and_partition, {"dist": "zero"}),
    (pins.test_f32_transform_order, {}),
    (pins.test_bruteforce_tiny_decoupled_buckets, {"n": 4}),
    (pins.test_closed_form_decoupled_buckets, {"kind": "zero", "t": 64, "s": 8, "m": 16, "b": 5}),
    (pins.test_bound_and_partition_decoupled_buckets, {"dist": "uniform", "b": 40}),
]


def _failing_pins():
    failed = []
    for fn, kw in PINS:
        try:
            fn(**kw)
        except Exception as e:  # an assertion, or an oracle error status
            failed.append("%s%s: %s" % (fn.__name__, kw, type(e).__name__))
    return failed


def test_unmutated_oracle_passes_the_pins(tmp_path):
    lib = oracle.compile_to(oracle._SRC, str(tmp_path / "liboracle_copy.so"))
    with oracle.use_library(lib):
        assert _failing_pins() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, tmp_path):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_to(str(path), str(tmp_path / ("liboracle_mutant_%d.so" % os.getpid())))
    with oracle.use_library(lib):
        failed = _failing_pins()
    assert failed, "planted mistake '%s' passes every pin" % name
