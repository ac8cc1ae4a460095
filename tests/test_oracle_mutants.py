"""Strength of the oracle's pins: copies of oracle.c with one plausible
mistake planted each (a swapped key word, a dropped term, an off-by-one,
a reversed comparison, a lost element, a wrong shift, signed bytes, ...)
are compiled into a temporary directory and loaded in a child process, and
the pins of test_oracle.py must fail against every one of them (a crash
counts as caught).  The mistakes live only in those temporary copies.  One
mutant -- a comparison of record keys on 9 bytes -- survived the record pin
as first written, which is why that pin now plants records equal in bytes
0..8; another -- a u32 radix key read as 8 bytes -- is why a pin takes
digits above bit 31.  Mistakes in the choice of splitters (an unsorted
sample, other sample positions) are not planted: a samplesort's result does
not depend on its splitters, only its recursion shape does, and the
deduplication step keeps any kept splitters strictly increasing.  CPU only.
"""
import ctypes
import os
import subprocess

import pytest
import torch.multiprocessing as mp

import oracle
import test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text in oracle.c, replacement, pins that must catch it)
MUTANTS = [
    ("quartet words compared c, b, a", "for (int w = 0; w < 3; w++) {",
     "for (int w = 2; w >= 0; w--) {",
     [lambda: pins.test_quartet_matches_numpy_lexsort("lexdup"),
      pins.test_quartet_word_order_by_hand]),
    ("equality class off by one", "cls[e] = (uint32_t)(2 * i + 1 - (uint64_t)key_less",
     "cls[e] = (uint32_t)(2 * i + 2 - (uint64_t)key_less",
     [lambda: pins.test_classify_equality_buckets_semantics(7), pins.test_classify_bruteforce_tiny]),
    ("search ignores the last padded splitter", "uint64_t lo = 0, hi = K - 1;",
     "uint64_t lo = 0, hi = K - 1 - (K > 2);",
     [lambda: pins.test_classify_no_equality_is_searchsorted(7), pins.test_classify_bruteforce_tiny]),
    ("f64 negatives not complemented", "return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);",
     "return (b >> 63) ? b : (b | 0x8000000000000000ULL);",
     [lambda: pins.test_sort_f64_matches_numpy("normal"),
      pins.test_f64_order_is_ieee754_total_order]),
    ("record key of 9 bytes", "return memcmp(a, b, 10) < 0;", "return memcmp(a, b, 9) < 0;",
     [lambda: pins.test_rec100_lexicographic_unsigned_bytes("uniform")]),
    ("record bytes compared as signed chars", "return memcmp(a, b, 10) < 0;",
     "{ for (int q = 0; q < 10; q++) if (a[q] != b[q]) return (signed char)a[q] < "
     "(signed char)b[q]; return 0; }",
     [lambda: pins.test_rec100_lexicographic_unsigned_bytes("uniform")]),
    ("distribution loses element 0", "for (uint64_t e = 0; e < n; e++) bucket_begin[cls[e] + 1]++;",
     "for (uint64_t e = 1; e < n; e++) bucket_begin[cls[e] + 1]++;",
     [lambda: pins.test_partition_level_boundaries_and_multisets(False),
      lambda: pins.test_sort_matches_numpy_every_distribution("uniform", "u64")]),
    ("insertion sort descending", "while (j > 0 && key_less(c->dt, c->swap, a + (j - 1) * D)) {",
     "while (j > 0 && key_less(c->dt, a + (j - 1) * D, c->swap)) {",
     [pins.test_bruteforce_insertion_sort_all_short_sequences]),
    ("bucket above every splitter not recursed", "if (eq && (j & 1) && j + 1 < B) continue;",
     "if (eq && (j & 1)) continue;",
     [lambda: pins.test_sort_matches_numpy_every_distribution("twodup", "u64"),
      lambda: pins.test_rootdup_closed_form(1 << 14)]),
    ("radix digit one bit too low", "cls[e] = (uint32_t)((shift >= 64 ? 0 : (k >> shift)) & mask);",
     "cls[e] = (uint32_t)((shift >= 63 ? 0 : (k >> (shift + 1))) & mask);",
     [lambda: pins.test_radix_classify_against_numpy("u64", 24, 8)]),
    ("base case when the parent is small, not the task", "if (n <= 2ULL * c->n0 || parent_n <= (uint64_t)c->k * c->n0) {",
     "if (n <= 2ULL * c->n0 && parent_n <= (uint64_t)c->k * c->n0) {",
     # still sorts correctly (only the recursion shape changes) unless the
     # partitioning path is exercised with tiny tasks: the brute force does
     [pins.test_bruteforce_all_short_sequences_partitioning_path]),
    ("pair ordered by its value word",
     "    case DT_U64:\n    case DT_PAIR:\n        return load_u64(a) < load_u64(b);",
     "    case DT_U64:\n        return load_u64(a) < load_u64(b);\n"
     "    case DT_PAIR:\n        return load_u64(a + 8) < load_u64(b + 8);",
     [pins.test_pair_keys_sorted_and_records_kept]),
    ("quartet third key word ignored", "for (int w = 0; w < 3; w++) {",
     "for (int w = 0; w < 2; w++) {",
     [pins.test_quartet_bruteforce_all_short_sequences, pins.test_quartet_word_order_by_hand]),
    ("f64 positives without the sign bit", "return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);",
     "return (b >> 63) ? ~b : b;",
     [lambda: pins.test_sort_f64_matches_numpy("normal"),
      pins.test_f64_order_is_ieee754_total_order]),
    ("u32 radix key read as 8 bytes",
     "    if (dt == DT_U32) {\n        uint32_t x;\n        memcpy(&x, a, 4);\n        return x;\n"
     "    }\n    return load_u64(a);",
     "    return load_u64(a);",
     [lambda: pins.test_radix_u32_digits_above_the_key_width_read_zero(28, 8)]),
    ("last bucket boundary not summed",
     "for (uint32_t j = 0; j < B; j++) bucket_begin[j + 1] += bucket_begin[j];",
     "for (uint32_t j = 0; j + 1 < B; j++) bucket_begin[j + 1] += bucket_begin[j];",
     [lambda: pins.test_partition_level_boundaries_and_multisets(False)]),
    ("tree size one power of two too large", "while (p < x) p <<= 1;", "while (p <= x) p <<= 1;",
     [lambda: pins.test_classify_no_equality_is_searchsorted(7)]),
    ("equality bucket and the bucket below it swapped",
     "cls[e] = (uint32_t)(2 * i + 1 - (uint64_t)key_less",
     "cls[e] = (uint32_t)(2 * i + (uint64_t)key_less",
     [lambda: pins.test_classify_equality_buckets_semantics(7)]),
    ("insertion sort leaves the first element", "for (uint64_t i = 1; i < n; i++) {\n        memcpy(c->swap",
     "for (uint64_t i = 2; i < n; i++) {\n        memcpy(c->swap",
     [pins.test_bruteforce_insertion_sort_all_short_sequences]),
    ("elements equal to a splitter classed above it",
     "            if (key_less(dt, spl + j * D, x))\n                lo = mid + 1;",
     "            if (!key_less(dt, x, spl + j * D))\n                lo = mid + 1;",
     [lambda: pins.test_classify_no_equality_is_searchsorted(7),
      lambda: pins.test_classify_equality_buckets_semantics(7)]),
]


def _build(tmpdir, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, "mutation site not unique: %s" % name
    path = os.path.join(tmpdir, "mutant.c")
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    lib = os.path.join(tmpdir, "libmutant_%d.so" % abs(hash(name)))
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", path, "-o", lib, "-lm"])
    return oracle._configure(ctypes.CDLL(lib))


def _run_checks(index, tmpdir, q):
    # child process: a mutant may also corrupt memory and crash, which the
    # parent counts as caught too
    name, old, new, checks = MUTANTS[index]
    oracle._lib = _build(tmpdir, name, old, new)
    caught = 0
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError):
            caught += 1
    q.put(caught)


@pytest.mark.parametrize("index", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(tmp_path, index):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_run_checks, args=(index, str(tmp_path), q))
    p.start()
    p.join(timeout=300)
    assert p.exitcode is not None, "mutant check did not finish"
    caught = q.get(timeout=5) if p.exitcode == 0 else 1  # a crash is caught too
    assert caught > 0, "no pin caught the mutant: %s" % MUTANTS[index][0]


def test_unmutated_oracle_passes_the_same_checks():
    for _, _, _, checks in MUTANTS:
        for check in checks:
            check()
