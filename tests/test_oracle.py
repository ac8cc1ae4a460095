"""Pins of the CPU oracle against facts that do not come from the oracle.

Every test here runs on the CPU.  Each pin is chosen so that a plausible slip
in oracle.c (a dropped term in the class formula, a reversed comparison, an
off-by-one in the padding, a lost or duplicated element in the distribution,
a wrong recursion rule) fails at least one of them:

  * brute force: every sequence of length <= 8 over a 4-letter alphabet,
    sorted by the samplesort with tiny k and n0 so it partitions, against
    Python's sorted();
  * library special cases: numpy.sort, numpy.searchsorted, numpy argsort;
  * closed forms: the histograms of RootDup / TwoDup / EightDup computed by
    counting the formulas of Sec. 6, never by sorting;
  * the decision-tree figure of Sec. 2 (7 splitters, 15 reachable buckets,
    7 of them equality buckets), stored in tests/golden/;
  * invariants: sortedness and order-independent multiset hashes.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2009_13569_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=1):
    return np.random.default_rng(seed)


def _multiset_hash(a):
    """Two commutative 64-bit hashes of the rows of a (sum of mixes)."""
    b = np.ascontiguousarray(a).view(np.uint8).reshape(len(a), -1).astype(np.uint64)
    w = np.arange(1, b.shape[1] + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h1 = (b * w * np.uint64(0x9E3779B97F4A7C15)).sum(axis=1)
        h1 ^= h1 >> np.uint64(29)
        h1 *= np.uint64(0xBF58476D1CE4E5B9)
        h2 = (b * (w + np.uint64(7))).sum(axis=1) * np.uint64(0x94D049BB133111EB)
        h2 ^= h2 >> np.uint64(31)
        return int(h1.sum()), int(h2.sum()), len(a)


# ---------------------------------------------------------------- brute force

def test_bruteforce_all_short_sequences_partitioning_path():
    # k=4, n0=1: tasks with more than 2 elements partition (Sec. 3.2 rule)
    for length in range(0, 9):
        for seq in itertools.product(range(4), repeat=length):
            a = np.array(seq, dtype=np.uint64)
            got = oracle.sort(a, "u64", k=4, n0=1, seed=length + 17)
            assert got.tolist() == sorted(seq), seq


def test_bruteforce_insertion_sort_all_short_sequences():
    for length in range(0, 8):
        for seq in itertools.product(range(3), repeat=length):
            a = np.array(seq, dtype=np.uint32)
            assert oracle.insertion_sort(a, "u32").tolist() == sorted(seq)


@pytest.mark.parametrize("k,n0", [(4, 1), (8, 2), (16, 4), (256, 16), (4, 16)])
def test_random_small_against_numpy(k, n0):
    rng = _rng(k * 31 + n0)
    for n in list(range(0, 70)) + [257, 1000, 2999]:
        for alphabet in (3, 50, 1 << 62):
            a = rng.integers(0, alphabet, size=n, dtype=np.uint64)
            got = oracle.sort(a, "u64", k=k, n0=n0, seed=n)
            np.testing.assert_array_equal(got, np.sort(a))


# ------------------------------------------------------- library special cases

@pytest.mark.parametrize("dist", inputs.INT_DISTS)
@pytest.mark.parametrize("dtype", ["u32", "u64"])
def test_sort_matches_numpy_every_distribution(dist, dtype):
    n = 20000
    a = inputs.to_numpy(inputs.generate(dist, dtype, n), dtype)
    got = oracle.sort(a, dtype)
    np.testing.assert_array_equal(got, np.sort(a))
    assert oracle.is_sorted(got, dtype)


@pytest.mark.parametrize("dist", inputs.F64_DISTS)
def test_sort_f64_matches_numpy(dist):
    a = inputs.to_numpy(inputs.generate(dist, "f64", 30000), "f64")
    got = oracle.sort(a, "f64")
    np.testing.assert_array_equal(got.view(np.uint64), np.sort(a).view(np.uint64))


def test_f64_order_is_total_and_refines_less_than():
    vals = np.array([3.5, -0.0, 0.0, -1e300, 1e-300, -1e-300, np.inf, -np.inf, 2.0, -2.0],
                    dtype=np.float64)
    got = oracle.sort(vals, "f64", k=4, n0=1)
    # -0.0 strictly before +0.0, otherwise numeric order
    expect = [-np.inf, -1e300, -2.0, -1e-300, -0.0, 0.0, 1e-300, 2.0, 3.5, np.inf]
    assert got.tolist() == expect
    assert np.signbit(got[4]) and not np.signbit(got[5])


def test_f64_order_is_ieee754_total_order():
    # IEEE 754-2008 totalOrder: -NaN (larger payload first) < -inf < negative
    # normals < negative subnormals < -0 < +0 < positive subnormals < normals
    # < +inf < +NaN (larger payload last).  Written out by hand from that
    # definition, as bit patterns.
    expect = [
        0xFFF8000000000001,  # -NaN, payload 0x8000000000001 (quiet)
        0xFFF0000000000001,  # -NaN, payload 1 (signalling)
        0xFFF0000000000000,  # -inf
        0xFFEFFFFFFFFFFFFF,  # -max double
        0xBFF0000000000000,  # -1.0
        0x8010000000000000,  # -smallest normal
        0x800FFFFFFFFFFFFF,  # -largest subnormal
        0x8000000000000001,  # -smallest subnormal
        0x8000000000000000,  # -0.0
        0x0000000000000000,  # +0.0
        0x0000000000000001,  # +smallest subnormal
        0x000FFFFFFFFFFFFF,  # +largest subnormal
        0x0010000000000000,  # +smallest normal
        0x3FF0000000000000,  # 1.0
        0x7FEFFFFFFFFFFFFF,  # max double
        0x7FF0000000000000,  # +inf
        0x7FF0000000000001,  # +NaN, payload 1
        0x7FF8000000000000,  # +NaN (the default quiet NaN)
    ]
    bits = np.array(expect, dtype=np.uint64)
    for seed in range(5):
        shuffled = bits[np.random.default_rng(seed).permutation(len(bits))]
        got = oracle.sort(shuffled.view(np.float64), "f64", k=4, n0=1, seed=seed)
        assert got.view(np.uint64).tolist() == expect


def test_pair_keys_sorted_and_records_kept():
    n = 5000
    a = inputs.to_numpy(inputs.generate("rootdup", "pair", n), "pair")
    got = oracle.sort(a, "pair", k=8, n0=2)
    np.testing.assert_array_equal(got[:, 0], np.sort(a[:, 0]))
    # each equal-key run holds the same set of records as the input
    for key in np.unique(a[:, 0])[:50]:
        assert sorted(got[got[:, 0] == key, 1].tolist()) == sorted(a[a[:, 0] == key, 1].tolist())
    assert _multiset_hash(got) == _multiset_hash(a)


@pytest.mark.parametrize("dist", inputs.REC_DISTS)
def test_rec100_lexicographic_unsigned_bytes(dist):
    n = 3000
    a = inputs.to_numpy(inputs.generate(dist, "rec100", n), "rec100").copy()
    # pairs of records equal in bytes 0..8 that differ only in byte 9, on
    # either side of 0x80, the larger one first (a 9-byte compare keeps
    # their input order, a signed-char compare reverses them)
    m = len(a[1::7])
    a[1::7, :9] = a[0::7, :9][:m]
    a[0::7, 9] = 0xF0
    a[1::7, 9] = 0x10
    got = oracle.sort(a, "rec100", k=16, n0=4)
    keys = [bytes(r[:10]) for r in got]
    assert keys == sorted(bytes(r[:10]) for r in a)  # Python bytes: unsigned
    assert _multiset_hash(got) == _multiset_hash(a)


def _qkeys(a):
    return [tuple(r) for r in a[:, :3].tolist()]


def test_quartet_bruteforce_all_short_sequences():
    # every sequence of length <= 5 over the 8 keys with words in {0, 1},
    # through the partitioning path (k=4, n0=1), against Python's tuple
    # order (lexicographic by definition); the value column keeps each
    # record's identity
    keys = list(itertools.product(range(2), repeat=3))
    for length in range(0, 6):
        for seq in itertools.product(range(8), repeat=length):
            a = np.array([keys[x] + (i,) for i, x in enumerate(seq)], dtype=np.uint64).reshape(-1, 4)
            got = oracle.sort(a, "quartet", k=4, n0=1, seed=length)
            assert _qkeys(got) == sorted(_qkeys(a)), seq
            assert sorted(map(tuple, got.tolist())) == sorted(map(tuple, a.tolist()))


def test_quartet_word_order_by_hand():
    a = np.array([[1, 0, 0, 0], [0, 9, 9, 1], [0, 9, 0, 2], [0, 0, 5, 3],
                  [0, 9, 9, 4], [2**64 - 1, 0, 0, 5], [0, 2**63, 0, 6]], dtype=np.uint64)
    got = oracle.sort(a, "quartet", k=4, n0=1)
    assert _qkeys(got) == [(0, 0, 5), (0, 9, 0), (0, 9, 9), (0, 9, 9), (0, 2**63, 0),
                           (1, 0, 0), (2**64 - 1, 0, 0)]
    assert oracle.insertion_sort(a, "quartet")[:, :3].tolist() == [list(k) for k in _qkeys(got)]


@pytest.mark.parametrize("dist", inputs.QUARTET_DISTS)
def test_quartet_matches_numpy_lexsort(dist):
    n = 20000
    a = inputs.to_numpy(inputs.generate(dist, "quartet", n), "quartet")
    got = oracle.sort(a, "quartet")
    ref = a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
    np.testing.assert_array_equal(got[:, :3], ref[:, :3])
    assert _multiset_hash(got) == _multiset_hash(a)
    assert oracle.is_sorted(got, "quartet")
    if dist not in ("uniform", "lexdup"):
        # the order-preserving embedding of the 64-bit value
        v = (got[:, 0] << np.uint64(40)) | (got[:, 1] << np.uint64(20)) | got[:, 2]
        u = inputs.to_numpy(inputs.generate(dist, "u64", n), "u64")
        np.testing.assert_array_equal(v, np.sort(u))


@pytest.mark.parametrize("eq", [False, True])
def test_quartet_classify_is_the_u64_classify_of_dense_ranks(eq):
    # a comparison-based classification depends on the key order only: map
    # every key to its dense rank in the lexicographic order (numpy sorts
    # rows lexicographically) and the classes must be the searchsorted /
    # equality-bucket classes of the ranks
    rng = _rng(11 + eq)
    n, m = 6000, 37
    a = np.stack([rng.integers(0, 3, n), rng.integers(0, 3, n), rng.integers(0, 50, n),
                  np.arange(n)], axis=1).astype(np.uint64)
    spl = a[rng.choice(n, m, replace=False)]
    spl = spl[np.lexsort((spl[:, 2], spl[:, 1], spl[:, 0]))]
    allk = np.concatenate([a[:, :3], spl[:, :3]])
    _, inv = np.unique(allk, axis=0, return_inverse=True)
    ra, rs = inv[:n].astype(np.uint64).ravel(), inv[n:].astype(np.uint64).ravel()
    cls, B = oracle.classify(a, "quartet", spl, eq)
    pad, K = _padded(rs, m)
    i = np.searchsorted(pad[:K - 1], ra, side="left")
    if not eq:
        assert B == K
        np.testing.assert_array_equal(cls, i)
    else:
        assert B == 2 * K
        hit = pad[np.minimum(i, K - 1)] == ra
        np.testing.assert_array_equal(cls, np.where(hit, 2 * i + 1, np.where(i == K - 1, 2 * K - 1, 2 * i)))


# ------------------------------------------------------------- closed forms

def _expect_from_hist(values, counts):
    return np.repeat(np.asarray(values, dtype=np.uint64), counts)


@pytest.mark.parametrize("n", [1 << 12, 1 << 14, 1 << 16])
def test_rootdup_closed_form(n):
    m = math.isqrt(n)
    a = inputs.to_numpy(inputs.generate("rootdup", "u64", n), "u64")
    # A[i] = i mod m: value v occurs ceil((n - v) / m) times
    counts = [(n - v + m - 1) // m for v in range(m)]
    assert set(counts) <= {n // m, -(-n // m)}
    np.testing.assert_array_equal(oracle.sort(a, "u64"), _expect_from_hist(range(m), counts))


@pytest.mark.parametrize("p", [2, 8])
@pytest.mark.parametrize("n", [1 << 12, 1 << 15])
def test_twodup_eightdup_closed_form(p, n):
    dist = "twodup" if p == 2 else "eightdup"
    a = inputs.to_numpy(inputs.generate(dist, "u64", n), "u64")
    hist = {}
    for i in range(n):  # (i^p + n/2) mod n, counted, never sorted
        v = (pow(i, p, 1 << 64) + n // 2) % n
        hist[v] = hist.get(v, 0) + 1
    vals = sorted(hist)
    np.testing.assert_array_equal(oracle.sort(a, "u64"),
                                  _expect_from_hist(vals, [hist[v] for v in vals]))


def test_zero_sorted_reverse():
    n = 4096
    z = inputs.to_numpy(inputs.generate("zero", "u64", n), "u64")
    assert not oracle.sort(z, "u64").any()
    s = inputs.to_numpy(inputs.generate("sorted", "u64", n), "u64")
    r = inputs.to_numpy(inputs.generate("reversesorted", "u64", n), "u64")
    assert oracle.is_sorted(s, "u64")
    np.testing.assert_array_equal(oracle.sort(s, "u64"), s)
    np.testing.assert_array_equal(oracle.sort(r, "u64"), s)


# ------------------------------------------------------- classification level

def _padded(spl, m):
    K = 1 << math.ceil(math.log2(m + 1))
    return np.concatenate([spl, np.repeat(spl[-1:], K - m)]), K


@pytest.mark.parametrize("m", [1, 2, 3, 7, 8, 100, 255])
def test_classify_no_equality_is_searchsorted(m):
    rng = _rng(m)
    a = rng.integers(0, 1000, size=20000, dtype=np.uint64)
    spl = np.sort(rng.integers(0, 1000, size=m, dtype=np.uint64))
    cls, B = oracle.classify(a, "u64", spl, False)
    pad, K = _padded(spl, m)
    assert B == K
    # smallest i with e <= s_i among s_0..s_{K-2}, else K-1
    np.testing.assert_array_equal(cls, np.searchsorted(pad[:K - 1], a, side="left"))


@pytest.mark.parametrize("m", [1, 3, 7, 31, 127])
def test_classify_equality_buckets_semantics(m):
    rng = _rng(100 + m)
    spl = np.sort(rng.choice(np.arange(0, 10 * m + 10, dtype=np.uint64), size=m, replace=False))
    a = np.concatenate([rng.integers(0, 10 * m + 20, size=5000, dtype=np.uint64), spl])
    cls, B = oracle.classify(a, "u64", spl, True)
    K = B // 2
    i = np.minimum(np.searchsorted(spl, a, side="left"), K - 1)
    is_eq = np.zeros(len(a), dtype=bool)
    inb = i < m
    is_eq[inb] = spl[i[inb]] == a[inb]
    above = a > spl[-1]
    # elements equal to s_i -> 2i+1; strictly between -> 2i; above all -> 2K-1
    np.testing.assert_array_equal(cls[is_eq], 2 * i[is_eq] + 1)
    between = ~is_eq & ~above
    np.testing.assert_array_equal(cls[between], 2 * i[between])
    assert (cls[above] == 2 * K - 1).all()
    assert not (cls == 2 * K - 2).any()


def test_decision_tree_figure_golden():
    facts = {}
    with open(os.path.join(GOLDEN, "decision_tree_fig.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                facts[k] = int(v)
    spl = np.arange(10, 10 * (facts["splitters"] + 1), 10, dtype=np.uint64)
    a = np.arange(0, 10 * facts["splitters"] + 20, dtype=np.uint64)  # every value
    cls, B = oracle.classify(a, "u64", spl, True)
    assert B == facts["class_ids"] == 2 * facts["leaf_buckets"]
    reached = set(cls.tolist())
    assert len(reached) == facts["reachable_buckets"]
    eq_buckets = {int(c) for c, e in zip(cls, a) if e in set(spl.tolist())}
    assert len(eq_buckets) == facts["equality_buckets"]
    assert facts["never_reached"] not in reached


def test_classify_bruteforce_tiny():
    # every array of length 4 over {0..4} and every sorted splitter multiset
    # of size 1..3 over {0..4}: compare with the definition by linear scan
    for m in (1, 2, 3):
        for spl in itertools.combinations_with_replacement(range(5), m):
            spl_a = np.array(spl, dtype=np.uint64)
            K = 1 << math.ceil(math.log2(m + 1))
            pad = list(spl) + [spl[-1]] * (K - m)
            a = np.array(list(itertools.product(range(5), repeat=4)), dtype=np.uint64).ravel()
            c0, _ = oracle.classify(a, "u64", spl_a, False)
            c1, _ = oracle.classify(a, "u64", spl_a, True)
            for e, x0, x1 in zip(a.tolist(), c0.tolist(), c1.tolist()):
                i = next((j for j in range(K - 1) if e <= pad[j]), K - 1)
                assert x0 == i
                assert x1 == (2 * i + 1 if e == pad[i] else (2 * i + 1 if e > pad[i] else 2 * i))


def test_zero_input_one_equality_bucket():
    a = np.zeros(1000, dtype=np.uint64)
    out, bb = oracle.partition_level(a, "u64", np.zeros(5, dtype=np.uint64), True)
    sizes = np.diff(bb.astype(np.int64))
    assert (sizes > 0).sum() == 1 and sizes[1] == 1000


@pytest.mark.parametrize("eq", [False, True])
def test_partition_level_boundaries_and_multisets(eq):
    rng = _rng(7)
    a = rng.integers(0, 300, size=10000, dtype=np.uint64)
    spl = np.sort(rng.integers(0, 300, size=40, dtype=np.uint64))
    cls, B = oracle.classify(a, "u64", spl, eq)
    out, bb = oracle.partition_level(a, "u64", spl, eq)
    assert bb[0] == 0 and bb[-1] == len(a) and (np.diff(bb.astype(np.int64)) >= 0).all()
    np.testing.assert_array_equal(bb, np.concatenate([[0], np.cumsum(np.bincount(cls, minlength=B))]))
    np.testing.assert_array_equal(out, a[np.argsort(cls, kind="stable")])
    if eq:  # each equality bucket 2i+1 holds exactly the copies of s_i
        uniq = np.unique(spl)
        for j in range(B // 2 - 1):
            s = spl[min(j, len(spl) - 1)]
            if j < len(spl) and (j == 0 or spl[j - 1] != s):
                assert bb[2 * j + 2] - bb[2 * j + 1] == (a == s).sum()
        assert len(uniq) <= len(spl)


@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
@pytest.mark.parametrize("shift,bits", [(0, 8), (24, 8), (56, 8), (4, 3), (0, 1)])
def test_radix_classify_against_numpy(dtype, shift, bits):
    if dtype == "u32" and shift + bits > 32:
        shift = 32 - bits
    a = inputs.to_numpy(inputs.generate("uniform", dtype, 5000), dtype)
    key = a[:, 0] if dtype == "pair" else a
    cls, B = oracle.radix_classify(a, dtype, shift, bits)
    assert B == 1 << bits
    expect = (key.astype(np.uint64) >> np.uint64(shift)) & np.uint64((1 << bits) - 1)
    np.testing.assert_array_equal(cls, expect.astype(np.uint32))
    out, bb = oracle.radix_level(a, dtype, shift, bits)
    np.testing.assert_array_equal(out, a[np.argsort(cls, kind="stable")])


@pytest.mark.parametrize("shift,bits", [(28, 8), (30, 4), (32, 8)])
def test_radix_u32_digits_above_the_key_width_read_zero(shift, bits):
    # a 32-bit key has no bits above bit 31: a digit that reaches past them
    # holds only the key's top bits, and one that starts at bit 32 is zero
    a = inputs.to_numpy(inputs.generate("uniform", "u32", 5000), "u32")
    cls, B = oracle.radix_classify(a, "u32", shift, bits)
    assert B == 1 << bits
    expect = (a.astype(np.uint64) >> np.uint64(shift)) & np.uint64((1 << bits) - 1)
    np.testing.assert_array_equal(cls, expect.astype(np.uint32))
    if shift >= 32:
        assert not cls.any()
    else:
        assert cls.max() == (1 << (32 - shift)) - 1  # the top bits do vary


def test_multiset_hash_detects_a_lost_element():
    a = _rng(3).integers(0, 1 << 62, size=1000, dtype=np.uint64)
    b = a.copy()
    b[5] = b[6]
    assert _multiset_hash(a) != _multiset_hash(b)
    assert _multiset_hash(a) == _multiset_hash(a[::-1].copy())
