"""The seeded input generators: chunked generation gives the same bits as
one-shot generation, and the segmented batch generator lays arrays out as
its offsets say.  (The generators hold none of the sorting method's
arithmetic.)"""
import pytest
import torch

from paper_2009_13569_gb300 import inputs


@pytest.mark.parametrize("dist", inputs.INT_DISTS)
@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
def test_generate_into_matches_generate(dtype, dist):
    n = 70_001
    ref = inputs.generate(dist, dtype, n, seed=5)
    out = torch.empty_like(ref)
    inputs.generate_into(out, dist, dtype, seed=5, chunk=4096)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("dist", inputs.QUARTET_DISTS)
def test_quartet_generate_into_matches_generate(dist):
    n = 30_001
    ref = inputs.generate(dist, "quartet", n, seed=9)
    out = torch.empty_like(ref)
    inputs.generate_into(out, dist, "quartet", seed=9, chunk=4096)
    assert torch.equal(out, ref)
    assert torch.equal(ref[:, 3], torch.arange(n))


def test_segmented_batch_layout():
    lengths = inputs.segment_lengths(50, 0, 12, seed=9)
    assert int(lengths.min()) >= 1 and int(lengths.max()) <= 1 << 12
    data, offsets = inputs.segmented_batch(lengths, seed=9, chunk_elems=3000)
    assert offsets[0] == 0 and int(offsets[-1]) == data.numel() == int(lengths.sum())
    assert torch.equal(offsets[1:] - offsets[:-1], lengths)
    # the twodup arrays (index 1 mod 3) hold (j^2 + m/2) mod m
    i = 1
    m = int(lengths[i])
    seg = data[int(offsets[i]):int(offsets[i + 1])]
    j = torch.arange(m, dtype=torch.int64)
    assert torch.equal(seg, (j * j + m // 2) % m)
    # the almost sorted arrays are permutations of 0..m-1
    i = 2
    m = int(lengths[i])
    seg = data[int(offsets[i]):int(offsets[i + 1])]
    assert torch.equal(torch.sort(seg).values, torch.arange(m, dtype=torch.int64))


def test_splitmix64_first_outputs_for_state_zero():
    # the generator's widely quoted first two outputs from state 0
    assert inputs.splitmix64_py(0, 0) == 0xE220A8397B1DCDAF
    assert inputs.splitmix64_py(1, 0) == 0x6E789E6AA1B965F4


def test_splitmix64_tensor_matches_big_integer_arithmetic():
    # the tensor form (int64 wrap-around, logical shifts made of arithmetic
    # ones) against the same definition in Python's unbounded integers
    import numpy as np
    idx = [0, 1, 2, 3, (1 << 31) + 7, (1 << 62) + 5]
    idx += np.random.default_rng(1).integers(0, 1 << 62, 200).tolist()
    for seed in (0, 1, inputs.DEFAULT_SEED, (1 << 64) - 1, 1 << 63):
        got = inputs.splitmix64(torch.tensor(idx, dtype=torch.int64), seed)
        for i, g in zip(idx, got.tolist()):
            assert g & ((1 << 64) - 1) == inputs.splitmix64_py(i, seed), (i, seed)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 1000, 4096, (1 << 40) + 3, (1 << 62) - 1])
def test_unsigned_modulo_of_bit_patterns(n):
    vals = [0, 1, 5, (1 << 63) - 1, 1 << 63, (1 << 64) - 1, 0xDEADBEEFCAFEF00D, 0x8000000000000001]
    x = torch.tensor([inputs._s64(v) for v in vals], dtype=torch.int64)
    assert inputs._umod(x, n).tolist() == [v % n for v in vals]


def _np(dist, dtype, n, seed=3):
    return inputs.to_numpy(inputs.generate(dist, dtype, n, seed=seed), dtype)


def _inversions(a):
    # Fenwick-tree count of pairs i < j with a[i] > a[j] (a a permutation)
    n = len(a)
    tree = [0] * (n + 1)
    inv = 0
    for seen, v in enumerate(a.tolist()):
        j, le = v + 1, 0
        while j > 0:
            le += tree[j]
            j -= j & -j
        inv += seen - le
        j = v + 1
        while j <= n:
            tree[j] += 1
            j += j & -j
    return inv


def test_integer_distributions_have_their_structure():
    import math
    import numpy as np
    n = 1 << 14
    u = _np("uniform", "u64", n)
    assert len(np.unique(u >> np.uint64(56))) == 256       # the top byte takes every value
    u32 = _np("uniform", "u32", n)
    assert u32.dtype == np.uint32 and len(np.unique(u32 >> np.uint32(24))) == 256
    e = _np("exponential", "u64", n)                        # 2^k <= v < 2^(k+1), k < log2 n
    assert e.min() >= 1 and e.max() < n
    octaves = np.bincount(np.floor(np.log2(e.astype(np.float64))).astype(int), minlength=14)
    assert len(octaves) == 14 and octaves.min() > n // 14 // 2
    m = math.isqrt(n)
    np.testing.assert_array_equal(_np("rootdup", "u64", n), np.arange(n) % m)
    a = _np("almostsorted", "u64", n)                       # sqrt(n) adjacent swaps
    np.testing.assert_array_equal(np.sort(a), np.arange(n))
    assert 0 < _inversions(a) <= m
    s, r = _np("sorted", "u64", n), _np("reversesorted", "u64", n)
    w = np.uint64((1 << 64) // n)                           # value i lies in stratum i
    np.testing.assert_array_equal(s // w, np.arange(n, dtype=np.uint64))
    np.testing.assert_array_equal(r, s[::-1])
    assert not _np("zero", "u64", n).any()


def test_zipf_frequencies():
    import numpy as np
    z = _np("zipf", "u64", 1 << 18)
    assert z.min() >= 1 and z.max() <= 10 ** 6
    c = np.bincount(z.astype(np.int64), minlength=4)
    assert c[1] == c.max()
    assert 1.45 < c[1] / c[2] < 1.95                        # 2^0.75 = 1.68


def test_f64_distributions():
    import numpy as np
    u = _np("uniform", "f64", 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    g = _np("normal", "f64", 1 << 16)
    assert np.isfinite(g).all() and abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02


def test_record_quartet_and_pair_layouts():
    import numpy as np
    n = 5000
    rec = _np("rootdup", "rec100", n)
    assert not rec[:, :2].any()
    key = np.zeros(n, dtype=np.uint64)
    for b in range(2, 10):                                   # big-endian i mod 2^14
        key = (key << np.uint64(8)) | rec[:, b].astype(np.uint64)
    np.testing.assert_array_equal(key, np.arange(n) % (1 << 14))
    idx = np.zeros(n, dtype=np.uint64)
    for b in range(8):                                       # payload: original index
        idx |= rec[:, 10 + b].astype(np.uint64) << np.uint64(8 * b)
    np.testing.assert_array_equal(idx, np.arange(n))
    for dist in ("exponential", "twodup", "uniform"):
        p = _np(dist, "pair", n)
        np.testing.assert_array_equal(p[:, 0], _np(dist, "u64", n))
        np.testing.assert_array_equal(p[:, 1], np.arange(n))
    for dist in ("exponential", "twodup", "zipf"):           # order-preserving embedding
        q = _np(dist, "quartet", n)
        assert (q[:, 1] < (1 << 20)).all() and (q[:, 2] < (1 << 20)).all()
        v = (q[:, 0] << np.uint64(40)) | (q[:, 1] << np.uint64(20)) | q[:, 2]
        np.testing.assert_array_equal(v, _np(dist, "u64", n))
        np.testing.assert_array_equal(q[:, 3], np.arange(n))
    lex = _np("lexdup", "quartet", n)
    assert set(np.unique(lex[:, 0])) <= {0, 1, 2, 3} and set(np.unique(lex[:, 1])) <= {0, 1, 2, 3}
