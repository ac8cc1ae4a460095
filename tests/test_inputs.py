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
