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
