"""Record parity past one partitioning level, and the sorter parameters that
change the block layout.

Pair, Quartet and 100-byte records are sorted with default parameters at
sizes where the sort takes at least two partitioning levels and its second
wave holds many segments cut into balanced stripes (2^22 100-byte records:
256 buckets of about 16,000 records, each partitioned again; 2^23 Pairs and
Quartets: 256 buckets of 32,768 records).  The key sequence is compared
with the oracle's element by element, and every record is checked whole
through the original index it carries.

Then every (k, block bytes) pair the autotuner searches (k * block bytes at
most 128 KiB, blocks up to 2 KiB) sorts every element type correctly, and
sorters created with different block sizes keep working side by side (the
classification kernel's shared-memory limit belongs to the kernel, not to
one sorter)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import autotune, inputs, ipsgpu
from _util import DEV, assert_level_parity, assert_record_parity, run_sort, stream, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,dist,log2n", [
    ("pair", "uniform", 23),
    ("pair", "rootdup", 23),
    ("pair", "zipf", 23),
    ("quartet", "uniform", 23),
    ("quartet", "lexdup", 23),
    ("rec100", "uniform", 22),
    ("rec100", "rootdup", 22),
])
def test_record_parity_multi_level_default_params(dtype, dist, log2n):
    host = inputs.generate(dist, dtype, 1 << log2n, seed=0xC0FFEE)
    inp = inputs.to_numpy(host, dtype)
    d = to_dev(host)
    with ipsgpu.Sorter(dtype) as s:
        s.set_timing(True)  # host-driven waves: count them
        s.sort(d.data_ptr(), 1 << log2n, stream())
        assert s.status(stream()) == ipsgpu.OK
        stats = s.kernel_stats()
    # two partitioning levels (and possibly a small third wave)
    assert stats["classify"][0] >= 2, stats["classify"]
    assert_record_parity(inputs.to_numpy(d.cpu(), dtype), inp, dtype)


KB = autotune.KB_PAIRS


@pytest.mark.parametrize("dtype", ["u32", "u64", "pair", "quartet", "rec100"])
@pytest.mark.parametrize("k,block_bytes", KB)
def test_every_kb_pair_sorts_every_type(dtype, k, block_bytes):
    n = 60_001 if dtype == "rec100" else 1_000_003
    dist = "rootdup" if dtype == "rec100" else ("lexdup" if dtype == "quartet" else "uniform")
    host = inputs.generate(dist, dtype, n, seed=k + block_bytes)
    got = run_sort(dtype, host, k=k, block_bytes=block_bytes)
    inp = inputs.to_numpy(host, dtype)
    if dtype in ("u32", "u64"):
        np.testing.assert_array_equal(got, oracle.sort(inp, dtype))
    else:
        assert_record_parity(got, inp, dtype)


@pytest.mark.parametrize("k,block_bytes", KB)
def test_every_kb_pair_partition_level(k, block_bytes):
    # one level with given splitters, blocks of 512 B to 2 KiB: boundaries
    # bit-exact and each bucket the oracle's multiset
    n, m = 500_009, k - 1
    host = inputs.generate("uniform", "pair", n, seed=k)
    a = inputs.to_numpy(host, "pair")
    spl = np.sort(a[np.random.default_rng(k).integers(0, n, size=m), 0])
    spl_rec = np.stack([spl, np.zeros_like(spl)], axis=1)
    d = to_dev(host)
    ds = to_dev(inputs.from_numpy(spl_rec, "pair"))
    bb = torch.zeros(k + 1, dtype=torch.int64, device=DEV)
    with ipsgpu.Sorter("pair", k=k, block_bytes=block_bytes) as s:
        s.partition_level(d.data_ptr(), n, ds.data_ptr(), m, False, bb.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK
    cls, _ = oracle.classify(a, "pair", spl_rec, False)
    assert_level_parity(inputs.to_numpy(d.cpu(), "pair"), bb.cpu().numpy().view(np.uint64), a,
                        "pair", cls, k)


def test_sorters_with_different_blocks_side_by_side():
    # sorter A (512-byte blocks) is created, then sorter B (256-byte blocks,
    # less classification shared memory), then the allocation-free level
    # runs; sorting with A afterwards, and with B, and the allocation-free
    # level again must all still match the oracle
    n = 2_000_003
    host = inputs.generate("uniform", "u64", n, seed=77)
    ref = oracle.sort(inputs.to_numpy(host, "u64"), "u64")
    a = ipsgpu.Sorter("u64", block_bytes=512)
    b = ipsgpu.Sorter("u64", block_bytes=256)
    try:
        for s in (a, b, a):
            d = to_dev(host)
            s.sort(d.data_ptr(), n, stream())
            assert s.status(stream()) == ipsgpu.OK
            np.testing.assert_array_equal(inputs.to_numpy(d.cpu(), "u64"), ref)
            m = 255
            spl = np.sort(ref[np.linspace(0, n - 1, m).astype(np.int64)])
            x = to_dev(host)
            ds = to_dev(inputs.from_numpy(spl, "u64"))
            bb = torch.full((257,), -1, dtype=torch.int64, device=DEV)
            ipsgpu.partition_level_noalloc("u64", x.data_ptr(), n, ds.data_ptr(), m, False,
                                           bb.data_ptr(), stream())
            torch.cuda.synchronize(DEV)
            cls, _ = oracle.classify(inputs.to_numpy(host, "u64"), "u64", spl, False)
            assert_level_parity(inputs.to_numpy(x.cpu(), "u64"), bb.cpu().numpy().view(np.uint64),
                                inputs.to_numpy(host, "u64"), "u64", cls, 256)
    finally:
        a.close()
        b.close()
