"""Parity at the full sizes of the plain-sort configurations, in the form
the bench times them (ipsgpu_sort through the sorter's CUDA graph): keys
non-decreasing and the multiset of words unchanged.  For u32 / u64 / f64
these two properties determine the output (the sorted permutation of a
multiset is unique), so the result equals the oracle's.  For records (Pair,
Quartet, 100-byte records) the check is by whole records: every output
record equals the input record of the original index it carries, every
index appears once, and a per-record hash signature is unchanged; with the
keys non-decreasing that is exactly the set of correct outputs of an
unstable sort."""
import pytest
import torch

from paper_2009_13569_gb300 import inputs, ipsgpu
from _util import (DEV, keys_nondecreasing, multiset_sig, record_sig, records_intact_dev,
                   stream)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,dist,log2n,algo", [
    ("u64", "uniform", 30, ipsgpu.SAMPLESORT),
    ("u64", "uniform", 30, ipsgpu.RADIX),
    ("u32", "exponential", 30, ipsgpu.SAMPLESORT),
    ("pair", "zipf", 28, ipsgpu.SAMPLESORT),
    ("quartet", "lexdup", 28, ipsgpu.SAMPLESORT),
])
def test_full_size_sort_properties(dtype, dist, log2n, algo):
    n = 1 << log2n
    shape = {"pair": (n, 2), "quartet": (n, 4)}.get(dtype, (n,))
    d = torch.empty(shape, dtype=torch.int32 if dtype == "u32" else torch.int64, device=DEV)
    inputs.generate_into(d, dist, dtype, seed=0x5EED)
    before = multiset_sig(d)
    records = dtype in ("pair", "quartet")
    if records:
        inp = d.clone()
        rsig = record_sig(d, dtype)
    with ipsgpu.Sorter(dtype, algo=algo) as s:
        s.sort(d.data_ptr(), n, stream())
        assert s.status(stream()) == ipsgpu.OK
    assert keys_nondecreasing(d, dtype)
    assert multiset_sig(d) == before
    if records:
        assert record_sig(d, dtype) == rsig
        assert records_intact_dev(d, inp, dtype)


@pytest.mark.parametrize("dtype,n,algo", [
    ("u32", (1 << 32) + 3, ipsgpu.SAMPLESORT),
    ("u64", (1 << 32) + 1, ipsgpu.RADIX),
])
def test_more_than_2_32_elements(dtype, n, algo):
    # element offsets past 2^32 (16 GiB of u32 keys, 32 GiB of u64 keys):
    # no index in the path may wrap at 32 bits
    d = torch.empty((n,), dtype=torch.int32 if dtype == "u32" else torch.int64, device=DEV)
    inputs.generate_into(d, "uniform", dtype, seed=0xB16)
    before = multiset_sig(d)
    with ipsgpu.Sorter(dtype, algo=algo) as s:
        s.sort(d.data_ptr(), n, stream())
        assert s.status(stream()) == ipsgpu.OK
    assert keys_nondecreasing(d, dtype)
    assert multiset_sig(d) == before


@pytest.mark.parametrize("dtype,dist", [("f64", "normal"), ("rec100", "uniform"),
                                        ("rec100", "rootdup"), ("pair", "uniform")])
def test_wide_record_configuration_2e28(dtype, dist):
    # the wider-record plain-sort configuration at its full size: 2^28
    # doubles (2 GiB), Pairs (4 GiB) or 100-byte records (25 GiB)
    n = 1 << 28
    d = inputs.generate(dist, dtype, n, seed=0x5EED, device=DEV)
    before = multiset_sig(d)
    records = dtype != "f64"
    if records:
        inp = d.clone()
        rsig = record_sig(d, dtype)
    with ipsgpu.Sorter(dtype) as s:
        s.sort(d.data_ptr(), n, stream())
        assert s.status(stream()) == ipsgpu.OK
    assert keys_nondecreasing(d, dtype)
    assert multiset_sig(d) == before
    if records:
        assert record_sig(d, dtype) == rsig
        assert records_intact_dev(d, inp, dtype)


def test_2e34_sort_and_its_task_metadata():
    # the serving configuration's huge request sorted alone: 2^34 uint64 keys
    # (128 GiB) in place, with the recursion's statistics: its pending
    # segments (the task metadata of Sec. 3.2 that App. B's strictly
    # in-place variant would keep in the array instead) stay far below the
    # sorter's fixed ring, whatever the size
    n = 1 << 34
    d = torch.empty((n,), dtype=torch.int64, device=DEV)
    inputs.generate_into(d, "uniform", "u64", seed=0x2E34)
    before = multiset_sig(d)
    with ipsgpu.Sorter("u64") as s:
        s.set_timing(True)
        s.sort(d.data_ptr(), n, stream())
        assert s.status(stream()) == ipsgpu.OK
        waves, pending, cap = s.wave_stats()
        s.kernel_stats()
    print("2^34 uint64: %d waves, at most %d segments pending (ring of %d)" % (waves, pending, cap))
    assert 3 <= waves and 0 < pending <= 1 << 17 and cap == 1 << 20
    assert keys_nondecreasing(d, "u64")
    assert multiset_sig(d) == before
