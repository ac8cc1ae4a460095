"""GPU parity of the segmented batch (many independent arrays sorted by one
device-planned launch sequence, Sec. 3.2 recursion breadth-first over the
whole batch) through the C ABI against the oracle, segment by segment: mixed
lengths that span tiny arrays, the base-case boundary and several
partitioning levels; every element type; the radix variant; the captured
CUDA graph replayed on refilled buffers; empty, single-element and uncovered
ranges; and invalid offsets."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu
from _util import DEV, assert_sorted_parity, stream, to_dev

pytestmark = pytest.mark.gpu

SMAX_U64 = 184 * 1024 // 8  # default base-case capacity for 8-byte elements


def _offsets_dev(offsets):
    return torch.as_tensor(offsets, dtype=torch.int64).to(DEV).contiguous()


def _check_segments(got, inp, offsets, dtype):
    for i in range(len(offsets) - 1):
        lo, hi = int(offsets[i]), int(offsets[i + 1])
        if hi - lo > 1:
            assert_sorted_parity(got[lo:hi], inp[lo:hi], dtype)
        elif hi - lo == 1:
            np.testing.assert_array_equal(got[lo:hi], inp[lo:hi])


def _run(dtype, host, offsets, **params):
    n = inputs.count(host, dtype)
    d = to_dev(host)
    off = _offsets_dev(offsets)
    with ipsgpu.Sorter(dtype, **params) as s:
        s.sort_segmented(d.data_ptr(), n, off.data_ptr(), len(offsets) - 1, stream())
        st = s.status(stream())
    assert st == ipsgpu.OK, ipsgpu.strerror(st)
    return inputs.to_numpy(d.cpu(), dtype)


def _concat(dtype, lengths, dists, seed):
    parts = [inputs.generate(dists[i % len(dists)], dtype, int(m), seed=seed + i)
             for i, m in enumerate(lengths)]
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    return torch.cat(parts, 0).contiguous(), offsets


@pytest.mark.parametrize("seed", [1, 2])
def test_segmented_u64_mixed_lengths(seed):
    # log-uniform lengths 2^0 .. 2^18: tiny arrays, the base case, one and two levels
    lengths = inputs.segment_lengths(300, 0, 18, seed=seed)
    data, offsets = inputs.segmented_batch(lengths, seed=seed)
    got = _run("u64", data, offsets.numpy())
    _check_segments(got, inputs.to_numpy(data, "u64"), offsets.numpy(), "u64")


def test_segmented_u64_base_case_boundary():
    lengths = [SMAX_U64 - 1, SMAX_U64, SMAX_U64 + 1, 2 * SMAX_U64 + 3, 1, 0, 2, 33, 200_001]
    data, offsets = inputs.segmented_batch(lengths, seed=9)
    got = _run("u64", data, offsets.numpy())
    _check_segments(got, inputs.to_numpy(data, "u64"), offsets.numpy(), "u64")


SHAPE_DISTS = {"f64": inputs.F64_DISTS, "rec100": inputs.REC_DISTS}


def _shape_cut_lengths(dtype):
    # segments of at most 88 KiB of records run on the 512-thread base-case
    # shape (two CTAs per SM), larger ones up to the 184 KiB capacity on the
    # 1024-thread shape, and larger still through a partitioning level
    small = 88 * 1024 // inputs.ELEM_BYTES[dtype]
    cap = 184 * 1024 // inputs.ELEM_BYTES[dtype]
    return [small - 1, small, small + 1, 2, cap, small, cap + 1, small + 1, 33, cap - 1]


@pytest.mark.parametrize("dtype", ["u32", "u64", "f64", "pair", "quartet", "rec100"])
def test_segmented_around_the_base_case_shapes(dtype):
    dists = SHAPE_DISTS.get(dtype, ("uniform", "twodup", "rootdup"))
    host, offsets = _concat(dtype, _shape_cut_lengths(dtype), dists, seed=31)
    got = _run(dtype, host, offsets)
    _check_segments(got, inputs.to_numpy(host, dtype), offsets, dtype)


@pytest.mark.parametrize("dtype", ["u32", "f64", "pair", "rec100", "quartet"])
def test_segmented_other_types(dtype):
    if dtype == "rec100":
        lengths, dists = [5000, 1, 30_000, 700, 9000, 12], inputs.REC_DISTS
    elif dtype == "quartet":
        # around the 5888-element base-case capacity, and several levels
        lengths, dists = [5887, 5888, 5889, 3, 80_000, 0, 33, 150_001], \
            ("uniform", "lexdup", "rootdup", "zipf")
    elif dtype == "f64":
        lengths, dists = [100_000, 3, 50_000, 20_000, 64, 130_000], inputs.F64_DISTS
    else:
        lengths, dists = [120_000, 3, 90_000, 20_000, 64, 130_000, 7], \
            ("uniform", "twodup", "zipf", "rootdup")
    host, offsets = _concat(dtype, lengths, dists, seed=77)
    got = _run(dtype, host, offsets)
    _check_segments(got, inputs.to_numpy(host, dtype), offsets, dtype)


@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
def test_segmented_radix(dtype):
    host, offsets = _concat(dtype, [150_000, 40_000, 5, 260_000], ("uniform", "exponential"),
                            seed=5)
    got = _run(dtype, host, offsets, algo=ipsgpu.RADIX)
    _check_segments(got, inputs.to_numpy(host, dtype), offsets, dtype)


@pytest.mark.parametrize("base_case", [32, 300])
def test_segmented_small_base_case_many_levels(base_case):
    lengths = inputs.segment_lengths(40, 4, 17, seed=base_case)
    data, offsets = inputs.segmented_batch(lengths, seed=base_case)
    got = _run("u64", data, offsets.numpy(), base_case=base_case)
    _check_segments(got, inputs.to_numpy(data, "u64"), offsets.numpy(), "u64")


def test_segmented_many_tiny():
    # 20,000 arrays of at most 64 elements: all go straight to the base case
    lengths = inputs.segment_lengths(20_000, 0, 6, seed=3)
    data, offsets = inputs.segmented_batch(lengths, seed=3)
    got = _run("u64", data, offsets.numpy())
    _check_segments(got, inputs.to_numpy(data, "u64"), offsets.numpy(), "u64")


def test_segmented_partial_cover_leaves_rest():
    # segments cover [100, 60100) and [70000, 190000) only; the gaps stay as they were
    host = inputs.generate("uniform", "u64", 200_000, seed=4)
    d = to_dev(host)
    off = _offsets_dev([100, 60_100, 70_000, 190_000])
    with ipsgpu.Sorter("u64") as s:
        s.sort_segmented(d.data_ptr(), 200_000, off.data_ptr(), 3, stream())
        assert s.status(stream()) == ipsgpu.OK
    got = inputs.to_numpy(d.cpu(), "u64")
    inp = inputs.to_numpy(host, "u64")
    np.testing.assert_array_equal(got[:100], inp[:100])
    np.testing.assert_array_equal(got[190_000:], inp[190_000:])
    _check_segments(got, inp, [100, 60_100, 70_000, 190_000], "u64")


def test_segmented_invalid_offsets_reported():
    host = inputs.generate("uniform", "u64", 50_000, seed=6)
    d = to_dev(host)
    # segment 1 runs backwards, segment 2 past the end: both skipped, E_INVAL recorded
    off = _offsets_dev([0, 30_000, 20_000, 60_000])
    with ipsgpu.Sorter("u64") as s:
        s.sort_segmented(d.data_ptr(), 50_000, off.data_ptr(), 3, stream())
        assert s.status(stream()) == ipsgpu.E_INVAL
        assert s.status(stream()) == ipsgpu.OK  # cleared by the read
    got = inputs.to_numpy(d.cpu(), "u64")
    inp = inputs.to_numpy(host, "u64")
    np.testing.assert_array_equal(got[:30_000], oracle.sort(inp[:30_000], "u64"))
    np.testing.assert_array_equal(got[30_000:], inp[30_000:])


def test_segmented_empty_batches():
    d = torch.zeros(16, dtype=torch.int64, device=DEV)
    off = _offsets_dev([0])
    with ipsgpu.Sorter("u64") as s:
        s.sort_segmented(d.data_ptr(), 16, off.data_ptr(), 0, stream())
        s.sort_segmented(d.data_ptr(), 0, off.data_ptr(), 0, stream())
        assert s.status(stream()) == ipsgpu.OK
        with pytest.raises(ipsgpu.IpsgpuError):
            s.sort_segmented(d.data_ptr(), 16, 0, 3, stream())


def test_segmented_graph_replay_refilled():
    lengths = inputs.segment_lengths(120, 2, 17, seed=21)
    data1, offsets = inputs.segmented_batch(lengths, seed=21)
    data2, _ = inputs.segmented_batch(lengths, seed=22)
    n = data1.numel()
    d = to_dev(data1)
    off = offsets.to(DEV)
    with ipsgpu.Sorter("u64") as s:
        g = s.segmented_graph(d.data_ptr(), n, off.data_ptr(), len(lengths))
        assert g.nodes() == 2  # the run's setup node and the WHILE loop over waves
        for host in (data1, data2, data1):
            d.copy_(host.to(DEV))
            g.launch(stream())
            assert s.status(stream()) == ipsgpu.OK
            _check_segments(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(host, "u64"),
                            offsets.numpy(), "u64")
        g.close()


def test_segmented_matches_per_array_sort():
    # the batch gives, array by array, exactly what one plain sort per array gives
    lengths = inputs.segment_lengths(25, 8, 17, seed=31)
    data, offsets = inputs.segmented_batch(lengths, seed=31)
    o = offsets.numpy()
    batch = _run("u64", data, o)
    d = to_dev(data)
    with ipsgpu.Sorter("u64") as s:
        for i in range(len(lengths)):
            lo, hi = int(o[i]), int(o[i + 1])
            s.sort(d[lo:hi].data_ptr(), hi - lo, stream())
        assert s.status(stream()) == ipsgpu.OK
    np.testing.assert_array_equal(batch, inputs.to_numpy(d.cpu(), "u64"))


def test_sort_batch_separate_arrays():
    # separate device tensors of one type, sorted by one batch call
    lengths = [70_000, 5, 0, 1, 23_552, 140_001, 999]
    hosts = [inputs.generate(("uniform", "twodup", "zipf")[i % 3], "u64", m, seed=40 + i)
             for i, m in enumerate(lengths)]
    devs = [to_dev(h) if h.numel() else torch.empty(0, dtype=torch.int64, device=DEV)
            for h in hosts]
    segs = torch.tensor([[t.data_ptr(), t.numel()] for t in devs], dtype=torch.int64).to(DEV)
    with ipsgpu.Sorter("u64") as s:
        s.sort_batch(segs.data_ptr(), len(devs), stream())
        assert s.status(stream()) == ipsgpu.OK
    for h, t in zip(hosts, devs):
        got = inputs.to_numpy(t.cpu(), "u64")
        if h.numel() > 1:
            assert_sorted_parity(got, inputs.to_numpy(h, "u64"), "u64")


def test_sort_batch_pairs_and_bad_entry():
    hosts = [inputs.generate("rootdup", "pair", m, seed=50 + m) for m in (30_000, 90_000, 300)]
    devs = [to_dev(h) for h in hosts]
    rows_ = [[t.data_ptr(), t.shape[0]] for t in devs]
    rows_.append([devs[0].data_ptr() + 8, 100])  # misaligned for 16-byte pairs: skipped
    segs = torch.tensor(rows_, dtype=torch.int64).to(DEV)
    with ipsgpu.Sorter("pair") as s:
        s.sort_batch(segs.data_ptr(), len(rows_), stream())
        assert s.status(stream()) == ipsgpu.E_INVAL
    for h, t in zip(hosts, devs):
        assert_sorted_parity(inputs.to_numpy(t.cpu(), "pair"), inputs.to_numpy(h, "pair"), "pair")


def test_sort_batch_quartets():
    hosts = [inputs.generate(d, "quartet", m, seed=60 + m)
             for d, m in (("lexdup", 40_000), ("uniform", 6000), ("rootdup", 70_001), ("zero", 500))]
    devs = [to_dev(h) for h in hosts]
    segs = torch.tensor([[t.data_ptr(), t.shape[0]] for t in devs], dtype=torch.int64).to(DEV)
    with ipsgpu.Sorter("quartet") as s:
        s.sort_batch(segs.data_ptr(), len(devs), stream())
        assert s.status(stream()) == ipsgpu.OK
    for h, t in zip(hosts, devs):
        assert_sorted_parity(inputs.to_numpy(t.cpu(), "quartet"), inputs.to_numpy(h, "quartet"),
                             "quartet")


@pytest.mark.parametrize("timing", [False, True])
def test_small_arena_forces_many_waves(timing):
    # a 2 MiB arena holds only a few segments per wave, so every level is
    # split over many waves; the host-driven loop (timing on) must agree
    lengths = inputs.segment_lengths(400, 10, 19, seed=61)
    data, offsets = inputs.segmented_batch(lengths, seed=61)
    n = data.numel()
    d = to_dev(data)
    off = offsets.to(DEV)
    big = inputs.generate("exponential", "u64", 3_000_000, seed=62)
    db = to_dev(big)
    with ipsgpu.Sorter("u64", arena_bytes=2 << 20) as s:
        s.set_timing(timing)
        s.sort_segmented(d.data_ptr(), n, off.data_ptr(), len(lengths), stream())
        s.sort(db.data_ptr(), big.numel(), stream())
        assert s.status(stream()) == ipsgpu.OK
        if timing:
            st = s.kernel_stats()
            # several waves, each with its own classification launch
            assert st["classify"][0] >= 5 and st["plan"][0] >= 2 * st["classify"][0]
    _check_segments(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(data, "u64"),
                    offsets.numpy(), "u64")
    assert_sorted_parity(inputs.to_numpy(db.cpu(), "u64"), inputs.to_numpy(big, "u64"), "u64")


def test_arena_too_small_rejected():
    with pytest.raises(ipsgpu.IpsgpuError):
        ipsgpu.Sorter("u64", arena_bytes=64 << 10)


def test_segmented_constant_and_two_valued_arrays():
    # base-case segments whose keys are all equal (the first pass finds a zero
    # key range) or take two values, next to ordinary ones
    lengths = [100, 5000, 23_552, 33, 17_000, 64, 20_000, 9_999]
    parts = []
    for i, m in enumerate(lengths):
        if i % 3 == 0:
            parts.append(torch.full((m,), 7 + i, dtype=torch.int64))
        elif i % 3 == 1:
            parts.append((torch.arange(m, dtype=torch.int64) % 2) * (1 << 40))
        else:
            parts.append(inputs.generate("uniform", "u64", m, seed=i))
    host = torch.cat(parts)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    got = _run("u64", host, offsets)
    _check_segments(got, inputs.to_numpy(host, "u64"), offsets, "u64")


@pytest.mark.parametrize("dist", ["exponential", "zipf", "eightdup"])
def test_sort_skewed_large(dist):
    # 2^23 keys: several partitioning waves with equality buckets, base-case
    # segments of few distinct values
    host = inputs.generate(dist, "u64", 1 << 23, seed=91)
    d = to_dev(host)
    with ipsgpu.Sorter("u64") as s:
        s.sort(d.data_ptr(), 1 << 23, stream())
        assert s.status(stream()) == ipsgpu.OK
    assert_sorted_parity(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(host, "u64"), "u64")
