"""GPU parity of the whole sort (levels + base case) through the C ABI
against the oracle, for every element type and input distribution, plus the
edge cases of the method (empty, tiny, base-case boundary, sorted, reversed,
all equal) and the bounded-wait failure path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu
from _util import DEV, assert_sorted_parity, run_sort, stream

pytestmark = pytest.mark.gpu

N = 300_007


@pytest.mark.parametrize("algo", [ipsgpu.SAMPLESORT, ipsgpu.RADIX])
def test_small_configuration_2e20_uniform_u64(algo):
    # the small plain-sort configuration: 2^20 uint64 keys, Uniform [0, 2^64),
    # default seed.  The oracle runs its parameters exactly (k = 256,
    # alpha = 0.2 log2 n, base case 16); the GPU runs its own block size (512 B:
    # 256 blocks of 2 KiB would need 512 KiB of shared memory).  The sorted
    # sequence is unique, so the two must agree bit for bit.
    host = inputs.generate("uniform", "u64", 1 << 20)
    ref = oracle.sort(inputs.to_numpy(host, "u64"), "u64", k=256, n0=16, alpha=0.2)
    got = run_sort("u64", host, algo=algo)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dist", inputs.INT_DISTS)
@pytest.mark.parametrize("dtype", ["u32", "u64"])
def test_sort_int_distributions(dtype, dist):
    host = inputs.generate(dist, dtype, N)
    assert_sorted_parity(run_sort(dtype, host), inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("dist", inputs.F64_DISTS)
def test_sort_f64(dist):
    host = inputs.generate(dist, "f64", N)
    assert_sorted_parity(run_sort("f64", host), inputs.to_numpy(host, "f64"), "f64")


@pytest.mark.parametrize("algo", [ipsgpu.SAMPLESORT, ipsgpu.SAMPLESORT_TREE])
def test_sort_f64_special_values(algo):
    # NaNs of both signs and several payloads, infinities, signed zeros and
    # subnormals among normal values: the GPU order must be the oracle's
    # (IEEE 754 totalOrder), bit for bit
    a = inputs.to_numpy(inputs.generate("normal", "f64", N, seed=4), "f64").copy()
    special = np.array([0xFFF8000000000001, 0xFFF0000000000001, 0xFFF0000000000000,
                        0x800FFFFFFFFFFFFF, 0x8000000000000001, 0x8000000000000000, 0,
                        1, 0x000FFFFFFFFFFFFF, 0x7FF0000000000000, 0x7FF0000000000001,
                        0x7FF8000000000000], dtype=np.uint64).view(np.float64)
    rng = np.random.default_rng(5)
    pos = rng.choice(N, size=20_000, replace=False)
    a[pos] = special[rng.integers(0, len(special), size=pos.size)]
    host = inputs.from_numpy(a, "f64")
    assert_sorted_parity(run_sort("f64", host, algo=algo), a, "f64")


@pytest.mark.parametrize("dist", ["uniform", "rootdup", "twodup", "zipf"])
def test_sort_pair(dist):
    host = inputs.generate(dist, "pair", N)
    assert_sorted_parity(run_sort("pair", host), inputs.to_numpy(host, "pair"), "pair")


@pytest.mark.parametrize("dist", inputs.REC_DISTS)
def test_sort_rec100(dist):
    host = inputs.generate(dist, "rec100", 60_001)
    assert_sorted_parity(run_sort("rec100", host), inputs.to_numpy(host, "rec100"), "rec100")


@pytest.mark.parametrize("dist", inputs.QUARTET_DISTS)
def test_sort_quartet(dist):
    host = inputs.generate(dist, "quartet", N)
    assert_sorted_parity(run_sort("quartet", host), inputs.to_numpy(host, "quartet"), "quartet")


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 5887, 5888, 5889, 2 ** 16 + 3])
def test_sort_quartet_sizes(n):
    # 5888 = 184 KiB / 32 B: the base-case capacity for quartets
    host = inputs.generate("lexdup", "quartet", n, seed=n + 3)
    assert_sorted_parity(run_sort("quartet", host), inputs.to_numpy(host, "quartet"), "quartet")


CAPACITY = {d: 184 * 1024 // inputs.ELEM_BYTES[d] for d in inputs.ELEM_BYTES}
BOUNDARY_DIST = {"u32": "uniform", "u64": "twodup", "f64": "normal", "pair": "rootdup",
                 "quartet": "uniform", "rec100": "uniform"}


@pytest.mark.parametrize("dtype", sorted(CAPACITY))
@pytest.mark.parametrize("rel", [-1, 0, 1, "2x+1", "small-1", "small", "small+1"])
def test_sort_around_base_case_capacity(dtype, rel):
    # the largest segment the shared-memory base case takes (184 KiB of
    # records) and its neighbours: one base-case call, or one level first;
    # and around 88 KiB, where the 512-thread base-case shape hands over to
    # the 1024-thread one
    cap = CAPACITY[dtype]
    small = 88 * 1024 // inputs.ELEM_BYTES[dtype]
    n = {"2x+1": 2 * cap + 1, "small-1": small - 1, "small": small,
         "small+1": small + 1}.get(rel)
    n = cap + rel if n is None else n
    host = inputs.generate(BOUNDARY_DIST[dtype], dtype, n, seed=cap % 97)
    assert_sorted_parity(run_sort(dtype, host), inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("dtype", ["u64", "pair", "quartet", "rec100"])
@pytest.mark.parametrize("k", [4, 32])
def test_sort_small_k_every_type(dtype, k):
    # few buckets per level: many levels, small class budgets
    dist = "rootdup" if dtype == "rec100" else "uniform"
    host = inputs.generate(dist, dtype, 60_001 if dtype == "rec100" else 200_003, seed=k)
    assert_sorted_parity(run_sort(dtype, host, k=k), inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("seed,alpha", [(1, 0.2), (0xDEADBEEF, 0.5), (7, 1.0)])
def test_sampling_choices_do_not_change_the_result(seed, alpha):
    # other sample positions and sizes give other splitters and levels, but
    # the sorted sequence is unique: identical to the oracle's bit for bit
    host = inputs.generate("zipf", "u64", 400_003, seed=11)
    got = run_sort("u64", host, seed=seed, alpha_scale=alpha, base_case=2048)
    np.testing.assert_array_equal(got, oracle.sort(inputs.to_numpy(host, "u64"), "u64"))


def test_sort_quartet_deep_ties():
    # long runs equal in the first word, then in the first two: the radix
    # passes of the base case move on to the second and third words, and
    # the splitters tie in their leading words
    n = 250_000
    host = inputs.generate("uniform", "quartet", n, seed=21)
    a = inputs.to_numpy(host, "quartet")
    a[:, 0] = np.uint64(7)
    a[: n // 2, 1] = a[: n // 2, 1] % np.uint64(3)
    a[n // 3: n // 2, 2] = a[n // 3: n // 2, 2] % np.uint64(5)
    a[::11, 0] = np.uint64(2 ** 64 - 1)
    a[5::13, :3] = np.uint64(0)
    host = inputs.from_numpy(a, "quartet")
    assert_sorted_parity(run_sort("quartet", host), a, "quartet")


@pytest.mark.parametrize("base_case", [32, 700])
@pytest.mark.parametrize("dist", ["uniform", "lexdup", "rootdup"])
def test_sort_quartet_small_base_case(base_case, dist):
    host = inputs.generate(dist, "quartet", 150_001, seed=base_case)
    got = run_sort("quartet", host, base_case=base_case)
    assert_sorted_parity(got, inputs.to_numpy(host, "quartet"), "quartet")


@pytest.mark.parametrize("dtype,dist", [("u64", "uniform"), ("u64", "exponential"), ("u32", "twodup"),
                                        ("f64", "normal"), ("pair", "zipf"), ("quartet", "lexdup")])
def test_sort_tree_walk_classifier(dtype, dist):
    host = inputs.generate(dist, dtype, N)
    got = run_sort(dtype, host, algo=ipsgpu.SAMPLESORT_TREE)
    assert_sorted_parity(got, inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("dtype", ["u64", "quartet"])
def test_sort_host_pinned_and_pageable(dtype):
    host = inputs.generate("uniform", dtype, 200_003, seed=8)
    inp = inputs.to_numpy(host, dtype)
    n = host.shape[0]
    pinned = host.pin_memory()
    out = torch.empty_like(host).pin_memory()
    work = torch.empty_like(host, device=DEV)
    with ipsgpu.Sorter(dtype) as s:
        s.sort_host(pinned.data_ptr(), out.data_ptr(), n, work.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK  # synchronizes the stream
        assert_sorted_parity(inputs.to_numpy(out, dtype), inp, dtype)
        assert torch.equal(pinned, host)  # the input is left as it was
        pageable = host.clone()  # pageable, sorted in place
        s.sort_host(pageable.data_ptr(), pageable.data_ptr(), n, work.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK
        assert_sorted_parity(inputs.to_numpy(pageable, dtype), inp, dtype)
        with pytest.raises(ipsgpu.IpsgpuError):
            s.sort_host(0, out.data_ptr(), n, work.data_ptr(), stream())
        with pytest.raises(ipsgpu.IpsgpuError):
            s.sort_host(pinned.data_ptr(), out.data_ptr(), n, work.data_ptr() + 4, stream())


def test_sort_host_two_streams_overlapped():
    # two sorters on two streams, each with its own device buffer, issued
    # back to back: the results are each the oracle's
    hosts = [inputs.generate(d, "u64", 1_000_003, seed=31 + i)
             for i, d in enumerate(("uniform", "twodup", "zipf", "exponential"))]
    pins = [h.pin_memory() for h in hosts]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]
    works = [torch.empty_like(hosts[0], device=DEV) for _ in range(2)]
    streams = [torch.cuda.Stream(DEV) for _ in range(2)]
    sorters = [ipsgpu.Sorter("u64") for _ in range(2)]
    try:
        for i in range(len(hosts)):
            j = i % 2
            sorters[j].sort_host(pins[i].data_ptr(), outs[i].data_ptr(), hosts[i].shape[0],
                                 works[j].data_ptr(), streams[j].cuda_stream)
        for j in range(2):
            assert sorters[j].status(streams[j].cuda_stream) == ipsgpu.OK
    finally:
        for s in sorters:
            s.close()
    for h, o in zip(hosts, outs):
        assert_sorted_parity(inputs.to_numpy(o, "u64"), inputs.to_numpy(h, "u64"), "u64")


def test_quartet_radix_unsupported():
    with pytest.raises(ipsgpu.IpsgpuError) as e:
        ipsgpu.Sorter("quartet", algo=ipsgpu.RADIX)
    assert e.value.code == ipsgpu.E_UNSUPPORTED


@pytest.mark.parametrize("dist", ["uniform", "twodup", "almostsorted", "exponential"])
@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
def test_sort_radix_variant(dtype, dist):
    host = inputs.generate(dist, dtype, N)
    got = run_sort(dtype, host, algo=ipsgpu.RADIX)
    assert_sorted_parity(got, inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("algo", [ipsgpu.SAMPLESORT, ipsgpu.RADIX])
@pytest.mark.parametrize("dist", ["uniform", "twodup", "eightdup"])
def test_sort_u32_buckets_of_2e14_key_values(algo, dist):
    # 2^22 keys below 2^22: the first level's children hold about 16,000 keys
    # over 2^13..2^14 key values each, which the base case sorts in one exact
    # pass in its large shape rather than in two-value digits in the small one
    host = inputs.generate(dist, "u32", 1 << 22, seed=21) & ((1 << 22) - 1)
    got = run_sort("u32", host, algo=algo)
    assert_sorted_parity(got, inputs.to_numpy(host, "u32"), "u32")


@pytest.mark.parametrize("pattern", ["pool", "clusters"])
@pytest.mark.parametrize("dtype", ["u64", "pair"])
def test_sort_duplicate_runs_in_small_ranges(pattern, dtype):
    # keys repeated many times: "pool" draws 2^22 keys from 2^22 / 50 random
    # 64-bit values, so a base-case digit often holds two or three values and
    # tens of copies (a small range peeled key by key); "clusters" draws runs
    # of 8 consecutive values, 8 copies each, so such ranges hold more
    # distinct keys than are peeled and fall back to ranking
    n = 1 << 22
    rng = np.random.default_rng(5 if pattern == "pool" else 6)
    if pattern == "pool":
        keys = rng.integers(0, 2 ** 64, size=n // 50, dtype=np.uint64)[rng.integers(0, n // 50, size=n)]
    else:
        base = rng.integers(0, 2 ** 63, size=n // 64, dtype=np.uint64)
        keys = base[rng.integers(0, n // 64, size=n)] + rng.integers(0, 8, size=n).astype(np.uint64)
    if dtype == "pair":
        a = np.stack([keys, np.arange(n, dtype=np.uint64)], axis=1)
    else:
        a = keys
    got = run_sort(dtype, inputs.from_numpy(a, dtype))
    assert_sorted_parity(got, a, dtype)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 1000, 23551, 23552, 23553, 24577,
                               49_155, 2 ** 17, 2 ** 17 + 1])
def test_sort_sizes(n):
    host = inputs.generate("uniform", "u64", n, seed=n + 11)
    assert_sorted_parity(run_sort("u64", host), inputs.to_numpy(host, "u64"), "u64")


@pytest.mark.parametrize("base_case", [32, 100, 4096])
def test_sort_small_base_case_forces_levels(base_case):
    # a small base case makes even modest inputs recurse through several levels
    host = inputs.generate("exponential", "u64", 200_000, seed=base_case)
    got = run_sort("u64", host, base_case=base_case)
    assert_sorted_parity(got, inputs.to_numpy(host, "u64"), "u64")


@pytest.mark.parametrize("k", [4, 16, 64])
def test_sort_small_k(k):
    host = inputs.generate("uniform", "u32", 250_000, seed=k)
    assert_sorted_parity(run_sort("u32", host, k=k), inputs.to_numpy(host, "u32"), "u32")


def test_sort_unaligned_view():
    host = inputs.generate("uniform", "u64", 100_001, seed=3)
    d = host.to(DEV)
    v = d[1:]
    with ipsgpu.Sorter("u64") as s:
        s.sort(v.data_ptr(), 100_000, stream())
        assert s.status(stream()) == ipsgpu.OK
    got = inputs.to_numpy(d.cpu(), "u64")
    assert got[0] == inputs.to_numpy(host, "u64")[0]
    assert_sorted_parity(got[1:], inputs.to_numpy(host[1:], "u64"), "u64")


def test_sort_on_side_stream_and_reuse():
    s_ = torch.cuda.Stream(DEV)
    with ipsgpu.Sorter("u64") as s:
        for seed in (1, 2, 3):
            host = inputs.generate("uniform", "u64", 70_000, seed=seed)
            d = host.to(DEV)
            torch.cuda.synchronize()
            s.sort(d.data_ptr(), 70_000, s_.cuda_stream)
            assert s.status(s_.cuda_stream) == ipsgpu.OK
            assert_sorted_parity(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(host, "u64"), "u64")


def test_bounded_wait_gives_up_with_timeout_status():
    with ipsgpu.Sorter("u64") as s:
        s.debug_bounded_wait(1000, stream())
        assert s.status(stream()) == ipsgpu.E_TIMEOUT
        # the status word was cleared and the sorter still works
        assert s.status(stream()) == ipsgpu.OK
        host = inputs.generate("uniform", "u64", 50_000)
        d = host.to(DEV)
        s.sort(d.data_ptr(), 50_000, stream())
        assert s.status(stream()) == ipsgpu.OK
    assert_sorted_parity(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(host, "u64"), "u64")
