"""GPU parity of one partitioning level (Sec. 3.1) through the C ABI:
bucket boundaries bit-exact against the oracle, each bucket the same
multiset of records, class ids of the branchless tree identical to the
oracle's binary search element by element."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu
from _util import DEV, assert_level_parity, stream, to_dev

pytestmark = pytest.mark.gpu

DTYPES = ["u32", "u64", "f64", "pair", "rec100", "quartet"]


def _input(dtype, n, dist, seed=5):
    if dtype == "f64":
        dist = "uniform" if dist != "normal" else dist
    elif dtype == "rec100":
        dist = "rootdup" if dist in ("rootdup", "twodup") else "uniform"
    elif dtype == "quartet" and dist == "twodup":
        dist = "lexdup"  # ties in the first two words
    return inputs.generate(dist, dtype, n, seed=seed)


def _splitters(host, dtype, m, seed):
    a = inputs.to_numpy(host, dtype)
    rng = np.random.default_rng(seed)
    pick = a[rng.integers(0, len(a), size=m)]
    return oracle.sort(pick, dtype)


def _run_level(dtype, host, spl, eq, offset=0, **params):
    n = inputs.count(host, dtype) - offset
    d = to_dev(host)
    dv = d[offset:]
    sd = to_dev(inputs.from_numpy(spl, dtype))
    K = 1 << int(np.ceil(np.log2(len(spl) + 1)))
    B = 2 * K if eq else K
    bb = torch.zeros(B + 1, dtype=torch.int64, device=DEV)
    with ipsgpu.Sorter(dtype, **params) as s:
        s.partition_level(dv.data_ptr(), n, sd.data_ptr(), len(spl), eq, bb.data_ptr(), stream())
        st = s.status(stream())
    assert st == ipsgpu.OK, ipsgpu.strerror(st)
    got = inputs.to_numpy(dv.cpu(), dtype)
    inp = inputs.to_numpy(host[offset:], dtype)
    cls, Bo = oracle.classify(inp, dtype, spl, eq)
    assert Bo == B
    assert_level_parity(got, bb.cpu().numpy().view(np.uint64), inp, dtype, cls, B)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("m,eq,dist", [(1, False, "uniform"), (1, True, "rootdup"),
                                        (7, True, "twodup"), (100, False, "uniform"),
                                        (127, True, "rootdup"), (255, False, "uniform")])
def test_partition_level_parity(dtype, m, eq, dist):
    if dtype == "rec100" and m > 63 and not eq:
        m = 63  # 4-record blocks: 64 classes x 400 B fit every buffer layout
    n = 200_003
    host = _input(dtype, n, dist)
    spl = _splitters(host, dtype, m, seed=m)
    _run_level(dtype, host, spl, eq)


@pytest.mark.parametrize("dtype", ["u64", "f64", "quartet"])
@pytest.mark.parametrize("m,eq", [(5, False), (255, False), (127, True)])
def test_partition_level_tree_walk_classifier(dtype, m, eq):
    # the classifier without the start-node table (every element walks from
    # the root, as Algorithm 1) gives the same level
    host = _input(dtype, 150_001, "twodup" if eq else "uniform", seed=m)
    spl = _splitters(host, dtype, m, seed=3 * m)
    _run_level(dtype, host, spl, eq, algo=ipsgpu.SAMPLESORT_TREE)


@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
def test_partition_level_unaligned_start(dtype):
    host = _input(dtype, 100_001, "uniform", seed=9)
    spl = _splitters(host, dtype, 31, seed=3)
    _run_level(dtype, host, spl, False, offset=1)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 129, 4096 * 3 + 5, 65_537])
def test_partition_level_small_and_ragged(n):
    host = _input("u64", n, "twodup", seed=n)
    spl = _splitters(host, "u64", 15, seed=n + 1)
    _run_level("u64", host, spl, True)
    _run_level("u64", host, spl, False)


def test_partition_level_all_equal_keys():
    host = inputs.generate("zero", "u64", 50_000)
    spl = np.zeros(3, dtype=np.uint64)
    _run_level("u64", host, spl, True)
    _run_level("u64", host, spl, False)


def test_partition_level_empty():
    bb = torch.full((5,), 7, dtype=torch.int64, device=DEV)
    spl = torch.zeros(1, dtype=torch.int64, device=DEV)
    d = torch.zeros(1, dtype=torch.int64, device=DEV)
    with ipsgpu.Sorter("u64") as s:
        s.partition_level(d.data_ptr(), 0, spl.data_ptr(), 1, True, bb.data_ptr(), stream())
    assert bb.cpu().tolist() == [0] * 5


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("m,eq", [(3, False), (7, True), (255, False), (127, True)])
def test_classify_ids_elementwise(dtype, m, eq):
    if dtype == "rec100" and m > 63:
        m = 63 if not eq else 31
    n = 100_000
    host = _input(dtype, n, "rootdup" if eq else "uniform", seed=m)
    spl = _splitters(host, dtype, m, seed=2 * m)
    d = to_dev(host)
    sd = to_dev(inputs.from_numpy(spl, dtype))
    out = torch.empty(n, dtype=torch.int32, device=DEV)
    with ipsgpu.Sorter(dtype) as s:
        s.classify(d.data_ptr(), n, sd.data_ptr(), m, eq, out.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK
    cls, _ = oracle.classify(inputs.to_numpy(host, dtype), dtype, spl, eq)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), cls)


@pytest.mark.parametrize("dtype", ["u32", "u64", "pair"])
@pytest.mark.parametrize("shift,bits", [(0, 8), (3, 5), (24, 8), (56, 8), (20, 1)])
def test_radix_level_parity(dtype, shift, bits):
    if dtype == "u32" and shift + bits > 32:
        shift = 32 - bits
    n = 150_001
    host = inputs.generate("uniform", dtype, n, seed=shift * 7 + bits)
    d = to_dev(host)
    B = 1 << bits
    bb = torch.zeros(B + 1, dtype=torch.int64, device=DEV)
    with ipsgpu.Sorter(dtype) as s:
        s.radix_level(d.data_ptr(), n, shift, bits, bb.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK
    inp = inputs.to_numpy(host, dtype)
    cls, _ = oracle.radix_classify(inp, dtype, shift, bits)
    assert_level_parity(inputs.to_numpy(d.cpu(), dtype), bb.cpu().numpy().view(np.uint64),
                        inp, dtype, cls, B)


def test_invalid_arguments_are_rejected():
    d = torch.zeros(16, dtype=torch.int64, device=DEV)
    bb = torch.zeros(600, dtype=torch.int64, device=DEV)
    with ipsgpu.Sorter("u64") as s:
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            s.partition_level(d.data_ptr(), 16, d.data_ptr(), 200, True, bb.data_ptr())
        assert e.value.code == ipsgpu.E_INVAL  # 2 * 256 classes > k
        with pytest.raises(ipsgpu.IpsgpuError):
            s.partition_level(d.data_ptr() + 4, 8, d.data_ptr(), 3, False, bb.data_ptr())
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            s.partition_level(d.data_ptr(), 8, d.data_ptr() + 4, 3, False, bb.data_ptr())
        assert e.value.code == ipsgpu.E_INVAL  # misaligned splitters
        out = torch.zeros(16, dtype=torch.int32, device=DEV)
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            s.classify(d.data_ptr(), 8, d.data_ptr() + 4, 3, False, out.data_ptr())
        assert e.value.code == ipsgpu.E_INVAL
    with ipsgpu.Sorter("quartet") as s:
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            s.partition_level(d.data_ptr() + 8, 2, d.data_ptr(), 1, False, bb.data_ptr())
        assert e.value.code == ipsgpu.E_INVAL  # quartets need 16-byte alignment
    with pytest.raises(ipsgpu.IpsgpuError) as e:
        ipsgpu.Sorter("f64", algo=ipsgpu.RADIX)
    assert e.value.code == ipsgpu.E_UNSUPPORTED


@pytest.mark.parametrize("dtype,spl_vals", [
    ("u64", [0, 1, 1 << 63, (1 << 64) - 2, (1 << 64) - 1]),
    ("u64", [5]),
    ("u64", [(1 << 64) - 1] * 3),
    ("u32", [0, 7, (1 << 31), (1 << 32) - 2, (1 << 32) - 1]),
    ("u32", [(1 << 32) - 3, (1 << 32) - 2]),
])
@pytest.mark.parametrize("eq", [False, True])
def test_partition_level_extreme_splitters(dtype, spl_vals, eq):
    # splitters at the ends of the key range and keys outside the splitter
    # range exercise every clamp of the classifier's start-node table
    n = 120_001
    host = inputs.generate("uniform", dtype, n, seed=len(spl_vals) + eq)
    a = inputs.to_numpy(host, dtype)
    a[::97] = spl_vals[0]
    a[1::89] = spl_vals[-1]
    a[2::83] = 0
    a[3::79] = np.iinfo(a.dtype).max
    host = inputs.from_numpy(a, dtype)
    spl = np.array(sorted(spl_vals), dtype=a.dtype)
    _run_level(dtype, host, spl, eq)


@pytest.mark.parametrize("dist", ["exponential", "zipf", "almostsorted", "eightdup"])
def test_partition_level_clustered_splitters(dist):
    host = _input("u64", 200_003, dist, seed=17)
    spl = _splitters(host, "u64", 255, seed=4)
    _run_level("u64", host, spl, False)
    spl = _splitters(host, "u64", 127, seed=5)
    _run_level("u64", host, spl, True)
