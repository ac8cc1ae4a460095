"""ipsgpu_partition_level_noalloc against ipsgpu_partition_level and the oracle.

The no-alloc entry point serves callers that cannot allocate device memory
(graph capture, allocator callbacks, services that reserve all memory up
front): it keeps its scratch in a fixed device array of the library instead
of a sorter's allocations.  Its result must equal the sorter-based level:
identical bucket boundaries (also equal to the oracle's classification
counts) and, bucket by bucket, the same multiset of elements (the order
inside a bucket is unspecified for both).  Two calls in
a row check that the shared array's leftovers from one call do not leak into
the next; between them a sorter with fewer classes and smaller blocks is
created (less classification shared memory than the fixed array's level
launches with), which must not disturb the second call.  This file is named
so that pytest collects it last; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu

pytestmark = pytest.mark.gpu


def _rows(a, dtype):
    if dtype in ("pair", "rec100", "quartet"):
        v = np.ascontiguousarray(a).view(np.uint8).reshape(len(a), -1)
        return v[np.lexsort(v.T[::-1])]
    return np.sort(a)


@pytest.mark.parametrize("dtype,n,m,eq,dist", [
    ("u64", 1_000_003, 255, False, "uniform"),
    ("u32", 300_001, 127, True, "twodup"),
    ("pair", 200_003, 63, False, "uniform"),
    ("quartet", 150_001, 127, True, "lexdup"),
    ("f64", 250_001, 100, False, "normal"),
    # 100-byte records: 4-byte alignment, 4-record (400-byte) blocks
    ("rec100", 100_003, 63, False, "uniform"),
    ("rec100", 60_001, 31, True, "rootdup"),
    # enough u32 keys that the fixed array's 64-stripe cap applies (a sorter
    # would cut this level into 2 stripes per SM)
    ("u32", 5_000_011, 255, False, "uniform"),
])
def test_noalloc_matches_sorter_level_twice(dtype, n, m, eq, dist):
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    K = 1 << int(np.ceil(np.log2(m + 1)))
    B = 2 * K if eq else K
    for call in range(2):
        host = inputs.generate(dist, dtype, n, seed=100 + call)
        a = inputs.to_numpy(host, dtype)
        pick = a[np.random.default_rng(call).integers(0, n, size=m)]
        spl_np = oracle.sort(pick, dtype)
        spl = inputs.from_numpy(spl_np, dtype).to(dev)
        # the bucket boundaries the paper's classification gives (the oracle)
        cls, B_or = oracle.classify(a, dtype, spl_np, eq)
        assert B_or == B
        bb_oracle = np.concatenate([[0], np.cumsum(np.bincount(cls, minlength=B))]).astype(np.uint64)

        ref = host.to(dev)
        bb_ref = torch.zeros(B + 1, dtype=torch.int64, device=dev)
        with ipsgpu.Sorter(dtype) as s:
            s.partition_level(ref.data_ptr(), n, spl.data_ptr(), m, eq, bb_ref.data_ptr(), stream)
            assert s.status(stream) == ipsgpu.OK

        got = host.to(dev)
        bb = torch.full((B + 1,), -1, dtype=torch.int64, device=dev)
        ipsgpu.partition_level_noalloc(dtype, got.data_ptr(), n, spl.data_ptr(), m, eq,
                                       bb.data_ptr(), stream)
        torch.cuda.synchronize(dev)
        bbn = bb.cpu().numpy().view(np.uint64)
        assert bbn[-1] == n, "kernel-side error reported by the no-alloc level"
        if call == 0:
            # a sorter whose classification needs less shared memory
            small = ipsgpu.Sorter(dtype, k=64, block_bytes=512 if dtype == "rec100" else 256)
        np.testing.assert_array_equal(bbn, bb_ref.cpu().numpy().view(np.uint64))
        np.testing.assert_array_equal(bbn, bb_oracle)
        g = inputs.to_numpy(got.cpu(), dtype)
        r = inputs.to_numpy(ref.cpu(), dtype)
        for j in range(B):
            lo, hi = int(bbn[j]), int(bbn[j + 1])
            if hi > lo:
                np.testing.assert_array_equal(_rows(g[lo:hi], dtype), _rows(r[lo:hi], dtype))
    small.close()


def test_noalloc_rejects_misaligned_splitters():
    d = torch.zeros(64, dtype=torch.int64, device="cuda:0")
    bb = torch.zeros(9, dtype=torch.int64, device="cuda:0")
    with pytest.raises(ipsgpu.IpsgpuError) as e:
        ipsgpu.partition_level_noalloc("quartet", d.data_ptr(), 8, d.data_ptr() + 8, 3, False,
                                       bb.data_ptr())
    assert e.value.code == ipsgpu.E_INVAL


def test_noalloc_rejects_too_many_classes():
    d = torch.zeros(16, dtype=torch.int64, device="cuda:0")
    bb = torch.zeros(600, dtype=torch.int64, device="cuda:0")
    with pytest.raises(ipsgpu.IpsgpuError) as e:
        ipsgpu.partition_level_noalloc("u64", d.data_ptr(), 16, d.data_ptr(), 255, True,
                                       bb.data_ptr())
    assert e.value.code == ipsgpu.E_INVAL
