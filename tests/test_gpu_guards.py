"""Out-of-bounds write detection on the GPU without a sanitizer: every device
buffer of a sorter lies between guard zones (ipsgpu_debug_check_guards).
Each operation below (every element type and algorithm, tiny, ragged and
multi-level sizes, batched and segmented runs that fill the scratch
capacities, invalid batch entries, one-level calls) must leave every guard
intact, besides giving the oracle's result."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu
from _util import DEV, assert_sorted_parity, stream, to_dev

pytestmark = pytest.mark.gpu


def _guards_intact(s):
    bad = s.check_guards()
    assert bad is None, "guard zone of device buffer %d changed" % bad


@pytest.mark.parametrize("dtype,dist", [("u32", "twodup"), ("u64", "uniform"), ("f64", "normal"),
                                        ("pair", "zipf"), ("quartet", "lexdup"),
                                        ("rec100", "rootdup")])
@pytest.mark.parametrize("n", [1, 33, 5889, 150_001])
def test_sorts_keep_guards(dtype, dist, n):
    host = inputs.generate(dist, dtype, n, seed=n)
    d = to_dev(host)
    with ipsgpu.Sorter(dtype) as s:
        s.sort(d.data_ptr(), n, stream())
        assert s.status(stream()) == ipsgpu.OK
        _guards_intact(s)
    if n > 1:
        assert_sorted_parity(inputs.to_numpy(d.cpu(), dtype), inputs.to_numpy(host, dtype), dtype)


@pytest.mark.parametrize("algo", [ipsgpu.RADIX, ipsgpu.SAMPLESORT_TREE])
def test_other_classifiers_keep_guards(algo):
    host = inputs.generate("exponential", "u64", 400_003, seed=3)
    d = to_dev(host)
    with ipsgpu.Sorter("u64", algo=algo, base_case=64) as s:  # many levels
        s.sort(d.data_ptr(), host.shape[0], stream())
        assert s.status(stream()) == ipsgpu.OK
        _guards_intact(s)
    assert_sorted_parity(inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(host, "u64"), "u64")


def test_batched_runs_at_capacity_keep_guards():
    # 20,000 tiny arrays and a small arena: many waves, full rings and lists
    lengths = inputs.segment_lengths(20_000, 0, 9, seed=4)
    data, offsets = inputs.segmented_batch(lengths, seed=4)
    d = to_dev(data)
    off = offsets.to(DEV)
    with ipsgpu.Sorter("u64", arena_bytes=1 << 21) as s:
        s.sort_segmented(d.data_ptr(), data.shape[0], off.data_ptr(), len(lengths), stream())
        assert s.status(stream()) == ipsgpu.OK
        _guards_intact(s)
        # a batch with a misaligned entry is reported and skipped
        segs = torch.tensor([[d.data_ptr(), 1000], [d.data_ptr() + 4, 10]], dtype=torch.int64,
                            device=DEV)
        s.sort_batch(segs.data_ptr(), 2, stream())
        assert s.status(stream()) == ipsgpu.E_INVAL
        _guards_intact(s)


@pytest.mark.parametrize("dtype,m,eq", [("u64", 255, False), ("quartet", 127, True),
                                        ("rec100", 31, True)])
def test_one_level_calls_keep_guards(dtype, m, eq):
    n = 100_003
    host = inputs.generate("uniform", dtype, n, seed=m)
    a = inputs.to_numpy(host, dtype)
    spl = oracle.sort(a[np.random.default_rng(m).integers(0, n, size=m)], dtype)
    sd = to_dev(inputs.from_numpy(spl, dtype))
    d = to_dev(host)
    K = 1 << int(np.ceil(np.log2(m + 1)))
    B = 2 * K if eq else K
    bb = torch.zeros(B + 1, dtype=torch.int64, device=DEV)
    cls = torch.zeros(n, dtype=torch.int32, device=DEV)
    with ipsgpu.Sorter(dtype) as s:
        s.classify(d.data_ptr(), n, sd.data_ptr(), m, eq, cls.data_ptr(), stream())
        s.partition_level(d.data_ptr(), n, sd.data_ptr(), m, eq, bb.data_ptr(), stream())
        assert s.status(stream()) == ipsgpu.OK
        _guards_intact(s)
    ref, rbb = oracle.partition_level(a, dtype, spl, eq)
    np.testing.assert_array_equal(bb.cpu().numpy().view(np.uint64), rbb)
