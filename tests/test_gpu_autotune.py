"""The autotuner on the GPU: the parameters it picks for a segmented batch
and for plain arrays sort correctly (checked against the oracle)."""
import pytest
import torch

from paper_2009_13569_gb300 import autotune, inputs, ipsgpu
from _util import DEV, assert_sorted_parity, stream, to_dev

pytestmark = pytest.mark.gpu


def test_autotune_segmented_params_sort_correctly():
    lengths = inputs.segment_lengths(200, 4, 17, seed=12)
    data, offsets = inputs.segmented_batch(lengths, seed=12, device=DEV)
    best, table = autotune.tune_segmented(torch, data, offsets, "u64", reps=2)
    # every (k, block bytes) pair of the grid is accepted and timed
    kb = {(p["k"], p["block_bytes"]) for p, t in table}
    assert kb == set(autotune.KB_PAIRS)
    assert all(t is not None and t > 0 for _, t in table), table
    d = data.clone()
    with ipsgpu.Sorter("u64", **best) as s:
        s.sort_segmented(d.data_ptr(), d.numel(), offsets.data_ptr(), lengths.numel(), stream())
        assert s.status(stream()) == ipsgpu.OK
    got, inp, o = inputs.to_numpy(d.cpu(), "u64"), inputs.to_numpy(data.cpu(), "u64"), offsets.cpu().numpy()
    for i in range(len(o) - 1):
        if o[i + 1] - o[i] > 1:
            assert_sorted_parity(got[o[i]:o[i + 1]], inp[o[i]:o[i + 1]], "u64")


@pytest.mark.parametrize("dtype", ["u32", "pair"])
def test_autotune_array_params_sort_correctly(dtype):
    host = inputs.generate("zipf", dtype, 1 << 20, seed=5)
    sample = to_dev(host)
    best, _ = autotune.tune_array(torch, sample, dtype, reps=2)
    d = to_dev(host)
    with ipsgpu.Sorter(dtype, **best) as s:
        s.sort(d.data_ptr(), host.shape[0], stream())
        assert s.status(stream()) == ipsgpu.OK
    assert_sorted_parity(inputs.to_numpy(d.cpu(), dtype), inputs.to_numpy(host, dtype), dtype)
