"""The parity checks the GPU tests rely on, on the CPU: the record
signature is blind to the order of records but not to words moved between
records (a signature over words alone is blind to both), and the
record-by-record check catches a lost, duplicated or split record."""
import numpy as np
import pytest
import torch

from paper_2009_13569_gb300 import inputs
from _util import assert_records_intact, multiset_sig, record_index, record_sig


@pytest.mark.parametrize("dtype", ["pair", "quartet", "rec100"])
def test_record_sig_ignores_order_sees_split_records(dtype):
    n = 5000
    t = inputs.generate("uniform", dtype, n, seed=3)
    sig = record_sig(t, dtype)
    perm = torch.from_numpy(np.random.default_rng(1).permutation(n))
    assert record_sig(t[perm], dtype) == sig
    # swap the last 8 bytes of two records: the words' multiset is kept
    u = t.clone()
    if dtype == "rec100":
        u[[10, 20], 92:100] = u[[20, 10], 92:100]
    else:
        u[[10, 20], -1] = u[[20, 10], -1]
    assert multiset_sig(u) == multiset_sig(t)
    assert record_sig(u, dtype) != sig


@pytest.mark.parametrize("dtype", ["pair", "quartet", "rec100"])
def test_records_intact_check(dtype):
    n = 3000
    inp = inputs.to_numpy(inputs.generate("uniform", dtype, n, seed=4), dtype)
    got = inp[np.random.default_rng(2).permutation(n)]
    assert_records_intact(got, inp, dtype)
    assert (record_index(got, dtype) >= 0).all()
    bad = got.copy()
    bad[5] = got[6]  # a record duplicated, another lost
    with pytest.raises(AssertionError):
        assert_records_intact(bad, inp, dtype)
    split = got.copy()
    if dtype == "rec100":
        split[7, 50] ^= 1  # payload of one record altered
    else:
        # first key words swapped between two records (distinct: Uniform keys)
        split[7, 0], split[8, 0] = got[8, 0], got[7, 0]
    with pytest.raises(AssertionError):
        assert_records_intact(split, inp, dtype)
