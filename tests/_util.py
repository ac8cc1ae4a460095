"""Helpers shared by the GPU parity tests (device placement, comparisons
against the oracle).  Expected values always come from the oracle package."""
import numpy as np
import torch

import oracle
from paper_2009_13569_gb300 import inputs, ipsgpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def stream():
    return torch.cuda.current_stream(DEV).cuda_stream


def to_dev(host):
    return host.to(DEV).contiguous()


def keys_of(a, dtype):
    """Order keys of a numpy array in oracle conventions, as something numpy
    compares in key order (rows of bytes for rec100)."""
    if dtype == "pair":
        return a[:, 0]
    if dtype == "rec100":
        return a[:, :10]
    if dtype == "quartet":
        return a[:, :3]
    if dtype == "f64":
        b = a.view(np.uint64)
        return np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))
    return a


def rows(a, dtype):
    """Canonically ordered copy of the records, to compare multisets."""
    if dtype in ("pair", "rec100", "quartet"):
        a = np.ascontiguousarray(a)
        v = a.view(np.uint8).reshape(len(a), a.itemsize * int(np.prod(a.shape[1:])))
        order = np.lexsort(v.T[::-1])
        return v[order]
    return np.sort(a.view(np.uint64) if dtype == "f64" else a)


def assert_sorted_parity(got, inp, dtype):
    """GPU sort output vs the oracle: identical keys everywhere; for u32 /
    u64 / f64 identical bits, for pair / rec100 the same multiset of records
    (which, with identical key sequences, means every equal-key run holds
    the same records)."""
    ref = oracle.sort(inp, dtype)
    if dtype in ("u32", "u64"):
        np.testing.assert_array_equal(got, ref)
        return
    if dtype == "f64":
        np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))
        return
    np.testing.assert_array_equal(keys_of(got, dtype), keys_of(ref, dtype))
    np.testing.assert_array_equal(rows(got, dtype), rows(inp, dtype))


def assert_level_parity(got, bb, inp, dtype, cls, B):
    """Partition-level parity: bucket boundaries bit-exact, each bucket the
    same multiset of records as the oracle's bucket."""
    ref, rbb = oracle.partition(inp, dtype, cls, B)
    np.testing.assert_array_equal(np.asarray(bb, dtype=np.uint64), rbb)
    for j in range(B):
        lo, hi = int(rbb[j]), int(rbb[j + 1])
        if hi - lo:
            np.testing.assert_array_equal(rows(got[lo:hi], dtype), rows(ref[lo:hi], dtype),
                                          err_msg="bucket %d" % j)


def run_sort(dtype, host, **params):
    n = inputs.count(host, dtype)
    d = to_dev(host)
    with ipsgpu.Sorter(dtype, **params) as s:
        s.sort(d.data_ptr(), n, stream())
        st = s.status(stream())
    assert st == ipsgpu.OK, ipsgpu.strerror(st)
    return inputs.to_numpy(d.cpu(), dtype)


def multiset_sig(t):
    """Order-independent signature of a device tensor's words (count, sum,
    xor, sum of squares, each mod 2^64): equal for any permutation, and
    changed by a lost, duplicated or altered word with overwhelming odds."""
    if t.dtype == torch.uint8:
        w = t.contiguous().view(torch.int32).reshape(-1).to(torch.int64)
    elif t.element_size() == 4:
        w = t.reshape(-1).view(torch.int32).to(torch.int64)
    else:
        w = t.reshape(-1).view(torch.int64)
    acc = [w.numel(), 0, 0, 0]
    for a in range(0, w.numel(), 1 << 27):
        x = w[a:a + (1 << 27)]
        acc[1] = (acc[1] + int(x.sum().item())) & ((1 << 64) - 1)
        while x.numel() > 1:
            if x.numel() % 2:
                x = torch.cat([x, torch.zeros(1, dtype=x.dtype, device=x.device)])
            x = x[0::2] ^ x[1::2]
        acc[2] ^= int(x[0].item()) & ((1 << 64) - 1)
        y = w[a:a + (1 << 27)]
        acc[3] = (acc[3] + int((y * y).sum().item())) & ((1 << 64) - 1)
    return tuple(acc)


def keys_nondecreasing(t, dtype, chunk=1 << 27):
    """Keys in non-decreasing order (unsigned; f64 by its order map;
    lexicographic for quartet and rec100 keys)."""
    if dtype == "rec100":
        chunk = min(chunk, 1 << 23)  # 10 int64 temporaries per record
    n = t.shape[0]
    for a in range(0, max(n - 1, 0), chunk):
        x = t[a:a + chunk + 1]
        if dtype == "u32":
            k = x.to(torch.int64) & 0xFFFFFFFF
        elif dtype in ("u64", "pair"):
            k = (x[:, 0] if dtype == "pair" else x) ^ (-(1 << 63))
        elif dtype == "f64":
            b = x.view(torch.int64)
            k = torch.where(b < 0, ~b, b | (-(1 << 63))) ^ (-(1 << 63))
        elif dtype == "rec100":
            # 10-byte keys compared as unsigned bytes: bytes 0..6 big-endian
            # in one int64 (56 bits, non-negative), bytes 7..9 in another
            kb = x[:, :10].to(torch.int64)
            hi = torch.zeros(kb.shape[0], dtype=torch.int64, device=x.device)
            for j in range(7):
                hi = hi * 256 + kb[:, j]
            lo = kb[:, 7] * 65536 + kb[:, 8] * 256 + kb[:, 9]
            dh = hi[1:] - hi[:-1]
            if not bool(((dh > 0) | ((dh == 0) & (lo[1:] >= lo[:-1]))).all().item()):
                return False
            continue
        elif dtype == "quartet":
            # lexicographic on the three key words, each unsigned
            w = [x[:, j] ^ (-(1 << 63)) for j in range(3)]
            lt = w[2][1:] < w[2][:-1]
            for j in (1, 0):
                lt = (w[j][1:] < w[j][:-1]) | ((w[j][1:] == w[j][:-1]) & lt)
            if bool(lt.any().item()):
                return False
            continue
        else:
            raise ValueError(dtype)
        if not bool((k[1:] >= k[:-1]).all().item()):
            return False
    return True
