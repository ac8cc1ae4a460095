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


def record_index(a, dtype):
    """Original index carried by every generated record (numpy): the value
    word of pair and quartet, payload bytes 10..17 (little-endian) of
    100-byte records."""
    if dtype == "pair":
        return a[:, 1].astype(np.int64)
    if dtype == "quartet":
        return a[:, 3].astype(np.int64)
    if dtype == "rec100":
        return np.ascontiguousarray(a[:, 10:18]).view("<u8").reshape(-1).astype(np.int64)
    raise ValueError(dtype)


def assert_records_intact(got, inp, dtype):
    """Every output record is a whole input record, each input record
    appears exactly once (record by record, through the original index
    each generated record carries)."""
    n = len(inp)
    assert len(got) == n
    idx = record_index(got, dtype)
    assert idx.min() >= 0 and idx.max() < n, "index payload out of range"
    assert np.bincount(idx, minlength=n).max() == 1, "a record lost or duplicated"
    np.testing.assert_array_equal(got, inp[idx], err_msg="a record came apart")


def assert_record_parity(got, inp, dtype):
    """Sort parity for records, element by element: the key sequence equals
    the oracle's (the sorted key sequence is unique) and the records are the
    input's, each whole and once (any order of equal keys is correct)."""
    ref = oracle.sort(inp, dtype)
    np.testing.assert_array_equal(keys_of(got, dtype), keys_of(ref, dtype))
    assert_records_intact(got, inp, dtype)


def _mix64(z):
    # splitmix64's finalizer (Steele, Lea, Flood 2014) on int64 bit patterns
    z = (z ^ inputs._lsr(z, 30)) * inputs._s64(0xBF58476D1CE4E5B9)
    z = (z ^ inputs._lsr(z, 27)) * inputs._s64(0x94D049BB133111EB)
    return z ^ inputs._lsr(z, 31)


def record_sig(t, dtype, chunk=1 << 24):
    """Order-independent signature of the records of a device tensor (one
    record per row): the words of each record are hashed together into one
    64-bit value, and the signature is the count, sum, xor and sum of
    squares of those values mod 2^64.  Any permutation of the records keeps
    it; a word moved from one record to another changes it with
    overwhelming odds (which a signature over words alone does not see)."""
    n = t.shape[0]
    acc = [n, 0, 0, 0]
    m = (1 << 64) - 1
    for a in range(0, n, chunk):
        x = t[a:a + chunk]
        if dtype == "rec100":
            w = x.contiguous().view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        else:
            w = x.reshape(x.shape[0], -1).view(torch.int64)
        h = torch.full((w.shape[0],), inputs._s64(0x9E3779B97F4A7C15), dtype=torch.int64,
                       device=t.device)
        for j in range(w.shape[1]):
            h = _mix64(h ^ (w[:, j] + inputs._s64(0x9E3779B97F4A7C15 * (j + 1))))
        acc[1] = (acc[1] + int(h.sum().item())) & m
        y = h
        while y.numel() > 1:
            if y.numel() % 2:
                y = torch.cat([y, torch.zeros(1, dtype=y.dtype, device=y.device)])
            y = y[0::2] ^ y[1::2]
        acc[2] ^= int(y[0].item()) & m
        acc[3] = (acc[3] + int((h * h).sum().item())) & m
    return tuple(acc)


def records_intact_dev(got, inp, dtype, chunk=1 << 24):
    """Device form of assert_records_intact (for inputs of many GiB):
    True iff the original indices of got are a permutation of 0..n-1 and
    every record of got equals the input record of its index."""
    n = got.shape[0]
    idx = torch.empty(n, dtype=torch.int64, device=got.device)
    for a in range(0, n, chunk):
        x = got[a:a + chunk]
        if dtype == "pair":
            idx[a:a + chunk] = x[:, 1]
        elif dtype == "quartet":
            idx[a:a + chunk] = x[:, 3]
        elif dtype == "rec100":
            b = x[:, 10:18].to(torch.int64)
            v = torch.zeros(x.shape[0], dtype=torch.int64, device=x.device)
            for j in range(8):
                v |= b[:, j] << (8 * j)
            idx[a:a + chunk] = v
        else:
            raise ValueError(dtype)
    if int(idx.min().item()) < 0 or int(idx.max().item()) >= n:
        return False
    cnt = torch.zeros(n, dtype=torch.int32, device=got.device)
    cnt.index_add_(0, idx, torch.ones(n, dtype=torch.int32, device=got.device))
    if not bool((cnt == 1).all().item()):
        return False
    del cnt
    for a in range(0, n, chunk):
        if not torch.equal(got[a:a + chunk], inp[idx[a:a + chunk]]):
            return False
    return True
