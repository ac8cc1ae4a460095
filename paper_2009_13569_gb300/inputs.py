"""Seeded synthetic inputs: the benchmark distributions of Sec. 6 of Axtmann et
al. (Uniform, Exponential, RootDup, TwoDup, EightDup, AlmostSorted, Zipf,
Sorted, ReverseSorted, Zero) for the element types of the same section.

This module holds none of the sorting method's arithmetic; it only makes
inputs.  It is written with plain torch integer ops so the same code runs on
the CPU (tests, oracle inputs) and on the GPU (large benchmark inputs) and
yields identical bits on both.

Random numbers come from splitmix64 (Steele, Lea and Flood, OOPSLA 2014) used
as a counter-based generator: draw i of stream s is the (i+1)-th output of a
splitmix64 sequence whose state starts at ``seed ^ stream_constant(s)``.

Storage formats (what the GPU library and ``to_numpy`` see):
  u32 -> torch.int32 (n,)   bit pattern of the unsigned value
  u64 -> torch.int64 (n,)   bit pattern of the unsigned value
  f64 -> torch.float64 (n,)
  pair -> torch.int64 (n, 2): key, value
  rec100 -> torch.uint8 (n, 100): 10-byte key, 90-byte payload
  quartet -> torch.int64 (n, 4): key words a, b, c (lexicographic), value

Quartet keys: "uniform" draws a, b and c as three independent uniform 64-bit
words (the Quartet workload of Sec. 6); every other integer distribution
draws its 64-bit value v and stores it as a = v >> 40, b = (v >> 20) mod
2^20, c = v mod 2^20, an order-preserving embedding (so the sorted key
sequence is that of v); "lexdup" draws a and b from {0, 1, 2, 3} and c
uniform, so that most comparisons are decided by the third word.
"""
import math

import numpy as np
import torch

DEFAULT_SEED = 0x1B54A32D192ED03
GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

INT_DISTS = ("uniform", "exponential", "rootdup", "twodup", "eightdup",
             "almostsorted", "zipf", "sorted", "reversesorted", "zero")
F64_DISTS = ("uniform", "normal")
REC_DISTS = ("uniform", "rootdup")
QUARTET_DISTS = INT_DISTS + ("lexdup",)
ELEM_BYTES = {"u32": 4, "u64": 8, "f64": 8, "pair": 16, "rec100": 100, "quartet": 32}


def _s64(x):
    """Python int (mod 2^64) -> signed int64 value with the same bits."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(z, s):
    """Logical right shift of int64 bit patterns."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64(idx, seed):
    """Counter-based splitmix64: output number idx (0-based) of the stream
    whose state starts at ``seed``.  idx is an int64 tensor; returns int64
    bit patterns."""
    z = idx * _s64(GOLDEN) + _s64(seed + GOLDEN)
    z = (z ^ _lsr(z, 30)) * _s64(MIX1)
    z = (z ^ _lsr(z, 27)) * _s64(MIX2)
    return z ^ _lsr(z, 31)


def splitmix64_py(i, seed):
    """Pure-Python splitmix64 (same definition), for checking the tensor one."""
    m = (1 << 64) - 1
    z = (seed + (i + 1) * GOLDEN) & m
    z = ((z ^ (z >> 30)) * MIX1) & m
    z = ((z ^ (z >> 27)) * MIX2) & m
    return z ^ (z >> 31)


def _stream(seed, s):
    return (seed ^ (s * 0xD1B54A32D192ED03)) & ((1 << 64) - 1)


def _draw(n, seed, stream, device):
    idx = torch.arange(n, dtype=torch.int64, device=device)
    return splitmix64(idx, _stream(seed, stream))


def _draw_at(idx, seed, stream):
    """Draws of stream `stream` at the given indices (same values as _draw)."""
    return splitmix64(idx, _stream(seed, stream))


def _umod(x, n):
    """Unsigned (x mod 2^64) mod n for int64 bit patterns, 0 < n < 2^62."""
    if n & (n - 1) == 0:
        return x & (n - 1)
    hi = _lsr(x, 1) % n
    return (hi * 2 + (x & 1)) % n


def _zipf_cdf(nvals=1_000_000, s=0.75):
    w = np.arange(1, nvals + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _int_values(dist, n, width, seed, device, i=None):
    """Values of an integer distribution as int64 tensors in [0, 2^width):
    the values at global positions i (an int64 tensor; default all of
    0..n-1) of an n-element input."""
    top = 1 << width
    if i is None:
        i = torch.arange(n, dtype=torch.int64, device=device)
    if dist == "uniform":
        r = _draw_at(i, seed, 1)
        return r if width == 64 else _lsr(r, 64 - width)
    if dist == "exponential":
        # pick e uniform in [0, log2 n), value uniform in [2^e, 2^(e+1))
        lg = max(1, int(math.floor(math.log2(max(n, 2)))))
        e = _umod(_draw_at(i, seed, 2), lg)
        r = _lsr(_draw_at(i, seed, 3), 1)
        return (torch.ones_like(e) << e) + (r & ((torch.ones_like(e) << e) - 1))
    if dist == "rootdup":
        return i % max(1, math.isqrt(n))
    if dist == "twodup":
        return _umod(i * i + n // 2, n)
    if dist == "eightdup":
        x = i * i
        x = x * x
        x = x * x
        return _umod(x + n // 2, n)
    if dist == "almostsorted":
        a = i.clone()
        swaps = math.isqrt(n)
        if n >= 2 and swaps > 0:
            p = _umod(_draw(swaps, seed, 4, "cpu"), n - 1).tolist()
            cur = {}
            for q in p:  # adjacent swaps applied in sequence
                x, y = cur.get(q, q), cur.get(q + 1, q + 1)
                cur[q], cur[q + 1] = y, x
            pos = torch.tensor(list(cur.keys()), dtype=torch.int64, device=device)
            val = torch.tensor(list(cur.values()), dtype=torch.int64, device=device)
            if i.numel():
                i0, i1 = int(i[0]), int(i[-1]) + 1  # i is a contiguous range
                keep = (pos >= i0) & (pos < i1)
                a[pos[keep] - i0] = val[keep]
        return a
    if dist == "zipf":
        cdf = torch.from_numpy(_zipf_cdf()).to(device)
        u = _lsr(_draw_at(i, seed, 5), 11).to(torch.float64) * 2.0 ** -53
        v = torch.searchsorted(cdf, u, right=True) + 1
        return torch.clamp(v, max=cdf.numel())
    if dist in ("sorted", "reversesorted"):
        # sorted uniform input, stratified: value j lies in [j*w, (j+1)*w)
        w = min(max(1, top // max(n, 1)), 1 << 62)
        j = i if dist == "sorted" else (n - 1) - i
        r = _draw_at(j, seed, 6)
        return j * w + _umod(r, w) if w > 1 else j
    if dist == "zero":
        return torch.zeros_like(i)
    raise ValueError("unknown distribution %r" % dist)


def _quartet_keys(dist, n, seed, device, i=None):
    """Key words (a, b, c) of a quartet input at global positions i."""
    if i is None:
        i = torch.arange(n, dtype=torch.int64, device=device)
    if dist == "uniform":
        return _draw_at(i, seed, 40), _draw_at(i, seed, 41), _draw_at(i, seed, 42)
    if dist == "lexdup":
        return _draw_at(i, seed, 43) & 3, _draw_at(i, seed, 44) & 3, _draw_at(i, seed, 45)
    v = _int_values(dist, n, 64, seed, device, i)
    return _lsr(v, 40), _lsr(v, 20) & 0xFFFFF, v & 0xFFFFF


def generate_into(out, dist, dtype, seed=DEFAULT_SEED, chunk=1 << 26):
    """Fill `out` (storage format above, any device) with the same values as
    generate(dist, dtype, len(out), seed), chunk by chunk, so that inputs of
    many GiB need little temporary memory.  u32, u64, pair and quartet."""
    n = out.shape[0]
    width = 32 if dtype == "u32" else 64
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        i = torch.arange(i0, i1, dtype=torch.int64, device=out.device)
        if dtype == "quartet":
            for w, x in enumerate(_quartet_keys(dist, n, seed, out.device, i)):
                out[i0:i1, w] = x
            out[i0:i1, 3] = i
            del i
            continue
        v = _int_values(dist, n, width, seed, out.device, i)
        if dtype == "u64":
            out[i0:i1] = v
        elif dtype == "u32":
            out[i0:i1] = (v - ((v >> 31) & 1) * (1 << 32)).to(torch.int32)
        elif dtype == "pair":
            out[i0:i1, 0] = v
            out[i0:i1, 1] = i
        else:
            raise ValueError("generate_into: u32, u64, pair and quartet only")
        del i, v
    return out


def generate(dist, dtype, n, seed=DEFAULT_SEED, device="cpu"):
    """Return a seeded synthetic input in the storage format above."""
    if dtype == "u64":
        return _int_values(dist, n, 64, seed, device)
    if dtype == "u32":
        v = _int_values(dist, n, 32, seed, device)
        return (v - ((v >> 31) & 1) * (1 << 32)).to(torch.int32)
    if dtype == "f64":
        if dist == "uniform":
            r = _draw(n, seed, 7, device)
            return _lsr(r, 11).to(torch.float64) * 2.0 ** -53
        if dist == "normal":  # Box-Muller
            u1 = (_lsr(_draw(n, seed, 8, device), 11) + 1).to(torch.float64) * 2.0 ** -53
            u2 = _lsr(_draw(n, seed, 9, device), 11).to(torch.float64) * 2.0 ** -53
            return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        raise ValueError("f64 distributions: %s" % (F64_DISTS,))
    if dtype == "pair":
        k = _int_values(dist, n, 64, seed, device)
        v = torch.arange(n, dtype=torch.int64, device=device)
        return torch.stack([k, v], dim=1).contiguous()
    if dtype == "quartet":
        if dist not in QUARTET_DISTS:
            raise ValueError("quartet distributions: %s" % (QUARTET_DISTS,))
        a, b, c = _quartet_keys(dist, n, seed, device)
        v = torch.arange(n, dtype=torch.int64, device=device)
        return torch.stack([a, b, c, v], dim=1).contiguous()
    if dtype == "rec100":
        out = torch.empty((n, 100), dtype=torch.uint8, device=device)
        if dist == "uniform":
            hi = _draw(n, seed, 10, device)
            lo = _draw(n, seed, 11, device)
        elif dist == "rootdup":
            # key = 80-bit big-endian value (i mod 2^14): 2 zero bytes + u64
            hi = torch.arange(n, dtype=torch.int64, device=device) % (1 << 14)
            lo = None
        else:
            raise ValueError("rec100 distributions: %s" % (REC_DISTS,))
        if lo is None:
            out[:, 0:2] = 0
            for b in range(8):
                out[:, 2 + b] = (_lsr(hi, 8 * (7 - b)) & 0xFF).to(torch.uint8)
        else:
            for b in range(8):
                out[:, b] = (_lsr(hi, 8 * (7 - b)) & 0xFF).to(torch.uint8)
            out[:, 8] = (_lsr(lo, 56) & 0xFF).to(torch.uint8)
            out[:, 9] = (_lsr(lo, 48) & 0xFF).to(torch.uint8)
        idx = torch.arange(n, dtype=torch.int64, device=device)
        for b in range(8):  # payload bytes 10..17: original index
            out[:, 10 + b] = (_lsr(idx, 8 * b) & 0xFF).to(torch.uint8)
        for w in range(11):  # payload bytes 18..99: seeded filler
            r = _draw(n, seed, 20 + w, device)
            for b in range(8):
                j = 18 + 8 * w + b
                if j < 100:
                    out[:, j] = (_lsr(r, 8 * b) & 0xFF).to(torch.uint8)
        return out
    raise ValueError("unknown dtype %r" % dtype)


SEG_DISTS = ("uniform", "twodup", "almostsorted")


def segment_lengths(nseg, lo_log2, hi_log2, seed=DEFAULT_SEED):
    """nseg lengths log-uniform in [2^lo_log2, 2^hi_log2]: length i is
    floor(2^(lo + u_i (hi - lo))) with u_i uniform in [0, 1) (stream 40).
    Returns an int64 CPU tensor."""
    u = _lsr(_draw(nseg, seed, 40, "cpu"), 11).to(torch.float64) * 2.0 ** -53
    return torch.floor(torch.pow(2.0, lo_log2 + u * (hi_log2 - lo_log2))).to(torch.int64)


def segmented_batch(lengths, dists=SEG_DISTS, seed=DEFAULT_SEED, device="cpu",
                    chunk_elems=1 << 26):
    """A batch of independent uint64 arrays stored back to back: array i has
    lengths[i] elements drawn from dists[i % len(dists)], where
      uniform       uniform in [0, 2^64)   (stream 41, by global position)
      twodup        (j^2 + m/2) mod m      (j: position in the array, m: its length)
      almostsorted  0..m-1 with about sqrt(m) disjoint adjacent swaps: pair
                    (2q, 2q+1) is swapped for every q drawn an odd number of
                    times among sqrt(m) draws q uniform in [0, (m-1)/2)
                    (stream 42, by array)
    Returns (data int64 (sum lengths,), offsets int64 (nseg + 1,)) on `device`;
    offsets[i] is the first element of array i.  Generated in chunks of whole
    arrays of about chunk_elems elements."""
    lengths = torch.as_tensor(lengths, dtype=torch.int64).cpu()
    nseg = lengths.numel()
    offsets = torch.zeros(nseg + 1, dtype=torch.int64)
    offsets[1:] = torch.cumsum(lengths, 0)
    total = int(offsets[-1])
    data = torch.empty(total, dtype=torch.int64, device=device)
    kind = torch.arange(nseg, dtype=torch.int64) % len(dists)
    codes = {"uniform": 0, "twodup": 1, "almostsorted": 2}
    kind = torch.tensor([codes[d] for d in dists], dtype=torch.int64)[kind]
    s0 = 0
    while s0 < nseg:
        s1 = s0
        acc = 0
        while s1 < nseg and (s1 == s0 or acc + int(lengths[s1]) <= chunk_elems):
            acc += int(lengths[s1])
            s1 += 1
        e0, e1 = int(offsets[s0]), int(offsets[s1])
        if e1 > e0:
            lens = lengths[s0:s1].to(device)
            sid = torch.repeat_interleave(torch.arange(s1 - s0, device=device), lens)
            start = offsets[s0:s1].to(device)
            gidx = torch.arange(e0, e1, dtype=torch.int64, device=device)
            loc = gidx - start[sid]
            m = lens[sid]
            k = kind[s0:s1].to(device)[sid]
            uni = _draw_at(gidx, seed, 41)
            two = (loc * loc + m // 2) % m
            v = torch.where(k == 0, uni, torch.where(k == 1, two, loc))
            data[e0:e1] = v
            # almost sorted arrays: disjoint adjacent swaps
            al = [i for i in range(s0, s1) if int(kind[i]) == 2 and int(lengths[i]) >= 4]
            for i in al:
                mlen = int(lengths[i])
                nsw = math.isqrt(mlen)
                npair = (mlen - 1) // 2
                q = _umod(_draw_at(torch.arange(nsw, dtype=torch.int64) + (i << 32), seed, 42),
                          npair)
                uq, cnt = torch.unique(q, return_counts=True)
                uq = uq[cnt % 2 == 1]
                if uq.numel():
                    a = int(offsets[i]) + 2 * uq.to(device)
                    x = data[a].clone()
                    data[a] = data[a + 1]
                    data[a + 1] = x
        s0 = s1
    return data, offsets.to(device)


def to_numpy(t, dtype):
    """Storage tensor -> numpy array in the oracle's conventions."""
    a = t.detach().cpu().contiguous().numpy()
    if dtype == "u32":
        return a.view(np.uint32)
    if dtype in ("u64", "pair", "quartet"):
        return a.view(np.uint64)
    return a


def from_numpy(a, dtype, device="cpu"):
    """numpy array in the oracle's conventions -> storage tensor."""
    a = np.ascontiguousarray(a)
    if dtype == "u32":
        a = a.view(np.int32)
    elif dtype in ("u64", "pair", "quartet"):
        a = a.view(np.int64)
    return torch.from_numpy(a.copy()).to(device)


def count(t, dtype):
    """Number of elements of a storage tensor."""
    return t.shape[0]
