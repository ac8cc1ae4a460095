"""CPU oracle for the in-place samplesort (IPS4o) and radix sort (IPS2Ra).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The GPU library and its
Python binding never import this package, and it never imports them.

The arithmetic lives in ``oracle.c`` (plain sequential C, see its header for
the passages of the paper each function follows); this module only compiles
it with gcc and marshals numpy arrays through ctypes.

Array conventions (shared with the GPU binding by convention only):
  'u32'    -> numpy uint32, shape (n,)
  'u64'    -> numpy uint64, shape (n,)
  'f64'    -> numpy float64, shape (n,)
  'pair'   -> numpy uint64, shape (n, 2): column 0 key, column 1 value
  'rec100' -> numpy uint8,  shape (n, 100): bytes 0..9 key, 10..99 payload
  'quartet'-> numpy uint64, shape (n, 4): columns 0..2 key (compared
              lexicographically), column 3 value
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

DTYPES = {"u32": 0, "u64": 1, "f64": 2, "pair": 3, "rec100": 4, "quartet": 5}
ELEM_BYTES = {"u32": 4, "u64": 8, "f64": 8, "pair": 16, "rec100": 100, "quartet": 32}

_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    lib.oracle_sort.argtypes = [i32, vp, u64, u32, u32, ctypes.c_double, u64]
    lib.oracle_sort.restype = i32
    lib.oracle_insertion_sort.argtypes = [i32, vp, u64]
    lib.oracle_insertion_sort.restype = i32
    lib.oracle_is_sorted.argtypes = [i32, vp, u64]
    lib.oracle_is_sorted.restype = i32
    lib.oracle_classify.argtypes = [i32, vp, u64, vp, u32, i32, vp]
    lib.oracle_classify.restype = u32
    lib.oracle_radix_classify.argtypes = [i32, vp, u64, u32, u32, vp]
    lib.oracle_radix_classify.restype = u32
    lib.oracle_partition.argtypes = [i32, vp, u64, vp, u32, vp, vp]
    lib.oracle_partition.restype = None
    lib.oracle_elem_size.argtypes = [i32]
    lib.oracle_elem_size.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def _count(a, dtype):
    a = np.asarray(a)
    if dtype in ("pair", "rec100", "quartet"):
        return a.shape[0]
    return a.size


def _check(a, dtype):
    want = {"u32": np.uint32, "u64": np.uint64, "f64": np.float64,
            "pair": np.uint64, "rec100": np.uint8, "quartet": np.uint64}[dtype]
    a = np.ascontiguousarray(a)
    if a.dtype != want:
        raise TypeError("oracle: %s array must be %s, got %s" % (dtype, want, a.dtype))
    if dtype == "pair" and (a.ndim != 2 or a.shape[1] != 2):
        raise ValueError("oracle: pair array must have shape (n, 2)")
    if dtype == "rec100" and (a.ndim != 2 or a.shape[1] != 100):
        raise ValueError("oracle: rec100 array must have shape (n, 100)")
    if dtype == "quartet" and (a.ndim != 2 or a.shape[1] != 4):
        raise ValueError("oracle: quartet array must have shape (n, 4)")
    return a


def sort(a, dtype, k=256, n0=16, alpha=0.2, seed=0x1B54A32D192ED03):
    """Return a sorted copy of ``a`` (sequential samplesort, Sec. 3 / Sec. 5)."""
    out = _check(a, dtype).copy()
    rc = _load().oracle_sort(DTYPES[dtype], out.ctypes.data, _count(out, dtype),
                             k, n0, alpha, seed)
    if rc != 0:
        raise ValueError("oracle_sort rejected its arguments")
    return out


def insertion_sort(a, dtype):
    """Return a copy of ``a`` sorted by insertion sort (the base case, Sec. 5)."""
    out = _check(a, dtype).copy()
    _load().oracle_insertion_sort(DTYPES[dtype], out.ctypes.data, _count(out, dtype))
    return out


def is_sorted(a, dtype):
    a = _check(a, dtype)
    return bool(_load().oracle_is_sorted(DTYPES[dtype], a.ctypes.data, _count(a, dtype)))


def classify(a, dtype, splitters, equal_buckets):
    """Class id of every element for sorted ``splitters`` (Sec. 2, Algorithm 1).

    Returns (cls uint32[n], B) with B = K or 2K, K = 2^ceil(log2(m+1)).
    """
    a = _check(a, dtype)
    s = _check(splitters, dtype)
    n, m = _count(a, dtype), _count(s, dtype)
    if m == 0:
        raise ValueError("at least one splitter is required")
    cls = np.empty(n, dtype=np.uint32)
    B = _load().oracle_classify(DTYPES[dtype], a.ctypes.data, n, s.ctypes.data, m,
                                1 if equal_buckets else 0, cls.ctypes.data)
    return cls, int(B)


def radix_classify(a, dtype, shift, bits):
    """Radix digit of every key (Sec. 5, IPS2Ra): (key >> shift) & (2^bits-1)."""
    if dtype not in ("u32", "u64", "pair"):
        raise ValueError("the radix extractor takes unsigned integer keys only")
    a = _check(a, dtype)
    n = _count(a, dtype)
    cls = np.empty(n, dtype=np.uint32)
    B = _load().oracle_radix_classify(DTYPES[dtype], a.ctypes.data, n, shift, bits,
                                      cls.ctypes.data)
    return cls, int(B)


def partition(a, dtype, cls, B):
    """Stable distribution by class: (partitioned copy, bucket_begin[B+1])."""
    a = _check(a, dtype)
    n = _count(a, dtype)
    cls = np.ascontiguousarray(cls, dtype=np.uint32)
    out = np.empty_like(a)
    bb = np.empty(B + 1, dtype=np.uint64)
    _load().oracle_partition(DTYPES[dtype], a.ctypes.data, n, cls.ctypes.data, B,
                             out.ctypes.data, bb.ctypes.data)
    return out, bb


def partition_level(a, dtype, splitters, equal_buckets):
    """One classification level, distributed: (partitioned copy, bucket_begin)."""
    cls, B = classify(a, dtype, splitters, equal_buckets)
    return partition(a, dtype, cls, B)


def radix_level(a, dtype, shift, bits):
    """One IPS2Ra level, distributed: (partitioned copy, bucket_begin)."""
    cls, B = radix_classify(a, dtype, shift, bits)
    return partition(a, dtype, cls, B)
