"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/ipsgpu.h declares; host-only entry points
behave.  No kernel runs here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2009_13569_gb300 import build, ipsgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ipsgpu.load()


def declared():
    with open(os.path.join(ROOT, "include", "ipsgpu.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ipsgpu_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(ipsgpu.exported_symbols()) == set(names)


def test_strerror_and_scratch_bytes(lib):
    assert ipsgpu.strerror(ipsgpu.OK) == "ok"
    assert "timed out" in ipsgpu.strerror(ipsgpu.E_TIMEOUT)
    b64 = ipsgpu.scratch_bytes("u64")
    assert b64 > 0
    # scratch does not depend on n: it is fixed by the parameters
    assert ipsgpu.scratch_bytes("u64", arena_bytes=1 << 20) < b64
    # radix takes unsigned keys only
    assert ipsgpu.scratch_bytes("f64", algo=ipsgpu.RADIX) == 0
    assert ipsgpu.scratch_bytes("u64", k=3) == 0
    assert ipsgpu.scratch_bytes("quartet") > 0
    assert ipsgpu.scratch_bytes("u64", algo=ipsgpu.SAMPLESORT_TREE) == b64
    assert ipsgpu.scratch_bytes("u64", algo=3) == 0
    assert ipsgpu.scratch_bytes("quartet", algo=ipsgpu.RADIX) == 0
    assert ipsgpu.scratch_bytes("rec100", algo=ipsgpu.RADIX) == 0


def test_dtype_enum_matches_binding():
    with open(os.path.join(ROOT, "include", "ipsgpu.h")) as f:
        text = f.read()
    enum = dict((k, int(v)) for k, v in re.findall(r"IPSGPU_(U32|U64|F64|PAIR_U64|REC100|QUARTET)"
                                                   r"\s*=\s*(\d+)", text))
    names = {"u32": "U32", "u64": "U64", "f64": "F64", "pair": "PAIR_U64", "rec100": "REC100",
             "quartet": "QUARTET"}
    assert {d: enum[names[d]] for d in names} == ipsgpu.DTYPES


def test_params_struct_layout():
    assert ctypes.sizeof(ipsgpu.Params) == 40
    assert ipsgpu.Params.arena_bytes.offset == 32


def test_server_config_struct_layout():
    assert ctypes.sizeof(ipsgpu.ServerConfig) == 40
    assert ipsgpu.ServerConfig.lanes.offset == 24
    assert ipsgpu.ServerConfig.batch_max_requests.offset == 32


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ipsgpu.h"
int main(void) {
    ipsgpu_params p;
    memset(&p, 0, sizeof p);
    size_t a = ipsgpu_scratch_bytes(&p, IPSGPU_U64);
    size_t b = ipsgpu_scratch_bytes(&p, IPSGPU_QUARTET);
    printf("%s|%llu|%llu\n", ipsgpu_strerror(IPSGPU_E_TIMEOUT),
           (unsigned long long)a, (unsigned long long)b);
    return (a > 0 && b > 0) ? 0 : 1;
}
"""


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_is_plain_c_and_links(lib, tmp_path, compiler, std):
    # the boundary carries no C++ or torch types: the header compiles as
    # strict C99 (and as C++), and a C program linked against the library
    # calls its host-only entry points
    src = tmp_path / ("t.c" if compiler == "gcc" else "t.cpp")
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(lib._name)
    exe = tmp_path / "t"
    subprocess.check_call([compiler, std, "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lipsgpu", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    msg, a, b = out.strip().split("|")
    assert msg == ipsgpu.strerror(ipsgpu.E_TIMEOUT)
    assert int(a) == ipsgpu.scratch_bytes("u64")
    assert int(b) == ipsgpu.scratch_bytes("quartet")


def _block_elems(block_bytes, D):
    b = 1
    while b * 2 * D <= block_bytes:
        b *= 2
    return b


@pytest.mark.parametrize("dtype", sorted(ipsgpu.ELEM_BYTES))
def test_parameter_ranges_of_the_header(lib, dtype):
    # every range the header states for ipsgpu_params, at its edges: inside,
    # scratch_bytes is positive; outside, it is 0 and creating a sorter
    # fails with E_INVAL before any CUDA call
    D = ipsgpu.ELEM_BYTES[dtype]
    cap = 184 * 1024 // D

    def ok(**p):
        return ipsgpu.scratch_bytes(dtype, **p) > 0

    def rejected(**p):
        if ipsgpu.scratch_bytes(dtype, **p) != 0:
            return False
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            ipsgpu.Sorter(dtype, **p)
        return e.value.code == ipsgpu.E_INVAL

    for k in (4, 8, 16, 32, 64, 128, 256):
        assert ok(k=k), k
    for k in (2, 3, 5, 12, 255, 257, 512):
        assert rejected(k=k), k
    assert ok(base_case=32) and ok(base_case=cap)
    assert rejected(base_case=31) and rejected(base_case=cap + 1)
    # blocks: b = largest power of two with b * D <= block_bytes; b * D a
    # multiple of 16, at most 2 KiB, and k * b * D at most 128 KiB
    for bb in (16, 64, 100, 400, 512, 1000, 1024, 2048, 4096):
        b = _block_elems(bb, D)
        for k in (4, 64, 128, 256):
            valid = (b * D) % 16 == 0 and b * D <= 2048 and k * b * D <= 128 * 1024
            assert ok(k=k, block_bytes=bb) == valid, (bb, k)
            if not valid:
                assert rejected(k=k, block_bytes=bb), (bb, k)
    # arena: at least (2k + 1) blocks and 1 KiB
    b = _block_elems(512, D)
    amin = (2 * 256 + 1) * b * D + 1024
    assert ok(arena_bytes=amin) and rejected(arena_bytes=amin - 1)
    assert rejected(algo=3) and rejected(algo=-1)


def test_server_config_checks_of_the_header(lib):
    # the argument checks of ipsgpu_server_create come before any CUDA call
    def code(budget, **kw):
        with pytest.raises(ipsgpu.IpsgpuError) as e:
            ipsgpu.Server(budget, **kw)
        return e.value.code

    big = 1 << 40
    assert code(0) == ipsgpu.E_INVAL
    assert code(big, lanes=65) == ipsgpu.E_INVAL
    assert code(big, small_reserve_bytes=big) == ipsgpu.E_INVAL
    assert code(big, dtypes=("u64", "f64"), algo=ipsgpu.RADIX) == ipsgpu.E_INVAL
    assert code(big, k=3) == ipsgpu.E_INVAL
    # a dtype_mask bit beyond the last type, through the raw call
    cfg = ipsgpu.ServerConfig(big, 0, 0, 0, 1 << (max(ipsgpu.DTYPES.values()) + 1), 0, 0)
    h = ctypes.c_void_p()
    assert lib.ipsgpu_server_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ipsgpu.E_INVAL
    # scratch of the lanes' sorters above the budget
    scratch = 4 * sum(ipsgpu.scratch_bytes(d) for d in ("u32", "u64", "pair"))
    assert code(scratch - 1) == ipsgpu.E_NOMEM


def test_noalloc_level_argument_checks(lib):
    # each call below breaks one stated limit, which the library checks
    # before any CUDA call (the pointers are placeholders, never read)
    P = 1 << 20  # a placeholder address, aligned for every type
    u64 = ipsgpu.DTYPES["u64"]
    f = lib.ipsgpu_partition_level_noalloc
    assert f(99, P, 10, P, 3, 0, P, None) == ipsgpu.E_INVAL          # no such dtype
    assert f(u64, P, 10, None, 3, 0, P, None) == ipsgpu.E_INVAL      # no splitters
    assert f(u64, P, 10, P, 3, 0, None, None) == ipsgpu.E_INVAL      # no bucket_begin
    assert f(u64, P, 10, P, 0, 0, P, None) == ipsgpu.E_INVAL         # zero splitters
    assert f(u64, P, 10, P, 128, 1, P, None) == ipsgpu.E_INVAL       # B = 512 > 256
    assert f(u64, P, 10, P, 256, 0, P, None) == ipsgpu.E_INVAL       # K = 512 > 256
    assert f(u64, P, 1 << 32, P, 3, 0, P, None) == ipsgpu.E_INVAL    # n > 2^32 - 1
    assert f(u64, None, 10, P, 3, 0, P, None) == ipsgpu.E_INVAL      # no data
    assert f(u64, P + 4, 10, P, 3, 0, P, None) == ipsgpu.E_INVAL     # misaligned data
    assert f(u64, P, 10, P + 4, 3, 0, P, None) == ipsgpu.E_INVAL     # misaligned splitters
    rec = ipsgpu.DTYPES["rec100"]
    assert f(rec, P + 2, 10, P, 3, 0, P, None) == ipsgpu.E_INVAL     # records: 4-byte aligned


def test_every_status_code_of_the_header_has_its_own_message(lib):
    with open(os.path.join(ROOT, "include", "ipsgpu.h")) as f:
        codes = dict((name, int(v)) for name, v in
                     re.findall(r"\b(IPSGPU_(?:OK|E_[A-Z]+))\s*=\s*(\d+)", f.read()))
    assert len(codes) >= 9 and sorted(codes.values()) == list(range(len(codes)))
    for name, v in codes.items():
        assert getattr(ipsgpu, name[len("IPSGPU_"):]) == v, name
    msgs = [ipsgpu.strerror(v) for v in codes.values()]
    assert len(set(msgs)) == len(msgs) and "unknown status" not in msgs
    assert ipsgpu.strerror(len(codes)) == ipsgpu.strerror(-1) == "unknown status"


def test_scratch_is_the_arena_plus_fixed_tables(lib):
    # the header's figures: tables of fixed capacity (by key width) plus the
    # arena, unchanged by k and by the arena's own size
    tables_mib = {"u32": 226.75, "u64": 234.75, "f64": 234.75, "pair": 234.75,
                  "rec100": 250.75, "quartet": 266.75}
    for dtype, mib in tables_mib.items():
        for arena in (256 << 20, 1 << 24):
            for k in (64, 256):
                got = ipsgpu.scratch_bytes(dtype, arena_bytes=arena, k=k) - arena
                assert got == int(mib * 2 ** 20) + 1024, (dtype, arena, k)  # + 1 KiB of state
