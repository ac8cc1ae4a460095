"""Thin ctypes binding of the C ABI in include/ipsgpu.h.

Every function here only marshals arguments: device pointers and sizes in,
status codes out.  All work runs in the CUDA kernels of libipsgpu.so.  There
is no fallback: if the library is missing, loading raises IpsgpuError (build
it with ``paper_2009_13569_gb300.build.build()``).
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libipsgpu.so")

DTYPES = {"u32": 0, "u64": 1, "f64": 2, "pair": 3, "rec100": 4, "quartet": 5}
ELEM_BYTES = {"u32": 4, "u64": 8, "f64": 8, "pair": 16, "rec100": 100, "quartet": 32}
SAMPLESORT, RADIX, SAMPLESORT_TREE = 0, 1, 2

OK, E_INVAL, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUSY, E_INTERNAL, E_CANCELED = range(9)


class IpsgpuError(RuntimeError):
    """A non-zero status of a C-ABI call (`code` is the ipsgpu status)."""
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (status %d)" % (what, strerror(code) if _lib else "?", code))


class Params(ctypes.Structure):
    """ipsgpu_params: zero fields take the library defaults."""
    _fields_ = [("k", ctypes.c_uint32), ("block_bytes", ctypes.c_uint32),
                ("alpha_scale", ctypes.c_float), ("base_case", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("algo", ctypes.c_int32),
                ("spin_limit", ctypes.c_uint32), ("arena_bytes", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    """ipsgpu_server_config: zero fields take the library defaults."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("batch_max_elems", ctypes.c_uint64),
                ("small_reserve_bytes", ctypes.c_uint64),
                ("lanes", ctypes.c_uint32), ("dtype_mask", ctypes.c_uint32),
                ("batch_max_requests", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_lib = None


def load():
    """Load libipsgpu.so (raises IpsgpuError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise IpsgpuError(E_CUDA, "libipsgpu.so not found at %s; run build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "ipsgpu_sorter_create": (i32, [ctypes.POINTER(Params), i32, ctypes.POINTER(vp)]),
        "ipsgpu_sorter_destroy": (i32, [vp]),
        "ipsgpu_scratch_bytes": (u64, [ctypes.POINTER(Params), i32]),
        "ipsgpu_sort": (i32, [vp, vp, u64, vp]),
        "ipsgpu_sort_host": (i32, [vp, vp, vp, u64, vp, vp]),
        "ipsgpu_partition_level": (i32, [vp, vp, u64, vp, u32, i32, vp, vp]),
        "ipsgpu_radix_level": (i32, [vp, vp, u64, u32, u32, vp, vp]),
        "ipsgpu_classify": (i32, [vp, vp, u64, vp, u32, i32, vp, vp]),
        "ipsgpu_status": (i32, [vp, vp]),
        "ipsgpu_strerror": (ctypes.c_char_p, [i32]),
        "ipsgpu_set_timing": (i32, [vp, i32]),
        "ipsgpu_kernel_stats": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), i32]),
        "ipsgpu_kernel_name": (ctypes.c_char_p, [i32]),
        "ipsgpu_wave_stats": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                    ctypes.POINTER(u64)]),
        "ipsgpu_debug_bounded_wait": (i32, [vp, u32, vp]),
        "ipsgpu_debug_check_guards": (i32, [vp, ctypes.POINTER(u64)]),
        "ipsgpu_partition_level_noalloc": (i32, [i32, vp, u64, vp, u32, i32, vp, vp]),
        "ipsgpu_sort_segmented": (i32, [vp, vp, u64, vp, u64, vp]),
        "ipsgpu_sort_batch": (i32, [vp, vp, u64, vp]),
        "ipsgpu_segmented_graph_create": (i32, [vp, vp, u64, vp, u64, ctypes.POINTER(vp)]),
        "ipsgpu_graph_launch": (i32, [vp, vp]),
        "ipsgpu_graph_nodes": (i32, [vp, ctypes.POINTER(u64)]),
        "ipsgpu_graph_destroy": (i32, [vp]),
        "ipsgpu_sorter_prepare": (i32, [vp]),
        "ipsgpu_server_create": (i32, [ctypes.POINTER(ServerConfig), ctypes.POINTER(Params),
                                       ctypes.POINTER(vp)]),
        "ipsgpu_server_destroy": (i32, [vp]),
        "ipsgpu_server_reserve": (i32, [vp, u64, i32, ctypes.POINTER(u64)]),
        "ipsgpu_server_start": (i32, [vp, u64, vp, vp]),
        "ipsgpu_server_submit": (i32, [vp, vp, u64, i32, ctypes.POINTER(u64)]),
        "ipsgpu_server_poll": (i32, [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ipsgpu_server_wait": (i32, [vp, u64]),
        "ipsgpu_server_times": (i32, [vp, u64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
        "ipsgpu_server_now_us": (ctypes.c_double, []),
        "ipsgpu_server_release": (i32, [vp, u64]),
        "ipsgpu_server_cancel": (i32, [vp, u64]),
        "ipsgpu_server_drain": (i32, [vp]),
        "ipsgpu_server_usage": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                      ctypes.POINTER(u64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C-ABI functions this binding declares."""
    return [
        "ipsgpu_sorter_create", "ipsgpu_sorter_destroy", "ipsgpu_scratch_bytes", "ipsgpu_sort",
        "ipsgpu_sort_host",
        "ipsgpu_partition_level", "ipsgpu_radix_level", "ipsgpu_classify", "ipsgpu_status",
        "ipsgpu_strerror", "ipsgpu_set_timing", "ipsgpu_kernel_stats", "ipsgpu_kernel_name",
        "ipsgpu_wave_stats",
        "ipsgpu_debug_bounded_wait", "ipsgpu_debug_check_guards",
        "ipsgpu_partition_level_noalloc", "ipsgpu_sort_segmented",
        "ipsgpu_sort_batch", "ipsgpu_segmented_graph_create", "ipsgpu_graph_launch",
        "ipsgpu_graph_nodes", "ipsgpu_graph_destroy", "ipsgpu_sorter_prepare",
        "ipsgpu_server_create", "ipsgpu_server_destroy", "ipsgpu_server_reserve",
        "ipsgpu_server_start", "ipsgpu_server_submit", "ipsgpu_server_poll", "ipsgpu_server_wait",
        "ipsgpu_server_times", "ipsgpu_server_now_us", "ipsgpu_server_release",
        "ipsgpu_server_drain", "ipsgpu_server_usage", "ipsgpu_server_cancel",
    ]


def strerror(code):
    """Message of an ipsgpu status code (ipsgpu_strerror)."""
    return load().ipsgpu_strerror(code).decode()


def _check(rc, what):
    if rc != OK:
        raise IpsgpuError(rc, what)


def partition_level_noalloc(dtype, ptr, n, spl_ptr, num_splitters, equal_buckets, bb_ptr,
                            stream=0):
    """ipsgpu_partition_level_noalloc: one level without a sorter and without
    allocating (scratch is a fixed device array inside the library)."""
    _check(load().ipsgpu_partition_level_noalloc(DTYPES[dtype], ptr, n, spl_ptr, num_splitters,
                                                 1 if equal_buckets else 0, bb_ptr, stream),
           "ipsgpu_partition_level_noalloc")


def make_params(k=0, block_bytes=0, alpha_scale=0.0, base_case=0, seed=0, algo=SAMPLESORT,
                spin_limit=0, arena_bytes=0):
    """An ipsgpu_params structure (see include/ipsgpu.h for each field)."""
    return Params(k, block_bytes, alpha_scale, base_case, seed, algo, spin_limit, arena_bytes)


def scratch_bytes(dtype, **params):
    """Device scratch of a sorter with these parameters (0: invalid)."""
    p = make_params(**params)
    return int(load().ipsgpu_scratch_bytes(ctypes.byref(p), DTYPES[dtype]))


class Sorter:
    """An ipsgpu_sorter (owns its device scratch).  Pointers are device
    addresses (ints), streams are cudaStream_t handles (ints, 0 = default)."""

    def __init__(self, dtype, **params):
        self.dtype = dtype
        self.elem_bytes = ELEM_BYTES[dtype]
        p = make_params(**params)
        h = ctypes.c_void_p()
        _check(load().ipsgpu_sorter_create(ctypes.byref(p), DTYPES[dtype], ctypes.byref(h)),
               "ipsgpu_sorter_create")
        self._h = h

    def close(self):
        """Free the underlying library object (also on leaving a with block)."""
        if self._h:
            load().ipsgpu_sorter_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def prepare(self):
        """Build the sorter's recursion graph now instead of on first use."""
        _check(load().ipsgpu_sorter_prepare(self._h), "ipsgpu_sorter_prepare")

    def sort(self, ptr, n, stream=0):
        """Sort ptr[0..n) in place on the device (ipsgpu_sort), queued on stream."""
        _check(load().ipsgpu_sort(self._h, ptr, n, stream), "ipsgpu_sort")

    def sort_host(self, in_ptr, out_ptr, n, work_ptr, stream=0):
        """Host array in (in_ptr), sorted result out (out_ptr, may equal
        in_ptr), through the device buffer work_ptr; queued on stream."""
        _check(load().ipsgpu_sort_host(self._h, in_ptr, out_ptr, n, work_ptr, stream),
               "ipsgpu_sort_host")

    def sort_segmented(self, ptr, n, offsets_ptr, num_segments, stream=0):
        """Sort segments [offsets[i], offsets[i+1]) of the n-element array in
        place; offsets_ptr points to num_segments + 1 u64 in device memory."""
        _check(load().ipsgpu_sort_segmented(self._h, ptr, n, offsets_ptr, num_segments, stream),
               "ipsgpu_sort_segmented")

    def sort_batch(self, segs_ptr, num_segments, stream=0):
        """Sort separate arrays in place; segs_ptr points to num_segments
        (device address, length) u64 pairs in device memory."""
        _check(load().ipsgpu_sort_batch(self._h, segs_ptr, num_segments, stream),
               "ipsgpu_sort_batch")

    def segmented_graph(self, ptr, n, offsets_ptr, num_segments):
        """Capture a segmented sort over these buffers into a CUDA graph."""
        return SegmentedGraph(self, ptr, n, offsets_ptr, num_segments)

    def partition_level(self, ptr, n, spl_ptr, num_splitters, equal_buckets, bb_ptr, stream=0):
        """One partitioning step with given sorted splitters; bucket begins
        (u64, B + 1 of them) to bb_ptr (ipsgpu_partition_level)."""
        _check(load().ipsgpu_partition_level(self._h, ptr, n, spl_ptr, num_splitters,
                                             1 if equal_buckets else 0, bb_ptr, stream),
               "ipsgpu_partition_level")

    def radix_level(self, ptr, n, shift, bits, bb_ptr, stream=0):
        """One IPS2Ra step on key bits [shift, shift + bits) (ipsgpu_radix_level)."""
        _check(load().ipsgpu_radix_level(self._h, ptr, n, shift, bits, bb_ptr, stream),
               "ipsgpu_radix_level")

    def classify(self, ptr, n, spl_ptr, num_splitters, equal_buckets, cls_ptr, stream=0):
        """Class id of every element to cls_ptr (u32), data not moved
        (ipsgpu_classify)."""
        _check(load().ipsgpu_classify(self._h, ptr, n, spl_ptr, num_splitters,
                                      1 if equal_buckets else 0, cls_ptr, stream),
               "ipsgpu_classify")

    def status(self, stream=0):
        """Synchronize, return and clear the device status word."""
        return load().ipsgpu_status(self._h, stream)

    def set_timing(self, enable=True):
        """Per-kernel CUDA-event timing on or off (ipsgpu_set_timing); while
        on, sorts run from the host-driven wave loop."""
        _check(load().ipsgpu_set_timing(self._h, 1 if enable else 0), "ipsgpu_set_timing")

    def kernel_stats(self):
        """{kernel name: (launches, ms, algorithmic bytes)} since the last call."""
        cap = 32
        la = (ctypes.c_uint64 * cap)()
        ms = (ctypes.c_double * cap)()
        by = (ctypes.c_double * cap)()
        nk = load().ipsgpu_kernel_stats(self._h, la, ms, by, cap)
        if nk < 0:
            raise IpsgpuError(-nk, "ipsgpu_kernel_stats")
        return {load().ipsgpu_kernel_name(i).decode(): (int(la[i]), float(ms[i]), float(by[i]))
                for i in range(nk)}

    def wave_stats(self):
        """(waves, largest ring occupancy, ring capacity) of the last run made
        with timing on (ipsgpu_wave_stats)."""
        w, m, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ipsgpu_wave_stats(self._h, ctypes.byref(w), ctypes.byref(m),
                                        ctypes.byref(c)), "ipsgpu_wave_stats")
        return int(w.value), int(m.value), int(c.value)

    def check_guards(self):
        """Synchronize and check the guard zones around every device buffer
        of the sorter: None if intact, else the index of the first buffer
        whose guard changed."""
        bad = ctypes.c_uint64(0)
        rc = load().ipsgpu_debug_check_guards(self._h, ctypes.byref(bad))
        if rc == OK:
            return None
        if rc == E_INTERNAL:
            return int(bad.value)
        raise IpsgpuError(rc, "ipsgpu_debug_check_guards")

    def debug_bounded_wait(self, spin_limit, stream=0):
        """Run the permutation's bounded wait on a flag nothing sets; the
        status then reads IPSGPU_E_TIMEOUT (ipsgpu_debug_bounded_wait)."""
        _check(load().ipsgpu_debug_bounded_wait(self._h, spin_limit, stream),
               "ipsgpu_debug_bounded_wait")


class SegmentedGraph:
    """An ipsgpu_graph: one segmented sort over fixed buffers, replayed by
    launch().  Keeps its sorter alive."""

    def __init__(self, sorter, ptr, n, offsets_ptr, num_segments):
        self.sorter = sorter
        h = ctypes.c_void_p()
        _check(load().ipsgpu_segmented_graph_create(sorter._h, ptr, n, offsets_ptr, num_segments,
                                                    ctypes.byref(h)),
               "ipsgpu_segmented_graph_create")
        self._h = h

    def launch(self, stream=0):
        """Launch the captured segmented sort (ipsgpu_graph_launch)."""
        _check(load().ipsgpu_graph_launch(self._h, stream), "ipsgpu_graph_launch")

    def nodes(self):
        """Top-level nodes of the captured graph (ipsgpu_graph_nodes)."""
        v = ctypes.c_uint64()
        _check(load().ipsgpu_graph_nodes(self._h, ctypes.byref(v)), "ipsgpu_graph_nodes")
        return int(v.value)

    def close(self):
        """Free the underlying library object (also on leaving a with block)."""
        if self._h:
            load().ipsgpu_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """An ipsgpu_server: admission by HBM footprint and continuous batching
    over CUDA streams.  Buffers stay owned by the caller."""

    def __init__(self, hbm_budget_bytes, lanes=0, dtypes=("u32", "u64", "pair"),
                 batch_max_elems=0, batch_max_requests=0, small_reserve_bytes=0, **params):
        mask = 0
        for d in dtypes:
            mask |= 1 << DTYPES[d]
        self.batch_max_elems = batch_max_elems or (1 << 22)
        cfg = ServerConfig(hbm_budget_bytes, batch_max_elems, small_reserve_bytes, lanes, mask,
                           batch_max_requests, 0)
        p = make_params(**params)
        h = ctypes.c_void_p()
        _check(load().ipsgpu_server_create(ctypes.byref(cfg), ctypes.byref(p), ctypes.byref(h)),
               "ipsgpu_server_create")
        self._h = h

    def reserve(self, n, dtype):
        """Ticket, or None if the footprint does not fit now (E_BUSY)."""
        t = ctypes.c_uint64()
        rc = load().ipsgpu_server_reserve(self._h, n, DTYPES[dtype], ctypes.byref(t))
        if rc == E_BUSY:
            return None
        _check(rc, "ipsgpu_server_reserve")
        return int(t.value)

    def start(self, ticket, ptr, ready_stream=0):
        """Queue a reserved request on data at ptr; the sort waits for the work
        queued so far on ready_stream (ipsgpu_server_start)."""
        _check(load().ipsgpu_server_start(self._h, ticket, ptr, ready_stream),
               "ipsgpu_server_start")

    def submit(self, ptr, n, dtype):
        """Ticket, or None if the footprint does not fit now (E_BUSY)."""
        t = ctypes.c_uint64()
        rc = load().ipsgpu_server_submit(self._h, ptr, n, DTYPES[dtype], ctypes.byref(t))
        if rc == E_BUSY:
            return None
        _check(rc, "ipsgpu_server_submit")
        return int(t.value)

    def poll(self, ticket):
        """(done, status)."""
        d, st = ctypes.c_int(), ctypes.c_int()
        _check(load().ipsgpu_server_poll(self._h, ticket, ctypes.byref(d), ctypes.byref(st)),
               "ipsgpu_server_poll")
        return bool(d.value), int(st.value)

    def wait(self, ticket):
        """Block until done; returns the request's status."""
        return load().ipsgpu_server_wait(self._h, ticket)

    def times(self, ticket):
        """(submit, launch, done) in microseconds of now_us()'s clock."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().ipsgpu_server_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c)), "ipsgpu_server_times")
        return a.value, b.value, c.value

    @staticmethod
    def now_us():
        """The server's clock in microseconds (ipsgpu_server_now_us)."""
        return load().ipsgpu_server_now_us()

    def release(self, ticket):
        """Give a finished request's footprint back (ipsgpu_server_release)."""
        _check(load().ipsgpu_server_release(self._h, ticket), "ipsgpu_server_release")

    def cancel(self, ticket):
        """Cancel a reserved or queued request (E_BUSY if it already runs)."""
        _check(load().ipsgpu_server_cancel(self._h, ticket), "ipsgpu_server_cancel")

    def drain(self):
        """Wait until no request is queued or running (ipsgpu_server_drain)."""
        _check(load().ipsgpu_server_drain(self._h), "ipsgpu_server_drain")

    def usage(self):
        """(used bytes incl. scratch, budget, scratch)."""
        u, b, s = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ipsgpu_server_usage(self._h, ctypes.byref(u), ctypes.byref(b),
                                          ctypes.byref(s)), "ipsgpu_server_usage")
        return int(u.value), int(b.value), int(s.value)

    def close(self):
        """Free the underlying library object (also on leaving a with block)."""
        if self._h:
            load().ipsgpu_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
