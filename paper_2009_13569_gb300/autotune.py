"""Autotuner for the sorter's parameters: (k, block bytes), the base-case
size and the oversampling factor, picked by timing candidate sorters on a
sample of the workload on the GPU.

The search is coordinate descent over three groups, in the order in which
they matter most: first the (k, block_bytes) pair (k in {256, 128, 64},
block bytes in {512, 1024, 2048}, k * block_bytes at most 128 KiB, the
classification buffer one CTA can hold), then the base-case size, then
alpha_scale (the paper's oversampling factor alpha = alpha_scale * log2 n).  Each candidate is timed `reps` times on fresh copies of the sample
(the sort is in place) and scored by its median.  The search logic is
independent of how a candidate is timed (search()), so it is testable on the
CPU; tune_array() and tune_segmented() time candidates through the C ABI.

Results can be kept in a JSON cache file (``cache=path``): the key is the
element type and a coarse signature of the workload (the array size, or the
number of arrays, total elements and a histogram of log2 array lengths), so
a later run on a workload of the same shape takes the stored parameters
without timing anything.
"""
import json
import math
import os
import statistics

from . import ipsgpu

# (k, block_bytes) with k * block_bytes <= 128 KiB: 256 buckets of 512 B
# blocks down to 64 buckets of 2 KiB
KB_PAIRS = ((256, 512), (128, 1024), (64, 2048), (128, 512), (64, 1024), (64, 512))
ALPHAS = (0.2, 0.5, 1.0)
BASE_FRACTIONS = (1.0, 0.5, 0.25)  # of the largest base case the type allows
BASE_SMEM_BYTES = 184 * 1024       # shared-memory element buffer of the base case


def base_cap(dtype):
    return BASE_SMEM_BYTES // ipsgpu.ELEM_BYTES[dtype]


def search(time_fn, dtype, kb_pairs=KB_PAIRS, base_fracs=BASE_FRACTIONS, alphas=ALPHAS):
    """Coordinate descent.  time_fn(params) -> seconds (smaller is better),
    or None if the parameters are rejected.  Returns (best params, table of
    every timed candidate as (params, seconds))."""
    table = []
    cache = {}

    def timed(p):
        key = tuple(sorted(p.items()))
        if key not in cache:
            cache[key] = time_fn(dict(p))
            table.append((dict(p), cache[key]))
        return cache[key]

    best = {"k": kb_pairs[0][0], "block_bytes": kb_pairs[0][1], "alpha_scale": alphas[0],
            "base_case": int(base_cap(dtype) * base_fracs[0])}
    groups = (
        [{"k": k, "block_bytes": b} for k, b in kb_pairs],
        [{"base_case": int(base_cap(dtype) * f)} for f in base_fracs],
        [{"alpha_scale": a} for a in alphas],
    )
    for options in groups:
        scored = []
        for opt in options:
            p = dict(best)
            p.update(opt)
            t = timed(p)
            if t is not None:
                scored.append((t, p))
        if scored:
            best = min(scored, key=lambda x: x[0])[1]
    return best, table


def cached(path, key, tune):
    """Run tune() -> (best params, table) unless the JSON file at `path`
    already holds parameters for `key`; store the result under `key`.
    Returns (best params, table); the table is empty on a cache hit."""
    if not path:
        return tune()
    store = {}
    if os.path.exists(path):
        with open(path) as f:
            store = json.load(f)
    if key in store:
        return dict(store[key]), []
    best, table = tune()
    store[key] = best
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(store, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best, table


def segmented_signature(lengths):
    """Coarse shape of a batch: arrays, total elements, and the count of
    arrays per log2 length class (0 for empty ones)."""
    hist = {}
    for m in lengths:
        c = 0 if m <= 0 else int(math.floor(math.log2(m))) + 1
        hist[c] = hist.get(c, 0) + 1
    return "arrays=%d,n=%d,log2hist=%s" % (
        len(lengths), sum(lengths), ",".join("%d:%d" % kv for kv in sorted(hist.items())))


def _median_time(torch, run, reps):
    ts = []
    for _ in range(reps):
        ts.append(run())
    return statistics.median(ts)


def tune_array(torch, sample, dtype, reps=3, cache=None, **kw):
    """Tune for plain sorts of arrays like `sample` (a device tensor in the
    storage format of paper_2009_13569_gb300.inputs)."""
    n = sample.shape[0]
    return cached(cache, "array:%s:n=%d" % (dtype, n),
                  lambda: _tune_array(torch, sample, dtype, reps, **kw))


def _tune_array(torch, sample, dtype, reps, **kw):
    n = sample.shape[0]
    work = torch.empty_like(sample)
    stream = torch.cuda.Stream(sample.device)

    def time_fn(params):
        try:
            s = ipsgpu.Sorter(dtype, **params)
        except ipsgpu.IpsgpuError:
            return None
        try:
            s.prepare()

            def run():
                work.copy_(sample)
                torch.cuda.synchronize(sample.device)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.sort(work.data_ptr(), n, stream.cuda_stream)
                e1.record(stream)
                stream.synchronize()
                return e0.elapsed_time(e1) * 1e-3

            run()  # warm-up
            t = _median_time(torch, run, reps)
            return t if s.status(stream.cuda_stream) == ipsgpu.OK else None
        finally:
            s.close()

    return search(time_fn, dtype, **kw)


def tune_segmented(torch, data, offsets, dtype, reps=3, cache=None, **kw):
    """Tune for segmented sorts of batches like (data, offsets): each
    candidate sorter captures the batch into a CUDA graph and is timed on
    graph launches."""
    lengths = (offsets[1:] - offsets[:-1]).cpu().tolist()
    return cached(cache, "segmented:%s:%s" % (dtype, segmented_signature(lengths)),
                  lambda: _tune_segmented(torch, data, offsets, dtype, reps, **kw))


def _tune_segmented(torch, data, offsets, dtype, reps, **kw):
    n = data.shape[0]
    nseg = offsets.numel() - 1
    work = torch.empty_like(data)
    stream = torch.cuda.Stream(data.device)

    def time_fn(params):
        try:
            s = ipsgpu.Sorter(dtype, **params)
        except ipsgpu.IpsgpuError:
            return None
        g = None
        try:
            g = s.segmented_graph(work.data_ptr(), n, offsets.data_ptr(), nseg)

            def run():
                work.copy_(data)
                torch.cuda.synchronize(data.device)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.launch(stream.cuda_stream)
                e1.record(stream)
                stream.synchronize()
                return e0.elapsed_time(e1) * 1e-3

            run()  # warm-up
            t = _median_time(torch, run, reps)
            return t if s.status(stream.cuda_stream) == ipsgpu.OK else None
        finally:
            if g is not None:
                g.close()
            s.close()

    return search(time_fn, dtype, **kw)
