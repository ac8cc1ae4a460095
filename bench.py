"""Benchmark: in-place GPU sort of n = 2^30 uint64 keys drawn uniformly from
[0, 2^64) (seeded, synthetic), k = 256 buckets, 512-byte blocks; next to it
the batched form (many arrays in one launch) and the serving form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one ipsgpu_sort call over the whole array (detection, every
partitioning wave, base case).  The input is restored from a pristine device
copy before each step, outside the timed region; 8 GiB of input is far larger
than the 126 MB L2, so no step runs from cache.  Each step is timed with CUDA
events on the sorting stream, bracketed by a barrier and a device
synchronize; the reported time is the maximum over ranks.  Two timed regions
of K steps each: the first (the value) runs every sort through the sorter's
CUDA graph, the second runs the same sorts from the host-driven wave loop
with CUDA events around every kernel, which give the per-kernel times and
the roofline.  With N > 1 every rank sorts its own array (independent
replicas, weak scaling).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
(sequential C samplesort) on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# request buffers of the serving run range from KiB to 128 GiB: let the
# caching allocator map memory on demand instead of keeping fixed segments
os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")

METRIC = "Gelem/s sorted (uint64, n=2^30)"
UNIT = "Gelem/s"
WORKLOAD = "in-place sort of 2^30 uint64 keys, Uniform [0, 2^64)"
LOG2N = 30
SEED = 0x1B54A32D192ED03
CPU_SAMPLE_LOG2 = 22


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--log2n", type=int, default=LOG2N)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--clocks-log", default=None,
                   help="file for the raw nvidia-smi clock samples of the timed region")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-segmented", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-radix", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="instead of the headline line: one JSON line per run of the plain-sort "
                        "configurations (u32/u64 x 10 distributions x IPS4o/IPS2Ra at 2^30; "
                        "f64, Pair, Quartet and 100-byte records at 2^28), with per-level "
                        "rooflines and full-size property checks")
    p.add_argument("--sweep-dtypes", default="u64,u32,f64,pair,quartet,rec100",
                   help="comma-separated element types the sweep runs")
    p.add_argument("--sweep-shift", type=int, default=0,
                   help="divide every sweep size by 2^shift (small cases for ncu captures)")
    p.add_argument("--sweep-algos", default="IPS4o,IPS2Ra",
                   help="comma-separated algorithms the sweep runs: IPS4o, IPS2Ra (u32/u64 "
                        "only) and IPS4o-tree (IPS4o walking every element from the tree's "
                        "root, without the start-node table)")
    p.add_argument("--serve-only", action="store_true",
                   help="only the serving run (200-request traces at three loads)")
    p.add_argument("--batched-only", action="store_true",
                   help="only the batched form's graph launches (both workloads), one JSON "
                        "line: the command of the batched launch-list profile")
    p.add_argument("--base-only", action="store_true",
                   help="only the base case: one ipsgpu_sort_batch of 8,192 arrays of 16,384 "
                        "uint64 Uniform keys (1 GiB; every array goes straight to the base "
                        "case), timed per kernel; the command of the base-case profile")
    p.add_argument("--instrumented", action="store_true",
                   help="run every sort from the host-driven wave loop (the same kernels, no "
                        "CUDA graph): the form the ncu captures in profiles/ use")
    return p.parse_args()


PARAM_KEYS = {"k": int, "block_bytes": int, "alpha_scale": float, "base_case": int,
              "seed": int, "spin_limit": int, "arena_bytes": int}


def env_params(text=None):
    """Sorter parameters of the headline sort from IPSGPU_PARAMS, e.g.
    "k=128,block_bytes=1024,alpha_scale=0.5" (empty: the library's
    defaults).  Unknown keys are an error."""
    text = os.environ.get("IPSGPU_PARAMS", "") if text is None else text
    out = {}
    for item in filter(None, (x.strip() for x in text.split(","))):
        key, _, val = item.partition("=")
        key = key.strip()
        if key not in PARAM_KEYS or not val:
            raise ValueError("IPSGPU_PARAMS: bad item %r (keys: %s)" % (item, sorted(PARAM_KEYS)))
        out[key] = PARAM_KEYS[key](val.strip())
    return out


def reduce_max_over_ranks(pg, values, device="cpu"):
    """Element-wise maximum over all ranks of a list of floats (the slowest
    rank's time, any rank's failure flag); every rank gets the result.  With
    no process group (one GPU) the values come back unchanged."""
    vals = [float(v) for v in values]
    if not pg:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_value(world, n, ms):
    """Whole-job throughput (Gelem/s) of `world` replicas that each sort n
    elements per step, the step taking the slowest rank's ms."""
    return world * n / (ms * 1e-3) / 1e9


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model, os.cpu_count()


def cpu_baseline(log2n=CPU_SAMPLE_LOG2, reps=1):
    """The oracle as it stands, single-threaded, on a 2^log2n sample of the
    same distribution; returns Gelem/s and a description."""
    import oracle
    from paper_2009_13569_gb300 import inputs
    a = inputs.to_numpy(inputs.generate("uniform", "u64", 1 << log2n, seed=SEED), "u64")
    oracle.build()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.sort(a, "u64")
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    model, ncpu = _cpu_info()
    return {"value": (1 << log2n) / best / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "2^%d uint64 Uniform keys, same generator, sequential C samplesort "
                      "(%s, %s host cores, 1 used), %.2f s" % (log2n, model or "cpu", ncpu, best)}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        import tempfile
        self.index = index
        self.proc = None
        # the raw samples: a file the caller names (--clocks-log), else a
        # temporary file
        self.path = path or os.path.join(tempfile.gettempdir(),
                                         "ipsgpu_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx = max(mx, float(c[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of the dominant kernel per element of a launch, from the ncu
# capture summarised in profiles/ (dram__bytes_read.sum + dram__bytes_write.sum
# of one launch divided by the elements it processed).  It is only valid for
# the kernel source it was measured on, identified by its sha256; otherwise
# the bench reports traffic as null.
NCU_TRAFFIC = {
    "classify": {"bytes_per_elem": 15.16,
                 "source": "paper_2009_13569_gb300/csrc/classify.cuh",
                 "sha256": "ed48567bb31a5be2e150d35747a43430c93d2bff2ee380beb86623724baeec42"},
    "permute": {"bytes_per_elem": 15.31,
                "source": "paper_2009_13569_gb300/csrc/level.cuh",
                "sha256": "b5623d4103c1706c66f1c80072bf3a4a49dfa222ba120374bbe295643b21cd47"},
    "base_case": {"bytes_per_elem": 15.11,
                  "source": "paper_2009_13569_gb300/csrc/base.cuh",
                  "sha256": "5cccd74924ea3ca59a0efbb8052a834a145853c84f3d757a5967503e70fccf28"},
}


def _traffic(kernel, elems_per_launch):
    import hashlib
    t = NCU_TRAFFIC.get(kernel)
    if not t:
        return None
    with open(os.path.join(ROOT, t["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
            return None
    return t["bytes_per_elem"] * elems_per_launch


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    # each step: the oracle on a bounded 2^22 sample of the workload
    vals = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(CPU_SAMPLE_LOG2)
        if i >= args.warmup:
            vals.append(r["value"])
            base = r
    v = statistics.mean(vals)
    n = 1 << CPU_SAMPLE_LOG2
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": n / v / 1e6,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + " (CPU oracle on a 2^22 sample per step)",
                       "n": 1 << LOG2N, "sample_n": n, "dist": "uniform", "seed": SEED},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _segments_sorted(torch, d, offsets):
    """Every adjacent pair inside a segment is ordered (as unsigned)."""
    x = d ^ (-(1 << 63))
    ok = x[1:] >= x[:-1]
    inner = offsets[1:-1]
    inner = inner[(inner > 0) & (inner < d.numel())]
    ok[inner - 1] = True
    return bool(ok.all().item())


SEG_WORKLOADS = (
    # (name, arrays, log2 of the shortest and longest length, total elements)
    ("100k_arrays", 100_000, 4.0, 17.65, None),
    ("loguniform_2^4_2^24", None, 4.0, 24.0, 1 << 31),
)


def run_segmented(torch, inputs, ipsgpu, dev, steps, graph_only=False, instrumented=False):
    """Batched form: many uint64 arrays of log-uniform lengths, mixed
    Uniform / TwoDup / AlmostSorted, sorted by one launch of a captured CUDA
    graph, against one plain ipsgpu_sort call per array on the same GPU.
    graph_only: the graph launches alone (no per-array baseline, no
    autotuning); with instrumented, the same sorts run from the host-driven
    wave loop (ipsgpu_sort_segmented with kernel timing), whose kernels a
    profiler can take one by one: the form of the batched launch-list
    profile."""
    out = {}
    st = torch.cuda.Stream(dev)
    for name, count, lo, hi, total in SEG_WORKLOADS:
        if count is None:
            lengths = inputs.segment_lengths(4096, lo, hi, seed=SEED)
            c = torch.cumsum(lengths, 0)
            lengths = lengths[:int((c <= total).sum())]
        else:
            lengths = inputs.segment_lengths(count, lo, hi, seed=SEED)
        src, offsets = inputs.segmented_batch(lengths, seed=SEED, device=dev)
        N = src.numel()
        work = torch.empty_like(src)
        sorter = ipsgpu.Sorter("u64")
        g = sorter.segmented_graph(work.data_ptr(), N, offsets.data_ptr(), lengths.numel())
        sorter.set_timing(instrumented)
        ts = []
        for i in range(2 + steps):
            work.copy_(src)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            if instrumented:
                sorter.sort_segmented(work.data_ptr(), N, offsets.data_ptr(), lengths.numel(),
                                      st.cuda_stream)
            else:
                g.launch(st.cuda_stream)
            e1.record(st)
            st.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1))
        ok = sorter.status(st.cuda_stream) == ipsgpu.OK and _segments_sorted(torch, work, offsets)
        gms = sum(ts) / len(ts)
        if graph_only:
            out[name] = {"arrays": int(lengths.numel()), "elements": N,
                         "form": "host-driven waves" if instrumented else "CUDA graph",
                         "ms": gms, "value": N / (gms * 1e-3) / 1e9, "unit": UNIT,
                         "result_sorted": ok}
            if instrumented:
                out[name]["kernels_ms"] = {k: round(v[1] / (2 + steps), 3)
                                           for k, v in sorter.kernel_stats().items() if v[0]}
            g.close()
            sorter.close()
            del src, work
            torch.cuda.empty_cache()
            continue
        # one plain sort call per array (the per-array baseline), one pass
        work.copy_(src)
        torch.cuda.synchronize(dev)
        o = offsets.cpu().tolist()
        base = work.data_ptr()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(lengths.numel()):
            a, b = o[i], o[i + 1]
            if b - a > 1:
                sorter.sort(base + 8 * a, b - a, st.cuda_stream)
        e1.record(st)
        st.synchronize()
        pms = e0.elapsed_time(e1)
        ok2 = sorter.status(st.cuda_stream) == ipsgpu.OK and _segments_sorted(torch, work, offsets)
        # the autotuner's pick (k, block bytes, base case, alpha) for this batch
        from paper_2009_13569_gb300 import autotune
        best, table = autotune.tune_segmented(torch, src, offsets, "u64", reps=2)
        ts_t = []
        with ipsgpu.Sorter("u64", **best) as s2:
            g2 = s2.segmented_graph(work.data_ptr(), N, offsets.data_ptr(), lengths.numel())
            for i in range(2 + steps):
                work.copy_(src)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                g2.launch(st.cuda_stream)
                e1.record(st)
                st.synchronize()
                if i >= 2:
                    ts_t.append(e0.elapsed_time(e1))
            ok3 = s2.status(st.cuda_stream) == ipsgpu.OK and _segments_sorted(torch, work, offsets)
            g2.close()
        tms = sum(ts_t) / len(ts_t)
        out[name] = {"arrays": int(lengths.numel()), "elements": N,
                     "lengths": "log-uniform [2^%g, 2^%g]" % (lo, hi),
                     "dists": "Uniform/TwoDup/AlmostSorted by array",
                     "graph_ms": gms, "value": N / (gms * 1e-3) / 1e9, "unit": UNIT,
                     "plain_per_array_ms": pms, "plain_value": N / (pms * 1e-3) / 1e9,
                     "speedup_vs_plain": pms / gms, "graph_nodes": g.nodes(),
                     "autotuned": {"params": best, "graph_ms": tms,
                                   "value": N / (tms * 1e-3) / 1e9,
                                   "candidates": [[p, t] for p, t in table]},
                     "result_sorted": ok and ok2 and ok3, "steps": steps,
                     "l2": "inputs larger than L2 (%.1f GiB)" % (N * 8 / 2 ** 30)}
        g.close()
        sorter.close()
        del src, work, offsets
        torch.cuda.empty_cache()
    return out


SERVE = {"requests": 200, "log2_lo": 10, "log2_hi": 32, "huge_log2": 34, "huge_every": 50,
         "budget_gb": 170, "lanes": 3, "loads": (0.5, 0.8, 0.95), "pool_log2": 30}
SERVE_DISTS = ("uniform", "exponential", "rootdup", "twodup", "eightdup", "almostsorted",
               "zipf", "sorted", "reversesorted", "zero")


def run_serve(torch, inputs, ipsgpu, dev):
    """Serving form: 200 sort requests (sizes log-uniform in [2^10, 2^32],
    uint32 / uint64 / Pair keys in turn, data from the ten plain-sort
    distributions; every 50th request a 2^34-element uint64 request, 128 GiB, sorted
    in place) arriving as a Poisson process at 50, 80 and 95 % of the plain
    sort's capacity, admitted by HBM footprint under a 170 GB budget.  The
    server (continuous batching over streams) runs every trace live; the
    plain form is first-in first-out, one plain sort at a time, whose
    latencies follow from the measured service time of each request sorted
    alone (a single-server queue: the order and the service times fix
    them).

    A request's data arrives in HBM when it is admitted: a copy from a
    pre-generated pool of its type (2^30 elements over the ten
    distributions); a request larger than the pool is tiled with pool
    copies, each tile's keys XORed with its own seeded 64-bit constant.
    Both forms include that copy in the service time and the latency.
    Every result is checked: keys non-decreasing, the multiset of words
    equal to the input's, and so each served result equal to the same
    request sorted alone (the sorted output is unique)."""
    import collections
    import numpy as np
    cfg = SERVE
    R = cfg["requests"]
    # the caching allocator keeps freed request buffers for reuse; held to
    # 85 % of the device it returns them before it would need more
    torch.cuda.set_per_process_memory_fraction(0.85, dev)
    rng = np.random.default_rng(SEED & 0xFFFFFFFF)
    sizes = inputs.segment_lengths(R, cfg["log2_lo"], cfg["log2_hi"], seed=SEED + 5).tolist()
    types = ["u32", "u64", "pair"]
    reqs = []
    for i, m in enumerate(sizes):
        if i % cfg["huge_every"] == cfg["huge_every"] // 2:
            reqs.append({"dtype": "u64", "n": 1 << cfg["huge_log2"], "huge": True,
                         "seed": SEED + 1000 + i})
        else:
            reqs.append({"dtype": types[i % 3], "n": int(m), "seed": SEED + 1000 + i})
    pmax = 1 << cfg["pool_log2"]
    pools = {}
    for t in types:
        shape = (pmax, 2) if t == "pair" else (pmax,)
        pool = torch.empty(shape, dtype=torch.int32 if t == "u32" else torch.int64, device=dev)
        step = pmax // len(SERVE_DISTS)
        for j, d in enumerate(SERVE_DISTS):
            part = pool[j * step:(j + 1) * step if j + 1 < len(SERVE_DISTS) else pmax]
            inputs.generate_into(part, d, t, seed=SEED + 17 * j)
        pools[t] = pool
    for r in reqs:
        r["pooled"] = r["n"] <= pmax
        r["off"] = int(rng.integers(0, pmax - r["n"] + 1)) if r["pooled"] else 0

    def fill(r, buf, stream):
        with torch.cuda.stream(stream):
            pool = pools[r["dtype"]]
            if r["pooled"]:
                buf.copy_(pool[r["off"]:r["off"] + r["n"]])
                return
            for q, a in enumerate(range(0, r["n"], pmax)):
                m = min(pmax, r["n"] - a)
                dst = buf[a:a + m]
                dst.copy_(pool[:m])
                c = inputs.splitmix64_py(q, r["seed"])
                keys = dst[:, 0] if r["dtype"] == "pair" else dst
                if r["dtype"] == "u32":  # int32 storage: the constant's low word, signed
                    c &= 0xFFFFFFFF
                    keys ^= c - (1 << 32) if c >> 31 else c
                else:
                    keys ^= inputs._s64(c)

    def alloc(r):
        shape = (r["n"], 2) if r["dtype"] == "pair" else (r["n"],)
        return torch.empty(shape, dtype=torch.int32 if r["dtype"] == "u32" else torch.int64,
                           device=dev)

    def sorted_ok(buf, t, chunk=1 << 27):
        # non-decreasing keys as unsigned, checked in chunks (bounded temporaries)
        k = buf[:, 0] if t == "pair" else buf
        res = torch.ones((), dtype=torch.bool, device=dev)
        for a in range(0, max(k.shape[0] - 1, 0), chunk):
            x = k[a:a + chunk + 1]
            x = x.to(torch.int64) & 0xFFFFFFFF if t == "u32" else x ^ (-(1 << 63))
            res &= (x[1:] >= x[:-1]).all()
        return res

    # phase A: every request alone, first-in first-out (service times,
    # reference results); the input's multiset is taken from a second fill
    st = torch.cuda.Stream(dev)
    sorters = {t: ipsgpu.Sorter(t) for t in types}
    for t in types:
        sorters[t].prepare()
    service, fifo_ok = [], True
    for r in reqs:
        buf = alloc(r)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fill(r, buf, st)
        sorters[r["dtype"]].sort(buf.data_ptr(), r["n"], st.cuda_stream)
        e1.record(st)
        st.synchronize()
        service.append(e0.elapsed_time(e1) * 1e3)  # us
        with torch.cuda.stream(st):
            ok = bool(sorted_ok(buf, r["dtype"]).item())
            r["sig"] = _multiset_sig_dev(torch, buf)
            fill(r, buf, st)
            ok = ok and bool(torch.equal(_multiset_sig_dev(torch, buf), r["sig"]))
        fifo_ok = fifo_ok and ok
        del buf
        if r.get("huge"):
            torch.cuda.empty_cache()
    fifo_ok = fifo_ok and all(sorters[t].status(st.cuda_stream) == ipsgpu.OK for t in types)
    for t in types:
        sorters[t].close()
    torch.cuda.synchronize(dev)
    total_service = sum(service)
    elems = sum(r["n"] for r in reqs)

    def fifo(arr):
        fin, prev = [], 0.0
        for a, sv in zip(arr, service):
            prev = max(prev, a) + sv
            fin.append(prev)
        return np.array(fin) - arr, (fin[-1] - arr[0]) * 1e-6

    # phase B: the server, live, on a trace of arrival times; requests'
    # data arrive on four copy streams in turn
    check_st = torch.cuda.Stream(dev)
    copy_sts = [torch.cuda.Stream(dev) for _ in range(4)]

    def serve_live(arr, check):
        srv = ipsgpu.Server(cfg["budget_gb"] * 10 ** 9, lanes=cfg["lanes"], dtypes=types)
        nfill = [0]
        t0 = srv.now_us() + 20_000.0
        pending = collections.deque(range(len(reqs)))
        live, lat, waits = {}, [0.0] * len(reqs), [0.0] * len(reqs)
        checks, t_last, huge_done = [], t0, 0
        while pending or live:
            now = srv.now_us()
            progressed = False
            for tk in list(live):
                done, stt = srv.poll(tk)
                if done:
                    i, buf, copy_st = live.pop(tk)
                    _, _, td = srv.times(tk)
                    lat[i] = td - (t0 + arr[i])
                    t_last = max(t_last, td)
                    # a checked run queues the check behind the sort on a
                    # stream of the lowest priority and reads it after the
                    # trace; the buffer is not reused before the check ran
                    if check:
                        check_st.wait_stream(copy_st)
                        with torch.cuda.stream(check_st):
                            checks.append((i, stt, sorted_ok(buf, reqs[i]["dtype"]),
                                           _multiset_sig_dev(torch, buf)))
                        buf.record_stream(check_st)
                    else:
                        checks.append((i, stt, None, None))
                    huge_done += 1 if reqs[i].get("huge") else 0
                    srv.release(tk)
                    del buf
                    progressed = True
            # admission in arrival order; while a large request waits for
            # memory, small ones behind it may still enter (the server keeps
            # a slice of the budget for them), large ones keep their order
            large_blocked = False
            for i in list(pending):
                if t0 + arr[i] > now:
                    break
                r = reqs[i]
                small = r["n"] <= srv.batch_max_elems
                if large_blocked and not small:
                    continue
                tk = srv.reserve(r["n"], r["dtype"])
                if tk is None:
                    if small:
                        break
                    large_blocked = True
                    continue
                waits[i] = srv.now_us() - (t0 + arr[i])
                copy_st = copy_sts[nfill[0] % len(copy_sts)]
                nfill[0] += 1
                buf = alloc(r)
                fill(r, buf, copy_st)
                srv.start(tk, buf.data_ptr(), copy_st.cuda_stream)
                live[tk] = (i, buf, copy_st)
                pending.remove(i)
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        srv.drain()
        torch.cuda.synchronize(dev)
        srv.close()
        ok_ = len(checks) == len(reqs) and all(
            stt == ipsgpu.OK and (not check or (bool(so.item()) and bool(torch.equal(sg, reqs[i]["sig"]))))
            for i, stt, so, sg in checks)
        del checks
        torch.cuda.empty_cache()
        return np.array(lat), max(waits), (t_last - t0) * 1e-6, ok_, huge_done

    def summary(lat):
        return {"p50_ms": float(np.percentile(lat, 50)) * 1e-3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e-3,
                "latency_ms": latency_summary(lat)}

    loads, all_ok, huge_all = [], fifo_ok, True
    gaps0 = rng.exponential(1.0, size=len(reqs))
    for rho in cfg["loads"]:
        lam = rho * len(reqs) / total_service  # arrivals per us
        gaps = gaps0 / lam
        arrival = np.cumsum(gaps) - gaps[0]
        lat, wait_max, span, ok, nh = serve_live(arrival, False)
        flat, fspan = fifo(arrival)
        all_ok = all_ok and ok
        huge_all = huge_all and nh == sum(1 for r in reqs if r.get("huge"))
        loads.append({"load": rho,
                      "server": dict(summary(lat), value=elems / span / 1e9, unit=UNIT,
                                     max_admission_wait_ms=wait_max * 1e-3, status_ok=ok),
                      "plain_fifo": dict(summary(flat), value=elems / fspan / 1e9, unit=UNIT)})
    _, _, sat_span, sat_ok, _ = serve_live(np.zeros(len(reqs)), False)
    # the same requests served once more with every result checked (untimed)
    _, _, _, chk_ok, chk_huge = serve_live(np.zeros(len(reqs)), True)
    all_ok = all_ok and sat_ok and chk_ok
    del pools
    torch.cuda.empty_cache()
    huge = [r for r in reqs if r.get("huge")]
    return {"requests": len(reqs), "elements": int(elems),
            "trace": "Poisson arrivals at %s of the plain sort's capacity; sizes log-uniform "
                     "[2^%d, 2^%d]; u32/u64/Pair in turn over pools of the ten plain-sort "
                     "distributions; "
                     "%d requests of 2^%d uint64 keys (%d GiB, %.0f %% of the requests) in place"
                     % ("/".join("%.0f%%" % (100 * x) for x in cfg["loads"]), cfg["log2_lo"],
                        cfg["log2_hi"], len(huge), cfg["huge_log2"], (1 << cfg["huge_log2"]) * 8 >> 30,
                        100.0 * len(huge) / len(reqs)),
            "data": "copies of a 2^%d-element pool per type (ten distributions); larger requests "
                    "tiled with pool copies, each tile's keys XORed with a seeded 64-bit "
                    "constant; inside service time and latency" % cfg["pool_log2"],
            "budget_gb": cfg["budget_gb"], "lanes": cfg["lanes"],
            "huge_requests_served_every_load": huge_all,
            "loads": loads,
            "saturated": {"server_value": elems / sat_span / 1e9,
                          "plain_fifo_value": elems / (total_service * 1e-6) / 1e9, "unit": UNIT,
                          "form": "every request available at once: elements / makespan"},
            "result_exact": all_ok,
            "latency": "arrival to completion, the arrival of the request's data included",
            "plain_fifo": "simulated single-server FIFO queue over the measured service times of "
                          "the requests sorted alone (fill + ipsgpu_sort each), not run live",
            "checks": "every result of the plain sorts, and of one more served run of all "
                      "requests (not timed; the timed runs check each request's status only): "
                      "keys non-decreasing and the multiset of words equal to the input's, so "
                      "each served result equals the same request sorted alone",
            "checked_run_huge_requests": chk_huge}


def latency_summary(lat_us):
    """Percentiles, mean and a histogram over powers of two of request
    latencies given in microseconds (all figures in milliseconds)."""
    import numpy as np
    a = np.asarray(lat_us, dtype=np.float64) * 1e-3
    if a.size == 0:
        return {"count": 0}
    hist = {}
    for x in a:
        e = int(np.floor(np.log2(x))) if x > 0 else -30
        hist[e] = hist.get(e, 0) + 1
    return {"count": int(a.size), "p50_ms": float(np.percentile(a, 50)),
            "p90_ms": float(np.percentile(a, 90)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max()),
            "histogram_ms": [[2.0 ** e, 2.0 ** (e + 1), c] for e, c in sorted(hist.items())]}


PARTITION_KERNELS = ("sample_tree", "classify", "prep", "fixup", "permute", "stage", "fill", "plan")


def level_roofline(stats, peak, D, n):
    """The distribution levels as a whole: their algorithmic bytes (each
    element read and written by classification and by the permutation,
    4 D per element and level) over the time of every kernel of the
    partitioning waves."""
    by = stats.get("classify", (0, 0.0, 0.0))[2] + stats.get("permute", (0, 0.0, 0.0))[2]
    ms = sum(stats.get(k, (0, 0.0, 0.0))[1] for k in PARTITION_KERNELS)
    if not by or not ms:
        return None
    ach = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "levels": by / (4.0 * D * n), "ms": ms, "bytes": by,
            "kernels": list(PARTITION_KERNELS)}


def _multiset_sig(torch, t):
    """Order-independent signature of a tensor's elements (count, sum, xor
    and sum of squares of its words, each mod 2^64; 32-bit words for u32
    and 100-byte records, 64-bit words otherwise)."""
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
        acc[2] ^= int(_xor_reduce(torch, x))
        acc[3] = (acc[3] + int((x * x).sum().item())) & ((1 << 64) - 1)
    return tuple(acc)


def _multiset_sig_dev(torch, t, chunk=1 << 27):
    """_multiset_sig without the host round trips: a device tensor (sum,
    xor, sum of squares of the words, wrapping int64), queued on the
    current stream, so that a check can run behind other work."""
    if t.dtype == torch.uint8:
        w = t.contiguous().view(torch.int32).reshape(-1).to(torch.int64)
    elif t.element_size() == 4:
        w = t.reshape(-1).view(torch.int32).to(torch.int64)
    else:
        w = t.reshape(-1).view(torch.int64)
    acc = torch.zeros(3, dtype=torch.int64, device=t.device)
    for a in range(0, w.numel(), chunk):
        x = w[a:a + chunk]
        acc[0] += x.sum()
        acc[2] += (x * x).sum()
        y = x
        while y.numel() > 1:
            if y.numel() % 2:
                y = torch.cat([y, torch.zeros(1, dtype=y.dtype, device=y.device)])
            y = y[0::2] ^ y[1::2]
        acc[1] ^= y[0]
    return acc


def _xor_reduce(torch, x):
    while x.numel() > 1:
        if x.numel() % 2:
            x = torch.cat([x, torch.zeros(1, dtype=x.dtype, device=x.device)])
        x = x[0::2] ^ x[1::2]
    return x[0].item() & ((1 << 64) - 1)


def _keys_sorted(torch, t, dtype, chunk=1 << 27):
    """Non-decreasing keys (as unsigned; f64 by its order map), chunked."""
    n = t.shape[0]
    ok = True
    for a in range(0, max(n - 1, 0), chunk):
        x = t[a:a + chunk + 1]
        if dtype == "u32":
            k = x.to(torch.int64) & 0xFFFFFFFF
            ok &= bool((k[1:] >= k[:-1]).all().item())
        elif dtype in ("u64", "pair"):
            k = (x[:, 0] if dtype == "pair" else x) ^ (-(1 << 63))
            ok &= bool((k[1:] >= k[:-1]).all().item())
        elif dtype == "f64":
            b = x.view(torch.int64)
            k = torch.where(b < 0, ~b, b | (-(1 << 63))) ^ (-(1 << 63))
            ok &= bool((k[1:] >= k[:-1]).all().item())
        elif dtype == "quartet":  # three unsigned words, lexicographic
            w = [x[:, j] ^ (-(1 << 63)) for j in range(3)]
            lt = w[2][1:] < w[2][:-1]
            for j in (1, 0):
                lt = (w[j][1:] < w[j][:-1]) | ((w[j][1:] == w[j][:-1]) & lt)
            ok &= not bool(lt.any().item())
        else:  # rec100: 10-byte big-endian unsigned keys, compared bytewise
            kb = x[:, :10].to(torch.int64)
            hi = torch.zeros(kb.shape[0], dtype=torch.int64, device=x.device)
            for j in range(7):
                hi = hi * 256 + kb[:, j]
            lo = kb[:, 7] * 65536 + kb[:, 8] * 256 + kb[:, 9]
            d_hi = hi[1:] - hi[:-1]
            ok &= bool(((d_hi > 0) | ((d_hi == 0) & (lo[1:] >= lo[:-1]))).all().item())
    return ok


E2E_LANES = 3  # streams (each with a sorter and a device buffer) of the end-to-end run


def e2e_lanes(array_bytes, ranks_per_node, mem_available=None):
    """Lanes of the end-to-end run: E2E_LANES, fewer when the pinned host
    buffers of every rank on the node (one input plus one output per lane)
    would take more than half of the host's available memory."""
    if mem_available is None:
        mem_available = 0
        try:
            with open("/proc/meminfo") as f:
                for line in f:
                    if line.startswith("MemAvailable:"):
                        mem_available = int(line.split()[1]) * 1024
        except OSError:
            pass
    if not mem_available:
        return 1
    lanes = E2E_LANES
    while lanes > 1 and (lanes + 1) * array_bytes * ranks_per_node > mem_available // 2:
        lanes -= 1
    return lanes

ALGO_CODES = {"IPS4o": 0, "IPS2Ra": 1, "IPS4o-tree": 2}  # ipsgpu_algo values
ALGO_NAMES = {v: k for k, v in ALGO_CODES.items()}

SWEEP_INT_DISTS = ("uniform", "exponential", "rootdup", "twodup", "eightdup", "almostsorted",
                   "zipf", "sorted", "reversesorted", "zero")


def run_sweep(args):
    """Plain-sort configurations: every distribution for u32/u64 with both
    algorithms at 2^30, and f64 / Pair / Quartet / 100-byte records at 2^28
    with IPS4o; one JSON line each.  Every run is checked at full size by
    properties: keys non-decreasing and the multiset of words unchanged."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2009_13569_gb300 import inputs, ipsgpu
    dev = torch.device("cuda", 0)
    peak, _ = _peak_hbm()
    stream = torch.cuda.Stream(dev)
    runs = []
    want = set(args.sweep_dtypes.split(","))
    algos = [ALGO_CODES[a] for a in args.sweep_algos.split(",")]
    for dtype in ("u64", "u32"):
        for dist in SWEEP_INT_DISTS:
            for algo in algos:
                runs.append((dtype, dist, algo, 30))
    for dtype, dists in (("f64", inputs.F64_DISTS), ("pair", ("uniform",)),
                         ("quartet", ("uniform", "lexdup")), ("rec100", inputs.REC_DISTS)):
        for dist in dists:
            for algo in algos:
                if algo != ipsgpu.RADIX:
                    runs.append((dtype, dist, algo, 28))
    runs = [r for r in runs if r[0] in want]
    cur = None
    for dtype, dist, algo, lg in runs:
        lg -= args.sweep_shift
        n = 1 << lg
        if cur != (dtype, dist, lg):
            src = None
            torch.cuda.empty_cache()
            if dtype in ("u32", "u64", "pair", "quartet"):
                shape = {"pair": (n, 2), "quartet": (n, 4)}.get(dtype, (n,))
                src = torch.empty(shape, dtype=torch.int32 if dtype == "u32" else torch.int64,
                                  device=dev)
                inputs.generate_into(src, dist, dtype, seed=SEED)
            else:
                src = inputs.generate(dist, dtype, n, seed=SEED, device=dev)
            work = torch.empty_like(src)
            sig = _multiset_sig(torch, src)
            cur = (dtype, dist, lg)
        D = ipsgpu.ELEM_BYTES[dtype]
        s = ipsgpu.Sorter(dtype, algo=algo)
        s.prepare()
        times = []
        for rep_ in range(1 + max(args.steps, 5)):
            work.copy_(src)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.sort(work.data_ptr(), n, stream.cuda_stream)
            e1.record(stream)
            stream.synchronize()
            if rep_ > 0:
                times.append(e0.elapsed_time(e1))
        s.set_timing(True)
        work.copy_(src)
        torch.cuda.synchronize(dev)
        s.sort(work.data_ptr(), n, stream.cuda_stream)
        stream.synchronize()
        st = s.status(stream.cuda_stream)
        stats = s.kernel_stats()
        s.close()
        ok = st == ipsgpu.OK and _keys_sorted(torch, work, dtype) and _multiset_sig(torch, work) == sig
        med = statistics.median(times)
        lv = level_roofline(stats, peak, D, n)
        line = {"sweep": True, "dtype": dtype, "dist": dist, "n": n,
                "algo": ALGO_NAMES[algo],
                "value": n / (med * 1e-3) / 1e9, "unit": UNIT, "ms_median": med,
                "ms_mean": statistics.mean(times), "runs": len(times),
                "level_roofline": lv,
                "level_roofline_lower_bound_2Dn": (
                    {"frac": lv["frac"] / 2, "note": "single read+write per level"} if lv else None),
                "kernels_ms": {k: round(v[1], 3) for k, v in stats.items() if v[0]},
                "result_sorted_and_same_multiset": ok}
        print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2009_13569_gb300 import inputs, ipsgpu

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)

    n = 1 << args.log2n
    src = inputs.generate("uniform", "u64", n, seed=SEED + rank, device=dev)
    work = torch.empty_like(src)
    stream = torch.cuda.Stream(dev)
    params = env_params()
    sorter = ipsgpu.Sorter("u64", **params)
    def timed_steps(count):
        ts = []
        for _ in range(count):
            work.copy_(src)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sorter.sort(work.data_ptr(), n, stream.cuda_stream)
            e1.record(stream)
            barrier()
            ts.append(e0.elapsed_time(e1))
        return ts

    # warm-up in both forms: the CUDA graph and the host-driven wave loop
    for mode in (False, True):
        sorter.set_timing(mode)
        for _ in range(args.warmup):
            work.copy_(src)
            torch.cuda.synchronize(dev)
            sorter.sort(work.data_ptr(), n, stream.cuda_stream)
            stream.synchronize()
    assert sorter.status(stream.cuda_stream) == ipsgpu.OK
    sorter.set_timing(False)
    sorter.kernel_stats()  # drop warm-up statistics
    clocks = ClockSampler(local, args.clocks_log)
    clocks.start()
    time.sleep(1.0)  # nvidia-smi is up before the first timed step
    # timed region 1 (the value): the production path, every wave of a sort
    # inside one launch of the sorter's CUDA graph
    times = [] if args.instrumented else timed_steps(args.steps)
    # timed region 2 (the per-kernel figures and the roofline): the same
    # sorts with CUDA events around every kernel, from the host-driven loop
    sorter.set_timing(True)
    itimes = timed_steps(args.steps)
    sorter.set_timing(False)
    clk = clocks.stop()
    stats = sorter.kernel_stats()
    if args.instrumented:
        times = itimes
    graph_ms = None if args.instrumented else sum(times) / len(times)
    inst_ms = sum(itimes) / len(itimes)
    st = sorter.status(stream.cuda_stream)
    # result check outside the timed region: non-decreasing as unsigned and
    # the same multiset of keys as the input (which together fix the output)
    sgn = -(1 << 63)
    src_sig = _multiset_sig(torch, src)
    ok = (bool(((work[1:] ^ sgn) >= (work[:-1] ^ sgn)).all().item()) and st == ipsgpu.OK
          and _multiset_sig(torch, work) == src_sig)
    ms = sum(times) / len(times)
    ms, bad = reduce_max_over_ranks(pg, [ms, 0.0 if ok else 1.0], dev)
    ok = bad == 0.0
    value = replica_value(world, n, ms)

    # roofline of the dominant kernel (algorithmic bytes / mean launch time)
    peak, peak_kind = _peak_hbm()
    kinds = {k: v for k, v in stats.items() if v[0] > 0 and v[2] > 0}
    dom = max(kinds, key=lambda k: kinds[k][1]) if kinds else None
    roof = None
    launches = sum(v[0] for v in stats.values())
    if dom:
        l, kms, by = kinds[dom]
        ach = (by / l) / (kms / l * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": _traffic(dom, by / l / 16.0),
                "peak_source": peak_kind,
                "bytes_per_launch": by / l, "ms_per_launch": kms / l}
    per_kernel = {k: {"launches": v[0] // args.steps, "ms": v[1] / args.steps,
                      "GBps": (v[2] / v[1] / 1e6) if v[1] and v[2] else None}
                  for k, v in stats.items() if v[0]}
    levels = level_roofline(stats, peak, 8, n * args.steps)

    # the radix variant (IPS2Ra) on the same input, both timed forms
    ips2ra = None
    if not args.no_radix:
        rs = ipsgpu.Sorter("u64", algo=ipsgpu.RADIX)
        for mode in (False, True):
            rs.set_timing(mode)
            for _ in range(args.warmup):
                work.copy_(src)
                torch.cuda.synchronize(dev)
                rs.sort(work.data_ptr(), n, stream.cuda_stream)
                stream.synchronize()
        rs.set_timing(False)
        rs.kernel_stats()
        sorter_saved = sorter
        sorter = rs
        rtimes = timed_steps(args.steps)
        rs.set_timing(True)
        ritimes = timed_steps(args.steps)
        rs.set_timing(False)
        sorter = sorter_saved
        rstats = rs.kernel_stats()
        rok = rs.status(stream.cuda_stream) == ipsgpu.OK and bool(
            ((work[1:] ^ sgn) >= (work[:-1] ^ sgn)).all().item()) and (
            _multiset_sig(torch, work) == src_sig)
        rms, rbad = reduce_max_over_ranks(pg, [sum(rtimes) / len(rtimes), 0.0 if rok else 1.0],
                                          dev)
        rok = rbad == 0.0
        ips2ra = {"value": replica_value(world, n, rms), "unit": UNIT, "ms_per_step": rms,
                  "instrumented_ms_per_step": sum(ritimes) / len(ritimes),
                  "level_roofline": level_roofline(rstats, peak, 8, n * args.steps),
                  "result_sorted": rok}
        rs.close()

    e2e = None
    if not args.no_e2e:
        # end to end through the public API (ipsgpu_sort_host): every step
        # copies its input from pinned host memory to the device, sorts it
        # and copies the result back to pinned host memory, all inside the
        # timed region.  Steps go round-robin over the lanes (streams), each
        # with its own sorter and device buffer, so the host->device copy of
        # one step, the kernels of another and the device->host copy of a
        # third run at once (the host link is full duplex).  The same steps
        # on one stream, one after another, are reported as `sequential`.
        lanes = e2e_lanes(n * 8, int(os.environ.get("LOCAL_WORLD_SIZE", "1")))
        hsrc = src.cpu().pin_memory()
        hdst = [torch.empty_like(hsrc).pin_memory() for _ in range(lanes)]
        works = [work] + [torch.empty_like(work) for _ in range(lanes - 1)]
        sorters = [sorter] + [ipsgpu.Sorter("u64", **params) for _ in range(lanes - 1)]
        for s_ in sorters[1:]:
            s_.prepare()
        streams = [stream] + [torch.cuda.Stream(dev) for _ in range(lanes - 1)]

        def e2e_steps(k, lanes):
            barrier()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(streams[0])
            for st_ in streams[1:]:
                st_.wait_event(t0)
            for i in range(k):
                j = i % lanes
                sorters[j].sort_host(hsrc.data_ptr(), hdst[j].data_ptr(), n, works[j].data_ptr(),
                                     streams[j].cuda_stream)
            for st_ in streams[1:]:
                join = torch.cuda.Event()
                join.record(st_)
                streams[0].wait_event(join)
            t1.record(streams[0])
            streams[0].synchronize()
            return t0.elapsed_time(t1) / k

        e2e_steps(lanes, lanes)  # warm-up of every sorter and the copy paths
        ems = e2e_steps(args.steps, lanes)
        sms = e2e_steps(args.steps, 1)
        eok = all(s_.status(st_.cuda_stream) == ipsgpu.OK for s_, st_ in zip(sorters, streams))
        for h in hdst:  # every result buffer checked on the device
            work.copy_(h)
            eok = eok and bool(((work[1:] ^ sgn) >= (work[:-1] ^ sgn)).all().item()) and (
                _multiset_sig(torch, work) == src_sig)
        ems, sms, ebad = reduce_max_over_ranks(pg, [ems, sms, 0.0 if eok else 1.0], dev)
        eok = ebad == 0.0
        e2e = {"value": replica_value(world, n, ems), "unit": UNIT,
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8, "ms_per_step": ems,
               "form": "ipsgpu_sort_host, pinned host buffers, steps round-robin over %d "
                       "streams (copies of some steps overlap the kernels of others)" % lanes,
               "lanes": lanes,
               "sequential": {"value": replica_value(world, n, sms), "ms_per_step": sms,
                              "form": "the same steps on one stream, one after another"},
               "result_sorted": eok}
        for s_ in sorters[1:]:
            s_.close()
        del hsrc, hdst, works

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
    sorter.close()
    del work, src
    torch.cuda.empty_cache()
    seg = None
    if world == 1 and not args.no_segmented:
        seg = run_segmented(torch, inputs, ipsgpu, dev, min(args.steps, 5))
        torch.cuda.empty_cache()
    serve = None
    if world == 1 and not args.no_serve:
        serve = run_serve(torch, inputs, ipsgpu, dev)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "dist": "uniform", "seed": SEED,
                           "k": params.get("k", 256), "block_bytes": params.get("block_bytes", 512),
                           "alpha": "%g*log2(n')" % params.get("alpha_scale", 0.2),
                           "params_override": params or None,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (8 GiB per array)"},
                "result_sorted": ok, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches // args.steps * args.steps, "clocks": clk,
                "timed_form": "CUDA graph" if graph_ms else "host-driven waves, kernel events",
                "instrumented_ms_per_step": inst_ms,
                "level_roofline": levels, "ips2ra": ips2ra,
                "kernels": per_kernel, "segmented": seg, "serve": serve}
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


def run_batched_only(args):
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2009_13569_gb300 import inputs, ipsgpu
    dev = torch.device("cuda", 0)
    seg = run_segmented(torch, inputs, ipsgpu, dev, args.steps, graph_only=True,
                        instrumented=args.instrumented)
    print(json.dumps({"batched_only": True, "segmented": seg}))


def run_base_only(args, nseg=8192, seglen=16384):
    """The base case alone: arrays of seglen keys (the size of a 2^30 sort's
    last-level buckets) sorted by one ipsgpu_sort_batch; every step restores
    the input, sorts with per-kernel timing and checks the result (each
    array non-decreasing, the multiset unchanged) outside the timed part."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2009_13569_gb300 import inputs, ipsgpu
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev).cuda_stream
    n = nseg * seglen
    src = inputs.generate("uniform", "u64", n, seed=SEED, device=dev)
    work = src.clone()
    segs = torch.stack([torch.arange(nseg, dtype=torch.int64, device=dev) * (seglen * 8)
                        + work.data_ptr(),
                        torch.full((nseg,), seglen, dtype=torch.int64, device=dev)], 1).contiguous()
    sig0 = _multiset_sig(torch, src)
    ms, ok = [], True
    with ipsgpu.Sorter("u64") as s:
        s.set_timing(True)
        for i in range(args.warmup + args.steps):
            work.copy_(src)
            torch.cuda.synchronize(dev)
            s.kernel_stats()
            s.sort_batch(segs.data_ptr(), nseg, st)
            if s.status(st) != ipsgpu.OK:
                raise SystemExit("base-only: sort failed")
            k = s.kernel_stats().get("base_case", (0, 0.0, 0.0))
            if i >= args.warmup:
                ms.append(k[1])
            u = work.view(nseg, seglen) ^ (-0x8000000000000000)
            ok = ok and bool((u[:, 1:] >= u[:, :-1]).all()) and _multiset_sig(torch, work) == sig0
    mean = sum(ms) / len(ms)
    print(json.dumps({"base_only": True, "arrays": nseg, "keys_per_array": seglen,
                      "base_case_ms": mean, "GBps": 2.0 * 8 * n / (mean * 1e-3) / 1e9,
                      "steps": args.steps, "warmup": args.warmup, "result_sorted": ok}))


def run_serve_only(args):
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2009_13569_gb300 import inputs, ipsgpu
    dev = torch.device("cuda", 0)
    print(json.dumps({"serve_only": True, "serve": run_serve(torch, inputs, ipsgpu, dev)}))


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.batched_only:
        run_batched_only(args)
    elif args.serve_only:
        run_serve_only(args)
    elif args.base_only:
        run_base_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
