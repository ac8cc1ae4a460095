"""Benchmark: in-place GPU sort of n = 2^30 uint64 keys drawn uniformly from
[0, 2^64) (seeded, synthetic), k = 256 buckets, 512-byte blocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one ipsgpu_sort call over the whole array (detection, every
partitioning level, base case).  The input is restored from a pristine
device copy before each step, outside the timed region; 8 GiB of input is
far larger than the 126 MB L2, so no step runs from cache.  Each step is
timed with CUDA events on the sorting stream, bracketed by a barrier and a
device synchronize; the reported time is the maximum over ranks.  With N > 1
every rank sorts its own array (independent replicas, weak scaling).

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
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


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

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

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
    "classify": {"bytes_per_elem": 15.1198,
                 "source": "paper_2009_13569_gb300/csrc/classify.cuh",
                 "sha256": "afc09346e15ad1910a79def3a02ff9f1c1171deb2be3c34107e535f22ece0623"},
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
    sorter = ipsgpu.Sorter("u64")
    for _ in range(args.warmup):
        work.copy_(src)
        torch.cuda.synchronize(dev)
        sorter.sort(work.data_ptr(), n, stream.cuda_stream)
        stream.synchronize()
    assert sorter.status(stream.cuda_stream) == ipsgpu.OK
    sorter.kernel_stats()  # drop warm-up statistics
    sorter.set_timing(True)
    clocks = ClockSampler(local)
    times = []
    clocks.start()
    for _ in range(args.steps):
        work.copy_(src)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sorter.sort(work.data_ptr(), n, stream.cuda_stream)
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    sorter.set_timing(False)
    stats = sorter.kernel_stats()
    st = sorter.status(stream.cuda_stream)
    # result check outside the timed region: non-decreasing as unsigned
    sgn = -(1 << 63)
    ok = bool(((work[1:] ^ sgn) >= (work[:-1] ^ sgn)).all().item()) and st == ipsgpu.OK
    ms = sum(times) / len(times)
    if pg:
        t = torch.tensor([ms, 0.0 if ok else 1.0], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms, bad = float(t[0]), float(t[1])
        ok = bad == 0.0
    value = world * n / (ms * 1e-3) / 1e9

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

    e2e = None
    if not args.no_e2e:
        # end to end through the public API: pinned host -> device, sort,
        # device -> host, all inside the timed region
        hsrc = src.cpu().pin_memory()
        hdst = torch.empty_like(hsrc).pin_memory()
        et = []
        for i in range(1 + args.steps):
            barrier()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                t0.record(stream)
                work.copy_(hsrc, non_blocking=True)
                sorter.sort(work.data_ptr(), n, stream.cuda_stream)
                hdst.copy_(work, non_blocking=True)
                t1.record(stream)
            stream.synchronize()
            if i > 0:
                et.append(t0.elapsed_time(t1))
        ems = sum(et) / len(et)
        if pg:
            t = torch.tensor([ems], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ems = float(t[0])
        e2e = {"value": world * n / (ems * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8, "ms_per_step": ems}
        del hsrc, hdst

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "dist": "uniform", "seed": SEED,
                           "k": 256, "block_bytes": 512, "alpha": "0.2*log2(n')",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (8 GiB per array)"},
                "result_sorted": ok, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches // args.steps * args.steps, "clocks": clk,
                "kernels": per_kernel}
        print(json.dumps(line))
    sorter.close()
    if pg:
        pg.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
