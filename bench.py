#!/usr/bin/env python3
"""Benchmark of the all-pairs Jaccard hot path (one JSON line on rank 0).

Workload (default): 1024 samples, values in [0, 2^32), log-normal set sizes
(median 1e6, range 1e5-1e7), 32 clades with a 30 % shared core and 0-40 %
substitution; about 1.3e9 values (10.5 GB) in total, seeded and synthetic.

A step is one jsim_all_pairs call on that collection: validation, every row
batch's filter, rank scan and bitmask pack, the AND+popcount product, and
the epilogue that writes C (uint32), |X_i| and J (binary64).

  value  dense AND+popcount bit-operations per second (Tbit-ops/s) of whole
         steps with the inputs resident in HBM: 64 * sum_l W_l * n(n+1)/2
         per step divided by the step time (CUDA events on the library's
         stream, max over ranks).
  e2e    the same metric through the same C-ABI call with pinned host input
         and host output buffers: host->device copy of the values and
         device->host copy of C, sizes and J inside the timed region.

--impl reference times the CPU oracle (pairwise sorted merge, all host
cores) on a bounded sample of pairs of the same workload, scaled to the same
metric.  Multi-GPU runs (torchrun) give every rank its own collection drawn
with a rank-specific seed (independent problems, weak scaling, no collective
on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2**20
METRIC = "AND-popcount Tbit-ops/s & all-pairs time vs roofline; query p50/p99 latency"
UNIT = "Tbit-ops/s"
POPC_PER_CLK_PER_SM = 16        # 32-bit population counts per clock per SM
SMS = 152
SM_MAX_MHZ = 2070.0
VARIANT_NAME = {"sparse": "block-sparse product", "tc2": "dense SM-pair product", "tc": "dense one-SM product",
                "popc": "CUDA-core product"}
LEGACY_INT_MMA_TOPS = 73.0      # mma.sync m16n8k32 s8 / m16n8k256 b1 multiply-adds per second, measured


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jsim", choices=["jsim", "reference"])
    ap.add_argument("--workload", default="clade1024",
                    choices=["clade1024", "ancestral64", "batched200", "stream4096", "serve2048",
                             "bernoulli10k", "density", "product", "serve-one"],
                    help="product: jsim_product alone on random packed words (--n, --words, --pad, --density, "
                         "--calls; the capture case of the product kernels); serve-one: a serving index of the "
                         "reference recipe at --median with requests submitted one at a time (the capture case "
                         "of the query kernel)")
    ap.add_argument("--variant", default="auto")
    ap.add_argument("--batch-rows", type=int, default=0)
    ap.add_argument("--filter-min", type=int, default=1, choices=[1, 2],
                    help="2: the filter keeps rows two or more samples hold (same C and J, fewer words)")
    ap.add_argument("--split", action="store_true",
                    help="strong scaling: every rank takes one part of the same collection's row batches "
                         "(jsim_all_pairs_part), one all-reduce sums the counts, rank 0 forms C and J "
                         "(the default for the default workload on more than one rank)")
    ap.add_argument("--replicas", action="store_true",
                    help="on more than one rank: every rank runs its own collection (weak scaling, no "
                         "collective) instead of the split contraction")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="default workload: skip the serving, batched and two-or-more-filter sub-measurements")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--words", type=int, default=32768)
    ap.add_argument("--pad", type=int, default=0, help="product: words of padding after every row")
    ap.add_argument("--density", type=float, default=0.25, help="product: bit density of the random words")
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--median", type=float, default=None,
                    help="serve-one: set-size median of the reference (default 2e4); clade1024: a smaller "
                         "set-size median than the recipe's 1e6, for profiler captures")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def bind_near_gpu(device):
    """Restrict this process to the host CPUs next to the GPU (its NUMA
    node, from sysfs), so that pinned host buffers, allocated after this,
    sit in the memory closest to the GPU.  Best effort: unchanged when sysfs
    says nothing or the sets do not meet."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(device)
        bdf = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bdf) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        near = cpus & os.sched_getaffinity(0)
        if near and near != os.sched_getaffinity(0):
            os.sched_setaffinity(0, near)
            return sorted(near)
    except Exception:
        pass
    return None


def aggregate_over_ranks(ms, work, device=None):
    """Whole-job timing over ranks: the slowest rank's time and the summed
    work (units every rank processed), one all-reduce each; identity on one
    process.  `device` is where the reduction tensors live (the rank's GPU
    under NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(work)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


def make_workload(name, rank, alloc=None, median=None):
    from paper_1911_04200_gb300 import synth
    if name == "ancestral64":
        off, ids = synth.ancestral64(seed=synth.SEED_BASE + 1 + 1000 * rank, alloc=alloc)
        cfg = {"workload": "ancestral64: n=64, values in [0,2^20), 8 ancestors x 50k, 0-60% replaced",
               "n": 64, "id_bits": 20}
    elif name == "bernoulli10k":
        off, ids = synth.bernoulli10k(seed=synth.SEED_BASE + 6 + 1000 * rank, alloc=alloc)
        cfg = {"workload": "bernoulli10k: n=10,000 samples, m=2^25 rows, every entry present with p=0.01 "
                           "(the paper's synthetic strong-scaling matrix)",
               "n": 10_000, "id_bits": 25}
    else:
        m = median or 1e6
        off, ids = synth.clade1024(seed=synth.SEED_BASE + 2 + 1000 * rank, alloc=alloc, median=m)
        cfg = {"workload": "clade1024: n=1024, values in [0,2^32), log-normal sizes median %.0e "
                           "(%.0e-%.0e), 32 clades, 30%% core, 0-40%% substitution" % (m, m / 10, m * 10),
               "n": 1024, "id_bits": 32}
    return off, ids, cfg


def dense_bitops(ids, n, batch_rows, id_bits):
    """64 * sum_l ceil(R_l / 64) * n(n+1)/2 for batches of batch_rows values."""
    from paper_1911_04200_gb300 import synth
    rb = int(math.log2(batch_rows))
    nr = max(1, (1 << id_bits) >> rb)
    counts = synth.range_distinct(ids, rb, nr)
    W = int(sum((int(c) + 63) // 64 for c in counts))
    return 64.0 * W * n * (n + 1) / 2.0, W


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # samples go to a scratch file; the JSON line carries their summary
        # (JSIM_CLOCKS_CSV keeps them at a chosen path)
        self.path = os.environ.get("JSIM_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "jsim_clocks_%d_rank%d.csv" % (os.getpid(), device))

    def __enter__(self):
        try:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r[2] > 300.0] or rows
        sm = sorted(r[0] for r in busy)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in busy:
            for nm, v in zip(names, r[3][1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "samples_under_load": len(busy),
                "power_w_max": max(r[2] for r in rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def roofline_for(variant, bitops_per_launch, ms_per_launch, peaks, traffic):
    achieved_t = bitops_per_launch / (ms_per_launch * 1e-3) / 1e12 if ms_per_launch > 0 else 0.0
    if variant in ("popc",):
        peak = SMS * POPC_PER_CLK_PER_SM * 32 * SM_MAX_MHZ * 1e6 / 1e12
        return {"bound": "alu", "achieved": round(achieved_t, 3), "peak": round(peak, 3), "unit": "Tbit-ops/s",
                "frac": round(achieved_t / peak, 4), "traffic": traffic,
                "peak_source": "derived: 152 SMs x 16 POPC/clk x 32 bits x 2070 MHz"}
    # tensor variants: one 0/1 multiply-add per bit-operation, 2 FLOP each;
    # fp8 dense peak = measured bf16 (sustained) x 2 (nominal fp8:bf16 ratio)
    pk, src = peaks
    if variant in ("i8", "b1"):
        # the legacy integer/binary mma.sync pipe: one bit-operation per 0/1
        # multiply-add (i8) or per AND+popcount bit (b1); its rate measured on
        # this GPU with the kernels' own instruction shapes
        peak = LEGACY_INT_MMA_TOPS
        return {"bound": "tensor", "achieved": round(achieved_t, 3), "peak": peak, "unit": "Tbit-ops/s",
                "frac": round(achieved_t / peak, 4), "traffic": traffic,
                "peak_source": "measured legacy mma.sync s8/b1 issue rate (%.0f T ops/s)" % peak}
    flops = 2.0 * achieved_t
    peak = pk.get("bf16_tflops_sustained", 1700.0) * 2.0
    return {"bound": "tensor", "achieved": round(flops, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(flops / peak, 4), "traffic": traffic,
            "peak_source": "%s bf16 sustained x 2 (fp8:bf16 nominal ratio)" % src}


def traffic_from_profiles(variant, workload):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        return d.get("%s/%s" % (variant, workload))
    except Exception:
        return None


def cpu_baseline(off, ids, n, bitops_total, seconds):
    """Oracle (pairwise sorted merge) on a bounded random sample of pairs, all host cores."""
    import oracle
    threads = oracle.default_threads()
    rng = np.random.default_rng(12345)
    total_pairs = n * (n + 1) // 2
    # merge random pairs in growing rounds until about `seconds` of work
    k2, dt, k = 0, 0.0, max(threads, 16)
    while dt < seconds and k2 < total_pairs:
        k = int(min(k, total_pairs - k2))
        pi = rng.integers(0, n, k).astype(np.uint64)
        pj = rng.integers(0, n, k).astype(np.uint64)
        t0 = time.perf_counter()
        oracle.pairs(off, ids, pi, pj, threads)
        dt += time.perf_counter() - t0
        k2 += k
        k *= 2
    value = bitops_total * (k2 / total_pairs) / dt / 1e12
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d random pairs of the %d-sample workload merged in %.1f s; scaled by pairs to the "
                      "dense bit-operations of all %d pairs" % (k2, n, dt, total_pairs),
            "seconds": dt, "pairs": k2, "projected_all_pairs_s": dt * total_pairs / k2}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    off, ids, cfg = make_workload(args.workload, 0)
    n = cfg["n"]
    br = args.batch_rows or (1 << min(28, cfg["id_bits"]))
    bitops, W = dense_bitops(ids, n, br, cfg["id_bits"])
    steps = []
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(off, ids, n, bitops, max(2.0, args.cpu_seconds / max(1, args.steps)))
        if s >= args.warmup:
            steps.append(cb)
    value = float(np.mean([c["value"] for c in steps]))
    cfg.update({"batch_rows": br, "words": W, "bitops_dense_per_step": bitops})
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([c["projected_all_pairs_s"] for c in steps])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": steps[0]["cores"], "kind": "oracle",
                             "sample": steps[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batched_measure(cols, steps, warmup, batch_rows=0):
    """Independent collections [(offsets, ids), ...] in device memory: one
    jsim_all_pairs_batched call per step (persistent multi-collection launch,
    CUDA-graph replay) against one jsim_all_pairs call per collection, same
    inputs and outputs; both checked equal.  Returns a dict of the timings."""
    import ctypes
    import torch
    from paper_1911_04200_gb300 import jsim
    dev = torch.device("cuda", 0)
    dcols = [(torch.from_numpy(o.view(np.int64)).to(dev), torch.from_numpy(i.view(np.int64)).to(dev)) for o, i in cols]
    N = sum(int(o[-1]) for o, _ in cols)
    ctx = jsim.Context(device=0, id_bits=32, profile=False, batch_rows=batch_rows)
    # preallocated outputs so the captured graph is replayed every step
    k = len(dcols)
    Cs = [torch.empty((len(o) - 1, len(o) - 1), dtype=torch.uint32, device=dev) for o, _ in cols]
    Ss = [torch.empty(len(o) - 1, dtype=torch.uint64, device=dev) for o, _ in cols]
    Js = [torch.empty((len(o) - 1, len(o) - 1), dtype=torch.float64, device=dev) for o, _ in cols]
    sets = (jsim.Sets * k)()
    for c, (o, i) in enumerate(dcols):
        sets[c] = jsim.Sets(len(cols[c][0]) - 1, o.data_ptr(), i.data_ptr() if i.numel() else None, jsim.MEM_DEVICE)
    arr = lambda L: (ctypes.c_void_p * k)(*[t.data_ptr() for t in L])
    Cp, Sp, Jp = arr(Cs), arr(Ss), arr(Js)
    lib = jsim.load()

    def call():
        ctx._order()
        rc = lib.jsim_all_pairs_batched(ctx._h, sets, k, Cp, Sp, Jp, jsim.MEM_DEVICE)
        jsim._check(rc, ctx._h)
        return ctx.stats()

    for _ in range(warmup):
        st = call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    bo = 0.0
    for _ in range(steps):
        st = call()
        bo += st["bitops_dense"]
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / steps
    variant = st["variant"]
    batched_J = [j.clone() for j in Js]
    # plain: one all-pairs call per collection
    pctx = jsim.Context(device=0, id_bits=32)
    plain_out = [(Cs[c], Ss[c], Js[c]) for c in range(k)]
    for c, (o, i) in enumerate(dcols):
        pctx.all_pairs(o, i, out=plain_out[c])
    torch.cuda.synchronize()
    e0.record(pctx.stream)
    for _ in range(steps):
        for c, (o, i) in enumerate(dcols):
            pctx.all_pairs(o, i, out=plain_out[c])
    e1.record(pctx.stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / steps
    same = all(bool(torch.equal(a.view(torch.int64), b.view(torch.int64))) for a, b in zip(batched_J, Js))
    ctx.close()
    pctx.close()
    bitops = bo / steps
    return {"ms_batched": ms_b, "ms_plain": ms_p, "speedup_vs_plain": ms_p / ms_b, "variant": variant,
            "bitops_dense_per_step": bitops, "value": bitops / (ms_b * 1e-3) / 1e12,
            "plain_value": bitops / (ms_p * 1e-3) / 1e12, "collections": k,
            "samples": sum(len(o) - 1 for o, _ in cols), "values": N, "same_J_as_plain": same}


def run_batched(args):
    """200 independent collections (n ~ U{8..512}, log-normal sizes, clade
    model): the batched call against one plain call per collection."""
    from paper_1911_04200_gb300 import synth
    median = float(os.environ.get("JSIM_BATCHED_MEDIAN", "2e4"))
    count = int(os.environ.get("JSIM_BATCHED_COUNT", "200"))
    cols = synth.batched_collections(median=median, lo=1e4, hi=5e6, count=count)
    m = batched_measure(cols, args.steps, args.warmup, args.batch_rows)
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_batched"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 ids, u32 counts, f64 J", "data": "synthetic",
            "config": {"workload": "batched200: %s%d collections, n ~ U{8..512}, log-normal sizes median %.0e, "
                                   "values in [0,2^32), ceil(n/32) clades"
                                   % ("the first " if count < 200 else "", count, median),
                       "collections": m["collections"], "samples": m["samples"], "values": m["values"],
                       "variant": m["variant"], "bitops_dense_per_step": m["bitops_dense_per_step"]},
            "plain": {"value": m["plain_value"], "ms_per_step": m["ms_plain"],
                      "how": "one jsim_all_pairs call per collection (AUTO variant), same inputs/outputs"},
            "speedup_vs_plain": m["speedup_vs_plain"], "same_J_as_plain": m["same_J_as_plain"]}
    print(json.dumps(line))
    return 0


def run_streamed(args):
    """The 4096-sample clade recipe over [0, 2^40) in (pageable) host memory,
    64-bit counts, row batches of 2^26 values: one jsim_all_pairs_streamed
    call per step (super-batches gathered into two pinned staging buffers,
    copies on a second stream overlapping the product) against one plain
    jsim_all_pairs call on the same host input (one copy of all values, then
    the batch loop).  Both write C, sizes and J to host memory; both are
    timed on the wall clock around the call, which returns after its last
    copy."""
    import torch
    from paper_1911_04200_gb300 import jsim, synth
    median = float(os.environ.get("JSIM_STREAM_MEDIAN", "2e5"))
    staging = int(os.environ.get("JSIM_STREAM_STAGING", str(1 << 30)))
    br = args.batch_rows or (1 << 26)
    off, ids = synth.clade4096(median=median)
    n = len(off) - 1
    N = int(off[-1])
    hC = torch.empty((n, n), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    hS = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    hJ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy()
    ctx = jsim.Context(device=0, variant=args.variant, batch_rows=br, count_bits=64, id_bits=40, profile=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        agg = {"ms_product": 0.0, "product_launches": 0, "launches": 0, "bitops": 0.0}
        for _ in range(args.steps):
            fn()
            st = ctx.stats()
            agg["ms_product"] += st["ms_product"]
            agg["product_launches"] += st["product_launches"]
            agg["launches"] += st["launches"]
            agg["bitops"] += st["bitops_dense"]
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / args.steps, st, agg

    with Clocks(0) as clk:
        dt_s, st_s, agg = timed(lambda: ctx.all_pairs_streamed(off, ids, staging_bytes=staging, out=(hC, hS, hJ)))
    J_s = hJ.copy()
    plain = os.environ.get("JSIM_STREAM_PLAIN", "1") != "0"
    if plain:
        # the plain form: one copy of all values to the device, then the batch
        # loop (jsim_all_pairs itself streams host input this large)
        dev = torch.device("cuda", 0)

        def plain_call():
            d_off = torch.from_numpy(off.view(np.int64)).to(dev)
            d_ids = torch.from_numpy(ids.view(np.int64)).to(dev)
            ctx.all_pairs(d_off, d_ids, out=(hC, hS, hJ), out_device=False)
        dt_p, st_p, _ = timed(plain_call)
        assert np.array_equal(J_s.view(np.uint64), hJ.view(np.uint64)), "streamed and plain results differ"
    bitops = st_s["bitops_dense"]
    variant = st_s["variant"]
    roof = roofline_for(variant, agg["bitops"] / max(1, agg["product_launches"]),
                        agg["ms_product"] / max(1, agg["product_launches"]), measured_peaks(),
                        traffic_from_profiles(variant, "stream4096"))
    stages = ("ms_h2d", "ms_validate", "ms_filter", "ms_scan", "ms_pack", "ms_product", "ms_epilogue", "ms_d2h")
    line = {"metric": METRIC, "value": bitops / dt_s / 1e12, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 ids, u64 counts, f64 J", "data": "synthetic",
            "config": {"workload": "stream4096: n=4096, values in [0,2^40), log-normal sizes median %.0e "
                                   "(x/10-10x), 64 clades, 30%% core, 0-40%% substitution" % median,
                       "values": N, "host_bytes": N * 8, "staging_bytes": staging, "batch_rows": br,
                       "batches": st_s["batches"], "words": st_s["words"], "rows_nonzero": st_s["rows_nonzero"],
                       "variant": variant, "bitops_dense_per_step": bitops,
                       "product_launches": st_s["product_launches"],
                       "h2d_gbs_effective": N * 8 / dt_s / 1e9,
                       "stage_ms": {k: round(st_s[k], 3) for k in stages},
                       "l2": "inputs (%.1f GB) larger than L2 (129 MB); no flush" % (N * 8 / 1e9)},
            "clocks": clk.summary(), "gpu_launches": agg["launches"], "roofline": roof,
            "e2e": {"value": bitops / dt_s / 1e12, "unit": UNIT, "h2d_bytes_per_step": int(N * 8 + (n + 1) * 8),
                    "d2h_bytes_per_step": int(n * n * 16 + n * 8)},
            "plain": {"value": bitops / dt_p / 1e12, "ms_per_step": dt_p * 1e3, "batches": st_p["batches"],
                      "how": "one copy of the pageable host input to the device, then one jsim_all_pairs "
                             "call (host outputs)",
                      "stage_ms": {k: round(st_p[k], 3) for k in stages}} if plain else None,
            "speedup_vs_plain": dt_p / dt_s if plain else None}
    print(json.dumps(line))
    ctx.close()
    return 0


def serve_measure(median, n_req, slots, warmup, pool=512, plain_requests=2):
    """Serving: a resident index of a 2048-sample reference (values in
    [0, 2^32), log-normal sizes of the given median, 64 clades) and requests
    of U{1..64} query samples from the same clades.  Capacity = requests/s of
    a closed burst; then Poisson arrivals at 0.5, 0.8 and 0.95 x capacity with
    p50/p99 request latency (submit to results ready, host clock).  The plain
    form answers a request with one jsim_all_pairs call on reference + query
    samples (the only way to get query x reference counts without an index);
    its results equal the index's.  Returns a dict."""
    from paper_1911_04200_gb300 import jsim, synth
    roff, rids = synth.serving_reference(median=median)
    qoff, qids = synth.serving_queries(0, pool, median=median)
    n_ref = len(roff) - 1
    rng = np.random.default_rng(11)

    def request():
        q = int(rng.integers(1, 65))
        a = int(rng.integers(0, pool - q + 1))
        return (qoff[a:a + q + 1] - qoff[a]).astype(np.uint64), qids[int(qoff[a]):int(qoff[a + q])]

    sizes = np.diff(qoff.astype(np.int64))
    max_vals = int(np.sort(sizes)[-64:].sum())
    ctx = jsim.Context(device=0, id_bits=32)
    t0 = time.perf_counter()
    ix = jsim.Index(ctx, roff, rids, max_batch_samples=64, max_batch_values=max_vals, slots=slots)
    build_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(warmup, 1)):
        ix.submit(*request()).wait()

    def run(reqs, gaps=None):
        st0 = ix.stats()
        handles = []
        t_begin = time.perf_counter()
        if gaps is None:
            handles = [ix.submit(*r) for r in reqs]
        else:
            t_next = t_begin
            for r, g in zip(reqs, gaps):
                t_next += g
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                handles.append(ix.submit(*r))
        for h in handles:
            h.wait()
        elapsed = time.perf_counter() - t_begin
        lat = np.array([h.latency()[1] for h in handles])
        st1 = ix.stats()
        for h in handles:
            h.free()
        d = {k: st1[k] - st0[k] for k in ("batches", "samples_done", "values_done", "ms_device", "ms_product",
                                          "index_bytes_read", "rows_read")}
        return elapsed, lat, d

    reqs = [request() for _ in range(n_req)]
    with Clocks(0) as clk:
        elapsed, lat, d = run(reqs)
    capacity = n_req / elapsed
    samples = sum(len(o) - 1 for o, _ in reqs)
    levels = {}
    for f in (0.5, 0.8, 0.95):
        lam = f * capacity
        rq = [request() for _ in range(n_req)]
        gaps = rng.exponential(1.0 / lam, n_req)
        el, lt, _ = run(rq, gaps)
        levels["%.2f" % f] = {"rate_rps": round(lam, 2), "achieved_rps": round(n_req / el, 2),
                              "p50_ms": round(float(np.percentile(lt, 50)), 3),
                              "p99_ms": round(float(np.percentile(lt, 99)), 3),
                              "mean_ms": round(float(lt.mean()), 3)}
    plain_ms = []
    pctx = jsim.Context(device=0, id_bits=32)
    for k in range(plain_requests):
        o, v = reqs[k]
        off = np.concatenate([roff, roff[-1] + o[1:]]).astype(np.uint64)
        ids = np.concatenate([rids, v])
        t0 = time.perf_counter()
        C, S, J = pctx.all_pairs(off, ids, want_J=True)
        plain_ms.append((time.perf_counter() - t0) * 1e3)
        h = ix.submit(o, v)
        Cs, Ss, Js = h.wait()
        h.free()
        assert np.array_equal(Cs, C[n_ref:, :n_ref]) and np.array_equal(Js.view(np.uint64),
                                                                         J[n_ref:, :n_ref].view(np.uint64))
    pctx.close()
    pk, src = measured_peaks()
    # algorithmic bytes of the query kernel: per row read, the row plus the
    # value's 8 bytes and its 16-byte filter entry (word, rank of its first bit)
    alg = d["index_bytes_read"] + 24.0 * d["rows_read"]
    achieved = alg / (d["ms_product"] * 1e-3) / 1e9 if d["ms_product"] else 0.0
    tq = traffic_from_profiles("qrows", "serve2048")
    traffic = (round(tq["bytes_per_row"] * d["rows_read"] / max(1, d["batches"]))
               if isinstance(tq, dict) and "bytes_per_row" in tq else None)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
            "kernel": "k_qrows", "peak_source": "%s HBM copy bandwidth" % src,
            "unit_bytes": "per query value the filter holds: its row (ceil(n_ref/64) x 8 B) + 8 B value + "
                          "16 B filter entry (word, rank of its first bit)"}
    out = {"capacity_rps": capacity, "elapsed_s": elapsed, "requests": n_req, "query_samples": samples,
           "samples_per_s": samples / elapsed, "latency": levels, "clocks": clk.summary(), "roofline": roof,
           "index_rows": ix.rows, "index_bytes": ix.rows * ((n_ref + 63) // 64) * 8, "build_ms": round(build_ms, 1),
           "batches": d["batches"], "samples_per_batch": d["samples_done"] / max(1, d["batches"]),
           "device_ms_per_batch": d["ms_device"] / max(1, d["batches"]),
           "qprod_ms_per_batch": d["ms_product"] / max(1, d["batches"]),
           "rows_read_per_batch": d["rows_read"] / max(1, d["batches"]),
           "values_per_request": d["values_done"] / n_req, "n_ref": n_ref, "slots": slots,
           "plain_ms_per_request": float(np.mean(plain_ms)),
           "speedup_vs_plain": capacity * float(np.mean(plain_ms)) / 1e3}
    ix.close()
    ctx.close()
    return out


def run_serve(args):
    """The serving workload (serve_measure) as its own JSON line."""
    median = float(os.environ.get("JSIM_SERVE_MEDIAN", "1e5"))
    n_req = int(os.environ.get("JSIM_SERVE_REQUESTS", "400"))
    slots = int(os.environ.get("JSIM_SERVE_SLOTS", "3"))
    m = serve_measure(median, n_req, slots, args.warmup)
    n_ref = m["n_ref"]
    line = {"metric": METRIC, "value": m["capacity_rps"], "unit": "requests/s", "n_gpus": 1, "steps": n_req,
            "warmup": args.warmup, "ms_per_step": m["elapsed_s"] / n_req * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 ids, u32 counts, f64 J", "data": "synthetic",
            "config": {"workload": "serve2048: reference n=2048, values in [0,2^32), log-normal sizes median "
                                   "%.0e (x/10-10x), 64 clades; requests of U{1..64} query samples of the same "
                                   "recipe" % median,
                       "index_rows": m["index_rows"], "index_bytes": m["index_bytes"], "build_ms": m["build_ms"],
                       "requests": n_req, "query_samples": m["query_samples"], "samples_per_s": m["samples_per_s"],
                       "batches": m["batches"], "samples_per_batch": m["samples_per_batch"],
                       "device_ms_per_batch": m["device_ms_per_batch"], "qprod_ms_per_batch": m["qprod_ms_per_batch"],
                       "rows_read_per_batch": m["rows_read_per_batch"],
                       "l2": "index (%.1f GB) larger than L2; no flush" % (m["index_bytes"] / 1e9)},
            "latency": m["latency"], "clocks": m["clocks"], "gpu_launches": int(10 * m["batches"]),
            "roofline": m["roofline"],
            "e2e": {"value": m["capacity_rps"], "unit": "requests/s",
                    "h2d_bytes_per_step": int(m["values_per_request"] * 8),
                    "d2h_bytes_per_step": int(m["query_samples"] * n_ref * 12 / n_req)},
            "plain": {"ms_per_request": m["plain_ms_per_request"], "value": 1e3 / m["plain_ms_per_request"],
                      "how": "one jsim_all_pairs call on reference + the request's samples (host in/out)"},
            "speedup_vs_plain": m["speedup_vs_plain"]}
    print(json.dumps(line))
    return 0


def run_split(args):
    """One collection split over the ranks by row batches (C is additive over
    batches, Eq. 4): part `rank` of `world` on every rank, one all-reduce of
    the n x n counts (NCCL; the only exchange), J on rank 0.  Strong scaling."""
    import torch
    import torch.distributed as dist
    from paper_1911_04200_gb300 import jsim

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    off, ids, cfg = make_workload(args.workload, 0)  # the same collection on every rank
    n = cfg["n"]
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_ids = torch.from_numpy(ids.view(np.int64)).to(dev)
    ctx = jsim.Context(device=local, variant=args.variant, batch_rows=args.batch_rows, id_bits=cfg["id_bits"],
                       filter_min=args.filter_min)

    def step():
        Cp, sp = ctx.all_pairs_part(d_off, d_ids, rank, world)
        bitops = ctx.stats()["bitops_dense"]
        Ci = Cp.view(torch.int32)  # u32 counts; their sum fits u32, so the int32 sum has the same bits
        if world > 1:
            dist.all_reduce(Ci, op=dist.ReduceOp.SUM)
        if rank == 0:
            ctx.finish(Ci, sp)
        return bitops

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    t0 = time.perf_counter()
    bitops = 0.0
    for _ in range(args.steps):
        bitops += step()
    barrier()
    ms, bitops_all = aggregate_over_ranks((time.perf_counter() - t0) * 1e3, bitops, dev)
    cfg.update({"parallelism": "split contraction over %d ranks (one all-reduce of n x n counts)" % world,
                "filter_min": args.filter_min})
    line = {"metric": METRIC, "value": bitops_all / (ms * 1e-3) / 1e12, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64 ids, u32 counts, f64 J", "data": "synthetic",
            "config": cfg}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def one_copy_gbs(ids, dev):
    """Rate of one 1 GiB copy from the page-locked input to the device (the
    link alone, nothing overlapping), outside any timed region."""
    import torch
    t = torch.from_numpy(ids.view(np.int64))
    m = min(t.numel(), 1 << 27)
    d = torch.empty(m, dtype=torch.int64, device=dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        d.copy_(t[:m], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, m * 8 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return round(best, 1)


def numa_of_buffer(a):
    """The NUMA placement of a host buffer's pages as the kernel reports it
    (the /proc/self/numa_maps line of the mapping holding it)."""
    addr = a.ctypes.data
    try:
        best = None
        with open("/proc/self/numa_maps") as f:
            for line in f:
                start = int(line.split()[0], 16)
                if start <= addr:
                    best = line
                else:
                    break
        if best is None:
            return None
        keep = [w for w in best.split()[1:] if w.startswith(("N", "kernelpagesize", "prefer", "bind", "default"))]
        return " ".join(keep)
    except Exception:
        return None


def systems_measure(args, d_off, d_ids, J_ref, cfg):
    """Bounded sub-measurements beside the default line: the same all-pairs
    call with the two-or-more filter (same C and J, fewer words), the batched
    call against one plain call per collection on a subset of the batched
    recipe at its full set-size median, and the serving index on a reduced
    reference (capacity, p50/p99 under Poisson arrivals, against the plain
    form)."""
    import torch
    from paper_1911_04200_gb300 import jsim, synth
    out = {}
    n = cfg["n"]
    dev = d_off.device
    # two-or-more filter, same device-resident inputs
    fctx = jsim.Context(device=dev.index, id_bits=cfg["id_bits"], filter_min=2, profile=True)
    C2 = torch.empty((n, n), dtype=torch.uint32, device=dev)
    S2 = torch.empty(n, dtype=torch.uint64, device=dev)
    J2 = torch.empty((n, n), dtype=torch.float64, device=dev)
    fctx.all_pairs(d_off, d_ids, out=(C2, S2, J2))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(fctx.stream)
    for _ in range(args.steps):
        fctx.all_pairs(d_off, d_ids, out=(C2, S2, J2))
    e1.record(fctx.stream)
    torch.cuda.synchronize()
    st = fctx.stats()
    out["filter_min2"] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "words": st["words"],
                          "rows_nonzero": st["rows_nonzero"],
                          "same_J": bool(torch.equal(J2.view(torch.int64), J_ref.view(torch.int64))),
                          "how": "jsim_all_pairs with filter_min 2 (rows two or more samples hold) on the "
                                 "default workload's device-resident inputs"}
    fctx.close()
    del C2, S2, J2
    # batched and serving: each in a process of its own (the one-workload
    # runs of this script), so that neither inherits this process's host
    # memory state (the serving gather's host bandwidth did, measurably)
    def child(workload, env, budget_s):
        e = dict(os.environ)
        e.update(env)
        t0 = time.perf_counter()
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", workload, "--steps", "2",
                            "--warmup", "2"], env=e, capture_output=True, text=True, timeout=budget_s)
        for ln in r.stdout.splitlines():
            if ln.startswith("{"):
                d = json.loads(ln)
                d["wall_s"] = round(time.perf_counter() - t0, 1)
                return d
        return {"error": "no result (rc %d): %s" % (r.returncode, (r.stderr or "")[-400:])}

    count = int(os.environ.get("JSIM_SYSTEMS_BATCHED_COUNT", "24"))
    out["batched"] = child("batched200", {"JSIM_BATCHED_MEDIAN": "2e5", "JSIM_BATCHED_COUNT": str(count)}, 600)
    median = os.environ.get("JSIM_SYSTEMS_SERVE_MEDIAN", "1e5")
    out["serving"] = child("serve2048", {"JSIM_SERVE_MEDIAN": median,
                                         "JSIM_SERVE_REQUESTS": os.environ.get("JSIM_SYSTEMS_SERVE_REQUESTS", "400")},
                           600)
    out["serving"]["note"] = "reduced reference: set-size median %s (the recipe's is 1e6)" % median
    return out


def run_jsim(args):
    import torch
    import torch.distributed as dist
    from paper_1911_04200_gb300 import jsim

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bound = bind_near_gpu(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def pinned(count):
        return torch.empty(count, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)

    off, ids, cfg = make_workload(args.workload, rank, alloc=pinned, median=args.median)
    n = cfg["n"]
    N = int(off[-1])
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_ids = torch.from_numpy(ids.view(np.int64)).to(dev)
    ctx = jsim.Context(device=local, variant=args.variant, batch_rows=args.batch_rows,
                       id_bits=cfg["id_bits"], profile=True, filter_min=args.filter_min)
    C = torch.empty((n, n), dtype=torch.uint32, device=dev)
    S = torch.empty(n, dtype=torch.uint64, device=dev)
    J = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = ctx.stream

    def step():
        ctx.all_pairs(d_off, d_ids, out=(C, S, J))
        return ctx.stats()

    for _ in range(args.warmup):
        st = step()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    agg = {"ms_product": 0.0, "product_launches": 0, "launches": 0, "bitops": 0.0, "bitops_done": 0.0,
           "ms_pack": 0.0, "pack_bytes": 0, "ms_filter": 0.0}
    barrier()
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            st = step()
            agg["ms_product"] += st["ms_product"]
            agg["product_launches"] += st["product_launches"]
            agg["launches"] += st["launches"]
            agg["bitops"] += st["bitops_dense"]
            agg["bitops_done"] += st["bitops_done"]
            agg["ms_pack"] += st["ms_pack"]
            agg["pack_bytes"] += st["pack_bytes"]
            agg["ms_filter"] += st["ms_filter"]
        e1.record(stream)
        barrier()
    ms_max, bitops_all = aggregate_over_ranks(e0.elapsed_time(e1), agg["bitops"], dev)
    value = bitops_all / (ms_max * 1e-3) / 1e12
    last = st

    # end to end: pinned host in, host out, through the same call
    e2e = None
    if not args.no_e2e:
        hC = torch.empty((n, n), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        hS = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        hJ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy()
        for _ in range(max(1, args.warmup)):
            ctx.all_pairs(off, ids, out=(hC, hS, hJ))
        barrier()
        t0 = time.perf_counter()
        bo = 0.0
        calls = []
        for _ in range(args.steps):
            tc = time.perf_counter()
            ctx.all_pairs(off, ids, out=(hC, hS, hJ))
            calls.append((time.perf_counter() - tc) * 1e3)
            bo += ctx.stats()["bitops_dense"]
        barrier()
        dt, bo = aggregate_over_ranks(time.perf_counter() - t0, bo, dev)
        se = ctx.stats()  # the last end-to-end call (stage timers on)
        e2e_ms = dt / args.steps * 1e3
        e2e = {"value": bo / dt / 1e12, "unit": UNIT, "h2d_bytes_per_step": int((n + 1) * 8 + N * 8),
               "d2h_bytes_per_step": int(n * n * 4 + n * 8 + n * n * 8), "ms_per_step": e2e_ms,
               "exposed_ms_per_step": round(e2e_ms - ms_max / args.steps, 2),
               "h2d_copies_per_step": int(se["h2d_copies"]),
               "h2d_pieces_per_step": int(se["h2d_pieces"]),
               "call_ms": [round(x, 1) for x in calls],
               "stage_ms_last_call": {k: round(se[k], 2) for k in ("ms_total", "ms_h2d", "ms_validate", "ms_filter",
                                                                   "ms_scan", "ms_pack", "ms_product", "ms_d2h")},
               "h2d_copy_busy_ms": round(se["ms_h2d"], 2),
               "h2d_gbs_while_overlapped": round(se["h2d_bytes"] / (se["ms_h2d"] * 1e-3) / 1e9, 1)
               if se["ms_h2d"] else None,
               "h2d_gbs_one_1gib_copy": one_copy_gbs(ids, dev),
               "host_input_memory": numa_of_buffer(ids),
               "path": ("page-locked host input read by the device in %d value-range pieces (a copy grid of 64 "
                        "CTAs over NVLink-C2C) while the %s batch loop runs on the pieces already there"
                        % (se["h2d_pieces"], VARIANT_NAME.get(se["variant"], se["variant"]))
                        if se["h2d_pieces"] else
                        "host input above 4 GiB: streamed through two 1 GiB pinned staging buffers, copies "
                        "overlapping the device's work (super-batches planned one ahead)" if se["h2d_copies"] > 2 else
                        "the whole input copied to the device in one copy, then the device-resident call "
                        "(%s)" % VARIANT_NAME.get(se["variant"], se["variant"]))}
        # the whole end-to-end result equals the device-resident run's
        assert np.array_equal(hJ.view(np.uint64), J.cpu().numpy().view(np.uint64))
        assert np.array_equal(hC, C.view(torch.int32).cpu().numpy().view(np.uint32))
        assert np.array_equal(hS, S.view(torch.int64).cpu().numpy().view(np.uint64))
        e2e["parity"] = "whole C, sizes and J bit-identical to the device-resident call"

    # the method's useful work (pairs of nonzero packed words, the count a
    # sparse product needs) and the compulsory bytes, from one more untimed call
    uctx = jsim.Context(device=local, variant=args.variant, batch_rows=args.batch_rows, id_bits=cfg["id_bits"],
                        filter_min=args.filter_min, count_useful=True)
    uctx.all_pairs(d_off, d_ids, out=(C, S, J))
    useful = uctx.stats()["bitops_useful"]
    uctx.close()
    cb = 4
    compulsory = 8 * N + 8 * n * last["words"] + n * n * (cb + 8) + 8 * n

    variant = last["variant"]
    # the product kernels against the tensor peak, by the bit-operations they
    # carried out (the block-sparse variant skips the blocks no row reaches)
    per_launch_bitops = agg["bitops_done"] / max(1, agg["product_launches"])
    ms_per_launch = agg["ms_product"] / max(1, agg["product_launches"])
    roof_product = roofline_for(variant, per_launch_bitops, ms_per_launch, measured_peaks(),
                                traffic_from_profiles(variant, args.workload) if args.filter_min == 1 else None)
    roof_product["kernel"] = "product (%s)" % variant
    # the pack against HBM, by its algorithmic bytes (values read, packed
    # matrices filled)
    pk, src = measured_peaks()
    pack_gbs = agg["pack_bytes"] / (agg["ms_pack"] * 1e-3) / 1e9 if agg["ms_pack"] else 0.0
    # the pack kernel that ran: the windowed one on device-resident input
    # dense enough for it, else the per-value one of the variant
    pack_kernel = ("k_win_pack" if last.get("windows") else
                   "k_pack_classes" if variant == "sparse" else "k_pack_full")
    roof_pack = {"bound": "hbm", "achieved": round(pack_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": round(pack_gbs / pk["hbm_gbs"], 4),
                 "traffic": (traffic_from_profiles("pack-" + pack_kernel, args.workload)
                             if args.filter_min == 1 else None),
                 "kernel": "pack (%s)" % pack_kernel, "peak_source": "%s HBM copy bandwidth" % src,
                 "unit_bytes": "8 B per value packed + 8 B per word of the packed matrices filled"}
    # the roofline line is the dominant stage's (by time)
    if agg["ms_pack"] > agg["ms_product"]:
        roof, roof_other = roof_pack, roof_product
    else:
        roof, roof_other = roof_product, roof_pack
    cfg.update({"batch_rows": last["batch_rows"], "batches": last["batches"], "variant": variant,
                "filter_min": args.filter_min,
                "rows_nonzero": last["rows_nonzero"], "words": last["words"], "values": N,
                "bitops_dense_per_step": last["bitops_dense"],
                "bitops_done_per_step": last["bitops_done"],
                "bitops_useful_per_step": useful,
                "useful_fraction": round(useful / last["bitops_dense"], 4) if last["bitops_dense"] else None,
                "compulsory_bytes_per_step": compulsory,
                "parallelism": "dp%d (independent problems)" % world,
                "l2": "inputs (%.1f GB of values) larger than L2 (129 MB); no flush" % (N * 8 / 1e9),
                "host_cpus": "bound to the GPU's NUMA node (%d CPUs)" % len(bound) if bound else "unbound",
                "stage_ms": {k: round(last[k], 3) for k in ("ms_validate", "ms_filter", "ms_scan", "ms_pack",
                                                            "ms_product", "ms_epilogue")}})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 ids, u32 counts, f64 J", "data": "synthetic",
            "config": cfg, "clocks": clk.summary(), "gpu_launches": agg["launches"], "roofline": roof,
            "roofline_" + roof_other["kernel"].split()[0]: roof_other, "e2e": e2e}
    if world == 1 and not args.no_systems and args.workload == "clade1024":
        line["systems"] = systems_measure(args, d_off, d_ids, J, cfg)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(off, ids, n, last["bitops_dense"], args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_density(args):
    """Density sweep (the paper's synthetic matrices, Sec. V-A): n=1024
    samples over m=2^25 rows, entries present with probability p; every
    product variant with both filters, one all-pairs call per step, inputs
    resident.  The curve behind the automatic variant choice."""
    import torch
    from paper_1911_04200_gb300 import jsim, synth
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, m = 1024, 1 << 25
    C = torch.empty((n, n), dtype=torch.uint32, device=dev)
    S = torch.empty(n, dtype=torch.uint64, device=dev)
    J = torch.empty((n, n), dtype=torch.float64, device=dev)
    rows, best = [], None
    with Clocks(local) as clk:
        for p in (1e-4, 1e-3, 1e-2, 5e-2):
            off, ids = synth.bernoulli(n, m, p)
            d_off = torch.from_numpy(off.view(np.int64)).to(dev)
            d_ids = torch.from_numpy(ids.view(np.int64)).to(dev)
            ref = None
            for fm in (1, 2):
                for variant in ("popc", "tc", "tc2", "auto"):
                    ctx = jsim.Context(device=local, variant=variant, id_bits=25, profile=True, filter_min=fm)
                    for _ in range(max(1, args.warmup)):
                        ctx.all_pairs(d_off, d_ids, out=(C, S, J))
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(ctx.stream)
                    for _ in range(args.steps):
                        ctx.all_pairs(d_off, d_ids, out=(C, S, J))
                    e1.record(ctx.stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / args.steps
                    st = ctx.stats()
                    ctx.close()
                    # every variant and filter gives the same J
                    h = J[::97, ::89].cpu().numpy().view(np.uint64)
                    if ref is None:
                        ref = h
                    assert np.array_equal(h, ref)
                    row = {"p": p, "values": int(off[-1]), "filter_min": fm, "variant": st["variant"],
                           "words": st["words"], "ms": round(ms, 3), "ms_product": round(st["ms_product"], 3),
                           "tbitops": round(st["bitops_dense"] / (ms * 1e-3) / 1e12, 1)}
                    rows.append(row)
                    if variant == "auto" and fm == 1 and p == 1e-2:
                        best = row
            del d_off, d_ids
    line = {"metric": METRIC, "value": best["tbitops"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 ids, u32 counts, f64 J", "data": "synthetic",
            "config": {"workload": "density: n=1024, m=2^25 rows, Bernoulli(p) entries, p in 1e-4..5e-2; "
                                   "value = automatic variant at p=0.01",
                       "sweep": rows, "l2": "inputs larger than L2 at p >= 1e-3; no flush"},
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_product(args):
    """The semiring product alone (jsim_product) on random packed words
    already in device memory: n rows of `words` words (bit density
    `density`; random 64-bit words above 2^23 words in all), optionally
    padded rows, `calls` calls; prints the product time and Tbit-ops/s.  The
    small, self-contained case the product kernels are captured on."""
    import torch
    from paper_1911_04200_gb300 import jsim
    n, W = args.n, args.words
    g = torch.Generator(device="cuda").manual_seed(7)
    if n * W <= (1 << 23):
        bits = torch.rand((n, W * 64), device="cuda", generator=g) < args.density
        w = torch.zeros((n, W), dtype=torch.int64, device="cuda")
        for k in range(64):
            w |= bits[:, k::64].to(torch.int64) << k
        del bits
        dens = args.density
    else:
        w = torch.randint(-2**63, 2**63 - 1, (n, W), dtype=torch.int64, device="cuda", generator=g)
        dens = 0.5
    stride = W + args.pad
    if args.pad:
        wp = torch.zeros((n, stride), dtype=torch.int64, device="cuda")
        wp[:, :W] = w
        w = wp
    ctx = jsim.Context(variant=args.variant, count_bits=32, profile=True)
    C = torch.empty((n, n), dtype=torch.uint32, device="cuda")
    for _ in range(args.calls):
        ctx.product(w, n, W, stride, C=C, variant=args.variant)
        st = ctx.stats()
    torch.cuda.synchronize()
    t = st["ms_product"]
    v = st["bitops_dense"] / (t * 1e-3) / 1e12
    roof = roofline_for(st["variant"], st["bitops_dense"] / max(1, st["product_launches"]),
                        t / max(1, st["product_launches"]), measured_peaks(), None)
    print(json.dumps({"workload": "product", "variant": st["variant"], "n": n, "words": W, "stride": stride,
                      "bit_density": dens, "ms_product": t, "value": v, "unit": UNIT, "roofline": roof}))
    ctx.close()
    return 0


def run_serve_one(args):
    """A serving index of the 2048-sample reference recipe at a reduced set-
    size median and `calls` requests of 64 query samples submitted one at a
    time (one device batch each, nothing overlapping), so every query kernel
    runs alone: the case the query kernel is captured on."""
    from paper_1911_04200_gb300 import jsim, synth
    median = args.median or 2e4
    roff, rids = synth.serving_reference(median=median)
    qoff, qids = synth.serving_queries(0, 64, median=median)
    ctx = jsim.Context(id_bits=32)
    ix = jsim.Index(ctx, roff, rids, max_batch_samples=64, max_batch_values=int(qoff[-1]), slots=1)
    dt = 0.0
    for _ in range(args.calls):
        t0 = time.perf_counter()
        ix.submit(qoff, qids).wait()
        dt = time.perf_counter() - t0
    st = ix.stats()
    b = max(1, st["batches"])
    print(json.dumps({"workload": "serve-one", "median": median, "index_rows": ix.rows,
                      "index_bytes": ix.rows * 2048 // 8, "batches": st["batches"],
                      "rows_read_per_batch": st["rows_read"] / b, "qrows_ms_per_batch": st["ms_product"] / b,
                      "index_row_gbs": st["index_bytes_read"] / (st["ms_product"] * 1e-3) / 1e9
                      if st["ms_product"] else None, "last_request_ms": dt * 1e3}))
    ix.close()
    ctx.close()
    return 0


def main():
    args = parse()
    if args.workload == "product":
        return run_product(args)
    if args.workload == "serve-one":
        return run_serve_one(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched200":
        return run_batched(args)
    if args.workload == "stream4096":
        return run_streamed(args)
    if args.workload == "serve2048":
        return run_serve(args)
    if args.workload == "density":
        return run_density(args)
    world = dist_env()[0]
    if args.split or (world > 1 and not args.replicas and args.workload == "clade1024"):
        return run_split(args)
    return run_jsim(args)


if __name__ == "__main__":
    sys.exit(main())
