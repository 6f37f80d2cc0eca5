#!/usr/bin/env python
"""Throughput of SDC-resilient block-wise SZ compression + decompression on GB300.

One step = compress one field and decompress it again (the whole hot path: range and input
checksums, prediction/quantization with the ABFT checks, Huffman code, encoding, decoding
with verification). Default workload: a 512^3 float32 field (8 sinusoids + noise + 1%
lognormal spikes, seeded), value-range relative bound 1e-3, 6^3 blocks, ABFT on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank runs an independent replica on its
own GPU (the blocks are independent; no collective on the data path) and the timing is the
maximum over ranks.
"""

from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s at rel eb 1e-3 (% HBM roofline), ABFT overhead %, p99 latency"
WORKLOADS = {
    "512cube": dict(shape=(512, 512, 512), block=6, spikes=0.01, seed=2010),
    "64cube": dict(shape=(64, 64, 64), block=6, spikes=0.0, seed=1),
    # profiling size for ncu captures: the same recipe, 226 MB (above L2), a few hundred MB held
    "384cube": dict(shape=(384, 384, 384), block=6, spikes=0.01, seed=2010),
    # the 2D single-field config: 1800 x 3600 float32 (Hurricane-sized slices), 12^2 blocks
    "1800x3600": dict(shape=(1800, 3600), block=12, spikes=0.01, seed=2010),
}
REL_EB = 1e-3

# DRAM traffic per launch from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum)
# of the full-block kernel of each stage, keyed by the hash of the stage's sources at capture
# time (a changed kernel reports null). The captures ran on the 384cube workload; the 512cube
# entries scale them by the point count (traffic grows in proportion to the blocks processed).
NCU_TRAFFIC = {
    ("512cube", "prep"): {"bytes": 553422999, "src": "9b0950b480de"},
    ("384cube", "prep"): {"bytes": 233475328, "src": "9b0950b480de"},
    ("512cube", "predict"): {"bytes": 966222734, "src": "377596b23cb1"},
    ("384cube", "predict"): {"bytes": 407625216, "src": "377596b23cb1"},
    ("512cube", "encode"): {"bytes": 465609007, "src": "1840fbc5c98b"},
    ("384cube", "encode"): {"bytes": 196428800, "src": "1840fbc5c98b"},
    ("512cube", "decode"): {"bytes": 448822689, "src": "244969bf7694"},
    ("384cube", "decode"): {"bytes": 189347072, "src": "244969bf7694"},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources that define each stage's kernels (the hash keys the stored ncu traffic)
KERNEL_SOURCES = {
    "prep": ("k_prep.cu", "sdcsz_internal.cuh"),
    "predict": ("predict.cuh", "predict_wave.cuh", "k_predict_f32.cu", "sdcsz_internal.cuh"),
    "codebook": ("k_codebook.cu", "sdcsz_internal.cuh"),
    "encode": ("k_encode.cu", "sdcsz_internal.cuh"),
    "decode": ("decode.cuh", "decode_wave.cuh", "k_decode_f32.cu", "k_decode_wave.cu", "sdcsz_internal.cuh"),
    "prep64": ("k_prep.cu", "sdcsz_internal.cuh"),
    "predict64": ("predict.cuh", "predict_wave.cuh", "k_predict_f64.cu", "sdcsz_internal.cuh"),
    "decode64": ("decode.cuh", "decode_wave.cuh", "k_decode_f64.cu", "k_decode_wave.cu", "sdcsz_internal.cuh"),
}


def _src_hash(stage):
    h = hashlib.sha1()
    try:
        for name in KERNEL_SOURCES[stage]:
            with open(os.path.join(ROOT, "paper_2010_03144_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[0]]
            rows = mine or rows
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[3 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce_max(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def weak_scaling_value(world: int, bytes_per_rank: float, steps: int, ms_max: float) -> float:
    """Whole-job GB/s: every rank processed `bytes_per_rank` per step; the slowest rank's time counts."""
    return world * bytes_per_rank * steps / (ms_max / 1e3) / 1e9


def algorithmic_bytes(N, s, nb, n_unpred, n_reg, stream_bytes, abft):
    """Bytes each kernel must move (inputs read once, outputs written once)."""
    meta_in = 16 + 16 + 8 + 1 if abft else 16 + 8 + 1
    return {
        "prep": N * s + nb * (meta_in),
        "predict": N * s + 2 * N + n_unpred * s + nb * (meta_in + (25 if abft else 1)) + n_reg * 4 * s,
        "codebook": 65536 * (8 + 4),
        "encode": 2 * N + n_unpred * s + nb * ((25 if abft else 1) + 1) + n_reg * 4 * s + stream_bytes,
        "decode": stream_bytes + N * s,
    }


def run_ours(args):
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    if rank == 0 or world > 1:
        libbuild.build()
    _barrier(world)
    sz.lib()

    wl = WORKLOADS[args.workload]
    shape, block = wl["shape"], wl["block"]
    x = synth.sinusoid_field(shape, wl["seed"] + rank, spikes=wl["spikes"])
    N, s_dt = x.size, 4
    d = torch.from_numpy(x).to(device)
    enc, ll = args.encoding, args.lossless
    p_on = sz.make_params(shape, np.float32, REL_EB, block=block, abft=True, encoding=enc, lossless=ll)
    p_off = sz.make_params(shape, np.float32, REL_EB, block=block, abft=False, encoding=enc, lossless=ll)
    ws_on = sz.Workspace(p_on, device)
    ws_off = sz.Workspace(p_off, device)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    dws = torch.empty(sz.decompress_workspace_size(), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)

    def step(ws, p):
        # the public API as a user calls it: compression without a host wait, then decompression
        # of the stream it wrote (the library reads the stream's header, a 128-byte host copy)
        s_full, _ = sz.compress(d, REL_EB, block=block, abft=bool(p.abft), workspace=ws, encoding=enc, lossless=ll,
                                sync=False)
        sz.decompress(s_full, out=out, status=st_dev, ws=dws, report=False)

    # reports of one run for counts and the compression ratio
    s_t, rep = sz.compress(d, REL_EB, block=block, workspace=ws_on, encoding=enc, lossless=ll)
    dws = torch.empty(sz.decompress_workspace_size(s_t), dtype=torch.uint8, device=device)
    stream_bytes = int(rep["compressed_bytes"])
    rc, y, st, rep_d = sz.decompress(s_t, out=out, ws=dws)
    assert rc == 0
    assert float((y - d).abs().max()) <= rep["eb_abs"]
    st_dev = torch.empty(max(int(rep["blocks"]), 1), dtype=torch.uint8, device=device)

    def timed(ws, p, steps, warmup, stage_acc=None):
        for _ in range(warmup):
            step(ws, p)
        torch.cuda.synchronize()
        _barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if stage_acc is not None:  # stage events inside the timed steps, read after them
            sz.trace_begin(2 * steps)
        n0 = sz.kernel_launches()
        e0.record(stream)
        for _ in range(steps):
            step(ws, p)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = sz.kernel_launches() - n0
        if stage_acc is not None:
            for kind, ms in sz.trace_end(2 * steps):
                if kind == "compress":
                    for k, v in zip(("reset", "prep", "predict", "codebook", "encode"), ms):
                        stage_acc[k] = stage_acc.get(k, 0.0) + v
                else:
                    stage_acc["decode"] = stage_acc.get("decode", 0.0) + ms[0]
        _barrier(world)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), launches

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        pass
    clk = ClockSampler(uuid)
    clk.start()
    stages = {}
    ms_on, launches = timed(ws_on, p_on, args.steps, args.warmup, stages)
    clocks = clk.stop()
    stages_off = {}
    ms_off, _ = timed(ws_off, p_off, args.steps, args.warmup, stages_off)
    ms_on_max = _reduce_max(ms_on, world, device)
    ms_off_max = _reduce_max(ms_off, world, device)
    per_step = ms_on_max / args.steps
    gb = N * s_dt / 1e9
    value = weak_scaling_value(world, N * s_dt, args.steps, ms_on_max)

    # per-kernel averages over the timed region, roofline of the dominant kernel
    avg = {k: v / args.steps for k, v in stages.items()}
    comp_ms = sum(avg[k] for k in ("reset", "prep", "predict", "codebook", "encode"))
    dec_ms = avg["decode"]
    alg = algorithmic_bytes(N, s_dt, rep["blocks"], rep["unpredictable_points"], rep["regression_blocks"],
                            stream_bytes, True)
    dom = max(("prep", "predict", "encode", "decode", "codebook"), key=lambda k: avg[k])
    peak, peak_kind = _peaks()
    achieved = alg[dom] / (avg[dom] / 1e3) / 1e9
    def traffic_of(stage):
        t = NCU_TRAFFIC.get((args.workload, stage))
        return t["bytes"] if t and t.get("src") == _src_hash(stage) else None

    kernels = {k: {"ms": round(avg[k], 4), "GB/s": round(alg[k] / (avg[k] / 1e3) / 1e9, 1) if avg[k] > 0 else None,
                   "frac": round(alg[k] / (avg[k] / 1e3) / 1e9 / peak, 3) if avg[k] > 0 else None,
                   "algorithmic_bytes": alg[k], "traffic": traffic_of(k)}
               for k in ("prep", "predict", "codebook", "encode", "decode")}

    # end to end through the public API with host buffers: H2D field, compress, D2H stream,
    # H2D stream, decompress, D2H field, every step. Steps rotate over three CUDA streams with
    # their own device buffers, and the host runs one step ahead: it enqueues step k+1's upload
    # and compression before it waits for step k's compression (to learn its stream size from
    # the header) and enqueues the rest of step k. So the upload of the next field overlaps the
    # previous steps' downloads (the host link carries both directions at once) and never waits
    # for the host.
    h_field = torch.from_numpy(x).pin_memory()
    n_slots = 3
    slots = []
    for q in range(n_slots):
        slots.append({
            "stream": torch.cuda.Stream(device),
            "ws": ws_on if q == 0 else sz.Workspace(p_on, device),
            "d_in": torch.empty_like(d),
            "d_s": torch.empty(ws_on.cap, dtype=torch.uint8, device=device),
            "out": out if q == 0 else torch.empty_like(out),
            "dws": dws if q == 0 else torch.empty_like(dws),
            "h_stream": torch.empty(ws_on.cap, dtype=torch.uint8).pin_memory(),
            "h_hdr": torch.empty(128, dtype=torch.uint8).pin_memory(),
            "h_out": torch.empty(shape, dtype=torch.float32).pin_memory(),
            "status": torch.empty(max(int(rep["blocks"]), 1), dtype=torch.uint8, device=device),
        })

    def e2e_front(k, ev0=None):
        sl = slots[k % n_slots]
        cs = sl["stream"]
        with torch.cuda.stream(cs):
            if ev0 is not None:
                ev0.record(cs)
            sl["d_in"].copy_(h_field, non_blocking=True)
            sz.compress(sl["d_in"], REL_EB, block=block, workspace=sl["ws"], encoding=enc, lossless=ll, stream=cs,
                        sync=False)
            sl["h_hdr"].copy_(sl["ws"].out[:128], non_blocking=True)

    def e2e_back(k, ev1=None):
        sl = slots[k % n_slots]
        cs = sl["stream"]
        with torch.cuda.stream(cs):
            cs.synchronize()  # the compression and its header copy
            n = sz.read_header_partial(sl["h_hdr"].numpy(), sl["ws"].cap)["total"]
            sl["h_stream"][:n].copy_(sl["ws"].out[:n], non_blocking=True)
            sl["d_s"][:n].copy_(sl["h_stream"][:n], non_blocking=True)
            sz.decompress(sl["d_s"][:n], out=sl["out"], status=sl["status"], ws=sl["dws"], report=False, cuda_stream=cs)
            sl["h_out"].copy_(sl["out"], non_blocking=True)
            if ev1 is not None:
                ev1.record(cs)
        return n

    def e2e_run(nsteps, ev_a=None, ev_b=None):
        e2e_front(0, ev_a[0] if ev_a else None)
        n = 0
        for q in range(nsteps):
            if q + 1 < nsteps:
                e2e_front(q + 1, ev_a[q + 1] if ev_a else None)
            n = e2e_back(q, ev_b[q] if ev_b else None)
        return n

    e2e_run(max(3, args.warmup))
    torch.cuda.synchronize()
    _barrier(world)
    # no collector pause between the enqueues of a step (it would show as a slow step)
    gc.collect()
    gc.disable()
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    first = torch.cuda.Event(enable_timing=True)
    last = torch.cuda.Event(enable_timing=True)
    first.record(slots[0]["stream"])
    for sl in slots[1:]:
        sl["stream"].wait_event(first)
    n_s = e2e_run(args.steps, ev_a, ev_b)
    for sl in slots[1:]:
        done = torch.cuda.Event()
        done.record(sl["stream"])
        slots[0]["stream"].wait_event(done)
    last.record(slots[0]["stream"])
    torch.cuda.synchronize()
    gc.enable()
    step_ms = [ev_a[q].elapsed_time(ev_b[q]) for q in range(args.steps)]
    e2e_ms = _reduce_max(first.elapsed_time(last), world, device)
    e2e_value = world * gb * args.steps / (e2e_ms / 1e3)

    result = None
    if rank == 0:
        cpu = cpu_baseline(args) if world == 1 and not args.no_cpu else None
        result = {
            "metric": METRIC,
            "value": round(value, 2),
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(per_step, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload} float32 {shape} sinusoids+noise+{wl['spikes']:.0%} spikes, "
                                   f"rel eb {REL_EB}, block {block}^{len(shape)}, ABFT on, {enc} encoding"
                                   f"{' + lossless stage' if ll else ''}; "
                                   "one step = compress + decompress",
                       "field_bytes": N * s_dt, "compressed_bytes": stream_bytes,
                       "compression_ratio": round(N * s_dt / stream_bytes, 3),
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"{world} independent replicas"},
            "compress_gbs": round(gb / (comp_ms / 1e3), 2),
            "decompress_gbs": round(gb / (dec_ms / 1e3), 2),
            "abft_overhead_pct": round(100.0 * (ms_on_max - ms_off_max) / ms_off_max, 2),
            "abft_off_value": round(world * gb * args.steps / (ms_off_max / 1e3), 2),
            "p99_latency_ms": round(float(np.percentile(step_ms, 99)), 4),
            "latency": {"p50_ms": round(float(np.percentile(step_ms, 50)), 4),
                        "p99_ms": round(float(np.percentile(step_ms, 99)), 4),
                        "what": "one end-to-end step through the public API (host field in, host field out), "
                                "from its upload to the end of its download; consecutive steps overlap on three "
                                "streams, the host enqueueing one step ahead"},
            "kernels": kernels,
            "kernels_abft_off_ms": {k: round(v / args.steps, 4) for k, v in stages_off.items()},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic_of(dom), "algorithmic_bytes": alg[dom]},
            "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": N * s_dt + n_s,
                    "d2h_bytes_per_step": 128 + n_s + N * s_dt},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def _oracle_sample(args):
    import synth
    wl = WORKLOADS[args.workload]
    shape = wl["shape"]
    # a slab of the same field recipe: the first quarter along the slowest axis
    slab = (max(1, shape[0] // 4),) + tuple(shape[1:])
    x = synth.sinusoid_field(slab, wl["seed"], spikes=wl["spikes"])
    return x, slab


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(conn, shape, seed, spikes, block, enc, ll, rel):
    """One host core's share of the all-cores oracle baseline: its own slab of the recipe,
    compressed and decompressed by the (single-threaded) oracle each time the parent says go."""
    import oracle
    import synth
    x = synth.sinusoid_field(shape, seed, spikes=spikes)
    oracle.lib()
    conn.send(x.nbytes)
    while True:
        abft = conn.recv()
        if abft is None:
            break
        t0 = time.perf_counter()
        s, _ = oracle.compress(x, rel, block=block, abft=abft, encoding=enc, lossless=ll)
        oracle.decompress(s)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OraclePool:
    """The oracle on every host core at once: one spawned process per core, each with its own
    block-aligned slab of the workload's recipe (independent blocks, so the slabs are
    independent problems). Spawned, not forked, so no CUDA state is inherited."""

    def __init__(self, args, cores=None, planes=96):
        import multiprocessing as mp
        wl = WORKLOADS[args.workload]
        self.cores = cores or os.cpu_count() or 1
        shape = (planes,) + tuple(wl["shape"][1:])
        self.slab = shape
        ctx = mp.get_context("spawn")
        self.procs, self.conns = [], []
        for r in range(self.cores):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, shape, wl["seed"] + 17 * r, wl["spikes"], wl["block"],
                                                         args.encoding, args.lossless, REL_EB), daemon=True)
            p.start()
            self.procs.append(p)
            self.conns.append(a)
        self.bytes = sum(c.recv() for c in self.conns)

    def round(self, abft=True):
        """Wall seconds for every core to compress + decompress its slab once."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(abft)
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(None)
        for p in self.procs:
            p.join(timeout=30)


def cpu_baseline(args):
    """The oracle as it stands (single-threaded C++): one core on a slab, and every host core at
    once on a slab each, ABFT on and off."""
    import oracle
    x, slab = _oracle_sample(args)
    oracle.lib()
    block = WORKLOADS[args.workload]["block"]

    def one(abft):
        t0 = time.perf_counter()
        s, rep = oracle.compress(x, REL_EB, block=block, abft=abft, encoding=args.encoding, lossless=args.lossless)
        oracle.decompress(s)
        return x.nbytes / 1e9 / (time.perf_counter() - t0)

    single_on, single_off = one(True), one(False)
    pool = OraclePool(args)
    try:
        pool.round(True)  # warm-up
        all_on = pool.bytes / 1e9 / pool.round(True)
        all_off = pool.bytes / 1e9 / pool.round(False)
    finally:
        pool.close()
    return {"value": round(all_on, 4), "unit": "GB/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"every host core compresses + decompresses its own {pool.slab} slab of the recipe "
                      f"({pool.bytes / pool.cores / 1e6:.0f} MB each) once; single core: one {slab} slab",
            "cpu_model": _cpu_model(),
            "single": {"value": round(single_on, 4), "cores": 1},
            "all_cores": {"value": round(all_on, 4), "cores": pool.cores},
            "abft_off": {"single": round(single_off, 4), "all_cores": round(all_off, 4)},
            "abft_overhead_pct": {"single": round(100.0 * (single_off / single_on - 1.0), 2),
                                  "all_cores": round(100.0 * (all_off / all_on - 1.0), 2)}}


def run_reference(args):
    """The reference arm: the CPU oracle on every host core, a slab per core per step, on rank 0."""
    world, rank, local = _dist()
    if rank != 0:
        return None
    pool = OraclePool(args)
    try:
        for _ in range(args.warmup):
            pool.round(True)
        dt = sum(pool.round(True) for _ in range(args.steps))
    finally:
        pool.close()
    block = WORKLOADS[args.workload]["block"]
    value = pool.bytes * args.steps / 1e9 / dt
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{args.workload} recipe, one {pool.slab} slab per host core per step, "
                                  f"rel eb {REL_EB}, block {block}^{len(pool.slab)}, ABFT on, {args.encoding} encoding; "
                                  "one step = compress + decompress"},
           "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": pool.cores, "kind": "oracle",
                            "sample": f"{pool.slab} slab per core per step", "cpu_model": _cpu_model()},
           "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)
    return res


# Batched workload: 13 float32 fields of uneven shapes, per-field value-range bound drawn from
# {1e-2, 1e-3, 1e-4} with a fixed seed, block edge per field class chosen by the autotuner.
BATCH13 = [((100, 500, 500), 6), ((512, 512, 512), 2), ((1800, 3600), 4), ((26, 1800, 3600), 1)]


def run_batch13(args):
    """Batched compression of the 13-field mix against per-field plain calls on the same GPU."""
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import autotune
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    libbuild.build()
    sz.lib()
    device = torch.device("cuda", 0)
    shapes = [shp for shp, k in BATCH13 for _ in range(k)]
    rng = np.random.default_rng(3)
    ebs = [float(rng.choice([1e-2, 1e-3, 1e-4])) for _ in shapes]
    t0 = time.perf_counter()
    fields = [torch.from_numpy(synth.sinusoid_field(shp, 3000 + i)).to(device) for i, shp in enumerate(shapes)]
    gen_s = time.perf_counter() - t0
    tuner = autotune.Tuner(None)
    t0 = time.perf_counter()
    blocks = [tuner.block_for(f, eb) for f, eb in zip(fields, ebs)]
    tune_s = time.perf_counter() - t0
    total_bytes = sum(f.numel() * 4 for f in fields)
    stream = torch.cuda.Stream(device)

    # per-field plain calls (asynchronous, one stream)
    wss = [sz.Workspace(sz.make_params(tuple(f.shape), np.float32, eb, block=bk), device)
           for f, eb, bk in zip(fields, ebs, blocks)]

    def plain_step():
        for f, eb, bk, w in zip(fields, ebs, blocks, wss):
            sz.compress(f, eb, block=bk, workspace=w, stream=stream, sync=False)

    batch = sz.Batch(fields, ebs, block=blocks, stream=stream)
    n0 = sz.kernel_launches()
    batch.capture(stream)
    graph_kernels = sz.kernel_launches() - n0  # kernels captured into the graph (one replay per step)

    def batch_step():
        batch.launch(stream)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n0 = sz.kernel_launches()
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1) / args.steps, (sz.kernel_launches() - n0) // args.steps

    clk = ClockSampler()
    clk.start()
    ms_batch, _ = timed(batch_step)
    clocks = clk.stop()
    ms_plain, launches_plain = timed(plain_step)
    # the batch's streams equal the per-field ones
    res = batch.results(stream)
    same = 0
    for (s_b, _), f, eb, bk in zip(res, fields, ebs, blocks):
        s_1, _ = sz.compress(f, eb, block=bk)
        same += int(s_b.numel() == s_1.numel() and bool(torch.equal(s_b, s_1)))
    comp = sum(int(r[1]["compressed_bytes"]) for r in res)
    value = total_bytes / (ms_batch * 1e-3) / 1e9
    print(json.dumps({
        "metric": "batched compression GB/s, 13 uneven float32 fields, one persistent launch per stage and shape",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_batch, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch13: 6x(100,500,500) 2x512^3 4x(1800,3600) 1x(26,1800,3600), rel eb per "
                               "field from {1e-2,1e-3,1e-4} (seed 3), ABFT on, blocks autotuned per field class",
                   "field_bytes": total_bytes, "compressed_bytes": comp, "blocks": blocks, "ebs": ebs,
                   "l2": "inputs larger than L2 (no flush)", "graph": "captured CUDA graph replayed per step"},
        "plain_per_field_gbs": round(total_bytes / (ms_plain * 1e-3) / 1e9, 2),
        "plain_ms_per_step": round(ms_plain, 4),
        "batch_over_plain": round(ms_plain / ms_batch, 3),
        "identical_streams": f"{same}/{len(fields)}",
        "gpu_launches": {"batch": graph_kernels, "plain": launches_plain},
        "tuning_s": round(tune_s, 2), "generation_s": round(gen_s, 1),
        "tuner": tuner.cache,
        "clocks": clocks,
    }), flush=True)
    batch.close()


def run_serve(args):
    """Serving: a Poisson stream of compress / decompress / verify requests through the server."""
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    libbuild.build()
    sz.lib()
    device = torch.device("cuda", 0)
    rng = np.random.default_rng(4)
    # input pool resident in HBM: float32 3D, edges uniform in 32..512; float64 2D, 256..4096
    pool = []
    for i in range(12):
        shp = tuple(int(v) for v in rng.integers(32, 513, size=3))
        pool.append(synth.device_field(shp, 400 + i, torch.float32, device))
    for i in range(6):
        shp = tuple(int(v) for v in rng.integers(256, 4097, size=2))
        pool.append(synth.device_field(shp, 500 + i, torch.float64, device))
    streams = [sz.compress(f, 1e-3)[0].clone() for f in pool]
    torch.cuda.synchronize()
    rate, seconds, warm_s = 2000.0, max(1.0, args.steps / 10.0), 0.5
    n_req = int(rng.poisson(rate * (seconds + warm_s)))
    gaps = rng.exponential(1.0 / rate, size=n_req)
    arrivals = np.cumsum(gaps)
    ops = rng.integers(0, 3, size=n_req)
    which = rng.integers(0, len(pool), size=n_req)
    ebs = 10.0 ** rng.uniform(-5, -2, size=n_req)
    flipped = rng.random(n_req) < 0.001
    srv = sz.Server(hbm_budget=60 << 30, slots=args.slots)
    done, lat, nbytes_done, peak_inflight = {}, [], 0, 0
    t0 = time.perf_counter()
    nxt = 0
    while len(done) < n_req:
        now = time.perf_counter() - t0
        while nxt < n_req and arrivals[nxt] <= now:
            k, op = int(which[nxt]), int(ops[nxt])
            fl = None
            if flipped[nxt]:
                fl = [("code", 1, 3, 2)] if op == 0 else ([("decomp", 1, 0, 0)] if op == 1 else None)
            if op == 0:
                srv.submit_compress(nxt, pool[k], float(ebs[nxt]), flips=fl)
            elif op == 1:
                srv.submit_decompress(nxt, streams[k], flips=fl)
            else:
                srv.submit_verify(nxt, streams[k])
            nxt += 1
        for c in srv.poll(256, wait_us=0 if nxt < n_req else 2000):
            rid = c["id"]
            done[rid] = c
            if c["status"] not in (0, sz.ESDC):
                raise RuntimeError(f"request {rid} failed: {c['status']}")
            if c["op"] in (sz.OP_COMPRESS, sz.OP_DECOMPRESS):
                srv.release(rid)
            if arrivals[rid] >= warm_s:
                lat.append(c["t_done"] - c["t_submit"])
                nbytes_done += pool[int(which[rid])].numel() * pool[int(which[rid])].element_size()
        st = srv.stats()
        peak_inflight = max(peak_inflight, st["in_flight"])
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat_ms = np.array(lat) * 1e3
    measured = [c for rid, c in done.items() if arrivals[rid] >= warm_s]
    span = max(c["t_done"] for c in measured) - min(c["t_submit"] for c in measured)
    print(json.dumps({
        "metric": "serving p50/p99 latency and GB/s, Poisson compress/decompress/verify requests",
        "value": round(nbytes_done / span / 1e9, 2), "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": "serve: Poisson 2000 req/s, thirds compress/decompress/verify, pool of 12 float32 3D "
                               "(edges U{32..512}) and 6 float64 2D (edges U{256..4096}) fields resident in HBM, "
                               "compress rel eb log-uniform 1e-5..1e-2, 0.1% of requests with one bit flip, "
                               f"60 GB admission budget, {args.slots} slots",
                   "requests": n_req, "measured_requests": len(lat), "warmup_s": warm_s, "seconds": seconds},
        "p50_latency_ms": round(float(np.percentile(lat_ms, 50)), 3),
        "p99_latency_ms": round(float(np.percentile(lat_ms, 99)), 3),
        "mean_latency_ms": round(float(lat_ms.mean()), 3),
        "achieved_req_per_s": round(len(lat) / span, 1),
        "wall_s": round(wall, 2), "peak_in_flight": peak_inflight, "peak_bytes": st["peak_bytes"],
        "flipped_requests": int(flipped.sum()),
    }), flush=True)


def run_faults(args):
    """Bit-flip rate sweep: soft errors in the input, the bin array and the regression
    coefficients during compression, and persistent corruption of the compressed stream;
    detection / correction counts, compression-ratio change and GB/s against the fault-free run."""
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    libbuild.build()
    sz.lib()
    dev = torch.device("cuda", 0)
    rel, rates = 1e-4, (1e-9, 1e-8, 1e-7, 1e-6, 1e-5)
    results = []
    for shape, tdt, B in (((1024, 1024, 1024), torch.float32, 8), ((512, 512, 512), torch.float64, 8)):
        W = 1 if tdt == torch.float32 else 2
        x0 = synth.device_field(shape, 21, tdt, dev, spikes=0.01)
        N = x0.numel()
        nbd = [n // B for n in shape]
        nb, P = nbd[0] * nbd[1] * nbd[2], B ** 3

        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                out = fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps, out

        def clean():
            s, rep = sz.compress(x0, rel, block=B)
            rc, y, st, rd = sz.decompress(s)
            return s, rep, y
        base_ms, (s0, rep0, _) = timed(clean)
        row = {"field": f"{tuple(shape)} {'f32' if W == 1 else 'f64'} block {B}^3 rel {rel}",
               "fault_free": {"ratio": round(N * 4 * W / s0.numel(), 3),
                              "gbs": round(N * 4 * W / (base_ms * 1e-3) / 1e9, 1)}, "rates": []}
        for rate in rates:
            rng = np.random.default_rng(int(round(-np.log10(rate))))
            n_in = int(rng.binomial(N * W, rate))
            words = np.unique(rng.integers(0, N * W, size=n_in))
            pts = words // W
            i, j, l = np.unravel_index(pts, shape)
            blk = ((i // B) * nbd[1] + j // B) * nbd[2] + l // B
            flips = [("input", int(bk), int(wd), int(bt)) for bk, wd, bt in
                     zip(blk, words, rng.integers(0, 32, size=words.size))]
            n_code = int(rng.binomial(N, rate))
            flips += [("code", int(bk), int(k), int(bt)) for bk, k, bt in
                      zip(rng.integers(0, nb, n_code), rng.integers(0, P, n_code), rng.integers(0, 16, n_code))]
            n_coef = int(rng.binomial(nb * 4, rate))
            flips += [("coef", int(bk), int(k), int(bt)) for bk, k, bt in
                      zip(rng.integers(0, nb, n_coef), rng.integers(0, 4, n_coef), rng.integers(0, 32 * W, n_coef))]
            x = x0.clone()

            def faulty():
                x.copy_(x0)
                s, rep = sz.compress(x, rel, block=B, flips=flips)
                rc, y, st, rd = sz.decompress(s)
                return s, rep, y
            ms, (s, rep, y) = timed(faulty)
            viol = int(((x0.double() - y.double()).abs() > rep["eb_abs"]).sum()) if W == 1 else \
                sum(int(((x0[q:q + 64].double() - y[q:q + 64].double()).abs() > rep["eb_abs"]).sum())
                    for q in range(0, shape[0], 64))
            # persistent corruption of the compressed stream (payload bits)
            hb = s[:128].cpu().numpy()
            pay_bytes = int(np.frombuffer(hb[96:104].tobytes(), "<u8")[0])
            pay0 = int(s.numel()) - pay_bytes  # the payload is the stream's last section
            npay = pay_bytes
            n_st = int(rng.binomial(npay // 4, rate))
            sc = s.clone()
            if n_st:
                pos = torch.from_numpy(rng.integers(pay0, s.numel(), size=n_st)).to(dev)
                sc[pos] ^= torch.from_numpy((1 << rng.integers(0, 8, size=n_st)).astype(np.uint8)).to(dev)
            rc2, y2, st2, rd2 = sz.decompress(sc)
            detected = int((st2 != 0).sum())
            ok_mask = (st2 == 0)
            row["rates"].append({
                "rate_per_word": rate, "input_flips": int(words.size), "code_flips": n_code, "coef_flips": n_coef,
                "input_corrected": rep["input_corrected"], "codes_corrected": rep["codes_corrected"],
                "uncorrectable_blocks": rep["uncorrectable_blocks"], "bound_violations_after_decompress": viol,
                "ratio": round(N * 4 * W / s.numel(), 3),
                "ratio_change_pct": round(100.0 * (s0.numel() - s.numel()) / s.numel(), 4),
                "gbs": round(N * 4 * W / (ms * 1e-3) / 1e9, 1),
                "stream_flips": n_st, "stream_blocks_flagged": detected, "stream_rc": rc2,
                "blocks_passing": int(ok_mask.sum())})
            del x, s, y, sc, y2
            torch.cuda.empty_cache()
        results.append(row)
        del x0
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "fault sweep: detection/correction, CR change and GB/s vs fault-free",
                      "unit": "GB/s", "data": "synthetic", "higher_is_better": True,
                      "config": {"workload": "faults: 1024^3 f32 and 512^3 f64, spikes 1%, rel 1e-4, 8^3 blocks; "
                                             "flips per word over input, bin array and coefficients at compression, "
                                             "and payload bits of the stream", "steps": "3 timed runs per rate"},
                      "sweep": results}), flush=True)


def run_region(args):
    """Random access: boxes of 32^3, 64^3 and 128^3 at random positions decoded out of the
    stream of a 1024^3 float32 field (6^3 blocks), each call timed end to end on the host
    (header read, decode, verification, report), against the full decompression."""
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    libbuild.build()
    sz.lib()
    dev = torch.device("cuda", 0)
    n = 1024
    f = synth.device_field((n, n, n), 11, torch.float32, dev, spikes=0.01)
    s, _ = sz.compress(f, 1e-4)
    s = s.clone()
    del f
    out_full = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    ws = torch.empty(sz.decompress_workspace_size(), dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(12)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return np.array(ts) * 1e3

    full_ms = timed(lambda: sz.decompress(s, out=out_full, ws=ws), max(3, args.steps // 4))
    rows = []
    for e in (32, 64, 128):
        out = torch.empty((e, e, e), dtype=torch.float32, device=dev)
        st = torch.empty(((e + 4) // 6 + 1) ** 3, dtype=torch.uint8, device=dev)
        boxes = [tuple(int(v) for v in rng.integers(0, n - e + 1, size=3)) for _ in range(args.steps)]
        it = iter(boxes * (1 + (args.warmup + args.steps) // len(boxes)))

        def one():
            lo = next(it)
            rc, _, _, _ = sz.decompress_region(s, lo, tuple(v + e for v in lo), out=out, status=st, ws=ws)
            assert rc == 0

        ms = timed(one, args.steps)
        rows.append({"box": f"{e}^3", "p50_ms": round(float(np.percentile(ms, 50)), 3),
                     "p99_ms": round(float(np.percentile(ms, 99)), 3),
                     "GB_per_s_of_box": round(e ** 3 * 4 / (np.median(ms) / 1e3) / 1e9, 2)})
    print(json.dumps({
        "metric": "random-access box decompression latency", "value": rows[1]["p50_ms"], "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "region: 1024^3 float32 (spikes 1%), rel 1e-4, 6^3 blocks; boxes at uniform random "
                               "positions, value = p50 of the 64^3 box, host-timed calls including the header read"},
        "boxes": rows, "full_decompress_p50_ms": round(float(np.percentile(full_ms, 50)), 3)}), flush=True)


# FP64 instructions (DADD + DMUL + DFMA, thread level) per point of each stage of the float64
# path, from an ncu capture (smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on.sum
# over every launch of the stage / points), keyed by the hash of the stage's sources.
NCU_FP64_PER_POINT = {
    "predict": {"per_point": 10.751, "src": "0d23c2e2396a"},
    "decode": {"per_point": 3.46, "src": "9a4285c83e39"},
}


def fp64_rate(device, reps=5):
    """Measured FP64 instruction rate of this GPU (separate DADD + DMUL, and DFMA), ops/s."""
    import ctypes

    import torch

    from paper_2010_03144_gb300 import build as libbuild
    L = ctypes.CDLL(libbuild.PEAK_LIB)
    L.sdcsz_peak_fp64.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_ulonglong)]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, iters = sms * 8, 4096
    out = torch.empty(blocks * 256, dtype=torch.float64, device=device)
    h = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    res = {}
    for fused in (0, 1):
        best = None
        for _ in range(reps):
            ms, n = ctypes.c_float(), ctypes.c_ulonglong()
            if L.sdcsz_peak_fp64(ctypes.c_void_p(out.data_ptr()), blocks, iters, fused, h, ctypes.byref(ms),
                                 ctypes.byref(n)):
                raise RuntimeError("FP64 rate kernel failed")
            r = n.value / (ms.value * 1e-3)
            best = r if best is None else max(best, r)
        res["fma" if fused else "add_mul"] = best
    return res


def run_fp64(args):
    """The float64 path against the FP64 instruction rate: 512^3 float64 (spikes; --fp64-size
    sets the edge), rel 1e-4, 8^3 blocks, ABFT on and off, with this GPU's measured DADD/DMUL rate beside it."""
    import torch

    import paper_2010_03144_gb300 as sz
    from paper_2010_03144_gb300 import build as libbuild
    import synth

    libbuild.build()
    sz.lib()
    dev = torch.device("cuda", 0)
    clk = ClockSampler()
    clk.start()
    rate = fp64_rate(dev)
    n = args.fp64_size
    shape, B, rel = (n, n, n), 8, 1e-4
    x = synth.device_field(shape, 21, torch.float64, dev, spikes=0.01)
    N = x.numel()
    rows = {}
    for abft in (True, False):
        p = sz.make_params(shape, torch.float64, rel, block=B, abft=abft)
        ws = sz.Workspace(p, dev)
        out = torch.empty_like(x)
        s_t, rep = sz.compress(x, rel, block=B, workspace=ws, abft=abft)
        dws = torch.empty(sz.decompress_workspace_size(s_t), dtype=torch.uint8, device=dev)
        st = torch.empty(max(int(rep["blocks"]), 1), dtype=torch.uint8, device=dev)

        def one():
            s_full, _ = sz.compress(x, rel, block=B, workspace=ws, abft=abft, sync=False)
            sz.decompress(s_full, out=out, status=st, ws=dws, report=False)

        for _ in range(args.warmup):
            one()
        torch.cuda.synchronize()
        acc = {}
        sz.trace_begin(2 * args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            one()
        e1.record()
        torch.cuda.synchronize()
        for kind, ms in sz.trace_end(2 * args.steps):
            if kind == "compress":
                for k, v in zip(("reset", "prep", "predict", "codebook", "encode"), ms):
                    acc[k] = acc.get(k, 0.0) + v / args.steps
            else:
                acc["decode"] = acc.get("decode", 0.0) + ms[0] / args.steps
        step = e0.elapsed_time(e1) / args.steps
        rows["abft_on" if abft else "abft_off"] = {
            "round_trip_gbs": round(N * 8 / (step * 1e-3) / 1e9, 1), "ms_per_step": round(step, 4),
            "stages_ms": {k: round(v, 4) for k, v in acc.items()},
            "compression_ratio": round(N * 8 / int(rep["compressed_bytes"]), 3)}
    clocks = clk.stop()
    fp = {}
    for stage in ("prep", "predict", "decode"):
        e = NCU_FP64_PER_POINT.get(stage)
        if e and e.get("src") == _src_hash(stage + "64"):
            t = rows["abft_on"]["stages_ms"][stage] * 1e-3
            ach = e["per_point"] * N / t
            fp[stage] = {"fp64_per_point": e["per_point"], "achieved_ops": round(ach / 1e9, 1),
                         "frac_of_add_mul_rate": round(ach / rate["add_mul"], 3)}
    print(json.dumps({
        "metric": "float64 round trip GB/s and FP64 instruction-rate fraction", "unit": "GB/s",
        "value": rows["abft_on"]["round_trip_gbs"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fp64: {n}^3 float64 sinusoids+noise+1% spikes, rel eb 1e-4, block 8^3; one step = "
                               "compress + decompress", "l2": "inputs larger than L2 (no flush)"},
        "fp64_rate_gops": {k: round(v / 1e9, 1) for k, v in rate.items()},
        "fp64_rate_what": "measured: independent DADD+DMUL chains (add_mul) and DFMA chains (fma), "
                          "thread-level instructions per second",
        "runs": rows, "fp64_roofline": fp or None, "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS) + ("batch13", "serve", "faults", "region", "fp64"),
                    default="512cube")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--fp64-size", type=int, default=512, help="float64 workload: edge of the cube")
    ap.add_argument("--block", type=int, default=0,
                    help="block edge for the single-field workloads (default: the workload's)")
    ap.add_argument("--rel", type=float, default=REL_EB,
                    help="value-range-relative error bound of the single-field workloads (default 1e-3)")
    ap.add_argument("--slots", type=int, default=16, help="serving: requests on the device at once")
    ap.add_argument("--encoding", choices=("raw", "compact"), default="raw",
                    help="stream encoding: raw coefficient/unpredictable sections, or compact (in the payload)")
    ap.add_argument("--lossless", action="store_true", help="add the lossless stage (rANS over the block data)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.block and args.workload in WORKLOADS and args.block != WORKLOADS[args.workload]["block"]:
        # another block edge is another workload (its own name, no stored ncu figures)
        name = f"{args.workload}_b{args.block}"
        WORKLOADS[name] = dict(WORKLOADS[args.workload], block=args.block)
        args.workload = name
    if args.rel != REL_EB and args.workload in WORKLOADS:  # likewise another bound
        globals()["REL_EB"] = args.rel
        name = f"{args.workload}_rel{args.rel:g}"
        WORKLOADS[name] = dict(WORKLOADS[args.workload])
        args.workload = name
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch13":
        run_batch13(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "faults":
        run_faults(args)
    elif args.workload == "region":
        run_region(args)
    elif args.workload == "fp64":
        run_fp64(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
