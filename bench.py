#!/usr/bin/env python
"""Benchmark of the B300 BOLT oblivious map: oblivious accesses/s and build
Mrec/s at N = 2^28 records of 32 B (8 B key + 24 B value).

One step = the whole hot path on one batch of synthetic input: the oblivious
build of the 2^28-record map (bolt_init), then 2^22 uniform accesses over its
keys (50% GET / 50% PUT, the paper's mix) in batches of 4096 (bolt_access).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bolt|reference]

value   accesses/s of the access phase, inputs resident in HBM, CUDA events on
        the launching stream; the build's Mrec/s is reported beside it;
e2e     the same through the host-pointer C-ABI calls (pinned host buffers,
        host<->device copies inside the timed region);
roofline  the bitonic global pass (the build's HBM-bound kernel), event-timed
        per launch inside the timed region, against the measured HBM copy peak;
cpu_baseline  the CPU oracle on a bounded sample of the same workload.
--impl reference times the CPU oracle itself (the only reference this method
has) on a bounded sample, on rank 0.
Multi-GPU (torchrun): independent replicas, one map per GPU ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_01742_b300 import workload as W  # noqa: E402

METRIC = "oblivious accesses/s and build Mrec/s at N=2^28; served p50/p99 latency"
LOG_N = 28
VAL_BYTES = 24
N_ACCESS = 1 << 22
BATCH = 4096
SEED_DATA = 0x5EED0003
SEED_OPS = 0x5EED0103
SEED_MAP = 0x5EED0203
def config_for(log_n: int, n_acc: int, lookahead: float = 0.0) -> dict:
    """The workload description of a headline-shaped run (N = 2^log_n)."""
    N = 1 << log_n
    tag_gib = 8 * N / 2**30
    return {
        "workload": f"N=2^{log_n} records x 32 B (8 B uint64 key + 24 B value), oblivious build, "
                    f"then {n_acc} uniform accesses to existing keys (50% GET / 50% PUT) in "
                    f"batches of {BATCH}",
        "records": N,
        "record_bytes": 8 + VAL_BYTES,
        "accesses_per_step": n_acc,
        "batch": BATCH,
        "c": 8,
        "alpha": 0.2,
        "l2": (f"inputs larger than L2 ({N * 32 / 2**30:.3g} GiB records, {tag_gib:.3g} GiB of "
               "sort tags, pages and position map larger still)"),
        "lookahead": lookahead,
    }


CONFIG = config_for(LOG_N, N_ACCESS)


def aggregate(local: dict, world: int, group=None) -> dict:
    """Whole-job figures over ranks: the slowest rank's times, the sum of the
    work.  With world == 1 the local figures are returned unchanged."""
    if world == 1:
        return dict(local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([local["build_s"], local["access_s"], local["step_s"]], dtype=torch.float64)
    w = torch.tensor([local["records"], local["accesses"]], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t, w = t.cuda(), w.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    t, w = t.cpu().tolist(), w.cpu().tolist()
    return {"build_s": t[0], "access_s": t[1], "step_s": t[2], "records": w[0],
            "accesses": w[1]}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def make_records(n: int, seed: int):
    keys = np.empty(n, dtype=np.uint64)
    step = 1 << 24
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        keys[lo:hi] = W.key_of(np.arange(lo, hi, dtype=np.uint64))
    rng = np.random.default_rng(seed)
    vals = np.frombuffer(rng.bytes(n * VAL_BYTES), dtype=np.uint8).reshape(n, VAL_BYTES)
    return keys, vals


def link_bandwidth(torch) -> dict:
    """Pinned host<->device copy bandwidth (1 GiB, best of 3), GB/s."""
    n = 1 << 30
    h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h", lambda: h.copy_(d, non_blocking=True))):
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            best = max(best, n / (a.elapsed_time(b) * 1e-3) / 1e9)
        out[name] = round(best, 1)
    del h, d
    return out


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_sample(seconds_hint: float = 15.0, multicore: bool = False) -> dict:
    """The oracle as it stands on a bounded sample of the workload: a
    2^21-record map of 32 B records, then accesses in batches of 4096 from
    the same op distribution.  Single-threaded (the oracle proper), or its
    OpenMP build on every host core (multicore: the same source, its
    independent loops -- PRF draws, per-round decisions, page decryption and
    encryption -- spread over the cores; byte-identical results)."""
    from oracle import oracle as O
    n_s = 1 << 21
    keys, vals = make_records(n_s, SEED_DATA)
    cores = 1
    if multicore:
        cores = O.threads(os.cpu_count() or 1)
    m = O.OracleMap(n_s, VAL_BYTES, trace=False, omp=multicore)
    t0 = time.perf_counter()
    rc = m.init(keys, vals, SEED_MAP)
    t_build = time.perf_counter() - t0
    assert rc == 0, rc
    done, t_acc, rep = 0, 0.0, 0
    while t_acc < seconds_hint and rep < 64:
        ops, k, vin = W.op_stream(n_s, BATCH, VAL_BYTES, SEED_OPS + rep, get_frac=0.5)
        t0 = time.perf_counter()
        rc, _, _ = m.access(ops, k, vin)
        t_acc += time.perf_counter() - t0
        assert rc == 0, rc
        done += BATCH
        rep += 1
    m.close()
    return {"value": round(done / t_acc, 1), "unit": "accesses/s", "cores": cores,
            "kind": "oracle (OpenMP build, all host cores)" if multicore else "oracle",
            "cpu": cpu_model(),
            "build_mrec_s": round(n_s / t_build / 1e6, 3),
            "sample": f"oracle map of 2^21 x 32 B records (build {t_build:.1f} s), then {done} "
                      f"uniform 50/50 GET/PUT accesses in batches of {BATCH} ({t_acc:.1f} s); "
                      + (f"{cores} host threads" if multicore else "single host thread")}


def one_op_calls(B, m, ops, keys, vin, count: int, warm: int = 100):
    """Wall time of `count` bolt_access calls of one operation each, through
    the C ABI on preallocated host arrays (the call's own cost: staging, the
    launch, the wait for its results), after `warm` untimed calls."""
    import ctypes
    vb = vin.shape[1]
    ops = np.ascontiguousarray(ops)
    keys = np.ascontiguousarray(keys)
    vin = np.ascontiguousarray(vin)
    out = np.zeros((len(ops), vb), dtype=np.uint8)
    st = np.zeros(len(ops), dtype=np.uint8)
    kb = keys.dtype.itemsize
    base = [a.ctypes.data for a in (ops, keys, vin, out, st)]
    lat = np.empty(count)
    for j in range(warm + count):
        i = j % len(ops)
        p = [ctypes.c_void_p(base[0] + i), ctypes.c_void_p(base[1] + kb * i),
             ctypes.c_void_p(base[2] + vb * i), ctypes.c_void_p(base[3] + vb * i),
             ctypes.c_void_p(base[4] + i)]
        t = time.perf_counter()
        rc = B.bolt_access(m.handle, *p, 1)
        dt = time.perf_counter() - t
        assert rc == 0, rc
        if j >= warm:
            lat[j - warm] = dt
    return lat


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    n_s = 1 << 21
    keys, vals = make_records(n_s, SEED_DATA)
    m = O.OracleMap(n_s, VAL_BYTES, trace=False)
    t0 = time.perf_counter()
    assert m.init(keys, vals, SEED_MAP) == 0
    t_build = time.perf_counter() - t0
    batches = [W.op_stream(n_s, BATCH, VAL_BYTES, SEED_OPS + i, get_frac=0.5)
               for i in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        assert m.access(*batches[i])[0] == 0
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        assert m.access(*batches[i])[0] == 0
    dt = time.perf_counter() - t0
    m.close()
    value = args.steps * BATCH / dt
    sample = (f"oracle (single thread) on a 2^21-record sample map of 32 B records (build "
              f"{t_build:.1f} s, untimed); each step = one batch of {BATCH} uniform 50/50 "
              "GET/PUT accesses")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "accesses/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/u64 (integer)",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": round(value, 1), "unit": "accesses/s", "cores": 1,
                             "kind": "oracle", "sample": sample,
                             "build_mrec_s": round(n_s / t_build / 1e6, 3)},
            "e2e": {"value": round(value, 1), "unit": "accesses/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_bolt(args) -> None:
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    group = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2509_01742_b300 import bolt as B

    N = 1 << args.log_n
    n_acc = args.accesses
    keys, vals = make_records(N, SEED_DATA + rank)
    ops, akeys, avin = W.op_stream(N, n_acc, VAL_BYTES, SEED_OPS + rank, get_frac=0.5)
    stream = torch.cuda.Stream()
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
    d_vals = torch.from_numpy(vals.copy()).cuda()
    d_ops = torch.from_numpy(ops).cuda()
    d_akeys = torch.from_numpy(akeys.view(np.int64)).cuda()
    d_avin = torch.from_numpy(avin).cuda()
    d_vout = torch.empty((n_acc, VAL_BYTES), dtype=torch.uint8, device="cuda")
    d_status = torch.empty(n_acc, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    m = B.BoltMap(N, VAL_BYTES)
    m.set_param(B.BOLT_PARAM_PROFILE, 1)
    m.set_param(B.BOLT_PARAM_LOOKAHEAD, args.lookahead)
    if args.defer is not None:
        m.set_param(B.BOLT_PARAM_DEFER_FLUSH, args.defer)
    info = m.info()
    nb = (n_acc + BATCH - 1) // BATCH

    def step(events=None):
        # event spans time the build's kernels (the roofline kernel among
        # them); the access batches run unprofiled, their kernel breakdown
        # comes from a separate pass after the timed region
        m.set_param(B.BOLT_PARAM_PROFILE, 1)
        if events:
            events[0].record(stream)
        rc = m.init_device(d_keys, d_vals, SEED_MAP, stream=stream)
        assert rc == 0, rc
        if events:
            events[1].record(stream)
        m.set_param(B.BOLT_PARAM_PROFILE, 0)
        rc = m.access_device_batches(d_ops, d_akeys, d_avin, d_vout, d_status, BATCH,
                                     stream=stream)
        assert rc == 0, rc
        if events:
            events[2].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    assert m.sync() == 0
    m.profile(reset=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            step(evs[k])
        barrier()
    assert m.sync() == 0
    prof = m.profile(reset=True)
    # correctness spot check of the last timed step's GETs against the inputs
    vout = d_vout.cpu().numpy()
    st = d_status.cpu().numpy()
    assert st.all(), "every accessed key exists"
    # untimed: the same access stream once more with kernel-class spans
    m.set_param(B.BOLT_PARAM_PROFILE, 1)
    assert m.access_device_batches(d_ops, d_akeys, d_avin, d_vout, d_status, BATCH,
                                   stream=stream) == 0
    assert m.sync() == 0
    aprof = m.profile(reset=True)
    m.set_param(B.BOLT_PARAM_PROFILE, 0)
    build_s = sum(e[0].elapsed_time(e[1]) for e in evs) * 1e-3
    access_s = sum(e[1].elapsed_time(e[2]) for e in evs) * 1e-3
    step_s = sum(e[0].elapsed_time(e[2]) for e in evs) * 1e-3
    agg = aggregate({"build_s": build_s, "access_s": access_s, "step_s": step_s,
                     "records": float(N * args.steps), "accesses": float(n_acc * args.steps)},
                    world, group)

    # secondary roofline: the build's grouping of host records by page (two
    # bucket passes), algorithmic bytes = a 4-byte destination read per
    # record, and per host-bin record its 8-byte tag written to its bucket,
    # read back and written to its page's run, against HBM.  The host-bin
    # record count comes from an untimed rebuild (same keys and seed: the same
    # placement), read from the bin loads before any access.
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    sg = prof["page_group"]
    m.set_param(B.BOLT_PARAM_PROFILE, 0)
    assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0
    assert m.sync() == 0
    n_host = int(m.loads()[info["K"]:].astype(np.int64).sum())
    bytes_per_launch = 4 * N + 24 * n_host
    avg_s = sg["ms"] / max(1, sg["spans"]) * 1e-3
    achieved = bytes_per_launch / avg_s / 1e9 if sg["spans"] else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f).get("page_group", {}).get("bytes_per_launch_full")
    roofline_hbm = {"bound": "hbm",
                    "kernel": "k_group_buckets + k_group_pages (host records grouped by page)",
                    "achieved": round(achieved, 1) if achieved else None,
                    "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(achieved / hbm_peak, 4) if achieved and hbm_peak else None,
                    "traffic": traffic, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"
                    if hbm_peak else "fallback 6400 GB/s",
                    "algorithmic_bytes_per_launch": bytes_per_launch,
                    "host_records": n_host,
                    "launches": sg["spans"], "avg_launch_ms": round(avg_s * 1e3, 4),
                    "share_of_step": round(sg["ms"] * 1e-3 / step_s, 4)}

    # pinned copy bandwidth of the host link (sequential, 1 GiB each way)
    link = link_bandwidth(torch) if rank == 0 else {}

    # one access per batch (Alg. 1 one command at a time) on the same map:
    # device rate of width-1 batches, and one host-pointer call per op
    w1_n = 2048
    a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    assert m.access_device_batches(d_ops[:64], d_akeys[:64], d_avin[:64], d_vout[:64],
                                   d_status[:64], 1, stream=stream) == 0  # warm-up
    a1.record(stream)
    assert m.access_device_batches(d_ops[:w1_n], d_akeys[:w1_n], d_avin[:w1_n], d_vout[:w1_n],
                                   d_status[:w1_n], 1, stream=stream) == 0
    b1.record(stream)
    b1.synchronize()
    assert m.sync() == 0
    w1_dev = w1_n / (a1.elapsed_time(b1) * 1e-3)
    m.set_param(B.BOLT_PARAM_BATCH, 1)
    lat = one_op_calls(B, m, ops[:1000], akeys[:1000], avin[:1000], 1000)
    w1 = {"device_accesses_per_s": round(w1_dev, 1),
          "device_us_per_access": round(1e6 / w1_dev, 2),
          "host_call_accesses_per_s": round(len(lat) / float(lat.sum()), 1),
          "host_call_p50_us": round(float(np.median(lat)) * 1e6, 1),
          "host_call_p99_us": round(float(np.percentile(lat, 99)) * 1e6, 1),
          "note": f"the same map and op stream, batches of one op: {w1_n} through "
                  "bolt_access_device_batches (device time), 1000 bolt_access calls of one op "
                  "through the C ABI on preallocated host arrays (host wall time per call)"}

    # the owner-side build (Sec. 4.2 "Fast data initialization"): the same
    # records prepared as an image on this device (bolt_prepare_device), then
    # loaded with sequential reads and writes (bolt_init_prepared), event-timed
    rc, img = m.prepare_device(d_keys, d_vals, SEED_MAP, stream=stream)
    assert rc == 0, rc
    load_ms = []
    for _ in range(3):
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        assert m.init_prepared(img, N, SEED_MAP, stream=stream) == 0
        b2.record(stream)
        b2.synchronize()
        load_ms.append(a2.elapsed_time(b2))
    del img
    torch.cuda.empty_cache()
    owner = {"load_ms": round(min(load_ms), 2),
             "load_mrec_s": round(N / (min(load_ms) * 1e-3) / 1e6, 2),
             "device_build_ms": round(build_s / args.steps * 1e3, 2),
             "note": "bolt_init_prepared of a device-resident image (keys, values, pairs, rows, "
                     "counts) that bolt_prepare_device exported for the same records and seed; "
                     "best of 3; the data owner's own preprocessing time is not included"}

    # end to end through the host-pointer ABI (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        hk = torch.from_numpy(keys.view(np.int64)).pin_memory()
        hv = torch.from_numpy(vals).pin_memory()
        ho = torch.from_numpy(ops).pin_memory()
        hak = torch.from_numpy(akeys.view(np.int64)).pin_memory()
        havin = torch.from_numpy(avin).pin_memory()
        hvout = torch.empty((n_acc, VAL_BYTES), dtype=torch.uint8).pin_memory()
        hst = torch.empty(n_acc, dtype=torch.uint8).pin_memory()
        import ctypes

        def ptr(t):
            return ctypes.c_void_p(t.data_ptr())

        m.set_param(B.BOLT_PARAM_BATCH, BATCH)

        def e2e_step():
            t0 = time.perf_counter()
            rc = B.bolt_init(m.handle, ptr(hk), ptr(hv), N, SEED_MAP)
            assert rc == 0, rc
            t1 = time.perf_counter()
            # one call over the whole op stream: batches of BATCH ops
            rc = B.bolt_access(m.handle, ptr(ho), ptr(hak), ptr(havin), ptr(hvout), ptr(hst),
                               n_acc)
            assert rc == 0, rc
            t2 = time.perf_counter()
            return t1 - t0, t2 - t1

        e2e_step()
        eb, ea = 0.0, 0.0
        e2e_steps = max(1, min(2, args.steps))
        for _ in range(e2e_steps):
            b_s, a_s = e2e_step()
            eb += b_s
            ea += a_s
        assert np.array_equal(hvout.numpy(), vout), "host and device paths agree"
        # whole job over ranks, as for the headline value: the slowest rank's
        # times, the sum of the work and of the copies
        agg_e = aggregate({"build_s": eb, "access_s": ea, "step_s": eb + ea,
                           "records": float(N * e2e_steps),
                           "accesses": float(n_acc * e2e_steps)}, world, group)
        e2e = {"value": round(agg_e["accesses"] / agg_e["access_s"], 1), "unit": "accesses/s",
               "h2d_bytes_per_step": world * (N * (8 + VAL_BYTES) + n_acc * (1 + 8 + VAL_BYTES)),
               "d2h_bytes_per_step": world * n_acc * (VAL_BYTES + 1),
               "build_mrec_s": round(agg_e["records"] / agg_e["build_s"] / 1e6, 2),
               "steps": e2e_steps}
        del hk, hv, ho, hak, havin, hvout, hst

    # The access path's roofline (the headline value): per batch, every
    # host page a read position names is read once and written back once
    # (2(1 - alpha) pages per op, page_bytes each way) -- algorithmic
    # host-link bytes per batch over the device time per batch -- against
    # the random-page rate of this map's own pinned store measured by
    # bolt_probe_link (one batch's pages read beside the previous batch's
    # write-back, no compute), and against the sequential pinned copies.
    page_bytes = info["page_bytes"]
    per_op = 2.0 * info["M"] / info["B"]  # expected host pages read per op
    probe = m.probe_link(int(round(per_op * BATCH)), 50)
    # (per GPU: each rank's share of the work over the slowest rank's time)
    acc_rate = agg["accesses"] / world / agg["access_s"]
    batch_s = BATCH / acc_rate
    link_bytes_per_batch = 2 * per_op * BATCH * page_bytes
    ach = link_bytes_per_batch / batch_s / 1e9
    peak_link = probe["pipelined_pages_per_s"] * 2 * page_bytes / 1e9
    per_dir = per_op * page_bytes * acc_rate / 1e9
    roofline = {"bound": "host-link", "kernel": "access batch of 4096 ops (k_lookup page reads "
                                                "+ k_flush write-back; the rest of the chain "
                                                "overlaps them)",
                "achieved": round(ach, 2), "peak": round(peak_link, 2), "unit": "GB/s",
                "frac": round(ach / peak_link, 4), "traffic": None,
                "traffic_note": "host-link bytes are not DRAM bytes; the algorithmic figure "
                                "counts each read position's page once read and once written",
                "peak_source": "bolt_probe_link in this run: random 512-byte page reads and "
                               "write-backs on this map's pinned store, no compute",
                "algorithmic_bytes_per_launch": int(round(link_bytes_per_batch)),
                "launch": "one access batch (device time per batch from CUDA events over the "
                          "timed access phase)",
                "ms_per_batch": round(batch_s * 1e3, 4),
                "pages_per_op": round(per_op, 4), "page_bytes": page_bytes,
                "achieved_pages_per_s": round(acc_rate * per_op, 1),
                "peak_pages_per_s": round(probe["pipelined_pages_per_s"], 1),
                "read_only_pages_per_s": round(probe["read_pages_per_s"], 1),
                "per_direction_gbs": round(per_dir, 2),
                "vs_pinned_copy": {"h2d_gbs": link.get("h2d"), "d2h_gbs": link.get("d2h"),
                                   "frac": round(per_dir / min(link["h2d"], link["d2h"]), 4)
                                   if link else None},
                "share_of_step": round(agg["access_s"] / agg["step_s"], 4)}

    # the build: its pages leave over the link (D2H copies of the staged
    # chunks); phase shares from the event-timed kernel classes
    build_ms = build_s / args.steps * 1e3
    page_store = info["M"] * page_bytes
    bk = {k: prof[k]["ms"] / args.steps for k in ("p2c_rounds", "page_group", "sort_global",
                                                   "sort_tile", "page_build", "key_check")}
    build = {"value": round(agg["records"] / agg["build_s"] / 1e6, 2), "unit": "Mrec/s",
             "ms_per_build": round(build_ms, 2),
             "share_of_step": round(agg["build_s"] / agg["step_s"], 4),
             "link": {"page_store_bytes": page_store,
                      "achieved_gbs": round(page_store / (build_ms * 1e-3) / 1e9, 2),
                      "d2h_copy_gbs": link.get("d2h"),
                      "frac": round(page_store / (build_ms * 1e-3) / 1e9 / link["d2h"], 4)
                      if link else None,
                      "note": "the whole build's time against the page store's D2H copy "
                              "at the pinned-copy rate"},
             "phase_ms": {k: round(v, 2) for k, v in bk.items()},
             "phase_note": "event-timed kernel classes; the key check and the placement "
                           "run on a side stream beside the page build, so shares overlap"}

    m.close()
    del d_keys, d_vals, d_ops, d_akeys, d_avin, d_vout, d_status
    torch.cuda.empty_cache()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = cpu_baseline_sample() if world == 1 and not args.no_cpu else None
    cpu_mt = cpu_baseline_sample(8.0, multicore=True) if world == 1 and not args.no_cpu else None
    serving = None
    if world == 1 and not args.no_serve:
        serving = serve_measure(16, 2000, 24.0, (0.5,))
    gat, ev = aprof["gather"], aprof["evict"]
    line = {
        "metric": METRIC,
        "value": round(agg["accesses"] / agg["access_s"], 1),
        "unit": "accesses/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(agg["step_s"] / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8/u64 (integer; ChaCha20 ARX)",
        "data": "synthetic (seeded; keys = bijective mix of the record index, random values)",
        "config": config_for(args.log_n, n_acc, args.lookahead),
        "build": build,
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        "w1": w1,
        "owner_build": owner,
        "link": {"h2d_gbs": link.get("h2d"), "d2h_gbs": link.get("d2h"),
                 "gather_ms_per_batch": round(gat["ms"] / max(1, gat["spans"]), 4),
                 "evict_ms_per_batch": round(ev["ms"] / max(1, ev["spans"]), 4),
                 "page_bytes": page_bytes},
        "kernel_ms": {k: round(v["ms"], 2) for k, v in prof.items()
                      if isinstance(v, dict) and v["spans"]},
        "access_kernel_ms_per_batch": {k: round(v["ms"] / nb, 4) for k, v in aprof.items()
                                       if isinstance(v, dict) and v["spans"]},
        "gpu_launches": prof["launches"],
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "cpu_baseline_multicore": cpu_mt,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args) -> None:
    """Batch-width sweep on the skewed workload: N = 2^24 records of 64 B
    (8 B key + 56 B value), a 2 GB HBM budget (alpha = 0.2), Zipf(0.99) keys,
    70% GET / 30% PUT; accesses/s for batch widths 1, 4, 16, ..., 65536 (one
    bolt_access_device_batches call over all the batches of a width).  Also one access per call vs batches of
    4096 on the headline map when --config w1 is given."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    if args.config == "zipf":
        log_n, vb, budget, get_frac, theta = 24, 56, 2 * 10**9, 0.7, 0.99
        widths = [1, 4, 16, 64, 256, 1024, 4096, 16384, 65536]
    else:
        log_n, vb, budget, get_frac, theta = args.log_n, VAL_BYTES, 2**64 - 1, 0.5, None
        widths = [1, 4096]
    N = 1 << log_n
    keys = np.empty(N, dtype=np.uint64)
    for lo in range(0, N, 1 << 24):
        keys[lo:lo + (1 << 24)] = W.key_of(np.arange(lo, min(N, lo + (1 << 24)), dtype=np.uint64))
    rng = np.random.default_rng(SEED_DATA)
    vals = np.frombuffer(rng.bytes(N * vb), dtype=np.uint8).reshape(N, vb)
    n_ops = 1 << 20
    ops, akeys, avin = W.op_stream(N, n_ops, vb, SEED_OPS, get_frac=get_frac, zipf_theta=theta)
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
    d_vals = torch.from_numpy(vals.copy()).cuda()
    d_ops = torch.from_numpy(ops).cuda()
    d_akeys = torch.from_numpy(akeys.view(np.int64)).cuda()
    d_avin = torch.from_numpy(avin).cuda()
    d_vout = torch.empty((n_ops, vb), dtype=torch.uint8, device="cuda")
    d_st = torch.empty(n_ops, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    m = B.BoltMap(N, vb, hbm_budget=budget)
    assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0
    rows = []
    for w in widths:
        count = min(n_ops, max(4096, 64 * w)) if w < 4096 else n_ops
        count -= count % w
        nb = count // w
        for _ in range(min(3, nb)):  # warm-up batches
            assert m.access_device(d_ops[:w], d_akeys[:w], d_avin[:w], d_vout[:w], d_st[:w],
                                   stream=stream) == 0
        assert m.sync() == 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        assert m.access_device_batches(d_ops[:count], d_akeys[:count], d_avin[:count],
                                       d_vout[:count], d_st[:count], w, stream=stream) == 0
        b.record(stream)
        b.synchronize()
        wall = time.perf_counter() - t0
        assert m.sync() == 0
        dev_s = a.elapsed_time(b) * 1e-3
        rows.append({"batch": w, "accesses": count, "accesses_per_s": round(count / dev_s, 1),
                     "wall_accesses_per_s": round(count / wall, 1),
                     "us_per_batch": round(dev_s / nb * 1e6, 2)})
    best = max(rows, key=lambda r: r["accesses_per_s"])
    line = {"metric": "oblivious accesses/s vs batch width", "config": {
        "workload": f"N=2^{log_n} records x {8 + vb} B, "
                    + ("Zipf(0.99) keys, 70% GET / 30% PUT, 2 GB HBM budget" if theta else
                       "uniform keys, 50% GET / 50% PUT"), "alpha": m.info()["alpha"]},
            "unit": "accesses/s", "sweep": rows, "best_batch": best["batch"],
            "value": best["accesses_per_s"], "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic"}
    print(json.dumps(line), flush=True)


def serve_measure(n_maps: int, n_requests: int, log_n_max: float = 26.0,
                  fractions=(0.5, 0.8)) -> dict:
    """Serving: n_maps maps with N log-uniform in [2^12, 2^log_n_max] (32 B
    records), admitted under a 120 GB HBM budget; Poisson request arrivals,
    request sizes log-uniform in 1..4096 ops, 70% GET / 30% PUT, Zipf(0.99)
    keys per map.  Saturation throughput is measured closed-loop (every
    request queued at once; the median of three runs); then open-loop at the
    given fractions of it:
    p50 / p99 latency from arrival to completed batch, and accesses/s."""
    import threading
    from paper_2509_01742_b300 import bolt as B

    rng = np.random.default_rng(0x5EED0005)
    vb, max_batch = VAL_BYTES, 4096
    log_ns = rng.uniform(12, log_n_max, n_maps)
    Ns = [int(2 ** x) for x in log_ns]
    srv = B.BoltServer(hbm_budget=120 * 10**9, max_batch=max_batch)
    t0 = time.perf_counter()
    mids = []
    for j, N in enumerate(Ns):
        keys, vals = make_records_vb(N, vb, SEED_DATA + j)
        mids.append(srv.add_map(N, vb, keys, vals, SEED_MAP + j))
    while any(srv.map_state(m) == 0 for m in mids):
        time.sleep(0.05)
    assert all(srv.map_state(m) == 1 for m in mids)
    build_s = time.perf_counter() - t0
    zipfs = {}

    import ctypes

    def gen_requests(count, seed):
        """(map, ops, keys, vin, C pointers) per request, built before the
        clock starts so that submitting is one C call per request"""
        g = np.random.default_rng(seed)
        out = []
        for _ in range(count):
            j = int(g.integers(0, n_maps))
            n = int(np.exp(g.uniform(0, np.log(max_batch))))
            N = Ns[j]
            if N not in zipfs:
                zipfs[N] = W.Zipf(N, 0.99)
            ranks = zipfs[N].sample(g, n)
            keys = np.ascontiguousarray(W.key_of(W.mix64(ranks) % np.uint64(N)))
            ops = (g.random(n) >= 0.7).astype(np.uint8)  # 70% GET (0), 30% PUT (1)
            vin = np.ascontiguousarray(g.integers(0, 256, size=(n, vb), dtype=np.uint8))
            ptrs = tuple(ctypes.c_void_p(a.ctypes.data) for a in (ops, keys, vin))
            out.append((j, ops, keys, vin, ptrs))
        return out

    def run(reqs, rate_ops=None):
        """Submit requests (at Poisson times for the given op rate, or all at
        once), wait for all; returns (latencies_us, ops, seconds)."""
        ids = [None] * len(reqs)
        lat = [0.0] * len(reqs)
        done_ev = threading.Event()
        failed = []

        def waiter():
            info = B.bolt_req_info_t()
            try:
                for i in range(len(reqs)):
                    while ids[i] is None:
                        if failed:
                            return
                        time.sleep(0)
                    j = reqs[i][0]
                    # timestamps only (the outputs are not copied out)
                    rc = B.bolt_server_wait(srv._s, ids[i], None, None, ctypes.byref(info), 60000)
                    if rc != 0:
                        why = B.bolt_strerror(rc).decode()
                        raise RuntimeError(f"request {i} on map {j}: {why} ({rc})")
                    lat[i] = (info.done_us - info.submit_us, info.submit_us, info.done_us)
            except BaseException as exc:  # reported by the submitting thread
                failed.append(exc)
            finally:
                done_ev.set()

        th = threading.Thread(target=waiter)
        th.start()
        total = sum(len(r[1]) for r in reqs)
        mean_n = total / len(reqs)
        start = time.perf_counter()

        def submit_many(lo, hi):
            P = ctypes.c_void_p * (hi - lo)
            part = reqs[lo:hi]
            mids_a = np.array([mids[r[0]] for r in part], dtype=np.uint32)
            ns_a = np.array([len(r[1]) for r in part], dtype=np.uint32)
            po, pk, pv = (P(*[r[4][x] for r in part]) for x in range(3))
            out = np.zeros(hi - lo, dtype=np.uint64)
            rc = B.bolt_server_submit_many(srv._s, hi - lo, mids_a.ctypes.data, po, pk, pv,
                                           ns_a.ctypes.data, out.ctypes.data)
            if rc != 0:
                raise RuntimeError(f"submit_many: {B.bolt_strerror(rc).decode()}")
            for i in range(lo, hi):
                ids[i] = int(out[i - lo])

        if not rate_ops:
            # closed loop: every request queued by one call (its arrival time
            # is the call's; the copies into the server count)
            submit_many(0, len(reqs))
        else:
            # open loop: Poisson arrival times at rate_ops; whenever requests
            # are due, all of them are queued by one call (a request's
            # arrival is that call), so the client keeps up with the rate
            arrive = np.cumsum(np.random.default_rng(7).exponential(mean_n / rate_ops, len(reqs)))
            k = 0
            while k < len(reqs) and not failed:
                m = int(np.searchsorted(arrive, time.perf_counter() - start, side="right"))
                if m > k:
                    submit_many(k, m)
                    k = m
                else:
                    time.sleep(0)
        done_ev.wait()
        th.join()
        if failed:
            raise failed[0]
        first = min(x[1] for x in lat)
        last = max(x[2] for x in lat)
        return np.array([x[0] for x in lat]), total, (last - first) * 1e-6

    warm = gen_requests(min(200, n_requests), 1)
    run(warm)
    # saturation: the median of three closed-loop runs (one run lasts a few
    # hundred ms and moves by tens of percent from run to run)
    sats = []
    for seed in (2, 7, 8):
        sat_reqs = gen_requests(n_requests, seed)
        lat, ops, secs = run(sat_reqs)
        sats.append(ops / secs)
    sat = float(np.median(sats))
    levels = []
    for frac, seed in zip(fractions, (3, 4, 5, 6)):
        reqs = gen_requests(n_requests, seed)
        lat, ops, secs = run(reqs, rate_ops=frac * sat)
        levels.append({"offered_fraction": frac, "offered_accesses_per_s": round(frac * sat, 1),
                       "accesses_per_s": round(ops / secs, 1),
                       "p50_us": round(float(np.percentile(lat, 50)), 1),
                       "p99_us": round(float(np.percentile(lat, 99)), 1),
                       "requests": len(reqs)})
    st = srv.stats()
    srv.close()
    return {"workload": f"{n_maps} maps, N log-uniform in [2^12, 2^{log_n_max:g}] "
                        "(32 B records), 120 GB HBM budget, Poisson arrivals, "
                        "request size log-uniform 1..4096, 70% GET / 30% PUT, "
                        "Zipf(0.99) keys", "records": int(sum(Ns)), "max_batch": max_batch,
            "saturation": {"accesses_per_s": round(sat, 1), "requests": len(sat_reqs),
                           "runs": [round(x, 1) for x in sats]},
            "levels": levels, "build_s": round(build_s, 2),
            "batches": st["batches"], "hbm_used_bytes": st["used"]}


def run_serve(args) -> None:
    """The serving configuration on its own line (64 maps by default)."""
    import torch
    torch.cuda.set_device(0)
    r = serve_measure(args.maps, args.requests)
    line = {"metric": "served p50/p99 latency and accesses/s", "unit": "accesses/s",
            "value": r["saturation"]["accesses_per_s"], "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic",
            "config": {"workload": r["workload"], "records": r["records"],
                       "max_batch": r["max_batch"]},
            "saturation": r["saturation"], "levels": r["levels"], "build_s": r["build_s"],
            "batches": r["batches"], "hbm_used_bytes": r["hbm_used_bytes"]}
    print(json.dumps(line), flush=True)


def host_mem_available() -> int:
    """MemAvailable of this host in bytes (0 if unknown)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_big(args) -> None:
    """The largest configuration: N = 2^30 records of 64 B (8 B key + 56 B
    value) under a 16 GB HBM budget (alpha = 0.1: ~120.8 M host pages of
    960 B, ~116 GB of pinned host memory), built from keys and values
    generated on the device; then 2^24 Zipf(0.99) accesses, 90% GET / 10%
    PUT, in batches of 4096 (a 2^20-op warm-up pass first).  The sampled GETs
    are checked against the initial values and the stream's own PUTs.  Skips
    (prints a "skipped" line) when the host cannot pin the page store."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    log_n = args.big_log_n
    N, vb, budget = 1 << log_n, 56, 16 * 10**9
    info = B.plan(N, vb, budget)
    pinned = info["M"] * info["page_bytes"]
    avail = host_mem_available()
    config = {"workload": f"N=2^{log_n} records x 64 B (8 B key + 56 B value), 16 GB HBM budget, "
                          "inputs generated on the device; 2^24 Zipf(0.99) accesses, 90% GET / "
                          "10% PUT, batches of 4096",
              "records": N, "alpha": info["alpha"], "pinned_page_bytes": pinned}
    line = {"metric": "oblivious accesses/s and build Mrec/s, largest map", "unit": "accesses/s",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "config": config}
    if not avail or pinned + (24 << 30) > avail:
        line["skipped"] = f"host memory: {pinned / 2**30:.1f} GiB of pinned pages needed, " \
                          f"{avail / 2**30:.1f} GiB available"
        print(json.dumps(line), flush=True)
        return
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d_keys = W.key_of_torch(torch.arange(N, device="cuda", dtype=torch.int64))
        d_vals = torch.empty((N, vb), dtype=torch.uint8, device="cuda")
        g = torch.Generator(device="cuda")
        g.manual_seed(SEED_DATA + 4)
        for lo in range(0, N, 1 << 26):
            hi = min(N, lo + (1 << 26))
            d_vals[lo:hi] = torch.randint(0, 256, (hi - lo, vb), dtype=torch.uint8,
                                          device="cuda", generator=g)
    torch.cuda.synchronize()
    n_warm, n_ops = 1 << 20, 1 << 24
    ops, akeys, avin, aidx = W.op_stream(N, n_warm + n_ops, vb, SEED_OPS + 4, get_frac=0.9,
                                         zipf_theta=0.99, return_index=True)
    d_ops = torch.from_numpy(ops).cuda()
    d_akeys = torch.from_numpy(akeys.view(np.int64)).cuda()
    d_avin = torch.from_numpy(avin).cuda()
    d_vout = torch.empty((n_warm + n_ops, vb), dtype=torch.uint8, device="cuda")
    d_st = torch.empty(n_warm + n_ops, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    m = B.BoltMap(N, vb, hbm_budget=budget)
    alloc_s = time.perf_counter() - t0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    assert m.init_device(d_keys, d_vals, SEED_MAP + 4, stream=stream) == 0
    ev[1].record(stream)
    assert m.access_device_batches(d_ops[:n_warm], d_akeys[:n_warm], d_avin[:n_warm],
                                   d_vout[:n_warm], d_st[:n_warm], BATCH, stream=stream) == 0
    ev[2].record(stream)
    with ClockSampler(0) as clk:
        assert m.access_device_batches(d_ops[n_warm:], d_akeys[n_warm:], d_avin[n_warm:],
                                       d_vout[n_warm:], d_st[n_warm:], BATCH,
                                       stream=stream) == 0
        ev[3].record(stream)
        ev[3].synchronize()
    assert m.sync() == 0
    build_s = ev[0].elapsed_time(ev[1]) * 1e-3
    acc_s = ev[2].elapsed_time(ev[3]) * 1e-3
    # check: every key exists; a sample of GETs returns the last PUT before it
    # in the stream, else the record's initial value
    st = d_st.cpu().numpy()
    assert st.all(), "every accessed key exists"
    rng = np.random.default_rng(5)
    gets = np.flatnonzero(ops == W.GET)
    sample = np.sort(rng.choice(gets, size=min(20000, len(gets)), replace=False))
    T = np.uint64(len(ops))
    puts = np.flatnonzero(ops == W.PUT).astype(np.uint64)
    put_key = np.sort(aidx[puts] * T + puts)
    q = aidx[sample] * T + sample.astype(np.uint64)
    j = np.searchsorted(put_key, q) - 1
    has = (j >= 0) & (put_key[np.maximum(j, 0)] // T == aidx[sample])
    last_put = (put_key[np.maximum(j, 0)] % T).astype(np.int64)
    init_vals = d_vals[torch.from_numpy(aidx[sample].astype(np.int64)).cuda()].cpu().numpy()
    expect = np.where(has[:, None], avin[last_put], init_vals)
    got = d_vout[torch.from_numpy(sample.astype(np.int64)).cuda()].cpu().numpy()
    assert np.array_equal(got, expect), "sampled GETs match the stream"
    per_op = 2.0 * info["M"] / info["B"]
    probe = m.probe_link(int(round(per_op * BATCH)), 20)
    rate = n_ops / acc_s
    line.update({
        "value": round(rate, 1),
        "build": {"value": round(N / build_s / 1e6, 2), "unit": "Mrec/s",
                  "ms_per_build": round(build_s * 1e3, 1),
                  "pinned_alloc_s": round(alloc_s, 1)},
        "access_link": {"achieved_pages_per_s": round(rate * per_op, 1),
                        "peak_pages_per_s": round(probe["pipelined_pages_per_s"], 1),
                        "frac": round(rate * per_op / probe["pipelined_pages_per_s"], 4),
                        "pages_per_op": round(per_op, 4), "page_bytes": info["page_bytes"]},
        "checked_gets": int(len(sample)),
        "clocks": clk.summary(),
    })
    m.close()
    print(json.dumps(line), flush=True)


def run_validate(args) -> None:
    """The paper's dimensional validation (Sec. 3.3 "Dimensions in
    practice", the table inside Fig. 5) on the device: N = 2^20 records, for
    c in {8, 16} and alpha in {0.01, 0.2, 0.5}, `--accesses` uniform random
    accesses (Get on present keys; every access remaps its key) in batches of
    `--width`; the peak bin load, peak HBM-store occupancy and peak stash
    occupancy since the build (device counters, bolt_get_stats) beside the
    analytical bounds and the paper's empirical maxima (bound - printed
    slack).  The paper accesses one key at a time: at the end of a batch of W
    the stash also holds that batch's own remapped keys (about W (1 - alpha)
    of them) that no page read has had a chance to evict yet."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    N, vb, W_ = 1 << 20, 8, args.width
    slack = {}
    with open(os.path.join(ROOT, "tests", "golden", "slack_table.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                metric, c, a, abs_s, _ = ln.split()
                slack[(metric, int(c), float(a))] = int(abs_s)
    keys = W.key_of(np.arange(N, dtype=np.uint64))
    vals = np.zeros((N, vb), dtype=np.uint8)
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
    d_vals = torch.from_numpy(vals).cuda()
    chunk = 1 << 22
    d_ops = torch.zeros(chunk, dtype=torch.uint8, device="cuda")
    d_vin = torch.zeros((chunk, vb), dtype=torch.uint8, device="cuda")
    d_out = torch.empty((chunk, vb), dtype=torch.uint8, device="cuda")
    d_st = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda")
    stream = torch.cuda.Stream()
    rows = []
    total = int(args.accesses)
    for c in (8, 16):
        for alpha in (0.01, 0.2, 0.5):
            m = B.BoltMap(N, vb, alpha=alpha, c=c)
            info = m.info()
            assert m.init_device(d_keys, d_vals, 0x5EED0007, stream=stream) == 0
            gen.manual_seed(int(c * 1000 + alpha * 100))
            t0 = time.perf_counter()
            done = 0
            while done < total:
                n = min(chunk, total - done)
                n -= n % W_ if n > W_ else 0
                with torch.cuda.stream(stream):
                    idx = torch.randint(0, N, (n,), device="cuda", generator=gen)
                    d_k = W.key_of_torch(idx)
                assert m.access_device_batches(d_ops[:n], d_k, d_vin[:n], d_out[:n], d_st[:n],
                                               W_, stream=stream) == 0
                done += n
            assert m.sync() == 0
            secs = time.perf_counter() - t0
            st = m.stats()
            assert bool(d_st[:n].all()), "every accessed key is present"
            emp = {k: (b - slack[(k, c, alpha)]) for k, b in
                   (("binload", info["lmax"]), ("hbm", info["beta1"]), ("stash", info["beta2"]))}
            rows.append({"c": c, "alpha": alpha, "accesses": done, "seconds": round(secs, 1),
                         "peak_load": st["peak_load"], "lmax": info["lmax"],
                         "paper_peak_load": emp["binload"],
                         "peak_hbm": st["peak_hbm"], "beta1": round(info["beta1"], 1),
                         "paper_peak_hbm": round(emp["hbm"], 1),
                         "peak_hbm_vs_paper": round(st["peak_hbm"] / emp["hbm"] - 1, 4),
                         "peak_stash": st["peak_stash"], "beta2": round(info["beta2"], 1),
                         "paper_peak_stash": round(emp["stash"], 1),
                         "peak_stash_vs_paper": round(st["peak_stash"] / emp["stash"] - 1, 4),
                         "batch_remap_term": round(W_ * (1 - alpha), 1)})
            print(json.dumps(rows[-1]), flush=True)
            m.close()
    line = {"metric": "dimensional validation: peak bin load, HBM store and stash (N=2^20)",
            "unit": "items", "n_gpus": 1, "data": "synthetic (uniform random accesses)",
            "config": {"workload": f"N=2^20 records, {total} uniform accesses per setting in "
                                   f"batches of {W_}, c in {{8,16}}, alpha in {{0.01,0.2,0.5}}"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_scaling(args) -> None:
    """The shape of the paper's scaling experiments (Sec. 5.4: entries from
    10^5 to 10^7 at 8-byte values; values from 8 to 256 bytes): for each map,
    the device build (init) time, Gets and Puts one operation per batch
    (Alg. 1, one command at a time; 2000 ops through bolt_access_device_batches
    of width 1, device time) and in batches of 4096 (2^20 ops), 50% GET / 50%
    PUT on present keys, uniform.  Keys and values are generated on the
    device."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    grid = [(n, 8) for n in (10**5, 10**6, 10**7)] + [(10**6, vb) for vb in (32, 128, 256)]
    rows = []
    for N, vb in grid:
        g = torch.Generator(device="cuda")
        g.manual_seed(N + vb)
        with torch.cuda.stream(stream):
            d_keys = W.key_of_torch(torch.arange(N, device="cuda", dtype=torch.int64))
            d_vals = torch.randint(0, 256, (N, vb), dtype=torch.uint8, device="cuda", generator=g)
        n_ops = 1 << 20
        ops, akeys, avin = W.op_stream(N, n_ops, vb, SEED_OPS + N + vb, get_frac=0.5)
        d_ops = torch.from_numpy(ops).cuda()
        d_ak = torch.from_numpy(akeys.view(np.int64)).cuda()
        d_av = torch.from_numpy(avin).cuda()
        d_out = torch.empty((n_ops, vb), dtype=torch.uint8, device="cuda")
        d_st = torch.empty(n_ops, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        m = B.BoltMap(N, vb)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0  # warm-up build
        ev[0].record(stream)
        assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0
        ev[1].record(stream)
        n1 = 2000
        assert m.access_device_batches(d_ops[:64], d_ak[:64], d_av[:64], d_out[:64], d_st[:64],
                                       1, stream=stream) == 0
        ev[2].record(stream)
        assert m.access_device_batches(d_ops[:n1], d_ak[:n1], d_av[:n1], d_out[:n1], d_st[:n1],
                                       1, stream=stream) == 0
        ev[3].record(stream)
        ev[4].record(stream)
        assert m.access_device_batches(d_ops, d_ak, d_av, d_out, d_st, BATCH, stream=stream) == 0
        ev[5].record(stream)
        ev[5].synchronize()
        assert m.sync() == 0
        assert bool(d_st.all()), "every accessed key is present"
        info = m.info()
        rows.append({"N": N, "val_bytes": vb, "alpha": info["alpha"],
                     "page_bytes": info["page_bytes"],
                     "init_ms": round(ev[0].elapsed_time(ev[1]), 2),
                     "init_mrec_s": round(N / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e6, 1),
                     "w1_accesses_per_s": round(n1 / (ev[2].elapsed_time(ev[3]) * 1e-3), 1),
                     "w1_us_per_access": round(ev[2].elapsed_time(ev[3]) * 1e3 / n1, 2),
                     "batched_accesses_per_s": round(n_ops / (ev[4].elapsed_time(ev[5]) * 1e-3), 1)})
        print(json.dumps(rows[-1]), flush=True)
        m.close()
        del d_keys, d_vals, d_ops, d_ak, d_av, d_out, d_st
        torch.cuda.empty_cache()
    line = {"metric": "init time and accesses/s vs entries and value size", "unit": "accesses/s",
            "n_gpus": 1, "data": "synthetic (device-generated keys and values)",
            "config": {"workload": "N in {1e5, 1e6, 1e7} at 8 B values; values in {8, 32, 128, "
                                   "256} B at N = 1e6; uniform 50/50 GET/PUT on present keys"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_integrity(args) -> None:
    """The cost of sealed pages (BOLT_PARAM_INTEGRITY: ChaCha20-Poly1305 per
    page, tag checked on every read): the headline map (N = 2^log_n records
    of 32 B, uniform 50/50 GET/PUT on present keys) built and accessed with
    plain pages, then with sealed pages -- device build time, one op per
    batch (2000 ops of width 1) and batches of 4096 (2^22 ops), CUDA events
    on the map's stream.  Keys and values are generated on the device."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    N, vb = 1 << args.log_n, VAL_BYTES
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED_DATA)
    with torch.cuda.stream(stream):
        d_keys = W.key_of_torch(torch.arange(N, device="cuda", dtype=torch.int64))
        d_vals = torch.randint(0, 256, (N, vb), dtype=torch.uint8, device="cuda", generator=g)
    n_ops = args.accesses
    ops, akeys, avin = W.op_stream(N, n_ops, vb, SEED_OPS, get_frac=0.5)
    d_ops = torch.from_numpy(ops).cuda()
    d_ak = torch.from_numpy(akeys.view(np.int64)).cuda()
    d_av = torch.from_numpy(avin).cuda()
    d_out = torch.empty((n_ops, vb), dtype=torch.uint8, device="cuda")
    d_st = torch.empty(n_ops, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rows = []
    for sealed in (0, 1):
        m = B.BoltMap(N, vb, integrity=bool(sealed))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0  # warm-up build
        ev[0].record(stream)
        assert m.init_device(d_keys, d_vals, SEED_MAP, stream=stream) == 0
        ev[1].record(stream)
        n1 = 2000
        assert m.access_device_batches(d_ops[:64], d_ak[:64], d_av[:64], d_out[:64], d_st[:64],
                                       1, stream=stream) == 0
        ev[2].record(stream)
        assert m.access_device_batches(d_ops[:n1], d_ak[:n1], d_av[:n1], d_out[:n1], d_st[:n1],
                                       1, stream=stream) == 0
        ev[3].record(stream)
        # warm-up batches, then the timed ones
        assert m.access_device_batches(d_ops[:8 * BATCH], d_ak[:8 * BATCH], d_av[:8 * BATCH],
                                       d_out[:8 * BATCH], d_st[:8 * BATCH], BATCH,
                                       stream=stream) == 0
        ev[4].record(stream)
        assert m.access_device_batches(d_ops, d_ak, d_av, d_out, d_st, BATCH, stream=stream) == 0
        ev[5].record(stream)
        ev[5].synchronize()
        assert m.sync() == 0
        assert bool(d_st.all()), "every accessed key is present"
        info = m.info()
        rows.append({"sealed": sealed, "page_bytes": info["page_bytes"],
                     "init_ms": round(ev[0].elapsed_time(ev[1]), 2),
                     "w1_us_per_access": round(ev[2].elapsed_time(ev[3]) * 1e3 / n1, 2),
                     "batched_accesses_per_s": round(n_ops / (ev[4].elapsed_time(ev[5]) * 1e-3), 1)})
        print(json.dumps(rows[-1]), flush=True)
        m.close()
        torch.cuda.empty_cache()
    line = {"metric": "accesses/s and build time, plain vs sealed pages", "unit": "accesses/s",
            "n_gpus": 1, "data": "synthetic (device-generated keys and values)",
            "config": {"workload": f"N=2^{args.log_n} x 32 B, uniform 50/50 GET/PUT on present "
                                   f"keys, {n_ops} accesses in batches of {BATCH}"},
            "rows": rows,
            "sealed_vs_plain": round(rows[1]["batched_accesses_per_s"] /
                                     rows[0]["batched_accesses_per_s"], 4)}
    print(json.dumps(line), flush=True)


def make_records_vb(n: int, vb: int, seed: int):
    keys = np.empty(n, dtype=np.uint64)
    for lo in range(0, n, 1 << 24):
        hi = min(n, lo + (1 << 24))
        keys[lo:hi] = W.key_of(np.arange(lo, hi, dtype=np.uint64))
    rng = np.random.default_rng(seed)
    vals = np.frombuffer(rng.bytes(n * vb), dtype=np.uint8).reshape(n, vb)
    return keys, vals


def run_paper_workload(args) -> None:
    """The paper's own query workload (Sec. 5.1 testbed: N = 10^6 records of
    4-byte keys and 8-byte values, then 2500 Get + 2500 Put on random present
    keys, processed one at a time): one bolt_access call per operation through
    host buffers, and the same 5000 operations as one call.  The paper's
    U55C figure (174 k queries/s, Table 2) is context for the first number;
    this path's design point is the batched call."""
    import torch
    from paper_2509_01742_b300 import bolt as B

    torch.cuda.set_device(0)
    N, vb, n_ops = 10**6, 8, 5000
    rng = np.random.default_rng(0x5EED0006)
    keys = rng.choice(2**32, size=N, replace=False).astype(np.uint32)
    vals = rng.integers(0, 256, (N, vb), dtype=np.uint8)
    idx = rng.integers(0, N, n_ops)
    ops = np.array([W.GET] * (n_ops // 2) + [W.PUT] * (n_ops - n_ops // 2), dtype=np.uint8)
    rng.shuffle(ops)
    vin = rng.integers(0, 256, (n_ops, vb), dtype=np.uint8)
    m = B.BoltMap(N, vb, key_bytes=4)
    t0 = time.perf_counter()
    assert m.init(keys, vals, SEED_MAP) == 0
    init_s = time.perf_counter() - t0
    lat = one_op_calls(B, m, ops, keys[idx], vin, n_ops, warm=200)
    one_s = float(lat.sum())
    t = time.perf_counter()
    assert m.access(ops, keys[idx], vin)[0] == 0
    batch_s = time.perf_counter() - t
    info = m.info()
    m.close()
    line = {"metric": "queries/s, the paper's workload one op per call", "unit": "queries/s",
            "value": round(n_ops / one_s, 1), "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic",
            "config": {"workload": "N=10^6, 4 B keys, 8 B values, 2500 Get + 2500 Put on "
                                   "random present keys, one bolt_access call per op through "
                                   "the C ABI (host buffers, preallocated)",
                       "alpha": info["alpha"]},
            "per_call_us": {"p50": round(float(np.median(lat)) * 1e6, 1),
                            "p99": round(float(np.percentile(lat, 99)) * 1e6, 1)},
            "one_call_of_5000": {"queries_per_s": round(n_ops / batch_s, 1),
                                 "seconds": round(batch_s, 6)},
            "init_s": round(init_s, 3),
            "paper_u55c_queries_per_s": 174000}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("bolt", "reference"), default="bolt")
    ap.add_argument("--config", choices=("headline", "zipf", "w1", "serve", "big", "paper",
                                         "validate", "scaling", "integrity"),
                    default="headline",
                    help="headline: the JSON line above; zipf: batch-width sweep on the "
                         "skewed 2^24 x 64 B map; w1: one access per call vs batches of 4096; "
                         "serve: 64 maps behind the continuous-batching server; big: the "
                         "2^30 x 64 B map under a 16 GB budget; paper: the paper's 10^6 x "
                         "(4 B key, 8 B value) workload, one op per call; integrity: plain "
                         "vs sealed pages on the headline map")
    ap.add_argument("--big-log-n", type=int, default=30)
    ap.add_argument("--width", type=int, default=4096,
                    help="batch width of --config validate")
    ap.add_argument("--maps", type=int, default=64)
    ap.add_argument("--requests", type=int, default=6000)
    ap.add_argument("--log-n", type=int, default=LOG_N)
    ap.add_argument("--accesses", type=int, default=N_ACCESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the bounded serving run of the headline line")
    ap.add_argument("--defer", type=int, default=None, choices=(0, 1, 2),
                    help="BOLT_PARAM_DEFER_FLUSH for the headline map (default: the library's, 0)")
    ap.add_argument("--lookahead", type=float, default=0.0,
                    help="share of each batch's pages read while the previous batch "
                         "finishes (0 = off)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "bolt" and args.config == "headline":
        print("note: at least 3 warm-up steps are required for a valid number", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "serve":
        run_serve(args)
    elif args.config == "big":
        run_big(args)
    elif args.config == "paper":
        run_paper_workload(args)
    elif args.config == "validate":
        run_validate(args)
    elif args.config == "scaling":
        run_scaling(args)
    elif args.config == "integrity":
        run_integrity(args)
    elif args.config != "headline":
        run_sweep(args)
    else:
        run_bolt(args)


if __name__ == "__main__":
    main()
