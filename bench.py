"""Benchmark of the HoSZp hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hoszp|reference]

Workload (the 3-D configuration of the benchmark set): two float32 Gaussian
random fields A and B of 512^3 values (E(k) ~ k^-5/3, seeds 1 and 2), value-range
relative bound 1e-4 (B is compressed with A's absolute bound so the two streams
can be added). One step runs every row of the hot path once:

    compress A, compress B        (range pass, Eq. 3, Eq. 4, BF encoding)
    negate A, add_scalar A 0.5, mul_scalar A 3.14, add A+B  (Sec. V-A, V-C)
    mean A, var A                 (Sec. V-B)
    decompress A                  (inverse pipeline)

value = original bytes the step's operators take as input (4N per input field,
10 fields' worth per step) / step time, in GB/s. The line also carries the
per-operator breakdown, the GPU decompress -> op -> recompress comparator built
from the same library, the roofline of the dominant operator, the oracle timed
on the host cores (cpu_baseline) and the end-to-end figure through host memory.
Multi-GPU (torchrun): every rank runs its own pair of fields (weak scaling, no
collective on the data path); time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("homomorphic op GB/s (original bytes) & % HBM roofline vs GPU "
          "decompress-op-recompress")
SHAPE = (512, 512, 512)
REL = 1e-4
DEFAULT_SHAPE = SHAPE
SCALAR_ADD = 0.5
SCALAR_MUL = 3.14


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2408_11971_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(op: str):
    """DRAM bytes per call of operator `op` (all its kernels, scaled to the 512^3
    workload) from the committed ncu summary, if the kernel sources have not
    changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        if d.get("csrc_sha") == csrc_hash():
            return d["ops"].get(op)
    except Exception:
        pass
    return None


# kernels of one benchmark step, operator by operator, in launch order
STEP_KERNELS = (("compress A", ("k_range", "k_compress", "k_place")),
                ("compress B", ("k_compress", "k_place")),
                ("negate", ("k_meta<1>",)), ("add_scalar", ("k_meta<0>",)),
                ("mul_scalar", ("k_mul_lanes", "k_place")),
                ("add", ("k_add", "k_place")), ("mean", ("k_mean",)),
                ("var", ("k_var",)), ("decompress", ("k_decompress_lanes",)))
KERNELS_PER_STEP = sum(len(ks) for _, ks in STEP_KERNELS)  # library launches per step


def traffic_from_csv(path: str, shape) -> dict:
    """Per-operator DRAM bytes from an ncu launch list of the benchmark step
    (metrics gpu__time_duration.sum, dram__bytes_read.sum, dram__bytes_write.sum),
    captured on fields of `shape`: the library's launches are matched against
    the step's kernel sequence, the first step is dropped (cold), the others
    averaged, and bytes are scaled to the 512^3 workload by the number of values.
    Writes profiles/traffic.json with the hash of the kernel sources."""
    import csv

    rows = list(csv.reader(open(path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ki, mi, vi, ii = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "ID"))
    launches = {}
    for r in rows[start + 1:]:
        if len(r) <= max(ki, mi, vi, ii):
            continue
        name = r[ki].split("(")[0].replace("void ", "").strip()
        if not name.startswith("hz::"):
            continue
        d = launches.setdefault(int(r[ii]), {"name": name[4:]})
        d[r[mi]] = float(r[vi].replace(",", ""))
    seq = [launches[k] for k in sorted(launches)]
    flat = [k for _, ks in STEP_KERNELS for k in ks]
    hits = [i for i in range(len(seq) - len(flat) + 1)
            if all(seq[i + j]["name"].startswith(flat[j]) for j in range(len(flat)))]
    if not hits:
        raise SystemExit("no complete benchmark step in " + path)
    use = hits[1:] or hits
    scale = float(np.prod(DEFAULT_SHAPE)) / float(np.prod(shape))
    ops = {}
    for s0 in use:
        i = s0
        for op, ks in STEP_KERNELS:
            part = seq[i:i + len(ks)]
            i += len(ks)
            o = ops.setdefault(op, {"kernels": list(ks), "us": 0.0, "dram_read": 0.0,
                                    "dram_write": 0.0})
            o["us"] += sum(p["gpu__time_duration.sum"] for p in part) / 1e3 / len(use)
            o["dram_read"] += sum(p["dram__bytes_read.sum"] for p in part) * scale / len(use)
            o["dram_write"] += sum(p["dram__bytes_write.sum"] for p in part) * scale / len(use)
    for o in ops.values():
        o["dram_bytes_per_launch"] = o["dram_read"] + o["dram_write"]
    out = {"csrc_sha": csrc_hash(), "capture_shape": list(shape), "scale_to_full": scale,
           "steps_averaged": len(use), "ops": ops}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("| op | kernels | us | DRAM read MB | DRAM write MB | read+write MB (scaled to 512^3) |")
    print("|---|---|---|---|---|---|")
    for op, o in ops.items():
        print(f"| {op} | {' '.join(o['kernels'])} | {o['us']:.1f} | {o['dram_read'] / scale / 1e6:.1f}"
              f" | {o['dram_write'] / scale / 1e6:.1f} | {o['dram_bytes_per_launch'] / 1e6:.1f} |")
    print(f"step under ncu: {sum(o['us'] for o in ops.values()):.1f} us")
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples: HOSZP_CLOCK_DIR if set, else the system's temporary directory
        import tempfile

        d = os.environ.get("HOSZP_CLOCK_DIR", tempfile.gettempdir())
        self.path = os.path.join(d, f"hoszp_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Median SM clock, max clock and throttle reasons over the samples taken
        between host times t0 and t1 (datetime; all samples if not given)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        import datetime

        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if t0 is not None and not (t0 <= ts <= t1):
                    continue
                sm.append(float(parts[2].split()[0]))
                smax = max(smax, float(parts[3].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU) arm
def oracle_step(O, a: np.ndarray, b: np.ndarray):
    """One step of the hot path on the CPU oracle; returns seconds."""
    t0 = time.perf_counter()
    ca = O.compress(a, eb=REL, mode="rel")
    e = float(O.header(ca)["eps_q"])
    cb = O.compress(b, eb=e)
    O.negate(ca)
    O.add_scalar(ca, SCALAR_ADD)
    O.mul_scalar(ca, SCALAR_MUL)
    O.add(ca, cb)
    O.mean(ca)
    O.var(ca)
    O.decompress(ca)
    return time.perf_counter() - t0


def run_oracle(a, b, steps: int, warmup: int):
    import oracle as O

    O.build()
    for _ in range(warmup):
        oracle_step(O, a, b)
    ts = [oracle_step(O, a, b) for _ in range(steps)]
    return sum(ts) / len(ts)


def host_cpu():
    """Core count and CPU model of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or platform.machine()


def run_omp_baseline(a, b, reps: int = 3):
    """The oracle's arithmetic with an OpenMP loop over blocks (the paper's CPU
    design) on every host core: median seconds of `reps` steps after one warm-up."""
    import oracle as O
    from oracle import omp

    omp.build()
    oracle_step(omp_ops(O, omp), a, b)
    ts = sorted(oracle_step(omp_ops(O, omp), a, b) for _ in range(reps))
    return ts[len(ts) // 2], omp.threads()


def omp_ops(O, omp):
    """The OpenMP baseline behind the oracle's call names (header from the oracle)."""
    class _Ops:
        compress = staticmethod(omp.compress)
        header = staticmethod(O.header)
        negate = staticmethod(omp.negate)
        add_scalar = staticmethod(omp.add_scalar)
        mul_scalar = staticmethod(omp.mul_scalar)
        add = staticmethod(omp.add)
        mean = staticmethod(omp.mean)
        var = staticmethod(omp.var)
        decompress = staticmethod(omp.decompress)
    return _Ops


REF_BUDGET_S = 120.0  # the reference arm's warm-up and timed steps together


def reference_sample(A: np.ndarray, B: np.ndarray, nsteps: int) -> int:
    """Values per field for the reference arm: one oracle step on a 2^18-value
    sample gives this host's time per value, and the sample is sized so that
    `nsteps` steps take about REF_BUDGET_S seconds (between 2^16 and 2^24
    values, whole 64-value blocks)."""
    import oracle as O

    O.build()
    a, b = sample_fields(A, B, 1 << 18)
    oracle_step(O, a, b)  # first call: loads the library
    per_value = oracle_step(O, a, b) / a.size
    n = int(REF_BUDGET_S / max(nsteps, 1) / max(per_value, 1e-12))
    return max(1 << 16, min(1 << 24, n)) // 64 * 64


def sample_fields(A: np.ndarray, B: np.ndarray, n: int):
    """Bounded CPU sample: the first n values (whole 64-value blocks) of each field."""
    n = min(n, A.size) // 64 * 64
    return np.ascontiguousarray(A.reshape(-1)[:n]), np.ascontiguousarray(B.reshape(-1)[:n])


def make_fields(seed_base: int):
    import datagen

    A = datagen.grf(SHAPE, seed=seed_base + 1)
    B = datagen.grf(SHAPE, seed=seed_base + 2)
    return A, B


# ---------------------------------------------------------------- profiling mode
def profile_op(op: str, shape):
    """Runs one operator 4 times on the workload's fields, holding only the
    buffers that operator needs (for an ncu capture of its kernels)."""
    import torch

    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build as hzbuild

    hzbuild.build()
    ctx = hz.Context(0)
    A, B = make_fields(0)
    xa = torch.from_numpy(A.reshape(-1)).cuda()
    ca = hz.compress(xa, eb=REL, mode="rel", ctx=ctx)
    e = hz.header(ca)["eps_q"]
    cb = None
    if op in ("add", "cov"):
        cb = hz.compress(torch.from_numpy(B.reshape(-1)).cuda(), eb=e, ctx=ctx)
    del B
    if op not in ("compress", "decompress"):
        del xa
    torch.cuda.synchronize()
    for _ in range(4):
        if op == "compress":
            hz.compress(xa, eb=REL, mode="rel", ctx=ctx)
        elif op == "decompress":
            hz.decompress(ca, out=xa, ctx=ctx)
        elif op == "negate":
            hz.negate(ca, ctx=ctx)
        elif op == "add_scalar":
            hz.add_scalar(ca, SCALAR_ADD, ctx=ctx)
        elif op == "mul_scalar":
            hz.mul_scalar(ca, SCALAR_MUL, ctx=ctx)
        elif op == "add":
            hz.add(ca, cb, ctx=ctx)
        elif op == "mean":
            hz.mean(ca, ctx=ctx)
        elif op == "var":
            hz.var(ca, ctx=ctx)
        elif op == "cov":
            hz.cov(ca, cb, ctx=ctx)
    torch.cuda.synchronize()
    ctx.check(op)
    print(f"profile-op {op} done: stream {ca.numel()} bytes")


# ---------------------------------------------------------------- serving
SERVE_MIX = (("mean", 0.20), ("var", 0.20), ("add_scalar", 0.15), ("mul_scalar", 0.15),
             ("add", 0.20), ("decompress", 0.10))


def serving_bench(hz, xa, xb, eps_q, nfields: int, budget: int, rates, per_rate: int,
                  slots: int, seed: int = 7):
    """Poisson streams of mixed requests over `nfields` resident compressed
    fields of the workload's size (seeded rolls, scales and offsets of fields A
    and B, all at A's absolute bound so any two can be added), served by
    hoszp_server under an HBM budget that covers the resident streams too.
    Returns p50 / p99 latency (arrival to completion) and throughput per rate."""
    import torch

    rng = np.random.default_rng(seed)
    n = xa.numel()
    cap = hz.compress_bound(n)
    buf = torch.empty(cap, dtype=torch.uint8, device=xa.device)
    size = torch.zeros(1, dtype=torch.int64, device=xa.device)
    tmp = torch.empty_like(xa)
    streams = []
    for k in range(nfields):
        base = xa if k % 2 == 0 else xb
        r = int(rng.integers(1, n))
        tmp[: n - r].copy_(base[r:])
        tmp[n - r:].copy_(base[:r])
        tmp.mul_(float(rng.uniform(0.5, 2.0))).add_(float(rng.uniform(-1.0, 1.0)))
        hz.compress(tmp, eb=eps_q, out=buf, out_bytes=size, sync=False)
        streams.append(buf[: int(size.item())].clone())
    del buf, tmp
    torch.cuda.synchronize()
    resident = sum(c.numel() for c in streams)
    srv = hz.Server(xa.device.index, slots=slots, hbm_budget=budget - resident, max_n=n)
    ids = [srv.register(c) for c in streams]
    names = [m for m, _ in SERVE_MIX]
    probs = np.array([p for _, p in SERVE_MIX])
    out = {"fields": nfields, "resident_gib": resident / 2**30, "budget_gib": budget / 2**30,
           "slots": slots, "mix": dict(SERVE_MIX), "requests_per_rate": per_rate, "rates": []}
    for rate in rates:
        ops = rng.choice(len(names), size=per_rate, p=probs)
        gaps = rng.exponential(1e6 / rate, per_rate)
        t0 = srv.now_us() + 5000
        arr = t0 + np.cumsum(gaps).astype(np.int64)
        orig = 0
        for i in range(per_rate):
            op = names[ops[i]]
            a, b = int(rng.integers(nfields)), int(rng.integers(nfields))
            orig += (2 if op == "add" else 1) * 4 * n
            srv.submit(op, ids[a], ids[b], 0.5 if op == "add_scalar" else 3.14, tag=i,
                       arrival_us=int(arr[i]))
        lat, done_t, errs = [], [], 0
        deadline = time.time() + 120
        while len(lat) < per_rate and time.time() < deadline:
            for c in srv.poll(256, wait_us=20000):
                if c["status"] != 0:
                    errs += 1
                srv.release(c)
                lat.append((c["done_us"] - c["arrival_us"]) / 1e3)
                done_t.append(c["done_us"])
        span_s = (max(done_t) - t0) / 1e6 if done_t else float("nan")
        out["rates"].append({"offered_req_s": rate, "completed": len(lat), "errors": errs,
                             "p50_ms": float(np.percentile(lat, 50)) if lat else None,
                             "p99_ms": float(np.percentile(lat, 99)) if lat else None,
                             "served_req_s": len(lat) / span_s, "orig_gbs": orig / span_s / 1e9})
    st = srv.stats()
    out["max_in_flight"] = st["max_in_flight"]
    out["arena_peak_gib"] = st["arena_peak"] / 2**30
    srv.close()
    del streams
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- batched
def batched_pools(device, seed: int = 3):
    """The batched workload's value pools: a 1-D sines signal with constant runs,
    a 2-D and a 3-D Gaussian random field, about 1e7 values each (the kinds of
    datagen.field_set_batched); every field is a seeded slice of its kind's pool."""
    import torch

    import datagen

    pools = {1: datagen.sines_1d(10_000_000, seed=seed, const_frac=0.1),
             2: datagen.grf((3163, 3163), seed=seed + 1).reshape(-1),
             3: datagen.grf((216, 216, 216), seed=seed + 2).reshape(-1)}
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in pools.items()}


def _timed(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_bench(hz, device, nfields: int, seed: int = 3, reps: int = 3):
    """One snapshot of `nfields` uneven fields: sizes log-uniform in 1e4..1e7
    values, relative bounds log-uniform in 1e-5..1e-2 and a 1-D/2-D/3-D kind per
    field (datagen.field_set_batched), each field a seeded slice of its kind's
    pool, compressed and kept resident. Every batched operator (one launch over
    all fields, plus a scan and a placement for the producing ones) is timed
    against the same operator called field by field, and the results of both
    are compared."""
    import torch

    import datagen

    specs, _ = datagen.field_set_batched(nfields, seed=seed)
    pools = batched_pools(device, seed)
    rng = np.random.default_rng(seed + 7)
    xs, xbs, rels = [], [], []
    for n, rel, kind in specs:
        pool = pools[kind]
        o1 = int(rng.integers(0, (pool.numel() - n) // 4 + 1)) * 4  # 16-byte aligned slices
        o2 = int(rng.integers(0, (pool.numel() - n) // 4 + 1)) * 4
        xs.append(pool[o1:o1 + n])
        xbs.append(pool[o2:o2 + n])
        rels.append(rel)
    sizes = np.array([n for n, _, _ in specs], np.int64)
    orig = 4 * int(sizes.sum())
    out = {"fields": nfields, "values": int(sizes.sum()),
           "recipe": "datagen.field_set_batched sizes, bounds and kinds; values are seeded "
                     "slices of a 1e7-value pool per kind"}
    # resident streams: A at its relative bound, B at A's absolute bound (for A + B)
    ca = hz.batch_compress(xs, rels, mode="rel")
    eqs = [float(hz.header(c)["eps_q"]) for c in ca]
    cb = hz.batch_compress(xbs, eqs, mode="abs")
    cbytes = sum(c.numel() for c in ca)
    out["compressed_gb"] = cbytes / 1e9
    peak = measured_peak()[0]
    bA, bB = hz.Batch(ca), hz.Batch(cb)
    res = torch.empty(nfields, dtype=torch.float64, device=device)
    per = torch.empty(nfields, dtype=torch.float64, device=device)
    offs = np.concatenate([[0], np.cumsum((sizes + 3) // 4 * 4)])
    big = torch.empty(int(offs[-1]), dtype=torch.float32, device=device)
    douts = [big[int(offs[i]):int(offs[i]) + int(sizes[i])] for i in range(nfields)]

    # the untuned shape (super-tile pipeline, 8 warps per block group, any rate)
    # against the autotuner's pick, which is then kept for the timings below
    def default_index(op):
        for i in range(bA.shapes(op)):
            bA.set_shape(op, i)
            c = bA.config(op)
            if c["warps_per_group"] == 8 and c["plane_groups"] == 4 and c["stages"] == 4:
                return i
        raise SystemExit("no default batched shape")
    runs = {0: lambda: bA.mean(out=res, sync=False), 1: lambda: bA.var(out=res, sync=False),
            2: lambda: bA.decompress(douts, sync=False)}
    untuned = {}
    for op, fn in runs.items():
        bA.set_shape(op, default_index(op))
        untuned[op] = _timed(fn, reps)
    t0 = time.perf_counter()
    picks = bA.tune(outs=douts)
    out["autotune"] = {"seconds": time.perf_counter() - t0, "picks": picks,
                       "shapes_tried": {o: bA.shapes(i) for i, o in enumerate(bA.OPS)}}
    for name, bfn, sfn in (("mean", bA.mean, hz.mean), ("var", bA.var, hz.var)):
        bms = _timed(lambda: bfn(out=res, sync=False), reps)

        def fields():
            for i, c in enumerate(ca):
                sfn(c, out=per[i:i + 1], sync=False)
        fms = _timed(fields, 1)
        bA.check(name)
        out[name] = {"batched_ms": bms, "untuned_ms": untuned[0 if name == "mean" else 1],
                     "per_field_ms": fms, "speedup": fms / bms,
                     "batched_orig_gbs": orig / bms / 1e6,
                     "batched_frac_of_measured_hbm": cbytes / bms / 1e6 / peak,
                     "identical_to_per_field": bool(torch.equal(res, per))}
    # decompression into one float arena
    bms = _timed(lambda: bA.decompress(douts, sync=False), reps)
    bA.check("decompress")
    first = big.clone()

    def dfields():
        for i, c in enumerate(ca):
            hz.decompress(c, out=douts[i], check=False)
    fms = _timed(dfields, 1)
    out["decompress"] = {"batched_ms": bms, "untuned_ms": untuned[2], "per_field_ms": fms,
                         "speedup": fms / bms,
                         "batched_orig_gbs": orig / bms / 1e6,
                         "batched_frac_of_measured_hbm": (cbytes + orig) / bms / 1e6 / peak,
                         "identical_to_per_field": bool(torch.equal(first, big))}
    del big, first, douts
    # producing operators: outputs in one arena per arm, compared byte for byte
    bounds = [hz.compress_bound(int(n)) for n in sizes]
    boffs = np.concatenate([[0], np.cumsum([(b + 255) // 256 * 256 for b in bounds])])

    def arena():
        buf = torch.empty(int(boffs[-1]), dtype=torch.uint8, device=device)
        return buf, [buf[int(boffs[i]):int(boffs[i]) + bounds[i]] for i in range(nfields)]

    a1, o1 = arena()
    a2, o2 = arena()
    sz1 = torch.zeros(nfields, dtype=torch.int64, device=device)
    cases = (
        ("mul_scalar", lambda: bA.mul_scalar(SCALAR_MUL, outs=o1, sync=False),
         lambda i: hz.mul_scalar(ca[i], SCALAR_MUL, out=o2[i], out_bytes=sz1[i:i + 1],
                                 sync=False), cbytes),
        ("add", lambda: bA.add(bB, outs=o1, sync=False),
         lambda i: hz.add(ca[i], cb[i], out=o2[i], out_bytes=sz1[i:i + 1], sync=False),
         cbytes + sum(c.numel() for c in cb)),
        ("compress", lambda: hz.batch_compress(xs, rels, mode="rel", outs=o1, sync=False),
         lambda i: hz.compress(xs[i], eb=rels[i], mode="rel", out=o2[i],
                               out_bytes=sz1[i:i + 1], sync=False), orig),
    )
    for name, bfn, sfn, in_bytes in cases:
        holder = {}

        def run_b():
            holder["r"] = bfn()
        bms = _timed(run_b, reps)
        sizes_b = holder["r"][1]

        def run_f():
            for i in range(nfields):
                sfn(i)
        fms = _timed(run_f, 1)
        same = bool(torch.equal(sizes_b, sz1))
        if same:
            nb = sizes_b.cpu().tolist()
            same = all(torch.equal(o1[i][:nb[i]], o2[i][:nb[i]]) for i in range(nfields))
        out_bytes = int(sizes_b.sum().item())
        out[name] = {"batched_ms": bms, "per_field_ms": fms, "speedup": fms / bms,
                     "batched_orig_gbs": orig / bms / 1e6,
                     "batched_frac_of_measured_hbm": (in_bytes + out_bytes) / bms / 1e6 / peak,
                     "identical_to_per_field": same}
    bA.close()
    bB.close()
    del a1, a2, o1, o2, ca, cb, pools, xs, xbs
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hoszp", choices=["hoszp", "reference"])
    ap.add_argument("--oracle-sample", type=int, default=None,
                    help="values per field in the CPU oracle sample (default: 2^24 for the "
                         "cpu_baseline leg; for --impl reference, sized so that its warm-up "
                         "and timed steps take about two minutes together)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched measurement")
    ap.add_argument("--batch-fields", type=int, default=4096)
    ap.add_argument("--serve-fields", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=1000, help="requests per offered rate")
    ap.add_argument("--shape", type=int, nargs=3, default=list(DEFAULT_SHAPE),
                    help="field shape (smaller cases are for profiling, not bench lines)")
    ap.add_argument("--profile-op", default=None,
                    choices=["compress", "decompress", "negate", "add_scalar", "mul_scalar", "add",
                             "mean", "var", "cov"],
                    help="run only this operator 4 times (for ncu captures; prints no bench line)")
    ap.add_argument("--traffic-from", default=None, metavar="CSV",
                    help="summarise an ncu launch list of the step (captured at --shape) into "
                         "profiles/traffic.json; needs no GPU")
    args = ap.parse_args()
    global SHAPE
    SHAPE = tuple(args.shape)
    if args.traffic_from:
        traffic_from_csv(args.traffic_from, SHAPE)
        return
    if args.profile_op:
        if args.impl != "hoszp":
            raise SystemExit("--profile-op runs the library only")
    warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    n = int(np.prod(SHAPE))
    config = {"workload": "grf3d_%dx%dx%d_rel1e-4_fieldsAB" % SHAPE, "shape": list(SHAPE), "n": n,
              "rel_eb": REL, "spectrum": "E(k)~k^-5/3", "fields": 2,
              "ops": ["compress A", "compress B", "negate", "add_scalar 0.5", "mul_scalar 3.14",
                      "add A+B", "mean", "var", "decompress"],
              "l2": "no flush: each field is 512 MiB and each stream > L2 (129 MB)",
              "parallelism": f"replica{world}"}

    if args.impl == "reference":
        # the reference arm is the oracle, as it stands, on the host cores
        if rank != 0:
            return
        A, B = make_fields(0)
        n_s = args.oracle_sample or reference_sample(A, B, args.steps + args.warmup)
        a, b = sample_fields(A, B, n_s)
        sec = run_oracle(a, b, args.steps, args.warmup)
        val = 40.0 * a.size / sec / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": f"first {a.size} values of each 512^3 field, one step of all rows"},
                "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    if args.profile_op:
        profile_op(args.profile_op, tuple(args.shape))
        return

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build as hzbuild

    hzbuild.build()
    hz.load_library()
    ctx = hz.Context(dev.index)
    ctx.reserve(n)
    stream = torch.cuda.current_stream(dev)

    A, B = make_fields(1000 * rank)
    xa = torch.from_numpy(A.reshape(-1)).to(dev)
    xb = torch.from_numpy(B.reshape(-1)).to(dev)
    cap = hz.compress_bound(n)
    bufs = {k: torch.empty(cap, dtype=torch.uint8, device=dev)
            for k in ("ca", "cb", "neg", "adds", "mul", "sum")}
    sizes = {k: torch.zeros(1, dtype=torch.int64, device=dev) for k in bufs}
    res = torch.zeros(2, dtype=torch.float64, device=dev)
    xr = torch.empty(n, dtype=torch.float32, device=dev)

    # first compression on the host's schedule: A's bound, used for B as well
    ca = hz.compress(xa, eb=REL, mode="rel", ctx=ctx)
    eps_q = hz.header(ca)["eps_q"]
    cb = hz.compress(xb, eb=eps_q, ctx=ctx)
    C = {"ca": ca.numel(), "cb": cb.numel()}
    for k, src in (("neg", hz.negate), ("adds", lambda c, **kw: hz.add_scalar(c, SCALAR_ADD, **kw)),
                   ("mul", lambda c, **kw: hz.mul_scalar(c, SCALAR_MUL, **kw))):
        C[k] = src(ca, ctx=ctx).numel()
    C["sum"] = hz.add(ca, cb, ctx=ctx).numel()

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ops = ["compress A", "compress B", "negate", "add_scalar", "mul_scalar", "add", "mean", "var",
           "decompress"]

    def step(record=None, io=None):
        """One pass of the path; io = (field A, field B, decompressed output,
        the two reductions) on the device, by default the benchmark's own."""
        xa_, xb_, xr_, res_ = io if io is not None else (xa, xb, xr, res)

        def mark(i):
            if record is not None:
                record[i].record(stream)

        ca_b, cb_b = bufs["ca"], bufs["cb"]
        mark(0)
        hz.compress(xa_, eb=REL, mode="rel", out=ca_b, out_bytes=sizes["ca"], ctx=ctx, sync=False)
        mark(1)
        hz.compress(xb_, eb=eps_q, out=cb_b, out_bytes=sizes["cb"], ctx=ctx, sync=False)
        mark(2)
        sa, sb = ca_b[:C["ca"]], cb_b[:C["cb"]]
        hz.negate(sa, out=bufs["neg"], out_bytes=sizes["neg"], ctx=ctx, sync=False)
        mark(3)
        hz.add_scalar(sa, SCALAR_ADD, out=bufs["adds"], out_bytes=sizes["adds"], ctx=ctx,
                      sync=False)
        mark(4)
        hz.mul_scalar(sa, SCALAR_MUL, out=bufs["mul"], out_bytes=sizes["mul"], ctx=ctx, sync=False)
        mark(5)
        hz.add(sa, sb, out=bufs["sum"], out_bytes=sizes["sum"], ctx=ctx, sync=False)
        mark(6)
        hz.mean(sa, out=res_[0:1], ctx=ctx, sync=False)
        mark(7)
        hz.var(sa, out=res_[1:2], ctx=ctx, sync=False)
        mark(8)
        hz.decompress(sa, n=n, out=xr_, ctx=ctx, check=False)
        mark(9)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.check("warmup")

    K = args.steps
    marks = [[ev() for _ in range(10)] for _ in range(K)]
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = ev(), ev()
    import datetime

    h0 = datetime.datetime.now()
    t_start.record(stream)
    for k in range(K):
        step(marks[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    h1 = datetime.datetime.now()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop(h0, h1)
    ctx.check("timed steps")
    total_ms = t_start.elapsed_time(t_end)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / K
    per_op_ms = {op: statistics.mean(marks[k][i].elapsed_time(marks[k][i + 1]) for k in range(K))
                 for i, op in enumerate(ops)}

    # algorithmic bytes per operator (reads + writes the operator must make)
    N4 = 4 * n
    alg = {"compress A": 2 * N4 + C["ca"], "compress B": N4 + C["cb"], "negate": 2 * C["ca"],
           "add_scalar": 2 * C["ca"], "mul_scalar": C["ca"] + C["mul"],
           "add": C["ca"] + C["cb"] + C["sum"], "mean": C["ca"], "var": C["ca"],
           "decompress": C["ca"] + N4}
    orig = {op: N4 for op in ops}
    orig["add"] = 2 * N4
    peak, peak_kind = measured_peak()
    per_op = {}
    for op in ops:
        ms = per_op_ms[op]
        per_op[op] = {"ms": round(ms, 4), "orig_gbs": orig[op] / ms / 1e6,
                      "alg_gbs": alg[op] / ms / 1e6, "frac_of_measured_hbm": alg[op] / ms / 1e6 / peak}

    # GPU decompress -> op -> recompress comparator (same kernels, not fused)
    base = {}
    tmp1 = torch.empty(n, dtype=torch.float32, device=dev)
    tmp2 = torch.empty(n, dtype=torch.float32, device=dev)
    tmp3 = torch.empty(n, dtype=torch.float32, device=dev)
    outb = torch.empty(cap, dtype=torch.uint8, device=dev)
    outs = torch.zeros(1, dtype=torch.int64, device=dev)
    sa, sb = bufs["ca"][:C["ca"]], bufs["cb"][:C["cb"]]

    def trad(op):
        hz.decompress(sa, n=n, out=tmp1, ctx=ctx, check=False)
        if op == "negate":
            hz.fop_axpb(tmp1, -1.0, 0.0, out=tmp2)
        elif op == "add_scalar":
            hz.fop_axpb(tmp1, 1.0, SCALAR_ADD, out=tmp2)
        elif op == "mul_scalar":
            hz.fop_axpb(tmp1, SCALAR_MUL, 0.0, out=tmp2)
        elif op == "add":
            hz.decompress(sb, n=n, out=tmp3, ctx=ctx, check=False)
            hz.fop_add(tmp1, tmp3, out=tmp2)
        elif op in ("mean", "var"):
            hz.fop_moments(tmp1, op == "var", out=res[0:1], ctx=ctx)
            return
        hz.compress(tmp2, eb=eps_q, out=outb, out_bytes=outs, ctx=ctx, sync=False)

    def homo(op):  # the homomorphic operator alone, timed the way trad() is
        if op == "negate":
            hz.negate(sa, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "add_scalar":
            hz.add_scalar(sa, SCALAR_ADD, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "mul_scalar":
            hz.mul_scalar(sa, SCALAR_MUL, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "add":
            hz.add(sa, sb, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "mean":
            hz.mean(sa, out=res[0:1], ctx=ctx, sync=False)
        elif op == "var":
            hz.var(sa, out=res[1:2], ctx=ctx, sync=False)

    def alone(fn, op, reps=5):
        for _ in range(2):
            fn(op)
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            fn(op)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for op in ("negate", "add_scalar", "mul_scalar", "add", "mean", "var"):
        tms = alone(trad, op)
        hms = alone(homo, op)
        # speedup: both workflows timed alone, back to back on the same stream;
        # in_step: against the operator's share of the benchmark step (which also
        # carries the write-back of the previous operator's output)
        base[op] = {"ms": round(tms, 4), "homomorphic_alone_ms": round(hms, 4),
                    "homomorphic_alone_frac_of_measured_hbm": alg[op] / hms / 1e6 / peak,
                    "speedup_homomorphic": tms / hms, "speedup_in_step": tms / per_op_ms[op]}
    ctx.check("baseline")

    # operators outside the step (Sec. V-A scalar subtraction, Sec. V-B standard
    # deviation and block-wise means, Sec. V-D covariance), each timed alone;
    # algorithmic bytes: what the operator must read and write
    nbk = (n + 63) // 64
    bmeans = torch.empty(nbk, dtype=torch.float64, device=dev)

    def xop(op):
        if op == "sub_scalar":
            hz.sub_scalar(sa, SCALAR_ADD, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "std":
            hz.std(sa, out=res[0:1], ctx=ctx, sync=False)
        elif op == "block_means":
            hz.block_means(sa, out=bmeans, ctx=ctx, sync=False)
        elif op == "cov":
            hz.cov(sa, sb, out=res[1:2], ctx=ctx, sync=False)
        elif op == "mul_scalar_exact":
            hz.mul_scalar_exact(sa, SCALAR_MUL, out=outb, out_bytes=outs, ctx=ctx, sync=False)
        elif op == "hadamard":
            hz.hadamard(sa, sb, out=outb, out_bytes=outs, scratch=qscratch, ctx=ctx, sync=False)

    # covariance reads A and B once (one pass, exact sums)
    xalg = {"sub_scalar": 2 * C["ca"], "std": C["ca"], "block_means": C["ca"] + 8 * nbk,
            "cov": C["ca"] + C["cb"], "mul_scalar_exact": None, "hadamard": None}
    qscratch = torch.empty(n, dtype=torch.int32, device=dev)  # B's integers (Hadamard product)
    extra = {}
    for op, nbytes in xalg.items():
        for _ in range(3):
            xop(op)
        e0, e1 = ev(), ev()
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            xop(op)
        e1.record(stream)
        torch.cuda.synchronize()
        xms = e0.elapsed_time(e1) / reps
        if nbytes is None:  # a produced stream: inputs plus the output's size
            nbytes = C["ca"] + (C["cb"] if op == "hadamard" else 0) + int(outs.item())
        extra[op] = {"ms": round(xms, 4),
                     "orig_gbs": (2 if op in ("cov", "hadamard") else 1) * N4 / xms / 1e6,
                     "alg_gbs": nbytes / xms / 1e6, "frac_of_measured_hbm": nbytes / xms / 1e6 / peak}
    ctx.check("operators outside the step")

    # compression ratio (Sec. VI-B3, Table 8): this layout stores no per-block
    # lengths; an SZp-style layout would add one 2-byte length per block
    # (a block's words are at most 264 bytes)
    cr = {"hoszp": N4 / C["ca"], "szp_style_per_block_lengths": N4 / (C["ca"] + 2 * nbk),
          "field": "A"}

    # roofline of the dominant operator (largest share of the step)
    dom = max(ops, key=lambda o: per_op_ms[o])
    kern_of = {"compress A": "k_compress", "compress B": "k_compress", "negate": "k_meta",
               "add_scalar": "k_meta", "mul_scalar": "k_mul_lanes", "add": "k_add",
               "mean": "k_mean", "var": "k_var", "decompress": "k_decompress_lanes"}
    achieved = alg[dom] / per_op_ms[dom] / 1e6
    tr = ncu_traffic(dom)
    roofline = {"bound": "hbm", "op": dom, "kernel": kern_of[dom], "achieved": achieved,
                "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                "frac": achieved / peak, "alg_bytes_per_launch": alg[dom],
                "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                "traffic_kernels": (tr["kernels"] if tr else None)}

    # end to end through host memory: pinned inputs in, results out, every step.
    # Serial: upload, step, download, one after the other. Pipelined: two
    # slots of device buffers; step k's download runs while step k+1's inputs
    # upload (the host link is full duplex) and step k+1 computes once they
    # have landed. Every step still moves all of its bytes inside the timed
    # region; events keep a slot from being reused before its step has read
    # its inputs and its results are back on the host.
    e2e = None
    if rank == 0 or world > 1:
        ha = torch.from_numpy(A.reshape(-1)).pin_memory()
        hb = torch.from_numpy(B.reshape(-1)).pin_memory()
        hout = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
        hres = [torch.empty(2, dtype=torch.float64).pin_memory() for _ in range(2)]
        slots = [(xa, xb, xr, res), (torch.empty_like(xa), torch.empty_like(xb),
                                     torch.empty_like(xr), torch.empty_like(res))]
        s_in = torch.cuda.Stream(device=dev)
        s_out = torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_back = [torch.cuda.Event() for _ in range(2)]

        def e2e_serial():
            xa.copy_(ha, non_blocking=True)
            xb.copy_(hb, non_blocking=True)
            step()
            hout[0].copy_(xr, non_blocking=True)
            hres[0].copy_(res, non_blocking=True)

        def e2e_pipelined(steps):
            s_in.wait_stream(stream)
            for k in range(steps):
                sl = k & 1
                a_, b_, r_, q_ = slots[sl]
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(ev_used[sl])  # step k-2 has read this slot's inputs
                    a_.copy_(ha, non_blocking=True)
                    b_.copy_(hb, non_blocking=True)
                    ev_in[sl].record(s_in)
                stream.wait_event(ev_in[sl])
                if k >= 2:
                    stream.wait_event(ev_back[sl])  # step k-2's results are on the host
                step(io=slots[sl])
                ev_used[sl].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_used[sl])
                    hout[sl].copy_(r_, non_blocking=True)
                    hres[sl].copy_(q_, non_blocking=True)
                    ev_back[sl].record(s_out)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)

        def timed(fn, steps):
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            fn(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            if dist is not None:
                t = torch.tensor([ms], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ms = float(t.item())
            return ms

        def serial_steps(steps):
            for _ in range(steps):
                e2e_serial()

        e2e_serial()
        e2e_pipelined(2)
        torch.cuda.synchronize()
        E = max(4, min(K, 20))
        s_ms = timed(serial_steps, E)
        ref_out, ref_res = hout[0].clone(), hres[0].clone()
        p_ms = timed(e2e_pipelined, E)
        # both slots of the pipeline give the serial results (same inputs, deterministic path)
        for sl in range(2):
            if not (torch.equal(hout[sl], ref_out) and torch.equal(hres[sl], ref_res)):
                raise SystemExit("pipelined end-to-end results differ from the serial ones")
        e2e = {"value": world * 40.0 * n / p_ms / 1e6, "unit": "GB/s",
               "h2d_bytes_per_step": 2 * N4, "d2h_bytes_per_step": N4 + 16, "ms_per_step": p_ms,
               "steps": E, "overlap": "double-buffered: step k's download with step k+1's upload",
               "serial": {"value": world * 40.0 * n / s_ms / 1e6, "ms_per_step": s_ms}}
    ctx.check("e2e")

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    batched = None
    if world == 1 and not args.no_batched:
        batched = batched_bench(hz, xa.device, args.batch_fields)

    serving = None
    if world == 1 and not args.no_serving:
        del tmp1, tmp2, tmp3, outb
        torch.cuda.empty_cache()
        serving = serving_bench(hz, xa, xb, eps_q, args.serve_fields, 120 << 30,
                                (200, 2000, 5000, 10000, 20000), args.serve_requests, slots=8)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        a, b = sample_fields(A, B, args.oracle_sample or (1 << 24))
        sec = run_oracle(a, b, 1, 0)
        cores, model = host_cpu()
        cpu = {"value": 40.0 * a.size / sec / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {a.size} values of fields A and B, one step of all rows",
               "seconds": sec, "host": {"nproc": cores, "cpu_model": model}}
        try:
            osec, threads = run_omp_baseline(a, b)
            cpu["all_cores"] = {
                "value": 40.0 * a.size / osec / 1e9, "unit": "GB/s", "cores": threads,
                "kind": "oracle arithmetic + OpenMP loop over blocks (the paper's CPU design)",
                "sample": "the same sample, median of 3 steps", "seconds": osec}
        except (OSError, subprocess.CalledProcessError) as ex:  # no OpenMP toolchain
            cpu["all_cores"] = {"unavailable": f"OpenMP build failed: {ex}"}

    value = world * 40.0 * n / ms_step / 1e6
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": config,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": KERNELS_PER_STEP * K, "clocks": clocks,
            "compressed_bytes": C, "per_op": per_op, "decompress_op_recompress": base,
            "extra_ops": extra, "compression_ratio": cr,
            "batched": batched, "serving": serving}
    print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
