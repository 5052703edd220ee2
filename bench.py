#!/usr/bin/env python3
"""Benchmark of the B300 interleaved rANS coder.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload chunked]
                    [--impl ours|reference]

Workload "chunked": 1 GiB of i.i.d. bytes, Zipf(s=1.1) over 256 symbols, a
static model quantized to M = 2^12, 16384 chunks of 64 KiB, 32 interleaved
coders per chunk.  One step is the whole hot path over that batch: encode
(coder kernel, offset-table scan, chunk packing) and then decode.  The
headline value is decoded GB/s (raw bytes out of the decode phase per
second); encode GB/s is reported beside it.  Inputs are resident in HBM when
the timed region starts and are larger than L2, so no flush is needed.

Under torchrun every rank codes its own batch (the chunks are independent,
so the path shards with no data exchange: weak scaling); rank 0 prints one
JSON line with the whole-job value and the max-over-ranks time.

--impl reference times the CPU oracle (the plain scalar C implementation the
tests compare against) on the host cores, on bounded samples of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1402_3392_b300 import workloads as wl  # noqa: E402

DECODE_SOURCES = [os.path.join(ROOT, "paper_1402_3392_b300", "csrc", f)
                  for f in ("rans_decode.cu", "decode_core.cuh", "device_util.cuh")]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "decode_kernel_chunked.md")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="chunked", choices=["chunked", "single"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true",
                    help="run the timed region without the clock sampler")
    ap.add_argument("--symbols", type=int, default=0,
                    help="override the workload's symbol count (small profiling cases)")
    ap.add_argument("--legs",
                    default="batched,binary,single,serving,bypass,bytes,adaptive,adaptive_n,"
                            "prefix,wide",
                    help="extra legs after the headline one: comma list of batched, binary, "
                         "single, serving, bypass, bytes, adaptive, adaptive_n, prefix, wide, "
                         "none")
    ap.add_argument("--serving-requests", type=int, default=5000)
    ap.add_argument("--batched-streams", type=int, default=0,
                    help="override the batched workload's stream count")
    ap.add_argument("--batched-layout", default="",
                    help="N,chunk_symbols,policy for the batched leg instead of the "
                         "autotuner's choice (e.g. 32,16384,fill)")
    ap.add_argument("--binary-layout", default="",
                    help="chunk_symbols,policy for the binary leg instead of the autotuner's "
                         "choice (e.g. 16384,fixed)")
    return ap.parse_args(argv)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the decoder's source code with comments and blank lines
    removed, so that a profile stays attached to the code it measured."""
    h = hashlib.sha256()
    for path in DECODE_SOURCES:
        with open(path) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per decode launch from the committed ncu summary, or None
    if there is none or the kernel source changed since it was captured."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"decode_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


class _Nvml:
    """The few NVML queries the clock sampler needs, called through ctypes on
    the driver's libnvidia-ml (read only: clocks and clock-event reasons)."""

    NVML_CLOCK_SM = 1

    def __init__(self, uuid: str):
        import ctypes

        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 returned {rc}")
        self.h = ctypes.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetHandleByUUID({uuid}) returned {rc}")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def max_sm_mhz(self):
        v = self.C.c_uint()
        rc = self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.NVML_CLOCK_SM, self.C.byref(v))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetMaxClockInfo returned {rc}")
        return int(v.value)

    def sample(self):
        mhz, bits = self.C.c_uint(), self.C.c_ulonglong()
        rc = self.lib.nvmlDeviceGetClockInfo(self.h, self.NVML_CLOCK_SM, self.C.byref(mhz))
        rc2 = self.reasons_fn(self.h, self.C.byref(bits))
        if rc or rc2:
            raise RuntimeError(f"nvml sample returned {rc}/{rc2}")
        return int(mhz.value), int(bits.value)


class ClockSampler:
    """Samples the SM clock and the clock-event reasons (read only) while the
    timed region runs: NVML in this process (the driver's libnvidia-ml through
    ctypes), else an `nvidia-smi -lms` child.  Either is started and has
    delivered its first sample before the timed region begins (an
    nvidia-smi started inside it was seen to hold up the region's CUDA calls
    for seconds), and only samples taken between mark_start() and
    mark_stop() are summarised."""

    REASONS = {
        0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
        0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
        0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
        0x100: "display_clock_setting",
    }
    SMI_FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
                  "clocks_event_reasons.hw_thermal_slowdown",
                  "clocks_event_reasons.sw_thermal_slowdown",
                  "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        import torch

        self.samples = []          # (time, MHz, reasons)
        self.max_mhz, self.mode, self.errors = None, None, []
        self.t_start = self.t_stop = None
        props = torch.cuda.get_device_properties(device_index)
        uuid = str(getattr(props, "uuid", ""))
        self.uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        self.pci = None
        if hasattr(props, "pci_bus_id"):
            self.pci = (int(getattr(props, "pci_domain_id", 0)), int(props.pci_bus_id),
                        int(getattr(props, "pci_device_id", 0)))
        self._stop = threading.Event()
        self._first = threading.Event()
        try:
            self.nv = _Nvml(self.uuid)
            self.max_mhz = self.nv.max_sm_mhz()
            self.mode = "nvml"
        except Exception as e:  # noqa: BLE001
            self.errors.append(f"nvml: {e!r}"[:160])
            self.mode = "nvidia-smi"

    def _record(self, mhz, reasons):
        self.samples.append((time.perf_counter(), float(mhz), frozenset(reasons)))
        self._first.set()

    def _run_nvml(self):
        nv = self.nv
        while not self._stop.is_set():
            try:
                mhz, bits = nv.sample()
                self._record(mhz, {n for b, n in self.REASONS.items() if bits & b})
            except Exception as e:  # noqa: BLE001
                if len(self.errors) < 4:
                    self.errors.append(f"nvml sample: {e!r}"[:160])
            time.sleep(0.005)

    def _run_smi(self):
        for line in self.proc.stdout:
            f = [v.strip() for v in line.split(",")]
            if len(f) != len(self.SMI_FIELDS):
                continue
            try:
                mhz = float(f[0])
                self.max_mhz = float(f[1])
            except ValueError:
                continue
            names = {n for n, v in zip(("hw_slowdown", "hw_thermal_slowdown",
                                        "sw_thermal_slowdown", "sw_power_cap"), f[2:])
                     if v.lower() == "active"}
            self._record(mhz, names)

    def start(self, wait_s: float = 15.0):
        """Start sampling and wait (bounded) for the first sample."""
        import subprocess

        if self.mode == "nvml":
            self.t = threading.Thread(target=self._run_nvml, daemon=True)
        else:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.uuid}",
                     "--query-gpu=" + ",".join(self.SMI_FIELDS),
                     "--format=csv,noheader,nounits", "-lms", "20"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception as e:  # noqa: BLE001
                self.errors.append(f"nvidia-smi: {e!r}"[:160])
                self.proc = None
                return self
            self.t = threading.Thread(target=self._run_smi, daemon=True)
        self.t.start()
        if not self._first.wait(wait_s):
            self.errors.append(f"no sample within {wait_s} s")
        return self

    def mark_start(self):
        self.t_start = time.perf_counter()

    def mark_stop(self):
        self.t_stop = time.perf_counter()

    def stop(self):
        self._stop.set()
        if self.mode != "nvml" and getattr(self, "proc", None) is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=10)
            except Exception:  # noqa: BLE001
                self.proc.kill()
        if getattr(self, "t", None) is not None:
            self.t.join(timeout=10)

    def summary(self):
        a = self.t_start if self.t_start is not None else -1e300
        b = self.t_stop if self.t_stop is not None else 1e300
        inside = [s for s in self.samples if a <= s[0] <= b]
        # a region shorter than the sampling period: the samples nearest to it
        if not inside and self.samples:
            inside = sorted(self.samples, key=lambda s: min(abs(s[0] - a), abs(s[0] - b)))[:2]
        reasons = set().union(*(s[2] for s in inside)) if inside else set()
        names = sorted(r for r in reasons if r != "gpu_idle")
        out = {"sm_mhz": statistics.median(s[1] for s in inside) if inside else None,
               "sm_max_mhz": self.max_mhz, "reasons": names, "samples": len(inside),
               "source": self.mode}
        if self.errors:
            out["errors"] = self.errors[:4]
        return out


# ---------------------------------------------------------------------------
# CPU oracle legs (the only places bench.py runs oracle/)
# ---------------------------------------------------------------------------

def oracle_decode_rate(chunks, freq, N, CS, threads, repeats=1):
    """Decode the given chunks with the CPU oracle on `threads` host threads;
    returns (decoded bytes per second, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    orc = oracle.default()

    def work(ch):
        orc.decode_chunk(ch, CS, freq, N=N)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for _ in range(repeats):
            list(ex.map(work, chunks))
    dt = time.perf_counter() - t0
    return len(chunks) * CS * repeats / dt, dt


def _oracle():
    import oracle

    return oracle.default()


def host_chunks(msg_dev, n_chunks: int, k: int):
    """The first k chunks of a message in device memory, as host arrays."""
    k = min(k, n_chunks)
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = msg_dev[32:32 + 4 * (k + 1)].cpu().numpy().view(np.uint32).astype(np.int64)
    data = msg_dev[data0:data0 + int(offs[k])].cpu().numpy()
    return [data[offs[c]:offs[c + 1]] for c in range(k)]


def oracle_leg_baseline(decode_one, chunks, symbols_per_chunk, unit_bytes=True):
    """The CPU oracle beside a leg: decode_one(chunk) over a bounded sample of
    the leg's own chunks on the host threads."""
    from concurrent.futures import ThreadPoolExecutor

    cores = host_cores()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(decode_one, chunks))
    dt = time.perf_counter() - t0
    rate = len(chunks) * symbols_per_chunk / dt / 1e9
    return {"value": rate, "unit": "GB/s" if unit_bytes else "G symbols/s", "cores": cores,
            "kind": "oracle",
            "sample": f"oracle decode of the leg's first {len(chunks)} chunks x "
                      f"{symbols_per_chunk} symbols on {cores} threads, {dt:.2f} s"}


def split_chunks(msg: np.ndarray, n_chunks: int):
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = msg[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)
    return [msg[data0 + offs[c]:data0 + offs[c + 1]] for c in range(n_chunks)]


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    cfg = wl.WORKLOADS[args.workload]
    N, CS = cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    orc = oracle.default()
    freq = orc.quantize(wl.weights_from_probs(p))
    cores = host_cores()
    per_step = max(1, min(cores * 2, 256))  # chunks decoded per step
    n = per_step * CS
    sym = wl.iid_symbols(wl.rng_for(args.workload), p, n)
    msg = orc.encode_message(sym, freq, N=N, chunk_symbols=CS)
    chunks = split_chunks(msg, per_step)
    for _ in range(args.warmup):
        oracle_decode_rate(chunks[:cores], freq, N, CS, cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_decode_rate(chunks, freq, N, CS, cores)
        times.append(dt)
    gbs = n * len(times) / sum(times) / 1e9
    sample = (f"{per_step} chunks x {CS} symbols of the {args.workload} workload per step, "
              f"oracle decode, {cores} threads")
    line = {
        "impl": "reference", "metric": "decoded GB/s", "value": gbs, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args.workload, 1),
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name, world, n_symbols=None):
    cfg = wl.WORKLOADS[name]
    d = {"workload": name, "n_symbols": n_symbols or cfg["n_symbols"], "alphabet": cfg["alphabet"],
         "zipf_s": cfg["zipf_s"], "n_lanes": cfg["n_lanes"],
         "chunk_symbols": cfg["chunk_symbols"], "log2_M": 12, "L": 65536, "b": 65536,
         "parallelism": f"independent batch per rank x{world}",
         "l2": "inputs larger than L2 (no flush needed)",
         "step": "encode + decode of the batch; value counts the decode phase"}
    return d


# ---------------------------------------------------------------------------
# Batched leg: 10,000 streams of uneven size, one model each
# ---------------------------------------------------------------------------

# A spin of about 0.1 ms queued before each timed call: the stream is then
# busy while the host enqueues the call, so the device time between the two
# events is the call's own, not the host's launch latency as well.
SPIN_CYCLES = 200_000


def _events(torch, fn, reps, stream=None):
    """Device time (ms) of each of reps calls of fn, between CUDA events
    recorded on the stream fn launches on (the current stream by default)."""
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if stream is None:
            torch.cuda._sleep(SPIN_CYCLES)
        else:
            with torch.cuda.stream(stream):
                torch.cuda._sleep(SPIN_CYCLES)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def batched_leg(rans, dev, args, hbm):
    """Batched encode and decode of the 10,000-stream workload, the
    autotuner's choice of layout, the CUDA-graph replay of the batched decoder
    and the plain one-launch-per-stream decoder for comparison."""
    import torch

    from paper_1402_3392_b300 import autotune
    from paper_1402_3392_b300 import batch as B

    cfg = wl.WORKLOADS["batched"]
    count = args.batched_streams or cfg["n_streams"]
    rng = wl.rng_for("batched")
    sizes = wl.log_uniform_sizes(rng, count, cfg["size_lo"], cfg["size_hi"])
    probs = wl.batched_models(rng, count, cfg["alpha_lo"], cfg["alpha_hi"], cfg["dirichlet"])
    tables = [rans.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    offs, arena_bytes = B.aligned_offsets(sizes)
    arena = wl.streams_on_device(probs, sizes, offs, arena_bytes, wl.seed_for("batched"), dev)
    tdev = B.upload_tables(tables, dev)
    table_idx = np.arange(count)
    total = int(sizes.sum())

    t0 = time.perf_counter()
    if args.batched_layout:
        n_l, ch, pol = args.batched_layout.split(",")
        best, tried = dict(n_lanes=int(n_l), chunk=int(ch), policy=pol), []
    else:
        sample = np.arange(0, count, 25)
        best, tried = autotune.autotune(arena, offs[sample], sizes[sample], tdev, sample, reps=3)
    tune_s = time.perf_counter() - t0
    N = best["n_lanes"]
    cs = autotune.chunk_sizes(sizes, best["chunk"], best["policy"])

    eb = B.encode_batch(arena, offs, sizes, tdev, table_idx, N, cs)
    torch.cuda.synchronize()
    assert not eb.status.any(), "batched encode failed"
    d_desc, scratch = eb._keep
    enc_ms = _events(torch, lambda: rans.rans_encode_batch(
        d_desc, count, tdev, count, eb.sizes, eb.status, scratch, scratch.numel()), 3)
    msg_sizes = eb.host_sizes()
    msg_total = int(msg_sizes.sum())
    del scratch, d_desc
    eb._keep = None

    dec = B.BatchDecoder(eb.arena, eb.offsets, msg_sizes, sizes, tdev, table_idx, N, cs,
                         out_offsets=offs,
                         out_arena=torch.zeros(arena_bytes, dtype=torch.uint8, device=dev))
    dec()
    torch.cuda.synchronize()
    s = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            dec(stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    dec_ms = _events(torch, g.replay, max(5, min(args.steps, 20)))
    # bit-exact check: the filler between streams is zero in both arenas, so
    # the arenas are equal exactly when every stream decoded to its input
    ok = (not dec.status.any()) and torch.equal(dec.out_arena, arena)

    # plain form: one rans_decode launch per stream
    st1 = torch.zeros(1, dtype=torch.int32, device=dev)
    base_m, base_o = eb.arena.data_ptr(), dec.out_arena.data_ptr()

    def plain():
        for k in range(count):
            rans.rans_decode(base_m + int(eb.offsets[k]), int(msg_sizes[k]), tables[k], N, int(cs[k]),
                             base_o + int(offs[k]), int(sizes[k]), st1)

    plain()
    torch.cuda.synchronize()
    plain_ms = _events(torch, plain, 2)
    ok = ok and int(st1.item()) == 0
    dm = statistics.median(dec_ms)
    achieved = (msg_total + total) / (dm * 1e-3) / 1e9
    return {
        "workload": f"{count} streams, sizes log-uniform {cfg['size_lo']}..{cfg['size_hi']} B "
                    f"(total {total / 2**30:.2f} GiB), alphabets {cfg['alpha_lo']}..{cfg['alpha_hi']}, "
                    f"Dirichlet({cfg['dirichlet']})",
        "decode_gbs": total / (dm * 1e-3) / 1e9, "decode_ms": dm,
        "encode_gbs": total / (statistics.median(enc_ms) * 1e-3) / 1e9,
        "encode_ms": statistics.median(enc_ms),
        "plain_decode_gbs": total / (statistics.median(plain_ms) * 1e-3) / 1e9,
        "plain_decode_ms": statistics.median(plain_ms),
        "batched_over_plain": statistics.median(plain_ms) / dm,
        "compression_ratio": msg_total / total, "bit_exact_roundtrip": bool(ok),
        "roofline": {"kernel": "batch_decode_kernel", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "algorithmic_bytes_per_launch": msg_total + total},
        "layout": {"n_lanes": N, "chunk": best["chunk"], "policy": best["policy"],
                   "chunk_symbols_min": int(cs.min()), "chunk_symbols_max": int(cs.max()),
                   "autotune_s": tune_s, "candidates": len(tried)},
        "graph": "setup + persistent decode kernel captured in one CUDA graph, replayed",
    }


# ---------------------------------------------------------------------------
# Binary and single-stream legs
# ---------------------------------------------------------------------------

def binary_leg(rans, dev, args, hbm):
    """4096 streams of 64 KiB {0,1} symbols, stream k with its own model
    p0 ~ U[0.5, 0.999] (one binary model per 64 KiB, as in the rABS-style
    workload), batched encode and decode with the autotuned layout."""
    import torch

    from paper_1402_3392_b300 import autotune
    from paper_1402_3392_b300 import batch as B

    cfg = wl.WORKLOADS["binary"]
    count = cfg["n_chunks"]
    per = cfg["n_symbols"] // count
    rng = wl.rng_for("binary")
    p0 = wl.binary_chunk_probs(rng, count, cfg["p0_lo"], cfg["p0_hi"])
    probs = [np.array([p, 1.0 - p]) for p in p0]
    tables = [rans.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    sizes = np.full(count, per, dtype=np.int64)
    offs, arena_bytes = B.aligned_offsets(sizes)
    sym = wl.streams_on_device(probs, sizes, offs, arena_bytes, wl.seed_for("binary"), dev)
    tdev = B.upload_tables(tables, dev)
    idx = np.arange(count)
    # 256 MiB in all: every stream goes into the tuning runs, so that each
    # candidate layout is timed with the whole GPU's worth of work (a sample
    # leaves a one-chunk-per-stream layout under one wave of warps)
    if args.binary_layout:
        ch, pol = args.binary_layout.split(",")
        best, tried = dict(n_lanes=32, chunk=int(ch), policy=pol), []
    else:
        best, tried = autotune.autotune(sym, offs, sizes, tdev, idx, widths=(32,), reps=3)
    cs = autotune.chunk_sizes(sizes, best["chunk"], best["policy"])
    eb = B.encode_batch(sym, offs, sizes, tdev, idx, 32, cs)
    torch.cuda.synchronize()
    assert not eb.status.any()
    d_desc, scratch = eb._keep
    enc_ms = _events(torch, lambda: rans.rans_encode_batch(
        d_desc, count, tdev, count, eb.sizes, eb.status, scratch, scratch.numel()), 3)
    msg_sizes = eb.host_sizes()
    dec = B.BatchDecoder(eb.arena, eb.offsets, msg_sizes, sizes, tdev, idx, 32, cs,
                         out_offsets=offs,
                         out_arena=torch.zeros(arena_bytes, dtype=torch.uint8, device=dev))
    dec()
    torch.cuda.synchronize()
    dec_ms = _events(torch, dec, 10)
    ok = (not dec.status.any()) and torch.equal(dec.out_arena, sym)
    total, msg_total = int(sizes.sum()), int(msg_sizes.sum())
    dm = statistics.median(dec_ms)
    achieved = (msg_total + total) / (dm * 1e-3) / 1e9
    return {"workload": f"{count} streams x {per} binary symbols (u8 in {{0,1}}), per-stream "
                        f"p0 ~ U[{cfg['p0_lo']}, {cfg['p0_hi']}]",
            "decode_gbs": total / (dm * 1e-3) / 1e9, "decode_ms": dm,
            "encode_gbs": total / (statistics.median(enc_ms) * 1e-3) / 1e9,
            "compression_ratio": msg_total / total, "bit_exact_roundtrip": bool(ok),
            "roofline": {"kernel": "batch_decode_kernel", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm},
            "layout": {"n_lanes": 32, "chunk": best["chunk"], "policy": best["policy"],
                       "chunk_symbols": int(cs[0]), "candidates": len(tried)}}


def bypass_leg(rans, dev, args, hbm):
    """Raw words with the coded symbols (bypass coding, Section 3): 512 Mi
    Zipf(1.1) symbols (a bypass message holds up to about 2^30 symbols, its
    worst case being 4 bytes per symbol), every symbol >= 16 followed by one
    raw 16-bit word; encode and decode timed with CUDA events, the round trip
    checked."""
    import torch

    cfg = wl.WORKLOADS["bypass"]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rans.rans_quantize_table(wl.weights_from_probs(p))
    flags = (np.arange(cfg["alphabet"]) >= cfg["raw_from"]).astype(np.uint8)
    sym = wl.iid_symbols_device(p, n, wl.seed_for("bypass"), dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed_for("bypass", 1) & 0x7FFFFFFFFFFFFFFF)
    raw = torch.randint(-(1 << 15), 1 << 15, (n,), generator=gen, device=dev, dtype=torch.int16)
    cap = rans.rans_max_encoded_size_bypass(n, N, CS)
    scap = rans.rans_encode_scratch_size_bypass(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode_bypass(sym, raw, n, freq, flags, N, CS, msg, cap, size, est,  # noqa: E731
                                          scratch, scap)
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    del scratch
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    rout = torch.empty(n, dtype=torch.int16, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode_bypass(msg, msg_size, freq, flags, N, CS, out, rout, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    has = sym >= cfg["raw_from"]                  # the symbols whose flag is set
    ok = (int(dst.item()) == 0 and torch.equal(out, sym)
          and torch.equal(rout, torch.where(has, raw, torch.zeros_like(raw))))
    n_raw = int(has.sum().item())
    dec_ms = statistics.median(_events(torch, dec, 10))
    orc = _oracle()
    cpu = oracle_leg_baseline(
        lambda ch: orc.decode_chunk_bypass(ch, CS, freq, flags, N=N),
        host_chunks(msg, n // CS, 16 * host_cores()), CS, unit_bytes=False)
    alg = msg_size + n + 2 * n   # message read, symbols and one raw word slot per symbol written
    return {"workload": f"{n} symbols, Zipf({cfg['zipf_s']}) over {cfg['alphabet']}, symbols >= "
                        f"{cfg['raw_from']} followed by a raw 16-bit word ({n_raw} raw words), "
                        f"{n // CS} chunks x {CS}, N = {N}",
            "decode_gsym_s": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "decoded_gbs": (n + 2 * n_raw) / (dec_ms * 1e-3) / 1e9,
            "encode_gsym_s": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "message_bytes": msg_size, "bit_exact_roundtrip": bool(ok), "cpu_baseline": cpu,
            "roofline": {"kernel": "decode_kernel (bypass)", "bound": "hbm",
                         "achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": alg}}


def bytes_leg(rans, dev, args, hbm):
    """The 1 GiB chunked workload as a byte-wise message (b = 2^8, up to two
    renormalization bytes per symbol read breadth-first across the N = 32
    lanes, Section 5): encode and decode timed, the round trip checked."""
    import torch

    cfg = wl.WORKLOADS["chunked"]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rans.rans_quantize_table(wl.weights_from_probs(p))
    sym = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), dev)
    cap = rans.rans_max_encoded_size_bytes(n, N, CS)
    scap = rans.rans_encode_scratch_size(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode_bytes(sym, n, freq, N, CS, msg, cap, size, est, scratch, scap)  # noqa: E731
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    del scratch
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode_bytes(msg, msg_size, freq, N, CS, out, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    ok = int(dst.item()) == 0 and torch.equal(out, sym)
    dec_ms = statistics.median(_events(torch, dec, 10))
    alg = msg_size + n
    orc = _oracle()
    cpu = oracle_leg_baseline(lambda ch: orc.decode_chunk_bytes(ch, CS, freq, N=N),
                              host_chunks(msg, n // CS, 16 * host_cores()), CS)
    return {"workload": f"{n} symbols, Zipf({cfg['zipf_s']}) over {cfg['alphabet']}, {n // CS} "
                        f"chunks x {CS}, N = {N}, byte-wise (L = 2^23, b = 2^8)", "cpu_baseline": cpu,
            "decode_gbs": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "encode_gbs": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "compression_ratio": msg_size / n, "bit_exact_roundtrip": bool(ok),
            "roofline": {"kernel": "decode_kernel (byte-wise)", "bound": "hbm",
                         "achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": alg}}


def adaptive_leg(rans, dev, args, hbm):
    """256 Mi bits whose statistics drift (P(0) constant over runs of 4096
    symbols, U[0.001, 0.999] per run), coded with one adaptive context per
    coder (Section 5): encode and decode timed, the round trip checked, the
    size set beside one static binary model for the whole message."""
    import torch

    cfg = wl.WORKLOADS["adaptive"]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    sym = wl.drifting_bits_device(n, cfg["segment"], wl.seed_for("adaptive"), dev, cfg["p0_lo"],
                                  cfg["p0_hi"])
    cap = rans.rans_max_encoded_size(n, N, CS)
    scap = rans.rans_encode_scratch_size_adaptive(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode_adaptive(sym, n, N, CS, msg, cap, size, est, scratch, scap)  # noqa: E731
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    p1 = float(sym.float().mean().item())
    freq = rans.rans_quantize_table(wl.weights_from_probs(np.array([1.0 - p1, p1])))
    del scratch
    static_size = int(rans.encode(sym, freq, N, CS)[1].item())   # not timed
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode_adaptive(msg, msg_size, N, CS, out, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    ok = int(dst.item()) == 0 and torch.equal(out, sym)
    dec_ms = statistics.median(_events(torch, dec, 10))
    alg = msg_size + n
    orc = _oracle()
    cpu = oracle_leg_baseline(lambda ch: orc.decode_chunk_adaptive(ch, CS, N=N),
                              host_chunks(msg, n // CS, 16 * host_cores()), CS, unit_bytes=False)
    return {"cpu_baseline": cpu,
            "workload": f"{n} bits, P(0) ~ U[{cfg['p0_lo']}, {cfg['p0_hi']}] per run of "
                        f"{cfg['segment']}, {n // CS} chunks x {CS}, N = {N}, one adaptive "
                        f"context per coder (rate 1/32)",
            "decode_gbs": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "encode_gbs": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "bits_per_symbol": 8 * msg_size / n, "static_bits_per_symbol": 8 * static_size / n,
            "bit_exact_roundtrip": bool(ok),
            "roofline": {"kernel": "decode_kernel (adaptive)", "bound": "hbm",
                         "achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": alg}}


def issue_peak_tops(dev, sm_max_mhz):
    """Instruction-issue peak in T lane-operations/s: every SM's 4 schedulers
    issue one 32-lane instruction a cycle each, at the SM's maximum clock
    (the recipe's 2032 MHz when NVML gives none).  An upper bound for any
    kernel bound by integer arithmetic."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 4 * 32 * float(sm_max_mhz or 2032) * 1e6 / 1e12


def adaptive_n_leg(rans, dev, args, hbm, sm_max_mhz=None):
    """256 Mi symbols over 16 whose distribution drifts (Dirichlet(0.5) per
    run of 4096 symbols), coded with one adaptive 16-symbol model per coder
    (Section 5): encode and decode timed, the round trip checked, the size set
    beside one static model for the whole message.  The decoder is bound by
    integer arithmetic, not memory: its roofline counts the model update's
    operations against the instruction-issue peak, its HBM figures beside."""
    import torch

    cfg = wl.WORKLOADS["adaptive_n"]
    n, k, N, CS = (args.symbols or cfg["n_symbols"]), cfg["n_alpha"], cfg["n_lanes"], \
        cfg["chunk_symbols"]
    sym = wl.drifting_symbols_device(n, k, cfg["segment"], wl.seed_for("adaptive_n"), dev,
                                     cfg["dirichlet"])
    cap = rans.rans_max_encoded_size(n, N, CS)
    scap = rans.rans_encode_scratch_size_adaptive_n(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode_adaptive_n(sym, n, k, N, CS, msg, cap, size, est,  # noqa: E731
                                              scratch, scap)
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    counts = torch.bincount(sym.long(), minlength=k).cpu().numpy().astype(np.float64)
    freq = rans.rans_quantize_table(wl.weights_from_probs(np.maximum(counts, 1) / counts.sum()))
    del scratch
    static_size = int(rans.encode(sym, freq, N, CS)[1].item())   # not timed
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode_adaptive_n(msg, msg_size, k, N, CS, out, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    ok = int(dst.item()) == 0 and torch.equal(out, sym)
    dec_ms = statistics.median(_events(torch, dec, 10))
    alg = msg_size + n
    # After every symbol each of the model's n - 1 interior boundaries moves:
    # a compare (which side of the coded symbol it lies), a subtraction (its
    # distance to its target), a shift and an add or subtract.  4 (n - 1)
    # integer operations a symbol; D and the renormalization are not counted.
    ops = 4 * (k - 1) * n
    peak_ops = issue_peak_tops(dev, sm_max_mhz)
    orc = _oracle()
    cpu = oracle_leg_baseline(lambda ch: orc.decode_chunk_adaptive_n(ch, CS, k, N=N),
                              host_chunks(msg, n // CS, 4 * host_cores()), CS, unit_bytes=False)
    return {"cpu_baseline": cpu,
            "workload": f"{n} symbols over {k}, Dirichlet({cfg['dirichlet']}) per run of "
                        f"{cfg['segment']}, {n // CS} chunks x {CS}, N = {N}, one adaptive "
                        f"{k}-symbol model per coder (rate 1/32)",
            "decode_gsym_s": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "encode_gsym_s": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "bits_per_symbol": 8 * msg_size / n, "static_bits_per_symbol": 8 * static_size / n,
            "bit_exact_roundtrip": bool(ok),
            "roofline": {"kernel": "decode_kernel (adaptive-n)", "bound": "alu",
                         "achieved": ops / (dec_ms * 1e-3) / 1e12, "peak": peak_ops,
                         "unit": "TOP/s", "frac": ops / (dec_ms * 1e-3) / 1e12 / peak_ops,
                         "peak_kind": "derived: SMs x 4 schedulers x 32 lanes x max SM clock",
                         "algorithmic_ops_per_launch": ops,
                         "hbm": {"achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm,
                                 "unit": "GB/s", "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                                 "algorithmic_bytes_per_launch": alg}}}


def prefix_leg(rans, dev, args, hbm):
    """Section 4: the 1 GiB chunked workload coded by 32 prefix coders per
    chunk (package-merge lengths <= 12 from the Zipf(1.1) weights), their
    words laid down in the decoders' read order; encode and decode timed,
    the round trip checked, the size set beside the rANS message's."""
    import torch

    cfg = wl.WORKLOADS["chunked"]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    ln = rans.rans_prefix_lengths(wl.weights_from_probs(p), rans.RANS_PREFIX_MAX_LEN)
    sym = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), dev)
    cap = rans.rans_max_encoded_size_prefix(n, N, CS)
    scap = rans.rans_encode_scratch_size_prefix(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode_prefix(sym, n, ln, N, CS, msg, cap, size, est, scratch, scap)  # noqa: E731
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    del scratch
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode_prefix(msg, msg_size, ln, N, CS, out, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    ok = int(dst.item()) == 0 and torch.equal(out, sym)
    dec_ms = statistics.median(_events(torch, dec, 10))
    alg = msg_size + n
    mean_len = float((p * ln[: p.size]).sum())
    orc = _oracle()
    cpu = oracle_leg_baseline(lambda ch: orc.decode_chunk_prefix(ch, CS, ln, N=N),
                              host_chunks(msg, n // CS, 16 * host_cores()), CS)
    return {"workload": f"{n} symbols, Zipf({cfg['zipf_s']}) over {cfg['alphabet']}, {n // CS} "
                        f"chunks x {CS}, N = {N} prefix coders (lengths <= 12, mean "
                        f"{mean_len:.3f} bits), words in the decoders' read order",
            "decode_gbs": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "encode_gbs": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "compression_ratio": msg_size / n, "bit_exact_roundtrip": bool(ok), "cpu_baseline": cpu,
            "roofline": {"kernel": "decode_kernel (prefix)", "bound": "hbm",
                         "achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": alg}}


def wide_leg(rans, dev, args, hbm):
    """The 1 GiB chunked workload with the model at 14 bits of probability
    resolution (M = 2^14, b = 2^16: still one renormalization per symbol,
    Section 5): encode and decode timed, the round trip checked, the size set
    beside the 12-bit model's."""
    import torch

    cfg = wl.WORKLOADS["chunked"]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rans.rans_quantize_table(wl.weights_from_probs(p), 14)
    sym = wl.iid_symbols_device(p, n, wl.seed_for("chunked"), dev)
    cap = rans.rans_max_encoded_size(n, N, CS)
    scap = rans.rans_encode_scratch_size(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    enc = lambda: rans.rans_encode(sym, n, freq, N, CS, msg, cap, size, est, scratch, scap)  # noqa: E731
    enc()
    torch.cuda.synchronize()
    assert int(est.item()) == 0
    msg_size = int(size.item())
    enc_ms = statistics.median(_events(torch, enc, 5))
    f12 = rans.rans_quantize_table(wl.weights_from_probs(p))
    size12 = int(rans.encode(sym, f12, N, CS, scratch=scratch)[1].item())   # not timed
    del scratch
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    dst = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode(msg, msg_size, freq, N, CS, out, n, dst)  # noqa: E731
    dec()
    torch.cuda.synchronize()
    ok = int(dst.item()) == 0 and torch.equal(out, sym)
    dec_ms = statistics.median(_events(torch, dec, 10))
    alg = msg_size + n
    orc = _oracle()
    cpu = oracle_leg_baseline(lambda ch: orc.decode_chunk(ch, CS, freq, N=N),
                              host_chunks(msg, n // CS, 16 * host_cores()), CS)
    return {"workload": f"{n} symbols, Zipf({cfg['zipf_s']}) over {cfg['alphabet']}, {n // CS} "
                        f"chunks x {CS}, N = {N}, model at 14 bits (M = 2^14)",
            "decode_gbs": n / (dec_ms * 1e-3) / 1e9, "decode_ms": dec_ms,
            "encode_gbs": n / (enc_ms * 1e-3) / 1e9, "encode_ms": enc_ms,
            "compression_ratio": msg_size / n, "compression_ratio_12_bits": size12 / n,
            "bit_exact_roundtrip": bool(ok), "cpu_baseline": cpu,
            "roofline": {"kernel": "decode_kernel (14-bit model)", "bound": "hbm",
                         "achieved": alg / (dec_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (dec_ms * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": alg}}


def single_leg(rans, dev, args):
    """One 1 MiB stream, Zipf(1.2) over 256 symbols, 32 coders in one chunk:
    a single warp's chain of 32768 dependent steps, so a latency figure."""
    import torch

    cfg = wl.WORKLOADS["single"]
    n, N, CS = cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rans.rans_quantize_table(wl.weights_from_probs(p))
    sym = torch.from_numpy(wl.iid_symbols(wl.rng_for("single"), p, n)).to(dev)
    msg, _, _ = rans.encode(sym, freq, N, CS)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    cap = rans.rans_max_encoded_size(n, N, CS)
    scap = rans.rans_encode_scratch_size(n, N, CS)
    ebuf = torch.empty(cap, dtype=torch.uint8, device=dev)
    escr = torch.empty(scap, dtype=torch.uint8, device=dev)
    esz = torch.zeros(1, dtype=torch.int64, device=dev)
    est = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = lambda: rans.rans_decode(msg, msg.numel(), freq, N, CS, out, n, st)  # noqa: E731
    enc = lambda: rans.rans_encode(sym, n, freq, N, CS, ebuf, cap, esz, est, escr, scap)  # noqa: E731
    dec()
    enc()
    torch.cuda.synchronize()
    d_ms = statistics.median(_events(torch, dec, 20))
    e_ms = statistics.median(_events(torch, enc, 20))
    ok = int(st.item()) == 0 and torch.equal(out, sym)
    return {"workload": "1 MiB, Zipf(1.2) over 256, one stream of 32 interleaved coders",
            "decode_us": d_ms * 1e3, "encode_us": e_ms * 1e3,
            "decode_gbs": n / (d_ms * 1e-3) / 1e9, "encode_gbs": n / (e_ms * 1e-3) / 1e9,
            "bit_exact_roundtrip": bool(ok)}


# ---------------------------------------------------------------------------
# Serving leg: Poisson arrivals through the continuous-batching server
# ---------------------------------------------------------------------------

def serving_leg(rans, dev, args):
    """Encode and decode requests (50/50) of log-uniform size 4 KiB..64 MiB,
    one Dirichlet(0.5) model over 64..256 symbols each, arriving as a Poisson
    process at several rates (args.serving_requests requests per rate),
    served from a 40 GiB device budget.  Two payload modes: host (inputs
    copied in from and outputs copied back to page-locked host memory) and
    device (inputs and outputs already in device memory, coded in place), so
    the GPU side's latency and throughput show apart from PCIe.  The requests
    are drawn from a pool of 256 distinct ones (payloads, models, output
    buffers); requests sharing a pool entry write the same bytes to the same
    output, so after a run every pool entry's output is checked against the
    batched path once.  Latency = completion - arrival."""
    import torch

    from paper_1402_3392_b300 import batch as B

    cfg = wl.WORKLOADS["serving"]
    pool = 256
    count = args.serving_requests
    rng = wl.rng_for("serving")
    sizes = wl.log_uniform_sizes(rng, pool, cfg["size_lo"], cfg["size_hi"])
    probs = wl.batched_models(rng, pool, cfg["alpha_lo"], cfg["alpha_hi"], cfg["dirichlet"])
    tables = [rans.rans_quantize_table(wl.weights_from_probs(p)) for p in probs]
    kinds = rng.integers(0, 2, size=pool)
    N, CS = 32, 1 << 16
    offs, arena_bytes = B.aligned_offsets(sizes)
    sym = wl.streams_on_device(probs, sizes, offs, arena_bytes, wl.seed_for("serving"), dev)
    tdev = B.upload_tables(tables, dev)
    eb = B.encode_batch(sym, offs, sizes, tdev, np.arange(pool), N, CS)
    torch.cuda.synchronize()
    assert not eb.status.any()
    msg_sizes = eb.host_sizes()
    in_sizes = np.where(kinds == rans.RANS_REQ_ENCODE, sizes, msg_sizes)
    caps = np.where(kinds == rans.RANS_REQ_ENCODE,
                    [rans.rans_max_encoded_size(int(n), N, CS) for n in sizes], sizes)
    in_offs, in_total = B.aligned_offsets(in_sizes)
    out_offs, out_total = B.aligned_offsets(caps)
    h_in = torch.empty(in_total, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(out_total, dtype=torch.uint8, pin_memory=True)
    d_in = torch.empty(in_total, dtype=torch.uint8, device=dev)
    d_out = torch.empty(out_total, dtype=torch.uint8, device=dev)
    want = []
    for i in range(pool):
        if kinds[i] == rans.RANS_REQ_ENCODE:
            src = sym[int(offs[i]):int(offs[i]) + int(sizes[i])]
            w = eb.arena[int(eb.offsets[i]):int(eb.offsets[i]) + int(msg_sizes[i])]
        else:
            src = eb.arena[int(eb.offsets[i]):int(eb.offsets[i]) + int(msg_sizes[i])]
            w = sym[int(offs[i]):int(offs[i]) + int(sizes[i])]
        h_in[int(in_offs[i]):int(in_offs[i]) + int(in_sizes[i])].copy_(src)
        d_in[int(in_offs[i]):int(in_offs[i]) + int(in_sizes[i])].copy_(src)
        want.append(w)
    budget = torch.empty(cfg["budget_bytes"], dtype=torch.uint8, device=dev)
    srv = rans.Server(tdev, budget, max_batch=64, n_slots=3)
    raw_pool = int(sizes.sum())
    modes = {}
    for mode in ("host", "device"):
        base_in = (h_in if mode == "host" else d_in).data_ptr()
        base_out = (h_out if mode == "host" else d_out).data_ptr()
        flag = 0 if mode == "host" else rans.RANS_REQ_DEVICE_MEMORY
        rows = []
        exact = True
        for rate in (1000.0, 5000.0, 20000.0, 50000.0):
            r = np.random.default_rng(int(rate) + (0 if mode == "host" else 7))
            pick = r.integers(0, pool, size=count)
            reqs = np.zeros(count, dtype=rans.REQUEST_DTYPE)
            reqs["kind"] = kinds[pick] | flag
            reqs["table"] = pick
            reqs["n_lanes"] = N
            reqs["chunk_symbols"] = CS
            reqs["input"] = base_in + in_offs[pick]
            reqs["input_size"] = in_sizes[pick]
            reqs["n_symbols"] = sizes[pick]
            reqs["output"] = base_out + out_offs[pick]
            reqs["output_cap"] = caps[pick]
            reqs["arrival_s"] = wl.poisson_arrivals(r, rate, count)
            (h_out if mode == "host" else d_out).zero_()
            torch.cuda.synchronize()
            res = srv.run(reqs)
            lat = (res["done_s"] - reqs["arrival_s"]) * 1e3
            span = float(res["done_s"].max() - reqs["arrival_s"].min())
            ok = bool((res["status"] == 0).all())
            used = np.unique(pick)
            out = h_out if mode == "host" else d_out
            for i in used:     # every pool entry this run served, checked once
                n_out = int(msg_sizes[i]) if kinds[i] == rans.RANS_REQ_ENCODE else int(sizes[i])
                got = out[int(out_offs[i]):int(out_offs[i]) + n_out]
                exact = exact and torch.equal(got.to(dev), want[i])
            exact = exact and ok and all(
                int(res["output_size"][k]) == (int(msg_sizes[pick[k]])
                                               if kinds[pick[k]] == rans.RANS_REQ_ENCODE
                                               else int(sizes[pick[k]])) for k in range(count))
            raw = int(sizes[pick].sum())
            rows.append({"rate_req_s": rate, "achieved_req_s": count / span,
                         "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "gbs": raw / span / 1e9,
                         "batches": int(res["batch"].max()) + 1, "all_ok": ok})
        modes[mode] = {"rates": rows, "bit_exact_vs_batched_path": bool(exact)}
    srv.close()
    return {"workload": f"{count} requests per rate drawn from {pool} distinct ones "
                        f"({raw_pool / 2**30:.2f} GiB raw), sizes log-uniform "
                        f"{cfg['size_lo']}..{cfg['size_hi']} B, encode/decode 50/50, "
                        f"Dirichlet({cfg['dirichlet']}) over {cfg['alpha_lo']}..{cfg['alpha_hi']} "
                        f"symbols, {cfg['budget_bytes'] >> 30} GiB device budget",
            "server": "max_batch 64, 3 slots", "host_payloads": modes["host"],
            "device_payloads": modes["device"]}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def rank_seed(workload: str, rank: int) -> int:
    """Seed of rank `rank`'s batch: every rank codes its own independent
    batch of the workload (weak scaling, no data exchange)."""
    return wl.seed_for(workload, rank)


def max_over_ranks(values, device, world: int):
    """Element-wise maximum of per-rank timings over all ranks (the job takes
    as long as its slowest rank); the identity on one rank."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(world: int, n_symbols: int, decode_ms: float) -> float:
    """Whole-job decoded GB/s: the symbols all ranks decoded over the
    slowest rank's decode time."""
    return world * n_symbols / (decode_ms * 1e-3) / 1e9


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1402_3392_b300 import rans

    cfg = wl.WORKLOADS[args.workload]
    n, N, CS = args.symbols or cfg["n_symbols"], cfg["n_lanes"], cfg["chunk_symbols"]
    p = wl.zipf_probs(cfg["alphabet"], cfg["zipf_s"])
    freq = rans.rans_quantize_table(wl.weights_from_probs(p))
    sym = wl.iid_symbols_device(p, n, rank_seed(args.workload, rank), dev)

    cap = rans.rans_max_encoded_size(n, N, CS)
    scap = rans.rans_encode_scratch_size(n, N, CS)
    msg = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    out_size = torch.zeros(1, dtype=torch.int64, device=dev)
    enc_status = torch.zeros(1, dtype=torch.int32, device=dev)
    dec = torch.empty(n, dtype=torch.uint8, device=dev)
    dec_status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)

    # Encode once to learn the message size the decode phase reads.
    rans.rans_encode(sym, n, freq, N, CS, msg, cap, out_size, enc_status, scratch, scap, stream)
    torch.cuda.synchronize(dev)
    msg_size = int(out_size.item())
    assert int(enc_status.item()) == 0 and msg_size > 0

    def step(evs):
        evs[0].record(stream)
        rans.rans_encode(sym, n, freq, N, CS, msg, cap, out_size, enc_status, scratch, scap,
                         stream)
        evs[1].record(stream)
        rans.rans_decode(msg, msg_size, freq, N, CS, dec, n, dec_status, stream)
        evs[2].record(stream)

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(3)]  # noqa: E731
    for _ in range(args.warmup):
        step(mk())
    torch.cuda.synchronize(dev)
    ok = (int(enc_status.item()) == 0 and int(dec_status.item()) == 0
          and int(out_size.item()) == msg_size and torch.equal(dec, sym))
    if not ok:
        raise SystemExit("round trip failed in warm-up")

    evs = [mk() for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    sampler.mark_start()
    t0 = time.perf_counter()
    for e in evs:
        step(e)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    sampler.mark_stop()
    sampler.stop()
    enc_ms = [a.elapsed_time(b) for a, b, _ in evs]
    dec_ms = [b.elapsed_time(c) for _, b, c in evs]
    step_ms = evs[0][0].elapsed_time(evs[-1][2]) / args.steps
    ok = int(dec_status.item()) == 0 and torch.equal(dec, sym)

    dec_mean, enc_mean, step_mean, wall_max = max_over_ranks(
        [statistics.mean(dec_ms), statistics.mean(enc_ms), step_ms, wall], dev, world)

    e2e = e2e_enc = None
    if not args.no_e2e:
        e2e = end_to_end(rans, msg[:msg_size], n, freq, N, CS, dev, max(3, min(args.steps, 10)),
                         sym)
        e2e_enc = end_to_end_encode(rans, sym, freq, N, CS, dev, max(3, min(args.steps, 10)),
                                    msg[:msg_size])

    ceiling = pipe_ceiling(rans, dev, (n / N) / (dec_mean * 1e-3)) if rank == 0 else None

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, cpu1 = cpu_baseline(msg[:msg_size].cpu().numpy(), freq, N, CS, n // CS)

    legs = [x for x in args.legs.split(",") if x and x != "none"]
    extra = {}
    if legs:
        del msg, scratch, dec, sym
        torch.cuda.empty_cache()
    if "batched" in legs:
        extra["batched"] = batched_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "binary" in legs:
        extra["binary"] = binary_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "single" in legs:
        extra["single"] = single_leg(rans, dev, args)
    if "serving" in legs:
        extra["serving"] = serving_leg(rans, dev, args)
        torch.cuda.empty_cache()
    if "bypass" in legs:
        extra["bypass"] = bypass_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "bytes" in legs:
        extra["bytes"] = bytes_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "adaptive" in legs:
        extra["adaptive"] = adaptive_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "adaptive_n" in legs:
        extra["adaptive_n"] = adaptive_n_leg(rans, dev, args, peaks()[0], sampler.max_mhz)
        torch.cuda.empty_cache()
    if "prefix" in legs:
        extra["prefix"] = prefix_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()
    if "wide" in legs:
        extra["wide"] = wide_leg(rans, dev, args, peaks()[0])
        torch.cuda.empty_cache()

    if ceiling and "batched" in extra:
        # the batched decoder's chunk-steps (32 symbols each) per second
        b = extra["batched"]
        rate = b["decode_gbs"] * 1e9 / 32
        b["roofline"]["pipe_ceiling_fraction"] = rate / ceiling["warp_steps_per_s"]
    if rank == 0:
        hbm, peak_kind = peaks()
        alg_bytes = msg_size + n
        achieved = alg_bytes / (dec_mean * 1e-3) / 1e9
        line = {
            "metric": "decoded GB/s", "value": job_value(world, n, dec_mean),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(args.workload, world, n),
            "decode_ms": dec_mean, "encode_ms": enc_mean,
            "encode_gbs": world * n / (enc_mean * 1e-3) / 1e9,
            "compression_ratio": msg_size / n, "bit_exact_roundtrip": bool(ok),
            "roofline": {"kernel": "decode_kernel12", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": profiled_traffic(),
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "pipe_ceiling": ceiling},
            "clocks": sampler.summary(),
            "device": {"name": torch.cuda.get_device_name(dev),
                       "sm_count": torch.cuda.get_device_properties(dev).multi_processor_count},
            # per step: encode_kernel (codes and places the chunks), settle_kernel
            # (the size of a rejected message), decode_kernel
            "gpu_launches": 3 * args.steps,
            "e2e": e2e,
            "e2e_encode": e2e_enc,
            "cpu_baseline": cpu,
            "cpu_baseline_1t": cpu1,
        }
        # the legs of the scope table's next rows first, the headline's
        # companions (batched, binary, serving) last: a reader that keeps only
        # the end of the line still sees them
        for k in ("bypass", "bytes", "adaptive", "adaptive_n", "prefix", "wide", "single",
                  "serving", "binary", "batched"):
            if k in extra:
                line[k] = extra[k]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def pipe_ceiling(rans, dev, decoder_warp_steps_per_s):
    """The rate of rans_check_gather_ceiling (the decode step's slot-table
    gather, ring window read and 32-byte symbol store, without its arithmetic,
    in the plain decoder's shape) beside the headline decoder's own rate, both
    in warp-steps per second."""
    import torch

    warps = rans.rans_check_gather_ceiling_warps()
    out = torch.empty(warps * 4096, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    steps = 6144  # three 64 Ki-symbol chunks per warp
    run = lambda: rans.rans_check_gather_ceiling(steps, out, out.numel(), sink)  # noqa: E731
    run()
    torch.cuda.synchronize(dev)
    ms = statistics.median(_events(torch, run, 10))
    rate = warps * steps / (ms * 1e-3)
    return {"kernel": "gather_ceiling_kernel", "warps": warps, "steps_per_warp": steps,
            "ms": ms, "warp_steps_per_s": rate,
            "decoder_warp_steps_per_s": decoder_warp_steps_per_s,
            "decoder_fraction": decoder_warp_steps_per_s / rate}


def end_to_end(rans, msg_dev, n, freq, N, CS, dev, steps, sym_dev):
    """Decoded GB/s through the C ABI with host buffers (rans_decode_host):
    each step copies the message in from pinned host memory, decodes, and
    copies the symbols and the status word back to pinned host memory, the
    copies of pieces overlapped with each other and with the decoding."""
    import torch

    h_msg = torch.empty(msg_dev.numel(), dtype=torch.uint8, pin_memory=True)
    h_msg.copy_(msg_dev)
    h_out = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h_st = torch.empty(1, dtype=torch.int32, pin_memory=True)
    work = torch.empty(rans.rans_decode_host_work_size(msg_dev.numel(), n), dtype=torch.uint8,
                       device=dev)
    s = torch.cuda.Stream(dev)

    def one():
        rans.rans_decode_host(h_msg, h_msg.numel(), freq, N, CS, h_out, n, h_st, work,
                              work.numel(), s)

    one()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(steps):
        one()
    b.record(s)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    assert int(h_st.item()) == 0
    assert torch.equal(h_out, sym_dev.cpu()), "end-to-end decode differs from the input"
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(msg_dev.numel()), "d2h_bytes_per_step": n + 4,
            "api": "rans_decode_host"}


def end_to_end_encode(rans, sym_dev, freq, N, CS, dev, steps, msg_dev):
    """Encoded input GB/s through the C ABI with host buffers
    (rans_encode_host): each step copies the symbols in from pinned host
    memory and the device writes the message straight into pinned host
    memory, pieces overlapped; the size and status words come back too."""
    import torch

    n = sym_dev.numel()
    h_sym = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h_sym.copy_(sym_dev)
    cap = rans.rans_max_encoded_size(n, N, CS)
    h_out = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    h_size = torch.zeros(1, dtype=torch.int64, pin_memory=True)
    h_st = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    work = torch.empty(rans.rans_encode_host_work_size(n, N, CS), dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(dev)

    def one():
        rans.rans_encode_host(h_sym, n, freq, N, CS, h_out, cap, h_size, h_st, work,
                              work.numel(), s)

    one()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(steps):
        one()
    b.record(s)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    size = int(h_size.item())
    assert int(h_st.item()) == 0 and size == msg_dev.numel()
    assert torch.equal(h_out[:size], msg_dev.cpu()), "end-to-end encode differs"
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "h2d_bytes_per_step": n, "d2h_bytes_per_step": size + 12,
            "api": "rans_encode_host"}


def cpu_baseline(msg, freq, N, CS, n_chunks):
    """The oracle decoding a bounded sample of the message's chunks on all
    host threads, and the first 256 of them on one thread."""
    cores = host_cores()
    chunks = split_chunks(msg, n_chunks)
    count = min(len(chunks), 256 * cores)       # about 20 s of CPU work
    rate, dt = oracle_decode_rate(chunks[:count], freq, N, CS, cores)
    one = min(len(chunks), 256)
    rate1, dt1 = oracle_decode_rate(chunks[:one], freq, N, CS, 1)
    all_threads = {"value": rate / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
                   "sample": f"oracle decode of {count} chunks x {CS} symbols of this workload's "
                             f"message ({count * CS / 2**20:.0f} MiB) on {cores} threads, "
                             f"{dt:.1f} s ({dt * cores:.0f} CPU-seconds)"}
    one_thread = {"value": rate1 / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                  "sample": f"oracle decode of the first {one} chunks x {CS} symbols on one "
                            f"thread, {dt1:.1f} s"}
    return all_threads, one_thread


if __name__ == "__main__":
    sys.exit(main())
