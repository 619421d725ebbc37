#!/usr/bin/env python
"""Benchmark of the NTT extractor path on GB300.

Default workload (one step = one extraction through the C ABI): the Circulant
extractor, single instance, n + 1 = 16777259 (the smallest prime >= 2^24 with
primitive root 2), x of n bits and seed y of n + 1 bits, i.i.d. Bernoulli(1/2)
from a fixed seed, m = n / 2 output bits.  Transform length L = 2^25.

Printed: ONE JSON line (rank 0) with the output throughput in Gbit/s (inputs
resident in HBM), the roofline of the dominant kernel (CUDA events on the
launching stream, via the library's tracing hook), the end-to-end figure
through cm_extract_host (host buffers, copies inside the timed region), the
CPU oracle timed on a bounded sample, SM clocks sampled during the timed
region, and the number of kernel launches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cm|reference]
                    [--workload circulant|toeplitz|dodis]

N > 1 runs N independent replicas (one extraction per GPU per step, no
collective on the data path); value is the sum over ranks divided by the
slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # kind, n (input length n_1), m, seed-length formula
    "circulant": dict(kind=1, n=16777258, m=8388629,
                      name="Circulant single instance: n+1 = 16777259 (smallest N_A prime >= 2^24), "
                           "m = n/2, Bernoulli(1/2) x and y"),
    "toeplitz": dict(kind=0, n=1 << 16, m=1 << 15,
                     name="Toeplitz single instance: n = 2^16, m = 2^15, Bernoulli(1/2) x and y"),
    "dodis": dict(kind=2, n=1073741789, m=429496715,
                  name="Dodis et al. single instance: n = 1073741789 (largest N_A prime <= 2^30), "
                       "m = floor(0.4 n), Bernoulli(1/2) x and y"),
    # the QRNG example of the paper: n1 = 6.5e9, k1 = 581295000, eps = 1e-10
    "qrng_toeplitz": dict(kind=0, n=6_500_000_000, m=581_294_933,
                          name="Toeplitz at the QRNG example's sizes: n = 6.5e9, m = 581294933, "
                               "Bernoulli(1/2) x and y"),
    # the QKD privacy-amplification example: n1 = 1.738e9 raw key bits, m = 41378264
    "qkd_toeplitz": dict(kind=0, n=1_738_000_000, m=41_378_264,
                         name="Toeplitz at the QKD example's sizes: n = 1.738e9, m = 41378264, "
                              "Bernoulli(1/2) x and y"),
    "qrng_circulant": dict(kind=1, n=6_500_000_068, m=581_294_933,
                           name="Circulant at the QRNG example's sizes: P = 6500000069, m = 581294933, "
                                "Bernoulli(1/2) x and y"),
}
KIND_NAMES = {0: "toeplitz", 1: "circulant", 2: "dodis"}
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def seed_bits(kind, n, m):
    return n + m - 1 if kind == 0 else (n + 1 if kind == 1 else n)


# The translation units a kernel's capture depends on: the unit that defines
# and launches it and, for the NTT-path kernels, the planner that picks their
# shapes (cm_api.cu).  A capture stays valid while only other units change.
# Any other kernel is keyed on every unit but those of the stand-alone
# extractors (Von Neumann, Trevisan, shared seed).  Each unit counts with the
# headers it includes (transitively).
OWN_UNITS = {"k_vn": ("cm_vn.cu",), "k_rsh": ("cm_trevisan.cu",), "k_ss": ("cm_shared_seed.cu",),
             "k_pass_fwd_bits_f25": ("cm_pass25.cu", "cm_api.cu"), "k_middle_f25": ("cm_pass25.cu", "cm_api.cu"),
             "k_pass_inv_parity_f25": ("cm_pass25.cu", "cm_api.cu"),
             "k_pack_tail": ("cm_launch_misc.cu", "cm_api.cu"), "k_cluster_f25": ("cm_cluster25.cu", "cm_api.cu"),
             "k_batch": ("cm_batch.cu", "cm_api.cu")}
_INCLUDE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _source_closure(units):
    """The units and every header they include with quotes, resolved in the
    kernel source directory, then the public include directory."""
    dirs = [os.path.join(ROOT, "paper_2402_09481_gb300", "csrc"), os.path.join(ROOT, "include")]
    seen, todo = set(), list(units)
    while todo:
        path = todo.pop()
        if path in seen:
            continue
        seen.add(path)
        with open(path, errors="replace") as fh:
            text = fh.read()
        for name in _INCLUDE.findall(text):
            for d in [os.path.dirname(path)] + dirs:
                cand = os.path.join(d, name)
                if os.path.exists(cand):
                    todo.append(os.path.normpath(cand))
                    break
    return sorted(seen)


def kernel_source_hash(kernel: str | None = None) -> str:
    """Hash of the code of the sources `kernel` is built from (every unit when
    None); comments do not count."""
    own = next((u for pre, u in OWN_UNITS.items() if kernel and kernel.startswith(pre)), None)
    csrc = os.path.join(ROOT, "paper_2402_09481_gb300", "csrc")
    units = [f for f in sorted(os.listdir(csrc)) if f.endswith(".cu")]
    if own:
        units = [f for f in units if f in own]
    elif kernel is not None:
        units = [f for f in units if f not in ("cm_vn.cu", "cm_trevisan.cu", "cm_shared_seed.cu")]
    h = hashlib.sha256()
    for path in _source_closure([os.path.join(csrc, f) for f in units]):
        h.update(os.path.relpath(path, ROOT).encode())
        with open(path, errors="replace") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


_COMMENT = re.compile(r"//[^\n]*|/\*.*?\*/", re.S)


def _code_only(text):
    """The source without its comments, blank lines and trailing spaces: what
    a comment edit leaves unchanged (no string literal in these sources holds
    a comment marker)."""
    lines = (ln.rstrip() for ln in _COMMENT.sub("", text).splitlines())
    return "\n".join(ln for ln in lines if ln)


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash(kernel)
    with open(path) as f:
        for line in f:
            p = line.split()
            if len(p) >= 4 and not line.startswith("#") and p[0] == kernel and p[1] == workload:
                return float(p[2]) if p[3] == src else None
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 100 ms, with host timestamps."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [s.strip() for s in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [s for (t, s) in self.samples if t0 <= t <= t1]
        if not inside and self.samples:
            # timed region shorter than the sampling period: nearest samples
            mid = 0.5 * (t0 + t1)
            inside = [min(self.samples, key=lambda ts: abs(ts[0] - mid))[1]]
        if not inside:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for s in inside:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if len(s) > 3 + k and s[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def field_of(kernel):
    """(kernel name without the field suffix, element bytes): the 32-bit field
    kernels carry the suffix _f30 or _f25, the Goldilocks ones none."""
    return (kernel[:-4], 4) if kernel.endswith(("_f30", "_f25")) else (kernel, 8)


def pass_split(L):
    """Column passes of a transform of length L (log2 R of each, outer first):
    none up to 2^13, one for lg - 13 <= 12, else ceil / floor halves."""
    rest = int(L).bit_length() - 1 - 13
    if rest <= 0:
        return []
    if rest <= 12:
        return [rest]
    return [(rest + 1) // 2, rest // 2]


FIELD_GL, FIELD_Q30, FIELD_Q25 = 1, 2, 3
FIELD_NAMES = {FIELD_GL: "Goldilocks p = 2^64 - 2^32 + 1", FIELD_Q30: "q = 3 * 2^30 + 1",
               FIELD_Q25: "q = 5 * 2^25 + 1"}


def element_bytes(field):
    return 8 if field == FIELD_GL else 4


def kernel_model(products, m):
    """Per-step algorithmic bytes and launches of each kernel (name without the
    field suffix), from the plan's product list (cm_plan_products), in the
    HBM model of the path: one write and one read of three L-element
    arrays per product with 8-byte field elements, 48 L bytes (a forward pass
    writes both operands, 16 L; the middle reads them and writes the product,
    24 L, or reads and writes the sum-group accumulator as well, 32 L; the
    inverse pass reads the product, 8 L), plus the bits.  "actual" is the same
    count with the path's own element size (4 bytes for the 32-bit fields)."""
    tot = {}

    def add(k, b, a):
        t = tot.setdefault(k, {"bytes": 0.0, "actual": 0.0, "launches": 0})
        t["bytes"] += b
        t["actual"] += a
        t["launches"] += 1

    for p in products:
        if p["sum"] == 4:  # dense tail: seed bits and z read, z written
            b = (p["m"] + p["tail_terms"]) / 8 + 2 * p["m"] / 8
            add("k_tail", b, b)
            continue
        L, e, s, mr = p["L"], element_bytes(p["field"]), p["sum"], p["m"]
        bits = (p["a_len"] + p["b_len"]) / 8
        split = pass_split(L)
        if not split:
            add("k_fused_small", bits + mr / 8, bits + mr / 8)
            continue
        if p["field"] == FIELD_Q25 and 2 ** 14 <= L <= 2 ** 17 and s == 0:
            # one launch on a thread-block cluster: the arrays never leave the chip
            add("k_cluster", 48 * L + bits + mr / 8, bits + mr / 8)
            continue
        for j, _ in enumerate(split):
            if j == 0:
                add("k_pass_fwd_bits", 16 * L + bits, 2 * e * L + bits)
            else:
                add("k_pass_fwd", 32 * L, 4 * e * L)
        w = 3 if s in (0, 1) else 4
        add("k_middle", 8 * w * L, e * w * L)
        if s in (0, 3):
            for j in reversed(range(len(split))):
                if j == 0:
                    add("k_pass_inv_parity", 8 * L + mr, e * L + mr)
                else:
                    add("k_pass_inv", 16 * L, 2 * e * L)
            add("k_pack", mr + mr / 8, mr + mr / 8)
    if "k_tail" in tot and tot.get("k_pack", {}).get("launches") == 1 and tot.get("k_middle"):
        # one window packed in place: the library folds the tail into that pack
        t, pk = tot.pop("k_tail"), tot.pop("k_pack")
        tot["k_pack_tail"] = {"bytes": t["bytes"] + pk["bytes"], "actual": t["actual"] + pk["actual"],
                              "launches": 1}
    return tot


# Trevisan's bit-product model uses the GPU's ALU lanes.
ALU_LANES_PER_SM = 64
NUM_SMS = 152


def path_model(products, n, seedlen, m):
    """Bytes and modular multiplies of the whole path:
    bytes48 = 48 L per product (8-byte elements) + the bit I/O once;
    bytes_actual = 6 e L per product with the path's element size e;
    modmuls_reference = 3 L (ceil(lg / 6) - 1) + L per product (the reference
    count: a radix-64 plan whose inner twiddles are shifts, as over
    Goldilocks); modmuls_radix2 = 3 (L / 2)(lg - 2) + L per product (the
    non-trivial twiddles of three radix-2 transforms and the pointwise
    product: the count without free twiddles, as over the 32-bit fields)."""
    io = (n + seedlen + m) / 8
    b48, bact, n_ref, n_r2 = io, io, 0.0, 0.0
    for p in products:
        if p["sum"] == 4:
            continue
        L = p["L"]
        lg = int(L).bit_length() - 1
        b48 += 48 * L
        bact += 6 * element_bytes(p["field"]) * L
        n_ref += 3 * L * (-(-lg // 6) - 1) + L
        n_r2 += 3 * (L // 2) * max(lg - 2, 0) + L
    return {"bytes48": b48, "bytes_actual": bact, "modmuls_reference": n_ref, "modmuls_radix2": n_r2}


def cpu_model_name():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_ntt_baseline(kind, n, m, xw, yw, z_gpu=None):
    """The bit-packed CPU NTT (cpu_ntt/) on the full workload: one thread and
    every core this process may run on (os.sched_getaffinity); None when the
    workload's transform exceeds its field (2^30)."""
    import numpy as np

    import cpu_ntt
    if cpu_ntt.transform_lg(kind, n, m) > 30:
        return None
    cores = len(os.sched_getaffinity(0))
    cpu_ntt.prepare(kind, n, m)
    t0 = time.perf_counter()
    z1 = cpu_ntt.extract(kind, xw, n, yw, m, 1)
    t1 = time.perf_counter() - t0
    tn = []
    for _ in range(3):
        t0 = time.perf_counter()
        zn = cpu_ntt.extract(kind, xw, n, yw, m, cores)
        tn.append(time.perf_counter() - t0)
    tn = statistics.median(tn)
    same = bool((z1 == zn).all())
    if z_gpu is not None:
        same = same and bool((np.asarray(z_gpu, dtype=np.uint64) == zn).all())
    return {"value": m / tn / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "cpu_ntt",
            "sample": "the whole workload, one extraction per timing (median of 3 on all cores)",
            "ms_per_step": tn * 1e3, "cpu_model": cpu_model_name(),
            "single_thread": {"value": m / t1 / 1e9, "unit": "Gbit/s", "cores": 1, "ms_per_step": t1 * 1e3},
            "bit_identical_to_gpu": same,
            "design": "C++ threads, field 3 * 2^30 + 1 (the paper's), radix-2 Shoup butterflies, "
                      "breadth-first then cache-blocked stages"}


def cpu_oracle_rate(kind, n, m, xw, yw, budget_s=12.0):
    """Oracle output bits per second on a bounded sample of output rows."""
    import numpy as np

    import oracle
    rows_fn = {0: lambda r: oracle.toeplitz_rows(xw, n, yw, m, r),
               1: lambda r: oracle.circulant_rows(xw, n, yw, m, r),
               2: lambda r: oracle.dodis_rows(xw, yw, n, m, r)}[kind]
    rng = np.random.default_rng(7)
    done, t_spent, batch = 0, 0.0, 16
    while t_spent < budget_s:
        rows = np.sort(rng.integers(0, m, size=batch))
        t0 = time.perf_counter()
        rows_fn(rows)
        t_spent += time.perf_counter() - t0
        done += batch
        batch = min(batch * 2, 4096)
    return done / t_spent, done, t_spent


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The oracle as it stands, on the host cores: each step computes a bounded
    sample of output rows of the same workload."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2402_09481_gb300 import inputs
    if args.workload == "von_neumann":
        run_reference_vn(args)
        return
    if args.workload == "trevisan":
        n, m, l = trevisan_shape()
        xw, sw = inputs.bernoulli_half(40, n), inputs.bernoulli_half(41, 2 * l * m)
        t0 = time.perf_counter()
        rates = [trevisan_reference_rate(xw, n, sw, l, 5.0)[0] for _ in range(args.steps)]
        secs = time.perf_counter() - t0
        value = statistics.median(rates) / 1e9
        print(json.dumps({"impl": "reference", "metric": "extracted output Gbit/s", "value": value,
                          "unit": "Gbit/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": 0,
                          "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "python int", "data": "synthetic",
                          "config": {"workload": f"Trevisan one-bit step: n = {n}, m = {m} RSH one-bit "
                                                 f"extractions, l = {l}", "n": n, "m": m, "l": l},
                          "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                           "sample": "one-bit extractions for 5 s per step"},
                          "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle arm for the {args.workload} workload"}))
        return
    wl = WORKLOADS[args.workload]
    kind, n, m = wl["kind"], wl["n"], wl["m"]
    xw = inputs.bernoulli_half(1, n)
    yw = inputs.bernoulli_half(2, seed_bits(kind, n, m))
    rows_per_step = int(os.environ.get("CM_REF_ROWS", "128"))
    rng = np.random.default_rng(11)
    fn = {0: lambda r: oracle.toeplitz_rows(xw, n, yw, m, r),
          1: lambda r: oracle.circulant_rows(xw, n, yw, m, r),
          2: lambda r: oracle.dodis_rows(xw, yw, n, m, r)}[kind]
    for _ in range(args.warmup):
        fn(np.sort(rng.integers(0, m, size=rows_per_step)))
    times = []
    for _ in range(args.steps):
        r = np.sort(rng.integers(0, m, size=rows_per_step))
        t0 = time.perf_counter()
        fn(r)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = rows_per_step / (ms * 1e-3) / 1e9
    sample = f"{rows_per_step} random output rows per step of the full-size workload (explicit GF(2) rows, numpy)"
    line = {
        "impl": "reference", "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": wl["name"], "n": n, "m": m},
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_vn(args):
    """Von Neumann oracle on the host cores: each step filters a 2^26-bit chunk
    of the 6.5e9-bit workload input."""
    from paper_2402_09481_gb300 import inputs
    n = int(os.environ.get("CM_VN_BITS", str(VN_BITS)))
    sample_bits = 1 << 26
    xw = inputs.bernoulli_half(30, sample_bits * 4)
    for _ in range(args.warmup):
        vn_reference_rate(xw, sample_bits * 4, 0.0)
    times, outs = [], 0
    for k in range(args.steps):
        rate, done_in, secs = vn_reference_rate(xw, sample_bits * 4, 0.0)
        times.append(secs)
        outs += rate * secs
    ms = 1e3 * sum(times) / len(times)
    value = outs / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"Von Neumann: n = {n} i.i.d. Bernoulli(1/2) bits (QRNG example length)", "n": n},
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                         "sample": "one 2^26-bit chunk of the same input per step (numpy, one thread)"},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched_a(args, world, rank, local, emit=True):
    """4096 Toeplitz extractions, n = floor(2^U), U ~ U[10, 22), m = n/2, each with
    its own Bernoulli(1/2) input and seed; one step = one replay of the planned
    batch (a single persistent work-list launch, CUDA-graph captured)."""
    import ctypes

    import numpy as np
    import torch

    from paper_2402_09481_gb300 import build, inputs, native

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    count = int(os.environ.get("CM_BATCH_COUNT", "4096"))
    ns = inputs.loguniform_lengths(1, count, 10, 22)
    ms = ns // 2
    xw_off = np.concatenate([[0], np.cumsum((ns + 63) // 64)])
    yw_off = np.concatenate([[0], np.cumsum((ns + ms - 1 + 63) // 64)])
    zw_off = np.concatenate([[0], np.cumsum((ms + 63) // 64)])
    xh = np.empty(int(xw_off[-1]), dtype=np.uint64)
    yh = np.empty(int(yw_off[-1]), dtype=np.uint64)
    for j in range(count):
        xh[xw_off[j]:xw_off[j + 1]] = inputs.bernoulli_half(10000 + 2 * j + 100000 * rank, int(ns[j]))
        yh[yw_off[j]:yw_off[j + 1]] = inputs.bernoulli_half(10001 + 2 * j + 100000 * rank,
                                                            int(ns[j] + ms[j] - 1))
    xd = torch.from_numpy(xh.view(np.int64)).cuda()
    yd = torch.from_numpy(yh.view(np.int64)).cuda()
    zd = torch.zeros(int(zw_off[-1]), dtype=torch.int64, device="cuda")
    ctx = native.Context(local)
    arr = (native.CmDesc * count)()
    for j in range(count):
        arr[j] = native.CmDesc(native.TOEPLITZ, 0, int(ns[j]), int(ms[j]),
                               xd.data_ptr() + 8 * int(xw_off[j]), yd.data_ptr() + 8 * int(yw_off[j]),
                               zd.data_ptr() + 8 * int(zw_off[j]))
    h = ctypes.c_void_p()
    t0 = time.time()
    st = native.lib().cm_batch_create(ctx.handle, ctypes.cast(arr, ctypes.c_void_p), count,
                                      native.BATCH_AUTOTUNE, ctypes.byref(h))
    if st != native.CM_OK:
        raise native.CMError(st, "cm_batch_create")
    b = native.Batch(ctx, h, [])
    plan_s = time.time() - t0
    info = b.info()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.launch()
    torch.cuda.synchronize()
    z_ref = zd.clone()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    for k in range(args.steps):
        ev[k][0].record(stream)
        b.launch()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    tw1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    out_bits = int(ms.sum())
    value = world * out_bits / (ms_per_step * 1e-3) / 1e9
    assert torch.equal(zd, z_ref), "replays differ"
    s_, f_ = ctx.device_status()
    if s_ != native.CM_OK:
        raise RuntimeError(f"device status {native.STATUS.get(s_)} flags {f_}")

    # the plain per-call form on the same inputs: one cm_toeplitz per instance
    compare = os.environ.get("CM_BENCH_NO_COMPARE") != "1"
    zp = zd.clone() if not compare else torch.zeros_like(zd)
    L_ = native.lib()
    sh = stream.cuda_stream

    def plain():
        for j in range(count):
            r = L_.cm_toeplitz(ctx.handle, arr[j].x, int(ns[j]), arr[j].y, int(ms[j]),
                               zp.data_ptr() + 8 * int(zw_off[j]), sh)
            if r != native.CM_OK:
                raise native.CMError(r, "cm_toeplitz")
    if compare:
        plain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_ms = [float("nan")]
    for _ in range(max(1, min(3, args.steps)) if compare else 0):
        e0.record(stream)
        plain()
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    if compare:
        plain_ms = plain_ms[1:]
    assert torch.equal(zp, zd), "batched output differs from the per-call output"
    plain_value = world * out_bits / (statistics.median(plain_ms) * 1e-3) / 1e9

    # roofline of the work-list kernel (the only kernel of a step), in the
    # path's HBM model: 48 L bytes per instance with 8-byte
    # elements (on-chip instances, L <= 2^13: the bits only) + the bit I/O; the
    # work list runs 4-byte elements, so it moves about half of that.  k_batch
    # runs the instances of the work list (L <= 2^21); the longer ones run the
    # single-call kernels in the same graph and count in the step's figure only
    Ls = np.array([native.plan_query(native.TOEPLITZ, int(n), int(m), plan_mode=native.PLAN_SINGLE)
                   ["transform_length"] for n, m in zip(ns, ms)])
    onlist = Ls <= (1 << 21)
    if int((~onlist).sum()) != int(info["solo_instances"]):
        raise RuntimeError("work-list split differs from the batch's own")
    big = (Ls > (1 << 13)) & onlist
    bits = (ns + (ns + ms - 1) + ms) / 8
    io = float(bits[onlist].sum())
    alg = float(48 * Ls[big].sum()) + io
    act = float(24 * Ls[big].sum()) + io
    alg_step = float(48 * Ls[Ls > (1 << 13)].sum() + bits.sum())
    peak, peak_src = measured_peaks()
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    for _ in range(args.steps):
        b.launch()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    kb = prof.get("k_batch", (1, ms_per_step))
    per_launch = kb[1] / kb[0]
    achieved = alg / (per_launch * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_batch", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "traffic": ncu_traffic("k_batch", "batched_a") if count == 4096 else None,  # the figure is for 4096
            "model": "48 L bytes per work-list instance with 2^13 < L <= 2^21 (8-byte elements) + their bit I/O",
            "algorithmic_bytes_per_launch": alg, "avg_launch_ms": per_launch,
            "work_list_instances": int(onlist.sum()), "single_call_instances": int((~onlist).sum()),
            "actual_element_bytes": {"bytes_per_launch": act, "achieved": act / (per_launch * 1e-3) / 1e9,
                                     "frac": act / (per_launch * 1e-3) / 1e9 / peak},
            "step": {"bytes": alg_step, "achieved": alg_step / (ms_per_step * 1e-3) / 1e9,
                     "frac": alg_step / (ms_per_step * 1e-3) / 1e9 / peak,
                     "model": "48 L bytes per instance with L > 2^13 + all bit I/O, over the whole step"}}

    # end to end: host inputs (pinned) -> device, batch, outputs -> host
    xp = torch.from_numpy(xh.view(np.int64)).pin_memory()
    yp = torch.from_numpy(yh.view(np.int64)).pin_memory()
    zh = torch.empty(zd.numel(), dtype=torch.int64).pin_memory()
    e2e_ms = []
    for _ in range(max(1, min(3, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd.copy_(xp, non_blocking=True)
        yd.copy_(yp, non_blocking=True)
        b.launch()
        zh.copy_(zd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": world * out_bits / (e2e_mean * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": 8 * (xh.size + yh.size), "d2h_bytes_per_step": 8 * int(zw_off[-1]),
           "ms_per_step": e2e_mean}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(3)
        done, secs = 0, 0.0
        while secs < 10.0:
            j = int(rng.integers(0, count))
            rows = np.sort(rng.integers(0, int(ms[j]), size=32))
            t0 = time.perf_counter()
            oracle.toeplitz_rows(xh[xw_off[j]:xw_off[j + 1]], int(ns[j]), yh[yw_off[j]:yw_off[j + 1]],
                                 int(ms[j]), rows)
            secs += time.perf_counter() - t0
            done += 32
        cpu = {"value": done / secs / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} output rows from random instances of the batch in {secs:.1f} s "
                         "(explicit GF(2) rows, numpy, one thread)"}
    clocks = sampler.summary(tw0, tw1)
    if rank == 0:
        line = {
            "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"Batched Toeplitz: {count} instances, n = floor(2^U), U ~ U[10, 22), "
                                   "m = floor(n/2), own Bernoulli(1/2) x and seed each",
                       "sum_n": int(ns.sum()), "sum_m": out_bits, "sum_L": int(Ls.sum()),
                       "l2": "working set (scratch %.1f GB) far larger than L2" % (info["scratch_bytes"] / 1e9),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "batch": {"work_items": info["work_items"], "tile_lg": info["tile_lg"], "grid": info["grid"],
                      "graph": info["graph"], "plan_seconds": plan_s},
            "plain_per_call": {"value": plain_value, "unit": "Gbit/s",
                               "ms_per_step": statistics.median(plain_ms),
                               "launches_per_step": sum(native.launch_count(native.TOEPLITZ, int(n), int(m))
                                                        for n, m in zip(ns, ms))},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": max(step_ms)},
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(info["kernel_launches"]) * args.steps,
        }
        if emit:
            print(json.dumps(line), flush=True)
    b.close()
    ctx.close()
    del xd, yd, zd, zp
    torch.cuda.empty_cache()
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_batched_b(args, world, rank, local):
    """65,536 inputs of n = 4096 bits under one shared Toeplitz seed, m = 2048:
    one step = the whole dense product toep(y) X over GF(2) (engine chosen by
    the library's autotuner), compared in the same run with each engine, the
    NTT work-list batch and the plain per-call NTT."""
    import ctypes

    import numpy as np
    import torch

    from paper_2402_09481_gb300 import build, inputs, native

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    count = int(os.environ.get("CM_SS_COUNT", "65536"))
    n, m = 4096, 2048
    wx, wz = n // 64, m // 64
    yw = inputs.bernoulli_half(20 + 1000 * rank, n + m - 1)
    X = inputs.bernoulli_half(21 + 1000 * rank, n * count)   # inputs back to back (n = 64 words each)
    Xd = torch.from_numpy(X.view(np.int64)).cuda()
    yd = torch.from_numpy(yw.view(np.int64)).cuda()
    Z = torch.zeros(wz * count, dtype=torch.int64, device="cuda")
    ctx = native.Context(local)
    stream = torch.cuda.current_stream()
    ctx.toeplitz_shared_seed(yd, n, m, Xd, count, Z)   # settles the AUTO engine
    engine = native.lib().cm_shared_seed_engine(n, m)

    def step(e=native.ENGINE_AUTO):
        ctx.toeplitz_shared_seed(yd, n, m, Xd, count, Z, engine=e)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    if dist:
        dist.barrier()
    tw0 = time.time()
    step_ms = timed(step, args.steps)
    tw1 = time.time()
    if dist:
        dist.barrier()
    time.sleep(0.25)
    sampler.stop()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    out_bits = count * m
    value = world * out_bits / (ms_per_step * 1e-3) / 1e9
    z_ref = Z.clone()

    others = {}
    compare = os.environ.get("CM_BENCH_NO_COMPARE") != "1"
    for name, e in ((("imma", native.ENGINE_IMMA), ("gf2", native.ENGINE_GF2), ("bmma", native.ENGINE_BMMA))
                    if compare else ()):
        Z.zero_()
        t = statistics.median(timed(lambda e=e: step(e), max(3, min(args.steps, 10))))
        assert torch.equal(Z, z_ref), name
        others[name] = {"value": world * out_bits / (t * 1e-3) / 1e9, "unit": "Gbit/s", "ms_per_step": t}
    # the NTT paths on the same inputs (each input its own Toeplitz extraction)
    Zn = torch.zeros_like(Z)
    count_cmp = count if compare else 0
    if compare:
        items = [(native.TOEPLITZ, n, m, Xd[c * wx:(c + 1) * wx], yd, Zn[c * wz:(c + 1) * wz])
                 for c in range(count_cmp)]
        b = ctx.batch(items, autotune=False)
        t = statistics.median(timed(b.launch, 3))
        assert torch.equal(Zn, z_ref), "ntt batch"
        others["ntt_worklist_batch"] = {"value": world * out_bits / (t * 1e-3) / 1e9, "unit": "Gbit/s",
                                        "ms_per_step": t}
        b.close()
        Zn.zero_()
        L_ = native.lib()
        sh = stream.cuda_stream

        def per_call():
            for c in range(count):
                L_.cm_toeplitz(ctx.handle, Xd.data_ptr() + 8 * wx * c, n, yd.data_ptr(), m,
                               Zn.data_ptr() + 8 * wz * c, sh)
        t = statistics.median(timed(per_call, 1))
        assert torch.equal(Zn, z_ref), "per call"
        others["plain_per_call_ntt"] = {"value": world * out_bits / (t * 1e-3) / 1e9, "unit": "Gbit/s",
                                        "ms_per_step": t}

    # roofline of the dense kernel
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    for _ in range(args.steps):
        step()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    kname = {native.ENGINE_GF2: "k_ss_gf2", native.ENGINE_BMMA: "k_ss_bmma"}.get(engine, "k_ss_imma")
    c_, t_ = prof[kname]
    per_launch = t_ / c_
    clocks = sampler.summary(tw0, tw1)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    if engine == native.ENGINE_GF2:
        ops = count * m * (n // 32)           # LOP3 (32 AND + 32 XOR) per (output bit, 32-bit word)
        peak = 152 * 64 * sm_mhz * 1e6        # ALU pipe: 64 lanes per SM per clock
        roof = {"bound": "alu", "kernel": kname, "achieved": ops / (per_launch * 1e-3) / 1e12,
                "peak": peak / 1e12, "unit": "T LOP3/s", "frac": ops / (per_launch * 1e-3) / peak,
                "peak_source": "152 SMs x 64 ALU lanes x measured SM clock",
                "traffic": ncu_traffic(kname, "batched_b"), "avg_launch_ms": per_launch}
    elif engine == native.ENGINE_BMMA:
        # algorithmic HBM bytes: the inputs once, the outputs once, the expanded matrix once
        alg = 8 * X.size + 8 * Z.numel() + (m + 63) // 64 * 64 * ((n + 1023) // 1024 * 1024) // 8
        hbm, hbm_src = measured_peaks()
        roof = {"bound": "hbm", "kernel": kname, "achieved": alg / (per_launch * 1e-3) / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": alg / (per_launch * 1e-3) / 1e9 / hbm,
                "peak_source": f"{hbm_src} HBM copy bandwidth (MEASURED_PEAKS.json)",
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": per_launch,
                "traffic": ncu_traffic(kname, "batched_b"),
                "b1_tensor_ops": {"value": count * m * n / (per_launch * 1e-3) / 1e12, "unit": "T bit-AND-POPC/s",
                                  "note": "no measured or nominal peak for b1 MMA on this GPU"}}
    else:
        ops = 2 * count * m * n
        roof = {"bound": "tensor", "kernel": kname, "achieved": ops / (per_launch * 1e-3) / 1e12,
                "peak": None, "unit": "T int8 op/s", "frac": None, "avg_launch_ms": per_launch,
                "traffic": ncu_traffic(kname, "batched_b")}
    # end to end: inputs from pinned host memory, outputs back
    Xp = torch.from_numpy(X.view(np.int64)).pin_memory()
    Zh = torch.empty_like(Z, device="cpu").pin_memory()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd.copy_(Xp, non_blocking=True)
        step()
        Zh.copy_(Z, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": world * out_bits / (e2e_mean * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": 8 * X.size, "d2h_bytes_per_step": 8 * Z.numel(), "ms_per_step": e2e_mean}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(5)
        done, secs = 0, 0.0
        while secs < 10.0:
            c = int(rng.integers(0, count))
            t0 = time.perf_counter()
            oracle.toeplitz_packed(X[c * wx:(c + 1) * wx], n, yw, m)
            secs += time.perf_counter() - t0
            done += m
        cpu = {"value": done / secs / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
               "sample": f"{done // m} whole inputs ({done} output bits) in {secs:.1f} s "
                         "(explicit GF(2) rows, numpy, one thread)"}
    if rank == 0:
        line = {
            "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": {native.ENGINE_GF2: "u32 (GF(2) words)",
                                                                 native.ENGINE_BMMA: "b1"}.get(engine, "s8"),
            "data": "synthetic",
            "config": {"workload": f"Shared Toeplitz seed: {count} inputs of n = 4096 bits, m = 2048, "
                                   "Bernoulli(1/2)", "engine": {1: "imma", 2: "gf2", 3: "bmma"}.get(engine),
                       "l2": "inputs (%d MB) larger than L2" % (8 * X.size >> 20),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "compare": others, "latency_ms": {"p50": statistics.median(step_ms), "p99": max(step_ms)},
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


VN_BITS = 6_500_000_000   # the input length of the paper's QRNG example


def vn_reference_rate(xw, n, budget_s, chunk_bits=1 << 26):
    """The Von Neumann oracle as it stands on consecutive chunks of the input,
    for about budget_s seconds: (output bits per second, input bits done, s)."""
    import oracle.von_neumann as ovn
    from oracle.extractors import unpack_bits
    done_in, done_out, secs, off = 0, 0, 0.0, 0
    while done_in == 0 or secs < budget_s:
        w0 = (off // 64) % max(1, (n - chunk_bits) // 64)
        t0 = time.perf_counter()
        out = ovn.von_neumann(unpack_bits(xw[w0:w0 + chunk_bits // 64], chunk_bits))
        secs += time.perf_counter() - t0
        done_in += chunk_bits
        done_out += out.size
        off += chunk_bits
    return done_out / secs, done_in, secs


def run_von_neumann(args, world, rank, local):
    """Von Neumann extraction (Alg. vn) of n = 6.5e9 i.i.d. Bernoulli(1/2) bits
    (the input length of the paper's QRNG example): one step = one
    cm_von_neumann call (pair filter + order-keeping compaction, one kernel)."""
    import numpy as np
    import torch

    from paper_2402_09481_gb300 import build, inputs, native

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    n = int(os.environ.get("CM_VN_BITS", str(VN_BITS)))
    xw = inputs.bernoulli_half(30 + 1000 * rank, n)
    xd = torch.from_numpy(xw.view(np.int64)).cuda()
    zd = torch.empty(native.words(n // 2), dtype=torch.int64, device="cuda")
    md = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx = native.Context(local)
    stream = torch.cuda.current_stream()

    def step():
        ctx.von_neumann(xd, n, zd, md)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    m = int(md.item())
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    time.sleep(0.25)
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * m / (ms_per_step * 1e-3) / 1e9
    # kernel time from the library's launch events (same stream)
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    for _ in range(args.steps):
        step()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    words = (2 * (n // 2) + 63) // 64
    out_bytes = 8 * ((m + 63) // 64)
    alg = {"k_vn_count": 8 * words, "k_vn_zero": None, "k_vn_write": 8 * words + out_bytes}
    kern = {}
    for name in ("k_vn_count", "k_vn_zero", "k_vn_write"):
        c_, t_ = prof[name]
        kern[name] = {"launches": c_, "avg_ms": t_ / c_}
    tot = sum(k["avg_ms"] for k in kern.values())
    for k in kern.values():
        k["share"] = k["avg_ms"] / tot
    top = max(kern, key=lambda k: kern[k]["avg_ms"])
    per_launch = kern[top]["avg_ms"]
    hbm_peak, peak_src = measured_peaks()
    achieved = alg[top] / (per_launch * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_source": peak_src,
            "traffic": ncu_traffic(top, "von_neumann"), "algorithmic_bytes_per_launch": alg[top],
            "avg_launch_ms": per_launch}
    # the whole path against one read of the input and one write of the output
    single = 8 * words + out_bytes
    path = {"algorithmic_bytes": single, "achieved_gbs": single / (ms_per_step * 1e-3) / 1e9,
            "frac_of_measured_hbm": single / (ms_per_step * 1e-3) / 1e9 / hbm_peak,
            "note": "two passes over the input: the count pass and the write pass"}
    # end to end through the host-buffer entry point
    xh = torch.from_numpy(xw.view(np.int64)).pin_memory()
    zh = torch.empty(native.words(n // 2), dtype=torch.int64).pin_memory()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        s_, m_e = ctx.von_neumann_host(xh, n, zh)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        assert s_ == native.CM_OK and m_e == m
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": world * m / (e2e_mean * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": 8 * ((n + 63) // 64), "d2h_bytes_per_step": 8 + 8 * ((m + 63) // 64),
           "ms_per_step": e2e_mean}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, done_in, secs = vn_reference_rate(xw, n, 10.0)
        cpu = {"value": rate / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
               "sample": f"{done_in} input bits in 2^26-bit chunks of the same input in {secs:.1f} s "
                         "(array form of the pair filter, numpy, one thread)"}
    if rank == 0:
        line = {
            "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (bit words)",
            "data": "synthetic",
            "config": {"workload": f"Von Neumann: n = {n} i.i.d. Bernoulli(1/2) bits (QRNG example length)",
                       "n": n, "m": m, "input_gbit_per_s": world * n / (ms_per_step * 1e-3) / 1e9,
                       "l2": "input (%d MB) larger than L2" % (8 * words >> 20),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": max(step_ms)},
            "roofline": roof, "path_roofline": path, "kernels": kern, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": sampler.summary(tw0, tw1), "gpu_launches": 3 * args.steps,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


TREV_N, TREV_M, TREV_EPS = 1 << 20, 1 << 16, 1e-10


def trevisan_shape():
    """n, m, l of the Trevisan one-bit-step workload: l from the per-bit error
    eps / m (the total error eps = m eps1)."""
    import math
    l = math.ceil(math.log2(TREV_N) + 2 * math.log2(2.0 / (TREV_EPS / TREV_M)))
    return TREV_N, TREV_M, l


def trevisan_reference_rate(xw, n, sw, l, budget_s):
    """Oracle one-bit extractions per second on the first outputs."""
    import oracle.trevisan as otv
    from oracle import extractors as ex
    xb = ex.unpack_bits(xw, n)
    f = otv.rsh_modulus(l)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        sb = ex.unpack_bits(sw, 2 * l * (done + 1))[2 * l * done:]
        otv.rsh_onebit(xb, n, sb, l, f)
        done += 1
    secs = time.perf_counter() - t0
    return done / secs, done, secs


def run_trevisan(args, world, rank, local):
    """Trevisan's one-bit step (Section "Trevisan implementation"): m = 2^16
    Reed-Solomon-Hadamard one-bit extractions of one input of n = 2^20
    Bernoulli(1/2) bits, each under its own 2l-bit seed (standing for the
    weak design's sub-seeds), l = ceil(log2 n + 2 log2(2 m / eps)), eps = 1e-10.
    One step = one cm_trevisan_rsh call."""
    import numpy as np
    import torch

    from paper_2402_09481_gb300 import build, inputs, native

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    n, m, l = trevisan_shape()
    xw = inputs.bernoulli_half(40 + 1000 * rank, n)
    sw = inputs.bernoulli_half(41 + 1000 * rank, 2 * l * m)
    xd = torch.from_numpy(xw.view(np.int64)).cuda()
    sd = torch.from_numpy(sw.view(np.int64)).cuda()
    zd = torch.empty(native.words(m), dtype=torch.int64, device="cuda")
    ctx = native.Context(local)
    stream = torch.cuda.current_stream()

    def step():
        ctx.trevisan_rsh(xd, n, l, sd, m, zd)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    time.sleep(0.25)
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * m / (ms_per_step * 1e-3) / 1e9
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    for _ in range(args.steps):
        step()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    c_, t_ = prof["k_rsh"]
    per_launch = t_ / c_
    s = -(-n // l)
    # schoolbook GF(2) work: (s - 1) products of l-bit polynomials (l^2 bit
    # AND-XORs each) per output; one LOP3 does 32 of them on one lane
    macs = float(m) * (s - 1) * l * l
    clk = (sampler.summary(tw0, tw1) or {}).get("sm_mhz") or 2070.0
    peak = NUM_SMS * ALU_LANES_PER_SM * clk * 1e6 * 32 / 1e9
    ach = macs / (per_launch * 1e-3) / 1e9
    roof = {"bound": "alu", "kernel": "k_rsh", "achieved": ach, "peak": peak, "unit": "G GF(2) bit-MACs/s",
            "frac": ach / peak,
            "peak_source": f"{NUM_SMS} SMs x {ALU_LANES_PER_SM} ALU lanes x {clk:.0f} MHz measured x 32 "
                           "(one LOP3 = 32 AND + 32 XOR)",
            "traffic": ncu_traffic("k_rsh", "trevisan"), "avg_launch_ms": per_launch,
            "gf2_bit_macs_per_launch": macs}
    # end to end: input and seeds from pinned host memory, output back
    xh = torch.from_numpy(xw.view(np.int64)).pin_memory()
    sh = torch.from_numpy(sw.view(np.int64)).pin_memory()
    zh = torch.empty(native.words(m), dtype=torch.int64).pin_memory()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd.copy_(xh, non_blocking=True)
        sd.copy_(sh, non_blocking=True)
        step()
        zh.copy_(zd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": world * m / (e2e_mean * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": 8 * (xw.size + sw.size), "d2h_bytes_per_step": 8 * native.words(m),
           "ms_per_step": e2e_mean}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, done, secs = trevisan_reference_rate(xw, n, sw, l, 10.0)
        cpu = {"value": rate / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} output bits (one-bit extractions) in {secs:.1f} s (Python integers, one thread)"}
    if rank == 0:
        line = {
            "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (GF(2^l) words)",
            "data": "synthetic",
            "config": {"workload": f"Trevisan one-bit step: n = {n} Bernoulli(1/2) input bits, m = {m} RSH "
                                   f"one-bit extractions, l = {l} (eps = {TREV_EPS}), random 2l-bit seeds",
                       "n": n, "m": m, "l": l, "chunks": s, "modulus_taps": native.rsh_modulus(l),
                       "l2": "input and chunks L2-resident (read by every thread)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": max(step_ms)},
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": sampler.summary(tw0, tw1), "gpu_launches": 2 * args.steps,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def served_trace(count, rate, seed_stream=3):
    """Poisson arrivals at `rate`/s; kinds Toeplitz / Circulant / Dodis et al.
    50/25/25; n = floor(2^U), U ~ U[12, 28), snapped to the next valid N_A
    length for Circulant (n + 1 prime) and Dodis et al. (n prime), the previous
    one above 2^28; m = floor(n / 2)."""
    import numpy as np

    from paper_2402_09481_gb300 import inputs, native
    arr = inputs.poisson_arrivals(seed_stream, count, rate)
    u = inputs.uniform01(seed_stream + 1, count)
    ns = inputs.loguniform_lengths(seed_stream + 2, count, 12, 28)
    out = []
    for j in range(count):
        kind = 0 if u[j] < 0.5 else (1 if u[j] < 0.75 else 2)
        n = int(ns[j])
        if kind == 1:
            P = native.next_na_prime(n + 1)
            if P > (1 << 28):
                P = native.prev_na_prime(n + 1)
            n = P - 1
        elif kind == 2:
            P = native.next_na_prime(n)
            if P > (1 << 28):
                P = native.prev_na_prime(n)
            n = P
        out.append((float(arr[j]), kind, n, max(1, n // 2)))
    return out


def run_served(args, world, rank, local, emit=True):
    """Requests of the served workload submitted at their arrival times to the
    library's continuous-batching server; end-to-end latency (arrival to
    completion), service time (admission to completion) and output Gbit/s at
    the 20k req/s rate and at fractions of the measured capacity."""
    import threading

    import numpy as np
    import torch

    from paper_2402_09481_gb300 import build, native

    torch.cuda.set_device(local)
    if rank != 0:
        return
    build.build()
    ctx = native.Context(local)
    express = int(os.environ.get("CM_SERVE_EXPRESS", "1"))
    streams = int(os.environ.get("CM_SERVE_SLOTS", "0"))  # 0: the server's default, 3 streams
    ctx.server_start(slots=streams,
                     express_slots=express if express > 0 else native.SERVER_NO_EXPRESS)
    pool_bits = (1 << 29) + (1 << 24)
    xpool = torch.randint(-(1 << 62), 1 << 62, ((pool_bits + 63) // 64,), dtype=torch.int64, device="cuda")
    ypool = torch.randint(-(1 << 62), 1 << 62, ((pool_bits + 63) // 64,), dtype=torch.int64, device="cuda")

    def run(trace):
        zwords = [native.words(m) for _, _, _, m in trace]
        zbuf = torch.empty(sum(zwords), dtype=torch.int64, device="cuda")
        zoff = np.concatenate([[0], np.cumsum(zwords)])
        rng = np.random.default_rng(len(trace))
        tickets, arrive, offs = [None] * len(trace), [0] * len(trace), [None] * len(trace)
        t0 = time.monotonic_ns() + 20_000_000

        def client():
            for j, (ta, kind, n, m) in enumerate(trace):
                due = t0 + int(ta * 1e9)
                while True:
                    d = due - time.monotonic_ns()
                    if d <= 0:
                        break
                    time.sleep(min(d, 2_000_000) / 1e9)
                ox, oy = int(rng.integers(0, 1 << 18)), int(rng.integers(0, 1 << 18))
                offs[j] = (ox, oy)
                arrive[j] = max(due, time.monotonic_ns())
                s, t = ctx.submit_raw(kind, n, m, xpool.data_ptr() + 8 * ox, ypool.data_ptr() + 8 * oy,
                                      zbuf.data_ptr() + 8 * int(zoff[j]))
                if s != native.CM_OK:
                    raise native.CMError(s, "cm_submit")
                tickets[j] = t

        th = threading.Thread(target=client)
        th.start()
        th.join()
        res = []
        for t in tickets:
            s, r = ctx.poll(t, 600.0)
            if s != native.CM_OK or r["status"] != native.CM_OK:
                raise RuntimeError(f"request failed: {native.STATUS.get(s)} {r}")
            res.append(r)
        lat = np.array([(r["t_done_ns"] - a) / 1e6 for r, a in zip(res, arrive)])
        svc = np.array([(r["t_done_ns"] - r["t_admit_ns"]) / 1e6 for r in res])
        span = (max(r["t_done_ns"] for r in res) - min(arrive)) / 1e9
        bits = sum(m for _, _, _, m in trace)
        stats = {"requests": len(trace), "output_gbits": bits / 1e9, "span_s": span,
                 "gbit_per_s": bits / span / 1e9, "req_per_s": len(trace) / span,
                 "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                 "service_ms": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
                 "waves": ctx.server_stats()["waves"], "_lat": lat.tolist()}
        return stats, zbuf, zoff, offs

    def plain(trace, zoff, offs, z):
        """The same requests and inputs as plain single calls, back to back on one stream."""
        Lb = native.lib()
        sh = torch.cuda.current_stream().cuda_stream
        for j, (_, kind, n, m) in enumerate(trace):
            px, py = xpool.data_ptr() + 8 * offs[j][0], ypool.data_ptr() + 8 * offs[j][1]
            pz = z.data_ptr() + 8 * int(zoff[j])
            if kind == 0:
                r = Lb.cm_toeplitz(ctx.handle, px, n, py, m, pz, sh)
            elif kind == 1:
                r = Lb.cm_circulant(ctx.handle, px, n, py, m, pz, sh)
            else:
                r = Lb.cm_dodis(ctx.handle, px, py, n, m, pz, sh)
            if r != native.CM_OK:
                raise native.CMError(r, "single call")

    def alone_ms(trace, zoff, offs):
        """Each request's time as a plain single call (CUDA events around it on
        one stream), and whether those outputs equal the served ones."""
        z = torch.zeros(int(zoff[-1]), dtype=torch.int64, device="cuda")
        sh = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in trace]
        for j in range(len(trace)):
            ev[j][0].record(sh)
            plain(trace[j:j + 1], zoff[j:j + 2] - zoff[j], [offs[j]], z[int(zoff[j]):])
            ev[j][1].record(sh)
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ev]), z

    def slowdown(stats, trace, zs, zoff, offs):
        """Served latency over the request's time alone, p50 / p99 (1 = no
        waiting behind other requests)."""
        t_alone, z = alone_ms(trace, zoff, offs)
        assert torch.equal(z, zs), "served outputs differ from the per-call outputs"
        r = np.array(stats.pop("_lat")) / np.maximum(t_alone, 1e-3)
        stats["slowdown"] = {"p50": float(np.percentile(r, 50)), "p99": float(np.percentile(r, 99)),
                             "alone_ms_p50": float(np.percentile(t_alone, 50)),
                             "alone_ms_p99": float(np.percentile(t_alone, 99))}
        return stats

    rate = float(os.environ.get("CM_SERVE_RATE", "20000"))
    count = int(os.environ.get("CM_SERVE_COUNT", "600"))
    run(served_trace(max(8, args.warmup * 4), rate, seed_stream=90))   # warm-up (its outputs are not kept)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    tw0 = time.time()
    trace = served_trace(count, rate)
    # three runs of the same trace (bit-identical outputs); the line reports
    # the run of median throughput, and the plain form below likewise
    runs = [run(trace) for _ in range(3)]
    for r_ in runs[1:]:
        assert torch.equal(r_[1], runs[0][1]), "served outputs differ between runs of one trace"
    runs.sort(key=lambda r_: r_[0]["gbit_per_s"])
    main_run, zs, zoff, offs = runs[1]
    main_run["gbit_per_s_runs"] = [r_[0]["gbit_per_s"] for r_ in runs]
    tw1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    slowdown(main_run, trace, zs, zoff, offs)
    # the plain per-call form on the same trace: outputs bit-identical, GPU
    # time of the calls back to back (their host-side enqueue included)
    zp = torch.zeros_like(zs)
    plain(trace, zoff, offs, zp)
    torch.cuda.synchronize()
    same = bool(torch.equal(zp, zs))
    p_ms = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plain(trace, zoff, offs, zp)
        e1.record()
        torch.cuda.synchronize()
        p_ms.append(e0.elapsed_time(e1))
    bits = sum(m for _, _, _, m in trace)
    assert same, "served outputs differ from the per-call outputs"

    def plain_paced():
        """The plain per-call form as a queue alone: each request becomes one
        single call on one stream at its arrival time (the served run's
        schedule); span from the first arrival to the last completion."""
        zq = torch.zeros_like(zs)
        sh = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.monotonic_ns() + 20_000_000
        for j, (ta, _, _, _) in enumerate(trace):
            due = t0 + int(ta * 1e9)
            while True:
                d = due - time.monotonic_ns()
                if d <= 0:
                    break
                time.sleep(min(d, 2_000_000) / 1e9)
            if j == 0:
                e0.record(sh)
            plain(trace[j:j + 1], zoff[j:j + 2] - zoff[j], [offs[j]], zq[int(zoff[j]):])
        e1.record(sh)
        torch.cuda.synchronize()
        assert torch.equal(zq, zs), "paced per-call outputs differ from the served ones"
        return e0.elapsed_time(e1)

    paced_runs = sorted(plain_paced() for _ in range(3))
    paced_ms = paced_runs[1]
    plain_stats = {"value": bits / (paced_ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms": paced_ms,
                   "gbit_per_s_runs": [bits / (t * 1e-3) / 1e9 for t in paced_runs[::-1]],
                   "form": "one single call per request on one stream at its arrival time (a queue alone)",
                   "bit_identical_to_served": same,
                   "back_to_back": {"value": bits / (min(p_ms) * 1e-3) / 1e9, "unit": "Gbit/s", "ms": min(p_ms),
                                    "form": "every request's single call enqueued at once, no arrival times"}}
    cap = main_run["req_per_s"]
    points = []
    for frac in (0.25, 0.5, 0.8):
        k = int(os.environ.get("CM_SERVE_SUB_COUNT", "120"))
        tr = served_trace(k, frac * cap, seed_stream=30 + int(frac * 100))
        pt, zq, zoq, ofq = run(tr)
        slowdown(pt, tr, zq, zoq, ofq)
        pt["offered_fraction_of_capacity"] = frac
        points.append(pt)
    st = ctx.server_stats()
    line = {
        "metric": "extracted output Gbit/s", "value": main_run["gbit_per_s"], "unit": "Gbit/s", "n_gpus": 1,
        "steps": 1, "warmup": args.warmup, "ms_per_step": main_run["span_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"Served: {count} requests, Poisson arrivals at {rate:g} req/s, Toeplitz/Circulant/"
                               "Dodis 50/25/25, n = floor(2^U), U ~ U[12, 28) (N_A-snapped), m = n/2, "
                               "Bernoulli(1/2) inputs", "streams": (st["slots"] - max(express, 0)) // 2,
                   "wave_slots": st["slots"],
                   "express_slots": max(express, 0),
                   "hbm_budget_bytes": st["budget_bytes"]},
        "served": main_run, "plain_per_call": plain_stats, "sub_saturation": points,
        "latency_ms": main_run["latency_ms"], "max_inflight_bytes": st["max_inflight_bytes"],
        "clocks": sampler.summary(tw0, tw1),
    }
    if emit:
        print(json.dumps(line), flush=True)
    ctx.server_stop()
    ctx.close()
    del xpool, ypool, zs, zp
    torch.cuda.empty_cache()
    return line


def roofline_of(prof, products, m, peak, peak_src, workload):
    """The dominant kernel's roofline: algorithmic bytes per launch (the scope's
    48 L model, with the path's own element size beside it) over its average
    launch time, against the measured HBM copy bandwidth."""
    kernels = {k: {"launches": c, "avg_ms": t / c, "share": 0.0} for k, (c, t) in prof.items()}
    tot = sum(t for _, t in prof.values()) or 1.0
    for k, (c, t) in prof.items():
        kernels[k]["share"] = t / tot
    dom = max(prof, key=lambda k: prof[k][1])
    per_launch = prof[dom][1] / prof[dom][0]
    base = dom[:-4] if dom.endswith(("_f30", "_f25")) else dom
    model = kernel_model(products, m).get(base)
    if not model:
        return None, kernels
    alg = model["bytes"] / model["launches"]
    act = model["actual"] / model["launches"]
    achieved = alg / (per_launch * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic(dom, workload),
            "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "model": "48 L bytes per product (three L-element arrays written and read once, "
                     "8-byte elements) split over the kernels, per launch",
            "algorithmic_bytes_per_launch": alg, "avg_launch_ms": per_launch,
            "launches_per_step": model["launches"],
            "actual_element_bytes": {"bytes_per_launch": act,
                                     "achieved": act / (per_launch * 1e-3) / 1e9,
                                     "frac": act / (per_launch * 1e-3) / 1e9 / peak}}
    return roof, kernels


def path_roofline_of(products, n, sb, m, ms_per_step, peak, rates):
    """The scope's path roofline: max(T_hbm, T_int) against the measured step
    time; T_hbm = the 48 L bytes (and the actual ones) over the measured HBM
    copy bandwidth, T_int = modular multiplies over the measured rate of the
    product of each product's own field (cm_modmul_rate)."""
    pm = path_model(products, n, sb, m)
    # modular multiplies per field
    t_ref = t_r2 = 0.0
    fields = set()
    for p in products:
        if p["sum"] == 4:
            continue
        L = p["L"]
        lg = int(L).bit_length() - 1
        r = rates[p["field"]]
        fields.add(p["field"])
        t_ref += (3 * L * (-(-lg // 6) - 1) + L) / r
        t_r2 += (3 * (L // 2) * max(lg - 2, 0) + L) / r
    t_hbm48 = pm["bytes48"] / (peak * 1e9) * 1e3
    t_hbm_act = pm["bytes_actual"] / (peak * 1e9) * 1e3
    t_ref *= 1e3
    t_r2 *= 1e3
    roof_ms = max(t_hbm48, t_ref)
    return {"definition": "max(T_hbm(48 L + bit I/O at the measured HBM bandwidth), T_int(the scope's "
                          "modular-multiply count at the measured rate of the path's field)) / measured step",
            "frac": roof_ms / ms_per_step, "roofline_ms": roof_ms,
            "bytes48": pm["bytes48"], "t_hbm48_ms": t_hbm48,
            "achieved_gbs_48L": pm["bytes48"] / (ms_per_step * 1e-3) / 1e9,
            "frac_of_8tbs_48L": pm["bytes48"] / (ms_per_step * 1e-3) / 1e9 / 8000.0,
            "modmuls_reference": pm["modmuls_reference"], "t_int_reference_ms": t_ref,
            "modmul_rate_per_s": {FIELD_NAMES[f]: rates[f] for f in sorted(fields)},
            "actual_element_bytes": {"bytes": pm["bytes_actual"], "t_hbm_ms": t_hbm_act,
                                     "frac": max(t_hbm_act, t_ref) / ms_per_step},
            "radix2_modmuls": {"count": pm["modmuls_radix2"], "t_int_ms": t_r2,
                               "frac": max(t_hbm48, t_r2) / ms_per_step}}


def run_single(args, world, rank, local, dist):
    """One single-extraction workload (WORKLOADS): the JSON line (rank 0)."""
    import numpy as np
    import torch

    from paper_2402_09481_gb300 import inputs, native, replicas

    wl = WORKLOADS[args.workload]
    kind, n, m = wl["kind"], wl["n"], wl["m"]
    sb = seed_bits(kind, n, m)
    fopt = {"auto": native.FIELD_AUTO, "q30": native.FIELD_Q30, "goldilocks": native.FIELD_GOLDILOCKS}[args.field]
    plan = native.plan_query(kind, n, m, field=fopt)
    products = native.plan_products(kind, n, m, field=fopt)
    L = plan["transform_length"]
    launches = plan["launches"]
    ctx = native.Context(local, field=fopt)
    tune_cache = os.environ.get("CM_TUNE_CACHE")
    if tune_cache:
        # the planner's figures timed on this GPU (or loaded from the cache);
        # the plan keys below stay the built-in planner's
        ctx.calibrate(tune_cache)
    stream = torch.cuda.current_stream()

    xw = inputs.bernoulli_half(1 + 1000 * rank, n)
    if kind == 2:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(2 + 1000 * rank, sb)
    xd = torch.from_numpy(xw.view(np.int64)).cuda()
    yd = torch.from_numpy(yw.view(np.int64)).cuda()
    zd = torch.empty(native.words(m), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    call = {0: lambda: ctx.toeplitz(xd, n, yd, m, zd),
            1: lambda: ctx.circulant(xd, n, yd, m, zd),
            2: lambda: ctx.dodis(xd, yd, n, m, zd)}[kind]

    for _ in range(args.warmup):
        flush.zero_()
        call()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for k in range(args.steps):
        flush.zero_()                     # L2 flush, outside the events
        ev[k][0].record(stream)
        call()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # replicas: every rank extracts its own instance; the slowest rank bounds the job
    units_per_s, total_ms = replicas.job_throughput(m * args.steps, sum(step_ms), device="cuda")
    ms_per_step = total_ms / args.steps
    value = units_per_s / 1e9
    s, flags = ctx.device_status()
    if s != native.CM_OK:
        raise RuntimeError(f"device status {native.STATUS.get(s)} flags {flags}")

    # per-kernel device times (tracing hook: events on the launching stream)
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    for _ in range(args.steps):
        flush.zero_()
        call()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    peak, peak_src = measured_peaks()
    roof, kernels = roofline_of(prof, products, m, peak, peak_src, args.workload)
    rates = {f: native.modmul_rate(local, f) for f in (native.FIELD_GOLDILOCKS, native.FIELD_Q30, native.FIELD_Q25)}
    path_roof = path_roofline_of(products, n, sb, m, ms_per_step, peak, rates)

    # the Dodis et al. workload as its configuration states it: one Goldilocks
    # transform of length 2^31 (single-transform plan); same bits
    as_configured = None
    if args.workload == "dodis":
        gctx = native.Context(local, field=native.FIELD_GOLDILOCKS, plan_mode=native.PLAN_SINGLE)
        zg = torch.empty_like(zd)
        gcall = lambda: gctx.dodis(xd, yd, n, m, zg)  # noqa: E731
        for _ in range(2):
            gcall()
        g_ms = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gcall()
            b.record(stream)
            torch.cuda.synchronize()
            g_ms.append(a.elapsed_time(b))
        assert torch.equal(zg, zd), "single-transform result differs"
        gq = native.plan_query(kind, n, m, field=native.FIELD_GOLDILOCKS, plan_mode=native.PLAN_SINGLE)
        as_configured = {"plan": "one Goldilocks transform of length 2^31 (CM_FIELD_GOLDILOCKS, CM_PLAN_SINGLE)",
                         "transform_length": gq["transform_length"], "ms_per_step": statistics.median(g_ms),
                         "value": world * m / (statistics.median(g_ms) * 1e-3) / 1e9, "unit": "Gbit/s",
                         "bit_identical": True}
        gctx.close()
        del zg
        torch.cuda.empty_cache()

    # end to end through the public API with host buffers
    xh = torch.from_numpy(xw.view(np.int64)).pin_memory()
    yh = torch.from_numpy(yw.view(np.int64)).pin_memory()
    zh = torch.empty(native.words(m), dtype=torch.int64).pin_memory()
    for _ in range(3):
        ctx.extract_host(kind, xh, n, yh, m, zh)
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 50))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.extract_host(kind, xh, n, yh, m, zh)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    z_gpu = zd.cpu()
    assert torch.equal(zh, z_gpu), "host-buffer result differs from device-buffer result"
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": world * m / (e2e_mean * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": 8 * (xw.size + yw.size), "d2h_bytes_per_step": 8 * native.words(m),
           "ms_per_step": e2e_mean}
    ctx.close()
    del xd, yd, zd, flush
    torch.cuda.empty_cache()

    # CPU baselines on the host cores: the bit-packed CPU NTT on the whole
    # workload (one thread and every core) and the oracle on a bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, rows, secs = cpu_oracle_rate(kind, n, m, xw, yw)
        cpu = {"value": rate / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
               "sample": f"{rows} random output rows of the full-size workload in {secs:.1f} s "
                         f"(explicit GF(2) rows, numpy, one thread)"}
        # the competent CPU implementation, timed in the same run beside the oracle
        cpu_ntt = cpu_ntt_baseline(kind, n, m, xw, yw, z_gpu.numpy().view(np.uint64))
        if cpu_ntt is None:
            cpu_ntt = {"unavailable": "the CPU NTT's field (3 * 2^30 + 1) holds transforms up to 2^30 only"}
        cpu["cpu_ntt"] = cpu_ntt

    clocks = sampler.summary(t_wall0, t_wall1)
    if rank != 0:
        return None
    pf = plan["field"]
    return {
        "metric": "extracted output Gbit/s", "value": value, "unit": "Gbit/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64" if pf == FIELD_GL else "u32", "data": "synthetic",
        "config": {"workload": wl["name"], "n": n, "m": m, "seed_bits": sb,
                   "plan": {"products": plan["products"], "windows": plan["windows"],
                            "transform_length": L, "field": FIELD_NAMES.get(pf, pf),
                            "tail_terms": plan["tail_terms"], "planner_estimate_ms": plan["est_ms"]},
                   "l2": "flushed between timed steps (256 MiB write)",
                   **({"calibrated_planner": os.environ.get("CM_TUNE_CACHE")} if os.environ.get("CM_TUNE_CACHE") else {}),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "roofline": roof, "path_roofline": path_roof, "kernels": kernels,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
        **({"as_configured": as_configured} if as_configured else {}),
        "gpu_launches": launches * args.steps,
    }


def dodis_extra(local, steps=5):
    """The Dodis et al. workload (n = 1073741789, m = floor(0.4 n)), Bernoulli(1/2)
    sources and a second run with x 0.8-biased (drawn on the device: timing
    only; the tests check this run's bits against the oracle)."""
    import numpy as np
    import torch

    from paper_2402_09481_gb300 import inputs, native
    n, m = 1073741789, 429496715
    ctx = native.Context(local)
    plan = native.plan_query(2, n, m)
    products = native.plan_products(2, n, m)
    nw = native.words(n)
    xu = torch.from_numpy(inputs.bernoulli_half(31, n).view(np.int64)).cuda()
    yd = torch.from_numpy(inputs.bernoulli_half(32, n).view(np.int64)).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(2402)
    bits = torch.rand((nw, 64), device="cuda", generator=g) < 0.8
    xb = (bits.to(torch.int64) << torch.arange(64, device="cuda", dtype=torch.int64)).sum(dim=1)
    del bits
    zd = torch.empty(native.words(m), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    peak, _ = measured_peaks()
    rates = {f: native.modmul_rate(local, f) for f in (native.FIELD_GOLDILOCKS, native.FIELD_Q30, native.FIELD_Q25)}
    out = {"workload": "Dodis et al.: n = 1073741789 (largest N_A prime <= 2^30), m = floor(0.4 n)",
           "plan": {"products": plan["products"], "transform_length": plan["transform_length"],
                    "field": FIELD_NAMES.get(plan["field"], plan["field"])}}
    for name, xd in (("bernoulli_half", xu), ("x_0p8_biased", xb)):
        for _ in range(2):
            ctx.dodis(xd, yd, n, m, zd)
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.dodis(xd, yd, n, m, zd)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        st, fl = ctx.device_status()
        assert st == native.CM_OK, native.STATUS.get(st)
        ms_ = statistics.median(ts)
        pr = path_roofline_of(products, n, n, m, ms_, peak, rates)
        out[name] = {"ms_per_step": ms_, "value": m / (ms_ * 1e-3) / 1e9, "unit": "Gbit/s",
                     "path_roofline_frac": pr["frac"], "frac_actual_element_bytes": pr["actual_element_bytes"]["frac"]}
    ctx.close()
    del xu, xb, yd, zd, flush
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cm", choices=["cm", "reference"])
    ap.add_argument("--workload", default="circulant",
                    choices=sorted(WORKLOADS) + ["batched_a", "batched_b", "served", "von_neumann", "trevisan"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line only: skip the Dodis et al., batched (a) and served summaries")
    ap.add_argument("--field", default="auto", choices=["auto", "q30", "goldilocks"],
                    help="transform fields of the single calls (cm_options.field)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched_a":
        run_batched_a(args, world, rank, local)
        return
    if args.workload == "batched_b":
        run_batched_b(args, world, rank, local)
        return
    if args.workload == "served":
        run_served(args, world, rank, local)
        return
    if args.workload == "von_neumann":
        run_von_neumann(args, world, rank, local)
        return
    if args.workload == "trevisan":
        run_trevisan(args, world, rank, local)
        return

    import torch

    from paper_2402_09481_gb300 import build

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    line = run_single(args, world, rank, local, dist)
    # the scope's other targets, measured in the same run (one GPU): Dodis et
    # al. at full size with both sources, the batched and served forms each
    # against the plain per-call form on the same inputs
    if (line is not None and world == 1 and args.workload == "circulant" and args.field == "auto"
            and not args.no_extras):
        t0 = time.time()
        line["dodis"] = dodis_extra(local)
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.no_cpu_baseline = 3, 3, True
        ba = run_batched_a(sub, 1, 0, local, emit=False)
        line["batched_a"] = {k: ba[k] for k in ("value", "unit", "ms_per_step", "plain_per_call", "config",
                                               "roofline", "gpu_launches")}
        line["batched_a"]["faster_than_plain"] = ba["value"] / ba["plain_per_call"]["value"]
        sv = run_served(sub, 1, 0, local, emit=False)
        line["served"] = {k: sv[k] for k in ("value", "unit", "served", "plain_per_call", "sub_saturation", "config")}
        line["served"]["faster_than_plain"] = sv["value"] / sv["plain_per_call"]["value"]
        line["extras_seconds"] = time.time() - t0
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
