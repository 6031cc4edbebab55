#!/usr/bin/env python
"""Benchmark: bulk AES-ECB on GB300, one JSON line on stdout (rank 0).

Workload (one "step"): AES-128, AES-192 and AES-256, one seeded random key each,
a 1 GiB device-resident buffer of seeded uniform random bytes per key size;
encrypt the buffer in one launch, then decrypt the ciphertext in one launch --
six launches, 6 GiB of plaintext-equivalent bytes per step and GPU.  The buffers
(1 GiB) are larger than the 129 MB L2, so no flush is needed between steps.

  value     GB/s (1e9 B/s) over all ranks: bytes all ranks processed / max-over-ranks
            device time of the K timed steps (CUDA events on the launching stream).
  roofline  the dominant launch (largest share of step time) against the
            shared-memory lookup bound of Eq. 1 (16*Nr conflict-free 4-byte lookups
            per block, 32 per clock per SM), in plaintext GB/s.
  e2e       the same workload with the data in pinned host memory, through the
            C-ABI host pipeline (aes_pipeline_ecb, direct mode: the kernel reads
            and writes the host buffers over the host link), every transfer inside
            the timed region; "staged_gbs" is the staged mode (chunked copy-engine
            copies in and out around the kernel, overlapped over four slots).
  cpu_baseline  the CPU oracle (plain byte-oriented AES) on all host cores on a
            bounded 64 MiB sample of each of the six operations (rank 0, N=1 only).
  batched   10,000 messages (log-uniform 16 B - 4 MiB, own key each, key sizes
            2:1:1, mixed directions) in one persistent launch, against the same
            messages issued as 10,000 single-message launches.
  modes     CTR and CBC decryption (Section 3) on the 1 GiB AES-128/256 buffers:
            GB/s and fraction of the lookup roofline.
  serving   open-loop Poisson arrivals (200k req/s for 10 s, 64 B - 1 MiB, 1,024
            resident keys, 8 GiB budget) through the server in resident mode (one
            kernel stays on the GPU and takes requests from a ring in page-locked
            memory): GB/s and p50/p99 latency from scheduled arrival to
            completion; "launch_per_batch" runs the same arrivals through the
            launch-per-micro-batch mode.

Launch shapes of the table kernel are chosen by the autotuner during setup
(untimed) and reported under "tuned_shapes".

--impl reference times the CPU oracle as the reference arm (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AES-128/256 ECB GB/s on 1 GB300 (% of roofline); batched GB/s and p99 latency"
WORKLOAD = "aes-ecb encrypt+decrypt, 1 GiB device-resident buffer per key size (128/192/256), one launch per op"
BITS = (128, 192, 256)
NR = {128: 10, 192: 12, 256: 14}
GiB = 1 << 30
MiB = 1 << 20
LOOKUPS_PER_CLK_PER_SM = 32  # 32 banks x 4 B: one conflict-free 32-bit lookup per lane per clock
ALU_LANES_PER_CLK_PER_SM = 64  # integer ALU pipe: 4 SM sub-partitions x 16 lanes
# The bitsliced kernel's integer-ALU instructions per 16-byte block, (Nr, decrypt) -> lane-ops, counted by ncu
# (ALU-pipe utilisation x 2 warp instructions per clock per SM x active cycles x SMs x 32 / blocks) in
# profiles/bitsliced_kernel_ecb_256MiB_1GiB_ncu_full.md.
BITSLICED_ALU_OPS_PER_BLOCK = {(10, 0): 562.5, (10, 1): 639.5, (14, 0): 752.3, (14, 1): 860.3}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--buffer-mib", type=int, default=1024, help="bytes per key size (default 1 GiB)")
    p.add_argument("--e2e-steps", type=int, default=0, help="0 = max(3, steps // 20)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (e2e) leg")
    p.add_argument("--kernel", choices=("table", "bitsliced"), default="table")
    p.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    p.add_argument("--no-batched", action="store_true", help="skip the batched (10,000-message) section")
    p.add_argument("--batch-steps", type=int, default=10)
    p.add_argument("--no-serving", action="store_true", help="skip the serving (open-loop) section")
    p.add_argument("--no-modes", action="store_true", help="skip the CTR / CBC-decryption section")
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--sweep", action="store_true",
                   help="size sweep 4 KiB - 16 GiB (powers of 4), AES-128/256 encrypt, table vs bitsliced kernel")
    p.add_argument("--sweep-max-gib", type=int, default=16)
    p.add_argument("--no-cpu-sweep", action="store_true", help="--sweep: skip the CPU rows")
    p.add_argument("--serve-sweep", action="store_true",
                   help="serving latency against offered load (both server modes), one JSON line per point")
    p.add_argument("--serve-sweep-seconds", type=float, default=2.0)
    p.add_argument("--serve-sweep-rates", default="200000,400000,800000,1600000,2400000",
                   help="--serve-sweep: offered request rates (requests/s), comma separated")
    p.add_argument("--serve-sweep-modes", default="resident,launch",
                   help="--serve-sweep: server modes to run (resident, launch)")
    p.add_argument("--serve-sweep-repeat", type=int, default=1, help="--serve-sweep: runs per point")
    p.add_argument("--serve-poll-ms", type=float, default=0.0,
                   help="--serve-sweep: take completions every this many ms during the replay (0: at the end)")
    p.add_argument("--serve-pin", action="store_true",
                   help="--serve-sweep: pin the server's scheduler and replay threads to their own CPUs")
    p.add_argument("--serve-host", action="store_true",
                   help="--serve-sweep: request payloads in page-locked host memory (1 GiB in-flight budget)")
    p.add_argument("--serve-sweep-shape", default="",
                   help="--serve-sweep: resident tile shape THREADSxBLOCKS_PER_THREAD (default 512x2)")
    p.add_argument("--profile-case", choices=PROFILE_CASES,
                   help="run one small fixed case for an ncu capture (no timing, no JSON line)")
    p.add_argument("--profile-warmup", type=int, default=2)
    p.add_argument("--profile-launches", type=int, default=3)
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_fingerprint() -> str:
    """Hash of the table kernel's device code (host launcher code excluded)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1201_0398_gb300", "csrc")
    for name in ("ecb_table.cu", "aes_rounds.cuh", "aes_tables.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            text = f.read()
        if name == "ecb_table.cu":
            text = text.split(b"// ------------------------------------------------------------------ launcher")[0]
        h.update(text)
    return h.hexdigest()[:16]


def dram_traffic(kernel_key: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    fp = kernel_fingerprint()
    for line in lines:
        parts = line.split()
        if len(parts) >= 3 and parts[0] == fp and parts[1] == kernel_key:
            return float(parts[2])
    return None


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"gbaes_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            import torch

            uuid = str(torch.cuda.get_device_properties(self.device_index).uuid)
            ident = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:
            ident = str(self.device_index)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", ident], stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]) if f[3] not in ("[N/A]", "N/A") else None, f[5:9],
                             f[4]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] is None or r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max((r[2] or 0.0) for r in rows)}


def barrier(ranks):
    from paper_1201_0398_gb300 import dist

    dist.barrier(ranks)


def max_over_ranks(ranks, value: float) -> float:
    from paper_1201_0398_gb300 import dist

    return dist.max_over_ranks(ranks, value)


# ------------------------------------------------------------------ reference arm


def oracle_rate(sample_bytes: int, seed_offset: int = 0):
    """Times the CPU oracle on sample_bytes of each of the six operations.
    Returns (bytes, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_1201_0398_gb300 import workloads

    threads = os.cpu_count() or 1
    total_b, total_t = 0, 0.0
    for bits in BITS:
        key = workloads.random_key(workloads.SEED_BULK[bits], bits)
        data = workloads.host_bytes(workloads.SEED_BULK[bits] + seed_offset, sample_bytes)
        t0 = time.perf_counter()
        ct = oracle.ecb(key, bits, data, nthreads=threads)
        pt = oracle.ecb(key, bits, ct, decrypt=True, nthreads=threads)
        total_t += time.perf_counter() - t0
        total_b += 2 * sample_bytes
        if not np.array_equal(pt, data):
            raise RuntimeError("oracle round trip failed")
    return total_b, total_t, threads


def run_e2e(g, torch, x, keys, kernel, stream, size, bytes_per_step, e2e_steps, ranks, dev):
    """The step's workload on pinned host buffers through the host pipeline,
    host<->device transfers inside the timed region.  The headline uses the
    direct pipeline (the table kernel reads and writes the host buffers over the
    host link); the staged pipeline (64 MiB chunks through device slots and the
    copy engines) is measured beside it.  The three key sizes are independent
    chains (encrypt, then decrypt the ciphertext), so each runs on its own stream
    and pipeline."""
    xh = {bits: torch.empty(size, dtype=torch.uint8, pin_memory=True) for bits in BITS}
    ch = {bits: torch.empty(size, dtype=torch.uint8, pin_memory=True) for bits in BITS}
    ph = {bits: torch.empty(size, dtype=torch.uint8, pin_memory=True) for bits in BITS}
    for bits in BITS:
        xh[bits].copy_(x[bits])
    direct = {bits: g.Pipeline(mode=g.PIPE_DIRECT) for bits in BITS}
    staged = {bits: g.Pipeline(64 * MiB, 4, mode=g.PIPE_STAGED) for bits in BITS}
    chains = {bits: torch.cuda.Stream(dev) for bits in BITS}

    def fan(op):
        for bits in BITS:
            chains[bits].wait_stream(stream)
            op(bits, chains[bits])
        for bits in BITS:
            stream.wait_stream(chains[bits])

    def through(pipes):
        def step():
            def op(bits, st):
                pipes[bits].ecb(keys[bits], xh[bits], ch[bits], decrypt=False, stream=st)
                pipes[bits].ecb(keys[bits], ch[bits], ph[bits], decrypt=True, stream=st)
            fan(op)
        return step

    def timed_host(fn, reps):
        for bits in BITS:
            ph[bits].zero_()
        fn()
        torch.cuda.synchronize()
        if not all(torch.equal(ph[bits], xh[bits]) for bits in BITS):
            raise RuntimeError("e2e round trip failed")
        barrier(ranks)
        torch.cuda.synchronize()
        s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s2.record(stream)
        for _ in range(reps):
            fn()
        e2.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(ranks, s2.elapsed_time(e2) / 1e3)

    e2e_s = timed_host(through(direct), e2e_steps)
    staged_s = timed_host(through(staged), e2e_steps)

    def link_probe(kind, reps=5):  # plain torch copies of 1 GiB: what the host link gives
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for _ in range(reps):
            if kind in ("h2d", "both"):
                with torch.cuda.stream(s_in):
                    x[128].copy_(xh[128], non_blocking=True)
            if kind in ("d2h", "both"):
                with torch.cuda.stream(s_out):
                    ch[128].copy_(x[192], non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize()
        return reps * size / (e0.elapsed_time(e1) / 1e3) / 1e9

    link = {"h2d_gbs": link_probe("h2d"), "d2h_gbs": link_probe("d2h"), "both_directions_gbs_each": link_probe("both")}
    return {"value": ranks.world * e2e_steps * bytes_per_step / e2e_s / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": bytes_per_step, "d2h_bytes_per_step": bytes_per_step, "steps": e2e_steps,
           "path": "aes_pipeline_ecb, direct mode: the table kernel loads the pinned host input and stores the "
                   "pinned host output over the host link (512 threads x 4 blocks per thread), one launch per "
                   "operation; one pipeline and stream per key size",
           "staged_gbs": ranks.world * e2e_steps * bytes_per_step / staged_s / 1e9,
           "staged_path": "aes_pipeline_ecb, staged mode: 64 MiB chunks over 4 device staging slots/streams "
                          "(copy engine in, table kernel in place, copy engine out, overlapped)",
           "link": link}



def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    per_step = 2 * MiB
    for i in range(args.warmup):
        oracle_rate(per_step, seed_offset=1000 + i)
    tb, tt = 0, 0.0
    threads = os.cpu_count() or 1
    for i in range(args.steps):
        b, t, threads = oracle_rate(per_step, seed_offset=i)
        tb += b
        tt += t
    value = tb / tt / 1e9
    sample = (f"each step: the first {per_step // MiB} MiB of each of the six operations "
              f"(AES-128/192/256 encrypt + decrypt), oracle on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded uniform random bytes and keys)",
        "config": {"workload": WORKLOAD, "sample_bytes_per_op": per_step},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------- our arm


def run_ours(args):
    import numpy as np
    import torch

    import paper_1201_0398_gb300 as g
    from paper_1201_0398_gb300 import workloads

    from paper_1201_0398_gb300 import dist

    ranks = dist.setup()
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.load()
    kernel = g.KERNEL_TABLE if args.kernel == "table" else g.KERNEL_BITSLICED
    size = args.buffer_mib * MiB
    nblocks = size // 16
    stream = torch.cuda.current_stream(dev)
    keys, x, c, p = {}, {}, {}, {}
    for bits in BITS:
        keys[bits] = g.Key(workloads.random_key(workloads.SEED_BULK[bits], bits))
        x[bits] = workloads.device_bytes(dist.shard_seed(workloads.SEED_BULK[bits], ranks), size, device=dev)
        c[bits] = torch.empty_like(x[bits])
        p[bits] = torch.empty_like(x[bits])
    ops = [(bits, dec) for bits in BITS for dec in (False, True)]
    tuned = {}
    if kernel == g.KERNEL_TABLE and not args.no_tune:
        from paper_1201_0398_gb300 import autotune

        tuned = autotune.tune_all_ecb(nbytes=min(size, 256 * MiB))

    def launch(bits, dec):
        src, dst = (c[bits], p[bits]) if dec else (x[bits], c[bits])
        g.ecb_ex(keys[bits], src, dst, decrypt=dec, kernel=kernel, stream=stream)

    for _ in range(args.warmup):
        for bits, dec in ops:
            launch(bits, dec)
    torch.cuda.synchronize()
    for bits in BITS:  # sanity (untimed): decrypt(encrypt(x)) == x on the device
        if not torch.equal(p[bits], x[bits]):
            raise RuntimeError(f"round trip failed for AES-{bits}")

    ev = {op: [] for op in ops}
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    with ClockSampler(local) as clocks:
        barrier(ranks)
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            for op in ops:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                launch(*op)
                e1.record(stream)
                ev[op].append((e0, e1))
        end.record(stream)
        torch.cuda.synchronize()
        barrier(ranks)
    elapsed_s = start.elapsed_time(end) / 1e3
    elapsed_max = max_over_ranks(ranks, elapsed_s)
    clk = clocks.summary()
    bytes_per_step = len(ops) * size
    value = world * args.steps * bytes_per_step / elapsed_max / 1e9

    peaks, peak_kind = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sms = props.multi_processor_count
    op_stats = {}
    for (bits, dec), pairs in ev.items():
        ms = statistics.mean(a.elapsed_time(b) for a, b in pairs)
        gbs = size / (ms / 1e3) / 1e9
        r_smem = sms * LOOKUPS_PER_CLK_PER_SM * f_max / NR[bits] / 1e9
        op_stats[f"aes{bits}_{'dec' if dec else 'enc'}"] = {
            "ms": ms, "gbs": gbs, "smem_roofline_gbs": r_smem, "frac": gbs / r_smem,
            "hbm_frac": 2 * gbs / float(peaks["hbm_gbs"])}
    dom_name, dom = max(op_stats.items(), key=lambda kv: kv[1]["ms"])
    bits_dom = int(dom_name[3:6])
    dec_dom = dom_name.endswith("dec")
    bpt_dom = tuned.get(dom_name, {}).get("blocks_per_thread", 2)
    ktpl = f"table_kernel<{NR[bits_dom]},{1 if dec_dom else 0},{bpt_dom}>"
    traffic = dram_traffic(f"table_kernel<{NR[bits_dom]},{1 if dec_dom else 0}>") if kernel == g.KERNEL_TABLE else None
    clock_frac = None
    if clk.get("sm_mhz"):
        r_clk = sms * LOOKUPS_PER_CLK_PER_SM * clk["sm_mhz"] * 1e6 / NR[bits_dom] / 1e9
        clock_frac = dom["gbs"] / r_clk
    roofline = {
        "bound": "smem", "achieved": dom["gbs"], "peak": dom["smem_roofline_gbs"], "unit": "GB/s",
        "frac": dom["frac"], "traffic": traffic, "kernel": ktpl,
        "peak_basis": (f"{sms} SMs x {LOOKUPS_PER_CLK_PER_SM} lookups/clk x {f_max / 1e6:.0f} MHz "
                       f"({peak_kind} sm_max_mhz) / {NR[bits_dom]} lookups per plaintext byte"),
        "frac_at_measured_clock": clock_frac,
        "hbm": {"achieved": 2 * dom["gbs"], "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": dom["hbm_frac"], "peak_kind": f"{peak_kind} hbm_gbs (copy)"},
    }
    if kernel == g.KERNEL_BITSLICED:  # bound by the integer ALU pipe, not by shared memory
        ops_blk = BITSLICED_ALU_OPS_PER_BLOCK.get((NR[bits_dom], int(dec_dom)))
        peak = sms * ALU_LANES_PER_CLK_PER_SM * f_max / ops_blk * 16 / 1e9 if ops_blk else None
        roofline.update({
            "bound": "alu", "peak": peak, "frac": dom["gbs"] / peak if peak else None,
            "kernel": f"bitsliced_kernel<{NR[bits_dom]},{int(dec_dom)}>",
            "peak_basis": (f"{sms} SMs x {ALU_LANES_PER_CLK_PER_SM} ALU lanes/clk x {f_max / 1e6:.0f} MHz / "
                           f"{ops_blk} ALU ops per 16-byte block (ncu)" if ops_blk else
                           "no ncu count of ALU ops per block for this launch"),
            "frac_at_measured_clock": (dom["gbs"] / (peak * clk["sm_mhz"] * 1e6 / f_max)
                                       if peak and clk.get("sm_mhz") else None)})

    # ---- e2e: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(g, torch, x, keys, kernel, stream, size, bytes_per_step,
                      args.e2e_steps or max(3, args.steps // 20), ranks, dev)

    # ---- the other parallel modes of Section 3 on the same 1 GiB buffers
    modes = None
    if not args.no_modes and kernel == g.KERNEL_TABLE:
        modes = bench_modes(g, torch, x, c, p, keys, stream, size, sms, f_max)

    batched = None
    if not args.no_batched:
        for t in (x, c, p):
            t.clear()
        torch.cuda.empty_cache()
        batched = bench_batched(g, args, stream, ranks)

    serving = None
    if not args.no_serving:
        torch.cuda.empty_cache()
        from paper_1201_0398_gb300 import serving as serving_mod

        seed = dist.shard_seed(workloads.SEED_SERVE, ranks)
        serving = serving_mod.run(duration_s=args.serve_seconds, seed=seed, resident=True)
        torch.cuda.empty_cache()
        serving["launch_per_batch"] = {k: v for k, v in serving_mod.run(duration_s=args.serve_seconds, seed=seed).items()
                                       if k != "workload"}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = 64 * MiB
        b, t, threads = oracle_rate(sample)
        cpu = {"value": b / t / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": f"first {sample // MiB} MiB of each of the six operations (AES-128/192/256 enc+dec), "
                         f"{threads} host threads"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded uniform random bytes and keys)",
            "config": {"workload": WORKLOAD, "buffer_bytes": size, "nblocks_per_op": nblocks,
                       "kernel": args.kernel, "launches_per_step": len(ops), "sms": sms,
                       "l2": "inputs larger than L2 (1 GiB > 129 MB), no flush",
                       "parallelism": f"replicas x{world} (independent buffers per rank)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": len(ops) * args.steps,
            "clocks": clk, "ops": op_stats, "tuned_shapes": {k: f"{v['threads']}x{v['blocks_per_thread']}"
                                                             for k, v in tuned.items()},
            "batched": batched, "serving": serving, "modes": modes,
        }), flush=True)
    dist.teardown(ranks)


def bench_modes(g, torch, x, c, p, keys, stream, size, sms, f_max, reps=10):
    """CTR (big-endian 128-bit counter) and CBC decryption (Eq. 2) on the 1 GiB
    AES-128 and AES-256 buffers, one launch each, CUDA events on the launching
    stream: GB/s of plaintext and the fraction of the same shared-memory lookup
    roofline as ECB (the modes add one 16-byte XOR per block, and CBC one
    cache-resident neighbour load)."""
    iv = bytes(range(16))
    out = {}
    for bits in (128, 256):
        for name, fn in (("ctr", lambda: g.ctr_xcrypt(keys[bits], iv, x[bits], c[bits], stream=stream)),
                         ("cbc_dec", lambda: g.cbc_decrypt(keys[bits], iv, x[bits], p[bits], stream=stream))):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = size / (ms / 1e3) / 1e9
            r = sms * LOOKUPS_PER_CLK_PER_SM * f_max / NR[bits] / 1e9
            out[f"{name}_{bits}"] = {"ms": ms, "gbs": gbs, "smem_roofline_gbs": r, "frac": gbs / r}
    return out


def bench_batched(g, args, stream, ranks):
    """10,000 messages (log-uniform 16 B - 4 MiB, own key each, key sizes 2:1:1,
    mixed directions) in one persistent launch; compared with the same messages
    issued as 10,000 single-message launches."""
    import numpy as np
    import torch

    from paper_1201_0398_gb300 import autotune, workloads

    from paper_1201_0398_gb300 import dist

    world = ranks.world
    w = workloads.batch_workload(seed=dist.shard_seed(workloads.SEED_BATCH, ranks))
    keys = [g.Key(k) for k in w.keys]
    nblocks = w.lengths // 16
    off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
    descs = g.make_descs(off, off, nblocks, np.arange(len(keys)), w.decrypt)
    x = workloads.device_bytes(dist.shard_seed(workloads.SEED_BATCH, ranks), w.total_bytes, device=torch.device("cuda"))
    y = torch.empty_like(x)
    plan, report = autotune.tune_batch(descs, keys, x, y)
    plan.launch(x, y, stream=stream)
    alone = torch.empty_like(x)
    for i in range(len(keys)):
        a, n = int(off[i]), int(w.lengths[i])
        g.ecb_ex(keys[i], x[a:a + n], alone[a:a + n], decrypt=bool(w.decrypt[i]), stream=stream)
    torch.cuda.synchronize()
    if not torch.equal(alone, y):
        raise RuntimeError("batched output differs from the single-message kernel")

    def timed(fn, reps):
        barrier(ranks)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(ranks, e0.elapsed_time(e1) / 1e3 / reps)

    reps = max(3, args.batch_steps)
    t_plan = timed(lambda: plan.launch(x, y, stream=stream), reps)
    t_graph = timed(lambda: plan.launch(x, y, stream=stream, graph=True), reps)

    def single_loop():
        for i in range(len(keys)):
            a, n = int(off[i]), int(w.lengths[i])
            g.ecb_ex(keys[i], x[a:a + n], alone[a:a + n], decrypt=bool(w.decrypt[i]), stream=stream)

    t_loop = timed(single_loop, 2)

    total = w.total_bytes
    nr_eff = float((w.lengths * np.vectorize(NR.get)(w.bits)).sum() / total)  # lookups per plaintext byte
    peaks, _ = measured_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    r_smem = sms * LOOKUPS_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / nr_eff / 1e9
    return {"value": world * total / t_plan / 1e9, "unit": "GB/s", "messages": len(keys), "bytes": total,
            "ms": 1e3 * t_plan, "graph_gbs": world * total / t_graph / 1e9,
            "single_launch_loop_gbs": world * total / t_loop / 1e9,
            "shape": report["best"],
            "nr_eff": nr_eff, "smem_roofline_gbs": r_smem, "frac": total / t_plan / 1e9 / r_smem,
            "candidates_ms": report["candidates_ms"], "launches_per_step": 1,
            "workload": "10,000 messages, log-uniform 16 B-4 MiB (x16 B), keys 128/192/256 at 2:1:1, "
                        "encrypt/decrypt 50/50, one persistent launch"}


def run_sweep(args):
    """One JSON line per (key size, kernel, buffer size): device-resident
    uniform random bytes; "ms" = CUDA-event time of reps back-to-back calls /
    reps, "graph_us" (up to 16 MiB) = device time per call replayed from a
    CUDA graph."""
    import torch

    import paper_1201_0398_gb300 as g
    from paper_1201_0398_gb300 import workloads

    g.load()
    peaks, peak_kind = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    stream = torch.cuda.current_stream()
    sizes = [4096 * 4 ** i for i in range(12) if 4096 * 4 ** i <= args.sweep_max_gib * GiB]
    x = workloads.device_bytes(31, sizes[-1])
    y = torch.empty_like(x)
    kernels = (("table", g.KERNEL_TABLE), ("table_compact", g.KERNEL_TABLE_COMPACT),
               ("table_replicated", g.KERNEL_TABLE_REPLICATED), ("bitsliced", g.KERNEL_BITSLICED))
    for bits in (128, 256):
        k = g.Key(workloads.random_key(40 + bits, bits))
        for kname, kid in kernels:
            for size in sizes:
                if kid == g.KERNEL_TABLE_COMPACT and size > 256 * MiB:
                    continue
                xs, ys = x[:size], y[:size]
                reps = max(5, min(200, int(2 * GiB // size)))
                for _ in range(3):
                    g.ecb_ex(k, xs, ys, kernel=kid, stream=stream)
                torch.cuda.synchronize()
                # Back-to-back calls between two events: per call, the larger of
                # the device time and the host's issue time (a small call from
                # Python is host bound; graph_us below takes the host out).
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    g.ecb_ex(k, xs, ys, kernel=kid, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                gbs = size / (ms / 1e3) / 1e9
                r_smem = sms * LOOKUPS_PER_CLK_PER_SM * f_max / NR[bits] / 1e9
                line = {"sweep": "aes-ecb-encrypt", "bits": bits, "kernel": kname, "bytes": size, "ms": ms,
                        "gbs": gbs, "reps": reps, "frac_smem_roofline": gbs / r_smem,
                        "hbm_frac": 2 * gbs / float(peaks["hbm_gbs"])}
                if size <= 16 * MiB:
                    line["graph_us"] = graph_launch_us(torch, g, k, xs, ys, kid)
                    line["graph_gbs"] = size / line["graph_us"] / 1e3
                print(json.dumps(line), flush=True)


def graph_launch_us(torch, g, k, xs, ys, kid, n=50, reps=5):
    """Device time per call with the host out of the way: n calls of the C ABI
    captured into one CUDA graph, the graph replayed, CUDA events around the
    replay (median of reps replays) / n."""
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        for _ in range(n):
            g.ecb_ex(k, xs, ys, kernel=kid)
    replay = torch.cuda.current_stream()  # CUDAGraph.replay launches on the current stream
    graph.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(replay)
        graph.replay()
        e1.record(replay)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3 / n)
    del graph
    return statistics.median(ts)


class OpenSSLECB:
    """OpenSSL's EVP AES-ECB from the system libcrypto, used as-is through ctypes
    (a hardware-accelerated CPU comparison point; absent libraries are skipped)."""

    def __init__(self):
        import ctypes
        import ctypes.util

        name = ctypes.util.find_library("crypto")
        cands = [name] if name else []
        cands += ["libcrypto.so.3", "libcrypto.so.1.1", "libcrypto.so"]
        self.lib = None
        for c in cands:
            try:
                self.lib = ctypes.CDLL(c)
                break
            except OSError:
                continue
        if self.lib is None:
            raise OSError("libcrypto not found")
        L, vp = self.lib, ctypes.c_void_p
        L.EVP_CIPHER_CTX_new.restype = vp
        L.EVP_CIPHER_CTX_free.argtypes = [vp]
        for n in ("EVP_aes_128_ecb", "EVP_aes_256_ecb"):
            getattr(L, n).restype = vp
        L.EVP_EncryptInit_ex.argtypes = [vp, vp, vp, ctypes.c_char_p, ctypes.c_char_p]
        L.EVP_CIPHER_CTX_set_padding.argtypes = [vp, ctypes.c_int]
        L.EVP_EncryptUpdate.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), vp, ctypes.c_int]
        self.version = None
        try:
            L.OpenSSL_version.restype = ctypes.c_char_p
            self.version = L.OpenSSL_version(0).decode()
        except AttributeError:
            pass

    def encrypt(self, key: bytes, bits: int, data, out) -> None:
        import ctypes

        L = self.lib
        ctx = L.EVP_CIPHER_CTX_new()
        cipher = L.EVP_aes_128_ecb() if bits == 128 else L.EVP_aes_256_ecb()
        L.EVP_EncryptInit_ex(ctx, cipher, None, key, None)
        L.EVP_CIPHER_CTX_set_padding(ctx, 0)
        n = ctypes.c_int(0)
        chunk = 1 << 30
        for off in range(0, data.size, chunk):
            m = min(chunk, data.size - off)
            L.EVP_EncryptUpdate(ctx, ctypes.c_void_p(out.ctypes.data + off), ctypes.byref(n),
                                ctypes.c_void_p(data.ctypes.data + off), m)
        L.EVP_CIPHER_CTX_free(ctx)


def run_cpu_sweep():
    """CPU comparison at the paper's Fig. 4 granularity (1, 2, 3, 4 cores and all
    cores): the oracle and, when present, OpenSSL's EVP AES-ECB; AES-128/256
    encryption of large buffers; then the oracle beside the bench's six
    operations: one core on a 64 MiB slice and all cores on the whole 1 GiB
    buffer, AES-128/192/256 encryption and decryption.  Reporting only."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_1201_0398_gb300 import workloads

    allc = os.cpu_count() or 1
    counts = sorted({1, 2, 3, 4, allc})
    try:
        ossl = OpenSSLECB()
    except OSError:
        ossl = None
    for bits in (128, 256):
        key = workloads.random_key(40 + bits, bits)
        for n in counts:
            data = workloads.host_bytes(5, 8 * MiB * n)
            t0 = time.perf_counter()
            oracle.ecb(key, bits, data, nthreads=n)
            dt = time.perf_counter() - t0
            print(json.dumps({"sweep": "cpu", "impl": "oracle", "bits": bits, "threads": n, "bytes": data.size,
                              "gbs": data.size / dt / 1e9}), flush=True)
            if ossl is None:
                continue
            per = 128 * MiB
            data = workloads.host_bytes(6, per * n)
            out = np.empty_like(data)
            parts = [(data[i * per:(i + 1) * per], out[i * per:(i + 1) * per]) for i in range(n)]
            best = None
            with ThreadPoolExecutor(n) as ex:
                for _ in range(3):
                    t0 = time.perf_counter()
                    list(ex.map(lambda pr: ossl.encrypt(key, bits, pr[0], pr[1]), parts))
                    dt = time.perf_counter() - t0
                    best = dt if best is None else min(best, dt)
            ok = np.array_equal(out[:4096], oracle.ecb(key, bits, data[:4096]))
            print(json.dumps({"sweep": "cpu", "impl": "openssl-evp", "version": ossl.version, "bits": bits,
                              "threads": n, "bytes": data.size, "gbs": data.size / best / 1e9,
                              "matches_oracle": bool(ok)}), flush=True)
    for bits in BITS:
        key = workloads.random_key(workloads.SEED_BULK[bits], bits)
        for n, size in ((1, 64 * MiB), (allc, GiB)):
            data = workloads.host_bytes(workloads.SEED_BULK[bits], size)
            for dec in (False, True):
                t0 = time.perf_counter()
                oracle.ecb(key, bits, data, decrypt=dec, nthreads=n)
                dt = time.perf_counter() - t0
                print(json.dumps({"sweep": "cpu-oracle-bench-ops", "impl": "oracle", "bits": bits,
                                  "op": "dec" if dec else "enc", "threads": n, "bytes": data.size,
                                  "gbs": data.size / dt / 1e9}), flush=True)


def run_serve_sweep(args):
    """Open-loop serving at 200k, 400k, 800k, 1.6M and 2.4M requests/s (the serving
    workload's sizes and keys), through the resident kernel and through launch
    per micro-batch: one JSON line per (mode, rate) with GB/s and latency
    percentiles."""
    import torch

    from paper_1201_0398_gb300 import load, serving

    load()
    modes = [m.strip() for m in args.serve_sweep_modes.split(",")]
    threads, bpt = (int(v) for v in args.serve_sweep_shape.split("x")) if args.serve_sweep_shape else (0, 0)
    rates = [float(r) for r in args.serve_sweep_rates.split(",") for _ in range(args.serve_sweep_repeat)]
    for rate in rates:
        for resident in (m == "resident" for m in modes):
            shape = dict(threads=threads, blocks_per_thread=bpt) if resident else {}
            r = serving.run(rate=rate, duration_s=args.serve_sweep_seconds, check_last=200, resident=resident,
                            pin_threads=args.serve_pin, poll_every_s=args.serve_poll_ms / 1e3,
                            host_payloads=args.serve_host, **({"budget_bytes": GiB} if args.serve_host else {}),
                            **shape)
            torch.cuda.empty_cache()
            keep = ("mode", "value", "offered_gbs", "requests", "completed_ok", "p50_ms", "p99_ms", "p999_ms",
                    "max_ms", "p50_queue_ms", "p50_service_ms", "max_queue", "max_inflight_bytes", "shape",
                    "mismatches", "mean_batch_msgs", "p50_service_ms", "p99_service_ms", "host_threads",
                    "kernel_launches", "payloads", "host_memory")
            print(json.dumps({"sweep": "serving", "rate": rate, "seconds": args.serve_sweep_seconds,
                              **{k: r[k] for k in keep if k in r}}), flush=True)


PROFILE_CASES = ("table", "table1g", "bitsliced", "bitsliced1g", "batch", "sweep", "singles")


def run_profile_case(args):
    """Small fixed cases for profiling one kernel at a time (ncu -k ... -s W -c N).

    Each case runs --profile-warmup launches then --profile-launches more of one
    kernel, on inputs larger than the 129 MB L2 but a few hundred MB in all (so a
    multi-pass capture ends in seconds), except table1g:
      table      256 MiB, AES-128 encryption + AES-256 decryption, table kernel
      table1g    1 GiB, the bench's launches (AES-128/192/256, encrypt + decrypt),
                 for single-pass DRAM-byte captures at the bench size only
      bitsliced  256 MiB, AES-128 encryption + decryption, then AES-256 encryption +
                 decryption, bitsliced kernel
      bitsliced1g the same four launches at 1 GiB (2 GiB on the device), the bench's size
      batch      10,000 messages, 16 B - 1 MiB (~0.95 GB), one batched launch each
      sweep      one AES-128 encryption per size, 4 KiB - 256 MiB: table (size-dispatched),
                 compact tables (up to 64 MiB), replicated tables, bitsliced
      singles    the 10,000-message batch as one batched launch, then as 10,000
                 single-message launches
    """
    import numpy as np
    import torch

    import paper_1201_0398_gb300 as g
    from paper_1201_0398_gb300 import workloads

    g.load()
    case, warm, launches = args.profile_case, args.profile_warmup, args.profile_launches
    if case in ("table", "table1g", "bitsliced", "bitsliced1g"):
        kid = g.KERNEL_BITSLICED if case.startswith("bitsliced") else g.KERNEL_TABLE
        size = {"table": 256 << 20, "table1g": GiB, "bitsliced": 256 << 20, "bitsliced1g": GiB}[case]
        ops = {"table": [(128, False), (256, True)],
               "bitsliced": [(128, False), (128, True), (256, False), (256, True)],
               "bitsliced1g": [(128, False), (128, True), (256, False), (256, True)],
               "table1g": [(b, d) for b in BITS for d in (False, True)]}[case]
        x = workloads.device_bytes(1, size)
        y = torch.empty_like(x)
        keys = {b: g.Key(workloads.random_key(b, b)) for b, _ in ops}
        for _ in range(warm + launches):
            for bits, dec in ops:
                g.ecb_ex(keys[bits], x, y, decrypt=dec, kernel=kid)
    elif case == "sweep":
        x = workloads.device_bytes(31, 256 * MiB)
        y = torch.empty_like(x)
        k = g.Key(workloads.random_key(168, 128))
        for kid in (g.KERNEL_TABLE, g.KERNEL_TABLE_COMPACT, g.KERNEL_TABLE_REPLICATED, g.KERNEL_BITSLICED):
            for size in (4096 * 4 ** i for i in range(9)):  # 4 KiB .. 256 MiB
                if kid != g.KERNEL_TABLE_COMPACT or size <= 64 * MiB:
                    g.ecb_ex(k, x[:size], y[:size], kernel=kid)
    else:
        w = workloads.batch_workload(n=10000, max_len=MiB) if case == "batch" else workloads.batch_workload()
        ks = [g.Key(k) for k in w.keys]
        off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
        d = g.make_descs(off, off, w.lengths // 16, np.arange(len(ks)), w.decrypt)
        x = workloads.device_bytes(4, w.total_bytes)
        y = torch.empty_like(x)
        plan = g.BatchPlan(d, ks, 512, 8)
        if case == "batch":
            for _ in range(warm + launches):
                plan.launch(x, y)
        else:
            plan.launch(x, y)
            for i in range(len(ks)):
                o, n = int(off[i]), int(w.lengths[i])
                g.ecb_ex(ks[i], x[o:o + n], y[o:o + n], decrypt=bool(w.decrypt[i]))
    torch.cuda.synchronize()
    print(f"profile case {case}: ok", file=sys.stderr)


def main():
    args = parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.serve_sweep:
        run_serve_sweep(args)
        return
    if args.sweep:
        run_sweep(args)
        if not args.no_cpu_sweep:
            run_cpu_sweep()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
