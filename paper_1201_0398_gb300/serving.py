"""Open-loop serving run: Poisson arrivals replayed into the native server.

Requests read slices of one input pool and write to an output ring, both in
device memory (or both in page-locked host memory: host_payloads).  Consecutive requests take consecutive ring space; the ring is larger
than the output bytes the budget lets be in flight (half the budget) plus the
largest request, so two requests that are in flight together never share
output bytes.  Latency is completion minus *scheduled* arrival.
"""
from __future__ import annotations

import numpy as np

from . import COMPLETION, REQUEST, Key, Server, ecb_ex, workloads

GiB = 1 << 30

_VM_KEYS = ("pgmigrate_success", "compact_migrate_scanned", "compact_daemon_migrate_scanned")


def _vmstat() -> dict:
    """The kernel's page-migration and compaction counters (empty if unreadable)."""
    try:
        with open("/proc/vmstat") as f:
            return {k: int(v) for k, v in (line.split() for line in f) if k in _VM_KEYS}
    except OSError:
        return {}


def _wait_compaction_quiet(max_s: float, quiet_s: float = 1.0) -> float:
    """Waits (at most max_s) until the kernel has migrated no page for quiet_s:
    memory compaction set off by the setup (GBs of buffers just allocated) moves
    pages under the server's threads and code, and a thread that touches a page
    being moved sleeps until the move ends.  Returns the seconds waited."""
    import time

    t0 = time.monotonic()
    last, since = _vmstat(), t0
    if not last:
        return 0.0
    while time.monotonic() - t0 < max_s:
        time.sleep(0.1)
        cur = _vmstat()
        if cur != last:
            last, since = cur, time.monotonic()
        elif time.monotonic() - since >= quiet_s:
            break
    return time.monotonic() - t0


def run(rate: float = 200_000.0, duration_s: float = 10.0, budget_bytes: int = 8 << 30, nkeys: int = 1024,
        nstreams: int = 4, threads: int = 0, blocks_per_thread: int = 0, max_batch_msgs: int = 4096,
        pool_bytes: int = GiB, check_last: int = 1000, seed: int = workloads.SEED_SERVE,
        resident: bool = False, pin_threads: bool = False, poll_every_s: float = 0.0,
        host_payloads: bool = False, warmup_s: float = 0.2, settle_max_s: float = 10.0) -> dict:
    """host_payloads: the input pool and the output ring live in page-locked host
    memory instead of device memory (the kernels read and write them over the host
    link); the ring then holds twice the in-flight budget, at least 1 GiB.
    warmup_s: the first warmup_s seconds of the schedule run first on a separate
    server with the same settings (untimed; every code path of the server, the
    driver calls and the kernel's launch, end and relaunch have then run once).
    settle_max_s: then wait at most this long for the kernel's memory compaction
    to go quiet before the measured replay (reported as host_memory.settle_s,
    with the pages migrated during the replay)."""
    import torch

    w = workloads.serve_workload(rate=rate, duration_s=duration_s, nkeys=nkeys, seed=seed)
    n = w.arrival_s.size
    keys = [Key(k) for k in w.keys]
    dev = torch.device("cuda")
    x = workloads.device_bytes(seed, pool_bytes, device=dev)
    max_len = int(w.lengths.max())
    ring = max(2 * (budget_bytes // 2), GiB if host_payloads else 4 * GiB) + 2 * max_len
    ring = (ring + 15) // 16 * 16
    if host_payloads:
        x = x.cpu().pin_memory()
        y = torch.empty(ring + max_len, dtype=torch.uint8, pin_memory=True)
    else:
        y = torch.empty(ring + max_len, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(seed + 1)
    in_off = rng.integers(0, (pool_bytes - w.lengths) // 16 + 1) * 16
    cum = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
    out_off = cum % ring
    reqs = np.zeros(n, REQUEST)
    reqs["id"] = np.arange(n)
    reqs["in_ptr"] = x.data_ptr() + in_off
    reqs["out_ptr"] = y.data_ptr() + out_off
    reqs["nblocks"] = w.lengths // 16
    reqs["key_index"] = w.key_index
    reqs["decrypt"] = w.decrypt
    reqs["arrival_s"] = w.arrival_s

    torch.cuda.synchronize()  # inputs complete before the first request

    def make_server():
        return Server(keys, budget_bytes=budget_bytes, nstreams=nstreams, threads=threads,
                      blocks_per_thread=blocks_per_thread, max_batch_msgs=max_batch_msgs, resident=resident,
                      pin_threads=pin_threads)

    if warmup_s > 0:
        k = max(1, int(np.searchsorted(w.arrival_s, warmup_s)))
        wsrv = make_server()
        wsrv.replay(reqs[:k])
        wsrv.replay_join()
        wsrv.drain(120.0)
        wsrv.poll_all()
        wsrv.close()
        torch.cuda.synchronize()
    settle_s = _wait_compaction_quiet(settle_max_s) if settle_max_s > 0 else 0.0
    vm0 = _vmstat()
    srv = make_server()
    parts = []
    polling = poll_every_s > 0
    if polling:  # a client that takes its completions as they come (the server's queue stays short)
        import threading
        import time

        stop = threading.Event()

        buf = np.zeros(1 << 16, COMPLETION)  # reused: the copy under the server's lock lands in touched memory

        def poller():
            while not stop.is_set():
                p = srv.poll(buf.size, out=buf)
                if p.size:
                    parts.append(p.copy())
                else:
                    time.sleep(poll_every_s)

        th = threading.Thread(target=poller)
        th.start()
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(120.0)
    vm1 = _vmstat()
    if polling:
        stop.set()
        th.join()
    parts.append(srv.poll_all())
    done = np.concatenate(parts)
    stats = srv.stats()
    diag = srv.diag()
    srv.close()
    ok = done["status"] == 0
    lat = (done["done_s"] - done["arrival_s"])[ok]
    wait = (done["launch_s"] - done["arrival_s"])[ok]  # arrival -> its batch's launch (resident: publication)
    service = (done["done_s"] - done["launch_s"])[ok]  # launch -> completion observed
    span = float(done["done_s"].max() - done["arrival_s"].min())
    total = int(w.lengths.sum())

    # The last requests' outputs are still in the ring: compare with the
    # single-message kernel on each request alone.
    torch.cuda.synchronize()
    mismatches = 0
    idx = np.arange(max(0, n - check_last), n)
    alone = torch.empty(int(w.lengths[idx].max()), dtype=torch.uint8, device=dev)
    if host_payloads:
        alone = alone.cpu().pin_memory()
    for i in idx:
        a, b, m = int(in_off[i]), int(out_off[i]), int(w.lengths[i])
        ecb_ex(keys[int(w.key_index[i])], x[a:a + m], alone[:m], decrypt=bool(w.decrypt[i]))
        if host_payloads:
            torch.cuda.synchronize()  # (host tensors: the comparison below does not wait for the stream)
        if not torch.equal(alone[:m], y[b:b + m]):
            mismatches += 1
    batches = np.unique(done["launch_s"])
    return {
        "mode": "resident kernel" if resident else "launch per micro-batch",
        "payloads": "page-locked host memory" if host_payloads else "device memory",
        "value": total / span / 1e9, "unit": "GB/s", "requests": int(n), "completed_ok": int(ok.sum()),
        "offered_gbs": total / duration_s / 1e9, "bytes": total,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "p999_ms": float(np.percentile(lat, 99.9) * 1e3), "max_ms": float(lat.max() * 1e3),
        "p50_queue_ms": float(np.percentile(wait, 50) * 1e3), "p99_queue_ms": float(np.percentile(wait, 99) * 1e3),
        "p50_service_ms": float(np.percentile(service, 50) * 1e3),
        "p99_service_ms": float(np.percentile(service, 99) * 1e3),
        "mean_batch_msgs": float(n / max(1, len(batches))),
        ("kernel_launches" if resident else "batches"): int(stats["batches"]),
        "max_queue": int(stats["max_queue"]), "lost_completions": int(stats["lost_completions"]), "max_inflight_bytes": int(stats["max_inflight_bytes"]),
        "budget_bytes": int(budget_bytes), "nstreams": nstreams, "shape": f"{threads or 512}x{blocks_per_thread or (2 if resident else 1)}",
        "checked_alone": int(len(idx)), "mismatches": mismatches,
        "host_memory": {"warmup_s": warmup_s, "settle_s": round(settle_s, 2),
                        "pages_migrated_during_replay": (vm1.get("pgmigrate_success", 0) - vm0.get("pgmigrate_success", 0))
                        if vm0 else None,
                        "compaction_pages_scanned_during_replay":
                            sum(vm1.get(k, 0) - vm0.get(k, 0) for k in _VM_KEYS[1:]) if vm0 else None},
        "host_threads": {
            "pinned_cpus": [int(diag["sched_cpu"]), int(diag["producer_cpu"])],
            "sched_passes": int(diag["sched_passes"]),
            "sched_worst_window_us": diag["sched_worst_window_ns"] / 1e3,
            "sched_worst_window_cpu_us": diag["sched_worst_window_cpu_ns"] / 1e3,
            "sched_worst_window_invol": int(diag["sched_worst_window_invol"]),
            "sched_worst_window_vol": int(diag["sched_worst_window_vol"]),
            "sched_worst_window_faults": [int(diag["sched_worst_window_minflt"]),
                                          int(diag["sched_worst_window_majflt"])],
            "sched_worst_window_at_s": diag["sched_worst_window_at_ns"] / 1e9,
            "sched_invol": int(diag["sched_invol"]),
            "page_faults": [int(diag["sched_minflt"]), int(diag["producer_minflt"])],
            "lock_wait_max_us": {k: v / 1e3 for k, v in zip(("inbox", "done", "stats"), diag["lock_wait_max_ns"])},
            "lock_wait_at_s": {k: v / 1e9 for k, v in zip(("inbox", "done", "stats"), diag["lock_wait_at_ns"])},
            "cuda_call_max_us": diag["cuda_call_max_ns"] / 1e3,
            "cuda_call_at_s": diag["cuda_call_at_ns"] / 1e9,
            "stream_queries": {"confirm_end": int(diag["stream_queries"][0]),
                               "no_progress": int(diag["stream_queries"][1])},
            "sched_phase_max_us": {k: v / 1e3 for k, v in zip(("inbox", "done", "query", "admit", "launch"),
                                                              diag["sched_phase_max_ns"])},
            "sched_phase_at_s": {k: v / 1e9 for k, v in zip(("inbox", "done", "query", "admit", "launch"),
                                                             diag["sched_phase_at_ns"])},
            "inbox_hold_max_us": [v / 1e3 for v in diag["inbox_hold_max_ns"]],
            "producer_late_max_us": diag["producer_late_max_ns"] / 1e3,
            "producer_late_at_s": diag["producer_late_at_ns"] / 1e9,
            "producer_late_invol": int(diag["producer_late_invol"]),
            "producer_invol": int(diag["producer_invol"]),
            "producer_check_max_us": diag["producer_check_max_ns"] / 1e3,
            "producer_check_at_s": diag["producer_check_at_ns"] / 1e9},
        "workload": f"Poisson {rate:.0f} req/s for {duration_s:g} s, sizes log-uniform 64 B-1 MiB (x16 B), "
                    f"{nkeys} resident keys (128/192/256), encrypt/decrypt 50/50, {budget_bytes >> 30} GiB budget",
    }
