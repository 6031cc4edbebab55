"""Small fixed cases for profiling one kernel at a time (ncu -k ... -s W -c N).

Each case runs `warmup` launches then `launches` more of one kernel on inputs
larger than the 129 MB L2 but a few hundred MB in all, so a multi-pass ncu
capture of a launch ends in seconds:

  python -m paper_1201_0398_gb300.profile_cases table      # 256 MiB, AES-128 enc + AES-256 dec
  python -m paper_1201_0398_gb300.profile_cases bitsliced  # 64 MiB, AES-128 enc + dec
  python -m paper_1201_0398_gb300.profile_cases batch      # 10,000 messages, 16 B - 1 MiB (~0.95 GB)
  python -m paper_1201_0398_gb300.profile_cases sweep      # one AES-128 encryption per size, 4 KiB - 1 GiB,
                                                           # table kernel then bitsliced kernel
  python -m paper_1201_0398_gb300.profile_cases singles    # the 10,000-message batch as one batched launch,
                                                           # then as 10,000 single-message launches
"""
from __future__ import annotations

import argparse

import numpy as np


def main(argv=None):
    import torch

    import paper_1201_0398_gb300 as g
    from paper_1201_0398_gb300 import workloads

    p = argparse.ArgumentParser()
    p.add_argument("case", choices=("table", "bitsliced", "batch", "sweep", "singles"))
    p.add_argument("--warmup", type=int, default=2)
    p.add_argument("--launches", type=int, default=3)
    a = p.parse_args(argv)
    g.load()
    if a.case in ("table", "bitsliced"):
        kid = g.KERNEL_TABLE if a.case == "table" else g.KERNEL_BITSLICED
        size = (256 if a.case == "table" else 64) << 20
        x = workloads.device_bytes(1, size)
        y = torch.empty_like(x)
        ops = [(128, False), (256, True)] if a.case == "table" else [(128, False), (128, True)]
        keys = {b: g.Key(workloads.random_key(b, b)) for b, _ in ops}
        for _ in range(a.warmup + a.launches):
            for bits, dec in ops:
                g.ecb_ex(keys[bits], x, y, decrypt=dec, kernel=kid)
    elif a.case == "sweep":
        x = workloads.device_bytes(31, 1 << 30)
        y = torch.empty_like(x)
        k = g.Key(workloads.random_key(168, 128))
        sizes = [4096 * 4 ** i for i in range(10)]  # 4 KiB .. 1 GiB
        for kid in (g.KERNEL_TABLE, g.KERNEL_BITSLICED):
            for size in sizes:
                g.ecb_ex(k, x[:size], y[:size], kernel=kid)
    elif a.case == "singles":
        w = workloads.batch_workload()
        ks = [g.Key(k) for k in w.keys]
        off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
        d = g.make_descs(off, off, w.lengths // 16, np.arange(len(ks)), w.decrypt)
        x = workloads.device_bytes(4, w.total_bytes)
        y = torch.empty_like(x)
        plan = g.BatchPlan(d, ks, 512, 8)
        plan.launch(x, y)
        for i in range(len(ks)):
            o, n = int(off[i]), int(w.lengths[i])
            g.ecb_ex(ks[i], x[o:o + n], y[o:o + n], decrypt=bool(w.decrypt[i]))
    else:
        w = workloads.batch_workload(n=10000, max_len=1 << 20)
        ks = [g.Key(k) for k in w.keys]
        off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
        d = g.make_descs(off, off, w.lengths // 16, np.arange(len(ks)), w.decrypt)
        x = workloads.device_bytes(4, w.total_bytes)
        y = torch.empty_like(x)
        plan = g.BatchPlan(d, ks, 512, 8)
        for _ in range(a.warmup + a.launches):
            plan.launch(x, y)
    torch.cuda.synchronize()
    print(f"{a.case}: ok")


if __name__ == "__main__":
    main()
