"""gbaes: bulk AES on GB300 (sm_103a) -- Python binding of the C ABI in include/gbaes.h.

This module only marshals arguments: torch CUDA tensors become device pointers,
the current torch stream becomes a cudaStream_t, and error codes become
``AesError``.  Every step of the cipher runs in the CUDA kernels of
``libgbaes.so``; there is no CPU fallback, and every call raises if the library
cannot be loaded.

The cipher is AES (Section 2.1 of the paper) with rounds in the T-table form of
Eq. 1; modes are those of Section 3 (ECB, CTR, CBC decryption).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "AesError",
    "Key",
    "load",
    "encrypt_ecb",
    "decrypt_ecb",
    "ecb_ex",
    "ctr_xcrypt",
    "cbc_decrypt",
    "set_kernel",
    "set_tuning",
    "device_status",
    "key_schedule",
    "host_tables",
    "MSG_DESC",
    "make_descs",
    "BatchPlan",
    "ecb_batch",
    "batch_tiles",
    "Pipeline",
    "Server",
    "SERVER_DRYRUN",
    "SERVER_RESIDENT",
    "SERVER_PIN_THREADS",
    "Router",
    "ROUTE_LEAST_LOADED",
    "ROUTE_BY_DEVICE",
    "REQUEST",
    "COMPLETION",
    "KERNEL_TABLE",
    "KERNEL_BITSLICED",
    "KERNEL_TABLE_COMPACT",
    "KERNEL_TABLE_REPLICATED",
    "CTR_BE128",
    "CTR_LE32_CARRY",
    "PIPE_STAGED",
    "PIPE_DIRECT",
]

KERNEL_TABLE = 0
KERNEL_BITSLICED = 1
KERNEL_TABLE_COMPACT = 2
KERNEL_TABLE_REPLICATED = 3
CTR_BE128 = 0
CTR_LE32_CARRY = 1
PIPE_STAGED = 0
PIPE_DIRECT = 1

ERRORS = {
    -1: "AES_ERR_ARG",
    -2: "AES_ERR_KEYSIZE",
    -3: "AES_ERR_ALIGN",
    -4: "AES_ERR_CUDA",
    -5: "AES_ERR_BUDGET",
    -6: "AES_ERR_NOMEM",
    -7: "AES_ERR_DEVICE",
    -8: "AES_ERR_STATE",
}

_lib = None
_lock = threading.Lock()


class AesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def library_path() -> str:
    from . import _build

    return _build.LIB


def _declare(lib):
    c = ctypes
    vp, sz, u8p, u32p = c.c_void_p, c.c_size_t, c.POINTER(c.c_uint8), c.POINTER(c.c_uint32)
    sig = {
        "aes_expand_key": (vp, [u8p, c.c_int]),
        "aes_free_ctx": (None, [vp]),
        "aes_ctx_bits": (c.c_int, [vp]),
        "aes_encrypt_ecb": (c.c_int, [vp, vp, vp, sz, vp]),
        "aes_decrypt_ecb": (c.c_int, [vp, vp, vp, sz, vp]),
        "aes_ecb_ex": (c.c_int, [vp, c.c_int, vp, vp, sz, c.c_int, c.c_int, c.c_int, vp]),
        "aes_ctr_xcrypt": (c.c_int, [vp, u8p, c.c_int, c.c_uint64, vp, vp, sz, vp]),
        "aes_cbc_decrypt": (c.c_int, [vp, u8p, vp, vp, sz, vp]),
        "aes_set_kernel": (c.c_int, [c.c_int]),
        "aes_set_tuning": (c.c_int, [c.c_int, c.c_int, c.c_int, c.c_int]),
        "aes_device_status": (c.c_int, [c.c_int]),
        "aes_last_error": (c.c_char_p, []),
        "aes_key_schedule": (c.c_int, [u8p, c.c_int, u32p, u32p]),
        "aes_host_tables": (c.c_int, [u32p, u32p, u8p, u8p]),
        "aes_batch_plan_create": (vp, [vp, sz, vp, sz, c.c_int, c.c_int]),
        "aes_batch_plan_launch": (c.c_int, [vp, vp, sz, vp, sz, vp]),
        "aes_batch_plan_launch_graph": (c.c_int, [vp, vp, sz, vp, sz, vp]),
        "aes_batch_plan_info": (c.c_int, [vp, c.POINTER(c.c_uint64), u32p, u32p]),
        "aes_batch_plan_free": (None, [vp]),
        "aes_ecb_batch": (c.c_int, [vp, sz, vp, sz, vp, sz, vp, sz, vp]),
        "aes_batch_tiles": (c.c_int, [vp, sz, vp, sz, c.c_int, u32p, sz]),
        "aes_ecb_batch_noalloc": (c.c_int, [vp, sz, vp, sz, vp, sz, vp, sz, vp]),
        "aes_pipeline_create": (vp, [sz, c.c_int]),
        "aes_pipeline_create_ex": (vp, [sz, c.c_int, c.c_int]),
        "aes_pipeline_ecb": (c.c_int, [vp, vp, c.c_int, vp, vp, sz, vp]),
        "aes_pipeline_free": (None, [vp]),
        "aes_server_create": (vp, [vp, sz, vp]),
        "aes_server_submit": (c.c_int, [vp, vp]),
        "aes_server_replay": (c.c_int, [vp, vp, sz]),
        "aes_server_replay_join": (c.c_int, [vp, c.c_int]),
        "aes_server_drain": (c.c_int, [vp, c.c_double]),
        "aes_server_poll": (c.c_int, [vp, vp, sz]),
        "aes_server_get_stats": (c.c_int, [vp, vp]),
        "aes_server_get_diag": (c.c_int, [vp, vp]),
        "aes_server_inject_fault": (c.c_int, [vp, c.c_uint64]),
        "aes_server_cancel": (c.c_int, [vp, c.c_uint64]),
        "aes_server_destroy": (None, [vp]),
        "aes_router_create": (vp, [vp, sz, c.c_int]),
        "aes_router_submit": (c.c_int, [vp, vp]),
        "aes_router_poll": (c.c_int, [vp, vp, sz]),
        "aes_router_drain": (c.c_int, [vp, c.c_double]),
        "aes_router_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def load(build_if_missing: bool = True):
    """Loads libgbaes.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build

            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise AesError(-4, f"CUDA library not found at {path}; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        msg = load().aes_last_error()
        raise AesError(rc, msg.decode() if msg else "")
    return rc


def _u8p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


_torch = None


def _torch_mod():
    global _torch
    if _torch is None:
        import torch

        _torch = torch
    return _torch


def _stream_handle(stream):
    torch = _torch_mod()
    if stream is None:
        # The current stream's raw handle without building a Stream object
        # (that costs microseconds per call, as much as the launch itself).
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if raw is not None:
            return ctypes.c_void_p(raw(torch.cuda.current_device()))
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _nblocks(t) -> int:
    n = t.numel() * t.element_size()
    if n % 16:
        raise ValueError(f"buffer of {n} bytes is not a whole number of 16-byte blocks")
    return n // 16


def _ptr(t):
    torch = _torch_mod()
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Key:
    """An expanded AES key (``aes_ctx``): encryption and decryption schedules."""

    def __init__(self, key, bits: int | None = None):
        k = np.ascontiguousarray(np.frombuffer(bytes(key), np.uint8) if isinstance(key, (bytes, bytearray))
                                 else np.asarray(key, np.uint8))
        bits = bits if bits is not None else 8 * k.size
        if k.size != bits // 8:
            raise ValueError(f"key has {k.size} bytes, expected {bits // 8}")
        lib = load()
        self._lib = lib
        h = lib.aes_expand_key(_u8p(k), int(bits))
        if not h:
            _check(-2 if bits not in (128, 192, 256) else -1)
        self._h = ctypes.c_void_p(h)
        self.bits = bits

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.aes_free_ctx(h)
            self._h = None


def _out_like(x, out):
    torch = _torch_mod()
    if out is None:
        out = torch.empty_like(x)
    if out.numel() * out.element_size() != x.numel() * x.element_size():
        raise ValueError("out must have the same byte size as the input")
    return out


def encrypt_ecb(key: Key, x, out=None, stream=None):
    """ECB encryption of a CUDA tensor (any dtype; its bytes are the blocks)."""
    out = _out_like(x, out)
    _check(load().aes_encrypt_ecb(key.handle, _ptr(x), _ptr(out), _nblocks(x), _stream_handle(stream)))
    return out


def decrypt_ecb(key: Key, x, out=None, stream=None):
    """ECB decryption of a CUDA tensor."""
    out = _out_like(x, out)
    _check(load().aes_decrypt_ecb(key.handle, _ptr(x), _ptr(out), _nblocks(x), _stream_handle(stream)))
    return out


def ecb_ex(key: Key, x, out=None, decrypt=False, kernel=KERNEL_TABLE, threads=0, blocks_per_thread=0,
           stream=None):
    """ECB with an explicit kernel variant and launch shape."""
    out = _out_like(x, out)
    _check(load().aes_ecb_ex(key.handle, int(bool(decrypt)), _ptr(x), _ptr(out), _nblocks(x), int(kernel),
                             int(threads), int(blocks_per_thread), _stream_handle(stream)))
    return out


def _iv(iv) -> np.ndarray:
    v = np.ascontiguousarray(np.frombuffer(bytes(iv), np.uint8))
    if v.size != 16:
        raise ValueError("iv must be 16 bytes")
    return v


def ctr_xcrypt(key: Key, iv, x, out=None, kind=CTR_BE128, first_block=0, stream=None):
    """CTR mode (Section 3): x XOR E_K(counter(first_block + i))."""
    out = _out_like(x, out)
    v = _iv(iv)
    _check(load().aes_ctr_xcrypt(key.handle, _u8p(v), int(kind), int(first_block), _ptr(x), _ptr(out),
                                 _nblocks(x), _stream_handle(stream)))
    return out


def cbc_decrypt(key: Key, iv, x, out=None, stream=None):
    """CBC decryption (Section 3, Eq. 2)."""
    out = _out_like(x, out)
    v = _iv(iv)
    _check(load().aes_cbc_decrypt(key.handle, _u8p(v), _ptr(x), _ptr(out), _nblocks(x), _stream_handle(stream)))
    return out


def set_kernel(which: int) -> int:
    return _check(load().aes_set_kernel(int(which)))


def set_tuning(bits: int, decrypt: bool, threads: int, blocks_per_thread: int) -> None:
    _check(load().aes_set_tuning(int(bits), int(bool(decrypt)), int(threads), int(blocks_per_thread)))


def device_status(clear: bool = False) -> int:
    """The library's device status word (0 = no kernel reported an error). Synchronises."""
    return _check(load().aes_device_status(int(bool(clear))))


def key_schedule(key, bits: int):
    """Host-side schedules (enc, dec) as (Nr+1, 4) uint32 arrays; needs no GPU."""
    k = np.ascontiguousarray(np.frombuffer(bytes(key), np.uint8))
    enc = np.zeros(60, np.uint32)
    dec = np.zeros(60, np.uint32)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    nr = _check(load().aes_key_schedule(_u8p(k), int(bits), enc.ctypes.data_as(u32), dec.ctypes.data_as(u32)))
    return enc[: 4 * (nr + 1)].reshape(nr + 1, 4), dec[: 4 * (nr + 1)].reshape(nr + 1, 4)


def host_tables():
    """The library's generated tables (Te0, Td0, S-box, inverse S-box); needs no GPU."""
    te0 = np.zeros(256, np.uint32)
    td0 = np.zeros(256, np.uint32)
    s = np.zeros(256, np.uint8)
    si = np.zeros(256, np.uint8)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    _check(load().aes_host_tables(te0.ctypes.data_as(u32), td0.ctypes.data_as(u32), _u8p(s), _u8p(si)))
    return te0, td0, s, si


# ------------------------------------------------------------------- batched

# Matches struct aes_msg_desc (32 bytes).
MSG_DESC = np.dtype([("in_off", "<u8"), ("out_off", "<u8"), ("nblocks", "<u8"), ("key_index", "<u4"),
                     ("decrypt", "<u4")])


def make_descs(in_off, out_off, nblocks, key_index, decrypt) -> np.ndarray:
    """Array of aes_msg_desc from per-message sequences (byte offsets, blocks, key index, direction)."""
    n = len(nblocks)
    d = np.zeros(n, MSG_DESC)
    d["in_off"] = np.asarray(in_off, np.uint64)
    d["out_off"] = np.asarray(out_off, np.uint64)
    d["nblocks"] = np.asarray(nblocks, np.uint64)
    d["key_index"] = np.asarray(key_index, np.uint32)
    d["decrypt"] = np.asarray(decrypt, np.uint32)
    return d


def _ctx_array(keys):
    arr = (ctypes.c_void_p * max(1, len(keys)))(*[k.handle.value for k in keys])
    return arr


class BatchPlan:
    """A reusable batched launch (aes_batch_plan): descriptors + key contexts."""

    def __init__(self, descs: np.ndarray, keys, threads: int = 0, blocks_per_thread: int = 0):
        descs = np.ascontiguousarray(descs, MSG_DESC)
        self._lib = load()
        self._keys = list(keys)  # keep the contexts alive
        ctxs = _ctx_array(self._keys)
        h = self._lib.aes_batch_plan_create(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(self._keys),
                                            int(threads), int(blocks_per_thread))
        if not h:
            _check(-1)
        self._h = ctypes.c_void_p(h)

    def info(self):
        tb = ctypes.c_uint64()
        nt = ctypes.c_uint32()
        tbl = ctypes.c_uint32()
        _check(self._lib.aes_batch_plan_info(self._h, ctypes.byref(tb), ctypes.byref(nt), ctypes.byref(tbl)))
        return {"total_blocks": tb.value, "ntiles": nt.value, "tile_blocks": tbl.value}

    def launch(self, inp, out, stream=None, graph: bool = False):
        fn = self._lib.aes_batch_plan_launch_graph if graph else self._lib.aes_batch_plan_launch
        _check(fn(self._h, _ptr(inp), inp.numel() * inp.element_size(), _ptr(out), out.numel() * out.element_size(),
                  _stream_handle(stream)))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.aes_batch_plan_free(h)
            self._h = None


def ecb_batch(descs: np.ndarray, keys, inp, out, stream=None):
    """One-shot batched launch (stream-ordered scratch for the plan tables)."""
    descs = np.ascontiguousarray(descs, MSG_DESC)
    ctxs = _ctx_array(list(keys))
    _check(load().aes_ecb_batch(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(keys), _ptr(inp),
                                inp.numel() * inp.element_size(), _ptr(out), out.numel() * out.element_size(),
                                _stream_handle(stream)))
    return out


def batch_tiles(descs: np.ndarray, keys, tile_blocks: int) -> np.ndarray:
    """Host-only tiling of a batch: caller's index of each tile's first message."""
    descs = np.ascontiguousarray(descs, MSG_DESC)
    ctxs = _ctx_array(list(keys))
    lib = load()
    n = _check(lib.aes_batch_tiles(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(keys), int(tile_blocks),
                                   None, 0))
    out = np.zeros(max(n, 1), np.uint32)
    _check(lib.aes_batch_tiles(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(keys), int(tile_blocks),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), out.size))
    return out[:n]


# ------------------------------------------------------------- host pipeline


class Pipeline:
    """ECB on page-locked host buffers (aes_pipeline): through device staging
    slots and copy engines (mode PIPE_STAGED), or with the kernel reading and
    writing the host buffers over the host link (PIPE_DIRECT)."""

    def __init__(self, chunk_bytes: int = 64 << 20, depth: int = 4, mode: int = 0):
        self._lib = load()
        h = self._lib.aes_pipeline_create_ex(int(chunk_bytes), int(depth), int(mode))
        if not h:
            _check(-1)
        self._h = ctypes.c_void_p(h)

    def ecb(self, key: Key, host_in, host_out=None, decrypt: bool = False, stream=None):
        """host_in/host_out: pinned CPU tensors (torch.empty(..., pin_memory=True))."""
        import torch

        if host_out is None:
            host_out = torch.empty_like(host_in).pin_memory()
        if host_out.numel() * host_out.element_size() != host_in.numel() * host_in.element_size():
            raise ValueError("host_out must have the same byte size as host_in")
        _check(self._lib.aes_pipeline_ecb(self._h, key.handle, int(bool(decrypt)), _ptr(host_in), _ptr(host_out),
                                          _nblocks(host_in), _stream_handle(stream)))
        return host_out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.aes_pipeline_free(h)
            self._h = None


# ------------------------------------------------------------------- serving

SERVER_DRYRUN = 1
SERVER_RESIDENT = 2
SERVER_PIN_THREADS = 4

# Match aes_server_request / aes_server_completion (48 and 40 bytes).
REQUEST = np.dtype([("id", "<u8"), ("in_ptr", "<u8"), ("out_ptr", "<u8"), ("nblocks", "<u8"), ("key_index", "<u4"),
                    ("decrypt", "<u4"), ("arrival_s", "<f8")])
COMPLETION = np.dtype([("id", "<u8"), ("status", "<i4"), ("batch_msgs", "<u4"), ("arrival_s", "<f8"),
                       ("launch_s", "<f8"), ("done_s", "<f8")])


class _ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("nstreams", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_thread", ctypes.c_int32), ("max_batch_msgs", ctypes.c_uint32),
                ("dryrun_batch_us", ctypes.c_uint32), ("max_batch_blocks", ctypes.c_uint64),
                ("resident_idle_us", ctypes.c_uint32), ("resident_lifetime_ms", ctypes.c_uint32),
                ("ring_tiles", ctypes.c_uint32), ("ring_items", ctypes.c_uint32),
                ("resident_restart_pct", ctypes.c_uint32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "rejected", "batches",
                                               "max_inflight_bytes", "max_queue", "max_batch_msgs", "budget_bytes",
                                               "recovered_tiles", "lost_completions")]


class _ServerDiag(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_uint64) for n in ("sched_passes", "sched_worst_window_ns", "sched_worst_window_cpu_ns",
                                                "sched_worst_window_invol", "sched_worst_window_vol",
                                                "sched_worst_window_at_ns", "sched_worst_window_minflt",
                                                "sched_worst_window_majflt", "sched_invol")] +
                [("lock_wait_max_ns", ctypes.c_uint64 * 3), ("lock_wait_at_ns", ctypes.c_uint64 * 3)] +
                [(n, ctypes.c_uint64) for n in ("cuda_call_max_ns", "cuda_call_at_ns")] +
                [("stream_queries", ctypes.c_uint64 * 2)] +
                [("sched_phase_max_ns", ctypes.c_uint64 * 5), ("sched_phase_at_ns", ctypes.c_uint64 * 5),
                 ("inbox_hold_max_ns", ctypes.c_uint64 * 2)] +
                [(n, ctypes.c_uint64) for n in ("producer_late_max_ns", "producer_late_at_ns", "producer_late_invol",
                                                "producer_invol", "producer_check_max_ns", "producer_check_at_ns")] +
                [("sched_cpu", ctypes.c_int64), ("producer_cpu", ctypes.c_int64),
                 ("sched_minflt", ctypes.c_uint64), ("producer_minflt", ctypes.c_uint64)])


class Server:
    """Continuous-batching server (aes_server) with resident keys.  resident=True:
    one kernel stays on the GPU and takes requests from a ring in page-locked
    memory (AES_SERVER_RESIDENT) instead of one launch per micro-batch."""

    def __init__(self, keys, budget_bytes: int = 8 << 30, nstreams: int = 4, threads: int = 0,
                 blocks_per_thread: int = 0, max_batch_msgs: int = 0, max_batch_blocks: int = 0, dryrun: bool = False,
                 dryrun_batch_us: int = 0, resident: bool = False, resident_idle_us: int = 0,
                 resident_lifetime_ms: int = 0, ring_tiles: int = 0, ring_items: int = 0,
                 resident_restart_pct: int = 0, pin_threads: bool = False):
        self._lib = load()
        self._keys = list(keys)
        flags = ((SERVER_DRYRUN if dryrun else 0) | (SERVER_RESIDENT if resident else 0) |
                 (SERVER_PIN_THREADS if pin_threads else 0))
        cfg = _ServerConfig(int(budget_bytes), int(nstreams), flags, int(threads), int(blocks_per_thread),
                            int(max_batch_msgs), int(dryrun_batch_us), int(max_batch_blocks), int(resident_idle_us),
                            int(resident_lifetime_ms), int(ring_tiles), int(ring_items), int(resident_restart_pct))
        h = self._lib.aes_server_create(_ctx_array(self._keys), len(self._keys), ctypes.byref(cfg))
        if not h:
            _check(-1)
        self._h = ctypes.c_void_p(h)

    def submit(self, req_id: int, key_index: int, in_ptr: int, out_ptr: int, nblocks: int, decrypt: bool = False):
        r = np.zeros(1, REQUEST)
        r["id"], r["in_ptr"], r["out_ptr"], r["nblocks"] = req_id, in_ptr, out_ptr, nblocks
        r["key_index"], r["decrypt"] = key_index, int(bool(decrypt))
        _check(self._lib.aes_server_submit(self._h, ctypes.c_void_p(r.ctypes.data)))

    def replay(self, reqs: np.ndarray):
        """Open-loop replay of a REQUEST array (arrival_s non-decreasing) on a native thread."""
        self._replay = np.ascontiguousarray(reqs, REQUEST)
        _check(self._lib.aes_server_replay(self._h, ctypes.c_void_p(self._replay.ctypes.data), self._replay.size))

    def replay_join(self, stop_early: bool = False):
        _check(self._lib.aes_server_replay_join(self._h, int(bool(stop_early))))

    def drain(self, timeout_s: float = -1.0):
        _check(self._lib.aes_server_drain(self._h, float(timeout_s)))

    def poll(self, max_items: int = 1 << 22, out: np.ndarray | None = None) -> np.ndarray:
        """Up to max_items completions (into `out`, a COMPLETION array, if given: a buffer reused across
        polls spares the server's lock a copy into fresh memory)."""
        if out is None:
            out = np.zeros(max_items, COMPLETION)
        max_items = min(max_items, out.size)
        n = _check(self._lib.aes_server_poll(self._h, ctypes.c_void_p(out.ctypes.data), max_items))
        return out[:n]

    def poll_all(self) -> np.ndarray:
        parts = []
        while True:
            p = self.poll()
            if p.size == 0:
                break
            parts.append(p)
        return np.concatenate(parts) if parts else np.zeros(0, COMPLETION)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(self._lib.aes_server_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in s._fields_}

    def diag(self) -> dict:
        """Host-thread diagnostics (aes_server_diag); lock waits by lock: submissions, completions, stats."""
        d = _ServerDiag()
        _check(self._lib.aes_server_get_diag(self._h, ctypes.byref(d)))
        out = {}
        for n, _ in d._fields_:
            v = getattr(d, n)
            out[n] = list(v) if isinstance(v, ctypes.Array) else v
        return out

    def cancel(self, req_id: int):
        """Cancels a request still waiting for admission (it completes with AES_ERR_STATE)."""
        _check(self._lib.aes_server_cancel(self._h, int(req_id)))

    def inject_fault(self, batch_index: int):
        _check(self._lib.aes_server_inject_fault(self._h, int(batch_index)))

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.aes_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


ROUTE_LEAST_LOADED = 0
ROUTE_BY_DEVICE = 1


class Router:
    """Several servers (e.g. one per GPU) behind one submission point (aes_router).
    The servers stay owned by the caller."""

    def __init__(self, servers, policy: int = ROUTE_LEAST_LOADED):
        self._lib = load()
        self._servers = list(servers)
        arr = (ctypes.c_void_p * len(self._servers))(*[srv._h for srv in self._servers])
        h = self._lib.aes_router_create(arr, len(self._servers), int(policy))
        if not h:
            _check(-1)
        self._h = ctypes.c_void_p(h)

    def submit(self, req_id: int, key_index: int, in_ptr: int, out_ptr: int, nblocks: int,
               decrypt: bool = False) -> int:
        """Returns the index of the server the request went to."""
        r = np.zeros(1, REQUEST)
        r["id"], r["in_ptr"], r["out_ptr"], r["nblocks"] = req_id, in_ptr, out_ptr, nblocks
        r["key_index"], r["decrypt"] = key_index, int(bool(decrypt))
        return _check(self._lib.aes_router_submit(self._h, ctypes.c_void_p(r.ctypes.data)))

    def drain(self, timeout_s: float = -1.0):
        _check(self._lib.aes_router_drain(self._h, float(timeout_s)))

    def poll(self, max_items: int = 1 << 22) -> np.ndarray:
        out = np.zeros(max_items, COMPLETION)
        n = _check(self._lib.aes_router_poll(self._h, ctypes.c_void_p(out.ctypes.data), max_items))
        return out[:n]

    def poll_all(self) -> np.ndarray:
        parts = []
        while True:
            p = self.poll()
            if p.size == 0:
                break
            parts.append(p)
        return np.concatenate(parts) if parts else np.zeros(0, COMPLETION)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.aes_router_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
