"""GB300-native percolation inspection (Xu, Xu & Yakobson, arXiv:1401.2130).

Thin Python binding of ``libpercol.so`` (C ABI in ``include/percol.h``).  The
functions keep the C names and only marshal arguments: every step of the
inspection runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpercol.so")

PC_OK = 0
PC_ERR_ARG = -1
PC_ERR_OOM = -2
PC_ERR_CUDA = -3
PC_ERR_TIMEOUT = -4
PC_ERR_BUSY = -5
PC_ERR_CANCELLED = -6
PC_ERR_INTERNAL = -7
PC_OUT_DEVICE = 0x1
PC_ASYNC = 0x2
PC_MODE_RESIDENT = 0x10
PC_MODE_STREAM = 0x20
PC_BITS_ONLY = 0x40
PC_VERDICT_FIRST = 0x80

_STATUS = {PC_ERR_ARG: "PC_ERR_ARG", PC_ERR_OOM: "PC_ERR_OOM", PC_ERR_CUDA: "PC_ERR_CUDA",
           PC_ERR_TIMEOUT: "PC_ERR_TIMEOUT", PC_ERR_BUSY: "PC_ERR_BUSY",
           PC_ERR_CANCELLED: "PC_ERR_CANCELLED", PC_ERR_INTERNAL: "PC_ERR_INTERNAL"}

# Every symbol include/percol.h declares, with its ctypes signature.
_i32, _i64, _u64, _dbl, _vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_void_p)
SIGNATURES = {
    "pc_lattice_info": [_i32, _i32, _vp, _vp],
    "pc_occupancy": [_i32, _i32, _dbl, _u64, _i64, _i64, _vp, _vp],
    "pc_occupancy_fixed": [_i32, _i32, _i64, _u64, _i64, _i64, _vp, _vp],
    "pc_inspect": [_i32, _i32, _dbl, _u64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp],
    "pc_inspect_occupancy": [_i32, _i32, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp],
    "pc_inspect_static": [_i32, _i32, _dbl, _u64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "pc_batch_run": [_vp, _i64, _vp, _i32, _vp],
    "pc_server_create": [_vp, _vp],
    "pc_server_submit": [_vp, _vp, _vp],
    "pc_server_poll": [_vp, ctypes.c_uint64, _vp, _i64],
    "pc_server_cancel": [_vp, ctypes.c_uint64],
    "pc_server_get_stats": [_vp, _vp],
    "pc_server_destroy": [_vp],
    "pc_lattice_layout": [_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "pc_stream_layout": [_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "pc_bits_blocked_shape": [_i32, _vp, _vp, _vp, _vp],
    "pc_lazy_mass": [_vp, _vp, _i64, _dbl, _vp, _i32, _vp],
    "pc_shutdown": [],
    "pc_last_error": [],
}


class PercolError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libpercol.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "pc_last_error" else ctypes.c_int32
    _lib = lib
    return lib


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def _check(st: int):
    if st != PC_OK:
        msg = load().pc_last_error()
        raise PercolError(st, msg.decode() if msg else "")


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def pc_lattice_info(W: int, L: int) -> tuple[int, int]:
    """(A, N): columns of the hexagon of radius W and A*L sites (Sec. II.A)."""
    a = ctypes.c_int64(); n = ctypes.c_int64()
    _check(load().pc_lattice_info(W, L, ctypes.byref(a), ctypes.byref(n)))
    return a.value, n.value


def pc_lattice_layout(W: int) -> dict:
    """Plane layout of radius W used by the FP arrays (see percol.h)."""
    lib = load()
    P, sb, ns = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.pc_lattice_layout(W, ctypes.addressof(P), ctypes.addressof(sb), ctypes.addressof(ns),
                                 None, None, None, None))
    A = 3 * W * (W + 1) + 1
    sr = np.zeros(ns.value, np.int16); ro = np.zeros((2 * W + 1, 4), np.int32)
    pp = np.zeros(A, np.int32); pcl = np.zeros(P.value, np.int32)
    _check(lib.pc_lattice_layout(W, None, None, None, _ptr(sr), _ptr(ro), _ptr(pp), _ptr(pcl)))
    return {"P": P.value, "s_begin": sb.value, "n_strips": ns.value, "strip_row": sr,
            "row_off": ro, "ppos": pp, "pcol": pcl}


def pc_bits_blocked_shape(W: int) -> dict | None:
    """Cluster shape of the verdict-only solver with temporal blocking for
    radius W on the current device, or None where the step-synchronous
    solver runs PC_BITS_ONLY inspections instead (see percol.h)."""
    lib = load()
    v = [ctypes.c_int32() for _ in range(4)]
    st = lib.pc_bits_blocked_shape(W, *[ctypes.addressof(x) for x in v])
    if st == PC_ERR_ARG and 0 <= W <= 255:
        return None
    _check(st)
    return dict(zip(("cluster_size", "columns_per_cta", "slab_rows", "clusters"), (x.value for x in v)))


def pc_stream_layout(W: int) -> dict:
    """Paired plane layout of radius W used by the streamed solver (see percol.h)."""
    lib = load()
    P, sb, ns = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.pc_stream_layout(W, ctypes.addressof(P), ctypes.addressof(sb), ctypes.addressof(ns),
                                None, None, None, None))
    A = 3 * W * (W + 1) + 1
    sr = np.zeros(ns.value, np.int16); ro = np.zeros((2 * W + 1, 4), np.int32)
    pp = np.zeros(A, np.int32); pcl = np.zeros(P.value, np.int32)
    _check(lib.pc_stream_layout(W, None, None, None, _ptr(sr), _ptr(ro), _ptr(pp), _ptr(pcl)))
    return {"P": P.value, "s_begin": sb.value, "n_strips": ns.value, "strip_row": sr,
            "row_off": ro, "ppos": pp, "pcol": pcl}


def words_per_config(W: int, L: int) -> int:
    return (pc_lattice_info(W, L)[1] + 31) // 32


def pc_occupancy(W: int, L: int, p: float, seed: int, config_begin: int, n_configs: int,
                 out=None, stream=None):
    """Bit-packed occupancy [n_configs, ceil(N/32)] (int32 view of uint32 words)
    on the current CUDA device (Sec. II.A)."""
    import torch
    wpc = words_per_config(W, L)
    if out is None:
        out = torch.empty((n_configs, wpc), dtype=torch.int32, device="cuda")
    assert out.is_cuda and out.is_contiguous() and out.numel() >= n_configs * wpc
    _check(load().pc_occupancy(W, L, float(p), int(seed) & (2**64 - 1), config_begin,
                               n_configs, _ptr(out), _stream_handle(stream)))
    return out


def pc_occupancy_fixed(W: int, L: int, n_metallic: int, seed: int, config_begin: int,
                       n_configs: int, out=None, stream=None):
    """Fixed-count occupancy (Sec. II.A: exactly n_metallic metallic sites per
    configuration, a uniformly random subset), in pc_occupancy's layout."""
    import torch
    wpc = words_per_config(W, L)
    if out is None:
        out = torch.empty((n_configs, wpc), dtype=torch.int32, device="cuda")
    assert out.is_cuda and out.is_contiguous() and out.numel() >= n_configs * wpc
    _check(load().pc_occupancy_fixed(W, L, int(n_metallic), int(seed) & (2**64 - 1), config_begin,
                                     n_configs, _ptr(out), _stream_handle(stream)))
    return out


def _alloc_outputs(n: int, device: bool, want: tuple):
    if device:
        import torch
        mk = lambda dt: torch.empty(n, dtype=dt, device="cuda")
        out = {"verdict": mk(torch.uint8)}
        if "first_hit" in want: out["first_hit"] = mk(torch.int32)
        if "mass" in want: out["mass"] = mk(torch.float32)
        if "m_stop" in want: out["m_stop"] = mk(torch.int32)
        out["n_percolating"] = torch.zeros(1, dtype=torch.int64, device="cuda")
        return out
    out = {"verdict": np.zeros(n, np.uint8)}
    if "first_hit" in want: out["first_hit"] = np.zeros(n, np.int32)
    if "mass" in want: out["mass"] = np.zeros(n, np.float32)
    if "m_stop" in want: out["m_stop"] = np.zeros(n, np.int32)
    return out


ALL_OUTPUTS = ("first_hit", "mass", "m_stop")


def pc_inspect(W: int, L: int, p: float, seed: int, config_begin: int, n_configs: int, *,
               device: bool = False, want: tuple = ALL_OUTPUTS, mode: int = 0,
               stream=None, out: dict | None = None, bits_only: bool = False,
               verdict_first: bool = False) -> dict:
    """Inspect configurations config_begin..+n_configs-1 (Sec. II.B, Eqs. (1)-(4)).

    bits_only: propagate the exact reached set alone (verdicts, first_hit,
    m_stop; mass is 0).
    verdict_first: the same outputs, bit for bit, with the FP32 recursion run
    only on the configurations that percolate (resident solver).

    device=False: numpy outputs plus ``n_percolating`` and ``Pi`` (the call
    synchronises).  device=True: torch CUDA tensors written asynchronously on
    ``stream``; ``n_percolating`` is a one-element int64 tensor.
    ``out`` may pass preallocated outputs of the same form.
    """
    o = out if out is not None else _alloc_outputs(n_configs, device, want)
    flags = (mode | (PC_OUT_DEVICE if device else 0) | (PC_BITS_ONLY if bits_only else 0)
             | (PC_VERDICT_FIRST if verdict_first else 0))
    npc = ctypes.c_int64(0); pi = ctypes.c_double(0.0)
    _check(load().pc_inspect(
        W, L, float(p), int(seed) & (2**64 - 1), config_begin, n_configs,
        _ptr(o["verdict"]), _ptr(o.get("first_hit")), _ptr(o.get("mass")), _ptr(o.get("m_stop")),
        _ptr(o["n_percolating"]) if device else ctypes.addressof(npc),
        None if device else ctypes.addressof(pi), flags, _stream_handle(stream)))
    if not device:
        o["n_percolating"] = npc.value
        o["Pi"] = pi.value
    return o


def pc_lazy_mass(first_hit, mass, hold: float, *, out=None, stream=None):
    """Mass at the first hit under the lazy walk hold * I + (1 - hold) * P
    (the self-loop remark of Sec. II.B), from pc_inspect's first_hit and mass:
    mass * (1 - hold)^first_hit, 0 where first_hit <= 0.  numpy arrays in,
    numpy out (synchronising); torch CUDA tensors in, a CUDA tensor out
    written asynchronously on ``stream``."""
    device = hasattr(mass, "is_cuda") and mass.is_cuda
    n = int(mass.shape[0])
    if device:
        import torch
        assert first_hit.is_cuda and first_hit.dtype == torch.int32 and mass.dtype == torch.float32
        assert first_hit.is_contiguous() and mass.is_contiguous() and first_hit.shape[0] == n
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=mass.device)
    else:
        first_hit = np.ascontiguousarray(first_hit, dtype=np.int32)
        mass = np.ascontiguousarray(mass, dtype=np.float32)
        if first_hit.shape[0] != n:
            raise ValueError("first_hit and mass differ in length")
        if out is None:
            out = np.zeros(n, np.float32)
    _check(load().pc_lazy_mass(_ptr(first_hit), _ptr(mass), n, float(hold), _ptr(out),
                               PC_OUT_DEVICE if device else 0, _stream_handle(stream)))
    return out


def pc_inspect_occupancy(W: int, L: int, occ_bits, *, device: bool = False,
                         want: tuple = ALL_OUTPUTS, mode: int = 0, stream=None,
                         out: dict | None = None) -> dict:
    """As pc_inspect for caller occupancies: ``occ_bits`` is a CUDA int32/uint32
    tensor [n_configs, ceil(N/32)] in pc_occupancy's layout."""
    wpc = words_per_config(W, L)
    assert occ_bits.is_cuda and occ_bits.is_contiguous() and occ_bits.element_size() == 4
    n = occ_bits.numel() // wpc if occ_bits.numel() else 0
    assert n * wpc == occ_bits.numel()
    o = out if out is not None else _alloc_outputs(n, device, want)
    flags = mode | (PC_OUT_DEVICE if device else 0)
    npc = ctypes.c_int64(0); pi = ctypes.c_double(0.0)
    _check(load().pc_inspect_occupancy(
        W, L, _ptr(occ_bits), n,
        _ptr(o["verdict"]), _ptr(o.get("first_hit")), _ptr(o.get("mass")), _ptr(o.get("m_stop")),
        _ptr(o["n_percolating"]) if device else ctypes.addressof(npc),
        None if device else ctypes.addressof(pi), flags, _stream_handle(stream)))
    if not device:
        o["n_percolating"] = npc.value
        o["Pi"] = pi.value
    return o


def pc_inspect_static(W: int, L: int, p: float, seed: int, config_begin: int,
                      n_configs: int, stream=None) -> dict:
    """pc_inspect without device allocation (host outputs; see percol.h):
    for callers that cannot call cudaMalloc, e.g. because their framework's
    pool allocator owns the device memory, or because an allocation could
    synchronise the device inside a latency-critical loop."""
    o = _alloc_outputs(n_configs, False, ALL_OUTPUTS)
    npc = ctypes.c_int64(0); pi = ctypes.c_double(0.0)
    _check(load().pc_inspect_static(
        W, L, float(p), int(seed) & (2**64 - 1), config_begin, n_configs,
        _ptr(o["verdict"]), _ptr(o["first_hit"]), _ptr(o["mass"]), _ptr(o["m_stop"]),
        ctypes.addressof(npc), ctypes.addressof(pi), _stream_handle(stream)))
    o["n_percolating"] = npc.value
    o["Pi"] = pi.value
    return o


class PcQuery(ctypes.Structure):
    """Mirror of pc_query (include/percol.h)."""
    _fields_ = [("W", ctypes.c_int32), ("L", ctypes.c_int32), ("p", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("config_begin", ctypes.c_int64),
                ("n_configs", ctypes.c_int64), ("verdicts", ctypes.c_void_p),
                ("first_hit", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("m_stop", ctypes.c_void_p), ("n_percolating", ctypes.c_void_p)]


class PcResult(ctypes.Structure):
    """Mirror of pc_result (include/percol.h)."""
    _fields_ = [("n_percolating", ctypes.c_int64), ("Pi", ctypes.c_double),
                ("solver", ctypes.c_int32), ("threads", ctypes.c_int32)]


def batch_queries(specs, *, device: bool, outs: list | None = None):
    """ctypes query array for specs [(W, L, p, seed, config_begin, n_configs)],
    with outputs allocated (or taken from ``outs``) per query."""
    outs = outs if outs is not None else [_alloc_outputs(sp[5], device, ALL_OUTPUTS) for sp in specs]
    arr = (PcQuery * len(specs))()
    for i, (W, L, p, seed, b, n) in enumerate(specs):
        o = outs[i]
        arr[i] = PcQuery(W, L, float(p), int(seed) & (2**64 - 1), b, n, _ptr(o["verdict"]),
                         _ptr(o.get("first_hit")), _ptr(o.get("mass")), _ptr(o.get("m_stop")),
                         _ptr(o["n_percolating"]) if device else None)
    return arr, outs


def pc_batch_run(specs, *, device: bool = False, async_: bool = False, stream=None,
                 outs: list | None = None, queries=None, bits_only: bool = False,
                 verdict_first: bool = False):
    """Inspect a batch of queries [(W, L, p, seed, config_begin, n_configs)] in
    one submission (one cached CUDA graph).  Returns (outs, results): per-query
    outputs (numpy, or torch CUDA tensors with ``device``) and the host
    summaries (None with ``async_``).  Passing the same ``outs`` (and
    ``queries``) again replays the cached graph."""
    if queries is None:
        queries, outs = batch_queries(specs, device=device, outs=outs)
    flags = ((PC_OUT_DEVICE if device else 0) | (PC_ASYNC if async_ else 0) | (PC_BITS_ONLY if bits_only else 0)
             | (PC_VERDICT_FIRST if verdict_first else 0))
    res = None if async_ else (PcResult * len(specs))()
    _check(load().pc_batch_run(ctypes.addressof(queries), len(specs),
                               None if res is None else ctypes.addressof(res), flags,
                               _stream_handle(stream)))
    if res is None:
        return outs, None
    results = [{"n_percolating": r.n_percolating, "Pi": r.Pi,
                "solver": {0: "resident", 1: "streamed", 2: "blocked"}.get(r.solver, str(r.solver)),
                "threads": r.threads}
               for r in res]
    if not device:
        for o, r in zip(outs, results):
            o["n_percolating"] = r["n_percolating"]
            o["Pi"] = r["Pi"]
    return outs, results


class PcServerOpts(ctypes.Structure):
    """Mirror of pc_server_opts."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("max_slots_per_query", ctypes.c_int32), ("ticks_per_poll", ctypes.c_int32),
                ("max_pending", ctypes.c_int64), ("max_W", ctypes.c_int32)]


class PcServerStats(ctypes.Structure):
    """Mirror of pc_server_stats."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("configs_completed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("configs_per_s", ctypes.c_double)]


def pc_server_create(hbm_budget_bytes: int = 8 << 30, max_slots: int = 256,
                     max_slots_per_query: int = 64, ticks_per_poll: int = 8,
                     max_pending: int = 1 << 16, max_W: int = 0) -> int:
    """Create a serving loop on the current CUDA device; returns its handle."""
    opts = PcServerOpts(hbm_budget_bytes, max_slots, max_slots_per_query, ticks_per_poll,
                        max_pending, max_W)
    h = ctypes.c_void_p()
    _check(load().pc_server_create(ctypes.addressof(opts), ctypes.addressof(h)))
    return h.value


def pc_server_submit(handle: int, spec, outs: dict) -> int:
    """Submit (W, L, p, seed, config_begin, n_configs); ``outs`` are host numpy
    buffers (from _alloc_outputs) that must stay alive until the poll."""
    W, L, p, seed, b, n = spec
    q = PcQuery(W, L, float(p), int(seed) & (2**64 - 1), b, n, _ptr(outs["verdict"]),
                _ptr(outs.get("first_hit")), _ptr(outs.get("mass")), _ptr(outs.get("m_stop")), None)
    t = ctypes.c_uint64()
    _check(load().pc_server_submit(handle, ctypes.addressof(q), ctypes.addressof(t)))
    return t.value


def pc_server_poll(handle: int, ticket: int, timeout_s: float = 0.0):
    """Result dict once the ticket is done, None while it runs (PC_ERR_BUSY)."""
    r = PcResult()
    st = load().pc_server_poll(handle, ticket, ctypes.addressof(r), int(timeout_s * 1e9))
    if st == PC_ERR_BUSY:
        return None
    _check(st)
    return {"n_percolating": r.n_percolating, "Pi": r.Pi,
            "solver": "resident" if r.solver == 0 else "streamed"}


def pc_server_cancel(handle: int, ticket: int):
    _check(load().pc_server_cancel(handle, ticket))


def pc_server_get_stats(handle: int) -> dict:
    st = PcServerStats()
    _check(load().pc_server_get_stats(handle, ctypes.addressof(st)))
    return {k: getattr(st, k) for k, _ in PcServerStats._fields_}


def pc_server_destroy(handle: int):
    _check(load().pc_server_destroy(handle))


class Server:
    """Convenience wrapper: keeps each submission's host outputs alive."""

    def __init__(self, **opts):
        self.handle = pc_server_create(**opts)
        self.outs: dict[int, dict] = {}

    def submit(self, spec) -> int:
        o = _alloc_outputs(spec[5], False, ALL_OUTPUTS)
        t = pc_server_submit(self.handle, spec, o)
        self.outs[t] = o
        return t

    def poll(self, ticket: int, timeout_s: float = 0.0):
        r = pc_server_poll(self.handle, ticket, timeout_s)
        if r is None:
            return None
        o = self.outs.pop(ticket)
        o.update(r)
        return o

    def cancel(self, ticket: int):
        pc_server_cancel(self.handle, ticket)

    def stats(self) -> dict:
        return pc_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            pc_server_destroy(self.handle)
            self.handle = None


def pc_shutdown():
    _check(load().pc_shutdown())


def site_updates(A: int, L: int, verdict, first_hit, m_stop) -> int:
    """Site updates the forward recursion performed: every computed step m
    sweeps the causal window of min(m + 1, L) layers of A sites.  A
    percolating configuration computes steps 1..first_hit-1 (step first_hit
    only reads the detector); a non-percolating one steps 1..m_stop."""
    v = np.asarray(verdict).astype(np.int64)
    fh = np.asarray(first_hit).astype(np.int64)
    ms = np.asarray(m_stop).astype(np.int64)
    M = np.maximum(np.where(v != 0, fh - 1, ms), 0)
    k = np.minimum(M, L - 1)
    s = k * (k + 3) // 2 + np.maximum(M - k, 0) * L
    return int(s.sum()) * A
