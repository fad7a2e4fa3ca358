"""Thin ctypes binding of libbpq (include/bpq.h).

Argument marshalling only: torch supplies device memory and streams, every
step of sampling and decoding runs in the library's CUDA kernels.  There is
no CPU fallback: if libbpq.so cannot be loaded, the import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

PLANAR, TORIC, XZZX = 0, 1, 2
PLAIN, MOMENTUM, ADAGRAD, EWAINIT, AEWA = 0, 1, 2, 3, 4
CODES = {"planar": PLANAR, "toric": TORIC, "xzzx": XZZX}
VARIANTS = {"plain": PLAIN, "momentum": MOMENTUM, "adagrad": ADAGRAD, "ewainit": EWAINIT, "aewa": AEWA}


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("gamma", ctypes.c_float), ("eps", ctypes.c_float),
                ("msg_clip", ctypes.c_float), ("adagrad_g_from_iter1", ctypes.c_int32)]


class BPQError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libbpq.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.OUT
        if _build._stale():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: the CUDA library was not built")
        L = ctypes.CDLL(path)
        P, i, u64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
        PP = ctypes.POINTER(ctypes.c_void_p)
        pi = ctypes.POINTER(ctypes.c_int)
        sig = {
            "bpq_default_params": (None, [i, ctypes.POINTER(Params)]),
            "bpq_build_tanner": (i, [i, i, PP]),
            "bpq_tanner_from_paulis": (i, [i, i, P, PP]),
            "bpq_tanner_set_logicals": (i, [P, i, P]),
            "bpq_tanner_upload": (i, [P, i]),
            "bpq_tanner_info": (i, [P, pi, pi, pi, pi]),
            "bpq_tanner_layout": (i, [P, pi]),
            "bpq_tanner_export": (i, [P, P, P, P]),
            "bpq_tanner_logicals": (i, [P, P]),
            "bpq_free_tanner": (None, [P]),
            "bpq_sample": (i, [P, d, d, d, u64, u64, i, P, P, P]),
            "bpq_decode_workspace_bytes": (sz, []),
            "bpq_decode": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, P]),
            "bpq_decode_status": (i, [P, P, pi]),
            "bpq_decode_host_bytes": (sz, [P, i]),
            "bpq_decode_host": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, sz, P]),
            "bpq_decode_trace": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, P, P]),
            "bpq_decode_serial": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, P]),
            "bpq_decode_serial_trace": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, P, P]),
            "bpq_decode_host_noalloc": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P]),
            "bpq_decode_host_noalloc_max_shots": (i, [P]),
            "bpq_set_launch": (i, [P, i, i]),
            "bpq_autotune": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, P, pi, pi,
                                 ctypes.POINTER(ctypes.c_float)]),
            "bpq_get_launch": (i, [P, pi, pi, pi]),
            "bpq_set_batch_launch": (i, [P, i]),
            "bpq_get_batch_launch": (i, [P, i, pi, pi, pi]),
            "bpq_autotune_batch": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P, sz, P, pi,
                                       ctypes.POINTER(ctypes.c_float)]),
            "bpq_set_shots_per_thread": (i, [P, i]),
            "bpq_set_debug_checks": (i, [P, i]),
            "bpq_set_serial_shots_per_warp": (i, [P, i]),
            "bpq_get_shots_per_thread": (i, [P, i, pi]),
            "bpq_check_logical": (i, [P, P, P, i, P, P]),
            "bpq_probe_peak": (i, [i, i, i, i, P, P]),
            "bpq_batch_workspace_bytes": (sz, [i]),
            "bpq_batch_plan": (i, [P, i, i, ctypes.POINTER(Params), i, P, sz, P, PP]),
            "bpq_batch_launch": (i, [P, P]),
            "bpq_batch_info": (i, [P, pi, pi, pi, ctypes.POINTER(ctypes.c_long)]),
            "bpq_batch_free": (None, [P]),
            "bpq_server_device_bytes": (sz, [P, i, i, i]),
            "bpq_server_create": (i, [P, P, i, i, ctypes.POINTER(Params), i, i, i, P, sz, PP]),
            "bpq_server_replay": (i, [P, i, P, P, P, P, P, P, sz, P, P, P, pi]),
            "bpq_server_host_stats": (i, [P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
            "bpq_server_stats": (i, [P, ctypes.POINTER(ctypes.c_long)]),
            "bpq_server_slot_device_bytes": (sz, [i]),
            "bpq_server_slot_stats": (i, [P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                          ctypes.POINTER(ctypes.c_long)]),
            "bpq_server_create_slots": (i, [P, P, i, i, ctypes.POINTER(Params), i, i, i, P, sz, PP]),
            "bpq_server_free": (None, [P]),
            "bpq_train_workspace_bytes": (sz, [P, i, i, i, i]),
            "bpq_train_forward": (i, [P, i, P, P, P, i, i, i, P, P, P, P, ctypes.c_float, P, P, P, P, sz, P]),
            "bpq_train_backward": (i, [P, i, P, P, P, i, i, i, P, P, P, P, ctypes.c_float, P, P, P, P, P, P, sz,
                                       P]),
            "bpq_last_error": (ctypes.c_char_p, []),
            "bpq_version": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().bpq_last_error().decode(errors="replace")
        raise BPQError(f"{what} failed ({rc}): {msg}")


def default_params(variant) -> Params:
    p = Params()
    lib().bpq_default_params(VARIANTS.get(variant, variant), ctypes.byref(p))
    return p


def make_params(variant, alpha=None, gamma=None, eps=None, msg_clip=None, adagrad_g_from_iter1=None) -> Params:
    p = default_params(variant)
    if alpha is not None:
        p.alpha = alpha
    if gamma is not None:
        p.gamma = gamma
    if eps is not None:
        p.eps = eps
    if msg_clip is not None:
        p.msg_clip = msg_clip
    if adagrad_g_from_iter1 is not None:
        p.adagrad_g_from_iter1 = int(adagrad_g_from_iter1)
    return p


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


class Tanner:
    """A code's Tanner graph, built on the host by the library and uploaded
    to a CUDA device on first GPU use (or explicitly with upload())."""

    def __init__(self, code="planar", d=5, H=None, logicals=None):
        self._h = ctypes.c_void_p()
        if H is not None:
            H = np.ascontiguousarray(H, dtype=np.uint8)
            _check(lib().bpq_tanner_from_paulis(H.shape[0], H.shape[1], _ptr(H), ctypes.byref(self._h)),
                   "bpq_tanner_from_paulis")
            if logicals is not None:
                Lg = np.ascontiguousarray(logicals, dtype=np.uint8)
                _check(lib().bpq_tanner_set_logicals(self._h, Lg.shape[0], _ptr(Lg)), "bpq_tanner_set_logicals")
        else:
            _check(lib().bpq_build_tanner(CODES.get(code, code), d, ctypes.byref(self._h)), "bpq_build_tanner")
        n, m, e, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bpq_tanner_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e), ctypes.byref(k)),
               "bpq_tanner_info")
        self.N, self.M, self.E, self.K = n.value, m.value, e.value, k.value
        self.W = (self.M + 31) // 32
        self.device = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.bpq_free_tanner(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def upload(self, device=None):
        if self.device is None:
            dev = torch.cuda.current_device() if device is None else int(device)
            _check(lib().bpq_tanner_upload(self._h, dev), "bpq_tanner_upload")
            self.device = dev
        return self

    def export(self):
        ptr = np.zeros(self.M + 1, dtype=np.int32)
        var = np.zeros(self.E, dtype=np.int32)
        pauli = np.zeros(self.E, dtype=np.uint8)
        _check(lib().bpq_tanner_export(self._h, _ptr(ptr), _ptr(var), _ptr(pauli)), "bpq_tanner_export")
        return ptr, var, pauli

    def dense(self) -> np.ndarray:
        ptr, var, pauli = self.export()
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        rows = np.repeat(np.arange(self.M), np.diff(ptr))
        H[rows, var] = pauli
        return H

    def logicals(self) -> np.ndarray:
        L = np.zeros((2 * max(self.K, 0), self.N), dtype=np.uint8)
        _check(lib().bpq_tanner_logicals(self._h, _ptr(L)), "bpq_tanner_logicals")
        return L

    def layout(self) -> int:
        """The decode kernels' message layout: 0 generic, 1 split, 2 split
        without padding (bpq_tanner_layout)."""
        v = ctypes.c_int()
        _check(lib().bpq_tanner_layout(self._h, ctypes.byref(v)), "bpq_tanner_layout")
        return v.value

    def set_launch(self, threads_per_shot=0, shots_per_cta=0):
        _check(lib().bpq_set_launch(self._h, threads_per_shot, shots_per_cta), "bpq_set_launch")

    def launch(self):
        t, s, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bpq_get_launch(self._h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(c)), "bpq_get_launch")
        return t.value, s.value

    def set_batch_launch(self, nodes_per_thread=0):
        """Nodes per thread (1 or 2; 0 = automatic) of this code inside the
        batched kernel and the servers (bpq_set_batch_launch)."""
        _check(lib().bpq_set_batch_launch(self._h, nodes_per_thread), "bpq_set_batch_launch")

    def batch_launch(self, variant="ewainit"):
        """(threads per shot group, groups per CTA, nodes per thread) inside
        the batched kernel (bpq_get_batch_launch)."""
        t, s, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bpq_get_batch_launch(self._h, VARIANTS.get(variant, variant), ctypes.byref(t), ctypes.byref(s),
                                          ctypes.byref(n)), "bpq_get_batch_launch")
        return t.value, s.value, n.value

    def set_shots_per_thread(self, k=0):
        """1: one shot per thread; 2: two shots per thread (split tables);
        0: automatic (bpq_set_shots_per_thread)."""
        _check(lib().bpq_set_shots_per_thread(self._h, k), "bpq_set_shots_per_thread")

    def set_serial_shots_per_warp(self, k=0):
        """Shots per warp of the serial-schedule kernel: 1, 2, or 0 =
        automatic (bpq_set_serial_shots_per_warp)."""
        _check(lib().bpq_set_serial_shots_per_warp(self._h, k), "bpq_set_serial_shots_per_warp")

    def set_debug_checks(self, on=True):
        """Run the bounds-checked decode kernels (bpq_set_debug_checks)."""
        _check(lib().bpq_set_debug_checks(self._h, 1 if on else 0), "bpq_set_debug_checks")

    def shots_per_thread(self, variant="ewainit") -> int:
        k = ctypes.c_int()
        _check(lib().bpq_get_shots_per_thread(self._h, VARIANTS.get(variant, variant), ctypes.byref(k)),
               "bpq_get_shots_per_thread")
        return k.value


def autotune(tanner: Tanner, syn, prior, variant="ewainit", params=None, max_iter=100, stream=None, **param_kw):
    """Time every candidate launch shape on this sample batch and keep the
    fastest in the handle; returns (threads_per_shot, shots_per_cta, ms)."""
    tanner.upload()
    v = VARIANTS.get(variant, variant)
    p = params if params is not None else make_params(v, **param_kw)
    B = syn.shape[0]
    dev = syn.device
    est = torch.empty((B, tanner.N), dtype=torch.uint8, device=dev)
    conv = torch.empty(B, dtype=torch.uint8, device=dev)
    iters = torch.empty(B, dtype=torch.uint8, device=dev)
    work = workspace(dev)
    t_, s_, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().bpq_autotune(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), max_iter, B, _ptr(est),
                              _ptr(conv), _ptr(iters), _ptr(work), _stream(stream), ctypes.byref(t_),
                              ctypes.byref(s_), ctypes.byref(ms)), "bpq_autotune")
    return t_.value, s_.value, ms.value


def autotune_batch(tanner: Tanner, syn, prior, variant="ewainit", params=None, max_iter=100, stream=None,
                   **param_kw):
    """Time a one-item batched plan of this sample with one and with two
    nodes per thread and keep the faster in the handle
    (bpq_autotune_batch); returns (nodes_per_thread, ms)."""
    tanner.upload()
    v = VARIANTS.get(variant, variant)
    p = params if params is not None else make_params(v, **param_kw)
    B = syn.shape[0]
    dev = syn.device
    est = torch.empty((B, tanner.N), dtype=torch.uint8, device=dev)
    conv = torch.empty(B, dtype=torch.uint8, device=dev)
    iters = torch.empty(B, dtype=torch.uint8, device=dev)
    nbytes = lib().bpq_batch_workspace_bytes(1)
    work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    n_, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().bpq_autotune_batch(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), max_iter, B,
                                    _ptr(est), _ptr(conv), _ptr(iters), _ptr(work), nbytes, _stream(stream),
                                    ctypes.byref(n_), ctypes.byref(ms)), "bpq_autotune_batch")
    return n_.value, ms.value


def workspace(device=None) -> torch.Tensor:
    n = lib().bpq_decode_workspace_bytes()
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def sample(tanner: Tanner, px, py, pz, seed, shot0, B, err=None, syn=None, stream=None):
    """Errors (B, N) uint8 and packed syndromes (B, W) int32 on the device."""
    tanner.upload()
    dev = f"cuda:{tanner.device}"
    if err is None:
        err = torch.empty((B, tanner.N), dtype=torch.uint8, device=dev)
    if syn is None:
        syn = torch.empty((B, tanner.W), dtype=torch.int32, device=dev)
    _check(lib().bpq_sample(tanner.handle, px, py, pz, seed, shot0, B, _ptr(err), _ptr(syn), _stream(stream)),
           "bpq_sample")
    return err, syn


def prior_rows(n_qubits: int, px, py, pz, jitter: float = 0.0) -> np.ndarray:
    """(N, 3) float32 rows (p^X, p^Y, p^Z) of an i.i.d. channel.  With
    jitter > 0, row j is scaled by 1 + jitter * u_j, where
    u_j = 2 * ((j * 2654435761) mod 2^32) / 2^32 - 1 lies in [-1, 1).  The
    result is computed in float64 and rounded once to float32.

    Uniform priors on the toric and planar codes put many trapping sets
    (Sec. II-B2) into a nearly symmetric oscillation.  Under the parallel
    schedule EWAInit-BP cannot break an exact symmetry by itself (Sec.
    IV-A); a near one breaks only through asymmetries far below binary32
    resolution, so whether a run escapes is decided by the working
    precision.  A jitter of 2^-16 puts the asymmetry into the input, where
    every precision resolves it, and it is far below any channel-estimation
    precision."""
    j = np.arange(n_qubits, dtype=np.uint64)
    u = ((j * np.uint64(2654435761)) % np.uint64(1 << 32)).astype(np.float64) / 2.0 ** 32 * 2.0 - 1.0
    ch = np.array([px, py, pz], dtype=np.float64)
    return (ch[None, :] * (1.0 + float(jitter) * u)[:, None]).astype(np.float32)


def prior_tensor(tanner: Tanner, px, py, pz, device=None, jitter: float = 0.0) -> torch.Tensor:
    """(N, 3) float32 probabilities of an i.i.d. channel, on the device;
    jitter is the relative per-qubit perturbation of prior_rows."""
    tanner.upload()
    p = torch.from_numpy(prior_rows(tanner.N, px, py, pz, jitter))
    return p.to(device or f"cuda:{tanner.device}")


def decode(tanner: Tanner, syn, prior, variant="ewainit", params=None, max_iter=50, out=None, work=None,
           stream=None, schedule="parallel", **param_kw):
    """Decode packed syndromes (B, W) int32 on the device.  schedule:
    "parallel" (flooding, bpq_decode) or "serial" (Algorithm 1's sweep,
    bpq_decode_serial).  Returns (est (B, N) uint8, conv (B,) uint8,
    iters (B,) uint8) device tensors."""
    tanner.upload()
    v = VARIANTS.get(variant, variant)
    p = params if params is not None else make_params(v, **param_kw)
    B = syn.shape[0]
    dev = syn.device
    if out is None:
        out = (torch.empty((B, tanner.N), dtype=torch.uint8, device=dev),
               torch.empty(B, dtype=torch.uint8, device=dev),
               torch.empty(B, dtype=torch.uint8, device=dev))
    est, conv, iters = out
    if work is None:
        work = workspace(dev)
    assert syn.is_contiguous() and prior.is_contiguous() and prior.dtype == torch.float32
    fn = {"parallel": "bpq_decode", "serial": "bpq_decode_serial"}[schedule]
    _check(getattr(lib(), fn)(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), max_iter, B, _ptr(est),
                              _ptr(conv), _ptr(iters), _ptr(work), _stream(stream)), fn)
    return est, conv, iters


def decode_status(work, stream=None) -> int:
    e = ctypes.c_int()
    _check(lib().bpq_decode_status(_ptr(work), _stream(stream), ctypes.byref(e)), "bpq_decode_status")
    return e.value


def decode_host_bytes(tanner: Tanner, B: int) -> int:
    return lib().bpq_decode_host_bytes(tanner.handle, B)


def decode_host(tanner: Tanner, syn_host, prior_host, variant="ewainit", params=None, max_iter=50, out=None,
                dev_buf=None, stream=None, **param_kw):
    """Decode host syndromes (B, W) int32 (pinned torch CPU tensors or numpy)
    through bpq_decode_host; returns host (est, conv, iters)."""
    tanner.upload()
    v = VARIANTS.get(variant, variant)
    p = params if params is not None else make_params(v, **param_kw)
    B = syn_host.shape[0]
    if out is None:
        out = (torch.empty((B, tanner.N), dtype=torch.uint8, pin_memory=True),
               torch.empty(B, dtype=torch.uint8, pin_memory=True),
               torch.empty(B, dtype=torch.uint8, pin_memory=True))
    est, conv, iters = out
    need = decode_host_bytes(tanner, B)
    if dev_buf is None:
        dev_buf = torch.empty(need, dtype=torch.uint8, device=f"cuda:{tanner.device}")
    _check(lib().bpq_decode_host(tanner.handle, _ptr(syn_host), _ptr(prior_host), v, ctypes.byref(p), max_iter, B,
                                 _ptr(est), _ptr(conv), _ptr(iters), _ptr(dev_buf), dev_buf.numel(),
                                 _stream(stream)), "bpq_decode_host")
    return est, conv, iters


def decode_trace(tanner: Tanner, syn, prior, variant="plain", T=5, params=None, stream=None, schedule="parallel",
                 **param_kw):
    """Run exactly T iterations and return the per-iteration record:
    m_v2c (B, T+1, E), m_c2v (B, T, E), Q (B, T, N, 3), dec (B, T, N)."""
    tanner.upload()
    v = VARIANTS.get(variant, variant)
    p = params if params is not None else make_params(v, **param_kw)
    B = syn.shape[0]
    dev = syn.device
    rec = dict(m_v2c=torch.zeros((B, T + 1, tanner.E), dtype=torch.float32, device=dev),
               m_c2v=torch.zeros((B, T, tanner.E), dtype=torch.float32, device=dev),
               Q=torch.zeros((B, T, tanner.N, 3), dtype=torch.float32, device=dev),
               dec=torch.zeros((B, T, tanner.N), dtype=torch.uint8, device=dev))
    work = workspace(dev)
    fn = {"parallel": "bpq_decode_trace", "serial": "bpq_decode_serial_trace"}[schedule]
    _check(getattr(lib(), fn)(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), T, B,
                              _ptr(rec["m_v2c"]), _ptr(rec["m_c2v"]), _ptr(rec["Q"]), _ptr(rec["dec"]),
                              _ptr(work), _stream(stream)), fn)
    return rec


def check_logical(tanner: Tanner, err, est, out=None, stream=None):
    """(B,) uint8: 0 success, 1 detected error, 2 undetected (logical) error."""
    tanner.upload()
    B = err.shape[0]
    if out is None:
        out = torch.empty(B, dtype=torch.uint8, device=err.device)
    _check(lib().bpq_check_logical(tanner.handle, _ptr(err), _ptr(est), B, _ptr(out), _stream(stream)),
           "bpq_check_logical")
    return out


def probe_peak(which: str, blocks: int, threads: int = 256, iters: int = 4096, stream=None) -> float:
    """Measured throughput of the probe kernel: SFU ex2 ops/s ("sfu") or
    FMA instructions/s ("fma"), timed with CUDA events on the stream."""
    w = {"sfu": 0, "fma": 1}[which]
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    for _ in range(2):
        _check(lib().bpq_probe_peak(w, blocks, threads, iters, _ptr(sink), _stream(st)), "bpq_probe_peak")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    _check(lib().bpq_probe_peak(w, blocks, threads, iters, _ptr(sink), _stream(st)), "bpq_probe_peak")
    e1.record(st)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    return blocks * threads * iters * 8 / sec


class BatchItem(ctypes.Structure):
    _fields_ = [("tanner", ctypes.c_void_p), ("syn_dev", ctypes.c_void_p), ("prior_dev", ctypes.c_void_p),
                ("B", ctypes.c_int), ("est_dev", ctypes.c_void_p), ("conv_dev", ctypes.c_void_p),
                ("iters_dev", ctypes.c_void_p)]


class BatchPlan:
    """Many codes decoded by one persistent launch (bpq_batch_*).

    items: list of (Tanner, syndromes (B, W) int32, prior (N, 3) float32).
    The plan owns its outputs (est, conv, iters per item) and its device
    workspace; run() enqueues one launch (capturable in a CUDA graph)."""

    def __init__(self, items, variant="ewainit", params=None, max_iter=100, stream=None,
                 **param_kw):
        v = VARIANTS.get(variant, variant)
        self.params = params if params is not None else make_params(v, **param_kw)
        self.tanners = [t.upload() for t, _, _ in items]
        self.inputs = [(syn, prior) for _, syn, prior in items]
        dev = items[0][1].device
        self.outputs = []
        arr = (BatchItem * len(items))()
        total = 0
        for k, (t, syn, prior) in enumerate(items):
            B = syn.shape[0]
            assert syn.is_contiguous() and prior.is_contiguous() and prior.dtype == torch.float32
            out = (torch.empty((B, t.N), dtype=torch.uint8, device=dev), torch.empty(B, dtype=torch.uint8, device=dev),
                   torch.empty(B, dtype=torch.uint8, device=dev))
            self.outputs.append(out)
            arr[k] = BatchItem(t.handle.value, syn.data_ptr(), prior.data_ptr(), B, out[0].data_ptr(),
                               out[1].data_ptr(), out[2].data_ptr())
            total += B
        nbytes = lib().bpq_batch_workspace_bytes(len(items))
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self._h = ctypes.c_void_p()
        _check(lib().bpq_batch_plan(arr, len(items), v, ctypes.byref(self.params), max_iter, _ptr(self.work), nbytes,
                                    _stream(stream), ctypes.byref(self._h)), "bpq_batch_plan")
        self.total_shots = total

    def run(self, stream=None):
        _check(lib().bpq_batch_launch(self._h, _stream(stream)), "bpq_batch_launch")
        return self.outputs

    def info(self):
        c, t, n, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
        _check(lib().bpq_batch_info(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(n), ctypes.byref(s)),
               "bpq_batch_info")
        return dict(ctas=c.value, items=t.value, npt_max=n.value, shots=s.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.bpq_batch_free(h)
            self._h = None


class Server:
    """Decoding server (bpq_server_*); replay() serves a request trace in real
    time and returns per-request outputs and completion times.

    mode="lanes": n_lanes streams with room for max_batch shots each, each
    dispatch a batched launch (bpq_server_create).  mode="slots": one
    persistent kernel whose shot groups take the next request as soon as they
    finish a shot, with slots_per_code request slots per code
    (bpq_server_create_slots)."""

    def __init__(self, codes, priors, variant="ewainit", params=None, max_iter=100, n_lanes=4, max_batch=4096,
                 mode="lanes", slots_per_code=1024, idle_timeout_us=200000, **param_kw):
        v = VARIANTS.get(variant, variant)
        self.params = params if params is not None else make_params(v, **param_kw)
        self.codes = [t.upload() for t in codes]
        self.priors = [p.contiguous() for p in priors]
        self.mode = mode
        n = len(codes)
        harr = (ctypes.c_void_p * n)(*[t.handle.value for t in self.codes])
        parr = (ctypes.c_void_p * n)(*[p.data_ptr() for p in self.priors])
        self._h = ctypes.c_void_p()
        if mode == "slots":
            nbytes = lib().bpq_server_slot_device_bytes(n)
            self.mem = torch.empty(nbytes, dtype=torch.uint8, device=self.priors[0].device)
            _check(lib().bpq_server_create_slots(harr, parr, n, v, ctypes.byref(self.params), max_iter,
                                                 slots_per_code, idle_timeout_us, _ptr(self.mem), nbytes,
                                                 ctypes.byref(self._h)), "bpq_server_create_slots")
            return
        nbytes = lib().bpq_server_device_bytes(harr, n, n_lanes, max_batch)
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=self.priors[0].device)
        _check(lib().bpq_server_create(harr, parr, n, v, ctypes.byref(self.params), max_iter, n_lanes, max_batch,
                                       _ptr(self.mem), nbytes, ctypes.byref(self._h)), "bpq_server_create")

    def replay(self, code, arrival_s, syn_list, pinned=None):
        """code: (R,) int; arrival_s: (R,) float, non-decreasing; syn_list:
        packed syndrome words (uint32 numpy) of each request.  pinned: the
        outputs live in page-locked memory at 16-byte aligned offsets, so the
        slot server writes them directly (else through its rings); default:
        for the slot server only (the lane server's host copies run faster
        into pageable memory).  Returns (est list, conv (R,), iters (R,),
        done_s (R,), lanes_used)."""
        if pinned is None:
            pinned = self.mode == "slots"
        code = np.ascontiguousarray(code, dtype=np.int32)
        arrival = np.ascontiguousarray(arrival_s, dtype=np.float64)
        R = code.size
        syn_off = np.zeros(R, dtype=np.int64)
        est_off = np.zeros(R, dtype=np.int64)
        Ns = [self.codes[c].N for c in code]
        lens = [len(x) for x in syn_list]
        syn_off[1:] = np.cumsum(lens)[:-1]
        stride = [(n + 15) & ~15 for n in Ns] if pinned else Ns
        est_off[1:] = np.cumsum(stride)[:-1]
        syn = np.ascontiguousarray(np.concatenate(syn_list).astype(np.uint32)) if R else np.zeros(1, np.uint32)
        n_est = max(16, int(sum(stride)))

        def buf(n):
            if pinned:
                return torch.zeros(n, dtype=torch.uint8, pin_memory=True).numpy()
            return np.zeros(n, dtype=np.uint8)

        est, conv, iters = buf(n_est), buf(max(1, R)), buf(max(1, R))
        done = np.zeros(max(1, R), dtype=np.float64)
        used = ctypes.c_int()
        _check(lib().bpq_server_replay(self._h, R, _ptr(code), _ptr(arrival), _ptr(syn), _ptr(syn_off), _ptr(est),
                                       _ptr(est_off), n_est, _ptr(conv), _ptr(iters), _ptr(done),
                                       ctypes.byref(used)),
               "bpq_server_replay")
        ests = [est[o:o + n] for o, n in zip(est_off, Ns)]
        return ests, conv[:R], iters[:R], done[:R], used.value

    def slot_stats(self):
        """Slot server counters of the last replay: (code switches, empty
        scans, empty claims)."""
        a, b, c = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        _check(lib().bpq_server_slot_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "bpq_server_slot_stats")
        return a.value, b.value, c.value

    def host_stats(self):
        """Slot server host loop of the last replay: (turns with work, seconds
        admitting, seconds reading completions)."""
        n, a, c = ctypes.c_long(), ctypes.c_double(), ctypes.c_double()
        _check(lib().bpq_server_host_stats(self._h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(c)),
               "bpq_server_host_stats")
        return n.value, a.value, c.value

    def launches(self):
        """Decode kernels launched since creation."""
        n = ctypes.c_long()
        _check(lib().bpq_server_stats(self._h, ctypes.byref(n)), "bpq_server_stats")
        return n.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.bpq_server_free(h)
            self._h = None


TRAIN_MODELS = {"ewainit": 0, "momentum": 1}


class TrainLoss(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("logicals_dev", ctypes.c_void_p), ("n_logicals", ctypes.c_int)]


TRAIN_LOSSES = {"posterior": 0, "coset": 1}


def _train_loss(tanner, kind, logicals, device):
    """bpq_train_loss for `kind`; the coset loss takes logical operators
    (n, N) Pauli codes, by default the tanner's own (bpq_tanner_logicals).
    Returns (struct, tensor keeping the device copy alive)."""
    k = TRAIN_LOSSES[kind]
    if k == 0:
        return TrainLoss(0, None, 0), None
    L = tanner.logicals() if logicals is None else np.asarray(logicals, dtype=np.uint8)
    Ld = torch.as_tensor(np.ascontiguousarray(L, dtype=np.uint8), device=device)
    return TrainLoss(k, Ld.data_ptr(), int(L.shape[0])), Ld


class _Unrolled(torch.autograd.Function):
    """Loss of an unrolled decoder (model EWAInit or Momentum) as a function
    of its parameters (alpha, beta, w, gamma); forward and backward run in
    libbpq's CUDA kernels (bpq_train_forward / bpq_train_backward)."""

    @staticmethod
    def forward(ctx, alpha, beta, w, gamma, model, tanner, syn, err, prior, T, ckpt_every, msg_clip, lossdef):
        alpha, beta, w = alpha.contiguous().float(), beta.contiguous().float(), w.contiguous().float()
        gamma = gamma.contiguous().float() if gamma is not None else None
        B = syn.shape[0]
        nbytes = lib().bpq_train_workspace_bytes(tanner.handle, model, B, T, ckpt_every)
        work = torch.empty(nbytes, dtype=torch.uint8, device=syn.device)
        loss = torch.empty(1, dtype=torch.float32, device=syn.device)
        _check(lib().bpq_train_forward(tanner.handle, model, _ptr(syn), _ptr(err), _ptr(prior), B, T, ckpt_every,
                                       _ptr(alpha), _ptr(beta), _ptr(gamma) if gamma is not None else None, _ptr(w),
                                       msg_clip, ctypes.byref(lossdef[0]), _ptr(loss), None, _ptr(work), nbytes,
                                       _stream(None)),
               "bpq_train_forward")
        ctx.save_for_backward(alpha, beta, w, *( [gamma] if gamma is not None else []))
        ctx.rest = (model, tanner, syn, err, prior, T, ckpt_every, msg_clip, work, nbytes, lossdef)
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        saved = ctx.saved_tensors
        alpha, beta, w = saved[:3]
        gamma = saved[3] if len(saved) > 3 else None
        model, tanner, syn, err, prior, T, ckpt_every, msg_clip, work, nbytes, lossdef = ctx.rest
        ga, gb, gw = torch.empty_like(alpha), torch.empty_like(beta), torch.empty_like(w)
        gg = torch.empty_like(gamma) if gamma is not None else None
        _check(lib().bpq_train_backward(tanner.handle, model, _ptr(syn), _ptr(err), _ptr(prior), syn.shape[0], T,
                                        ckpt_every, _ptr(alpha), _ptr(beta),
                                        _ptr(gamma) if gamma is not None else None, _ptr(w), msg_clip,
                                        ctypes.byref(lossdef[0]), _ptr(ga), _ptr(gb),
                                        _ptr(gg) if gg is not None else None, _ptr(gw), _ptr(work), nbytes,
                                        _stream(None)), "bpq_train_backward")
        return (ga * gout, gb * gout, gw * gout, gg * gout if gg is not None else None,
                None, None, None, None, None, None, None, None, None)


def unrolled_loss(tanner: Tanner, syn, err, prior, alpha, beta, w, T=25, ckpt_every=5, msg_clip=30.0,
                  model="ewainit", gamma=None, loss="posterior", logicals=None):
    """Differentiable loss of the unrolled decoder (see bpq_train_forward):
    model "ewainit" (EWA weights alpha) or "momentum" (steps alpha, rates
    gamma); loss "posterior" (cross-entropy of the final posterior) or
    "coset" (every iteration's soft decision in the syndrome's and the true
    error's coset, with logical operators `logicals`, by default the
    tanner's); gradients flow to alpha (T,), beta (T,), w (E,) and gamma
    (T,)."""
    tanner.upload()
    m = TRAIN_MODELS[model]
    if m == 1 and gamma is None:
        raise BPQError("the Momentum model needs gamma")
    lossdef = _train_loss(tanner, loss, logicals, syn.device)
    return _Unrolled.apply(alpha, beta, w, gamma if m == 1 else None, m, tanner, syn, err, prior, T, ckpt_every,
                           msg_clip, lossdef)


def unrolled_posterior(tanner: Tanner, syn, err, prior, alpha, beta, w, T=25, ckpt_every=5, msg_clip=30.0,
                       model="ewainit", gamma=None, loss="posterior", logicals=None):
    """Final posterior Q^(T) (B, N, 3) and the loss of the unrolled decoder."""
    tanner.upload()
    m = TRAIN_MODELS[model]
    B = syn.shape[0]
    nbytes = lib().bpq_train_workspace_bytes(tanner.handle, m, B, T, ckpt_every)
    work = torch.empty(nbytes, dtype=torch.uint8, device=syn.device)
    out = torch.empty(1, dtype=torch.float32, device=syn.device)
    Q = torch.empty((B, tanner.N, 3), dtype=torch.float32, device=syn.device)
    a, b, ww = alpha.contiguous().float(), beta.contiguous().float(), w.contiguous().float()
    g = gamma.contiguous().float() if gamma is not None else None
    lossdef = _train_loss(tanner, loss, logicals, syn.device)
    _check(lib().bpq_train_forward(tanner.handle, m, _ptr(syn), _ptr(err), _ptr(prior), B, T, ckpt_every, _ptr(a),
                                   _ptr(b), _ptr(g) if g is not None else None, _ptr(ww), msg_clip,
                                   ctypes.byref(lossdef[0]), _ptr(out), _ptr(Q), _ptr(work), nbytes, _stream(None)),
           "bpq_train_forward")
    return Q, out[0]
