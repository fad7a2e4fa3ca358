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
PLAIN, MOMENTUM, ADAGRAD, EWAINIT = 0, 1, 2, 3
CODES = {"planar": PLANAR, "toric": TORIC, "xzzx": XZZX}
VARIANTS = {"plain": PLAIN, "momentum": MOMENTUM, "adagrad": ADAGRAD, "ewainit": EWAINIT}


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
            "bpq_decode_host_noalloc": (i, [P, P, P, i, ctypes.POINTER(Params), i, i, P, P, P, P]),
            "bpq_decode_host_noalloc_max_shots": (i, [P]),
            "bpq_set_launch": (i, [P, i, i]),
            "bpq_get_launch": (i, [P, pi, pi, pi]),
            "bpq_check_logical": (i, [P, P, P, i, P, P]),
            "bpq_probe_peak": (i, [i, i, i, i, P, P]),
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

    def set_launch(self, threads_per_shot=0, shots_per_cta=0):
        _check(lib().bpq_set_launch(self._h, threads_per_shot, shots_per_cta), "bpq_set_launch")

    def launch(self):
        t, s, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bpq_get_launch(self._h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(c)), "bpq_get_launch")
        return t.value, s.value


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


def prior_tensor(tanner: Tanner, px, py, pz, device=None) -> torch.Tensor:
    """(N, 3) float32 probabilities of an i.i.d. channel, on the device."""
    tanner.upload()
    p = torch.tensor([px, py, pz], dtype=torch.float32).repeat(tanner.N, 1)
    return p.to(device or f"cuda:{tanner.device}")


def decode(tanner: Tanner, syn, prior, variant="ewainit", params=None, max_iter=50, out=None, work=None,
           stream=None, **param_kw):
    """Decode packed syndromes (B, W) int32 on the device.  Returns
    (est (B, N) uint8, conv (B,) uint8, iters (B,) uint8) device tensors."""
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
    _check(lib().bpq_decode(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), max_iter, B, _ptr(est),
                            _ptr(conv), _ptr(iters), _ptr(work), _stream(stream)), "bpq_decode")
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


def decode_trace(tanner: Tanner, syn, prior, variant="plain", T=5, params=None, stream=None, **param_kw):
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
    _check(lib().bpq_decode_trace(tanner.handle, _ptr(syn), _ptr(prior), v, ctypes.byref(p), T, B,
                                  _ptr(rec["m_v2c"]), _ptr(rec["m_c2v"]), _ptr(rec["Q"]), _ptr(rec["dec"]),
                                  _ptr(work), _stream(stream)), "bpq_decode_trace")
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
