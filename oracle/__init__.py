"""FP64 CPU oracle for GF(4) belief-propagation decoding (Plain, Momentum-BP,
AdaGrad-BP, EWAInit-BP; flooding schedule) and for the Philox noise sampler.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2407_11523_gb300``) and never imports it.

The arithmetic lives in ``bp_oracle.c`` (decoder) and ``noise_oracle.c``
(sampler), compiled with gcc into ``_oracle.so`` beside them; this module only
marshals numpy arrays.  Code construction and GF(2) tools are in
``codes.py``.

``decode`` and ``trace`` take ``precision``: "f64" (the oracle proper,
double precision), "ext" (the same source computing in long double) or
"f32" (double arithmetic with every stored message, posterior, prior and
state value rounded to binary32).  The two other builds exist to show which
results the working precision decides; parity is measured against "f64".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import codes  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = [os.path.join(_HERE, f) for f in ("bp_oracle.c", "noise_oracle.c")]
# precision -> (shared object, extra gcc flags); only the f64 build carries the sampler
_BUILDS = {
    "f64": (os.path.join(_HERE, "_oracle.so"), [], _SOURCES),
    "ext": (os.path.join(_HERE, "_oracle_ext.so"), ["-DORACLE_REAL=long double"], _SOURCES[:1]),
    "f32": (os.path.join(_HERE, "_oracle_f32.so"), ["-DORACLE_STORE_F32"], _SOURCES[:1]),
}
_SO = _BUILDS["f64"][0]

PLAIN, MOMENTUM, ADAGRAD, EWAINIT, AEWA = 0, 1, 2, 3, 4
VARIANTS = {"plain": PLAIN, "momentum": MOMENTUM, "adagrad": ADAGRAD, "ewainit": EWAINIT, "aewa": AEWA}

# Parameters taken from the paper (Sec. III-A2, Sec. IV-A, Table I):
# AdaGrad alpha = 5; Momentum gamma = 0 with alpha = 0.5; EWAInit alpha = 0.5.
DEFAULT_PARAMS = {
    PLAIN: dict(alpha=1.0, gamma=0.0),
    MOMENTUM: dict(alpha=0.5, gamma=0.0),
    ADAGRAD: dict(alpha=5.0, gamma=0.0),
    EWAINIT: dict(alpha=0.5, gamma=0.0),
    AEWA: dict(alpha=1.0, gamma=0.0),  # alpha is swept 1.0 .. 0.0 (Appendix C)
}


def build(force: bool = False, precision: str | None = None) -> str:
    """Compile the oracle's C sources (plain gcc -O2): _oracle.so, and the
    extended-precision and binary32-storage builds of the decoder.  With
    `precision`, only that build."""
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    for prec, (so, flags, srcs) in _BUILDS.items():
        if precision is not None and prec != precision:
            continue
        if force or not os.path.exists(so) or os.path.getmtime(so) < newest:
            tmp = so + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, *srcs, "-lm", "-lpthread"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, so)
    return _SO


_libs = {}


def lib(precision: str = "f64"):
    if precision not in _BUILDS:
        raise ValueError(f"precision must be one of {sorted(_BUILDS)}")
    if precision not in _libs:
        build(precision=precision)
        L = ctypes.CDLL(_BUILDS[precision][0])
        P = ctypes.c_void_p
        i, d, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        L.oracle_decode.argtypes = [i, i, P, i, P, P, i, d, d, d, d, i, i, i, P, P, P, i]
        L.oracle_decode.restype = i
        L.oracle_trace.argtypes = [i, i, P, P, P, i, d, d, d, d, i, i, i, P, P, P, P, P, P]
        L.oracle_trace.restype = i
        if precision == "f64":
            L.oracle_sample.argtypes = [i, i, P, d, d, d, u64, u64, i, P, P]
            L.oracle_sample.restype = i
            L.oracle_philox4x64_10.argtypes = [P, P, P]
            L.oracle_philox4x64_10.restype = None
        L.oracle_num_edges.argtypes = [i, i, P]
        L.oracle_num_edges.restype = i
        L.oracle_hard_decision.argtypes = [P]
        L.oracle_hard_decision.restype = i
        _libs[precision] = L
    return _libs[precision]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x64_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample(H: np.ndarray, px: float, py: float, pz: float, seed: int, shot0: int, B: int):
    """Errors (B x N Pauli codes) and syndromes (B x M bytes) of shots
    shot0 .. shot0+B-1 of the i.i.d. Pauli channel."""
    H = np.ascontiguousarray(H, dtype=np.uint8)
    M, N = H.shape
    err = np.zeros((B, N), dtype=np.uint8)
    syn = np.zeros((B, M), dtype=np.uint8)
    rc = lib().oracle_sample(N, M, _ptr(H), px, py, pz, seed, shot0, B, _ptr(err), _ptr(syn))
    if rc:
        raise ValueError(f"oracle_sample failed ({rc})")
    return err, syn


def _params(variant, alpha, gamma, eps, msg_clip, adagrad_g_from_iter1):
    dp = DEFAULT_PARAMS[variant]
    return (dp["alpha"] if alpha is None else alpha,
            dp["gamma"] if gamma is None else gamma,
            1e-8 if eps is None else eps,
            30.0 if msg_clip is None else msg_clip,
            1 if adagrad_g_from_iter1 is None else int(adagrad_g_from_iter1))


SCHEDULES = {"parallel": 0, "serial": 1}


def decode(H, syn, prior, variant=PLAIN, max_iter=50, alpha=None, gamma=None, eps=None,
           msg_clip=None, adagrad_g_from_iter1=None, nthreads=1, schedule="parallel", precision="f64"):
    """Decode B syndromes. syn: (B, M) 0/1; prior: (N, 3) probabilities
    (p^X, p^Y, p^Z).  schedule: "parallel" (flooding) or "serial"
    (Algorithm 1's qubit-by-qubit sweep).  precision: "f64", "ext" or
    "f32" (see the module docstring).  Returns (est (B,N) codes,
    conv (B,) bool, iters (B,))."""
    H = np.ascontiguousarray(H, dtype=np.uint8)
    M, N = H.shape
    syn = np.ascontiguousarray(np.atleast_2d(syn), dtype=np.uint8).reshape(-1, M)
    prior = np.ascontiguousarray(np.broadcast_to(np.asarray(prior, dtype=np.float64), (N, 3)))
    variant = VARIANTS.get(variant, variant)
    B = syn.shape[0]
    est = np.zeros((B, N), dtype=np.uint8)
    conv = np.zeros(B, dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    a, g, e, c, f = _params(variant, alpha, gamma, eps, msg_clip, adagrad_g_from_iter1)
    rc = lib(precision).oracle_decode(N, M, _ptr(H), B, _ptr(syn), _ptr(prior), variant, a, g, e, c, f,
                             SCHEDULES[schedule], max_iter, _ptr(est), _ptr(conv), _ptr(iters), nthreads)
    if rc:
        raise ValueError(f"oracle_decode failed ({rc})")
    return est, conv.astype(bool), iters


def trace(H, syn, prior, variant=PLAIN, T=5, alpha=None, gamma=None, eps=None, msg_clip=None,
          adagrad_g_from_iter1=None, schedule="parallel", precision="f64"):
    """Run exactly T iterations on one syndrome and return every intermediate
    quantity: dict with m_v2c (T+1, E), m_c2v (T, E), S, Q, aux (T, N, 3) and
    dec (T, N).  Edges are in check-major order (row i of H, columns j
    increasing)."""
    H = np.ascontiguousarray(H, dtype=np.uint8)
    M, N = H.shape
    syn = np.ascontiguousarray(syn, dtype=np.uint8).reshape(M)
    prior = np.ascontiguousarray(np.broadcast_to(np.asarray(prior, dtype=np.float64), (N, 3)))
    variant = VARIANTS.get(variant, variant)
    E = lib().oracle_num_edges(N, M, _ptr(H))
    out = dict(m_v2c=np.zeros((T + 1, E)), m_c2v=np.zeros((T, E)), S=np.zeros((T, N, 3)),
               Q=np.zeros((T, N, 3)), aux=np.zeros((T, N, 3)), dec=np.zeros((T, N), dtype=np.uint8))
    a, g, e, c, f = _params(variant, alpha, gamma, eps, msg_clip, adagrad_g_from_iter1)
    rc = lib(precision).oracle_trace(N, M, _ptr(H), _ptr(syn), _ptr(prior), variant, a, g, e, c, f,
                            SCHEDULES[schedule], T,
                            _ptr(out["m_v2c"]), _ptr(out["m_c2v"]), _ptr(out["S"]), _ptr(out["Q"]),
                            _ptr(out["aux"]), _ptr(out["dec"]))
    if rc:
        raise ValueError(f"oracle_trace failed ({rc})")
    return out


def hard_decision(q) -> int:
    """Pauli code chosen by the hard decision for one (Q_X, Q_Y, Q_Z) triple."""
    a = np.ascontiguousarray(q, dtype=np.float64).reshape(3)
    return int(lib().oracle_hard_decision(_ptr(a)))


def edges(H):
    """Check-major edge list (check, qubit, Pauli) of H, the order used by trace()."""
    H = np.asarray(H)
    ii, jj = np.nonzero(H)
    return ii.astype(np.int64), jj.astype(np.int64), H[ii, jj].astype(np.uint8)


def depolarizing(p: float):
    """(p^X, p^Y, p^Z) of the depolarising channel: p/3 each (Sec. IV)."""
    return (p / 3.0, p / 3.0, p / 3.0)


def biased(p: float, eta: float):
    """Z-biased channel with bias eta = p^Z / (p^X + p^Y) and total p."""
    pz = p * eta / (1.0 + eta)
    px = p / (2.0 * (1.0 + eta))
    return (px, px, pz)
