"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds none of the decoding arithmetic: it only draws random
Tanner graphs, priors and syndromes from numpy's seeded generator.  Noise on
the surface codes is drawn by each side's own Philox sampler instead.
"""
from __future__ import annotations

import numpy as np

X, Y, Z = 1, 2, 3


def random_tree_code(n_qubits: int, seed: int, max_check_deg: int = 4, max_qubit_deg: int = 4):
    """A GF(4) check matrix whose Tanner graph is a tree: every new check is
    attached to one existing qubit and to 1..3 fresh qubits, with random
    Pauli entries.  Every check has degree >= 2."""
    rng = np.random.default_rng(seed)
    rows = []
    qdeg = [0]
    n = 1
    while n < n_qubits:
        anchors = [q for q in range(n) if qdeg[q] < max_qubit_deg]
        a = int(rng.choice(anchors))
        k = int(rng.integers(1, max_check_deg))
        k = min(k, n_qubits - n)
        members = [a] + list(range(n, n + k))
        row = {q: int(rng.integers(1, 4)) for q in members}
        rows.append(row)
        qdeg[a] += 1
        qdeg.extend([1] * k)
        n += k
    H = np.zeros((len(rows), n_qubits), dtype=np.uint8)
    for i, row in enumerate(rows):
        for q, p in row.items():
            H[i, q] = p
    return H


def random_priors(n_qubits: int, seed: int, lo: float = 0.02, hi: float = 0.2):
    """Per-qubit (p^X, p^Y, p^Z), each in [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_qubits, 3))


def jittered_priors(n_qubits: int, px: float, py: float, pz: float, rel: float):
    """(N, 3) float32 rows (p^X, p^Y, p^Z) of an i.i.d. channel, row j scaled
    by 1 + rel * u_j with u_j = 2 * ((j * 2654435761) mod 2^32) / 2^32 - 1 in
    [-1, 1) (Knuth's multiplicative hash of the qubit index).  The arithmetic
    is done in float64 and rounded once to float32, so the rows are exact
    and identical wherever they are built.  rel = 0 gives the uniform rows.
    A tiny rel breaks the exact symmetric ties that uniform priors leave on
    the toric and planar codes (Sec. II-B2, Sec. IV-A)."""
    j = np.arange(n_qubits, dtype=np.uint64)
    u = ((j * np.uint64(2654435761)) % np.uint64(1 << 32)).astype(np.float64) / 2.0 ** 32 * 2.0 - 1.0
    ch = np.array([px, py, pz], dtype=np.float64)
    return (ch[None, :] * (1.0 + rel * u)[:, None]).astype(np.float32)


def random_syndromes(m_checks: int, count: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(count, m_checks)).astype(np.uint8)


def trapping_set_code(check_pauli: int = Z):
    """The (4,0) trapping set of Sec. II-B2: four checks of one type and
    four qubits on an 8-cycle; qubit j lies on checks j and j+1 (mod 4)."""
    H = np.zeros((4, 4), dtype=np.uint8)
    for j in range(4):
        H[j, j] = check_pauli
        H[(j + 1) % 4, j] = check_pauli
    return H


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(B, M) 0/1 -> (B, ceil(M/32)) uint32 words, bit i%32 of word i//32."""
    bits = np.asarray(bits, dtype=np.uint8)
    B, M = bits.shape
    W = (M + 31) // 32
    padded = np.zeros((B, W * 32), dtype=np.uint64)
    padded[:, :M] = bits
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (padded.reshape(B, W, 32) * weights).sum(axis=2).astype(np.uint32)


def unpack_bits(words: np.ndarray, M: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32)
    B, W = words.shape
    bits = (words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(B, W * 32)[:, :M].astype(np.uint8)
