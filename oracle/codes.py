"""Oracle code construction and GF(2) tools for the surface codes of the paper.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  Shares no code with the CUDA path.

Codes (Sec. II-A and Sec. IV-B):
  * toric code [[2L^2, 2, L]]: hypergraph product (HGP) of the cyclic [L,1]
    repetition code with itself (Sec. IV-B2 builds it this way; the printed
    "[[2n^2, 1, n]]" there contradicts Sec. II-A, and K = 2 is what the
    construction gives);
  * planar (unrotated) surface code [[2L^2-2L+1, 1, L]]: HGP of the open
    [L,1] repetition code (Sec. II-A, Fig. 1);
  * XZZX surface code: the planar HGP code with a Hadamard applied to every
    qubit of the second HGP block, so that every bulk stabilizer reads
    X Z Z X (Sec. II-A, Sec. IV-B3).

HGP of H1 (m1 x n1) and H2 (m2 x n2), written out as the textbook definition:
    H_X = [ H1 (x) I_n2 | I_m1 (x) H2^T ]      (m1 n2 X-type checks)
    H_Z = [ I_n1 (x) H2 | H1^T (x) I_m2 ]      (n1 m2 Z-type checks)
Qubit order: block 1 then block 2 (row-major Kronecker order); check order:
X-type checks then Z-type checks.

Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z.  A Pauli string is also written as a
binary symplectic vector (x | z) with X = (1,0), Z = (0,1), Y = (1,1).
"""
from __future__ import annotations

import itertools

import numpy as np

I, X, Y, Z = 0, 1, 2, 3


def repetition_open(L: int) -> np.ndarray:
    """Parity checks of the open [L,1] repetition code: (L-1) x L."""
    H = np.zeros((L - 1, L), dtype=np.uint8)
    for r in range(L - 1):
        H[r, r] = 1
        H[r, r + 1] = 1
    return H


def repetition_cyclic(L: int) -> np.ndarray:
    """Parity checks of the cyclic [L,1] repetition code: L x L."""
    H = np.zeros((L, L), dtype=np.uint8)
    for r in range(L):
        H[r, r] = 1
        H[r, (r + 1) % L] = 1
    return H


def hypergraph_product(H1: np.ndarray, H2: np.ndarray):
    """Return (H_X, H_Z) of the HGP code, as 0/1 matrices."""
    m1, n1 = H1.shape
    m2, n2 = H2.shape
    HX = np.hstack([np.kron(H1, np.eye(n2, dtype=np.uint8)),
                    np.kron(np.eye(m1, dtype=np.uint8), H2.T)]) % 2
    HZ = np.hstack([np.kron(np.eye(n1, dtype=np.uint8), H2),
                    np.kron(H1.T, np.eye(m2, dtype=np.uint8))]) % 2
    return HX.astype(np.uint8), HZ.astype(np.uint8), n1 * n2


def css_to_pauli(HX: np.ndarray, HZ: np.ndarray) -> np.ndarray:
    """GF(4) check matrix: X-type rows carry X on their support, Z-type rows Z."""
    return np.vstack([HX * X, HZ * Z]).astype(np.uint8)


def build_code(kind: str, L: int):
    """Return (H, K) where H is the M x N Pauli check matrix."""
    if kind == "planar":
        R = repetition_open(L)
        HX, HZ, _ = hypergraph_product(R, R)
        return css_to_pauli(HX, HZ), 1
    if kind == "toric":
        R = repetition_cyclic(L)
        HX, HZ, _ = hypergraph_product(R, R)
        return css_to_pauli(HX, HZ), 2
    if kind == "xzzx":
        R = repetition_open(L)
        HX, HZ, n_block1 = hypergraph_product(R, R)
        H = css_to_pauli(HX, HZ)
        second = H[:, n_block1:]
        swapped = second.copy()
        swapped[second == X] = Z
        swapped[second == Z] = X
        H[:, n_block1:] = swapped
        return H, 1
    raise ValueError(kind)


# ----------------------------------------------------------------- symplectic

def to_symplectic(P: np.ndarray) -> np.ndarray:
    """Pauli codes (..., N) -> binary (..., 2N) vectors (x | z)."""
    P = np.asarray(P)
    x = ((P == X) | (P == Y)).astype(np.uint8)
    z = ((P == Z) | (P == Y)).astype(np.uint8)
    return np.concatenate([x, z], axis=-1)


def from_symplectic(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v).astype(np.uint8)
    n = v.shape[-1] // 2
    x, z = v[..., :n], v[..., n:]
    out = np.zeros(x.shape, dtype=np.uint8)
    out[(x == 1) & (z == 0)] = X
    out[(x == 1) & (z == 1)] = Y
    out[(x == 0) & (z == 1)] = Z
    return out


def symplectic_product(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """<a, b> = a_x . b_z + a_z . b_x (mod 2); 1 means the Paulis anticommute.
    a: (..., 2N), b: (K, 2N) -> (..., K)."""
    n = a.shape[-1] // 2
    ax, az = a[..., :n].astype(np.int64), a[..., n:].astype(np.int64)
    bx, bz = b[:, :n].astype(np.int64), b[:, n:].astype(np.int64)
    return ((ax @ bz.T + az @ bx.T) % 2).astype(np.uint8)


def syndrome(H: np.ndarray, E: np.ndarray) -> np.ndarray:
    """s_i = <E, row_i of H> for each check; E: (..., N) codes -> (..., M)."""
    return symplectic_product(to_symplectic(E), to_symplectic(H))


# ----------------------------------------------------------------- GF(2) algebra

def gf2_rref(A: np.ndarray):
    """Reduced row echelon form over GF(2); returns (R, pivot_columns)."""
    R = (np.asarray(A) % 2).astype(np.uint8).copy()
    rows, cols = R.shape
    pivots = []
    r = 0
    for c in range(cols):
        if r >= rows:
            break
        nz = np.nonzero(R[r:, c])[0]
        if nz.size == 0:
            continue
        p = r + nz[0]
        if p != r:
            R[[r, p]] = R[[p, r]]
        mask = R[:, c].astype(bool)
        mask[r] = False
        R[mask] ^= R[r]
        pivots.append(c)
        r += 1
    return R[:r], pivots


def gf2_rank(A: np.ndarray) -> int:
    return len(gf2_rref(A)[1])


def gf2_nullspace(A: np.ndarray) -> np.ndarray:
    """Basis (rows) of {v : A v = 0 mod 2}."""
    A = (np.asarray(A) % 2).astype(np.uint8)
    cols = A.shape[1]
    R, piv = gf2_rref(A)
    free = [c for c in range(cols) if c not in set(piv)]
    basis = []
    for f in free:
        v = np.zeros(cols, dtype=np.uint8)
        v[f] = 1
        for k, p in enumerate(piv):
            v[p] = R[k, f]
        basis.append(v)
    return np.array(basis, dtype=np.uint8).reshape(len(basis), cols)


class StabilizerGroup:
    """Row space of the check matrix in symplectic form, for membership tests."""

    def __init__(self, H: np.ndarray):
        self.H = np.asarray(H, dtype=np.uint8)
        self.R, self.piv = gf2_rref(to_symplectic(self.H))

    def contains(self, P: np.ndarray) -> np.ndarray:
        """True where the Pauli string(s) P (..., N) lie in the stabilizer group
        (up to phase): reduce against the row-echelon basis and test for 0."""
        v = to_symplectic(np.atleast_2d(P)).copy()
        for k, p in enumerate(self.piv):
            hit = v[:, p] == 1
            v[hit] ^= self.R[k]
        res = ~v.any(axis=1)
        return res if np.ndim(P) > 1 else bool(res[0])


def logical_operators(H: np.ndarray) -> np.ndarray:
    """A basis of N(S) modulo S (2K Pauli strings), from linear algebra alone.

    N(S) is the kernel of the symplectic form against the rows of H:
    v with [H_z | H_x] v = 0.  Its elements outside the row space of S give
    the logical operators; greedy extension of a basis of S picks 2K of them."""
    Hs = to_symplectic(H)
    n = H.shape[1]
    swap = np.concatenate([Hs[:, n:], Hs[:, :n]], axis=1)
    normalizer = gf2_nullspace(swap)
    basis = gf2_rref(Hs)[0]
    rank = basis.shape[0]
    logicals = []
    for v in normalizer:
        trial = np.vstack([basis, v[None, :]])
        r = gf2_rank(trial)
        if r > rank:
            basis = gf2_rref(trial)[0]
            rank = r
            logicals.append(v)
    return from_symplectic(np.array(logicals, dtype=np.uint8))


def logical_failure(H: np.ndarray, E: np.ndarray, Ehat: np.ndarray, group: StabilizerGroup | None = None):
    """Success criterion of Sec. IV: E^ in E S, i.e. the residual E^ E is a
    stabilizer.  Returns (fail, detected): fail when the residual is not in
    S; detected when it also anticommutes with some stabilizer."""
    group = group or StabilizerGroup(H)
    R = from_symplectic(to_symplectic(E) ^ to_symplectic(Ehat))
    ok = group.contains(R)
    detected = syndrome(H, R).any(axis=-1)
    return ~ok, detected


def min_logical_weight(H: np.ndarray, max_weight: int, paulis=(X, Y, Z)) -> int | None:
    """Smallest weight w <= max_weight of a Pauli string (entries from
    `paulis`) that commutes with every check but is not a stabilizer.
    Brute force over all supports; None if there is none up to max_weight."""
    N = H.shape[1]
    group = StabilizerGroup(H)
    Hs = to_symplectic(H)
    for w in range(1, max_weight + 1):
        for support in itertools.combinations(range(N), w):
            for ops in itertools.product(paulis, repeat=w):
                P = np.zeros(N, dtype=np.uint8)
                P[list(support)] = ops
                if symplectic_product(to_symplectic(P)[None, :], Hs).any():
                    continue
                if not group.contains(P):
                    return w
    return None
