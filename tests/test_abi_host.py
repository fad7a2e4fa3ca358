"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every symbol include/bpq.h declares, builds the same Tanner graphs as the
oracle's hypergraph-product construction, and rejects bad arguments."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from inputs import random_tree_code
from oracle import codes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    bpq.lib()
    return bpq


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bpq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bpq_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(bpq):
    L = bpq.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert L.bpq_version() >= 100


@pytest.mark.parametrize("kind", ["planar", "toric", "xzzx"])
@pytest.mark.parametrize("d", [3, 4, 5, 7, 9, 15])
def test_tanner_matches_oracle_construction(bpq, kind, d):
    t = bpq.Tanner(kind, d)
    H_oracle, K = codes.build_code(kind, d)
    assert (t.M, t.N, t.K) == (H_oracle.shape[0], H_oracle.shape[1], K)
    assert t.E == int((H_oracle != 0).sum())
    ptr, var, pauli = t.export()
    ii, jj, pp = oracle.edges(H_oracle)
    assert (np.repeat(np.arange(t.M), np.diff(ptr)) == ii).all()
    assert (var == jj).all() and (pauli == pp).all()


@pytest.mark.parametrize("kind,d", [("planar", 3), ("planar", 7), ("toric", 4), ("toric", 6), ("xzzx", 5)])
def test_library_logicals_are_valid(bpq, kind, d):
    t = bpq.Tanner(kind, d)
    H = t.dense()
    Lg = t.logicals()
    assert Lg.shape == (2 * t.K, t.N)
    Hs, Ls = codes.to_symplectic(H), codes.to_symplectic(Lg)
    assert not codes.symplectic_product(Ls, Hs).any()
    group = codes.StabilizerGroup(H)
    assert not group.contains(Lg).any()
    assert codes.gf2_rank(codes.symplectic_product(Ls, Ls)) == 2 * t.K
    # together with the checks they span a space of dimension N - K + 2K
    assert codes.gf2_rank(np.vstack([Hs, Ls])) == t.N - t.K + 2 * t.K


def test_custom_tanner_roundtrip(bpq):
    H = random_tree_code(7, seed=3)
    t = bpq.Tanner(H=H)
    assert (t.dense() == H).all() and t.K == -1


def test_rejects_bad_arguments(bpq):
    with pytest.raises(bpq.BPQError):
        bpq.Tanner("toric", 2)
    with pytest.raises(bpq.BPQError):
        bpq.Tanner("planar", 33)
    with pytest.raises(bpq.BPQError):
        bpq.Tanner(7, 5)
    H = np.zeros((1, 6), dtype=np.uint8)
    H[0, :5] = 1  # weight-5 check exceeds the padded degree
    with pytest.raises(bpq.BPQError):
        bpq.Tanner(H=H)
    H = np.array([[4, 1]], dtype=np.uint8)
    with pytest.raises(bpq.BPQError):
        bpq.Tanner(H=H)
    t = bpq.Tanner("planar", 5)
    with pytest.raises(bpq.BPQError):
        t.set_launch(48, 1)   # not a multiple of 32
    with pytest.raises(bpq.BPQError):
        bpq.Tanner("toric", 15).set_launch(32, 1)  # 450 nodes > 4 per thread x 32
    # GPU entry points refuse a handle that was never uploaded, before any CUDA call
    L = bpq.lib()
    rc = L.bpq_decode(t.handle, None, None, 0, None, 10, 0, None, None, None, None, None)
    assert rc == -4


def test_launch_shapes(bpq):
    t = bpq.Tanner("toric", 15)
    t.set_shots_per_thread(1)
    assert t.shots_per_thread("ewainit") == 1
    assert t.launch() == (256, 1)
    t.set_launch(256, 2)
    assert t.launch() == (256, 2)
    p = bpq.Tanner("planar", 5)
    p.set_shots_per_thread(1)
    assert p.launch()[0] == 32


def test_two_shots_per_thread_shapes(bpq):
    """Split tables decode two shots per thread by default (two nodes per
    thread, about 256 threads per CTA); AEWA-BP and the generic layout keep
    one shot per thread."""
    t = bpq.Tanner("toric", 15)
    assert t.shots_per_thread("ewainit") == 2 and t.shots_per_thread("plain") == 2
    assert t.shots_per_thread("aewa") == 1
    assert t.launch() == (256, 1)
    t.set_launch(480, 1)  # one node per thread
    assert t.launch() == (480, 1)
    t.set_launch(128, 1)  # four nodes per thread: only one shot per thread fits
    assert t.shots_per_thread("ewainit") == 1
    with pytest.raises(bpq.BPQError):
        t.set_shots_per_thread(2)  # the stored shape has four nodes per thread
    t.set_launch(0, 0)
    t.set_shots_per_thread(2)
    assert t.shots_per_thread("ewainit") == 2 and t.launch() == (256, 1)
    with pytest.raises(bpq.BPQError):
        t.set_launch(128, 1)
    with pytest.raises(bpq.BPQError):
        t.set_shots_per_thread(3)
    assert bpq.Tanner("planar", 5).launch() == (32, 8)
    H = bpq.Tanner("toric", 5).dense()
    H[0, np.nonzero(H[0])[0][0]] = 2  # a Y entry: generic layout
    g = bpq.Tanner(H=H)
    assert g.shots_per_thread("ewainit") == 1
    with pytest.raises(bpq.BPQError):
        g.set_shots_per_thread(2)


def test_default_params_follow_the_paper(bpq):
    p = bpq.default_params("adagrad")
    assert p.alpha == 5.0 and p.msg_clip == 30.0 and p.adagrad_g_from_iter1 == 1
    p = bpq.default_params("momentum")
    assert p.alpha == 0.5 and p.gamma == 0.0
    assert bpq.default_params("ewainit").alpha == 0.5


def test_workspace_and_host_buffer_sizes(bpq):
    L = bpq.lib()
    assert L.bpq_decode_workspace_bytes() >= 8
    t = bpq.Tanner("toric", 15)
    n = bpq.decode_host_bytes(t, 1000)
    assert n >= 1000 * (t.N + 2) + 1000 * t.W * 4 + 3 * t.N * 4


def test_prior_rows_match_the_shared_input_generator(bpq):
    from inputs import jittered_priors
    for n, ch, rel in ((450, (0.02 / 3,) * 3, 2.0 ** -16), (313, (0.01, 0.002, 0.05), 2.0 ** -8), (7, (0.1,) * 3, 0.0)):
        a = bpq.prior_rows(n, *ch, jitter=rel)
        b = jittered_priors(n, *ch, rel)
        assert a.dtype == np.float32 and a.shape == (n, 3)
        assert np.array_equal(a, b)
    # the perturbation is relative, bounded by rel, and not constant
    a = bpq.prior_rows(450, 0.01, 0.01, 0.01, jitter=2.0 ** -16).astype(np.float64)
    r = a / 0.01 - 1.0
    assert np.abs(r).max() <= 2.0 ** -16 + 2.0 ** -23 and np.unique(a[:, 0]).size > 300  # float32 resolves about 330 levels here
    assert (a[:, 0] == a[:, 1]).all() and (a[:, 1] == a[:, 2]).all()
    assert np.array_equal(bpq.prior_rows(9, 0.01, 0.02, 0.03), np.tile(np.float32([0.01, 0.02, 0.03]), (9, 1)))


def test_message_layout_of_each_code_family(bpq):
    """Toric codes have no padding slots (every check of degree 4, every
    qubit two X and two Z edges); planar and XZZX codes use the split layout
    with padding; a Y entry, or three edges of one type on a qubit, forces the
    generic layout."""
    for d in (3, 6, 15):
        assert bpq.Tanner("toric", d).layout() == 2
    for kind in ("planar", "xzzx"):
        for d in (3, 7):
            assert bpq.Tanner(kind, d).layout() == 1
    H = bpq.Tanner("toric", 5).dense()
    Hy = H.copy()
    Hy[0, np.nonzero(H[0])[0][0]] = 2  # one Y entry
    assert bpq.Tanner(H=Hy).layout() == 0
    Hx = np.concatenate([H, np.zeros((H.shape[0], 1), dtype=np.uint8)], axis=1)  # an isolated qubit
    assert bpq.Tanner(H=Hx).layout() == 1
    assert bpq.Tanner(H=random_tree_code(10, seed=3)).layout() in (0, 1)
    T = np.zeros((3, 1), dtype=np.uint8)
    T[:, 0] = 1  # one qubit on three X checks
    assert bpq.Tanner(H=T).layout() == 0


def test_batch_shapes(bpq):
    """Shot groups of a code inside the batched kernel: the fewest threads per
    group for the chosen nodes per thread, as many groups as fit in 1024
    threads (15 multi-warp, 32 one-warp at most); automatic = the choice with
    more busy node slots per CTA, two nodes per thread on a tie; independent
    of the one-code launch shape."""
    assert bpq.Tanner("planar", 17).batch_launch() == (288, 3, 2)   # 3 x 545 / 2048 > 1 x 545 / 1024
    assert bpq.Tanner("planar", 9).batch_launch() == (160, 6, 1)    # 6 x 145 / 1024 > 10 x 145 / 2048
    assert bpq.Tanner("toric", 8).batch_launch() == (128, 8, 1)
    assert bpq.Tanner("toric", 16).batch_launch() == (256, 4, 2)    # tie: 2 x 512 / 1024 = 4 x 512 / 2048
    assert bpq.Tanner("planar", 5).batch_launch() == (32, 32, 2)    # one-warp groups
    assert bpq.Tanner("planar", 25).batch_launch() == (608, 1, 2)   # 1201 nodes: no one-node shape
    t = bpq.Tanner("planar", 17)
    t.set_launch(160, 1)   # four nodes per thread in bpq_decode
    assert t.batch_launch() == (288, 3, 2)
    t.set_batch_launch(1)
    assert t.batch_launch() == (576, 1, 1)
    t.set_batch_launch(0)
    assert t.batch_launch() == (288, 3, 2)
    with pytest.raises(bpq.BPQError):
        t.set_batch_launch(3)
    with pytest.raises(bpq.BPQError):
        bpq.Tanner("planar", 25).set_batch_launch(1)    # 1201 threads per group
    with pytest.raises(bpq.BPQError):
        t.batch_launch("aewa")


def test_serial_shots_per_warp_refusals(bpq):
    t = bpq.Tanner("planar", 5)
    for k in (0, 1, 2):
        t.set_serial_shots_per_warp(k)
    for k in (3, -1):
        with pytest.raises(bpq.BPQError):
            t.set_serial_shots_per_warp(k)


def test_batch_plan_refuses_a_misaligned_workspace(bpq):
    """A workspace that does not start on a 16-byte boundary is refused on the
    host (BPQ_EINVAL) before the items are looked at; an aligned one goes on
    to the next check (here: an item without an uploaded Tanner graph).  The
    addresses are never dereferenced."""
    from paper_2407_11523_gb300 import _binding as B

    L = bpq.lib()
    items = (B.BatchItem * 1)()
    items[0] = B.BatchItem(None, None, None, 1, None, None, None)
    p = bpq.make_params("ewainit")
    out = ctypes.c_void_p()
    rc = L.bpq_batch_plan(items, 1, 3, ctypes.byref(p), 100, ctypes.c_void_p(0x100008), 1 << 20, None,
                          ctypes.byref(out))
    assert rc == -1 and b"16-byte" in L.bpq_last_error()
    rc = L.bpq_batch_plan(items, 1, 3, ctypes.byref(p), 100, ctypes.c_void_p(0x100000), 1 << 20, None,
                          ctypes.byref(out))
    assert rc == -4 and b"uploaded" in L.bpq_last_error()
    assert not out.value
